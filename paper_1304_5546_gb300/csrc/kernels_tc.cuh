// FP32 stage kernel with the element-local products on the 5th-generation
// tensor cores (tcgen05; operand A and the accumulator in tensor memory).
//
// Same result as dg_stage_kernel (kernels.cuh): right-hand side of Eq.
// dg-strong-explicit -- volume derivative by Dr/Ds and the chain rule of Eq.
// dg-diff-local-to-global, upwind flux of Eq. max2d-numflux at every face
// node, LIFT of Eq. dg-lift -- followed by one 2N-storage LSRK(5,4) stage
// update, or written out as the right-hand side.
//
// The products of a block of E elements form one dense contraction.  With
// X rows per element (u_d = u minus its linear interpolant through the
// element's vertex nodes; A = rx Hy_d - ry Hx_d, B = sx Hy_d - sy Hx_d;
// F_c = Fscale/2 * flux_c):
//   row      e = [ -ry Ez_d | -sy Ez_d | F_x | L_x ]  ->  dHx/dt
//   row  E + e = [  rx Ez_d |  sx Ez_d | F_y | L_y ]  ->  dHy/dt
//   row 2E + e = [  A       |  B       | F_z | L_z ]  ->  dEz/dt
// (each part of a row starts on a 16-byte boundary, see tc_kd; the last
// column L of a row holds the chain-rule combination of the linear part's
// exact derivatives, (u_v2 - u_v1)/2 along r and (u_v3 - u_v1)/2 along s,
// and the operator tile holds 1 there for every node) the right-hand side
// is the GEMM D = X [Dr | Ds | LIFT | 1]^T, with no further term.
// The deflation keeps the products' operands O(h^2) for smooth fields, so
// their TF32 rounding stays far below FP32 accuracy.  M = 3E rows in one
// 128-row tile (E = 40), or in two tiles at N <= 3 (E = 80: each tile is its
// own MMA group and each operand-row and epilogue thread owns one row per
// tile), K = 2 Np + Nafp + 1 (padded to 8), N = Np (padded to 16).  FP32 accuracy
// comes from three TF32 products, X_hi Op_hi + X_hi Op_lo + X_lo Op_hi: X_hi
// keeps the top 11 significand bits of X, X_lo = X - X_hi (exact in FP32,
// truncated to TF32 by the tensor core); Op's hi/lo split is made on the host
// from FP64 with round-to-nearest.  One MMA of N = 2 Np' computes X_hi
// [Op_hi ; Op_lo] so that X_hi is read once; a second adds X_lo Op_hi (at
// N = 7 all three products go to one accumulator of Np' columns, see
// TcLayout).
//
// X never touches shared memory: the build warps write it straight into
// tensor memory (tcgen05.st; lane = row, one column per K index), and the
// MMAs read operand A from there (double-buffered where the 512 columns
// allow).  Shared memory carries only the stage data, the operator tiles
// (operand B) and the face fluxes.  Rows are ordered field-major, so the 32
// rows of a TMEM lane quarter -- the rows one warp may access -- are
// consecutive elements, whose shared-memory reads at a stride of Np words
// spread over 32 / gcd(Np, 32) banks.
//
// Warp roles: 4 epilogue warps (one per lane quarter: accumulator ->
// LSRK update in place in the stage buffer), 8 flux warps (upwind flux at
// every face node into a double-buffered shared-memory array, up to two
// blocks ahead; neighbour traces gathered one block ahead), 8 operand-row
// warps (two per lane quarter, each a share of its rows' volume-part and
// LIFT-part column chunks balanced by a work model, with packed FP32x2
// arithmetic; the LIFT part waits for the block's fluxes), one MMA warp, one
// memory warp (1D TMA bulk loads into a ring of stage buffers, bulk stores
// of full blocks from the same buffers, a stage refilled once the stores of
// the block after it are issued).  Every wait is bounded; on expiry the CTA
// sets the status word, drains its copies (bounded), frees its TMEM and
// returns.
#pragma once

#include "kernels.cuh"

namespace dgw {

template <int N, int PREC_, bool MEDIA_ = false, bool ALT_ = false>
struct TcLayout {
  static constexpr int PREC = PREC_;
  static constexpr bool MEDIA = MEDIA_;
  static constexpr int GEO = MEDIA ? kGeoMedia : kGeo;  // geometry record length
  static constexpr bool BF = tc_is_bf16(PREC);  // BF16 operands (else TF32)
  static constexpr int NS = tc_nsplit(PREC);     // X parts and operator tiles (hi, lo)
  static constexpr int Np = Order<N>::Np;
  static constexpr int Nfp = Order<N>::Nfp;
  static constexpr int Nafp = Order<N>::Nafp;
  static constexpr int KD = tc_kd(N), KP = tc_kpp(N, PREC);
  static constexpr int EB = BF ? 2 : 4;         // operand element bytes
  static constexpr int KG = KP * EB / 16;       // core matrices along K
  static constexpr int XPART = BF ? KP / 2 : KP;  // TMEM columns of one X part
  static constexpr int NN = tc_nn(N);
  // GEMM row tiles of 128 TMEM lanes per block (tc_tiles: two at N <= 3,
  // where two tiles' double-buffered operands and (split) accumulators fit
  // the 512 columns, one above; ALT_: the other count where both fit).  A
  // block of 80 elements shares the per-block hand-offs.
  static constexpr int TILES = tc_tiles(N, PREC_, ALT_);
  static constexpr int E = 40 * TILES;  // 3E <= 128 TILES GEMM rows, E % 4 == 0
  static constexpr int ROWS = 3 * E;
  static constexpr int NPAD = tc_npad(N);
  static constexpr int IV = NPAD / 4;          // volume chunks of 4 nodes
  static constexpr int LCOLS = KP - 2 * NPAD;  // LIFT-part columns (zero beyond Nafp)
  // tensor memory: two accumulators, then XBUF operand buffers of NS parts.
  // Split variants (ACC_SPLIT): an accumulator has 2 NN columns, [0, NN)
  // holding X_hi Op_hi + X_lo Op_hi and [NN, 2 NN) holding X_hi Op_lo (one
  // MMA of N = 2 NN reads X_hi once for both operator tiles); where that
  // leaves no room for two operand buffers (N = 7) all three products go to
  // the same NN columns instead, so that operand building and MMAs still
  // overlap.  An operand buffer holds X_hi, then X_lo.  Single-product
  // variants: NN columns, X.
  // With TILES = 2 every buffer holds one such part per tile (accumulator
  // buffer b, tile t at (b TILES + t) ACC_COLS; operand buffer x, tile t at
  // OFF_XT + (x TILES + t) XCOLS).
  static constexpr int XCOLS = NS * XPART;
  static constexpr bool ACC_SPLIT = NS == 2 && TILES * (2 * (2 * NN) + 2 * XCOLS) <= 512;
  static constexpr int ACC_COLS = ACC_SPLIT ? 2 * NN : NN;
  static constexpr int XBUF = TILES * (2 * ACC_COLS + 2 * XCOLS) <= 512 ? 2 : 1;
  static constexpr int OFF_XT = 2 * TILES * ACC_COLS;
  static constexpr int TMEM_COLS = 512;
  // warp roles: 0-3 epilogue; 4-11 operand rows (warp w serves lane quarter
  // w % 4 and takes share (w - 4) / 4 of its rows' chunks); 12-19 face flux
  // and neighbour gathers; 20 MMA; 21 memory
  static constexpr int EPI_WARPS = 4, X_WARPS = 8, FLUX_WARPS = 8;
  // memory warp: the bulk copies of a block issued by several lanes at once
  // at N >= 5 (2-9 % faster there on GB300), by lane 0 alone at N <= 4
  // (where several issuing lanes measured 2-6 % slower)
  static constexpr bool IO_LANES = N >= 5;
  // widest tcgen05.st of an operand-row run (columns): 8 (1-4 % faster than
  // 4 at every order on GB300), 16 at N = 7 (where it measured faster
  // still; at N = 6 it was slower than 8)
  static constexpr int ST_W = N == 7 ? 16 : 8;
  static constexpr int FLUX_WARP0 = EPI_WARPS + X_WARPS;
  static constexpr int MMA_WARP = FLUX_WARP0 + FLUX_WARPS, IO_WARP = MMA_WARP + 1;
  static constexpr int THREADS = 32 * (IO_WARP + 1);
  static constexpr int X_THREADS = 32 * X_WARPS, FLUX_THREADS = 32 * FLUX_WARPS;
  static constexpr int TASKS = E * Nafp;
  static constexpr int TPT = (TASKS + FLUX_THREADS - 1) / FLUX_THREADS;
  // LIFT-part chunks read with one 16-byte load each (N = 3 and 5, where
  // that measured 0.4-1.5 % faster on GB300; about even elsewhere).  The
  // face-flux row stride is then 4 x odd words, so that the 16-byte loads of
  // 8 consecutive rows by a quarter warp fall on distinct banks; otherwise it
  // is odd, for conflict-free 4-byte row reads.
  static constexpr bool LIFT_V4 = N == 3 || N == 5;
  static constexpr int FES = !LIFT_V4                         ? (Nafp | 1)
                             : ((Nafp + 3) / 4) % 2 == 1      ? (Nafp + 3) / 4 * 4
                                                              : (Nafp + 3) / 4 * 4 + 4;
  // deflation of a node pair as one subtraction and two FMAs instead of two
  // subtractions, a product and an FMA (N = 5 and 6, where that measured
  // 0.4 % and 5 % faster; 2 % slower at N = 7, even at N <= 4)
  static constexpr bool DEFL_FMA = N == 5 || N == 6;
  // operand-row field loads without the row-validity predicate (N <= 5,
  // 0.2-1.3 % faster there; 1 % and 10 % slower at N = 6 and 7): a row that
  // is not valid reads an address inside the stage buffer, and its values
  // reach only its own GEMM row, which the epilogue never writes back
  static constexpr bool ROW_LOADS_UNPRED = N <= 5;
  static constexpr int FB = 3 * E * FES * 4;  // one face-flux buffer [3][E][FES]
  static constexpr int QB = E * Np * 4;
  static constexpr int GB = E * GEO * 4;
  static constexpr int CB = E * 3 * 4;
  static constexpr int STAGE_BYTES = round_up(6 * QB + GB + CB, 128);
  static constexpr int OB = NN * KP * EB;  // one operator tile
  static constexpr int HEADER = 1024;
  static constexpr int OFF_OP = HEADER;
  static constexpr int OFF_F = OFF_OP + NS * OB;
  static constexpr int OFF_STAGES = round_up(OFF_F + 2 * FB, 128);
  static constexpr int SMAX = 232448;
  static constexpr int S_FIT = (SMAX - OFF_STAGES) / STAGE_BYTES;
  static constexpr int S = S_FIT < 6 ? S_FIT : 6;  // stage buffers
  // at least half of the SM's shared memory: one CTA per SM, which owns all
  // 512 TMEM columns (a second resident CTA would wait in tcgen05.alloc)
  static constexpr size_t SMEM_USED = OFF_STAGES + S * STAGE_BYTES;
  static constexpr size_t SMEM_BYTES = SMEM_USED > 118784 ? SMEM_USED : 118784;
  // S >= 3: a stage is refilled one block after its stores are issued, and
  // the flux warps wait for the next block's stage while on this one
  static_assert(S >= 3 && S <= 8, "stage ring / header layout");
  static_assert(SMEM_BYTES <= SMAX, "shared memory");
  static_assert(QB % 16 == 0 && GB % 16 == 0 && CB % 16 == 0 && OB % 16 == 0, "TMA chunks");
  static_assert(!LIFT_V4 || (FES % 4 == 0 && FES >= (Nafp + 3) / 4 * 4 && OFF_F % 16 == 0 &&
                             FB % 16 == 0),
                "16-byte face-flux loads: aligned rows, chunks inside a row");
  static_assert(ROWS <= 128 * TILES && NN <= 256 && NN % 16 == 0 && KP % (BF ? 16 : 8) == 0,
                "UMMA shape");
  static_assert(LCOLS % 4 == 0 && LCOLS >= Nafp + 1, "LIFT part and linear-part column");
  static_assert(TILES * (2 * ACC_COLS + XBUF * XCOLS) <= TMEM_COLS, "tensor memory");
  static_assert(X_WARPS % 4 == 0, "operand-row warps come in lane-quarter groups");
};

// The column chunks (4 columns each) of one X row that build warp share
// ROLE of a lane quarter writes: a contiguous range of volume chunks and a
// contiguous range of LIFT-part chunks taken from the other end, so that the
// NR shares are even.
template <class L, int ROLE>
struct RowShare {
  static constexpr int NR = L::X_WARPS / 4, LC = L::LCOLS / 4;
  // work model of a chunk (instructions, roughly): a volume chunk converts
  // and stores two parts (16) and computes 6 per node inside the element; a
  // LIFT-part chunk loads, converts and stores one part (12)
  static constexpr int vol_w(int v) {
    return 16 + 6 * (L::Np - 4 * v >= 4 ? 4 : (L::Np - 4 * v > 0 ? L::Np - 4 * v : 0));
  }
  static constexpr int vol_sum(int a, int b) { return a >= b ? 0 : vol_w(a) + vol_sum(a + 1, b); }
  // two shares: share 0 takes volume chunks [0, k) and LIFT chunks [l, LC),
  // share 1 the rest; (k, l) minimises the larger share's work
  static constexpr int cost(int k, int l) {
    return vol_sum(0, k) + 12 * (LC - l) > vol_sum(k, L::IV) + 12 * l
               ? vol_sum(0, k) + 12 * (LC - l)
               : vol_sum(k, L::IV) + 12 * l;
  }
  static constexpr int best(int k, int l, int bk, int bl) {
    return k > L::IV ? bk * 64 + bl
           : l > LC  ? best(k + 1, 0, bk, bl)
                     : best(k, l + 1, cost(k, l) < cost(bk, bl) ? k : bk,
                            cost(k, l) < cost(bk, bl) ? l : bl);
  }
  static constexpr int SPLIT = best(0, 0, L::IV / 2, LC / 2);
  static constexpr int K2 = SPLIT / 64, L2 = SPLIT % 64;
  static constexpr int VLO = NR == 2 ? (ROLE == 0 ? 0 : K2) : ROLE * L::IV / NR;
  static constexpr int VHI = NR == 2 ? (ROLE == 0 ? K2 : L::IV) : (ROLE + 1) * L::IV / NR;
  static constexpr int LLO = NR == 2 ? (ROLE == 0 ? L2 : 0) : (NR - 1 - ROLE) * LC / NR;
  static constexpr int LHI = NR == 2 ? (ROLE == 0 ? LC : L2) : (NR - ROLE) * LC / NR;
};

// Four consecutive K columns (k0, a multiple of 4) of this thread's X row
// into tensor memory at xh (and xl for the split variants), in the operand
// format of the launch's product variant:
//   kTcTf32x3  hi = top 11 significand bits (TF32), lo = the exact rest
//   kTcTf32    rounded to the nearest TF32
//   kTcBf16    rounded to the nearest BF16, two per column
//   kTcBf16x3  hi = nearest BF16, lo = nearest BF16 of the rest
template <class L>
__device__ __forceinline__ void x_emit4(uint32_t xh, uint32_t xl, int k0, float v0, float v1,
                                        float v2, float v3) {
  if constexpr (L::PREC == kTcTf32x3) {
    const f32x2 p0 = f32x2_pack(v0, v1), p1 = f32x2_pack(v2, v3);
    const f32x2 h0 = f32x2_tf32_trunc(p0), h1 = f32x2_tf32_trunc(p1);
    float h[4], l[4];
    f32x2_unpack(h0, h[0], h[1]);
    f32x2_unpack(h1, h[2], h[3]);
    f32x2_unpack(f32x2_sub(p0, h0), l[0], l[1]);
    f32x2_unpack(f32x2_sub(p1, h1), l[2], l[3]);
    tmem_st4(xh + k0, h);
    tmem_st4(xl + k0, l);
  } else if constexpr (L::PREC == kTcTf32) {
    const float h[4] = {tf32_rna(v0), tf32_rna(v1), tf32_rna(v2), tf32_rna(v3)};
    tmem_st4(xh + k0, h);
  } else if constexpr (L::PREC == kTcBf16) {
    tmem_st2(xh + k0 / 2, bf16x2_rn(v0, v1), bf16x2_rn(v2, v3));
  } else {
    const uint32_t h01 = bf16x2_rn(v0, v1), h23 = bf16x2_rn(v2, v3);
    const uint32_t l01 = bf16x2_rn(v0 - bf16_lo_f32(h01), v1 - bf16_hi_f32(h01));
    const uint32_t l23 = bf16x2_rn(v2 - bf16_lo_f32(h23), v3 - bf16_hi_f32(h23));
    tmem_st2(xh + k0 / 2, h01, h23);
    tmem_st2(xl + k0 / 2, l01, l23);
  }
}

// Eight (sixteen) consecutive K columns from k0 as in x_emit4, in one
// tcgen05.st per part.
template <class L>
__device__ __forceinline__ void x_emit8(uint32_t xh, uint32_t xl, int k0, const float* v) {
  if constexpr (L::PREC == kTcTf32x3) {
    float h[8], l[8];
#pragma unroll
    for (int i = 0; i < 8; i += 2) {
      const f32x2 p = f32x2_pack(v[i], v[i + 1]);
      const f32x2 hh = f32x2_tf32_trunc(p);
      f32x2_unpack(hh, h[i], h[i + 1]);
      f32x2_unpack(f32x2_sub(p, hh), l[i], l[i + 1]);
    }
    tmem_st8(xh + k0, h);
    tmem_st8(xl + k0, l);
  } else {
    x_emit4<L>(xh, xl, k0, v[0], v[1], v[2], v[3]);
    x_emit4<L>(xh, xl, k0 + 4, v[4], v[5], v[6], v[7]);
  }
}

template <class L>
__device__ __forceinline__ void x_emit16(uint32_t xh, uint32_t xl, int k0, const float* v) {
  if constexpr (L::PREC == kTcTf32x3) {
    float h[16], l[16];
#pragma unroll
    for (int i = 0; i < 16; i += 2) {
      const f32x2 p = f32x2_pack(v[i], v[i + 1]);
      const f32x2 hh = f32x2_tf32_trunc(p);
      f32x2_unpack(hh, h[i], h[i + 1]);
      f32x2_unpack(f32x2_sub(p, hh), l[i], l[i + 1]);
    }
    tmem_st16(xh + k0, h);
    tmem_st16(xl + k0, l);
  } else {
    x_emit8<L>(xh, xl, k0, v);
    x_emit8<L>(xh, xl, k0 + 8, v + 8);
  }
}

// A run of NC chunks of 4 columns (values v[0 .. 4 NC)) from column k0, in
// stores of at most L::ST_W columns.
template <class L, int NC>
__device__ __forceinline__ void x_emit_run(uint32_t xh, uint32_t xl, int k0, const float* v) {
  constexpr int N16 = L::ST_W >= 16 ? NC / 4 : 0;
  constexpr int R = NC - 4 * N16, N8 = R / 2, N4 = R % 2;
#pragma unroll
  for (int c = 0; c < N16; ++c) x_emit16<L>(xh, xl, k0 + 16 * c, v + 16 * c);
#pragma unroll
  for (int c = 0; c < N8; ++c) x_emit8<L>(xh, xl, k0 + 16 * N16 + 8 * c, v + 16 * N16 + 8 * c);
  if constexpr (N4) {
    constexpr int o = 16 * N16 + 8 * N8;
    x_emit4<L>(xh, xl, k0 + o, v[o], v[o + 1], v[o + 2], v[o + 3]);
  }
}

// One thread's share of its X row into tensor memory at xh / xl (this warp's
// lane quarter), in two calls: the volume part, then the LIFT part (which
// waits for the face fluxes).  Each call computes every value first and then
// converts and stores them (x_emit4), so the loads of all its chunks can be
// in flight at once.  rc: output field of the row; qe: the element's fields
// in the stage buffer; fr: the row's face fluxes; (a1, a2, a3) / (b1, b2,
// b3): vertex values of u (Ez for rc < 2, Hx for rc = 2) / of w (Hy, rc = 2).
//
// Volume part: nodes 4ch .. 4ch+3 in pairs (packed FP32x2): deflated u (and
// w), then the Dr part cr1 u + cr2 w and the Ds part cs1 u + cs2 w with
// (cr1, cs1, cr2, cs2) = (-ry, -sy, 0, 0), (rx, sx, 0, 0), (-ry, -sy, rx, sx)
// for output field Hx, Hy, Ez.  Nodes >= Np come out exactly zero (u = u1
// there, and the zero-padded weights).  Rows that are not valid have zero
// vertex values and factors; with L::ROW_LOADS_UNPRED they still read their
// stage entries, which may hold anything (their GEMM rows are discarded).
template <int N, class L, int ROLE>
__device__ __forceinline__ void build_x_vol(const float* qe, const float* lam, uint32_t xh,
                                            uint32_t xl, bool row_ok, int rc, float rx, float ry,
                                            float sx, float sy, float a1, float a2, float a3,
                                            float b1, float b2, float b3) {
  using R = RowShare<L, ROLE>;
  constexpr int Np = L::Np, E = L::E, NPAD = L::NPAD;
  constexpr int NV = R::VHI - R::VLO;
  if constexpr (NV > 0) {
    float vr[4 * NV], vs[4 * NV];
    const int fu = rc < 2 ? 2 * E * Np : 0;  // field u in the stage buffer
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int m0 = 4 * (R::VLO + v);
      const float4 l2v = *reinterpret_cast<const float4*>(lam + m0);
      const float4 l3v = *reinterpret_cast<const float4*>(lam + NPAD + m0);
#pragma unroll
      for (int pp = 0; pp < 2; ++pp) {
        const int m = m0 + 2 * pp;
        const f32x2 l2 = pp == 0 ? f32x2_pack(l2v.x, l2v.y) : f32x2_pack(l2v.z, l2v.w);
        const f32x2 l3 = pp == 0 ? f32x2_pack(l3v.x, l3v.y) : f32x2_pack(l3v.z, l3v.w);
        const bool in0 = (L::ROW_LOADS_UNPRED || row_ok) && m < Np;
        const bool in1 = (L::ROW_LOADS_UNPRED || row_ok) && m + 1 < Np;
        const f32x2 uq = f32x2_pack(in0 ? qe[fu + m] : a1, in1 ? qe[fu + m + 1] : a1);
        f32x2 ud = f32x2_sub(uq, f32x2_dup(a1));
        if constexpr (L::DEFL_FMA) {
          ud = f32x2_fma(f32x2_dup(a1 - a2), l2, ud);
          ud = f32x2_fma(f32x2_dup(a1 - a3), l3, ud);
        } else {
          ud = f32x2_sub(ud, f32x2_fma(f32x2_dup(a2 - a1), l2, f32x2_mul(f32x2_dup(a3 - a1), l3)));
        }
        f32x2 pr = f32x2_mul(f32x2_dup(rc == 1 ? rx : -ry), ud);
        f32x2 ps = f32x2_mul(f32x2_dup(rc == 1 ? sx : -sy), ud);
        if (rc == 2) {
          const f32x2 wq = f32x2_pack(in0 ? qe[E * Np + m] : b1, in1 ? qe[E * Np + m + 1] : b1);
          f32x2 wd = f32x2_sub(wq, f32x2_dup(b1));
          if constexpr (L::DEFL_FMA) {
            wd = f32x2_fma(f32x2_dup(b1 - b2), l2, wd);
            wd = f32x2_fma(f32x2_dup(b1 - b3), l3, wd);
          } else {
            wd = f32x2_sub(wd, f32x2_fma(f32x2_dup(b2 - b1), l2, f32x2_mul(f32x2_dup(b3 - b1), l3)));
          }
          pr = f32x2_fma(f32x2_dup(rx), wd, pr);
          ps = f32x2_fma(f32x2_dup(sx), wd, ps);
        }
        const int i = 4 * v + 2 * pp;
        f32x2_unpack(pr, vr[i], vr[i + 1]);
        f32x2_unpack(ps, vs[i], vs[i + 1]);
      }
    }
    __syncwarp();
    x_emit_run<L, NV>(xh, xl, 4 * R::VLO, vr);
    x_emit_run<L, NV>(xh, xl, NPAD + 4 * R::VLO, vs);
  }
}

// LIFT part: the row's face fluxes, then (column Nafp of the part) the
// chain-rule combination of the linear part's exact derivatives, which the
// operator tile multiplies by 1 for every node; zero beyond.
template <int N, class L, int ROLE>
__device__ __forceinline__ void build_x_lift(const float* fr, uint32_t xh, uint32_t xl,
                                             bool row_ok, int rc, float rx, float ry, float sx,
                                             float sy, float a1, float a2, float a3, float b1,
                                             float b2, float b3) {
  using R = RowShare<L, ROLE>;
  constexpr int NPAD = L::NPAD, Nafp = L::Nafp;
  constexpr int NL = R::LHI - R::LLO;
  if constexpr (NL > 0) {
    float x[4 * NL];
    float lin = 0.f;
    if (row_ok) {
      if (rc < 2) {  // a = Ez vertex values
        const float grz = 0.5f * (a2 - a1), gsz = 0.5f * (a3 - a1);
        lin = (rc == 0) ? -(ry * grz + sy * gsz) : (rx * grz + sx * gsz);
      } else {  // a = Hx, b = Hy vertex values
        lin = 0.5f * (rx * (b2 - b1) - ry * (a2 - a1) + sx * (b3 - b1) - sy * (a3 - a1));
      }
    }
    if constexpr (L::LIFT_V4) {
      // fr is 16-byte aligned (FES a multiple of 4) and a chunk that starts
      // below Nafp ends inside the row's FES entries
#pragma unroll
      for (int c = 0; c < NL; ++c) {
        const int j0 = 4 * (R::LLO + c);
        float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
        if (j0 < Nafp && row_ok) f = *reinterpret_cast<const float4*>(fr + j0);
        const float fv[4] = {f.x, f.y, f.z, f.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int jj = j0 + i;
          x[4 * c + i] = jj < Nafp ? fv[i] : (jj == Nafp ? lin : 0.f);
        }
      }
    } else {
#pragma unroll
      for (int v = 0; v < 4 * NL; ++v) {
        const int jj = 4 * R::LLO + v;
        x[v] = 0.f;
        if (jj < Nafp)
          x[v] = row_ok ? fr[jj] : 0.f;
        else if (jj == Nafp)
          x[v] = lin;
      }
    }
    __syncwarp();
    x_emit_run<L, NL>(xh, xl, 2 * NPAD + 4 * R::LLO, x);
  }
}

// Upwind flux of Eq. max2d-numflux with parameter alpha at one face node,
// times Fscale/2 (fsc), for the jumps dH = q- - q+ (at a PEC face dH = 0,
// dEz = 2 Ez-).  Every operation is explicitly rounded: the two sides of a
// face computed in one task (face pairs) then round exactly as when each
// side's own task computes it.
__device__ __forceinline__ void upwind_flux(float nx, float ny, float fsc, float alpha, float dHx,
                                            float dHy, float dEz, float& fx, float& fy,
                                            float& fz) {
  const float fa = __fmul_rn(fsc, alpha);
  const float ndotdH = __fmaf_rn(nx, dHx, __fmul_rn(ny, dHy));
  fx = __fmaf_rn(fa, __fmaf_rn(ndotdH, nx, -dHx), __fmul_rn(__fmul_rn(fsc, ny), dEz));
  fy = __fmaf_rn(fa, __fmaf_rn(ndotdH, ny, -dHy), -__fmul_rn(__fmul_rn(fsc, nx), dEz));
  fz = __fmaf_rn(-fa, dEz, __fmul_rn(fsc, __fmaf_rn(ny, dHx, -__fmul_rn(nx, dHy))));
}
// The same for a per-element permittivity: the exact interface Riemann
// solution fz = cH [Ht] - cE [Ez], lifted as (-Z- ny fz, Z- nx fz, fz).
__device__ __forceinline__ void media_flux(float nx, float ny, float cH, float cE, float zM,
                                           float dHx, float dHy, float dEz, float& fx, float& fy,
                                           float& fz) {
  const float f = __fmaf_rn(cH, __fmaf_rn(ny, dHx, -__fmul_rn(nx, dHy)), -__fmul_rn(cE, dEz));
  fx = -__fmul_rn(__fmul_rn(zM, ny), f);
  fy = __fmul_rn(__fmul_rn(zM, nx), f);
  fz = f;
}

// One CTA's share of a stage launch: the blocks first, first + G, ... of
// the launch (TABLE: from the block table p.blocks; else contiguous blocks of
// E elements over [0, K)).  smem: the CTA's dynamic shared memory (1024-byte
// aligned, L::SMEM_BYTES).  PAIRS: face pairs (a face whose two elements are
// both in the block is done once, by the lower-numbered element's task, for
// both sides, with every flux operation explicitly rounded so that an
// element's result does not depend on whether its neighbour shares its
// block); otherwise each side's task computes its own face nodes.
template <int N, int MODE, int PREC, bool MEDIA, bool TABLE, bool PAIRS = false, bool ALT = false>
__device__ __forceinline__ void tc_stage_body(const StageArgs<float>& p, const int first,
                                              const int G, unsigned char* smem) {
  using L = TcLayout<N, PREC, MEDIA, ALT>;
  constexpr int Np = L::Np, Nfp = L::Nfp, Nafp = L::Nafp, E = L::E, S = L::S;
  constexpr int KP = L::KP, NN = L::NN, NPAD = L::NPAD, FES = L::FES, XBUF = L::XBUF;
  constexpr int FT = L::FLUX_THREADS, TASKS = L::TASKS, TPT = L::TPT;
  constexpr int NQ = (MODE == kModeStage) ? 6 : 3;
  constexpr int GEO = L::GEO;

  // header: mbarriers, TMEM base, abort flag, tables
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);              // [S] stage loaded
  uint64_t* out_ready = reinterpret_cast<uint64_t*>(smem + 64);    // [S] outputs written
  uint64_t* mma_done = reinterpret_cast<uint64_t*>(smem + 128);    // [2] accumulator ready
  uint64_t* tmem_free = reinterpret_cast<uint64_t*>(smem + 144);   // [2] accumulator read
  uint64_t* xfull = reinterpret_cast<uint64_t*>(smem + 160);       // [2] operand rows written
  uint64_t* op_bar = reinterpret_cast<uint64_t*>(smem + 176);      // operator tiles landed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + 184);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + 188);
  int* nbr = reinterpret_cast<int*>(smem + 192);      // [6][Nfp] neighbour face-node table
  float* lam = reinterpret_cast<float*>(smem + 384);  // [2][NPAD] vertex-interpolant weights
  uint64_t* fs_full = reinterpret_cast<uint64_t*>(smem + 704);   // [2] face fluxes written
  uint64_t* fs_empty = reinterpret_cast<uint64_t*>(smem + 720);  // [2] face fluxes read
  unsigned char* stages = smem + L::OFF_STAGES;
  float* Fs = reinterpret_cast<float*>(smem + L::OFF_F);  // [2][3][E][FES] face fluxes

  const int t = threadIdx.x;
  const int warp = t >> 5, lane = t & 31;
  const int K = static_cast<int>(p.K);
  const int nblk = TABLE ? __ldg(p.nblocks) : (K + E - 1) / E;
  const int niter = first < nblk ? (nblk - 1 - first) / G + 1 : 0;
  const int64_t fs = p.fstride;
  // first element and element count of this CTA's block `it`
  auto block_at = [&](int it, int& k0, int& n) {
    const int b = first + it * G;
    if constexpr (TABLE) {
      const int2 d = __ldg(p.blocks + b);
      k0 = d.x;
      n = d.y;
#ifdef DGW_DEVICE_CHECKS
      if (!block_ok(k0, n, E, fs, Np)) {  // no access to the block; the CTA stops
        atomicOr(p.status, kStatusIndex);
        *abort_flag = 1;
        k0 = 0;
        n = 0;
      }
#endif
    } else {
      k0 = b * E;
      n = (K - k0) < E ? (K - k0) : E;
    }
  };

  if (t == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&out_ready[s], 32 * L::EPI_WARPS);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&mma_done[b], 1);
      mbar_init(&tmem_free[b], 32 * L::EPI_WARPS);
      mbar_init(&xfull[b], L::X_THREADS);
      mbar_init(&fs_full[b], FT);
      mbar_init(&fs_empty[b], L::X_THREADS);
    }
    mbar_init(op_bar, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(tmem_slot, L::TMEM_COLS);
  if (t < 6 * Nfp) {
    const int c = t / Nfp, jj = t - c * Nfp;
    nbr[t] = face_node_dev(N, c >> 1, (c & 1) ? (N - jj) : jj);
  }
  if (t < 2 * NPAD) {  // [2][NPAD], zero beyond Np
    const int m = t % NPAD;
    lam[t] = m < Np ? __ldg(p.lam + (t / NPAD) * Np + m) : 0.f;
  }
  for (int idx = t; idx < 2 * L::FB / 4; idx += L::THREADS) Fs[idx] = 0.f;
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  auto fail = [&]() {
    *abort_flag = 1;
    atomicOr(p.status, kStatusTimeout);
  };

  if (warp == L::IO_WARP) {
    if constexpr (L::IO_LANES) {
      // ======================= memory warp: TMA loads, bulk stores.  The copies
      // of a block are issued by several lanes in one instruction (lane f: q
      // field f, 3 + f: res field f, 6: geometry, 7: face codes; stores: lane
      // f field f of q, 3 + f of res); lane 0 alone arms the mbarriers.  Bulk
      // async-groups are per thread, so every lane commits and waits on its own.
      int issued = 0;
      auto issue = [&](int it) {
        const int s = it % S;
        int k0, n;
        block_at(it, k0, n);
#ifdef DGW_DEVICE_CHECKS
        if (n == 0) return;  // rejected block: the abort flag ends every wait
#endif
        const uint32_t qb = round16(static_cast<uint32_t>(n * Np * 4));
        const uint32_t gb = round16(static_cast<uint32_t>(n * GEO * 4));
        const uint32_t cb = round16(static_cast<uint32_t>(n * 3 * 4));
        unsigned char* st = stages + s * L::STAGE_BYTES;
        if (lane == 0) mbar_expect_tx(&full[s], NQ * qb + gb + cb);
        __syncwarp();
        if (lane < 3) {
          tma_load_1d(st + lane * L::QB, p.qin + lane * fs + k0 * Np, qb, &full[s]);
        } else if (lane < 6) {
          if (MODE == kModeStage)
            tma_load_1d(st + lane * L::QB, p.res + (lane - 3) * fs + k0 * Np, qb, &full[s]);
        } else if (lane == 6) {
          tma_load_1d(st + 6 * L::QB, p.geo + static_cast<int64_t>(k0) * GEO, gb, &full[s]);
        } else if (lane == 7) {
          tma_load_1d(st + 6 * L::QB + L::GB, p.conn + static_cast<int64_t>(k0) * 3, cb, &full[s]);
        }
      };
      bool ok = true;
      if (p.stall_gate) {  // timeout test: a flag that nothing sets, bounded wait
        if (lane == 0) {
          const unsigned long long t0 = global_ns();
          while (*reinterpret_cast<const volatile int*>(p.stall_gate) == 0) {
            if (global_ns() - t0 > kGateLimitNs) {
              ok = false;
              break;
            }
            __nanosleep(1000);
          }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
      }
      if (ok) {
        if (lane == 0) {
          mbar_expect_tx(op_bar, L::NS * L::OB);
          tma_load_1d(smem + L::OFF_OP, p.tc_op, L::NS * L::OB, op_bar);
        }
        for (; issued < niter && issued < S; ++issued) issue(issued);
      }
      for (int jj = 0; ok && jj < niter; ++jj) {
        const int s = jj % S;
        ok = __all_sync(0xffffffffu, mbar_wait_or_abort(&out_ready[s],
                                                        static_cast<uint32_t>((jj / S) & 1),
                                                        abort_flag));
        if (!ok) break;
        int k0, nv;
        block_at(jj, k0, nv);
        if (nv == E && lane < 6) {
          const float* sq = reinterpret_cast<const float*>(stages + s * L::STAGE_BYTES);
          if (MODE == kModeRhs) {
            if (lane < 3) tma_store_1d(p.rhs + lane * fs + k0 * Np, sq + lane * E * Np, L::QB);
          } else if (lane < 3) {
            tma_store_1d(p.qout + lane * fs + k0 * Np, sq + lane * E * Np, L::QB);
          } else {
            tma_store_1d(p.res + (lane - 3) * fs + k0 * Np, sq + lane * E * Np, L::QB);
          }
        }
        bulk_commit();
        if (jj >= 1 && issued < niter) {  // issued == jj - 1 + S: the stage of block jj - 1
          bulk_wait_read_but_last();
          __syncwarp();
          fence_proxy_async();
          issue(issued);
          ++issued;
        }
      }
      if (!ok) {
        if (lane == 0) {
          fail();
          // let this CTA's loads in flight land (each wait bounded)
          for (int jj = (issued > S ? issued - S : 0); jj < issued; ++jj)
            mbar_wait_bounded(&full[jj % S], static_cast<uint32_t>((jj / S) & 1), kWaitLimitNs);
        }
      }
      bulk_wait_all();
    } else {
      // ======================= memory warp: TMA loads, bulk stores (lane 0)
      if (lane == 0) {
        int issued = 0;
        auto issue = [&](int it) {
          const int s = it % S;
          int k0, n;
          block_at(it, k0, n);
#ifdef DGW_DEVICE_CHECKS
          if (n == 0) return;  // rejected block: the abort flag ends every wait
#endif
          const uint32_t qb = round16(static_cast<uint32_t>(n * Np * 4));
          const uint32_t gb = round16(static_cast<uint32_t>(n * GEO * 4));
          const uint32_t cb = round16(static_cast<uint32_t>(n * 3 * 4));
          unsigned char* st = stages + s * L::STAGE_BYTES;
          mbar_expect_tx(&full[s], NQ * qb + gb + cb);
#pragma unroll
          for (int f = 0; f < 3; ++f)
            tma_load_1d(st + f * L::QB, p.qin + f * fs + k0 * Np, qb, &full[s]);
          if (MODE == kModeStage) {
#pragma unroll
            for (int f = 0; f < 3; ++f)
              tma_load_1d(st + (3 + f) * L::QB, p.res + f * fs + k0 * Np, qb, &full[s]);
          }
          tma_load_1d(st + 6 * L::QB, p.geo + static_cast<int64_t>(k0) * GEO, gb, &full[s]);
          tma_load_1d(st + 6 * L::QB + L::GB, p.conn + static_cast<int64_t>(k0) * 3, cb, &full[s]);
        };
        bool ok = true;
        if (p.stall_gate) {  // timeout test: a flag that nothing sets, bounded wait
          const unsigned long long t0 = global_ns();
          while (*reinterpret_cast<const volatile int*>(p.stall_gate) == 0) {
            if (global_ns() - t0 > kGateLimitNs) {
              ok = false;
              break;
            }
            __nanosleep(1000);
          }
        }
        if (ok) {
          mbar_expect_tx(op_bar, L::NS * L::OB);
          tma_load_1d(smem + L::OFF_OP, p.tc_op, L::NS * L::OB, op_bar);
          for (; issued < niter && issued < S; ++issued) issue(issued);
        }
        // outputs of block jj leave by bulk stores, one bulk group per block
        // (empty for a short block, whose epilogue writes global memory); the
        // stage of block jj - 1 is refilled once that block's stores have read
        // it, so the warp never waits for the stores it has just issued
        for (int jj = 0; ok && jj < niter; ++jj) {
          const int s = jj % S;
          ok = mbar_wait_or_abort(&out_ready[s], static_cast<uint32_t>((jj / S) & 1), abort_flag);
          if (!ok) break;
          int k0, nv;
          block_at(jj, k0, nv);
          if (nv == E) {
            const float* sq = reinterpret_cast<const float*>(stages + s * L::STAGE_BYTES);
            if (MODE == kModeRhs) {
#pragma unroll
              for (int f = 0; f < 3; ++f)
                tma_store_1d(p.rhs + f * fs + k0 * Np, sq + f * E * Np, L::QB);
            } else {
#pragma unroll
              for (int f = 0; f < 3; ++f) {
                tma_store_1d(p.qout + f * fs + k0 * Np, sq + f * E * Np, L::QB);
                tma_store_1d(p.res + f * fs + k0 * Np, sq + (3 + f) * E * Np, L::QB);
              }
            }
          }
          bulk_commit();
          if (jj >= 1 && issued < niter) {  // issued == jj - 1 + S: the stage of block jj - 1
            bulk_wait_read_but_last();
            fence_proxy_async();
            issue(issued);
            ++issued;
          }
        }
        if (!ok) {
          fail();
          // let this CTA's loads in flight land (each wait bounded)
          for (int jj = (issued > S ? issued - S : 0); jj < issued; ++jj)
            mbar_wait_bounded(&full[jj % S], static_cast<uint32_t>((jj / S) & 1), kWaitLimitNs);
        }
        bulk_wait_all();
      }
    }
  } else if (warp == L::MMA_WARP) {
    // ======================= MMA warp: 2 x (KP / 8) tcgen05.mma per block (lane 0)
    if (lane == 0) {
      bool ok = mbar_wait_or_abort(op_bar, 0, abort_flag);
      const uint32_t oaddr = smem_u32(smem + L::OFF_OP);
      constexpr uint32_t LBO = 128, SBO = L::KG * 128;
      constexpr int KS = KP / (L::BF ? 16 : 8);  // MMA K steps (8 TMEM columns each)
      constexpr uint32_t IDESC2 =                // B = [Op_hi ; Op_lo]
          L::BF ? umma_idesc_bf16(128, 2 * NN) : umma_idesc_tf32(128, 2 * NN);
      constexpr uint32_t IDESC1 = L::BF ? umma_idesc_bf16(128, NN) : umma_idesc_tf32(128, NN);
      auto mma = [&](uint32_t d, uint32_t a, int ks, uint32_t idesc, uint32_t acc,
                     uint32_t b_off = 0) {  // b_off: byte offset of the operator tile
        const uint64_t bd = umma_desc(oaddr + b_off + ks * 256, LBO, SBO);
        if constexpr (L::BF)
          umma_bf16_ta(d, a, bd, idesc, acc);
        else
          umma_tf32_ta(d, a, bd, idesc, acc);
      };
      int mma_pending = -1;  // block whose MMA group may still run
      for (int j = 0; ok && j < niter; ++j) {
        const int xb = j % XBUF;
        ok = mbar_wait_or_abort(&xfull[xb], static_cast<uint32_t>((j / XBUF) & 1), abort_flag);
        if (ok && j >= 2)
          ok = mbar_wait_or_abort(&tmem_free[j & 1], static_cast<uint32_t>(((j - 2) >> 1) & 1),
                                  abort_flag);
        if (!ok) break;
        tc_fence_after();
#pragma unroll
        for (int tile = 0; tile < L::TILES; ++tile) {
        const uint32_t dacc =
            tmem + static_cast<uint32_t>(((j & 1) * L::TILES + tile) * L::ACC_COLS);
        const uint32_t xh =
            tmem + static_cast<uint32_t>(L::OFF_XT + (xb * L::TILES + tile) * L::XCOLS);
        if constexpr (L::NS == 2 && L::ACC_SPLIT) {
#pragma unroll
          for (int ks = 0; ks < KS; ++ks)  // X_hi [Op_hi ; Op_lo] -> columns [0, 2 NN)
            mma(dacc, xh + 8 * ks, ks, IDESC2, ks > 0 ? 1u : 0u);
#pragma unroll
          for (int ks = 0; ks < KS; ++ks)  // + X_lo Op_hi -> columns [0, NN)
            mma(dacc, xh + L::XPART + 8 * ks, ks, IDESC1, 1u);
        } else if constexpr (L::NS == 2) {
#pragma unroll
          for (int ks = 0; ks < KS; ++ks)  // X_hi Op_hi -> columns [0, NN)
            mma(dacc, xh + 8 * ks, ks, IDESC1, ks > 0 ? 1u : 0u);
#pragma unroll
          for (int ks = 0; ks < KS; ++ks)  // + X_hi Op_lo (the lo tile follows the hi tile)
            mma(dacc, xh + 8 * ks, ks, IDESC1, 1u, L::OB);
#pragma unroll
          for (int ks = 0; ks < KS; ++ks)  // + X_lo Op_hi
            mma(dacc, xh + L::XPART + 8 * ks, ks, IDESC1, 1u);
        } else {
#pragma unroll
          for (int ks = 0; ks < KS; ++ks)  // X Op -> columns [0, NN)
            mma(dacc, xh + 8 * ks, ks, IDESC1, ks > 0 ? 1u : 0u);
        }
        }  // tile
        umma_commit(&mma_done[j & 1]);
        mma_pending = j;
      }
      if (!ok) {
        fail();
        if (mma_pending >= 0)
          mbar_wait_bounded(&mma_done[mma_pending & 1],
                            static_cast<uint32_t>((mma_pending >> 1) & 1), kWaitLimitNs);
      }
    }
  } else if (warp >= L::FLUX_WARP0) {
    // ======================= flux warps: upwind flux at every face node
    // into the double-buffered face-flux array, up to two blocks ahead of the
    // operand-row warps; neighbour traces gathered one block ahead
    const int ft = t - 32 * L::FLUX_WARP0;
    const float* qin[3] = {p.qin, p.qin + fs, p.qin + 2 * fs};
    // flux tasks of this thread (the same in every block): element slot,
    // offsets of its own face node, face code, face geometry and flux slot
    int task_e[TPT], task_jj[TPT], task_nm[TPT], task_cf[TPT], task_gf[TPT], task_fo[TPT];
#pragma unroll
    for (int u = 0; u < TPT; ++u) {
      const int tau = ft + u * FT;
      const int ee = tau / Nafp, j = tau - ee * Nafp, f = j / Nfp, jj = j - f * Nfp;
      task_e[u] = tau < TASKS ? ee : E;
      task_jj[u] = jj;
      task_nm[u] = ee * Np + face_node_dev(N, f, jj);
      task_cf[u] = ee * 3 + f;
      task_gf[u] = ee * GEO + 4 + (MEDIA ? 4 : 3) * f;
      task_fo[u] = ee * FES + j;
    }
    float trc[TPT][3];
    auto gather = [&](int it) {
      const int32_t* sc = reinterpret_cast<const int32_t*>(stages + (it % S) * L::STAGE_BYTES +
                                                           6 * L::QB + L::GB);
      int k0, nv;
      block_at(it, k0, nv);
#pragma unroll
      for (int u = 0; u < TPT; ++u) {
        trc[u][0] = trc[u][1] = trc[u][2] = 0.f;
        const int ee = task_e[u];
        if (ee < nv) {
          const int32_t code = sc[task_cf[u]];
#ifdef DGW_DEVICE_CHECKS
          if (!nbr_code_ok(code, fs, Np)) {
            atomicOr(p.status, kStatusIndex);
            continue;
          }
#endif
          // face pairs: a neighbour inside the block is read from the stage
          if (code >= 0 && !(PAIRS && static_cast<unsigned>((code >> 3) - k0) <
                                           static_cast<unsigned>(nv))) {
            const int gP = (code >> 3) * Np + nbr[(code & 7) * Nfp + task_jj[u]];
            trc[u][0] = __ldg(qin[0] + gP);
            trc[u][1] = __ldg(qin[1] + gP);
            trc[u][2] = __ldg(qin[2] + gP);
          }
        }
      }
    };
    bool ok = true;
    if (niter > 0) {
      ok = mbar_wait_or_abort(&full[0], 0, abort_flag);
      if (ok) gather(0);
    }
    for (int j = 0; ok && j < niter; ++j) {
      const int s = j % S;
      ok = mbar_wait_or_abort(&full[s], static_cast<uint32_t>((j / S) & 1), abort_flag);
      // the operand-row warps are done with this flux buffer (block j - 2)
      if (ok && j >= 2)
        ok = mbar_wait_or_abort(&fs_empty[j & 1], static_cast<uint32_t>(((j - 2) >> 1) & 1),
                                abort_flag);
      if (!ok) break;
      int k0, nvalid;
      block_at(j, k0, nvalid);
      const unsigned char* st = stages + s * L::STAGE_BYTES;
      const float* sq = reinterpret_cast<const float*>(st);
      const float* sg = reinterpret_cast<const float*>(st + 6 * L::QB);
      const int32_t* sc = reinterpret_cast<const int32_t*>(st + 6 * L::QB + L::GB);
      float* Fb = Fs + (j & 1) * (L::FB / 4);
      // ---- upwind flux at every face node -> Fb[c][e][j], scaled by Fscale/2
      if constexpr (PAIRS) {
#pragma unroll
        for (int u = 0; u < TPT; ++u) {
          const int ee = task_e[u];
          if (ee < nvalid) {
            const int nM = task_nm[u];
            const int32_t code = sc[task_cf[u]];
            // face pairs: a face whose neighbour eP lies in this block is done
            // once, by the task of the lower-numbered element, for both sides
            // (each side with its own geometry and its own flux slot)
            const int eP = code >= 0 ? (code >> 3) - k0 : -1;
            bool pair = eP >= 0 && eP < nvalid && eP != ee;
#ifdef DGW_DEVICE_CHECKS
            pair = pair && nbr_code_ok(code, fs, Np);  // the gather flagged a bad code
#endif
            if (pair && eP < ee) continue;  // the neighbour's task writes this slot
            const float hxM = sq[nM], hyM = sq[E * Np + nM], ezM = sq[2 * E * Np + nM];
            float hxP, hyP, ezP;
            if (pair) {
              const int nP = eP * Np + nbr[(code & 7) * Nfp + task_jj[u]];
              hxP = sq[nP];
              hyP = sq[E * Np + nP];
              ezP = sq[2 * E * Np + nP];
            } else {
              hxP = trc[u][0];
              hyP = trc[u][1];
              ezP = trc[u][2];
            }
            float dHx, dHy, dEz;
            if (code < 0) {  // PEC wall: Ez+ = -Ez-, H+ = H-
              dHx = 0.f;
              dHy = 0.f;
              dEz = 2.f * ezM;
            } else {
              dHx = hxM - hxP;
              dHy = hyM - hyP;
              dEz = ezM - ezP;
            }
            const float* gf = sg + task_gf[u];
            float* fo = Fb + task_fo[u];
            float fx, fy, fz;
            if constexpr (MEDIA) {
              media_flux(gf[0], gf[1], gf[2], gf[3], sg[ee * GEO + 16], dHx, dHy, dEz, fx, fy, fz);
            } else {
              upwind_flux(gf[0], gf[1], gf[2], p.alpha, dHx, dHy, dEz, fx, fy, fz);
            }
            fo[0] = fx;
            fo[E * FES] = fy;
            fo[2 * E * FES] = fz;
            if (pair) {  // the neighbour's side: its jumps are the negated ones
              const int fP = (code >> 1) & 3;
              const int jjP = (code & 1) ? N - task_jj[u] : task_jj[u];
              const float* gP = sg + eP * GEO + 4 + (MEDIA ? 4 : 3) * fP;
              float* foP = Fb + eP * FES + fP * Nfp + jjP;
              if constexpr (MEDIA) {
                media_flux(gP[0], gP[1], gP[2], gP[3], sg[eP * GEO + 16], hxP - hxM, hyP - hyM,
                           ezP - ezM, fx, fy, fz);
              } else {
                upwind_flux(gP[0], gP[1], gP[2], p.alpha, hxP - hxM, hyP - hyM, ezP - ezM, fx, fy,
                            fz);
              }
              foP[0] = fx;
              foP[E * FES] = fy;
              foP[2 * E * FES] = fz;
            }
          }
        }
      } else {
#pragma unroll
        for (int u = 0; u < TPT; ++u) {
          const int ee = task_e[u];
          if (ee < nvalid) {
            const int nM = task_nm[u];
            const float hxM = sq[nM], hyM = sq[E * Np + nM], ezM = sq[2 * E * Np + nM];
            float dHx, dHy, dEz;
            if (sc[task_cf[u]] < 0) {  // PEC wall: Ez+ = -Ez-, H+ = H-
              dHx = 0.f;
              dHy = 0.f;
              dEz = 2.f * ezM;
            } else {
              dHx = hxM - trc[u][0];
              dHy = hyM - trc[u][1];
              dEz = ezM - trc[u][2];
            }
            const float* gf = sg + task_gf[u];
            float* fo = Fb + task_fo[u];
            if constexpr (MEDIA) {
              // exact interface Riemann solution: fz = cH [Ht] - cE [Ez]
              const float nx = gf[0], ny = gf[1], cH = gf[2], cE = gf[3];
              const float zM = sg[ee * GEO + 16];
              const float fz = cH * (ny * dHx - nx * dHy) - cE * dEz;
              fo[0] = -zM * ny * fz;
              fo[E * FES] = zM * nx * fz;
              fo[2 * E * FES] = fz;
            } else {
              // Eq. max2d-numflux with parameter alpha (1: upwind, 0: central)
              const float nx = gf[0], ny = gf[1], fsc = gf[2], fa = fsc * p.alpha;
              const float ndotdH = nx * dHx + ny * dHy;
              fo[0] = fsc * ny * dEz + fa * (ndotdH * nx - dHx);
              fo[E * FES] = -fsc * nx * dEz + fa * (ndotdH * ny - dHy);
              fo[2 * E * FES] = fsc * (ny * dHx - nx * dHy) - fa * dEz;
            }
          }
        }
      }
      mbar_arrive(&fs_full[j & 1]);
      if (j + 1 < niter) {  // next block's traces, one block ahead
        ok = mbar_wait_or_abort(&full[(j + 1) % S], static_cast<uint32_t>(((j + 1) / S) & 1),
                                abort_flag);
        if (ok) gather(j + 1);
      }
    }
    if (!ok) fail();
  } else if (warp >= L::EPI_WARPS) {
    // ======================= operand-row warps: the GEMM rows into TMEM
    const int quarter = warp & 3;                 // TMEM lanes 32 quarter .. + 31
    const int role = (warp - L::EPI_WARPS) >> 2;  // share of the row's chunks
    const uint32_t lane_base = static_cast<uint32_t>(32 * quarter) << 16;
    bool ok = true;
    for (int j = 0; j < niter; ++j) {
      const int s = j % S;
      ok = ok && mbar_wait_or_abort(&full[s], static_cast<uint32_t>((j / S) & 1), abort_flag);
      // the MMAs that last read this operand buffer are done
      if (ok && j >= XBUF)
        ok = mbar_wait_or_abort(&mma_done[(j - XBUF) & 1],
                                static_cast<uint32_t>(((j - XBUF) >> 1) & 1), abort_flag);
      if (!__all_sync(0xffffffffu, ok)) {
        ok = false;
        break;
      }
      tc_fence_after();
      int k0, nvalid;
      block_at(j, k0, nvalid);
      const unsigned char* st = stages + s * L::STAGE_BYTES;
      const float* sq = reinterpret_cast<const float*>(st);
      const float* sg = reinterpret_cast<const float*>(st + 6 * L::QB);
      const float* Fb = Fs + (j & 1) * (L::FB / 4);

      // ---- this thread's X rows (one per row tile), split into TF32 hi /
      // lo, into tensor memory.  The X_WARPS / 4 warps of a lane quarter share
      // a row's chunks of 4 columns: a contiguous range of volume chunks (Dr
      // and Ds parts) and a contiguous range of LIFT-part chunks, taken from
      // the other end.
      bool row_ok[L::TILES];
      int rc[L::TILES];
      const float* qe[L::TILES];
      const float* fr[L::TILES];
      uint32_t xh[L::TILES], xl[L::TILES];
      float rx[L::TILES], ry[L::TILES], sx[L::TILES], sy[L::TILES];
      float a1[L::TILES], a2[L::TILES], a3[L::TILES], b1[L::TILES], b2[L::TILES], b3[L::TILES];
#pragma unroll
      for (int tile = 0; tile < L::TILES; ++tile) {
        const int r = 128 * tile + 32 * quarter + lane;  // this thread's X row of the tile
        const int c = r / E, re = r - c * E;              // its output field and element
        rc[tile] = c;
        row_ok[tile] = r < L::ROWS && re < nvalid;
        xh[tile] = tmem + lane_base +
                   static_cast<uint32_t>(L::OFF_XT + ((j % XBUF) * L::TILES + tile) * L::XCOLS);
        xl[tile] = xh[tile] + L::XPART;
        qe[tile] = sq + re * Np;
        fr[tile] = Fb + c * E * FES + re * FES;
        rx[tile] = ry[tile] = sx[tile] = sy[tile] = 0.f;
        a1[tile] = a2[tile] = a3[tile] = b1[tile] = b2[tile] = b3[tile] = 0.f;  // vertex values
        if (row_ok[tile]) {
          const float* ge = sg + re * GEO;
          const float* q = qe[tile];
          rx[tile] = ge[0];
          ry[tile] = ge[1];
          sx[tile] = ge[2];
          sy[tile] = ge[3];
          if (c < 2) {  // u = Ez
            a1[tile] = q[2 * E * Np];
            a2[tile] = q[2 * E * Np + N];
            a3[tile] = q[2 * E * Np + Np - 1];
          } else {  // u = Hx, w = Hy
            a1[tile] = q[0];
            a2[tile] = q[N];
            a3[tile] = q[Np - 1];
            b1[tile] = q[E * Np];
            b2[tile] = q[E * Np + N];
            b3[tile] = q[E * Np + Np - 1];
          }
        }
      }
#define DG_BUILD_SHARE(R_)                                                                     \
  do {                                                                                         \
    _Pragma("unroll") for (int tile = 0; tile < L::TILES; ++tile)                              \
      build_x_vol<N, L, R_>(qe[tile], lam, xh[tile], xl[tile], row_ok[tile], rc[tile],         \
                            rx[tile], ry[tile], sx[tile], sy[tile], a1[tile], a2[tile],         \
                            a3[tile], b1[tile], b2[tile], b3[tile]);                           \
    ok = mbar_wait_or_abort(&fs_full[j & 1], static_cast<uint32_t>((j >> 1) & 1), abort_flag); \
    if (__all_sync(0xffffffffu, ok)) {                                                         \
      _Pragma("unroll") for (int tile = 0; tile < L::TILES; ++tile)                            \
        build_x_lift<N, L, R_>(fr[tile], xh[tile], xl[tile], row_ok[tile], rc[tile],           \
                               rx[tile], ry[tile], sx[tile], sy[tile], a1[tile], a2[tile],      \
                               a3[tile], b1[tile], b2[tile], b3[tile]);                        \
    } else {                                                                                   \
      ok = false;                                                                              \
    }                                                                                          \
  } while (0)
      switch (role) {  // compile-time chunk ranges: each share unrolls
        case 0:
          DG_BUILD_SHARE(0);
          break;
        case 1:
          if constexpr (L::X_WARPS / 4 > 1) DG_BUILD_SHARE(1);
          break;
        case 2:
          if constexpr (L::X_WARPS / 4 > 2) DG_BUILD_SHARE(2);
          break;
        default:
          if constexpr (L::X_WARPS / 4 > 3) DG_BUILD_SHARE(3);
          break;
      }
#undef DG_BUILD_SHARE
      tmem_st_wait();
      tc_fence_before();
      if (!ok) break;
      mbar_arrive(&xfull[j % XBUF]);
      mbar_arrive(&fs_empty[j & 1]);
    }
    if (!ok) fail();
  } else {
    // ======================= epilogue warps: accumulator -> stage update
    bool ok = true;
    for (int j = 0; j < niter; ++j) {
      const int s = j % S;
      ok = ok && mbar_wait_or_abort(&mma_done[j & 1], static_cast<uint32_t>((j >> 1) & 1),
                                    abort_flag);
      ok = ok && mbar_wait_or_abort(&full[s], static_cast<uint32_t>((j / S) & 1), abort_flag);
      if (!__all_sync(0xffffffffu, ok)) {
        ok = false;
        break;
      }
      tc_fence_after();
      float acc_t[L::TILES][NN];  // this thread's accumulator row of each tile
#pragma unroll
      for (int tile = 0; tile < L::TILES; ++tile) {
        float* acc = acc_t[tile];
        const uint32_t dacc = tmem +
                              static_cast<uint32_t>(((j & 1) * L::TILES + tile) * L::ACC_COLS) +
                              (static_cast<uint32_t>(32 * warp) << 16);
#pragma unroll
        for (int c0 = 0; c0 < NN; c0 += 16) {
          if constexpr (L::NS == 2 && L::ACC_SPLIT) {
            float va[16], vb[16];
            tmem_ld16(dacc + c0, va);       // X_hi Op_hi + X_lo Op_hi
            tmem_ld16(dacc + NN + c0, vb);  // X_hi Op_lo
#pragma unroll
            for (int q = 0; q < 16; q += 2)
              f32x2_unpack(f32x2_add(f32x2_pack(va[q], va[q + 1]), f32x2_pack(vb[q], vb[q + 1])),
                           acc[c0 + q], acc[c0 + q + 1]);
          } else {
            float va[16];
            tmem_ld16(dacc + c0, va);  // X Op
#pragma unroll
            for (int q = 0; q < 16; ++q) acc[c0 + q] = va[q];
          }
        }
      }
      tmem_ld_wait();
      tc_fence_before();
      mbar_arrive(&tmem_free[j & 1]);

      int k0, nvalid;
      block_at(j, k0, nvalid);
      float* sq = reinterpret_cast<float*>(stages + s * L::STAGE_BYTES);  // q, then outputs
      float* sres = sq + 3 * E * Np;
      // each thread updates its own row of every tile: no ordering with other rows
#pragma unroll
      for (int tile = 0; tile < L::TILES; ++tile) {
        const int r = 128 * tile + 32 * warp + lane;
        const float* acc = acc_t[tile];
        const int c = r / E, e = r - c * E;
        // each thread updates only its own row: no ordering with other rows
        const bool row_ok = r < L::ROWS && e < nvalid;
        // the row's scale of the right-hand side (media records: sH or sE)
        float srow = 1.f;
        if constexpr (MEDIA) {
          if (row_ok) srow = sq[6 * E * Np + e * GEO + (c < 2 ? 17 : 18)];
        }
        const float drow = MEDIA ? p.dt * srow : p.dt;
        // point source on this row (batched launch, Ez row of a source element)
        float samp = 0.f;
        const float* sw = nullptr;
        if constexpr (TABLE && MEDIA && MODE != kModeRhs) {
          const int sid = row_ok && c == 2 ? static_cast<int>(sq[6 * E * Np + e * GEO + 19]) - 1 : -1;
          if (sid >= 0) {
            const double* m = p.src_meta + 4 * sid;
            const double t =
                (static_cast<double>(__ldg(p.step_ctr) - __ldg(p.src_step + sid)) + p.c_stage) * m[0];
            const double aa = (t - m[1]) * m[2];
            samp = static_cast<float>(m[3] * (1.0 - 2.0 * aa * aa) * exp(-aa * aa));
            sw = p.src_w + sid * kSrcStride;
          }
        }
        if (row_ok && nvalid == E) {
          // full block: in place in the stage buffer, node pairs in packed
          // FP32x2 arithmetic (res = a res + dt rhs, q = q + b res)
          float* rq = sq + c * E * Np + e * Np;
          float* rr = sres + c * E * Np + e * Np;
          const f32x2 a2 = f32x2_dup(p.a), b2 = f32x2_dup(p.b), dt2 = f32x2_dup(drow);
#pragma unroll
          for (int n = 0; n + 1 < Np; n += 2) {
            if (MODE == kModeRhs) {
              rq[n] = MEDIA ? srow * acc[n] : acc[n];
              rq[n + 1] = MEDIA ? srow * acc[n + 1] : acc[n + 1];
            } else {
              f32x2 rn = f32x2_mul(dt2, f32x2_pack(acc[n], acc[n + 1]));
              if (MODE == kModeStage) rn = f32x2_fma(a2, f32x2_pack(rr[n], rr[n + 1]), rn);
              const f32x2 qn = f32x2_fma(b2, rn, f32x2_pack(rq[n], rq[n + 1]));
              f32x2_unpack(qn, rq[n], rq[n + 1]);
              f32x2_unpack(rn, rr[n], rr[n + 1]);
            }
          }
          if (Np & 1) {
            constexpr int n = Np - 1;
            if (MODE == kModeRhs) {
              rq[n] = MEDIA ? srow * acc[n] : acc[n];
            } else {
              float rn = __fmul_rn(drow, acc[n]);
              if (MODE == kModeStage) rn = __fmaf_rn(p.a, rr[n], rn);
              rq[n] = __fmaf_rn(p.b, rn, rq[n]);
              rr[n] = rn;
            }
          }
          if constexpr (TABLE && MEDIA && MODE != kModeRhs) {
            if (sw) {  // res += s w, q += b s w
              for (int n = 0; n < Np; ++n) {
                const float v = __fmul_rn(samp, __ldg(sw + n));
                rr[n] = __fadd_rn(rr[n], v);
                rq[n] = __fmaf_rn(p.b, v, rq[n]);
              }
            }
          }
        } else if (row_ok) {
          // ragged last block: straight to global memory, with the same
          // rounded operations as a full block, so that an element's result
          // does not depend on the block it falls in
          const int off = c * E * Np + e * Np;
          const int64_t g = static_cast<int64_t>(c) * fs + static_cast<int64_t>(k0 + e) * Np;
#pragma unroll
          for (int n = 0; n < Np; ++n) {
            if (MODE == kModeRhs) {
              p.rhs[g + n] = MEDIA ? srow * acc[n] : acc[n];
            } else {
              float rn = __fmul_rn(drow, acc[n]);
              if (MODE == kModeStage) rn = __fmaf_rn(p.a, sres[off + n], rn);
              float qn = __fmaf_rn(p.b, rn, sq[off + n]);
              if constexpr (TABLE && MEDIA) {
                if (sw) {
                  const float v = __fmul_rn(samp, __ldg(sw + n));
                  rn = __fadd_rn(rn, v);
                  qn = __fmaf_rn(p.b, v, qn);
                }
              }
              p.qout[g + n] = qn;
              p.res[g + n] = rn;
            }
          }
        }
      }  // tile
      fence_proxy_async();
      mbar_arrive(&out_ready[s]);
    }
    if (!ok) fail();
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, L::TMEM_COLS);
}

template <int N, int MODE, int PREC, bool MEDIA, bool PAIRS, bool ALT>
__global__ void __launch_bounds__(TcLayout<N, PREC, MEDIA, ALT>::THREADS, 1)
    dg_stage_tc_kernel(const __grid_constant__ StageArgs<float> p) {
  extern __shared__ __align__(1024) unsigned char smem[];
  tc_stage_body<N, MODE, PREC, MEDIA, false, PAIRS, ALT>(p, blockIdx.x, gridDim.x, smem);
}

template <int N, int MODE, int PREC, bool MEDIA, bool PAIRS, bool ALT>
cudaError_t launch_stage_tc_mode(const StageArgs<float>& args, int num_sms, cudaStream_t stream) {
  using L = TcLayout<N, PREC, MEDIA, ALT>;
  static std::atomic<uint64_t> configured{0};
  cudaError_t err = configure_once_per_device(configured, [] {
    return cudaFuncSetAttribute(dg_stage_tc_kernel<N, MODE, PREC, MEDIA, PAIRS, ALT>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(L::SMEM_BYTES));
  });
  if (err != cudaSuccess) return err;
  const int64_t nblk = (args.K + L::E - 1) / L::E;
  int64_t grid = num_sms;  // one CTA per SM (shared memory and TMEM sized for it)
  if (grid > nblk) grid = nblk;
  if (grid < 1) grid = 1;
  dg_stage_tc_kernel<N, MODE, PREC, MEDIA, PAIRS, ALT>
      <<<static_cast<unsigned>(grid), L::THREADS, L::SMEM_BYTES, stream>>>(args);
  return cudaGetLastError();
}

template <int N, int PREC, bool MEDIA, bool PAIRS, bool ALT = false>
cudaError_t launch_stage_tc_modes(const StageArgs<float>& args, int mode, int num_sms,
                                  cudaStream_t stream) {
  if (mode == kModeRhs)
    return launch_stage_tc_mode<N, kModeRhs, PREC, MEDIA, PAIRS, ALT>(args, num_sms, stream);
  if (mode == kModeFirstStage)
    return launch_stage_tc_mode<N, kModeFirstStage, PREC, MEDIA, PAIRS, ALT>(args, num_sms, stream);
  return launch_stage_tc_mode<N, kModeStage, PREC, MEDIA, PAIRS, ALT>(args, num_sms, stream);
}

// face pairs (args.face_pairs) and the alternative block size (args.tc_alt)
// exist for the 3xTF32 products, the FP32 path's default; the other product
// variants compute every face node per side in blocks of the default size.
// With both set, face pairs run with the default block size.
template <int N, int PREC, bool MEDIA>
cudaError_t launch_stage_tc_any(const StageArgs<float>& args, int mode, int num_sms,
                                cudaStream_t stream) {
  if constexpr (PREC == kTcTf32x3) {
    if (args.face_pairs)
      return launch_stage_tc_modes<N, PREC, MEDIA, true>(args, mode, num_sms, stream);
    if constexpr (tc_has_alt(N, PREC)) {
      if (args.tc_alt)
        return launch_stage_tc_modes<N, PREC, MEDIA, false, true>(args, mode, num_sms, stream);
    }
  }
  return launch_stage_tc_modes<N, PREC, MEDIA, false>(args, mode, num_sms, stream);
}

template <int N, int PREC>
cudaError_t launch_stage_tc(const StageArgs<float>& args, int mode, int num_sms,
                            cudaStream_t stream) {
  return launch_stage_tc_any<N, PREC, false>(args, mode, num_sms, stream);
}

template <int N>
cudaError_t launch_stage_tc_media(const StageArgs<float>& args, int mode, int num_sms,
                                  cudaStream_t stream) {
  return launch_stage_tc_any<N, kTcTf32x3, true>(args, mode, num_sms, stream);
}

// ------------------------------------------------------------ batched launch
// One persistent launch over every order group of a batch (BatchArgs):
// CTA b runs the body of the order whose CTA range holds b, over that
// group's block table.  Every order's CTA has the same warp layout, so the
// launch has one block size; its dynamic shared memory is the largest any
// present order needs.
constexpr int kTcThreads = TcLayout<5, kTcTf32x3, true>::THREADS;

// one order's share of a batched launch, compiled as a function of its own:
// its registers are allocated for that order alone, so the two-tile bodies
// at N <= 3 fit as in the single-operator kernel (inlined into one kernel,
// the seven bodies spilled, and the launch kept one tile at every order)
template <int N, int MODE>
__device__ __noinline__ void batch_order_body(const StageArgs<float>& g, int first, int G,
                                              unsigned char* smem) {
  tc_stage_body<N, MODE, kTcTf32x3, true, true>(g, first, G, smem);
}

template <int MODE>
__global__ void __launch_bounds__(kTcThreads, 1)
    dg_batch_tc_kernel(const __grid_constant__ BatchArgs p) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int b = blockIdx.x;
  // CTA ranges of the order groups, from device memory
  int c0[8];
#pragma unroll
  for (int g = 0; g < 8; ++g) c0[g] = __ldg(p.cta0 + g);
  // tuning launches: each CTA's start and end time (ns)
  const unsigned long long t_start = p.cta_clock ? global_ns() : 0ull;
#define DG_BATCH_GROUP(NN_)                                                              \
  if (b >= c0[NN_ - 1] && b < c0[NN_]) {                                                 \
    static_assert(TcLayout<NN_, kTcTf32x3, true>::THREADS == kTcThreads, "block size");   \
    batch_order_body<NN_, MODE>(p.g[NN_ - 1], b - c0[NN_ - 1], c0[NN_] - c0[NN_ - 1], smem); \
    if (p.cta_clock && threadIdx.x == 0) {                                               \
      p.cta_clock[2 * b] = t_start;                                                      \
      p.cta_clock[2 * b + 1] = global_ns();                                              \
    }                                                                                    \
    return;                                                                              \
  }
  DG_BATCH_GROUP(1)
  DG_BATCH_GROUP(2)
  DG_BATCH_GROUP(3)
  DG_BATCH_GROUP(4)
  DG_BATCH_GROUP(5)
  DG_BATCH_GROUP(6)
  DG_BATCH_GROUP(7)
#undef DG_BATCH_GROUP
}

// The concurrent launch mode of a batch: each order's share of a stage is a
// kernel of its own (the body inlined, so the stage arguments are kernel
// parameters rather than data reached through a pointer), with one CTA per
// SM striding over the order's block table; the orders' kernels run side by
// side and the hardware gives SMs to whichever has CTAs waiting.  CTAs past
// the order's block count (read from device memory, so that a captured
// graph replays unchanged when problems join or leave) return at once.
template <int N, int MODE, bool ALT>
__global__ void __launch_bounds__(kTcThreads, 1)
    dg_batch_order_kernel(const __grid_constant__ StageArgs<float> g) {
  extern __shared__ __align__(1024) unsigned char smem[];
  if (static_cast<int>(blockIdx.x) >= __ldg(g.nblocks)) return;
  static_assert(TcLayout<N, kTcTf32x3, true, ALT>::THREADS == kTcThreads, "block size");
  tc_stage_body<N, MODE, kTcTf32x3, true, true, false, ALT>(g, blockIdx.x, gridDim.x, smem);
}

// ALT: the order's alternative block size (tc_tiles(N, prec, true)); the
// block table must hold blocks of at most that many elements
template <int N, int MODE, bool ALT>
cudaError_t launch_batch_order(const StageArgs<float>& g, int grid, cudaStream_t stream) {
  if constexpr (ALT && !tc_has_alt(N, kTcTf32x3)) {
    return cudaErrorInvalidValue;
  } else {
    using L = TcLayout<N, kTcTf32x3, true, ALT>;
    static std::atomic<uint64_t> configured{0};
    cudaError_t err = configure_once_per_device(configured, [] {
      return cudaFuncSetAttribute(dg_batch_order_kernel<N, MODE, ALT>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(L::SMEM_BYTES));
    });
    if (err != cudaSuccess) return err;
    if (grid < 1) return cudaSuccess;
    dg_batch_order_kernel<N, MODE, ALT><<<grid, kTcThreads, L::SMEM_BYTES, stream>>>(g);
    return cudaGetLastError();
  }
}

template <int MODE>
cudaError_t launch_batch_tc(const BatchArgs& args, int grid, size_t smem, cudaStream_t stream) {
  static std::atomic<uint64_t> configured{0};
  cudaError_t err = configure_once_per_device(configured, [] {
    return cudaFuncSetAttribute(dg_batch_tc_kernel<MODE>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                TcLayout<5, kTcTf32x3, true>::SMAX);
  });
  if (err != cudaSuccess) return err;
  if (grid < 1) return cudaSuccess;
  dg_batch_tc_kernel<MODE><<<grid, kTcThreads, smem, stream>>>(args);
  return cudaGetLastError();
}

}  // namespace dgw
