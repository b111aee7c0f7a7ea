// FP32 stage kernel with one thread per element ("element threads"), for the
// low orders.
//
// Same result as dg_stage_kernel (kernels.cuh): right-hand side of Eq.
// dg-strong-explicit -- volume derivative by Dr/Ds and the chain rule of Eq.
// dg-diff-local-to-global, upwind flux of Eq. max2d-numflux (parameter
// alpha; PEC by the mirror state Ez+ = -Ez-, H+ = H-) at every face node,
// LIFT of Eq. dg-lift scaled by Fscale/2 -- followed by one 2N-storage
// LSRK(5,4) stage update, or written out as the right-hand side.  The
// products take the same deflated operands (fields minus their linear
// interpolant through the vertex nodes, whose exact derivatives are added
// back per element) and the same four-product form of the volume term,
//   dEz/dt = Dr (rx Hy - ry Hx) + Ds (sx Hy - sy Hx).
//
// At low order the element-local matrices are small (Np = 3 .. 21 nodes), so
// each product is a short dot product whose matrix operand is the same for
// every element.  Here one thread evaluates one element: its nodal values,
// deflated operands and face fluxes stay in registers, and Dr, Ds, LIFT and
// the vertex-interpolant weights are a by-value kernel parameter.  With every
// loop unrolled each matrix entry is a compile-time offset into the
// parameter (constant) bank, which an FMA takes as an operand directly: a
// product term costs one FMA and no load, where the tensor-core kernel
// spends most of its instructions building operand rows and hand-offs.  At
// N = 4, 5 the matrices outgrow the fast constant cache and the unrolled code
// grows large; there they are read from a table in shared memory instead
// (ept_table).  MEDIA: per-element-permittivity records (launch.h), the flux
// of the exact interface Riemann solution and the row scales of the
// right-hand side.
//
// Work decomposition.  A CTA is one warp (residency is then set warp by warp
// by shared memory).  The warp walks blocks of 32 consecutive elements, block
// blockIdx.x + it * gridDim.x, lane e owning element 32 block + e.  All a
// block owns is contiguous in HBM (its q and residual values per field, its
// geometry records and face codes) and is fetched by the warp's lanes with
// 16-byte cp.async copies, one commit group per block, one block ahead: the
// values, residual and geometry into a ring of S = 2 stage buffers (from
// N = 2 on the residual into one buffer of its own, fetched as its block
// starts: ept_res_single), the face codes -- all the neighbour gather needs
// -- one block earlier still, into a ring of three.  So the gather of block
// it + 1 is issued as block it starts and has that whole block to land, and
// so do block it + 1's bulk copies.
// A lane reads its element's values from the stage buffer (a stride of Np
// words: conflict-free for odd Np, 8-byte loads for even Np), gathers its
// neighbours' face-node traces from global memory (L2) into registers, writes
// its updated values back into its own stage slots, and the warp stores the
// block's valid elements with coalesced 16-byte stores.  No wait spins on a
// flag: cp.async.wait_group returns when the warp's own copies have landed.
#pragma once

#include <atomic>
#include <cstring>

#include "kernels.cuh"

namespace dgw {

template <int N>
struct EptOps {
  static constexpr int Np = Order<N>::Np, Nafp = Order<N>::Nafp;
  float dr[Np * Np];    // Dr, row-major
  float ds[Np * Np];    // Ds, row-major
  float lf[Np * Nafp];  // LIFT, row-major (face-node columns, face by face)
  float l2[Np];         // (1 + r_n) / 2: weight of vertex 2 in the linear interpolant
  float l3[Np];         // (1 + s_n) / 2: weight of vertex 3
};

// Stage buffers per warp: two at every order -- one block computed while
// the next one lands.  Deeper rings measured slower on GB300 (N = 1, ms per
// step on the order-sweep mesh: 0.542 with two, 0.598 with three, 0.620 with
// four; N = 2: 0.666 with two, 0.673 with three), because the shared memory
// they take leaves fewer warps resident per SM, and more warps hide more of
// the latency of a block's loads and gathers.
__host__ __device__ constexpr int ept_stages(int) { return 2; }

// Where the products read the reference matrices: false -- the by-value
// parameter, every output node unrolled, each entry an FMA's constant
// operand; true -- a table in shared memory (one row per output node:
// [Dr | Ds over the interior nodes | LIFT], each part padded to 4), read
// with 16-byte broadcast loads in a loop over the output nodes, which keeps
// the code and the constant working set small at the higher orders.
__host__ __device__ constexpr bool ept_table(int N) { return N >= 4; }

// Register and shared-memory economies, per order (each measured A/B on
// GB300, order-sweep meshes, ms per step):
//   ept_prefetch  -- the neighbour traces of the next block are gathered
//                    while this block computes (true), or this block's own
//                    at its start, used after the deflation (false: the
//                    traces are live only until the flux; 80 instead of 128
//                    registers at N = 2, but slower: N = 2 0.703 vs 0.503,
//                    N = 3 0.791 vs 0.615 with a single residual buffer);
//   ept_reread    -- the update reads the element's values back from its
//                    stage slots instead of keeping them in registers (with
//                    the traces not prefetched: N = 2 0.681, N = 3 0.725);
//   ept_res_single -- one residual buffer per warp instead of one per stage
//                    buffer, fetched as its block starts and waited for just
//                    before the update: less shared memory a warp, and the
//                    residual no longer gates the block's start (N = 2 0.503
//                    vs 0.639, N = 3 0.615 vs 0.645, N = 5 1.102 vs 1.131,
//                    N = 4 even; N = 1 0.705 vs 0.675, so not there).
__host__ __device__ constexpr bool ept_prefetch(int) { return true; }
__host__ __device__ constexpr bool ept_reread(int) { return false; }
__host__ __device__ constexpr bool ept_res_single(int N) { return N >= 2; }

// c-th node of an element that is not a vertex node (0, N, Np - 1): the
// deflated operands are zero at the vertex nodes
__host__ __device__ constexpr int ept_interior_node(int N, int c) {
  return c < N - 1 ? c + 1 : c + 2;
}

template <int N, bool MEDIA = false>
struct EptLayout {
  static constexpr int Np = Order<N>::Np, Nfp = Order<N>::Nfp, Nafp = Order<N>::Nafp;
  static constexpr int E = 32;             // elements per block: one per lane
  static constexpr int S = ept_stages(N);  // stage buffers of the warp's ring
  static constexpr int FQ = E * Np;        // floats of one field of a block
  // geometry record length (MEDIA: the per-element-permittivity records,
  // launch.h)
  static constexpr int GEO = MEDIA ? kGeoMedia : kGeo;
  static constexpr int QB = FQ * 4;
  static constexpr int GB = E * GEO * 4;
  static constexpr int CB = E * 3 * 4;
  static constexpr bool PREFETCH = ept_prefetch(N), REREAD = ept_reread(N);
  static constexpr bool RES1 = ept_res_single(N);
  // stage buffer: q[3][E Np], then (unless RES1) res[3][E Np], then
  // geo[E][GEO]
  static constexpr int GEO_OFF = (RES1 ? 3 : 6) * FQ;  // floats
  static constexpr int STAGE_BYTES = GEO_OFF * 4 + GB;
  // RES1: the warp's single residual buffer [3][E Np]
  static constexpr int RES_OFF = S * STAGE_BYTES;
  // face codes: a ring of three blocks' codes, one block ahead of the stages
  static constexpr int CONN_OFF = RES_OFF + (RES1 ? 3 * QB : 0), CONN_BYTES = 3 * CB;
  // operator table (ept_table): row width RS floats, Dr and Ds parts DW
  // wide (Np - 3 interior nodes, padded to 4), LIFT part LW wide
  static constexpr bool TBL = ept_table(N);
  static constexpr int DW = (Np - 3 + 3) / 4 * 4, LW = (Nafp + 3) / 4 * 4;
  static constexpr int RS = 2 * DW + LW;
  static constexpr int TBL_BYTES = TBL ? Np * RS * 4 : 0;
  static constexpr int TBL_OFF = CONN_OFF + CONN_BYTES;
  static constexpr int SMEM_BYTES = TBL_OFF + TBL_BYTES;
  static_assert(S == 2, "the pipeline below waits for one group per block");
  static_assert(Np <= 32, "neighbour node numbers are packed in 5 bits (ept_nbr_nodes)");
  static_assert(QB % 16 == 0 && GB % 16 == 0 && CB % 16 == 0, "16-byte copies");
  static_assert(sizeof(EptOps<N>) == 4 * ept_ops_floats(N), "parameter layout");
};

// Neighbour node for own face-node slot jj, for each value sel = fP * 2 + rev
// of a face connection code's low bits: 5 bits per sel (Np <= 32).
template <int N>
__host__ __device__ constexpr uint32_t ept_nbr_nodes(int jj) {
  uint32_t v = 0;
  for (int sel = 0; sel < 6; ++sel)
    v |= static_cast<uint32_t>(face_node_dev(N, sel >> 1, (sel & 1) ? (N - jj) : jj)) << (5 * sel);
  return v;
}

template <int Np>
__device__ __forceinline__ void ept_ld_row(float (&v)[Np], const float* s) {
  if constexpr (Np % 2 == 0) {  // 8-byte aligned: lane * Np words, Np even
#pragma unroll
    for (int j = 0; j < Np; j += 2) {
      const float2 t = *reinterpret_cast<const float2*>(s + j);
      v[j] = t.x;
      v[j + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int j = 0; j < Np; ++j) v[j] = s[j];
  }
}

// the warp copies PIECES 16-byte pieces global -> shared
template <int PIECES>
__device__ __forceinline__ void ept_fetch(void* dst, const void* src, int lane) {
#pragma unroll
  for (int c = lane; c < PIECES; c += 32)
    cp_async16(static_cast<char*>(dst) + 16 * c, static_cast<const char*>(src) + 16 * c);
}

// the warp stores the first n elements' values of one field of a block
// (FQ = 32 Np floats in shared memory) to global memory
template <int Np>
__device__ __forceinline__ void ept_store(float* dst, const float* src, int n, int lane) {
  constexpr int P = 8 * Np;  // 16-byte pieces of a whole block
  if (n == 32) {
#pragma unroll
    for (int c = lane; c < P; c += 32)
      *reinterpret_cast<float4*>(dst + 4 * c) = *reinterpret_cast<const float4*>(src + 4 * c);
  } else {
    const int nv = n * Np;
    for (int c = lane; 4 * c < nv; c += 32) {
      if (4 * c + 4 <= nv) {
        *reinterpret_cast<float4*>(dst + 4 * c) = *reinterpret_cast<const float4*>(src + 4 * c);
      } else {
        for (int v = 4 * c; v < nv; ++v) dst[v] = src[v];
      }
    }
  }
}

template <int N, int MODE, bool MEDIA>
__global__ void __launch_bounds__(32) dg_stage_ept_kernel(const StageArgs<float> p,
                                                          const EptOps<N> ops) {
  using L = EptLayout<N, MEDIA>;
  constexpr int GEO = L::GEO;
  constexpr int Np = L::Np, Nfp = L::Nfp, Nafp = L::Nafp, S = L::S, FQ = L::FQ;
  extern __shared__ __align__(128) unsigned char smem[];

  const int lane = threadIdx.x;
  const int K = static_cast<int>(p.K);
  const int nblk = (K + 31) >> 5;
  const int G = gridDim.x;
  const int b0 = blockIdx.x;
  const int niter = b0 < nblk ? (nblk - 1 - b0) / G + 1 : 0;
  if (niter == 0) return;
  const float* q0 = p.qin;
  const float* q1 = p.qin + p.fstride;
  const float* q2 = p.qin + 2 * p.fstride;

  auto stage = [&](int it) {
    return reinterpret_cast<float*>(smem + (it % S) * L::STAGE_BYTES);
  };
  auto codes = [&](int it) {
    return reinterpret_cast<int*>(smem + L::CONN_OFF + (it % 3) * L::CB);
  };
  // one commit group per block: the warp fetches block `it`'s values,
  // residual and geometry into its stage buffer, and the face codes of block
  // it + 1 into the code ring (the next block's neighbour gather needs only
  // those).  The first stage of a step does not read the residual (a_1 = 0),
  // nor does the right-hand-side mode.  A block never reaches past the
  // records' padding (Kpad, a multiple of 64) nor past a field (fstride >=
  // Kpad Np).
  auto fetch_codes = [&](int it) {
    const int64_t k0 = static_cast<int64_t>(b0 + it * G) * 32;
    ept_fetch<L::CB / 16>(codes(it), p.conn + k0 * 3, lane);
  };
  auto issue = [&](int it) {
    float* st = stage(it);
    const int64_t k0 = static_cast<int64_t>(b0 + it * G) * 32;
#pragma unroll
    for (int f = 0; f < 3; ++f)
      ept_fetch<L::QB / 16>(st + f * FQ, p.qin + f * p.fstride + k0 * Np, lane);
    if (MODE == kModeStage && !L::RES1) {
#pragma unroll
      for (int f = 0; f < 3; ++f)
        ept_fetch<L::QB / 16>(st + (3 + f) * FQ, p.res + f * p.fstride + k0 * Np, lane);
    }
    ept_fetch<L::GB / 16>(st + L::GEO_OFF, p.geo + k0 * GEO, lane);
    if (it + 1 < niter) fetch_codes(it + 1);
  };
  float* resbuf = reinterpret_cast<float*>(smem + L::RES_OFF);  // RES1
  auto fetch_res = [&](int it) {
    const int64_t k0 = static_cast<int64_t>(b0 + it * G) * 32;
#pragma unroll
    for (int f = 0; f < 3; ++f)
      ept_fetch<L::QB / 16>(resbuf + f * FQ, p.res + f * p.fstride + k0 * Np, lane);
  };

  // neighbour traces (Hx, Hy, Ez) of this lane's element at its Nafp face
  // nodes, for block `it` (its face codes are in the code ring); zero at
  // PEC faces (code -1), whose flux takes the mirror state instead
  float trc[3][Nafp];
  auto gather = [&](int it) {
    const int* sc = codes(it);
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      const int code = sc[lane * 3 + f];
      bool ok = code >= 0;
#ifdef DGW_DEVICE_CHECKS
      if (!nbr_code_ok(code, p.fstride, Np)) {
        atomicOr(p.status, kStatusIndex);
        ok = false;
      }
#endif
      const int base = (code >> 3) * Np;
      const uint32_t sh = 5u * static_cast<uint32_t>(code & 7);
#pragma unroll
      for (int jj = 0; jj < Nfp; ++jj) {
        const int j = f * Nfp + jj;
        trc[0][j] = trc[1][j] = trc[2][j] = 0.f;
        if (ok) {
          const int g = base + static_cast<int>((ept_nbr_nodes<N>(jj) >> sh) & 31u);
          trc[0][j] = __ldg(q0 + g);
          trc[1][j] = __ldg(q1 + g);
          trc[2][j] = __ldg(q2 + g);
        }
      }
    }
  };

  float* tbl = reinterpret_cast<float*>(smem + L::TBL_OFF);
  if constexpr (L::TBL) {
    // the operator table, from the operator's device copies of Dr, Ds, LIFT
    for (int idx = lane; idx < Np * L::RS; idx += 32) {
      const int i = idx / L::RS, c = idx - i * L::RS;
      float v = 0.f;
      if (c < L::DW) {
        if (c < Np - 3) v = __ldg(p.Dr + i * Np + ept_interior_node(N, c));
      } else if (c < 2 * L::DW) {
        if (c - L::DW < Np - 3) v = __ldg(p.Ds + i * Np + ept_interior_node(N, c - L::DW));
      } else if (c - 2 * L::DW < Nafp) {
        v = __ldg(p.LIFT + i * Nafp + (c - 2 * L::DW));
      }
      tbl[idx] = v;
    }
  }

  // prologue: block 0's codes and group 0, then block 0's gather
  fetch_codes(0);
  issue(0);
  cp_async_commit();
  cp_async_wait<0>();
  __syncwarp();
  if (L::PREFETCH) gather(0);

  for (int it = 0; it < niter; ++it) {
    // RES1: this block's residual into the buffer the previous block
    // released (its own group, waited for before the update)
    if (L::RES1) {
      if (MODE == kModeStage) fetch_res(it);
      cp_async_commit();
    }
    // refill the stage the previous block released; then block it has
    // landed (its group was committed one block ago), and so have the codes
    // of block it + 1
    if (it + 1 < niter) issue(it + 1);
    cp_async_commit();
    if (L::RES1)
      cp_async_wait<2>();
    else
      cp_async_wait<1>();
    __syncwarp();
    if (!L::PREFETCH) gather(it);

    float* sq = stage(it);
    const float* sg = sq + L::GEO_OFF;
    const int* sc = codes(it);
    const int k0 = (b0 + it * G) * 32;
    float* own = sq + lane * Np;  // this lane's slot in field 0 (fields FQ apart)

    float hx[Np], hy[Np], ez[Np];
    ept_ld_row<Np>(hx, own);
    ept_ld_row<Np>(hy, own + FQ);
    ept_ld_row<Np>(ez, own + 2 * FQ);
    const float* ge = sg + lane * GEO;
    const float rx = ge[0], ry = ge[1], sx = ge[2], sy = ge[3];
    // row scales of the right-hand side (media records; 1 otherwise)
    const float sH = MEDIA ? ge[17] : 1.f, sE = MEDIA ? ge[18] : 1.f;

    // ---- volume operands minus their linear part (exactly zero at the
    // vertex nodes 0, N, Np - 1), and the linear part's derivatives
    float zd[Np], A[Np], B[Np];
    float lin0, lin1, lin2;
    auto deflate = [&]() {
      const float x1 = hx[0], x2 = hx[N], x3 = hx[Np - 1];
      const float y1 = hy[0], y2 = hy[N], y3 = hy[Np - 1];
      const float z1 = ez[0], z2 = ez[N], z3 = ez[Np - 1];
#pragma unroll
      for (int j = 0; j < Np; ++j) {
        if (j == 0 || j == N || j == Np - 1) {
          zd[j] = A[j] = B[j] = 0.f;
        } else {
          const float dhx = (hx[j] - x1) - ((x2 - x1) * ops.l2[j] + (x3 - x1) * ops.l3[j]);
          const float dhy = (hy[j] - y1) - ((y2 - y1) * ops.l2[j] + (y3 - y1) * ops.l3[j]);
          zd[j] = (ez[j] - z1) - ((z2 - z1) * ops.l2[j] + (z3 - z1) * ops.l3[j]);
          A[j] = rx * dhy - ry * dhx;
          B[j] = sx * dhy - sy * dhx;
        }
      }
      const float grz = 0.5f * (z2 - z1), gsz = 0.5f * (z3 - z1);
      lin0 = -(ry * grz + sy * gsz);
      lin1 = rx * grz + sx * gsz;
      lin2 = 0.5f * (rx * (y2 - y1) - ry * (x2 - x1) + sx * (y3 - y1) - sy * (x3 - x1));
    };
    if (!L::PREFETCH) deflate();

    // ---- upwind flux (Eq. max2d-numflux) times Fscale/2 at every face node
    float F0[Nafp], F1[Nafp], F2[Nafp];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      const bool pec = sc[lane * 3 + f] < 0;
      if constexpr (MEDIA) {
        // the exact interface Riemann solution: fz = cH [Ht] - cE [Ez],
        // lifted terms (-Z- ny fz, Z- nx fz, fz)
        const float nx = ge[4 + 4 * f], ny = ge[5 + 4 * f], cH = ge[6 + 4 * f],
                    cE = ge[7 + 4 * f], zM = ge[16];
#pragma unroll
        for (int jj = 0; jj < Nfp; ++jj) {
          const int n = face_node_dev(N, f, jj);
          const int j = f * Nfp + jj;
          const float dHx = pec ? 0.f : hx[n] - trc[0][j];
          const float dHy = pec ? 0.f : hy[n] - trc[1][j];
          const float dEz = pec ? 2.f * ez[n] : ez[n] - trc[2][j];
          const float fz = cH * (ny * dHx - nx * dHy) - cE * dEz;
          F0[j] = -zM * ny * fz;
          F1[j] = zM * nx * fz;
          F2[j] = fz;
        }
      } else {
        const float nx = ge[4 + 3 * f], ny = ge[5 + 3 * f], fsc = ge[6 + 3 * f];
        const float fa = fsc * p.alpha, fnx = fsc * nx, fny = fsc * ny;
#pragma unroll
        for (int jj = 0; jj < Nfp; ++jj) {
          const int n = face_node_dev(N, f, jj);
          const int j = f * Nfp + jj;
          const float dHx = pec ? 0.f : hx[n] - trc[0][j];
          const float dHy = pec ? 0.f : hy[n] - trc[1][j];
          const float dEz = pec ? 2.f * ez[n] : ez[n] - trc[2][j];
          const float ndH = nx * dHx + ny * dHy;
          F0[j] = fny * dEz + fa * (ndH * nx - dHx);
          F1[j] = -fnx * dEz + fa * (ndH * ny - dHy);
          F2[j] = fny * dHx - fnx * dHy - fa * dEz;
        }
      }
    }

    // ---- the next block's neighbour traces (their L2 latency hides behind
    // this block's products and stores)
    if (L::PREFETCH) {
      if (it + 1 < niter) gather(it + 1);
      deflate();
    }
    // RES1: the residual of this block has landed
    if (L::RES1 && MODE == kModeStage) {
      cp_async_wait<1>();
      __syncwarp();
    }
    float* rown = L::RES1 ? resbuf + lane * Np : own + 3 * FQ;  // residual slot, field 0


    // right-hand side at node i: volume products, chain rule, lift
    auto rhs_at = [&](int i, float& rHx, float& rHy, float& rEz) {
      float dzr = 0.f, dzs = 0.f, ca = 0.f, cb = 0.f;
#pragma unroll
      for (int j = 0; j < Np; ++j) {
        if (j == 0 || j == N || j == Np - 1) continue;
        dzr = fmaf(ops.dr[i * Np + j], zd[j], dzr);
        dzs = fmaf(ops.ds[i * Np + j], zd[j], dzs);
        ca = fmaf(ops.dr[i * Np + j], A[j], ca);
        cb = fmaf(ops.ds[i * Np + j], B[j], cb);
      }
      float l0 = lin0, l1 = lin1, l2 = lin2;
#pragma unroll
      for (int k = 0; k < Nafp; ++k) {
        l0 = fmaf(ops.lf[i * Nafp + k], F0[k], l0);
        l1 = fmaf(ops.lf[i * Nafp + k], F1[k], l1);
        l2 = fmaf(ops.lf[i * Nafp + k], F2[k], l2);
      }
      rHx = l0 - (ry * dzr + sy * dzs);
      rHy = l1 + (rx * dzr + sx * dzs);
      rEz = l2 + (ca + cb);
      if (MEDIA) {
        rHx *= sH;
        rHy *= sH;
        rEz *= sE;
      }
    };

    // ---- stage update (or the right-hand side) into this lane's own slots
    auto update = [&](int i, float rHx, float rHy, float rEz, float& o0, float& o1, float& o2,
                      float& n0, float& n1, float& n2, float r0, float r1, float r2) {
      if (MODE == kModeFirstStage) {
        n0 = p.dt * rHx;
        n1 = p.dt * rHy;
        n2 = p.dt * rEz;
      } else {
        n0 = fmaf(p.a, r0, p.dt * rHx);
        n1 = fmaf(p.a, r1, p.dt * rHy);
        n2 = fmaf(p.a, r2, p.dt * rEz);
      }
      o0 = fmaf(p.b, n0, L::REREAD ? own[i] : hx[i]);
      o1 = fmaf(p.b, n1, L::REREAD ? own[FQ + i] : hy[i]);
      o2 = fmaf(p.b, n2, L::REREAD ? own[2 * FQ + i] : ez[i]);
    };
    if constexpr (L::TBL) {
      // one output node per trip; own values re-read from the stage slots
#pragma unroll 1
      for (int i = 0; i < Np; ++i) {
        const float* row = tbl + i * L::RS;
        float dzr = 0.f, dzs = 0.f, ca = 0.f, cb = 0.f;
#pragma unroll
        for (int c4 = 0; c4 < L::DW; c4 += 4) {
          const float4 d4 = *reinterpret_cast<const float4*>(row + c4);
          const float4 e4 = *reinterpret_cast<const float4*>(row + L::DW + c4);
          const float dv[4] = {d4.x, d4.y, d4.z, d4.w}, ev[4] = {e4.x, e4.y, e4.z, e4.w};
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            if (c4 + u < Np - 3) {
              const int j = ept_interior_node(N, c4 + u);
              dzr = fmaf(dv[u], zd[j], dzr);
              dzs = fmaf(ev[u], zd[j], dzs);
              ca = fmaf(dv[u], A[j], ca);
              cb = fmaf(ev[u], B[j], cb);
            }
          }
        }
        float l0 = lin0, l1 = lin1, l2 = lin2;
#pragma unroll
        for (int c4 = 0; c4 < L::LW; c4 += 4) {
          const float4 f4 = *reinterpret_cast<const float4*>(row + 2 * L::DW + c4);
          const float fv[4] = {f4.x, f4.y, f4.z, f4.w};
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            if (c4 + u < Nafp) {
              l0 = fmaf(fv[u], F0[c4 + u], l0);
              l1 = fmaf(fv[u], F1[c4 + u], l1);
              l2 = fmaf(fv[u], F2[c4 + u], l2);
            }
          }
        }
        float rHx = l0 - (ry * dzr + sy * dzs);
        float rHy = l1 + (rx * dzr + sx * dzs);
        float rEz = l2 + (ca + cb);
        if (MEDIA) {
          rHx *= sH;
          rHy *= sH;
          rEz *= sE;
        }
        if (MODE == kModeRhs) {
          own[i] = rHx;
          own[FQ + i] = rHy;
          own[2 * FQ + i] = rEz;
        } else {
          float n0 = p.dt * rHx, n1 = p.dt * rHy, n2 = p.dt * rEz;
          if (MODE == kModeStage) {
            n0 = fmaf(p.a, rown[i], n0);
            n1 = fmaf(p.a, rown[FQ + i], n1);
            n2 = fmaf(p.a, rown[2 * FQ + i], n2);
          }
          own[i] = fmaf(p.b, n0, own[i]);
          own[FQ + i] = fmaf(p.b, n1, own[FQ + i]);
          own[2 * FQ + i] = fmaf(p.b, n2, own[2 * FQ + i]);
          rown[i] = n0;
          rown[FQ + i] = n1;
          rown[2 * FQ + i] = n2;
        }
      }
    } else if constexpr (Np % 2 == 0) {
#pragma unroll
      for (int i = 0; i < Np; i += 2) {
        float a0, a1, a2, b0_, b1, b2;
        rhs_at(i, a0, a1, a2);
        rhs_at(i + 1, b0_, b1, b2);
        if (MODE == kModeRhs) {
          *reinterpret_cast<float2*>(own + i) = make_float2(a0, b0_);
          *reinterpret_cast<float2*>(own + FQ + i) = make_float2(a1, b1);
          *reinterpret_cast<float2*>(own + 2 * FQ + i) = make_float2(a2, b2);
        } else {
          float2 r0 = make_float2(0.f, 0.f), r1 = r0, r2 = r0;
          if (MODE == kModeStage) {
            r0 = *reinterpret_cast<const float2*>(rown + i);
            r1 = *reinterpret_cast<const float2*>(rown + FQ + i);
            r2 = *reinterpret_cast<const float2*>(rown + 2 * FQ + i);
          }
          float oa0, oa1, oa2, na0, na1, na2, ob0, ob1, ob2, nb0, nb1, nb2;
          update(i, a0, a1, a2, oa0, oa1, oa2, na0, na1, na2, r0.x, r1.x, r2.x);
          update(i + 1, b0_, b1, b2, ob0, ob1, ob2, nb0, nb1, nb2, r0.y, r1.y, r2.y);
          *reinterpret_cast<float2*>(own + i) = make_float2(oa0, ob0);
          *reinterpret_cast<float2*>(own + FQ + i) = make_float2(oa1, ob1);
          *reinterpret_cast<float2*>(own + 2 * FQ + i) = make_float2(oa2, ob2);
          *reinterpret_cast<float2*>(rown + i) = make_float2(na0, nb0);
          *reinterpret_cast<float2*>(rown + FQ + i) = make_float2(na1, nb1);
          *reinterpret_cast<float2*>(rown + 2 * FQ + i) = make_float2(na2, nb2);
        }
      }
    } else {
#pragma unroll
      for (int i = 0; i < Np; ++i) {
        float a0, a1, a2;
        rhs_at(i, a0, a1, a2);
        if (MODE == kModeRhs) {
          own[i] = a0;
          own[FQ + i] = a1;
          own[2 * FQ + i] = a2;
        } else {
          float r0 = 0.f, r1 = 0.f, r2 = 0.f;
          if (MODE == kModeStage) {
            r0 = rown[i];
            r1 = rown[FQ + i];
            r2 = rown[2 * FQ + i];
          }
          float o0, o1, o2, n0, n1, n2;
          update(i, a0, a1, a2, o0, o1, o2, n0, n1, n2, r0, r1, r2);
          own[i] = o0;
          own[FQ + i] = o1;
          own[2 * FQ + i] = o2;
          rown[i] = n0;
          rown[FQ + i] = n1;
          rown[2 * FQ + i] = n2;
        }
      }
    }

    // ---- the warp stores the block's valid elements
    __syncwarp();
    const int n = (K - k0) < 32 ? (K - k0) : 32;
    const int64_t g0 = static_cast<int64_t>(k0) * Np;
    if (MODE == kModeRhs) {
#pragma unroll
      for (int f = 0; f < 3; ++f) ept_store<Np>(p.rhs + f * p.fstride + g0, sq + f * FQ, n, lane);
    } else {
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        ept_store<Np>(p.qout + f * p.fstride + g0, sq + f * FQ, n, lane);
        ept_store<Np>(p.res + f * p.fstride + g0,
                      (L::RES1 ? resbuf : sq + 3 * FQ) + f * FQ, n, lane);
      }
    }
    __syncwarp();  // the stage is free for the next refill
  }
}

template <int N, int MODE, bool MEDIA>
cudaError_t launch_stage_ept_mode(const StageArgs<float>& args, const EptOps<N>& ops, int num_sms,
                                  cudaStream_t stream) {
  using L = EptLayout<N, MEDIA>;
  // per (N, MODE, MEDIA): shared-memory attribute and resident CTAs per SM,
  // set on the first launch on each device
  static std::atomic<uint64_t> configured{0};
  static std::atomic<int> blocks_per_sm{1};
  cudaError_t err = configure_once_per_device(configured, [] {
    cudaError_t e = cudaFuncSetAttribute(dg_stage_ept_kernel<N, MODE, MEDIA>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         L::SMEM_BYTES);
    int nb = 0;
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, dg_stage_ept_kernel<N, MODE, MEDIA>,
                                                        32, L::SMEM_BYTES);
    if (e == cudaSuccess) blocks_per_sm.store(nb > 0 ? nb : 1);
    return e;
  });
  if (err != cudaSuccess) return err;
  const int64_t nblk = (args.K + 31) / 32;
  int64_t grid = static_cast<int64_t>(blocks_per_sm.load()) * num_sms;
  if (grid > nblk) grid = nblk;
  if (grid < 1) grid = 1;
  dg_stage_ept_kernel<N, MODE, MEDIA>
      <<<static_cast<unsigned>(grid), 32, L::SMEM_BYTES, stream>>>(args, ops);
  return cudaGetLastError();
}

template <int N, bool MEDIA>
cudaError_t launch_stage_ept_any(const StageArgs<float>& args, const float* ops_host, int mode,
                                 int num_sms, cudaStream_t stream) {
  EptOps<N> ops;
  std::memcpy(&ops, ops_host, sizeof(ops));
  if (mode == kModeRhs)
    return launch_stage_ept_mode<N, kModeRhs, MEDIA>(args, ops, num_sms, stream);
  if (mode == kModeFirstStage)
    return launch_stage_ept_mode<N, kModeFirstStage, MEDIA>(args, ops, num_sms, stream);
  return launch_stage_ept_mode<N, kModeStage, MEDIA>(args, ops, num_sms, stream);
}

// Definitions of the launchers declared in launch.h; explicitly instantiated
// per order in kernels_ept_N*.cu.
template <int N>
cudaError_t launch_stage_ept(const StageArgs<float>& args, const float* ops_host, int mode,
                             int num_sms, cudaStream_t stream) {
  return launch_stage_ept_any<N, false>(args, ops_host, mode, num_sms, stream);
}
template <int N>
cudaError_t launch_stage_ept_media(const StageArgs<float>& args, const float* ops_host, int mode,
                                   int num_sms, cudaStream_t stream) {
  return launch_stage_ept_any<N, true>(args, ops_host, mode, num_sms, stream);
}

}  // namespace dgw
