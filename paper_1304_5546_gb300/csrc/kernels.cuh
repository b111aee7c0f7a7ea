// Fused nodal-DG stage kernel for the 2D TM Maxwell system.
//
// One launch evaluates the right-hand side of Eq. dg-strong-explicit for
// every element -- the volume derivative (Dr/Ds and the chain rule of
// Eq. dg-diff-local-to-global), the face-trace gather with the upwind flux
// of Eq. max2d-numflux (alpha = 1, PEC by the mirror state Ez+ = -Ez-,
// H+ = H-), and the LIFT apply of Eq. dg-lift scaled by Fscale/2 -- and,
// depending on MODE, writes it out or applies one stage of the 2N-storage
// LSRK(5,4) update res <- a res + dt rhs, q_out <- q_in + b res.
//
// Work decomposition.  The grid is persistent; a CTA walks element blocks
// blk = blockIdx.x + it * gridDim.x of E consecutive elements, one thread
// per (element, output node).  Each thread keeps its rows of Dr, Ds and LIFT
// in registers for the whole launch, so the element-local products read
// only field vectors, from shared memory, as 16-byte vectors broadcast to
// the threads of an element.  The volume term uses the algebraically equal
//   dEz/dt = Dr (rx Hy - ry Hx) + Ds (sx Hy - sy Hx)
// (geometric factors are constant on an affine element): four products per
// node instead of six.  The product operands are the fields minus their
// linear interpolant through the element's three vertex nodes; Dr and Ds
// differentiate that linear part exactly ((u_v2 - u_v1)/2 along r,
// (u_v3 - u_v1)/2 along s), which is added back per element.  Equal in exact
// arithmetic, this keeps FP32 products small for smooth fields (no
// cancellation of O(|u|) or O(h |grad u|) terms).
//
// Memory pipeline.  Everything a block owns is contiguous in HBM (its q and
// residual values per field, its geometry records and face codes), so it is
// fetched by 1D TMA bulk copies into a ring of kStages shared-memory stage
// buffers, completion tracked by one mbarrier per stage; loads for block
// it + kStages are issued while block it computes.  The neighbour traces a
// block needs are gathered into registers one iteration ahead (their
// addresses come from the next stage's face codes), so their L2 latency
// hides behind the current block's products.  Every mbarrier wait is bounded
// (about two seconds); on expiry the CTA sets the status word, waits
// (bounded) for its own copies in flight and returns.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "launch.h"
#include "ptx.cuh"

namespace dgw {

template <int N>
struct Order {
  static constexpr int Np = (N + 1) * (N + 2) / 2;
  static constexpr int Nfp = N + 1;
  static constexpr int Nafp = 3 * (N + 1);
};

// Elements per block: simt_block_elems (launch.h, with the reasons).
template <typename T, int N>
constexpr int elems_per_block() {
  return simt_block_elems(N, sizeof(T) == 8);
}

constexpr int kStages = 3;

template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
  static constexpr int width = 4;
};
template <>
struct Vec16<double> {
  using type = double2;
  static constexpr int width = 2;
};

constexpr int round_up(int x, int m) { return (x + m - 1) / m * m; }

template <typename T, int N, bool MEDIA = false>
struct Layout {
  static constexpr int GEO = MEDIA ? kGeoMedia : kGeo;  // geometry record length
  static constexpr int Np = Order<N>::Np;
  static constexpr int Nfp = Order<N>::Nfp;
  static constexpr int Nafp = Order<N>::Nafp;
  static constexpr int E = elems_per_block<T, N>();
  static constexpr int VW = Vec16<T>::width;
  static constexpr int NPAD = round_up(Np, VW);
  static constexpr int FPAD = round_up(Nafp, VW);
  static constexpr int THREADS = E * Np;
  static constexpr int TASKS = E * Nafp;                       // flux tasks per block
  static constexpr int TPT = (TASKS + THREADS - 1) / THREADS;  // per thread
  // stage buffer: q[3][E Np], res[3][E Np], geo[E][kGeo], conn[E][3]
  static constexpr int QB = E * Np * static_cast<int>(sizeof(T));
  static constexpr int GB = E * GEO * static_cast<int>(sizeof(T));
  static constexpr int CB = E * 3 * 4;
  static constexpr int STAGE_BYTES = round_up(6 * QB + GB + CB, 128);
  // double-buffered work arrays: centred volume operands and lifted fluxes
  static constexpr int W_ELEMS = 3 * E * NPAD;
  static constexpr int F_ELEMS = 3 * E * FPAD;
  static constexpr int HEADER = 512;  // mbarriers + neighbour face-node table
  static_assert(64 + 6 * Nfp * 4 <= HEADER, "header");
  static constexpr size_t SMEM_BYTES =
      HEADER + kStages * STAGE_BYTES + 2 * sizeof(T) * (W_ELEMS + F_ELEMS);
  static_assert(QB % 16 == 0 && GB % 16 == 0 && CB % 16 == 0, "16-byte TMA chunks");
};

__host__ __device__ constexpr int face_node_dev(int N, int f, int j) {
  return f == 0 ? j
                : (f == 1 ? j * (N + 1) - j * (j - 1) / 2 + (N - j) : j * (N + 1) - j * (j - 1) / 2);
}

template <typename T, int W>
__device__ __forceinline__ void load_vec(T (&dst)[W], const T* src) {
  using V = typename Vec16<T>::type;
  *reinterpret_cast<V*>(dst) = *reinterpret_cast<const V*>(src);
}

__host__ __device__ constexpr uint32_t round16(uint32_t x) { return (x + 15u) & ~15u; }

// ------------------------------------------------------------ kernel
// Offsets inside one field are 32-bit (the host guarantees field_stride <
// 2^31); each field has its own 64-bit base pointer.  MEDIA: geometry
// records of kGeoMedia values (per-element permittivity, see launch.h): the
// flux of the exact interface Riemann solution and per-row scales of the
// right-hand side.
template <typename T, int N, int MODE, bool MEDIA>
__global__ void __launch_bounds__(Layout<T, N, MEDIA>::THREADS)
    dg_stage_kernel(const StageArgs<T> p) {
  using L = Layout<T, N, MEDIA>;
  constexpr int GEO = L::GEO;
  constexpr int Np = L::Np, Nfp = L::Nfp, Nafp = L::Nafp;
  constexpr int E = L::E, NPAD = L::NPAD, FPAD = L::FPAD, VW = L::VW;
  constexpr int THREADS = L::THREADS, TASKS = L::TASKS, TPT = L::TPT;
  constexpr int NQ = (MODE == kModeStage) ? 6 : 3;  // field chunks fetched per block

  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  int* nbr = reinterpret_cast<int*>(smem + 64);  // [6][Nfp] neighbour face-node table
  unsigned char* stages = smem + L::HEADER;
  T* Wbuf = reinterpret_cast<T*>(stages + kStages * L::STAGE_BYTES);  // [2][3][E][NPAD]
  T* Fbuf = Wbuf + 2 * L::W_ELEMS;                                    // [2][3][E][FPAD]

  const int t = threadIdx.x;
  const int e = t / Np;
  const int i = t - e * Np;

  const int K = static_cast<int>(p.K);
  const int nblk = (K + E - 1) / E;
  const int G = gridDim.x;
  const int first = blockIdx.x;
  const int niter = first < nblk ? (nblk - 1 - first) / G + 1 : 0;
  const T* qin[3] = {p.qin, p.qin + p.fstride, p.qin + 2 * p.fstride};

  if (t == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
  }
  // neighbour's node for face code bits (fP, rev) and own face-node slot jj:
  // nbr[(2 fP + rev) * Nfp + jj]
  if (t < 6 * Nfp) {
    const int c = t / Nfp, jj = t - c * Nfp;
    nbr[t] = face_node_dev(N, c >> 1, (c & 1) ? (N - jj) : jj);
  }
  __syncthreads();

  // thread 0: fetch everything block `it` owns into stage it % kStages
  auto issue = [&](int it) {
    const int s = it % kStages;
    const int k0 = (first + it * G) * E;
    const int n = (K - k0) < E ? (K - k0) : E;
    const uint32_t qb = round16(static_cast<uint32_t>(n * Np * sizeof(T)));
    const uint32_t gb = round16(static_cast<uint32_t>(n * GEO * sizeof(T)));
    const uint32_t cb = round16(static_cast<uint32_t>(n * 3 * 4));
    unsigned char* st = stages + s * L::STAGE_BYTES;
    mbar_expect_tx(&bars[s], NQ * qb + gb + cb);
#pragma unroll
    for (int f = 0; f < 3; ++f)
      tma_load_1d(st + f * L::QB, p.qin + f * p.fstride + k0 * Np, qb, &bars[s]);
    if (MODE == kModeStage) {
#pragma unroll
      for (int f = 0; f < 3; ++f)
        tma_load_1d(st + (3 + f) * L::QB, p.res + f * p.fstride + k0 * Np, qb, &bars[s]);
    }
    tma_load_1d(st + 6 * L::QB, p.geo + static_cast<int64_t>(k0) * GEO, gb, &bars[s]);
    tma_load_1d(st + 6 * L::QB + L::GB, p.conn + static_cast<int64_t>(k0) * 3, cb, &bars[s]);
  };

  int issued = 0;  // (thread 0) iterations whose loads were issued
  if (t == 0) {
    for (; issued < niter && issued < kStages; ++issued) issue(issued);
  }

  // this thread's rows of Dr, Ds and LIFT, kept in registers
  const T lam2 = __ldg(p.lam + i), lam3 = __ldg(p.lam + Np + i);
  T dr[Np], ds[Np], lf[Nafp];
#pragma unroll
  for (int m = 0; m < Np; ++m) {
    dr[m] = __ldg(p.Dr + i * Np + m);
    ds[m] = __ldg(p.Ds + i * Np + m);
  }
#pragma unroll
  for (int j = 0; j < Nafp; ++j) lf[j] = __ldg(p.LIFT + i * Nafp + j);

  // this thread's flux tasks (the same in every block): element slot, face
  // node slot, face, node on the face
  int task_e[TPT], task_j[TPT], task_f[TPT], task_jj[TPT];
#pragma unroll
  for (int u = 0; u < TPT; ++u) {
    const int tau = t + u * THREADS;
    task_e[u] = tau < TASKS ? tau / Nafp : E;  // E marks "no task"
    task_j[u] = tau - (tau / Nafp) * Nafp;
    task_f[u] = task_j[u] / Nfp;
    task_jj[u] = task_j[u] - task_f[u] * Nfp;
  }

  // neighbour traces of this thread's flux tasks, one block ahead
  T trc[TPT][3];
  auto gather = [&](int it) {
    const int s = it % kStages;
    const int32_t* sc =
        reinterpret_cast<const int32_t*>(stages + s * L::STAGE_BYTES + 6 * L::QB + L::GB);
    const int k0 = (first + it * G) * E;
#pragma unroll
    for (int u = 0; u < TPT; ++u) {
      trc[u][0] = trc[u][1] = trc[u][2] = T(0);
      const int ee = task_e[u];
      if (ee < E && k0 + ee < K) {
        const int32_t code = sc[ee * 3 + task_f[u]];
#ifdef DGW_DEVICE_CHECKS
        if (!nbr_code_ok(code, p.fstride, Np)) {
          atomicOr(p.status, kStatusIndex);
          continue;
        }
#endif
        if (code >= 0) {
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
    ok = mbar_wait_bounded(&bars[0], 0, kWaitLimitNs);
    if (ok) gather(0);
  }

  int it = 0;
  for (; it < niter; ++it) {
    const int s = it % kStages;
    const uint32_t parity = static_cast<uint32_t>((it / kStages) & 1);
    if (ok) ok = mbar_wait_bounded(&bars[s], parity, kWaitLimitNs);
    const int k0 = (first + it * G) * E;
    const bool valid = k0 + e < K;
    const int g = k0 * Np + t;  // == k * Np + i
    const unsigned char* st = stages + s * L::STAGE_BYTES;
    const T* sq = reinterpret_cast<const T*>(st);
    const T* sg = reinterpret_cast<const T*>(st + 6 * L::QB);
    const int32_t* sc = reinterpret_cast<const int32_t*>(st + 6 * L::QB + L::GB);
    T* Wb = Wbuf + (it & 1) * L::W_ELEMS;
    T* Fb = Fbuf + (it & 1) * L::F_ELEMS;

    // ---- phase 1: own values, residual, geometry; volume operands minus
    // their linear part
    T hx = 0, hy = 0, ez = 0, r0 = 0, r1 = 0, r2 = 0, rx = 0, ry = 0, sx = 0, sy = 0;
    T lin0 = 0, lin1 = 0, lin2 = 0;
    T sH = 1, sE = 1;  // row scales of the right-hand side (media records)
    if (ok) {
      hx = sq[t];
      hy = sq[E * Np + t];
      ez = sq[2 * E * Np + t];
      if (MODE == kModeStage) {
        r0 = sq[3 * E * Np + t];
        r1 = sq[4 * E * Np + t];
        r2 = sq[5 * E * Np + t];
      }
      rx = sg[e * GEO + 0];
      ry = sg[e * GEO + 1];
      sx = sg[e * GEO + 2];
      sy = sg[e * GEO + 3];
      if (MEDIA) {
        sH = sg[e * GEO + 17];
        sE = sg[e * GEO + 18];
      }
      const T* qe = sq + e * Np;  // vertex nodes: 0, N, Np - 1
      const T x1 = qe[0], x2 = qe[N], x3 = qe[Np - 1];
      const T y1 = qe[E * Np], y2 = qe[E * Np + N], y3 = qe[E * Np + Np - 1];
      const T z1 = qe[2 * E * Np], z2 = qe[2 * E * Np + N], z3 = qe[2 * E * Np + Np - 1];
      const T dhx = (hx - x1) - ((x2 - x1) * lam2 + (x3 - x1) * lam3);
      const T dhy = (hy - y1) - ((y2 - y1) * lam2 + (y3 - y1) * lam3);
      Wb[(0 * E + e) * NPAD + i] = (ez - z1) - ((z2 - z1) * lam2 + (z3 - z1) * lam3);
      Wb[(1 * E + e) * NPAD + i] = rx * dhy - ry * dhx;
      Wb[(2 * E + e) * NPAD + i] = sx * dhy - sy * dhx;
      // derivatives of the linear part along r and s
      const T grz = T(0.5) * (z2 - z1), gsz = T(0.5) * (z3 - z1);
      lin0 = -(ry * grz + sy * gsz);
      lin1 = rx * grz + sx * gsz;
      lin2 = T(0.5) * (rx * (y2 - y1) - ry * (x2 - x1) + sx * (y3 - y1) - sy * (x3 - x1));
    }
    if (__syncthreads_or(!ok)) break;

    // ---- phase 2: upwind flux at every face node, scaled by Fscale/2
#pragma unroll
    for (int u = 0; u < TPT; ++u) {
      const int ee = task_e[u];
      if (ee < E && k0 + ee < K) {
        const int f = task_f[u], j = task_j[u];
        const int nM = ee * Np + face_node_dev(N, f, task_jj[u]);
        const T hxM = sq[nM], hyM = sq[E * Np + nM], ezM = sq[2 * E * Np + nM];
        T dHx, dHy, dEz;
        if (sc[ee * 3 + f] < 0) {  // PEC wall: Ez+ = -Ez-, H+ = H-
          dHx = 0;
          dHy = 0;
          dEz = 2 * ezM;
        } else {
          dHx = hxM - trc[u][0];
          dHy = hyM - trc[u][1];
          dEz = ezM - trc[u][2];
        }
        if constexpr (MEDIA) {
          // exact interface Riemann solution: fz = cH [Ht] - cE [Ez]
          const T* gf = sg + ee * GEO + 4 + 4 * f;
          const T nx = gf[0], ny = gf[1], cH = gf[2], cE = gf[3];
          const T zM = sg[ee * GEO + 16];
          const T fz = cH * (ny * dHx - nx * dHy) - cE * dEz;
          Fb[(0 * E + ee) * FPAD + j] = -zM * ny * fz;
          Fb[(1 * E + ee) * FPAD + j] = zM * nx * fz;
          Fb[(2 * E + ee) * FPAD + j] = fz;
        } else {
          // Eq. max2d-numflux with parameter alpha (1: upwind, 0: central)
          const T* gf = sg + ee * GEO + 4 + 3 * f;
          const T nx = gf[0], ny = gf[1], fsc = gf[2], fa = fsc * p.alpha;
          const T ndotdH = nx * dHx + ny * dHy;
          Fb[(0 * E + ee) * FPAD + j] = fsc * ny * dEz + fa * (ndotdH * nx - dHx);
          Fb[(1 * E + ee) * FPAD + j] = -fsc * nx * dEz + fa * (ndotdH * ny - dHy);
          Fb[(2 * E + ee) * FPAD + j] = fsc * (ny * dHx - nx * dHy) - fa * dEz;
        }
      }
    }
    // next block's traces: their addresses are in the next stage's codes
    if (it + 1 < niter) {
      const uint32_t par1 = static_cast<uint32_t>(((it + 1) / kStages) & 1);
      ok = mbar_wait_bounded(&bars[(it + 1) % kStages], par1, kWaitLimitNs);
      if (ok) gather(it + 1);
    }
    if (__syncthreads_or(!ok)) break;
    // stage s is no longer read: refill it with block it + kStages
    if (t == 0 && issued < niter) {
      fence_proxy_async();
      issue(issued);
      ++issued;
    }

    // ---- phase 3: volume products, lift, stage update (seven independent
    // accumulation chains)
    T dEzdr = 0, dEzds = 0, cA = 0, cB = 0;
    T l0 = 0, l1 = 0, l2 = 0;
    const T* pEz = Wb + (0 * E + e) * NPAD;
    const T* pA = Wb + (1 * E + e) * NPAD;
    const T* pB = Wb + (2 * E + e) * NPAD;
    const T* pF0 = Fb + (0 * E + e) * FPAD;
    const T* pF1 = Fb + (1 * E + e) * FPAD;
    const T* pF2 = Fb + (2 * E + e) * FPAD;
#pragma unroll
    for (int m0 = 0; m0 < NPAD; m0 += VW) {
      if (m0 < Np) {
        T vz[VW], va[VW], vb[VW];
        load_vec<T, VW>(vz, pEz + m0);
        load_vec<T, VW>(va, pA + m0);
        load_vec<T, VW>(vb, pB + m0);
#pragma unroll
        for (int u = 0; u < VW; ++u) {
          if (m0 + u < Np) {
            dEzdr += dr[m0 + u] * vz[u];
            dEzds += ds[m0 + u] * vz[u];
            cA += dr[m0 + u] * va[u];
            cB += ds[m0 + u] * vb[u];
          }
        }
      }
      if (m0 < Nafp) {
        T f0[VW], f1[VW], f2[VW];
        load_vec<T, VW>(f0, pF0 + m0);
        load_vec<T, VW>(f1, pF1 + m0);
        load_vec<T, VW>(f2, pF2 + m0);
#pragma unroll
        for (int u = 0; u < VW; ++u) {
          if (m0 + u < Nafp) {
            l0 += lf[m0 + u] * f0[u];
            l1 += lf[m0 + u] * f1[u];
            l2 += lf[m0 + u] * f2[u];
          }
        }
      }
    }
    if (FPAD > NPAD) {  // lift columns beyond the volume loop (N = 1, 2)
#pragma unroll
      for (int m0 = NPAD; m0 < Nafp; m0 += VW) {
        T f0[VW], f1[VW], f2[VW];
        load_vec<T, VW>(f0, pF0 + m0);
        load_vec<T, VW>(f1, pF1 + m0);
        load_vec<T, VW>(f2, pF2 + m0);
#pragma unroll
        for (int u = 0; u < VW; ++u) {
          if (m0 + u < Nafp) {
            l0 += lf[m0 + u] * f0[u];
            l1 += lf[m0 + u] * f1[u];
            l2 += lf[m0 + u] * f2[u];
          }
        }
      }
    }
    T rhsHx = -(ry * dEzdr + sy * dEzds) + lin0 + l0;
    T rhsHy = (rx * dEzdr + sx * dEzds) + lin1 + l1;
    T rhsEz = (cA + cB) + lin2 + l2;
    if (MEDIA) {
      rhsHx *= sH;
      rhsHy *= sH;
      rhsEz *= sE;
    }

    if (valid) {
      if (MODE == kModeRhs) {
        p.rhs[g] = rhsHx;
        p.rhs[p.fstride + g] = rhsHy;
        p.rhs[2 * p.fstride + g] = rhsEz;
      } else {
        T n0, n1, n2;
        if (MODE == kModeFirstStage) {
          n0 = p.dt * rhsHx;
          n1 = p.dt * rhsHy;
          n2 = p.dt * rhsEz;
        } else {
          n0 = p.a * r0 + p.dt * rhsHx;
          n1 = p.a * r1 + p.dt * rhsHy;
          n2 = p.a * r2 + p.dt * rhsEz;
        }
        p.res[g] = n0;
        p.res[p.fstride + g] = n1;
        p.res[2 * p.fstride + g] = n2;
        p.qout[g] = hx + p.b * n0;
        p.qout[p.fstride + g] = hy + p.b * n1;
        p.qout[2 * p.fstride + g] = ez + p.b * n2;
      }
    }
  }

  if (it < niter && t == 0) {
    // a wait expired: report, then let this CTA's copies in flight land
    // (each wait bounded) before the CTA's shared memory is released
    atomicOr(p.status, kStatusTimeout);
    for (int j = it; j < issued; ++j)
      mbar_wait_bounded(&bars[j % kStages], static_cast<uint32_t>((j / kStages) & 1),
                        kWaitLimitNs);
  }
}

template <typename T, int N, int MODE, bool MEDIA>
cudaError_t launch_stage_mode(const StageArgs<T>& args, int num_sms, cudaStream_t stream) {
  using L = Layout<T, N, MEDIA>;
  // per (T, N, MODE, MEDIA): shared-memory attribute and resident CTAs per
  // SM, set on the first launch on each device
  static std::atomic<uint64_t> configured{0};
  static std::atomic<int> blocks_per_sm{1};
  cudaError_t err = configure_once_per_device(configured, [] {
    cudaError_t e = cudaFuncSetAttribute(dg_stage_kernel<T, N, MODE, MEDIA>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(L::SMEM_BYTES));
    int nb = 0;
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, dg_stage_kernel<T, N, MODE, MEDIA>,
                                                        L::THREADS, L::SMEM_BYTES);
    if (e == cudaSuccess) blocks_per_sm.store(nb > 0 ? nb : 1);
    return e;
  });
  if (err != cudaSuccess) return err;
  const int64_t nblk = (args.K + L::E - 1) / L::E;
  int64_t grid = static_cast<int64_t>(blocks_per_sm.load()) * num_sms;
  if (grid > nblk) grid = nblk;
  if (grid < 1) grid = 1;
  dg_stage_kernel<T, N, MODE, MEDIA>
      <<<static_cast<unsigned>(grid), L::THREADS, L::SMEM_BYTES, stream>>>(args);
  return cudaGetLastError();
}

template <typename T, int N, bool MEDIA>
cudaError_t launch_stage_any(const StageArgs<T>& args, int mode, int num_sms,
                             cudaStream_t stream) {
  if (mode == kModeRhs) return launch_stage_mode<T, N, kModeRhs, MEDIA>(args, num_sms, stream);
  if (mode == kModeFirstStage)
    return launch_stage_mode<T, N, kModeFirstStage, MEDIA>(args, num_sms, stream);
  return launch_stage_mode<T, N, kModeStage, MEDIA>(args, num_sms, stream);
}

// Definitions of the launchers declared in launch.h; explicitly instantiated
// per order in kernels_N*.cu.
template <typename T, int N>
cudaError_t launch_stage(const StageArgs<T>& args, int mode, int num_sms, cudaStream_t stream) {
  return launch_stage_any<T, N, false>(args, mode, num_sms, stream);
}
template <typename T, int N>
cudaError_t launch_stage_media(const StageArgs<T>& args, int mode, int num_sms,
                               cudaStream_t stream) {
  return launch_stage_any<T, N, true>(args, mode, num_sms, stream);
}

}  // namespace dgw
