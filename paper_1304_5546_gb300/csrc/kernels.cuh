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
// Work decomposition: a CTA owns a block of E consecutive elements and has
// one thread per (element, output node).  The CTAs are persistent and loop
// over element blocks.  Each thread keeps its rows of Dr, Ds and LIFT in
// registers for the whole launch (loaded once), so the element-local
// matrix-vector products read only the field vectors, which sit in shared
// memory and are read as 16-byte vectors broadcast to all threads of an
// element.  Volume terms use the algebraically equal form
//   dEz/dt = Dr (rx Hy - ry Hx) + Ds (sx Hy - sy Hx)
// (geometric factors are constant on an affine element), which needs four
// products per node instead of six.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "launch.h"

namespace dgw {

template <int N>
struct Order {
  static constexpr int Np = (N + 1) * (N + 2) / 2;
  static constexpr int Nfp = N + 1;
  static constexpr int Nafp = 3 * (N + 1);
};

// elements per CTA (E * Np threads).  ptxas budgets registers for the CTA
// rounded up to 4 warps, so E keeps E * Np <= 512 from N = 4 on: each
// thread then has up to 128 registers for its matrix rows (2 Np + Nafp
// values) without spilling.
template <typename T, int N>
constexpr int elems_per_block() {
  constexpr int e32[8] = {0, 64, 32, 32, 32, 24, 18, 14};
  constexpr int e64[8] = {0, 32, 16, 16, 16, 12, 9, 7};
  return sizeof(T) == 8 ? e64[N] : e32[N];
}

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

template <typename T, int N>
struct Layout {
  static constexpr int Np = Order<N>::Np;
  static constexpr int Nafp = Order<N>::Nafp;
  static constexpr int E = elems_per_block<T, N>();
  static constexpr int VW = Vec16<T>::width;
  static constexpr int NPAD = round_up(Np, VW);
  static constexpr int FPAD = round_up(Nafp, VW);
  static constexpr int THREADS = E * Np;
  // shared: Hx, Hy, Ez (raw, for the traces); Ez - Ez_0,
  // A = rx (Hy - Hy_0) - ry (Hx - Hx_0), B = sx (Hy - Hy_0) - sy (Hx - Hx_0)
  // (centred on the element's node 0, for the volume products); 3 fluxes
  static constexpr int SMEM_ELEMS = 6 * E * NPAD + 3 * E * FPAD;
  static constexpr size_t SMEM_BYTES = sizeof(T) * SMEM_ELEMS;
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

template <typename T, int N, int MODE>
__global__ void __launch_bounds__(Layout<T, N>::THREADS)
    dg_stage_kernel(const StageArgs<T> p) {
  using L = Layout<T, N>;
  constexpr int Np = L::Np, Nfp = Order<N>::Nfp, Nafp = L::Nafp;
  constexpr int E = L::E, NPAD = L::NPAD, FPAD = L::FPAD, VW = L::VW;
  constexpr int THREADS = L::THREADS;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sHx = reinterpret_cast<T*>(smem_raw);
  T* sHy = sHx + E * NPAD;
  T* sEz = sHy + E * NPAD;
  T* sA = sEz + E * NPAD;
  T* sB = sA + E * NPAD;
  T* sEc = sB + E * NPAD;
  T* sF = sEc + E * NPAD;  // 3 x E x FPAD

  const int t = threadIdx.x;
  const int e = t / Np;
  const int i = t - e * Np;

  // this thread's rows of Dr, Ds and LIFT, kept in registers
  T dr[Np], ds[Np], lf[Nafp];
#pragma unroll
  for (int m = 0; m < Np; ++m) {
    dr[m] = __ldg(p.Dr + i * Np + m);
    ds[m] = __ldg(p.Ds + i * Np + m);
  }
#pragma unroll
  for (int j = 0; j < Nafp; ++j) lf[j] = __ldg(p.LIFT + i * Nafp + j);

  const int64_t K = p.K;
  const int64_t nblk = (K + E - 1) / E;
  const int64_t fs = p.fstride;

  for (int64_t blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    const int64_t k0 = blk * E;
    const int64_t k = k0 + e;
    const bool valid = k < K;
    const int64_t g = k0 * Np + t;  // == k * Np + i

    // ---- phase 1: own nodal values, residual, geometry
    T hx = 0, hy = 0, ez = 0, r0 = 0, r1 = 0, r2 = 0;
    T rx = 0, ry = 0, sx = 0, sy = 0;
    if (valid) {
      hx = __ldg(p.qin + g);
      hy = __ldg(p.qin + fs + g);
      ez = __ldg(p.qin + 2 * fs + g);
      if (MODE == kModeStage) {
        r0 = p.res[g];
        r1 = p.res[fs + g];
        r2 = p.res[2 * fs + g];
      }
      const T* gk = p.geo + k * kGeo;
      rx = __ldg(gk + 0);
      ry = __ldg(gk + 1);
      sx = __ldg(gk + 2);
      sy = __ldg(gk + 3);
    }
    __syncthreads();  // previous block's readers of shared memory are done
    sHx[e * NPAD + i] = hx;
    sHy[e * NPAD + i] = hy;
    sEz[e * NPAD + i] = ez;
    __syncthreads();

    // ---- volume operands, centred on the element's node 0.  Dr 1 = Ds 1 = 0,
    // so this changes nothing in exact arithmetic; in FP32 it removes the
    // cancellation of O(|u|) products that sum to O(h |grad u|).
    {
      const T hx0 = sHx[e * NPAD], hy0 = sHy[e * NPAD], ez0 = sEz[e * NPAD];
      const T dhx = hx - hx0, dhy = hy - hy0;
      sEc[e * NPAD + i] = ez - ez0;
      sA[e * NPAD + i] = rx * dhy - ry * dhx;
      sB[e * NPAD + i] = sx * dhy - sy * dhx;
    }

    // ---- phase 2: face-trace gather and upwind flux, one task per face node
    for (int tau = t; tau < E * Nafp; tau += THREADS) {
      const int ee = tau / Nafp;
      const int j = tau - ee * Nafp;
      const int64_t kk = k0 + ee;
      if (kk >= K) continue;
      const int f = j / Nfp;
      const int jj = j - f * Nfp;
      const int nM = face_node_dev(N, f, jj);
      const T hxM = sHx[ee * NPAD + nM];
      const T hyM = sHy[ee * NPAD + nM];
      const T ezM = sEz[ee * NPAD + nM];
      const int32_t code = __ldg(p.conn + kk * 3 + f);
      T dHx, dHy, dEz;
      if (code < 0) {  // PEC wall: Ez+ = -Ez-, H+ = H-
        dHx = 0;
        dHy = 0;
        dEz = 2 * ezM;
      } else {
        const int64_t kP = code >> 3;
        const int fP = (code >> 1) & 3;
        const int jP = (code & 1) ? (N - jj) : jj;
        const int64_t gP = kP * Np + face_node_dev(N, fP, jP);
        dHx = hxM - __ldg(p.qin + gP);
        dHy = hyM - __ldg(p.qin + fs + gP);
        dEz = ezM - __ldg(p.qin + 2 * fs + gP);
      }
      const T* gk = p.geo + kk * kGeo + 4 + 3 * f;
      const T nx = __ldg(gk + 0), ny = __ldg(gk + 1), fsc = __ldg(gk + 2);
      const T ndotdH = nx * dHx + ny * dHy;
      const T fHx = ny * dEz + (ndotdH * nx - dHx);
      const T fHy = -nx * dEz + (ndotdH * ny - dHy);
      const T fEz = ny * dHx - nx * dHy - dEz;
      sF[(0 * E + ee) * FPAD + j] = fsc * fHx;
      sF[(1 * E + ee) * FPAD + j] = fsc * fHy;
      sF[(2 * E + ee) * FPAD + j] = fsc * fEz;
    }
    __syncthreads();

    // ---- phase 3: volume products, lift, stage update
    T dEzdr = 0, dEzds = 0, cEz = 0;
    const T* pEz = sEc + e * NPAD;
    const T* pA = sA + e * NPAD;
    const T* pB = sB + e * NPAD;
#pragma unroll
    for (int m0 = 0; m0 < Np; m0 += VW) {
      T vz[VW], va[VW], vb[VW];
      load_vec<T, VW>(vz, pEz + m0);
      load_vec<T, VW>(va, pA + m0);
      load_vec<T, VW>(vb, pB + m0);
#pragma unroll
      for (int u = 0; u < VW; ++u) {
        if (m0 + u < Np) {
          dEzdr += dr[m0 + u] * vz[u];
          dEzds += ds[m0 + u] * vz[u];
          cEz += dr[m0 + u] * va[u] + ds[m0 + u] * vb[u];
        }
      }
    }
    T l0 = 0, l1 = 0, l2 = 0;
    const T* pF0 = sF + (0 * E + e) * FPAD;
    const T* pF1 = sF + (1 * E + e) * FPAD;
    const T* pF2 = sF + (2 * E + e) * FPAD;
#pragma unroll
    for (int j0 = 0; j0 < Nafp; j0 += VW) {
      T f0[VW], f1[VW], f2[VW];
      load_vec<T, VW>(f0, pF0 + j0);
      load_vec<T, VW>(f1, pF1 + j0);
      load_vec<T, VW>(f2, pF2 + j0);
#pragma unroll
      for (int u = 0; u < VW; ++u) {
        if (j0 + u < Nafp) {
          l0 += lf[j0 + u] * f0[u];
          l1 += lf[j0 + u] * f1[u];
          l2 += lf[j0 + u] * f2[u];
        }
      }
    }
    const T rhsHx = -(ry * dEzdr + sy * dEzds) + l0;
    const T rhsHy = (rx * dEzdr + sx * dEzds) + l1;
    const T rhsEz = cEz + l2;

    if (valid) {
      if (MODE == kModeRhs) {
        p.rhs[g] = rhsHx;
        p.rhs[fs + g] = rhsHy;
        p.rhs[2 * fs + g] = rhsEz;
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
        p.res[fs + g] = n1;
        p.res[2 * fs + g] = n2;
        p.qout[g] = hx + p.b * n0;
        p.qout[fs + g] = hy + p.b * n1;
        p.qout[2 * fs + g] = ez + p.b * n2;
      }
    }
  }
}

template <typename T, int N, int MODE>
cudaError_t launch_stage_mode(const StageArgs<T>& args, int num_sms, cudaStream_t stream) {
  using L = Layout<T, N>;
  static int blocks_per_sm = 0;  // per (T, N, MODE), set on the first launch
  if (blocks_per_sm == 0) {
    cudaError_t err = cudaFuncSetAttribute(dg_stage_kernel<T, N, MODE>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(L::SMEM_BYTES));
    if (err != cudaSuccess) return err;
    int nb = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, dg_stage_kernel<T, N, MODE>,
                                                        L::THREADS, L::SMEM_BYTES);
    if (err != cudaSuccess) return err;
    blocks_per_sm = nb > 0 ? nb : 1;
  }
  const int64_t nblk = (args.K + L::E - 1) / L::E;
  int64_t grid = static_cast<int64_t>(blocks_per_sm) * num_sms;
  if (grid > nblk) grid = nblk;
  if (grid < 1) grid = 1;
  dg_stage_kernel<T, N, MODE>
      <<<static_cast<unsigned>(grid), L::THREADS, L::SMEM_BYTES, stream>>>(args);
  return cudaGetLastError();
}

// Definition of the launcher declared in launch.h; explicitly instantiated
// per order in kernels_N*.cu.
template <typename T, int N>
cudaError_t launch_stage(const StageArgs<T>& args, int mode, int num_sms, cudaStream_t stream) {
  if (mode == kModeRhs) return launch_stage_mode<T, N, kModeRhs>(args, num_sms, stream);
  if (mode == kModeFirstStage) return launch_stage_mode<T, N, kModeFirstStage>(args, num_sms, stream);
  return launch_stage_mode<T, N, kModeStage>(args, num_sms, stream);
}

}  // namespace dgw
