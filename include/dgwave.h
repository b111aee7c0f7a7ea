/*
 * dgwave.h -- C ABI of the GB300 nodal discontinuous Galerkin wave solver.
 *
 * The library evaluates the semi-discrete right-hand side of the 2D
 * transverse-magnetic Maxwell system (Hx, Hy, Ez; eps = mu = 1; PEC walls)
 * on an unstructured, straight-sided triangle mesh with the nodal DG method
 * of Kloeckner, Warburton and Hesthaven, "Solving Wave Equations on
 * Unstructured Geometries", and advances it with the five-stage fourth-order
 * low-storage Runge-Kutta scheme LSRK(5,4).
 *
 *   Problem:  Eq. tm-maxwells (Section "A Precise Mathematical Problem
 *             Statement"), PEC condition Ez = 0 on the boundary.
 *   Method:   Eq. dg-strong with the upwind flux of Eq. max2d-numflux
 *             (alpha = 1), in the explicit form Eq. dg-strong-explicit:
 *             element-local differentiation (Eq. dg-diff-local-to-global),
 *             face-trace gather + flux, surface lift (Eq. dg-lift).
 *   Time:     "a simple Runge-Kutta time integrator" (Section "Computing
 *             the Surface Contribution"), here LSRK(5,4).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Node numbering inside an element: Warburton warp-and-blend nodes of
 *   order N on the reference triangle v1 = (-1,-1), v2 = (1,-1), v3 = (-1,1),
 *   numbered row by row of the equidistant lattice (rows of constant s from
 *   s = -1 upwards, r increasing within a row).  Np = (N+1)(N+2)/2.
 * - Element k's vertices are EToV[3k..3k+2]; clockwise input triangles are
 *   re-listed counter-clockwise by swapping their 2nd and 3rd vertex, and
 *   the element's node coordinates follow that (possibly swapped) order.
 *   Faces: face 0 = v1v2, face 1 = v2v3, face 2 = v3v1.
 * - Field buffers ("q", "rhs", "res") are device arrays of 3 fields in the
 *   order Hx, Hy, Ez.  Field f of element k, node n lives at index
 *   f * field_stride + k * Np + n (element-major, node-minor, no padding
 *   inside an element).  field_stride >= K * Np comes from dg_get_info; it
 *   rounds K up to a whole number of kernel blocks and keeps every field
 *   256-byte aligned.  A buffer therefore holds 3 * field_stride values of
 *   the operator's precision (float for DG_FP32, double for DG_FP64).
 *   Entries beyond K * Np in a field are never read for results and never
 *   written.
 * - Ownership: the caller owns every host array it passes in (the library
 *   copies what it keeps) and every device field buffer (the library never
 *   frees or reallocates them).  Handles are owned by the library until
 *   their *_destroy call.  Streams belong to the caller; `stream` is a
 *   cudaStream_t passed as void* (NULL = the legacy default stream).
 * - Asynchrony: dg_rhs, dg_step and dg_solve only enqueue work on `stream`
 *   and return; dg_step_host returns after its results are in host memory.
 *   Launch errors are reported by the call; errors raised while kernels run
 *   surface at the next dg_sync_check (or any later CUDA call).
 * - Errors never abort the process.  A non-zero dg_status leaves every output
 *   untouched for argument errors; dg_last_error() returns a thread-local
 *   message describing the last failure on the calling thread.
 */
#ifndef DGWAVE_H
#define DGWAVE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dg_mesh dg_mesh;
typedef struct dg_op dg_op;
typedef struct dg_batch dg_batch;
typedef int32_t dg_status;

/* A point source (dg_operator_set_source, dg_batch_add, dg_server_submit):
 * the source term f of the problem statement (which the paper leaves
 * unspecified), read as
 *     dEz/dt += s(t) delta(x - (x, y)),
 *     s(t) = amplitude (1 - 2 a^2) exp(-a^2),  a = pi f (t - t0)
 * (a Ricker wavelet of peak frequency f).  For an operator, t is the time
 * dg_step and dg_rhs are given (dg_solve starts at 0); in a batch or a
 * server it is measured from the problem's first step.  The delta is
 * projected onto the nodal basis of the element that contains the point
 * (the lowest-numbered one, barycentric coordinates >= -1e-12):
 * w = M^-1 l(x_s) / J_k, l the element's Lagrange basis at the point; the
 * Ez right-hand side of that element gains s(t) w, after the division by
 * eps.  Stage times are t_n + c_i dt.                                      */
typedef struct dg_point_source {
  double x, y;       /* location, inside the mesh                          */
  double f;          /* peak frequency, > 0                                */
  double t0;         /* time of the peak (1.2 / f is customary)            */
  double amplitude;  /* peak value of s                                    */
} dg_point_source;

#define DG_OK 0
#define DG_ERR_ARG 1                /* bad pointer, size or value            */
#define DG_ERR_MESH_DEGENERATE 2    /* zero-area triangle                    */
#define DG_ERR_MESH_NONCONFORMING 3 /* face shared by more than two elements */
#define DG_ERR_ORDER 4              /* N outside 1..DG_N_MAX                 */
#define DG_ERR_CUDA 5               /* CUDA runtime error / no device        */
#define DG_ERR_OOM 6                /* device or host allocation failed      */
#define DG_ERR_NONFINITE 7          /* NaN or Inf found in a field           */
#define DG_ERR_NO_DEVICE 8          /* operator was set up host-only         */
#define DG_ERR_TIMEOUT 9            /* a kernel's bounded wait expired       */
#define DG_ERR_IO 10                /* a checkpoint file could not be read or
                                       written                               */
#define DG_ERR_INDEX 11             /* a checked build (libdgwave_checked.so)
                                       found an index in device tables out of
                                       range and skipped the access          */

#define DG_FP64 0
#define DG_FP32 1

#define DG_SETUP_HOST_ONLY 1 /* dg_operator_setup flag: skip device upload */
#define DG_SETUP_SIMT 2      /* FP32: element-local products on the CUDA cores
                                instead of the tensor cores (3xTF32)         */
/* FP32 tensor-core product variants (at most one; default: three TF32
 * products per term, hi/lo split of both operands, FP32 accuracy).  Fields,
 * accumulation and the LSRK update stay FP32; only the element-local
 * products (Dr, Ds, LIFT) change precision:                                */
#define DG_SETUP_TC_TF32 4   /* one product, both operands rounded to TF32   */
#define DG_SETUP_TC_BF16 8   /* one product, both operands rounded to BF16   */
#define DG_SETUP_TC_BF16X3 16 /* three BF16 products: hi/lo split of both
                                 operands (X_hi Op_hi + X_hi Op_lo + X_lo Op_hi) */
/* Default FP32 products per order: the element-thread kernel at N <= 2,
 * the tensor cores (3xTF32) from N = 3 on -- the fastest measured at each
 * order, with or without a permittivity.  Overrides:                      */
#define DG_SETUP_TC 32       /* FP32: tensor cores (3xTF32) at every order   */
#define DG_SETUP_ELEMENT_THREADS 64 /* FP32, N <= 5: the CUDA cores with one
                                thread per element, the reference matrices
                                as constant operands                        */

#define DG_N_MAX 7

/* ---------------------------------------------------------------- mesh ---
 * dg_mesh_create: build a conforming triangle mesh from vertex coordinates
 * (vx[Nv], vy[Nv], FP64, host) and a 0-based element-to-vertex table
 * (EToV[3K], int32, host).  Computes element-to-element / element-to-face
 * connectivity (two faces are the same face when they join the same vertex
 * pair; a boundary face points to itself), and re-lists clockwise triangles
 * counter-clockwise.  This is the mesh of Section "Construction of the
 * Method": disjoint, straight-sided, face-conforming triangles.
 * Errors: DG_ERR_ARG (NULL pointer, K < 1, Nv < 3, vertex index out of
 * range, K >= 2^28), DG_ERR_MESH_DEGENERATE (zero area),
 * DG_ERR_MESH_NONCONFORMING (a face shared by three or more elements),
 * DG_ERR_OOM.  *out is written only on success.                           */
dg_status dg_mesh_create(const double* vx, const double* vy, int64_t Nv,
                         const int32_t* EToV, int64_t K, dg_mesh** out);

/* K, number of triangles re-listed counter-clockwise, number of boundary
 * faces.  Any output pointer may be NULL.                                  */
dg_status dg_mesh_info(const dg_mesh* mesh, int64_t* K, int64_t* n_flipped,
                       int64_t* n_boundary_faces);

/* Host copies (K*3 int32 each) of the connectivity: face f of element k
 * joins face EToF[3k+f] of element EToE[3k+f]; boundary faces point to
 * themselves.  Also the oriented EToV (K*3) if EToV_out is not NULL.       */
dg_status dg_mesh_connectivity(const dg_mesh* mesh, int32_t* EToE, int32_t* EToF,
                               int32_t* EToV_out);

void dg_mesh_destroy(dg_mesh* mesh);

/* ----------------------------------------------------------- operator ---
 * dg_operator_setup: everything that needs FP64 is computed on the host in
 * FP64 (Section "Implementation Aspects"): Warburton nodes (cited there for
 * numerical stability), the orthonormal-basis Vandermonde matrix, the
 * reference differentiation matrices Dr, Ds (Eq. dg-diff-local-to-global),
 * face mass matrices and LIFT = M^-1 M^dI (Eq. dg-lift), the affine
 * Jacobians and chain-rule factors rx, ry, sx, sy, outward unit normals and
 * Fscale = surface Jacobian / volume Jacobian (Section "Computing the
 * Surface Contribution"), and the trace maps.  FP32 operators run the
 * element-local products (Dr, Ds, LIFT) on the tensor cores as three TF32
 * products per term (hi/lo splits of both operands, FP32 accumulation) from
 * N = 3 on, and on the CUDA cores below, one thread per element (the
 * element-thread kernel).  DG_SETUP_TC selects the
 * tensor cores at every order, DG_SETUP_SIMT the node-thread CUDA-core FP32
 * kernel, DG_SETUP_ELEMENT_THREADS the element-thread kernel (N <= 5), and
 * one of DG_SETUP_TC_TF32 / _BF16 / _BF16X3 a
 * lower-precision product variant (the precision path of the element-local
 * contractions).  FP64
 * operators always use the CUDA cores.  Unless flags has
 * DG_SETUP_HOST_ONLY, device-ready copies are uploaded once, cast to the
 * operator's precision (DG_FP32 or DG_FP64), to the current CUDA device.
 * The operator keeps its own copy of the mesh data; the mesh may be
 * destroyed afterwards.
 * Errors: DG_ERR_ARG (unknown flags; more than one product variant, or one
 * with DG_FP64 or DG_SETUP_SIMT; DG_SETUP_TC with DG_FP64 or DG_SETUP_SIMT;
 * DG_SETUP_ELEMENT_THREADS with DG_FP64, N > 5 or another kernel or product
 * flag;
 * also when a field would hold 2^31 or more values:
 * kernel offsets inside a field are 32-bit), DG_ERR_ORDER (N < 1 or
 * N > DG_N_MAX), DG_ERR_CUDA, DG_ERR_OOM.  *out is written only on success. */
dg_status dg_operator_setup(const dg_mesh* mesh, int32_t N, int32_t precision,
                            int32_t flags, dg_op** out);

/* dg_operator_setup_media: dg_operator_setup for a medium with a
 * piecewise-constant permittivity, eps[k] > 0 on element k (host, K
 * doubles, copied), and mu = 1: the variable-coefficient form of Eq.
 * tm-maxwells, eps dEz/dt = dHy/dx - dHx/dy (the H equations unchanged).
 * The paper treats eps = mu = 1 only; the flux at an interface between
 * different media is the upwind flux of the exact Riemann solution along the
 * face normal (impedance Z = 1/sqrt(eps), Z- own, Z+ the neighbour's; at a
 * PEC face Z+ = Z-).  With jumps [u] = u- - u+ and [Ht] = ny [Hx] - nx [Hy]:
 *     n.(F - F*) for Ez      = (Z+ [Ht] - [Ez]) / (Z- + Z+)
 *     n.(F - F*) for (Hx,Hy) = (ny, -nx) Z- ([Ez] - Z+ [Ht]) / (Z- + Z+)
 * lifted with Fscale (no extra 1/2), and the Ez right-hand side divided by
 * eps[k].  For eps = 1 this equals the right-hand side of dg_operator_setup
 * up to rounding.  dg_cfl_dt uses min over elements of inradius *
 * sqrt(eps[k]) (the wave speed is 1/sqrt(eps)).  The hot-path calls and
 * their conventions are those of any operator.
 * Errors: those of dg_operator_setup; DG_ERR_ARG when eps is NULL or an
 * entry is not a positive finite number, or with the lower-precision
 * product variants (DG_SETUP_TC_*), which have no per-element-permittivity
 * kernel.                                                                  */
dg_status dg_operator_setup_media(const dg_mesh* mesh, int32_t N, const double* eps,
                                  int32_t precision, int32_t flags, dg_op** out);

/* dg_operator_set_alpha: the flux parameter alpha of Eq. max2d-numflux for
 * later calls on the operator: 1 (the default) is the upwind flux, 0 the
 * central flux n.(F - {F}) of Eq. dg-strong, values between blend the two
 * (the dissipative alpha-terms scale with alpha).  Not for operators with a
 * per-element permittivity.  Errors: DG_ERR_ARG (NULL, alpha outside
 * [0, 1], a media operator).  Calls already enqueued keep their alpha.    */
dg_status dg_operator_set_alpha(dg_op* op, double alpha);

/* dg_operator_set_face_pairs: with enable = 1, later calls on the operator
 * compute the numerical flux of a face whose two elements lie in the same
 * element block of the tensor-core stage kernel once, for both sides, with
 * the neighbour's traces read from the block's shared-memory copy instead
 * of being gathered again (Section "Further Tuning Opportunities": each
 * face pair is otherwise fetched twice, once by each side).  Faces across
 * blocks and PEC faces are computed per side as before.  Each side keeps
 * its own normal and Fscale, and every flux operation is explicitly
 * rounded, so an element's result does not depend on which task computed
 * its faces (partitions, whose blocks differ, agree bit for bit); it
 * differs from enable = 0 by rounding only (the default kernel lets the
 * compiler contract multiply-adds).  It applies to the default 3xTF32
 * products; the other product variants, operators on the CUDA-core kernel
 * (FP64, DG_SETUP_SIMT), the element-thread kernel (FP32 at N <= 2 by
 * default, DG_SETUP_ELEMENT_THREADS) and batches ignore it.
 * Measured slower than the default on GB300 at every order, so off by
 * default.  Errors: DG_ERR_ARG (NULL, enable not 0 or 1).                  */
dg_status dg_operator_set_face_pairs(dg_op* op, int32_t enable);

/* dg_operator_set_source: attach a point source (dg_point_source, copied)
 * to the operator, or remove it (src = NULL).  Later dg_rhs, dg_step,
 * dg_solve, dg_step_host, dg_step_host_jobs and dg_step_static calls add
 * s(t) w to the Ez right-hand side of the element that contains the point:
 * after each stage launch one small kernel adds dt s(t) w to that element's
 * residual and b_i dt s(t) w to its fields (t: the stage time t0 + (n + c_i)
 * dt), which is the stage update with the source in the right-hand side.
 * The projected load w is computed on the host in FP64 and uploaded once
 * (an allocation of Np values, made here, not by the stepping calls).
 * Batches and servers take their own sources and ignore this one;
 * dg_partition_create refuses an operator with a source.
 * Errors: DG_ERR_ARG (NULL operator, parameters not finite or f <= 0, the
 * point outside the mesh), DG_ERR_CUDA, DG_ERR_OOM.                       */
dg_status dg_operator_set_source(dg_op* op, const dg_point_source* src);

/* Np, Nfp = N+1, K and field_stride (see conventions).  NULL outputs are
 * skipped.                                                                 */
dg_status dg_get_info(const dg_op* op, int32_t* Np, int32_t* Nfp, int64_t* K,
                      int64_t* field_stride);

/* Host copies of the physical node coordinates, x[K*Np], y[K*Np] (FP64),
 * index k*Np + n.                                                          */
dg_status dg_get_nodes(const dg_op* op, double* x, double* y);

/* Host copies of the reference element (FP64): r[Np], s[Np], Dr[Np*Np] and
 * Ds[Np*Np] (row-major, row = output node), LIFT[Np*3Nfp] (row-major,
 * column j = face j/Nfp, face node j%Nfp), Fmask[3*Nfp] (node index of each
 * face node, increasing along each face).  NULL outputs are skipped.       */
dg_status dg_get_reference(const dg_op* op, double* r, double* s, double* Dr,
                           double* Ds, double* LIFT, int32_t* Fmask);

/* Host copies of the FP64 geometry: per element rx, ry, sx, sy, J [K];
 * per element face (index 3k+f) nx, ny, Fscale [3K].  NULL outputs are
 * skipped.                                                                 */
dg_status dg_get_geometry(const dg_op* op, double* rx, double* ry, double* sx,
                          double* sy, double* J, double* nx, double* ny,
                          double* Fscale);

/* Host copies of the trace maps, vmapM[K*3Nfp] and vmapP[K*3Nfp] (int64
 * global node numbers k*Np + n of the interior and exterior trace of every
 * face node; boundary face nodes have vmapP = vmapM).                     */
dg_status dg_get_maps(const dg_op* op, int64_t* vmapM, int64_t* vmapP);

/* dg_operator_tune: the kernel and element-block size of an FP32 operator,
 * by measurement.  Times `reps` stage launches of each candidate on the
 * operator's own mesh (scratch fields, allocated and freed here; synchronises
 * `stream`) and keeps the fastest for later calls.  The candidates are:
 *   - the tensor-core kernel (3xTF32) in its default element-block size;
 *   - the same in its alternative size where there is one (40 elements at
 *     N = 1..3, where the default is 80; 80 at N = 4, where it is 40);
 *   - unless DG_SETUP_TC, the CUDA cores: the node-thread kernel, and the
 *     element-thread kernel at N <= 5.
 * Writes the milliseconds per launch of the fastest tensor-core candidate
 * and of the fastest CUDA-core candidate (NULL outputs skipped; -1 where not
 * timed).  Operators whose set-up fixed the kernel and products (FP64,
 * DG_SETUP_SIMT, DG_SETUP_ELEMENT_THREADS, DG_SETUP_TC_*) are left as they
 * are.  dg_operator_kernel
 * reports the choice.  Call it before stepping, not while calls on the
 * operator are in flight.
 * Errors: DG_ERR_ARG (NULL, reps < 1), DG_ERR_NO_DEVICE, DG_ERR_OOM,
 * DG_ERR_CUDA.                                                             */
dg_status dg_operator_tune(dg_op* op, int32_t reps, void* stream, double* ms_tc,
                           double* ms_cuda_cores);

/* dg_operator_set_block_elems: the element-block size of the operator's
 * kernel for later calls: 0 or the default size, or the tensor-core
 * kernel's alternative size where it has one (3xTF32 products; see
 * dg_operator_tune).  The blocks are a kernel's unit of work: each CTA of
 * the persistent launch walks blocks of this many consecutive elements.
 * Results do not depend on the size beyond rounding.  With face pairs on,
 * the default size is used.
 * Errors: DG_ERR_ARG (NULL, a size the operator's kernel does not have). */
dg_status dg_operator_set_block_elems(dg_op* op, int32_t elems);

/* dg_operator_kernel: the kernel the operator's hot-path calls run
 * (DG_KERNEL_*) and its elements per block (the element-thread kernel: 32,
 * one per lane of a warp).  Errors: DG_ERR_ARG (NULL).                    */
#define DG_KERNEL_TENSOR_CORES 0
#define DG_KERNEL_CUDA_CORES 1
#define DG_KERNEL_ELEMENT_THREADS 2
dg_status dg_operator_kernel(const dg_op* op, int32_t* kernel, int32_t* elems);

/* CFL time step: cfl * (2/3) * min over elements of the inradius *
 * (spacing of the first two Gauss-Lobatto points of order N).             */
dg_status dg_cfl_dt(const dg_op* op, double cfl, double* dt);

/* LSRK(5,4) coefficients used by dg_step (each array of 5 doubles, NULL
 * skipped): a, b (Carpenter-Kennedy 2N-storage) and stage times c.        */
dg_status dg_lsrk_coefficients(double* a, double* b, double* c);

void dg_op_destroy(dg_op* op);

/* --------------------------------------------------------- hot path ----
 * dg_rhs: rhs = the semi-discrete right-hand side of Eq. dg-strong-explicit
 * for the three fields in d_q: volume derivative (Dr/Ds + chain rule),
 * face-trace gather with the upwind flux (PEC: Ez+ = -Ez-, H+ = H-), LIFT
 * apply with the factor Fscale/2.  d_q and d_rhs are device field buffers
 * of the operator's precision (3 * field_stride values each, 16-byte
 * aligned; the kernels read whole per-block chunks with bulk copies) and
 * must not overlap.  t is the time of the evaluation: it only matters with
 * a point source (dg_operator_set_source), whose s(t) w is added; without
 * one the system is autonomous.  Enqueued on `stream`.
 * Errors: DG_ERR_ARG (NULL / overlapping / misaligned buffers),
 * DG_ERR_NO_DEVICE, DG_ERR_CUDA (launch failure).                          */
dg_status dg_rhs(const dg_op* op, const void* d_q, void* d_rhs, double t, void* stream);

/* dg_step: nsteps >= 0 LSRK(5,4) steps of size dt starting at t0, in place
 * on d_q.  Each of the 5 stages is ONE fused kernel: right-hand side of the
 * stage's input plus the 2N-storage update
 *     res <- a_i res + dt rhs,   q <- q + b_i res.
 * d_res is a caller-owned device field buffer for the residual (same size
 * as d_q); it needs no initialisation (a_1 = 0: the first stage overwrites
 * it) and holds the last stage's residual on return.  Stages alternate
 * between d_q and an operator-owned device buffer; when nsteps is odd the
 * result is copied back into d_q with one device-to-device copy.  Enqueued
 * on `stream`.  Calls on one operator must not overlap in time (they share
 * that buffer).
 * With a point source, stage i of step n is at time t0 + (n + c_i) dt.
 * Errors: DG_ERR_ARG (NULL/overlapping buffers, nsteps < 0, dt or t0 not
 * finite), DG_ERR_NO_DEVICE, DG_ERR_CUDA.                                  */
dg_status dg_step(const dg_op* op, void* d_q, void* d_res, double t0, double dt,
                  int32_t nsteps, void* stream);

/* dg_solve: advance d_q from t = 0 to T.  dt <= 0 selects dg_cfl_dt(op, 1).
 * The step count is ceil(T/dt) and dt is shrunk to land on T exactly.
 * Writes the step count and the final time (host values, known at enqueue
 * time).  Same buffers and errors as dg_step.                              */
dg_status dg_solve(const dg_op* op, void* d_q, void* d_res, double T, double dt,
                   int32_t* nsteps_out, double* t_reached, void* stream);

/* dg_step_host: dg_step on fields held in HOST memory.  Copies h_q (3 *
 * field_stride values, pinned memory recommended) to the device buffer d_q,
 * runs nsteps steps with d_res as residual buffer, copies the result back
 * into h_q, and synchronises `stream` before returning.                    */
dg_status dg_step_host(const dg_op* op, void* h_q, void* d_q, void* d_res, double t0,
                       double dt, int32_t nsteps, void* stream);

/* dg_step_host_jobs: many independent host-resident field sets, each
 * copied to the device, advanced by nsteps steps and copied back into its
 * own host buffer, with the copies of one job overlapping the steps of the
 * next: job j's copy in runs on one internal stream while job j - 1 steps on
 * `stream`, and job j - 2 is copied out on another.  h_q[j] (j < njobs) are
 * host buffers of 3 * field_stride values each (pinned memory, or the
 * copies do not overlap); a buffer may be listed more than once, and a job
 * then reads it after every earlier job's result has been written there.
 * d_work is caller-owned device memory of dg_step_host_jobs_work_bytes(op)
 * bytes (16-byte aligned): three job slots of two field buffers each and
 * one shared residual buffer.  Every job's stage launches run in order on
 * `stream`, so each result equals that of dg_step_host on the same fields.
 * Returns after every result is in host memory.  Errors: those of
 * dg_step_host, DG_ERR_ARG (njobs < 0, a NULL buffer).                     */
dg_status dg_step_host_jobs(const dg_op* op, int32_t njobs, void* const* h_q, void* d_work,
                            double t0, double dt, int32_t nsteps, void* stream);
int64_t dg_step_host_jobs_work_bytes(const dg_op* op);

/* Size of the scratch array that dg_step_static uses (per device).        */
#define DG_STATIC_SCRATCH_BYTES (32u * 1024u * 1024u)

/* dg_step_static: dg_step whose second field buffer is a fixed array inside
 * the library rather than memory owned by the operator.  The paper has no
 * counterpart; this is a library convenience.
 *
 * Which callers need it: callers that may not allocate device memory when
 * they step, for instance under a fixed device-memory budget that is already
 * handed out, or in a loop that must not call cudaMalloc/cudaFree, which
 * synchronise the whole device.  The call allocates nothing: it uses the
 * caller's d_q and d_res and a DG_STATIC_SCRATCH_BYTES array, one instance
 * per device, that exists as soon as the library's device code is loaded.
 *
 * Result: the same as dg_step with the same arguments (same kernels, same
 * launch order).  Limit: the fields must fit the array, i.e.
 * 3 * field_stride * (4 for DG_FP32, 8 for DG_FP64) <= DG_STATIC_SCRATCH_BYTES
 * (32 MiB: about 133,000 elements at N = 5 in FP32).  Larger operators get
 * DG_ERR_ARG and a message naming the size; use dg_step for them.
 *
 * Nothing in the array has to start at zero.  Each call zeroes the entries
 * of each field beyond K*Np, which the per-block copies read but no result
 * uses.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with the operator's device current), which may load
 * the library's device code.  Make that first call before any stream
 * capture.  The address is kept per device and per context: after the
 * device's context is destroyed and created again (cudaDeviceReset), the
 * next call looks it up afresh, so make that call before any capture too.  Every call with any operator on one device shares the one array:
 * calls that overlap on the GPU (other streams, or other threads' calls not
 * ordered by the caller) race and give wrong results.
 * Errors: those of dg_step; DG_ERR_ARG for fields larger than the array;
 * DG_ERR_CUDA if the address lookup fails.                                 */
dg_status dg_step_static(const dg_op* op, void* d_q, void* d_res, double t0, double dt,
                         int32_t nsteps, void* stream);

/* ------------------------------------------------------------ batches ---
 * A batch steps many independent problems of mixed orders together: each
 * LSRK stage of every problem in the batch is ONE persistent launch (all
 * orders at once; the launch's CTAs are split among the orders), and a step
 * (five stages) is replayed from a captured CUDA graph.  Problems join and
 * leave between steps (continuous batching); each keeps its own time step.
 * Computation: FP32 fields, tensor-core 3xTF32 products, the per-element
 * permittivity flux of dg_operator_setup_media (eps = 1 for operators set
 * up without one).  The paper has no batches: this is the element-blocked,
 * many-problem form of its right-hand side and time stepping.
 *
 * Memory: one pool per order with the element capacity given at creation
 * (about 36 Np + 92 bytes per element of capacity: two field buffers, the
 * residual, geometry records, face codes), allocated by dg_batch_create and
 * freed by dg_batch_destroy.  A problem occupies K elements (rounded up to a
 * multiple of 4) of its order's pool.
 * Fields: the batch owns them.  Problem i's fields are copied in and out
 * with dg_batch_set_fields / dg_batch_get_fields, in the layout of a single
 * operator (field f, element k, node n at f * stride + k * Np + n) with a
 * stride the caller chooses.                                               */
#define DG_BATCH_NO_GRAPH 1 /* dg_batch_create flag: launch the five stage
                               kernels directly instead of replaying graphs */
#define DG_BATCH_NO_ADAPT 2 /* dg_batch_create flag: keep the CTA split fixed
                               between joins and leaves (see dg_batch_step) */
#define DG_BATCH_SPLIT 4    /* dg_batch_create flag: the split launch mode
                               only (see below)                            */

/* Launch modes.  Concurrent (the default): each order's share of a stage
 * is a kernel of its own with one CTA per SM over that order's blocks; the
 * orders' kernels run side by side on streams of the batch, joined once per
 * step, and the hardware hands SMs to whichever order has CTAs waiting, so
 * orders do not wait for each other at every stage.  Split (DG_BATCH_SPLIT,
 * or when dg_batch_tune measures it faster): one launch per stage over all
 * orders, its CTAs split among the orders by the planner.                  */
/* dg_batch_create: capacity[N-1] = elements of order N the batch can hold
 * (N = 1..DG_N_MAX, 0 = none), on the current device.
 * Errors: DG_ERR_ARG (NULL, unknown flags, capacities all zero or one
 * >= 2^27 or too large for 32-bit field offsets), DG_ERR_OOM, DG_ERR_CUDA. */
dg_status dg_batch_create(const int64_t* capacity, int32_t flags, dg_batch** out);
/* flags: DG_BATCH_NO_GRAPH, DG_BATCH_NO_ADAPT (either or both).           */

/* Waits for the device, then frees the batch and its device memory.      */
void dg_batch_destroy(dg_batch* batch);


/* dg_batch_add: admit the problem of operator `op` (DG_FP32; set up on any
 * device or host-only: the batch copies what it needs from the operator's
 * host data, and the operator may be destroyed afterwards) with time step
 * dt (<= 0: the operator's dg_cfl_dt with cfl = 1) and an optional point
 * source (NULL: none; copied).  Its geometry is uploaded asynchronously on
 * `stream`.  Its fields are unspecified until dg_batch_set_fields; it is
 * stepped by every later dg_batch_step, its time starting at 0 with the
 * first of them.  Writes the problem's slot number.
 * Errors: DG_ERR_ARG (NULL, not DG_FP32, no capacity for its order, bad
 * source parameters or a source point outside the mesh), DG_ERR_OOM (no
 * free range of its size in the pool), DG_ERR_CUDA.                       */
dg_status dg_batch_add(dg_batch* batch, const dg_op* op, double dt, const dg_point_source* src,
                       void* stream, int32_t* slot);

/* dg_batch_remove: the problem in `slot` leaves the batch; its range of the
 * pool and its slot number become free.  Copy its fields out first.       */
dg_status dg_batch_remove(dg_batch* batch, int32_t slot);

/* Order, K, time step and pool field stride of the problem in `slot`.     */
dg_status dg_batch_info(const dg_batch* batch, int32_t slot, int32_t* N, int64_t* K, double* dt,
                        int64_t* field_stride);

/* Copy the problem's three fields in (set) or out (get): src / dst hold
 * field f, element k, node n at f * stride + k * Np + n (float), stride >=
 * K * Np, in host (pageable or pinned) or device memory; set with src NULL
 * zeroes the fields.  Enqueued on `stream`, ordered with dg_batch_step calls
 * on the same stream.  set copies a pageable host source into a pinned
 * buffer of the batch first, so it returns without waiting for the device;
 * get into pageable host memory returns once the copy is done (use pinned
 * memory, or dg_server, to keep the host ahead of the device).            */
dg_status dg_batch_set_fields(dg_batch* batch, int32_t slot, const void* src, int64_t src_stride,
                              void* stream);
dg_status dg_batch_get_fields(dg_batch* batch, int32_t slot, void* dst, int64_t dst_stride,
                              void* stream);

/* dg_batch_step: nsteps LSRK(5,4) steps of every problem in the batch, each
 * with its own dt; per stage one launch over all problems.  The first call
 * after a problem joined or left uploads the block tables and CTA split
 * (asynchronously on `stream`).  Calls on one batch must be ordered (one
 * stream, or the caller's synchronisation).  Unless DG_BATCH_NO_ADAPT, the
 * split adapts online: every launch records each CTA's start and end time;
 * every 8 steps a snapshot is copied to host memory, and once it has arrived
 * (checked at a later call, never waited for) each order's cost moves
 * halfway to the cost observed in that launch and the split is re-planned,
 * switching when the predicted makespan is at least 3 % shorter.  The split
 * changes only which CTA computes a block, never a result.
 * Errors: DG_ERR_ARG (nsteps < 0; more orders present than SMs),
 * DG_ERR_OOM, DG_ERR_CUDA.                                                 */
dg_status dg_batch_step(dg_batch* batch, int32_t nsteps, void* stream);

/* dg_batch_tune: the autotuner.  Times `reps` stage launches of each order
 * alone on all SMs (cost of one block iteration per CTA) and plans the CTA
 * split from those costs; then, up to six times, runs the mixed launch with
 * per-CTA clocks, takes each order's cost from its observed finish time
 * (the orders share HBM and L2 there) and re-plans, until the plan no longer
 * changes; finally tries moving single CTAs between orders and keeps every
 * move that measures at least 0.5 % faster.  The fastest measured plan is
 * kept.  Synchronises `stream`; leaves the fields unchanged.  Later joins
 * and leaves re-plan with the last costs.                                  */
dg_status dg_batch_tune(dg_batch* batch, int32_t reps, void* stream);

/* The current plan: CTAs and blocks per order (index N-1) and the per-block
 * cost the planner used (seconds per block iteration of one CTA: measured
 * by dg_batch_tune, before it a table measured on a GB300).  NULL outputs
 * are skipped.                                                             */
dg_status dg_batch_plan(const dg_batch* batch, int32_t* cta, int64_t* nblocks, double* cost);

/* dg_batch_launch_mode: the batch's current launch mode (DG_BATCH_MODE_*)
 * and the last dg_batch_tune timings of `reps` stage launches in each mode
 * (0 before any tuning; the split time is that of the tuned split).      */
#define DG_BATCH_MODE_CONCURRENT 0
#define DG_BATCH_MODE_SPLIT 1
dg_status dg_batch_launch_mode(const dg_batch* batch, int32_t* mode, double* split_ms,
                               double* concurrent_ms);

/* dg_batch_set_block_elems: the element-block size of order N's kernel in
 * the concurrent launch mode: 0 or the default, or the alternative where
 * the order has one (40 at N = 1..3, where the default is 80; 80 at N = 4,
 * where it is 40).  The block tables are rebuilt and the step graphs
 * captured again before the next dg_batch_step.  dg_batch_tune chooses the
 * size per order by measurement (in the concurrent mode).
 * Errors: DG_ERR_ARG (no pool for N, a size order N does not have, the
 * alternative in the split mode).                                          */
dg_status dg_batch_set_block_elems(dg_batch* batch, int32_t N, int32_t elems);

/* dg_batch_block_elems: elems[N-1] = order N's elements per block (0 where
 * the batch has no pool), and the last dg_batch_tune timings of `reps`
 * stage launches of the order alone in its default and alternative size
 * (ms_default / ms_alt, 7 values each, may be NULL; 0 where not timed).   */
dg_status dg_batch_block_elems(const dg_batch* batch, int32_t* elems, double* ms_default,
                               double* ms_alt);

/* The planner on its own (host only): CTAs per order for block counts
 * nblocks[7] and per-block costs cost[7] on num_ctas CTAs.  Every order with
 * blocks gets one CTA; each further CTA goes to the order with the largest
 * ceil(nblocks / cta) * cost that has fewer CTAs than blocks.
 * Errors: DG_ERR_ARG (NULL, num_ctas < 1, more orders with blocks than
 * CTAs).                                                                   */
dg_status dg_batch_plan_ctas(const int64_t* nblocks, const double* cost, int32_t num_ctas,
                             int32_t* cta);

/* Synchronises `stream`, reports pending CUDA errors and the kernels'
 * status word (DG_ERR_TIMEOUT after an expired bounded wait).             */
dg_status dg_batch_sync_check(dg_batch* batch, void* stream);

/* Kernel launches enqueued by the batch: per step five stage launches and
 * one single-thread launch that advances the step counter the point sources
 * read.                                                                   */
int64_t dg_batch_launch_count(const dg_batch* batch);

/* ------------------------------------------------------------ serving ---
 * A solve server: continuous batching of wave-propagation solves on the
 * current device.  A worker thread owns a batch (above) and a stream; it
 * admits submitted requests, oldest first, whenever their order's pool has
 * room (the memory budget is the pools' capacity), steps every admitted
 * request together (one dg_batch_step per chunk of up to 4 steps, so
 * requests that arrive while others run join at the next chunk boundary),
 * and retires each request at its final time: its fields go to host memory
 * and its pool range is free for the next admission.  A request's result
 * does not depend on what else runs with it.  The paper has no server: this
 * is the serving form of dg_solve with a point source.                    */
#define DG_SERVER_SEQUENTIAL 1 /* dg_server_create flag: admit a request only
                                  when none is running (one solve at a time) */

#define DG_REQUEST_QUEUED 0
#define DG_REQUEST_RUNNING 1
#define DG_REQUEST_DONE 2
#define DG_REQUEST_FAILED 3
#define DG_REQUEST_CANCELLED 4

typedef struct dg_server dg_server;

/* Times in seconds on the library's steady clock (dg_server_clock).       */
typedef struct dg_request_info {
  int32_t state;    /* DG_REQUEST_*                                        */
  int32_t status;   /* why a failed request failed (DG_ERR_OOM: it does not
                       fit the pool of its order even when empty)          */
  int32_t N;
  int64_t K;
  int64_t nsteps;   /* LSRK steps to the final time                        */
  double dt;        /* step: T / ceil(T / dg_cfl_dt(op, 1))                */
  double t_submit, t_admit, t_done;
  double t_retired; /* left the batch: its last step enqueued (0 if it never
                       ran to its final time)                              */
} dg_request_info;

/* The steady clock of the request times (seconds).                        */
double dg_server_clock(void);

/* capacity[N-1]: elements of order N the server's batch can hold.  Starts
 * the worker thread.  Errors: those of dg_batch_create.                   */
dg_status dg_server_create(const int64_t* capacity, int32_t flags, dg_server** out);

/* Finishes every submitted request, stops the worker and frees everything. */
void dg_server_destroy(dg_server* server);

/* dg_server_set_work_limit: bound on the work stepped together.  While
 * requests run, the oldest queued request is admitted only if the running
 * requests' K * Np (nodal values per field) plus its own stay within
 * max_nodes; otherwise it, and every request behind it, waits (first come,
 * first served: a large request is not passed by later small ones).  A
 * request is always admitted when none runs, so one larger than the limit
 * runs alone.  This caps the processor sharing that stretches long solves;
 * 0 (the default) means no limit beyond the memory budget.  Takes effect at
 * the worker's next admission pass.  Errors: DG_ERR_ARG (NULL,
 * max_nodes < 0).                                                          */
dg_status dg_server_set_work_limit(dg_server* server, int64_t max_nodes);

/* dg_server_submit: queue the solve of operator `op` (DG_FP32, host-only is
 * enough; it must stay alive until the request is released) from t = 0 to
 * T with the optional point source `src` (copied; NULL: none), starting
 * from the host fields q0 (3 * K * Np floats in the layout of
 * dg_batch_set_fields with stride K * Np; NULL: zero fields; read at
 * admission, so it must stay valid until then) and writing the fields at T
 * to `out` (same layout; NULL: discard), host memory that must stay valid
 * until the request is done.  Returns at once with the request id.
 * Errors: DG_ERR_ARG (NULL, not DG_FP32, T not positive, step count out
 * of range, server stopping), DG_ERR_OOM.                                  */
dg_status dg_server_submit(dg_server* server, const dg_op* op, double T,
                           const dg_point_source* src, const void* q0, void* out,
                           int64_t* request_id);

/* Waits until the request is done or failed (timeout_s < 0: no limit) and
 * fills info.  Errors: DG_ERR_ARG (unknown id), DG_ERR_TIMEOUT.            */
dg_status dg_server_wait(dg_server* server, int64_t request_id, double timeout_s,
                         dg_request_info* info);

/* The request's current state and times, without waiting.                 */
dg_status dg_server_info(dg_server* server, int64_t request_id, dg_request_info* info);

/* dg_server_cancel: a queued request is dropped at the worker's next
 * admission pass, a running one leaves the batch at the next chunk boundary
 * without its result (`out` is not written); either then reports
 * DG_REQUEST_CANCELLED.  A request whose result is already on its way to
 * host memory completes normally.
 * Errors: DG_ERR_ARG (unknown id, or the request already finished).       */
dg_status dg_server_cancel(dg_server* server, int64_t request_id);

/* Forget a finished request (its id becomes unknown).                     */
dg_status dg_server_release(dg_server* server, int64_t request_id);

/* Requests completed and failed, LSRK steps taken by the batch, and its
 * kernel launches.  NULL outputs are skipped.                              */
dg_status dg_server_stats(dg_server* server, int64_t* completed, int64_t* failed, int64_t* steps,
                          int64_t* launches);

/* ---------------------------------------------------------- checkpoints ---
 * The state of a solve between steps is its three fields, its time and its
 * step count (the LSRK residual needs no saving: the first stage of a step
 * overwrites it).  dg_checkpoint_save writes q's first K * Np values of each
 * field (field f at f * q_stride) to the file `path`, with t and step, in
 * the operator's precision.  The header records the operator (N, K,
 * precision, medium) and a hash of its node coordinates and permittivities.
 * The file is written under a temporary name and then renamed.
 * dg_checkpoint_load refuses a file written for another operator or mesh,
 * or whose field data no longer match their hash, and otherwise fills q (the
 * entries beyond K * Np are left alone) and returns t and step.  Resuming
 * from a checkpoint gives bit for bit what running on would have given.
 * q is device memory of the operator's device, or host memory with
 * DG_CKPT_HOST.  Both calls are synchronous.
 * Errors: DG_ERR_ARG (NULL, unknown flags, q_stride < K * Np, a file for
 * another operator or mesh, damaged data), DG_ERR_NO_DEVICE (device fields
 * with a host-only operator), DG_ERR_IO (open, read, write, rename),
 * DG_ERR_OOM, DG_ERR_CUDA.                                                 */
#define DG_CKPT_HOST 1 /* the fields are in host memory */

dg_status dg_checkpoint_save(const dg_op* op, const void* q, int64_t q_stride, int32_t flags,
                             double t, int64_t step, const char* path);
dg_status dg_checkpoint_load(const dg_op* op, const char* path, void* q, int64_t q_stride,
                             int32_t flags, double* t, int64_t* step);

/* ----------------------------------------------------------- partitions ---
 * A mesh partition of one operator into P parts, each with its own element
 * tables and field buffers, stepped with one halo exchange per LSRK stage:
 * the multi-GPU decomposition of Section "Further Tuning Opportunities"
 * (only the face traces that the flux needs cross a cut), emulated on one
 * device.  Parts are recursive coordinate bisections of the element
 * centroids (sizes within one element of K / P); each part keeps its
 * elements in increasing global order.  Every element whose face meets a
 * cut gets, in each part across that face, a ghost slot whose face nodes
 * receive its traces.  A stage is: pack (one kernel: every part's outgoing
 * traces into a send buffer, one contiguous message per (sender, receiver)
 * pair), the transfer (between GPUs one send / receive per pair; on one
 * device a single copy of all messages into the receive buffer), unpack
 * (one kernel into the ghost slots), then one stage launch per part, each
 * on a stream of the partition's own (the parts' launches of a stage are
 * independent), which `stream` waits for.  The result equals, bit for bit,
 * the unpartitioned operator's.
 *
 * dg_partition_create: partitions `op` (not owned; it must outlive the
 * partition) into P parts, 1 <= P <= min(K, 64).  With a device operator it
 * builds the parts' device tables and buffers on op's device; with a
 * host-only operator only the plan (parts, ghosts, exchange lists).
 * dg_partition_info: part p's element count, ghost count, the number of
 * parts it receives from and sends to, and the node values (per field) it
 * receives and sends per exchange.
 * dg_partition_elements / dg_partition_ghosts: global element ids of part
 * p's elements (K_p) and of its ghost slots (G_p), host int64 arrays.
 * dg_partition_conn: part p's face connection codes (3 K_p, int32): -1 on a
 * boundary face, otherwise e * 8 + f * 2 + rev with e the neighbour's slot in
 * part p (an element index below K_p, or ghost slot g at index Kpad_p + g).
 * dg_partition_exchange_plan: what part p sends and receives per exchange,
 * as node offsets into one field of its local layout (element slot * Np +
 * node): send_peer[i] gets send_count[i] values at the next send_count[i]
 * entries of send_off, in that order; recv_peer[i] sends recv_count[i]
 * values, stored at the next recv_count[i] entries of recv_off.  The lists
 * of a sender and its receiver match entry for entry.  Any pointer may be
 * NULL; arrays are sized by dg_partition_info.
 * dg_partition_set_fields / dg_partition_get_fields: scatter the global
 * fields q (device, the operator's precision, field f at f * q_stride) into
 * the parts, or gather them back.  Asynchronous on `stream`.
 * dg_partition_exchange: one halo exchange on the parts' current fields.
 * dg_partition_step: nsteps LSRK(5,4) steps of size dt of every part.
 * dg_partition_sync_check: dg_sync_check of every part.
 * Errors: DG_ERR_ARG (NULL, P out of range, p out of range, q_stride <
 * K * Np, nsteps < 0, dt not finite), DG_ERR_NO_DEVICE (a device call on a
 * plan-only partition), DG_ERR_OOM, DG_ERR_CUDA, DG_ERR_TIMEOUT.          */
typedef struct dg_partition dg_partition;

dg_status dg_partition_create(const dg_op* op, int32_t P, dg_partition** out);
void dg_partition_destroy(dg_partition* part);
dg_status dg_partition_info(const dg_partition* part, int32_t p, int64_t* K_p, int64_t* G_p,
                            int32_t* n_recv_peers, int32_t* n_send_peers, int64_t* n_recv,
                            int64_t* n_send);
dg_status dg_partition_elements(const dg_partition* part, int32_t p, int64_t* gid);
dg_status dg_partition_ghosts(const dg_partition* part, int32_t p, int64_t* gid);
dg_status dg_partition_conn(const dg_partition* part, int32_t p, int32_t* conn);
dg_status dg_partition_exchange_plan(const dg_partition* part, int32_t p, int32_t* send_peer,
                                     int64_t* send_count, int32_t* send_off, int32_t* recv_peer,
                                     int64_t* recv_count, int32_t* recv_off);
dg_status dg_partition_set_fields(dg_partition* part, const void* q, int64_t q_stride,
                                  void* stream);
dg_status dg_partition_get_fields(dg_partition* part, void* q, int64_t q_stride, void* stream);
dg_status dg_partition_exchange(dg_partition* part, void* stream);
dg_status dg_partition_step(dg_partition* part, double dt, int32_t nsteps, void* stream);
dg_status dg_partition_sync_check(dg_partition* part, void* stream);

/* dg_check_finite: synchronises `stream`, then scans the first K*Np values
 * of each field of d_q for NaN/Inf.  Returns DG_ERR_NONFINITE if any is
 * found (blow-up detection), DG_OK otherwise.                              */
dg_status dg_check_finite(const dg_op* op, const void* d_q, void* stream);

/* dg_sync_check: synchronises `stream` and reports any pending CUDA error
 * (DG_ERR_CUDA with its message in dg_last_error()), then reads and clears
 * the operator's kernel status word: DG_ERR_TIMEOUT if a stage kernel gave
 * up waiting for its own shared-memory copies (bounded waits, ~2 s), and
 * DG_ERR_INDEX if a checked build's kernel found a face connection code or
 * a block-table entry out of range (the access is skipped, the result is
 * not valid).  The checked build is the same library compiled with
 * DGW_DEVICE_CHECKS into libdgwave_checked.so; the Python binding loads it
 * when DGWAVE_CHECKED=1.                                                    */
dg_status dg_sync_check(const dg_op* op, void* stream);

/* dg_test_fail_alloc: allocation failures made on the host.  The n-th
 * device allocation the library makes from now on (n >= 1) fails with
 * DG_ERR_OOM without allocating; n = 0 switches this off.  Each set-up call
 * must then return DG_ERR_OOM, free what it had allocated and leave the
 * library usable.  dg_test_fail_alloc_pending: allocations left before the
 * planted failure (0: it happened, or none is planted).  Process-wide; for
 * tests only.  Errors: DG_ERR_ARG (n < 0).                                 */
dg_status dg_test_fail_alloc(int32_t n);
int32_t dg_test_fail_alloc_pending(void);

/* dg_test_wait_timeout: the timeout path, exercised without any fault.
 * Launches one right-hand-side pass of a tensor-core operator whose memory
 * warp first waits, bounded by 0.1 s, for a device flag that nothing sets.
 * The wait runs out, the CTAs set the operator's status word, stop their
 * other warps through their shared abort flag, free their tensor memory and
 * return, having read and written no field.  Synchronises `stream`.  A
 * following dg_sync_check returns DG_ERR_TIMEOUT (and clears the word); the
 * operator stays usable.  The paper has no counterpart: this tests the
 * failure detection of the bounded waits.
 * Errors: DG_ERR_ARG (NULL, not a tensor-core operator), DG_ERR_NO_DEVICE,
 * DG_ERR_CUDA.                                                             */
dg_status dg_test_wait_timeout(const dg_op* op, void* stream);

/* Number of kernel launches enqueued by this operator since setup (one per
 * dg_rhs, five per step, one per dg_check_finite, and 2 (reps + 1) per
 * dg_operator_tune that measured).                                         */
int64_t dg_launch_count(const dg_op* op);

/* Thread-local message of the last failing call on this thread ("" if
 * none).  The pointer stays valid until the next call on the thread.      */
const char* dg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* DGWAVE_H */
