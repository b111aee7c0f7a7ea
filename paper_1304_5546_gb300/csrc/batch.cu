// Batched solves: many independent problems of mixed orders stepped by one
// persistent launch per LSRK stage (dg_batch_* of the C ABI).
//
// Each order N has a pool: element capacity fixed at creation, field buffers
// (two for the stage ping-pong, one residual), geometry records of
// kGeoMedia values and face codes.  A problem occupies a range of its
// order's pool (first fit, 4-element aligned so that every block's chunks
// start on 16 bytes); its face codes point at pool element numbers, so the
// kernels never look outside the problem.  The problem's own time step is
// folded into its records' row scales (sH = dt, sE = dt / eps_k) and the
// launch runs with dt = 1, so problems with different steps share a launch.
//
// A launch walks a block table per order (E-element blocks that never span
// two problems; the last block of a problem may be short).  Tables, block
// counts and the split of the launch's CTAs among the orders live in device
// memory and are rewritten when problems join or leave, so the two captured
// one-step graphs (starting from either ping-pong buffer) stay valid for the
// batch's lifetime.
//
// The CTA split: order N's blocks take ceil(nblk_N / c_N) iterations of
// tau_N seconds on each of its c_N CTAs; the planner gives every order with
// blocks one CTA and then hands out the rest one at a time to the order with
// the largest ceil(nblk_N / c_N) tau_N.  tau_N starts from a table measured
// on a GB300 and is replaced by the batch's own measurements by
// dg_batch_tune, which also tries moving single CTAs between orders and
// keeps what measures faster.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "internal.h"
#include "launch.h"
#include "staging.h"

using dgw::fail;

namespace {

constexpr int kOrders = DG_N_MAX;
constexpr int kPadElems = 8;  // pool tail read by the last block's 16-byte rounding

dg_status cuda_fail(cudaError_t err, const char* where) {
  return fail(err == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA, "%s: %s (%s)", where,
              cudaGetErrorName(err), cudaGetErrorString(err));
}

struct Pool {
  int N = 0, Np = 0, E = 0;
  bool alt = false;  // concurrent mode: the order's alternative block size (E follows)
  int64_t cap = 0;      // element capacity
  int64_t fstride = 0;  // values between fields
  float* q[2] = {nullptr, nullptr};
  float* res = nullptr;
  float* geo = nullptr;
  int32_t* conn = nullptr;
  float* lam = nullptr;
  void* tcop = nullptr;
  int2* blocks = nullptr;
  int64_t max_blocks = 0;
  std::map<int64_t, int64_t> free_ranges;  // start -> length
  size_t smem = 0;
};

struct Problem {
  bool live = false;
  bool source = false;
  int N = 0;
  int64_t K = 0, off = 0, len = 0;
  double dt = 0.0;
};

}  // namespace

struct dg_batch {
  int device = 0;
  int num_sms = 0;
  int flags = 0;
  Pool pools[kOrders];
  int* d_meta = nullptr;  // [0, 7): block counts per order, [8, 16): CTA split cta0,
                          // [16]: steps completed (stage time of the point sources)
  int* d_status = nullptr;
  // point sources, indexed by problem slot
  int64_t max_slots = 0;
  float* d_src_w = nullptr;      // [slot][kSrcStride]
  double* d_src_meta = nullptr;  // [slot][4]: dt, t0, pi f, amplitude
  int* d_src_step = nullptr;     // [slot]: steps enqueued when the problem joined
  int64_t steps = 0;             // steps enqueued so far
  std::vector<Problem> probs;
  int cur = 0;  // ping-pong buffer holding the current fields
  bool dirty = true;
  int64_t nblk[kOrders] = {};
  int cta[kOrders] = {};
  double cost[kOrders] = {};  // seconds (or model units) per block iteration of one CTA
  bool measured = false;
  size_t smem = 0;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  cudaStream_t capture = nullptr;
  // launch mode: concurrent (each order's stage a kernel of its own, the
  // orders side by side on streams of their own, joined once per step) or,
  // with DG_BATCH_SPLIT or when dg_batch_tune measures it faster, split (one
  // launch per stage, its CTAs split among the orders)
  bool concurrent = true;
  float tuned_split_ms = 0.f, tuned_concurrent_ms = 0.f;  // dg_batch_tune's last timings
  float tuned_order_ms[kOrders][2] = {};  // per order: default, alternative block size
  cudaStream_t ostream[kOrders] = {};
  cudaEvent_t fork_ev = nullptr;
  cudaEvent_t join_ev[kOrders] = {};
  double lsrk_a[5], lsrk_b[5], lsrk_c[5];
  int64_t launches = 0;
  dgw::Staging staging;
  // online adaptation of the CTA split: every launch writes each CTA's start
  // and end time to d_clock; every kAdaptSteps steps a snapshot goes to
  // pinned host memory, and once it has arrived the per-order costs are
  // updated from the observed finish times and the split re-planned
  unsigned long long* d_clock = nullptr;
  unsigned long long* h_clock = nullptr;
  cudaEvent_t clock_ev = nullptr;
  bool clock_pending = false;
  int clock_cta[kOrders] = {};
  int64_t clock_nblk[kOrders] = {};
  int64_t steps_since_snapshot = 0;
  int64_t replans = 0;
};

namespace {

// ----------------------------------------------------------- planning
// CTAs per order for block counts nblk and per-block costs cost: every
// order with blocks gets one, the rest go one at a time to the order whose
// ceil(nblk / c) * cost is largest (an order never gets more CTAs than
// blocks).  Returns false if there are more orders with blocks than CTAs.
bool plan_ctas(const int64_t* nblk, const double* cost, int num_ctas, int* cta) {
  int used = 0;
  for (int g = 0; g < kOrders; ++g) {
    cta[g] = nblk[g] > 0 ? 1 : 0;
    used += cta[g];
  }
  if (used > num_ctas) return false;
  auto finish = [&](int g, int c) {
    return static_cast<double>((nblk[g] + c - 1) / c) * cost[g];
  };
  for (; used < num_ctas; ++used) {
    int best = -1;
    double worst = -1.0;
    for (int g = 0; g < kOrders; ++g) {
      if (cta[g] == 0 || cta[g] >= nblk[g]) continue;
      const double f = finish(g, cta[g]);
      if (f > worst) {
        worst = f;
        best = g;
      }
    }
    if (best < 0) break;
    ++cta[best];
  }
  return true;
}

// cost of one block iteration per CTA before dg_batch_tune measures it:
// seconds, the medians of four dg_batch_tune runs on a GB300 (152 CTAs, a
// batch of all seven orders with about 3000 blocks each, of 80 elements at
// N <= 3 and 40 above; costs observed in the mixed launch).  The bytes a
// block moves predict these badly: a block has a fixed cost in hand-offs
// and instruction issue.
double model_cost(int N) {
  static const double us[8] = {0.0, 1.55, 1.98, 2.22, 2.18, 2.68, 2.92, 2.93};
  return 1e-6 * us[N];
}

void free_pool(Pool& p) {
  void* ptrs[] = {p.q[0], p.q[1], p.res, p.geo, p.conn, p.lam, p.tcop, p.blocks};
  for (void* x : ptrs)
    if (x) cudaFree(x);
  p.q[0] = p.q[1] = p.res = p.geo = p.lam = nullptr;
  p.conn = nullptr;
  p.tcop = nullptr;
  p.blocks = nullptr;
}

void destroy_batch(dg_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  cudaDeviceSynchronize();
  for (cudaGraphExec_t& g : b->graph)
    if (g) cudaGraphExecDestroy(g);
  if (b->capture) cudaStreamDestroy(b->capture);
  for (int g = 0; g < kOrders; ++g) {
    if (b->ostream[g]) cudaStreamDestroy(b->ostream[g]);
    if (b->join_ev[g]) cudaEventDestroy(b->join_ev[g]);
  }
  if (b->fork_ev) cudaEventDestroy(b->fork_ev);
  for (Pool& p : b->pools) free_pool(p);
  if (b->d_meta) cudaFree(b->d_meta);
  if (b->d_status) cudaFree(b->d_status);
  if (b->d_clock) cudaFree(b->d_clock);
  if (b->h_clock) cudaFreeHost(b->h_clock);
  if (b->clock_ev) cudaEventDestroy(b->clock_ev);
  if (b->d_src_w) cudaFree(b->d_src_w);
  if (b->d_src_meta) cudaFree(b->d_src_meta);
  if (b->d_src_step) cudaFree(b->d_src_step);
  b->staging.release();
  delete b;
}

dg_status alloc_pool(dg_batch* b, int N, int64_t cap) {
  Pool& p = b->pools[N - 1];
  p.N = N;
  p.cap = cap;
  const dgw::RefElement ref = dgw::build_reference(N);
  p.Np = ref.Np;
  p.E = dgw::batch_tc_block_elems(N);
  p.smem = dgw::batch_tc_smem_bytes(N);
  const int64_t rows = cap + kPadElems;
  p.fstride = (rows * p.Np + 63) / 64 * 64;
  if (p.fstride >= (int64_t(1) << 31) || rows * 8 >= (int64_t(1) << 31))
    return fail(DG_ERR_ARG, "dg_batch_create: capacity %lld at N = %d exceeds 32-bit offsets",
                static_cast<long long>(cap), N);
  p.max_blocks = cap / 4 + 1;  // problems are >= 1 element at 4-element alignment
  const size_t fb = 3 * static_cast<size_t>(p.fstride) * sizeof(float);
  struct A {
    void** dst;
    size_t bytes;
  } allocs[] = {
      {reinterpret_cast<void**>(&p.q[0]), fb},
      {reinterpret_cast<void**>(&p.q[1]), fb},
      {reinterpret_cast<void**>(&p.res), fb},
      {reinterpret_cast<void**>(&p.geo), static_cast<size_t>(rows) * dgw::kGeoMedia * 4},
      {reinterpret_cast<void**>(&p.conn), static_cast<size_t>(rows) * 3 * 4},
      {reinterpret_cast<void**>(&p.blocks), static_cast<size_t>(p.max_blocks) * sizeof(int2)},
  };
  for (const A& a : allocs) {
    cudaError_t err = dgw::dev_malloc(a.dst, a.bytes);
    if (err != cudaSuccess) return cuda_fail(err, "dg_batch_create: cudaMalloc");
    err = cudaMemset(*a.dst, 0, a.bytes);
    if (err != cudaSuccess) return cuda_fail(err, "dg_batch_create: cudaMemset");
  }
  std::vector<float> lam(2 * static_cast<size_t>(p.Np));
  for (int n = 0; n < p.Np; ++n) {
    lam[n] = static_cast<float>(0.5 * (1.0 + ref.r[n]));
    lam[p.Np + n] = static_cast<float>(0.5 * (1.0 + ref.s[n]));
  }
  const std::vector<unsigned char> tiles = dgw::tc_operator_tiles(ref, dgw::kTcTf32x3);
  cudaError_t err = dgw::dev_malloc(reinterpret_cast<void**>(&p.lam), lam.size() * 4);
  if (err == cudaSuccess) err = cudaMemcpy(p.lam, lam.data(), lam.size() * 4, cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = dgw::dev_malloc(&p.tcop, tiles.size());
  if (err == cudaSuccess) err = cudaMemcpy(p.tcop, tiles.data(), tiles.size(), cudaMemcpyHostToDevice);
  if (err != cudaSuccess) return cuda_fail(err, "dg_batch_create: operator upload");
  p.free_ranges[0] = cap;
  return DG_OK;
}

// first-fit range of `len` elements; -1 if none
int64_t take_range(Pool& p, int64_t len) {
  for (auto it = p.free_ranges.begin(); it != p.free_ranges.end(); ++it) {
    if (it->second >= len) {
      const int64_t start = it->first, rest = it->second - len;
      p.free_ranges.erase(it);
      if (rest > 0) p.free_ranges[start + len] = rest;
      return start;
    }
  }
  return -1;
}

void give_range(Pool& p, int64_t start, int64_t len) {
  auto next = p.free_ranges.lower_bound(start);
  if (next != p.free_ranges.end() && next->first == start + len) {
    len += next->second;
    next = p.free_ranges.erase(next);
  }
  if (next != p.free_ranges.begin()) {
    auto prev = std::prev(next);
    if (prev->first + prev->second == start) {
      prev->second += len;
      return;
    }
  }
  p.free_ranges[start] = len;
}

dgw::BatchArgs batch_args(const dg_batch* b, int src, int stage) {
  dgw::BatchArgs a;
  for (int g = 0; g < kOrders; ++g) {
    const Pool& p = b->pools[g];
    dgw::StageArgs<float>& s = a.g[g];
    if (p.cap == 0) continue;
    s.K = p.cap;
    s.fstride = p.fstride;
    s.qin = p.q[src];
    s.qout = p.q[src ^ 1];
    s.res = p.res;
    s.geo = p.geo;
    s.conn = p.conn;
    s.lam = p.lam;
    s.tc_op = p.tcop;
    s.status = b->d_status;
    s.blocks = p.blocks;
    s.nblocks = b->d_meta + g;
    s.a = static_cast<float>(b->lsrk_a[stage]);
    s.b = static_cast<float>(b->lsrk_b[stage]);
    s.dt = 1.0f;  // each problem's step is in its row scales
    s.src_w = b->d_src_w;
    s.src_meta = b->d_src_meta;
    s.src_step = b->d_src_step;
    s.step_ctr = b->d_meta + 16;
    s.c_stage = b->lsrk_c[stage];
  }
  a.cta0 = b->d_meta + 8;
  return a;
}

// end of a step: the device step counter that the source times read
__global__ void batch_tick_kernel(int* ctr) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *ctr += 1;
}

cudaError_t launch_tick(dg_batch* b, cudaStream_t s) {
  batch_tick_kernel<<<1, 32, 0, s>>>(b->d_meta + 16);
  cudaError_t err = cudaGetLastError();
  if (err == cudaSuccess) ++b->launches;
  return err;
}

cudaError_t launch_stage(dg_batch* b, int src, int stage, cudaStream_t s) {
  dgw::BatchArgs a = batch_args(b, src, stage);
  a.cta_clock = b->d_clock;
  cudaError_t err = stage == 0 ? dgw::launch_batch_tc<dgw::kModeFirstStage>(a, b->num_sms, b->smem, s)
                               : dgw::launch_batch_tc<dgw::kModeStage>(a, b->num_sms, b->smem, s);
  if (err == cudaSuccess) ++b->launches;
  return err;
}

// Order g's kernel of the concurrent mode for stage `stage`, reading field
// buffer src; grid 0 only configures the kernel.
cudaError_t launch_order_stage(dg_batch* b, int g, int src, int stage, int grid, cudaStream_t s) {
  const dgw::BatchArgs a = batch_args(b, src, stage);
  const dgw::StageArgs<float>& ga = a.g[g];
  const bool first = stage == 0;
  cudaError_t err = cudaErrorInvalidValue;
  const bool alt = b->pools[g].alt;
#define DG_ORDER_CASE(NN_)                                                                 \
  case NN_:                                                                                \
    if (alt)                                                                               \
      err = first ? dgw::launch_batch_order<NN_, dgw::kModeFirstStage, true>(ga, grid, s)  \
                  : dgw::launch_batch_order<NN_, dgw::kModeStage, true>(ga, grid, s);      \
    else                                                                                   \
      err = first ? dgw::launch_batch_order<NN_, dgw::kModeFirstStage>(ga, grid, s)        \
                  : dgw::launch_batch_order<NN_, dgw::kModeStage>(ga, grid, s);            \
    break;
  switch (g + 1) {
    DG_ORDER_CASE(1)
    DG_ORDER_CASE(2)
    DG_ORDER_CASE(3)
    DG_ORDER_CASE(4)
    DG_ORDER_CASE(5)
    DG_ORDER_CASE(6)
    DG_ORDER_CASE(7)
    default:
      break;
  }
#undef DG_ORDER_CASE
  if (err == cudaSuccess && grid > 0) ++b->launches;
  return err;
}

// `reps` launches of stage `stage` (reading buffer src) of every order with
// a pool, each order on its own stream, forked from and joined back into s.
cudaError_t launch_concurrent(dg_batch* b, int src, int stage, int reps, bool whole_step,
                              cudaStream_t s) {
  cudaError_t err = cudaEventRecord(b->fork_ev, s);
  for (int g = 0; g < kOrders && err == cudaSuccess; ++g) {
    if (b->pools[g].cap == 0) continue;
    err = cudaStreamWaitEvent(b->ostream[g], b->fork_ev, 0);
    if (whole_step) {
      for (int i = 0; i < 5 && err == cudaSuccess; ++i)
        err = launch_order_stage(b, g, src ^ (i & 1), i, b->num_sms, b->ostream[g]);
    } else {
      for (int r = 0; r < reps && err == cudaSuccess; ++r)
        err = launch_order_stage(b, g, src, stage, b->num_sms, b->ostream[g]);
    }
    if (err == cudaSuccess) err = cudaEventRecord(b->join_ev[g], b->ostream[g]);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(s, b->join_ev[g], 0);
  }
  return err;
}

// One LSRK step of every problem, from field buffer src, in the batch's
// launch mode, followed by the step-counter tick.
cudaError_t launch_step(dg_batch* b, int src, cudaStream_t s) {
  cudaError_t err = cudaSuccess;
  if (b->concurrent) {
    err = launch_concurrent(b, src, 0, 1, true, s);
  } else {
    for (int i = 0; i < 5 && err == cudaSuccess; ++i) err = launch_stage(b, src ^ (i & 1), i, s);
  }
  if (err == cudaSuccess) err = launch_tick(b, s);
  return err;
}

// block tables, counts and CTA split -> device (asynchronously on s)
dg_status upload_tables(dg_batch* b, cudaStream_t s) {
  std::vector<int2> tab[kOrders];
  for (const Problem& pr : b->probs) {
    if (!pr.live) continue;
    const int E = b->pools[pr.N - 1].E;
    for (int64_t k = 0; k < pr.K; k += E)
      tab[pr.N - 1].push_back(make_int2(static_cast<int>(pr.off + k),
                                        static_cast<int>(std::min<int64_t>(E, pr.K - k))));
  }
  for (int g = 0; g < kOrders; ++g) {
    // longest problems first inside an order is not needed: blocks are
    // handed out strided over the CTAs, so neighbours in the table spread
    std::sort(tab[g].begin(), tab[g].end(), [](const int2& x, const int2& y) { return x.x < y.x; });
    b->nblk[g] = static_cast<int64_t>(tab[g].size());
  }
  if (!plan_ctas(b->nblk, b->cost, b->num_sms, b->cta))
    return fail(DG_ERR_ARG, "dg_batch_step: more orders with problems than CTAs");
  size_t total = 0;
  for (int g = 0; g < kOrders; ++g) total += tab[g].size();
  const size_t bytes = 16 * sizeof(int) + total * sizeof(int2);
  size_t idx = 0;
  unsigned char* h = static_cast<unsigned char*>(b->staging.get(bytes, &idx));
  if (!h) return fail(DG_ERR_OOM, "dg_batch_step: pinned staging buffer");
  int* meta = reinterpret_cast<int*>(h);
  int2* blk = reinterpret_cast<int2*>(h + 16 * sizeof(int));
  meta[7] = 0;
  meta[8] = 0;
  for (int g = 0; g < kOrders; ++g) {
    meta[g] = static_cast<int>(b->nblk[g]);
    meta[9 + g] = meta[8 + g] + b->cta[g];
  }
  cudaError_t err = cudaMemcpyAsync(b->d_meta, meta, 16 * sizeof(int), cudaMemcpyHostToDevice, s);
  size_t o = 0;
  for (int g = 0; g < kOrders && err == cudaSuccess; ++g) {
    if (tab[g].empty()) continue;
    std::memcpy(blk + o, tab[g].data(), tab[g].size() * sizeof(int2));
    err = cudaMemcpyAsync(b->pools[g].blocks, blk + o, tab[g].size() * sizeof(int2),
                          cudaMemcpyHostToDevice, s);
    o += tab[g].size();
  }
  if (err == cudaSuccess) err = b->staging.mark(idx, s);
  if (err != cudaSuccess) return cuda_fail(err, "dg_batch_step: table upload");
  b->dirty = false;
  return DG_OK;
}

dg_status capture_graphs(dg_batch* b) {
  if (!b->capture) {
    cudaError_t err = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
    if (err != cudaSuccess) return cuda_fail(err, "dg_batch_step: stream");
  }
  // set the kernels' shared-memory attribute outside the capture (a launch
  // of zero CTAs only configures)
  const dgw::BatchArgs a0 = batch_args(b, 0, 0);
  cudaError_t cerr = dgw::launch_batch_tc<dgw::kModeFirstStage>(a0, 0, 0, b->capture);
  if (cerr == cudaSuccess) cerr = dgw::launch_batch_tc<dgw::kModeStage>(a0, 0, 0, b->capture);
  for (int g = 0; g < kOrders && cerr == cudaSuccess; ++g) {
    if (b->pools[g].cap == 0) continue;
    cerr = launch_order_stage(b, g, 0, 0, 0, b->capture);
    if (cerr == cudaSuccess) cerr = launch_order_stage(b, g, 0, 1, 0, b->capture);
  }
  if (cerr != cudaSuccess) return cuda_fail(cerr, "dg_batch_step: kernel attributes");
  for (int src = 0; src < 2; ++src) {
    cudaGraph_t graph = nullptr;
    cudaError_t err = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
    if (err != cudaSuccess) return cuda_fail(err, "dg_batch_step: begin capture");
    const int64_t before = b->launches;
    const cudaError_t lerr = launch_step(b, src, b->capture);
    b->launches = before;  // captured, not run
    err = cudaStreamEndCapture(b->capture, &graph);
    if (lerr != cudaSuccess) err = lerr;
    if (err == cudaSuccess) err = cudaGraphInstantiate(&b->graph[src], graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (err != cudaSuccess) return cuda_fail(err, "dg_batch_step: graph capture");
  }
  return DG_OK;
}

// Order g's block size: the default, or (alt) its alternative.  The block
// tables are rebuilt before the next launch, and the step graphs, which hold
// the order's kernel, are captured again.
void set_order_alt(dg_batch* b, int g, bool alt) {
  Pool& p = b->pools[g];
  if (p.alt == alt) return;
  p.alt = alt;
  p.E = dgw::batch_tc_block_elems(g + 1, alt);
  b->dirty = true;
  for (cudaGraphExec_t& ge : b->graph) {
    if (ge) cudaGraphExecDestroy(ge);
    ge = nullptr;
  }
}

// kernel launches of one step in the batch's mode (stages and the tick)
int64_t launches_per_step(const dg_batch* b) {
  if (!b->concurrent) return 6;
  int64_t n = 1;
  for (int g = 0; g < kOrders; ++g) n += b->pools[g].cap > 0 ? 5 : 0;
  return n;
}

dg_status check_batch(dg_batch* b, const char* where) {
  if (!b) return fail(DG_ERR_ARG, "%s: NULL batch", where);
  cudaError_t err = cudaSetDevice(b->device);
  if (err != cudaSuccess) return cuda_fail(err, where);
  return DG_OK;
}

dg_status check_slot(const dg_batch* b, int32_t slot, const char* where) {
  if (slot < 0 || slot >= static_cast<int32_t>(b->probs.size()) || !b->probs[slot].live)
    return fail(DG_ERR_ARG, "%s: no problem in slot %d", where, slot);
  return DG_OK;
}

}  // namespace

// ============================================================ C ABI
extern "C" dg_status dg_batch_plan_ctas(const int64_t* nblocks, const double* cost,
                                        int32_t num_ctas, int32_t* cta) {
  dgw::clear_error();
  if (!nblocks || !cost || !cta || num_ctas < 1)
    return fail(DG_ERR_ARG, "dg_batch_plan_ctas: bad argument");
  int c[kOrders];
  if (!plan_ctas(nblocks, cost, num_ctas, c))
    return fail(DG_ERR_ARG, "dg_batch_plan_ctas: more orders with blocks than CTAs");
  for (int g = 0; g < kOrders; ++g) cta[g] = c[g];
  return DG_OK;
}

extern "C" dg_status dg_batch_create(const int64_t* capacity, int32_t flags, dg_batch** out) {
  dgw::clear_error();
  if (!capacity || !out) return fail(DG_ERR_ARG, "dg_batch_create: NULL argument");
  if (flags & ~(DG_BATCH_NO_GRAPH | DG_BATCH_NO_ADAPT | DG_BATCH_SPLIT))
    return fail(DG_ERR_ARG, "dg_batch_create: unknown flags 0x%x", flags);
  bool any = false;
  for (int g = 0; g < kOrders; ++g) {
    if (capacity[g] < 0 || capacity[g] >= (int64_t(1) << 27))
      return fail(DG_ERR_ARG, "dg_batch_create: capacity[%d] = %lld out of range", g,
                  static_cast<long long>(capacity[g]));
    any = any || capacity[g] > 0;
  }
  if (!any) return fail(DG_ERR_ARG, "dg_batch_create: every capacity is zero");
  dg_batch* b = new (std::nothrow) dg_batch;
  if (!b) return fail(DG_ERR_OOM, "dg_batch_create: out of host memory");
  b->flags = flags;
  b->concurrent = !(flags & DG_BATCH_SPLIT);
  dgw::lsrk_coefficients(b->lsrk_a, b->lsrk_b, b->lsrk_c);
  cudaError_t err = cudaGetDevice(&b->device);
  if (err == cudaSuccess)
    err = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
  if (err != cudaSuccess) {
    delete b;
    return cuda_fail(err, "dg_batch_create: device");
  }
  for (int g = 0; g < kOrders; ++g) {
    if (capacity[g] == 0) continue;
    const dg_status st = alloc_pool(b, g + 1, capacity[g]);
    if (st != DG_OK) {
      destroy_batch(b);
      return st;
    }
    b->smem = std::max(b->smem, b->pools[g].smem);
    b->cost[g] = model_cost(g + 1);
  }
  for (int g = 0; g < kOrders; ++g) b->max_slots += capacity[g] > 0 ? capacity[g] / 4 + 1 : 0;
  err = dgw::dev_malloc(reinterpret_cast<void**>(&b->d_meta), 17 * sizeof(int));
  if (err == cudaSuccess) err = cudaMemset(b->d_meta, 0, 17 * sizeof(int));
  if (err == cudaSuccess)
    err = dgw::dev_malloc(reinterpret_cast<void**>(&b->d_src_w), b->max_slots * dgw::kSrcStride * 4);
  if (err == cudaSuccess)
    err = dgw::dev_malloc(reinterpret_cast<void**>(&b->d_src_meta), b->max_slots * 4 * sizeof(double));
  if (err == cudaSuccess)
    err = dgw::dev_malloc(reinterpret_cast<void**>(&b->d_src_step), b->max_slots * sizeof(int));
  const size_t clock_bytes = 2 * static_cast<size_t>(b->num_sms) * sizeof(unsigned long long);
  if (err == cudaSuccess) err = dgw::dev_malloc(reinterpret_cast<void**>(&b->d_clock), clock_bytes);
  if (err == cudaSuccess) err = cudaMemset(b->d_clock, 0, clock_bytes);
  if (err == cudaSuccess) err = cudaMallocHost(reinterpret_cast<void**>(&b->h_clock), clock_bytes);
  if (err == cudaSuccess) err = cudaEventCreateWithFlags(&b->clock_ev, cudaEventDisableTiming);
  if (err == cudaSuccess) err = dgw::dev_malloc(reinterpret_cast<void**>(&b->d_status), sizeof(int));
  if (err == cudaSuccess) err = cudaMemset(b->d_status, 0, sizeof(int));
  if (err == cudaSuccess) err = cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming);
  for (int g = 0; g < kOrders && err == cudaSuccess; ++g) {
    if (capacity[g] == 0) continue;
    err = cudaStreamCreateWithFlags(&b->ostream[g], cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&b->join_ev[g], cudaEventDisableTiming);
  }
  if (err != cudaSuccess) {
    destroy_batch(b);
    return cuda_fail(err, "dg_batch_create: cudaMalloc");
  }
  *out = b;
  return DG_OK;
}

extern "C" void dg_batch_destroy(dg_batch* b) { destroy_batch(b); }

extern "C" dg_status dg_batch_add(dg_batch* b, const dg_op* op, double dt,
                                  const dg_point_source* src, void* stream, int32_t* slot) {
  dgw::clear_error();
  dg_status st = check_batch(b, "dg_batch_add");
  if (st) return st;
  if (!op || !slot) return fail(DG_ERR_ARG, "dg_batch_add: NULL argument");
  if (op->precision != DG_FP32)
    return fail(DG_ERR_ARG, "dg_batch_add: the batch computes in FP32; set the operator up with DG_FP32");
  Pool& p = b->pools[op->N - 1];
  if (p.cap == 0)
    return fail(DG_ERR_ARG, "dg_batch_add: the batch has no capacity for order N = %d", op->N);
  if (!(dt > 0.0)) dt = (2.0 / 3.0) * op->min_inradius_over_c * op->ref.lgl_gap;
  if (!std::isfinite(dt)) return fail(DG_ERR_ARG, "dg_batch_add: dt is not finite");
  int64_t src_k = -1;
  std::vector<double> src_wt;
  if (src) {
    if (!std::isfinite(src->x) || !std::isfinite(src->y) || !(src->f > 0.0) ||
        !std::isfinite(src->t0) || !std::isfinite(src->amplitude))
      return fail(DG_ERR_ARG, "dg_batch_add: bad point source parameters");
    src_k = dgw::point_source(op->ref, op->geo, op->K, src->x, src->y, src_wt);
    if (src_k < 0)
      return fail(DG_ERR_ARG, "dg_batch_add: source point (%g, %g) is outside the mesh", src->x,
                  src->y);
  }
  // slot: the lowest free number (below max_slots: every live problem holds
  // at least 4 elements of some pool)
  int32_t id = -1;
  for (size_t i = 0; i < b->probs.size(); ++i)
    if (!b->probs[i].live) {
      id = static_cast<int32_t>(i);
      break;
    }
  if (id < 0) id = static_cast<int32_t>(b->probs.size());
  const int64_t K = op->K, len = (K + 3) / 4 * 4;
  const int64_t off = take_range(p, len);
  if (off < 0)
    return fail(DG_ERR_OOM, "dg_batch_add: no free range of %lld elements in the N = %d pool",
                static_cast<long long>(len), op->N);
  // records with this problem's step folded in, face codes in pool numbering
  std::vector<double> rec;
  try {
    dgw::media_records(*op, dt, rec);
  } catch (const std::bad_alloc&) {
    give_range(p, off, len);
    return fail(DG_ERR_OOM, "dg_batch_add: out of host memory");
  }
  if (src) rec[src_k * dgw::kGeoMedia + 19] = id + 1.0;
  const size_t rb = static_cast<size_t>(K) * dgw::kGeoMedia * 4, cb = static_cast<size_t>(K) * 12;
  const size_t sb = dgw::kSrcStride * 4 + 4 * sizeof(double) + sizeof(int);
  const size_t so = (rb + cb + 15) / 16 * 16;  // source block, 16-byte aligned
  size_t idx = 0;
  unsigned char* h = static_cast<unsigned char*>(b->staging.get(so + sb, &idx));
  if (!h) {
    give_range(p, off, len);
    return fail(DG_ERR_OOM, "dg_batch_add: pinned staging buffer");
  }
  float* hg = reinterpret_cast<float*>(h);
  int32_t* hc = reinterpret_cast<int32_t*>(h + rb);
  for (size_t i = 0; i < rec.size(); ++i) hg[i] = static_cast<float>(rec[i]);
  for (int64_t i = 0; i < 3 * K; ++i) {
    const int32_t code = op->geo.conn[i];
    hc[i] = code < 0 ? -1 : static_cast<int32_t>(((code >> 3) + off) * 8 + (code & 7));
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t err = cudaMemcpyAsync(p.geo + off * dgw::kGeoMedia, hg, rb, cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess) err = cudaMemcpyAsync(p.conn + off * 3, hc, cb, cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess && src) {
    // weights times this problem's dt, wavelet parameters, starting step
    double* hm = reinterpret_cast<double*>(h + so);
    float* hw = reinterpret_cast<float*>(h + so + 4 * sizeof(double));
    int* hs = reinterpret_cast<int*>(h + so + 4 * sizeof(double) + dgw::kSrcStride * 4);
    hm[0] = dt;
    hm[1] = src->t0;
    hm[2] = 3.14159265358979323846 * src->f;
    hm[3] = src->amplitude;
    for (int n = 0; n < dgw::kSrcStride; ++n)
      hw[n] = n < op->Np ? static_cast<float>(dt * src_wt[n]) : 0.0f;
    *hs = static_cast<int>(b->steps);
    err = cudaMemcpyAsync(b->d_src_meta + 4 * id, hm, 4 * sizeof(double), cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(b->d_src_w + dgw::kSrcStride * id, hw, dgw::kSrcStride * 4,
                            cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(b->d_src_step + id, hs, sizeof(int), cudaMemcpyHostToDevice, s);
  }
  if (err == cudaSuccess) err = b->staging.mark(idx, s);
  if (err != cudaSuccess) {
    give_range(p, off, len);
    return cuda_fail(err, "dg_batch_add: upload");
  }
  Problem pr;
  pr.live = true;
  pr.source = src != nullptr;
  pr.N = op->N;
  pr.K = K;
  pr.off = off;
  pr.len = len;
  pr.dt = dt;
  if (id == static_cast<int32_t>(b->probs.size()))
    b->probs.push_back(pr);
  else
    b->probs[id] = pr;
  b->dirty = true;
  *slot = id;
  return DG_OK;
}

extern "C" dg_status dg_batch_remove(dg_batch* b, int32_t slot) {
  dgw::clear_error();
  dg_status st = check_batch(b, "dg_batch_remove");
  if (st) return st;
  if ((st = check_slot(b, slot, "dg_batch_remove"))) return st;
  Problem& pr = b->probs[slot];
  give_range(b->pools[pr.N - 1], pr.off, pr.len);
  pr.live = false;
  b->dirty = true;
  return DG_OK;
}

extern "C" dg_status dg_batch_info(const dg_batch* b, int32_t slot, int32_t* N, int64_t* K,
                                   double* dt, int64_t* field_stride) {
  dgw::clear_error();
  if (!b) return fail(DG_ERR_ARG, "dg_batch_info: NULL batch");
  dg_status st = check_slot(b, slot, "dg_batch_info");
  if (st) return st;
  const Problem& pr = b->probs[slot];
  if (N) *N = pr.N;
  if (K) *K = pr.K;
  if (dt) *dt = pr.dt;
  if (field_stride) *field_stride = b->pools[pr.N - 1].fstride;
  return DG_OK;
}

namespace {

dg_status copy_fields(dg_batch* b, int32_t slot, void* other, int64_t other_stride, bool to_pool,
                      void* stream, const char* where) {
  dg_status st = check_batch(b, where);
  if (st) return st;
  if ((st = check_slot(b, slot, where))) return st;
  const Problem& pr = b->probs[slot];
  const Pool& p = b->pools[pr.N - 1];
  const int64_t n = pr.K * p.Np;
  float* dev = p.q[b->cur] + pr.off * p.Np;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t width = static_cast<size_t>(n) * 4;
  const size_t pitch_pool = static_cast<size_t>(p.fstride) * 4;
  if (!other) {
    if (!to_pool) return fail(DG_ERR_ARG, "%s: NULL buffer", where);
    cudaError_t err = cudaMemset2DAsync(dev, pitch_pool, 0, width, 3, s);  // zero fields
    if (err != cudaSuccess) return cuda_fail(err, where);
    return DG_OK;
  }
  if (other_stride < n) return fail(DG_ERR_ARG, "%s: field stride %lld < K * Np = %lld", where,
                                    static_cast<long long>(other_stride), static_cast<long long>(n));
  const size_t pitch_other = static_cast<size_t>(other_stride) * 4;
  cudaPointerAttributes attr;
  const bool pageable = cudaPointerGetAttributes(&attr, other) == cudaSuccess &&
                        attr.type == cudaMemoryTypeUnregistered;
  cudaGetLastError();  // clear a failed attribute query
  cudaError_t err;
  if (to_pool && pageable) {
    // through a pinned buffer, so that the call does not wait for the device
    size_t idx = 0;
    unsigned char* h = static_cast<unsigned char*>(b->staging.get(3 * width, &idx));
    if (!h) return fail(DG_ERR_OOM, "%s: pinned staging buffer", where);
    for (int f = 0; f < 3; ++f)
      std::memcpy(h + f * width, static_cast<const unsigned char*>(other) + f * pitch_other, width);
    err = cudaMemcpy2DAsync(dev, pitch_pool, h, width, width, 3, cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess) err = b->staging.mark(idx, s);
  } else {
    err = to_pool
              ? cudaMemcpy2DAsync(dev, pitch_pool, other, pitch_other, width, 3, cudaMemcpyDefault, s)
              : cudaMemcpy2DAsync(other, pitch_other, dev, pitch_pool, width, 3, cudaMemcpyDefault, s);
  }
  if (err != cudaSuccess) return cuda_fail(err, where);
  return DG_OK;
}

}  // namespace

extern "C" dg_status dg_batch_set_fields(dg_batch* b, int32_t slot, const void* src,
                                         int64_t src_stride, void* stream) {
  dgw::clear_error();
  return copy_fields(b, slot, const_cast<void*>(src), src_stride, true, stream,
                     "dg_batch_set_fields");
}

extern "C" dg_status dg_batch_get_fields(dg_batch* b, int32_t slot, void* dst,
                                         int64_t dst_stride, void* stream) {
  dgw::clear_error();
  return copy_fields(b, slot, dst, dst_stride, false, stream, "dg_batch_get_fields");
}

namespace {

constexpr int64_t kAdaptSteps = 8;  // steps between clock snapshots

// Per-order cost of one block iteration, from one launch's per-CTA clocks
// under the split cta[] with block counts nblk[]: the order's finish time
// after the launch's first CTA start over its block iterations per CTA.
void observed_costs(const unsigned long long* clk, const int* cta, const int64_t* nblk,
                    double* cost) {
  unsigned long long t0 = ~0ull;
  int c = 0;
  for (int g = 0; g < kOrders; ++g) c += cta[g];
  for (int i = 0; i < c; ++i) t0 = std::min(t0, clk[2 * i]);
  int first = 0;
  for (int g = 0; g < kOrders; ++g) {
    unsigned long long end = t0;
    for (int i = first; i < first + cta[g]; ++i) end = std::max(end, clk[2 * i + 1]);
    first += cta[g];
    if (cta[g] > 0 && nblk[g] > 0 && end > t0) {
      const int64_t iters = (nblk[g] + cta[g] - 1) / cta[g];
      cost[g] = 1e-9 * static_cast<double>(end - t0) / static_cast<double>(iters);
    }
  }
}

double makespan(const int64_t* nblk, const double* cost, const int* cta) {
  double m = 0.0;
  for (int g = 0; g < kOrders; ++g)
    if (cta[g] > 0) m = std::max(m, static_cast<double>((nblk[g] + cta[g] - 1) / cta[g]) * cost[g]);
  return m;
}

// a clock snapshot has arrived: move the costs halfway to the observed ones
// and switch to a new split when it predicts a makespan at least 3 % shorter
dg_status adapt_split(dg_batch* b, cudaStream_t s) {
  double obs[kOrders];
  std::copy(b->cost, b->cost + kOrders, obs);
  observed_costs(b->h_clock, b->clock_cta, b->clock_nblk, obs);
  for (int g = 0; g < kOrders; ++g) b->cost[g] = 0.5 * (b->cost[g] + obs[g]);
  int next[kOrders];
  if (!plan_ctas(b->nblk, b->cost, b->num_sms, next)) return DG_OK;
  if (std::equal(next, next + kOrders, b->cta)) return DG_OK;
  if (makespan(b->nblk, b->cost, next) > 0.97 * makespan(b->nblk, b->cost, b->cta)) return DG_OK;
  size_t idx = 0;
  int* meta = static_cast<int*>(b->staging.get(8 * sizeof(int), &idx));
  if (!meta) return fail(DG_ERR_OOM, "dg_batch_step: pinned staging buffer");
  meta[0] = 0;
  for (int g = 0; g < kOrders; ++g) meta[g + 1] = meta[g] + next[g];
  cudaError_t err = cudaMemcpyAsync(b->d_meta + 8, meta, 8 * sizeof(int), cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess) err = b->staging.mark(idx, s);
  if (err != cudaSuccess) return cuda_fail(err, "dg_batch_step: split upload");
  std::copy(next, next + kOrders, b->cta);
  ++b->replans;
  return DG_OK;
}

}  // namespace

extern "C" dg_status dg_batch_step(dg_batch* b, int32_t nsteps, void* stream) {
  dgw::clear_error();
  dg_status st = check_batch(b, "dg_batch_step");
  if (st) return st;
  if (nsteps < 0) return fail(DG_ERR_ARG, "dg_batch_step: nsteps = %d < 0", nsteps);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (b->dirty && (st = upload_tables(b, s))) return st;
  const bool use_graph = !(b->flags & DG_BATCH_NO_GRAPH);
  if (use_graph && !b->graph[0] && (st = capture_graphs(b))) return st;
  for (int32_t n = 0; n < nsteps; ++n) {
    if (use_graph) {
      cudaError_t err = cudaGraphLaunch(b->graph[b->cur], s);
      if (err != cudaSuccess) return cuda_fail(err, "dg_batch_step: graph launch");
      b->launches += launches_per_step(b);
    } else {
      cudaError_t err = launch_step(b, b->cur, s);
      if (err != cudaSuccess) return cuda_fail(err, "dg_batch_step: kernel launch");
    }
    b->cur ^= 1;
    ++b->steps;
  }
  if (!(b->flags & DG_BATCH_NO_ADAPT) && !b->concurrent && nsteps > 0) {
    if (b->clock_pending && cudaEventQuery(b->clock_ev) == cudaSuccess) {
      b->clock_pending = false;
      if (!b->dirty && (st = adapt_split(b, s))) return st;
    }
    b->steps_since_snapshot += nsteps;
    if (!b->clock_pending && b->steps_since_snapshot >= kAdaptSteps) {
      cudaError_t err = cudaMemcpyAsync(b->h_clock, b->d_clock,
                                        2 * static_cast<size_t>(b->num_sms) * sizeof(unsigned long long),
                                        cudaMemcpyDeviceToHost, s);
      if (err == cudaSuccess) err = cudaEventRecord(b->clock_ev, s);
      if (err != cudaSuccess) return cuda_fail(err, "dg_batch_step: clock snapshot");
      std::copy(b->cta, b->cta + kOrders, b->clock_cta);
      std::copy(b->nblk, b->nblk + kOrders, b->clock_nblk);
      b->clock_pending = true;
      b->steps_since_snapshot = 0;
    }
  }
  return DG_OK;
}

extern "C" dg_status dg_batch_tune(dg_batch* b, int32_t reps, void* stream) {
  dgw::clear_error();
  dg_status st = check_batch(b, "dg_batch_tune");
  if (st) return st;
  if (reps < 1) return fail(DG_ERR_ARG, "dg_batch_tune: reps = %d < 1", reps);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((st = upload_tables(b, s))) return st;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaError_t err = cudaSuccess;
  std::vector<unsigned long long> clk(2 * static_cast<size_t>(b->num_sms));
  int meta[16];
  auto set_plan = [&](const int* cta) -> cudaError_t {
    meta[7] = 0;
    meta[8] = 0;
    for (int g = 0; g < kOrders; ++g) {
      meta[g] = static_cast<int>(b->nblk[g]);
      meta[9 + g] = meta[8 + g] + cta[g];
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_meta, meta, sizeof(meta), cudaMemcpyHostToDevice);
    return e;
  };
  // time `reps` stage launches (stage 2 form: reads q[cur] and the residual,
  // writes the other buffer and the residual; the fields stay as they are)
  auto timed = [&](const int* cta, float* ms) -> cudaError_t {
    cudaError_t e = set_plan(cta);
    if (e == cudaSuccess) e = launch_stage(b, b->cur, 1, s);  // warm
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_stage(b, b->cur, 1, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    return e;
  };
  // one launch with per-CTA clocks: each order's finish time after the
  // launch's first CTA start, divided by its block iterations per CTA
  auto observed = [&](const int* cta, double* cost) -> cudaError_t {
    cudaError_t e = set_plan(cta);
    if (e == cudaSuccess) e = launch_stage(b, b->cur, 1, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess)
      e = cudaMemcpy(clk.data(), b->d_clock, clk.size() * sizeof(unsigned long long),
                     cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) observed_costs(clk.data(), cta, b->nblk, cost);
    return e;
  };
  // 1. each order alone on all SMs
  int alone[kOrders];
  for (int g = 0; g < kOrders && err == cudaSuccess; ++g) {
    if (b->nblk[g] == 0) continue;
    for (int h = 0; h < kOrders; ++h) alone[h] = 0;
    alone[g] = b->num_sms;
    float ms = 0.f;
    err = timed(alone, &ms);
    const int64_t iters = (b->nblk[g] + b->num_sms - 1) / b->num_sms;
    b->cost[g] = 1e-3 * ms / reps / static_cast<double>(iters);
  }
  // 2. plan, then re-plan from the costs observed in the mixed launch (the
  //    orders share HBM and L2 there) while the plan changes
  int best[kOrders], plan[kOrders];
  float best_ms = 0.f;
  if (err == cudaSuccess) {
    plan_ctas(b->nblk, b->cost, b->num_sms, plan);
    std::copy(plan, plan + kOrders, best);
    err = timed(best, &best_ms);
  }
  for (int it = 0; it < 6 && err == cudaSuccess; ++it) {
    double cost[kOrders];
    std::copy(b->cost, b->cost + kOrders, cost);
    err = observed(plan, cost);
    if (err != cudaSuccess) break;
    std::copy(cost, cost + kOrders, b->cost);
    int next[kOrders];
    plan_ctas(b->nblk, b->cost, b->num_sms, next);
    if (std::equal(next, next + kOrders, plan)) break;
    std::copy(next, next + kOrders, plan);
    float ms = 0.f;
    err = timed(plan, &ms);
    if (err == cudaSuccess && ms < best_ms) {
      best_ms = ms;
      std::copy(plan, plan + kOrders, best);
    }
  }
  // 3. single-CTA moves between orders that measure faster
  for (int round = 0; round < 2 && err == cudaSuccess; ++round) {
    bool improved = false;
    for (int from = 0; from < kOrders && err == cudaSuccess; ++from) {
      for (int to = 0; to < kOrders && err == cudaSuccess; ++to) {
        if (from == to || best[from] <= 1 || best[to] == 0 || best[to] >= b->nblk[to]) continue;
        int trial[kOrders];
        std::copy(best, best + kOrders, trial);
        --trial[from];
        ++trial[to];
        float ms = 0.f;
        err = timed(trial, &ms);
        if (err == cudaSuccess && ms < 0.995f * best_ms) {
          std::copy(trial, trial + kOrders, best);
          best_ms = ms;
          improved = true;
        }
      }
    }
    if (!improved) break;
  }
  if (err != cudaSuccess) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return cuda_fail(err, "dg_batch_tune");
  }
  b->measured = true;
  std::copy(best, best + kOrders, b->cta);
  err = set_plan(b->cta);
  // 4. launch mode: the tuned split against the orders' own kernels side by
  //    side (same stage, same reps); the faster one is kept (DG_BATCH_SPLIT
  //    keeps the split)
  if (err == cudaSuccess && !(b->flags & DG_BATCH_SPLIT)) {
    float conc_ms = 0.f;
    err = launch_concurrent(b, b->cur, 1, 1, false, s);  // warm
    if (err == cudaSuccess) err = cudaEventRecord(e0, s);
    if (err == cudaSuccess) err = launch_concurrent(b, b->cur, 1, reps, false, s);
    if (err == cudaSuccess) err = cudaEventRecord(e1, s);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    if (err == cudaSuccess) err = cudaEventElapsedTime(&conc_ms, e0, e1);
    if (err == cudaSuccess) {
      const bool conc = conc_ms <= best_ms;
      if (conc != b->concurrent) {
        for (cudaGraphExec_t& g : b->graph) {
          if (g) cudaGraphExecDestroy(g);
          g = nullptr;
        }
      }
      b->concurrent = conc;
      b->tuned_split_ms = best_ms;
      b->tuned_concurrent_ms = conc_ms;
    }
  }
  if (err == cudaSuccess && !b->concurrent) {  // the split mode runs the default block sizes
    for (int g = 0; g < kOrders; ++g) set_order_alt(b, g, false);
    if (b->dirty && upload_tables(b, s) != DG_OK) err = cudaErrorUnknown;
  }
  // 5. concurrent mode: each order's element-block size, the default against
  //    the alternative where there is one, each timed alone on all SMs over
  //    the order's own blocks (tables rebuilt for each size); the faster kept
  for (int g = 0; g < kOrders && err == cudaSuccess && b->concurrent; ++g) {
    if (b->nblk[g] == 0 || dgw::batch_tc_block_elems(g + 1, true) == dgw::batch_tc_block_elems(g + 1, false))
      continue;
    float t[2] = {0.f, 0.f};
    for (int v = 0; v < 2 && err == cudaSuccess; ++v) {
      set_order_alt(b, g, v == 1);
      if (upload_tables(b, s) != DG_OK) {
        err = cudaErrorUnknown;
        break;
      }
      err = launch_order_stage(b, g, b->cur, 1, b->num_sms, s);  // warm
      if (err == cudaSuccess) err = cudaEventRecord(e0, s);
      for (int r = 0; r < reps && err == cudaSuccess; ++r)
        err = launch_order_stage(b, g, b->cur, 1, b->num_sms, s);
      if (err == cudaSuccess) err = cudaEventRecord(e1, s);
      if (err == cudaSuccess) err = cudaEventSynchronize(e1);
      if (err == cudaSuccess) err = cudaEventElapsedTime(&t[v], e0, e1);
    }
    if (err == cudaSuccess) {
      set_order_alt(b, g, t[1] < t[0]);
      b->tuned_order_ms[g][0] = t[0];
      b->tuned_order_ms[g][1] = t[1];
      if (b->dirty && upload_tables(b, s) != DG_OK) err = cudaErrorUnknown;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return cuda_fail(err, "dg_batch_tune: plan upload / launch mode");
  return DG_OK;
}

extern "C" dg_status dg_batch_plan(const dg_batch* b, int32_t* cta, int64_t* nblocks,
                                   double* cost) {
  dgw::clear_error();
  if (!b) return fail(DG_ERR_ARG, "dg_batch_plan: NULL batch");
  for (int g = 0; g < kOrders; ++g) {
    // concurrent mode: each order's kernel has one CTA per SM, of which as
    // many as it has blocks do work
    if (cta)
      cta[g] = b->concurrent ? static_cast<int32_t>(std::min<int64_t>(b->num_sms, b->nblk[g]))
                             : b->cta[g];
    if (nblocks) nblocks[g] = b->nblk[g];
    if (cost) cost[g] = b->cost[g];
  }
  return DG_OK;
}

extern "C" dg_status dg_batch_launch_mode(const dg_batch* b, int32_t* mode, double* split_ms,
                                          double* concurrent_ms) {
  dgw::clear_error();
  if (!b) return fail(DG_ERR_ARG, "dg_batch_launch_mode: NULL batch");
  if (mode) *mode = b->concurrent ? DG_BATCH_MODE_CONCURRENT : DG_BATCH_MODE_SPLIT;
  if (split_ms) *split_ms = b->tuned_split_ms;
  if (concurrent_ms) *concurrent_ms = b->tuned_concurrent_ms;
  return DG_OK;
}

extern "C" dg_status dg_batch_set_block_elems(dg_batch* b, int32_t N, int32_t elems) {
  dgw::clear_error();
  const char* where = "dg_batch_set_block_elems";
  dg_status st = check_batch(b, where);
  if (st) return st;
  if (N < 1 || N > kOrders || b->pools[N - 1].cap == 0)
    return fail(DG_ERR_ARG, "%s: the batch has no pool for order N = %d", where, N);
  const int def = dgw::batch_tc_block_elems(N, false), alt = dgw::batch_tc_block_elems(N, true);
  if (elems == 0 || elems == def) {
    set_order_alt(b, N - 1, false);
  } else if (elems == alt && alt != def) {
    if (!b->concurrent)
      return fail(DG_ERR_ARG, "%s: the split launch mode runs the default size (%d)", where, def);
    set_order_alt(b, N - 1, true);
  } else {
    return fail(DG_ERR_ARG, "%s: %d elements per block is not a size of order %d (%d%s)", where,
                elems, N, def, alt != def ? (" or " + std::to_string(alt)).c_str() : "");
  }
  return DG_OK;
}

extern "C" dg_status dg_batch_block_elems(const dg_batch* b, int32_t* elems, double* ms_default,
                                          double* ms_alt) {
  dgw::clear_error();
  if (!b || !elems) return fail(DG_ERR_ARG, "dg_batch_block_elems: NULL argument");
  for (int g = 0; g < kOrders; ++g) {
    elems[g] = b->pools[g].cap > 0 ? b->pools[g].E : 0;
    if (ms_default) ms_default[g] = b->tuned_order_ms[g][0];
    if (ms_alt) ms_alt[g] = b->tuned_order_ms[g][1];
  }
  return DG_OK;
}

extern "C" dg_status dg_batch_sync_check(dg_batch* b, void* stream) {
  dgw::clear_error();
  dg_status st = check_batch(b, "dg_batch_sync_check");
  if (st) return st;
  cudaError_t err = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (err == cudaSuccess) err = cudaGetLastError();
  if (err != cudaSuccess) return cuda_fail(err, "dg_batch_sync_check");
  int status = 0;
  err = cudaMemcpy(&status, b->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (err != cudaSuccess) return cuda_fail(err, "dg_batch_sync_check: status read");
  if (status != 0) {
    cudaMemset(b->d_status, 0, sizeof(int));
    if (status & dgw::kStatusIndex)
      return fail(DG_ERR_INDEX,
                  "dg_batch_sync_check: a checked kernel found an index out of range");
    return fail(DG_ERR_TIMEOUT, "dg_batch_sync_check: a kernel's bounded wait expired");
  }
  return DG_OK;
}

extern "C" int64_t dg_batch_launch_count(const dg_batch* b) { return b ? b->launches : 0; }
