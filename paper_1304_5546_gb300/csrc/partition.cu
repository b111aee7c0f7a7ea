// Mesh partitions with a halo exchange per stage (dg_partition_*).
//
// The solver shards by mesh partition: each part owns a set of elements and
// needs, per LSRK stage, only the face traces of the elements across its
// cuts (Section "Further Tuning Opportunities": only face data crosses
// between GPUs).  Here the P parts live on one device.  Each part is an
// operator of its own (element records, connection codes, field buffers)
// whose connection codes point either at its own elements or at ghost slots
// placed after its padded element range; an exchange packs every part's
// outgoing traces into one message per (sender, receiver) pair, transfers
// the messages (one copy on one device, where separate devices would send /
// receive per pair) and unpacks them into the receivers' ghost slots.  The stage kernels are the single-operator ones, unchanged: they
// read neighbour traces through the connection codes, wherever they point.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <numeric>
#include <stdexcept>
#include <vector>

#include "internal.h"
#include "launch.h"

using dgw::fail;

namespace {

constexpr int kMaxParts = 64;
// same padding rule as a single operator: whole blocks of <= 64 elements
// plus a spare element for the bulk copies' 16-byte rounding
constexpr int64_t kBlockPad = 64;

dg_status cuda_fail(cudaError_t err, const char* where) {
  return fail(err == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA, "%s: %s (%s)", where,
              cudaGetErrorName(err), cudaGetErrorString(err));
}

// one (sender, receiver) pair of an exchange: node offsets in one field of
// the sender's layout and of the receiver's, entry for entry
struct Pair {
  int src = 0, dst = 0;
  std::vector<int32_t> src_off, dst_off;
  int64_t send_pos = 0, recv_pos = 0;  // first entry in the send / receive buffers
};

// pack / unpack entry: part, node offset in one field of that part, position
// of field 0 in the exchange buffer, and the pair's entry count (field f of
// the entry sits at pos + f * count, so that a pair's three fields are one
// contiguous run of the buffer)
struct Entry {
  int32_t part, off;
  int64_t pos, count;
};

template <typename T>
__global__ void halo_pack_kernel(const Entry* __restrict__ ent, int64_t n,
                                 T* const* __restrict__ base, const int64_t* __restrict__ fs,
                                 T* __restrict__ buf) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const Entry e = ent[i];
    const T* q = base[e.part];
    const int64_t s = fs[e.part];
    buf[e.pos] = q[e.off];
    buf[e.pos + e.count] = q[s + e.off];
    buf[e.pos + 2 * e.count] = q[2 * s + e.off];
  }
}

template <typename T>
__global__ void halo_unpack_kernel(const Entry* __restrict__ ent, int64_t n,
                                   T* const* __restrict__ base, const int64_t* __restrict__ fs,
                                   const T* __restrict__ buf) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const Entry e = ent[i];
    T* q = base[e.part];
    const int64_t s = fs[e.part];
    q[e.off] = buf[e.pos];
    q[s + e.off] = buf[e.pos + e.count];
    q[2 * s + e.off] = buf[e.pos + 2 * e.count];
  }
}

// element copies between the global fields (stride gs) and a part (stride
// ls): part element e is global element gid[e]; to_part copies global ->
// part, otherwise part -> global
template <typename T>
__global__ void part_copy_kernel(const T* __restrict__ src, T* __restrict__ dst, int64_t gs,
                                 int64_t ls, const int64_t* __restrict__ gid, int64_t Kp, int Np,
                                 bool to_part) {
  const int64_t n = Kp * Np;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t e = i / Np;
    const int64_t g = gid[e] * Np + (i - e * Np);
    for (int f = 0; f < 3; ++f) {
      if (to_part)
        dst[f * ls + i] = src[f * gs + g];
      else
        dst[f * gs + g] = src[f * ls + i];
    }
  }
}

// Recursive coordinate bisection of the elements `ids` (centroids cx, cy)
// into parts first .. first + P - 1: split across the wider extent at the
// element that gives the two halves P_left / P shares of the elements.
void rcb(std::vector<int64_t>::iterator lo, std::vector<int64_t>::iterator hi, int P, int first,
         const std::vector<double>& cx, const std::vector<double>& cy, std::vector<int>& owner) {
  if (P == 1) {
    for (auto it = lo; it != hi; ++it) owner[*it] = first;
    return;
  }
  double x0 = 1e300, x1 = -1e300, y0 = 1e300, y1 = -1e300;
  for (auto it = lo; it != hi; ++it) {
    x0 = std::min(x0, cx[*it]);
    x1 = std::max(x1, cx[*it]);
    y0 = std::min(y0, cy[*it]);
    y1 = std::max(y1, cy[*it]);
  }
  const std::vector<double>& c = (x1 - x0 >= y1 - y0) ? cx : cy;
  const int Pl = P / 2;
  const int64_t n = hi - lo;
  const int64_t nl = n * Pl / P;
  // ties broken by element id, so that the split is deterministic
  std::nth_element(lo, lo + nl, hi, [&](int64_t a, int64_t b) {
    return c[a] < c[b] || (c[a] == c[b] && a < b);
  });
  rcb(lo, lo + nl, Pl, first, cx, cy, owner);
  rcb(lo + nl, hi, P - Pl, first + Pl, cx, cy, owner);
}

}  // namespace

struct dg_partition {
  const dg_op* op = nullptr;
  int P = 0;
  bool device = false;
  std::vector<std::vector<int64_t>> own, ghost;
  std::vector<std::vector<int32_t>> conn;
  std::vector<int64_t> Kpad, fstride;
  std::vector<Pair> pairs;  // sorted by (src, dst)
  int64_t n_entries = 0;    // per field, over all pairs
  // device state
  std::vector<dg_op*> sub;
  std::vector<void*> d_q, d_res;  // per part, 3 * fstride values each
  std::vector<int64_t*> d_gid;
  void** d_base = nullptr;  // [2][P]: parity 0 = d_q, parity 1 = the part's ping-pong buffer
  int64_t* d_fs = nullptr;
  Entry* d_pack = nullptr;
  Entry* d_unpack = nullptr;
  void* d_send = nullptr;
  void* d_recv = nullptr;
  int cur = 0;  // parity of the buffers holding the current fields
  // one stream per part: the parts' stage launches of one stage are
  // independent, so a part's CTAs start on the SMs that the previous part's
  // tail leaves idle
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> part_done;
  cudaEvent_t exchanged = nullptr;

  ~dg_partition() {
    for (cudaStream_t st : streams) {
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    }
    for (cudaEvent_t e : part_done) cudaEventDestroy(e);
    if (exchanged) cudaEventDestroy(exchanged);
    for (dg_op* s : sub) dg_op_destroy(s);
    for (void* p : d_q) cudaFree(p);
    for (void* p : d_res) cudaFree(p);
    for (int64_t* p : d_gid) cudaFree(p);
    void* ptrs[] = {d_base, d_fs, d_pack, d_unpack, d_send, d_recv};
    for (void* p : ptrs)
      if (p) cudaFree(p);
  }
};

namespace {

// The plan: owners by RCB, each part's elements in increasing global order,
// ghost slots in order of first use, connection codes, exchange pairs.
void build_plan(dg_partition& pt) {
  const dg_op& op = *pt.op;
  const int64_t K = op.K;
  const int Np = op.Np, Nfp = op.Nfp, N = op.N;
  const int P = pt.P;
  std::vector<double> cx(K), cy(K);
  for (int64_t k = 0; k < K; ++k) {
    const int64_t b = k * Np;
    cx[k] = (op.geo.x[b] + op.geo.x[b + N] + op.geo.x[b + Np - 1]) / 3.0;
    cy[k] = (op.geo.y[b] + op.geo.y[b + N] + op.geo.y[b + Np - 1]) / 3.0;
  }
  std::vector<int64_t> ids(K);
  std::iota(ids.begin(), ids.end(), int64_t(0));
  std::vector<int> owner(K, 0);
  rcb(ids.begin(), ids.end(), P, 0, cx, cy, owner);

  pt.own.assign(P, {});
  std::vector<int64_t> local(K);
  for (int64_t k = 0; k < K; ++k) {
    local[k] = static_cast<int64_t>(pt.own[owner[k]].size());
    pt.own[owner[k]].push_back(k);
  }
  pt.ghost.assign(P, {});
  pt.conn.assign(P, {});
  pt.Kpad.assign(P, 0);
  pt.fstride.assign(P, 0);
  std::map<std::pair<int, int>, Pair> pairs;
  for (int p = 0; p < P; ++p) {
    const std::vector<int64_t>& el = pt.own[p];
    const int64_t Kp = static_cast<int64_t>(el.size());
    const int64_t Kpad = (Kp + 1 + kBlockPad - 1) / kBlockPad * kBlockPad;
    pt.Kpad[p] = Kpad;
    std::map<int64_t, int64_t> slot;  // global id -> ghost slot
    // (global node) values part p receives, deduplicated per sender
    std::map<int, std::vector<int64_t>> want;
    pt.conn[p].assign(3 * Kp, -1);
    for (int64_t e = 0; e < Kp; ++e) {
      for (int f = 0; f < 3; ++f) {
        const int32_t code = op.geo.conn[3 * el[e] + f];
        if (code < 0) continue;
        const int64_t kP = code >> 3;
        int64_t idx;
        if (owner[kP] == p) {
          idx = local[kP];
        } else {
          auto it = slot.find(kP);
          if (it == slot.end()) it = slot.emplace(kP, static_cast<int64_t>(slot.size())).first;
          idx = Kpad + it->second;
          const int fP = (code >> 1) & 3;
          for (int j = 0; j < Nfp; ++j)
            want[owner[kP]].push_back(kP * Np + dgw::face_node(N, fP, j));
        }
        pt.conn[p][3 * e + f] = static_cast<int32_t>(idx * 8 + (code & 7));
      }
    }
    pt.ghost[p].resize(slot.size());
    for (const auto& kv : slot) pt.ghost[p][kv.second] = kv.first;
    const int64_t G = static_cast<int64_t>(slot.size());
    pt.fstride[p] = ((Kpad + G) * Np + 63) / 64 * 64;
    if (pt.fstride[p] >= (int64_t(1) << 31) || (Kpad + G) * 8 >= (int64_t(1) << 31))
      throw std::length_error("a part's field exceeds 2^31 - 1 values");
    for (auto& kv : want) {
      std::vector<int64_t>& nodes = kv.second;
      std::sort(nodes.begin(), nodes.end());
      nodes.erase(std::unique(nodes.begin(), nodes.end()), nodes.end());
      Pair& pr = pairs[{kv.first, p}];
      pr.src = kv.first;
      pr.dst = p;
      for (int64_t gn : nodes) {
        const int64_t k = gn / Np, n = gn - k * Np;
        pr.src_off.push_back(static_cast<int32_t>(local[k] * Np + n));
        pr.dst_off.push_back(static_cast<int32_t>((Kpad + slot[k]) * Np + n));
      }
    }
  }
  pt.pairs.clear();
  for (auto& kv : pairs) pt.pairs.push_back(std::move(kv.second));  // (src, dst) order
  // the messages of all pairs, in (src, dst) order, are consecutive runs of
  // one send buffer and sit at the same place in one receive buffer
  int64_t pos = 0;
  for (Pair& pr : pt.pairs) {
    pr.send_pos = pr.recv_pos = pos;
    pos += static_cast<int64_t>(pr.src_off.size());
  }
  pt.n_entries = pos;
}

template <typename T>
dg_status build_device(dg_partition& pt) {
  const dg_op& op = *pt.op;
  const int P = pt.P;
  std::vector<double> rec;
  std::vector<int32_t> conn_full;
  dgw::operator_records(op, rec, conn_full);
  const int R = op.media() ? dgw::kGeoMedia : dgw::kGeo;
  for (int p = 0; p < P; ++p) {
    dg_op* s = new dg_op;
    pt.sub.push_back(s);
    s->N = op.N;
    s->Np = op.Np;
    s->Nfp = op.Nfp;
    s->Nafp = op.Nafp;
    s->precision = op.precision;
    s->flags = op.flags;
    s->ref = op.ref;
    s->alpha = op.alpha;
    s->face_pairs = op.face_pairs;
    s->use_tc = op.use_tc;
    s->use_ept = op.use_ept;
    s->tc_prec = op.tc_prec;
    s->elem_size = op.elem_size;
    s->device = op.device;
    s->num_sms = op.num_sms;
    s->min_inradius_over_c = op.min_inradius_over_c;
    std::memcpy(s->lsrk_a, op.lsrk_a, sizeof(op.lsrk_a));
    std::memcpy(s->lsrk_b, op.lsrk_b, sizeof(op.lsrk_b));
    std::memcpy(s->lsrk_c, op.lsrk_c, sizeof(op.lsrk_c));
    const std::vector<int64_t>& el = pt.own[p];
    s->K = static_cast<int64_t>(el.size());
    s->Kpad = pt.Kpad[p];
    s->fstride = pt.fstride[p];
    if (op.media())
      for (int64_t k : el) s->eps.push_back(op.eps[k]);
    std::vector<double> rp(static_cast<size_t>(s->K) * R);
    for (int64_t e = 0; e < s->K; ++e)
      std::copy(&rec[el[e] * R], &rec[el[e] * R] + R, &rp[e * R]);
    dg_status st = dgw::upload_operator(s, rp, pt.conn[p]);
    if (st) return st;
    s->has_device = true;
    const size_t fb = 3 * static_cast<size_t>(s->fstride) * sizeof(T);
    void* q = nullptr;
    void* r = nullptr;
    int64_t* g = nullptr;
    cudaError_t err = dgw::dev_malloc(&q, fb);
    if (err == cudaSuccess) pt.d_q.push_back(q);
    if (err == cudaSuccess) err = dgw::dev_malloc(&r, fb);
    if (err == cudaSuccess) pt.d_res.push_back(r);
    if (err == cudaSuccess) err = dgw::dev_malloc(&g, std::max<size_t>(el.size(), 1) * 8);
    if (err == cudaSuccess) pt.d_gid.push_back(g);
    if (err == cudaSuccess) err = cudaMemset(q, 0, fb);
    if (err == cudaSuccess) err = cudaMemset(r, 0, fb);
    if (err == cudaSuccess && !el.empty())
      err = cudaMemcpy(g, el.data(), el.size() * 8, cudaMemcpyHostToDevice);
    if (err != cudaSuccess) return cuda_fail(err, "dg_partition_create: part buffers");
  }
  std::vector<void*> base(2 * static_cast<size_t>(P));
  for (int p = 0; p < P; ++p) {
    base[p] = pt.d_q[p];
    base[P + p] = pt.sub[p]->d_qtmp;
  }
  std::vector<Entry> pack, unpack;
  pack.reserve(pt.n_entries);
  unpack.resize(pt.n_entries);
  for (const Pair& pr : pt.pairs) {
    const int64_t c = static_cast<int64_t>(pr.src_off.size());
    for (int64_t i = 0; i < c; ++i) {
      pack.push_back({pr.src, pr.src_off[i], 3 * pr.send_pos + i, c});
      unpack[pr.recv_pos + i] = {pr.dst, pr.dst_off[i], 3 * pr.recv_pos + i, c};
    }
  }
  const size_t nb = std::max<size_t>(3 * static_cast<size_t>(pt.n_entries), 1) * sizeof(T);
  const size_t eb = std::max<size_t>(static_cast<size_t>(pt.n_entries), 1) * sizeof(Entry);
  cudaError_t err = dgw::dev_malloc(&pt.d_base, base.size() * sizeof(void*));
  if (err == cudaSuccess) err = dgw::dev_malloc(&pt.d_fs, P * sizeof(int64_t));
  if (err == cudaSuccess) err = dgw::dev_malloc(&pt.d_pack, eb);
  if (err == cudaSuccess) err = dgw::dev_malloc(&pt.d_unpack, eb);
  if (err == cudaSuccess) err = dgw::dev_malloc(&pt.d_send, nb);
  if (err == cudaSuccess) err = dgw::dev_malloc(&pt.d_recv, nb);
  if (err == cudaSuccess)
    err = cudaMemcpy(pt.d_base, base.data(), base.size() * sizeof(void*), cudaMemcpyHostToDevice);
  if (err == cudaSuccess)
    err = cudaMemcpy(pt.d_fs, pt.fstride.data(), P * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (err == cudaSuccess && pt.n_entries > 0) {
    err = cudaMemcpy(pt.d_pack, pack.data(), pack.size() * sizeof(Entry), cudaMemcpyHostToDevice);
    if (err == cudaSuccess)
      err = cudaMemcpy(pt.d_unpack, unpack.data(), unpack.size() * sizeof(Entry),
                       cudaMemcpyHostToDevice);
  }
  if (err != cudaSuccess) return cuda_fail(err, "dg_partition_create: exchange tables");
  err = cudaEventCreateWithFlags(&pt.exchanged, cudaEventDisableTiming);
  for (int p = 0; p < P && err == cudaSuccess; ++p) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    err = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (err == cudaSuccess) pt.streams.push_back(st);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (err == cudaSuccess) pt.part_done.push_back(ev);
  }
  if (err != cudaSuccess) return cuda_fail(err, "dg_partition_create: streams");
  return DG_OK;
}

int grid_for(int64_t n, int num_sms) {
  const int64_t g = (n + 255) / 256;
  return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(g, int64_t(num_sms) * 8)));
}

template <typename T>
cudaError_t exchange(dg_partition& pt, cudaStream_t s) {
  if (pt.n_entries == 0) return cudaSuccess;
  const int grid = grid_for(pt.n_entries, pt.op->num_sms);
  T* const* base = reinterpret_cast<T* const*>(pt.d_base) + pt.cur * pt.P;
  halo_pack_kernel<T><<<grid, 256, 0, s>>>(pt.d_pack, pt.n_entries, base, pt.d_fs,
                                           static_cast<T*>(pt.d_send));
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  // the transfer: every pair's message at once (one device, one copy; between
  // devices, one send / receive per pair)
  err = cudaMemcpyAsync(pt.d_recv, pt.d_send, 3 * static_cast<size_t>(pt.n_entries) * sizeof(T),
                        cudaMemcpyDeviceToDevice, s);
  if (err != cudaSuccess) return err;
  halo_unpack_kernel<T><<<grid, 256, 0, s>>>(pt.d_unpack, pt.n_entries, base, pt.d_fs,
                                             static_cast<const T*>(pt.d_recv));
  return cudaGetLastError();
}

dg_status check_part(const dg_partition* pt, int32_t p, const char* where) {
  if (!pt) return fail(DG_ERR_ARG, "%s: NULL partition", where);
  if (p < 0 || p >= pt->P) return fail(DG_ERR_ARG, "%s: part %d outside [0, %d)", where, p, pt->P);
  return DG_OK;
}

dg_status check_device_part(const dg_partition* pt, const char* where) {
  if (!pt) return fail(DG_ERR_ARG, "%s: NULL partition", where);
  if (!pt->device)
    return fail(DG_ERR_NO_DEVICE, "%s: partition of a host-only operator (plan only)", where);
  cudaError_t err = cudaSetDevice(pt->op->device);
  if (err != cudaSuccess) return cuda_fail(err, where);
  return DG_OK;
}

// global fields q <-> the parts' current fields; q is only read when
// to_part is set
template <typename T>
dg_status copy_fields(dg_partition& pt, T* q, int64_t q_stride, bool to_part, cudaStream_t s,
                      const char* where) {
  for (int p = 0; p < pt.P; ++p) {
    const int64_t Kp = static_cast<int64_t>(pt.own[p].size());
    if (Kp == 0) continue;
    T* loc = static_cast<T*>(pt.cur ? pt.sub[p]->d_qtmp : pt.d_q[p]);
    part_copy_kernel<T><<<grid_for(Kp * pt.op->Np, pt.op->num_sms), 256, 0, s>>>(
        to_part ? q : loc, to_part ? loc : q, q_stride, pt.fstride[p], pt.d_gid[p], Kp,
        pt.op->Np, to_part);
    const cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return cuda_fail(err, where);
  }
  return DG_OK;
}

}  // namespace

extern "C" dg_status dg_partition_create(const dg_op* op, int32_t P, dg_partition** out) {
  dgw::clear_error();
  const char* where = "dg_partition_create";
  if (!op || !out) return fail(DG_ERR_ARG, "%s: NULL argument", where);
  *out = nullptr;
  if (op->has_src)
    return fail(DG_ERR_ARG, "%s: the operator has a point source; partitions step without one",
                where);
  if (P < 1 || P > kMaxParts || P > op->K)
    return fail(DG_ERR_ARG, "%s: P = %d outside [1, min(K = %lld, %d)]", where, P,
                static_cast<long long>(op->K), kMaxParts);
  dg_partition* pt = nullptr;
  try {
    pt = new dg_partition;
    pt->op = op;
    pt->P = P;
    build_plan(*pt);
  } catch (const std::bad_alloc&) {
    delete pt;
    return fail(DG_ERR_OOM, "%s: out of host memory", where);
  } catch (const std::exception& ex) {
    delete pt;
    return fail(DG_ERR_ARG, "%s: %s", where, ex.what());
  }
  if (op->has_device) {
    cudaError_t err = cudaSetDevice(op->device);
    if (err != cudaSuccess) {
      delete pt;
      return cuda_fail(err, where);
    }
    dg_status st;
    try {
      st = (op->precision == DG_FP32) ? build_device<float>(*pt) : build_device<double>(*pt);
    } catch (const std::bad_alloc&) {
      st = fail(DG_ERR_OOM, "%s: out of host memory", where);
    }
    if (st) {
      delete pt;
      return st;
    }
    pt->device = true;
  }
  *out = pt;
  return DG_OK;
}

extern "C" void dg_partition_destroy(dg_partition* part) {
  if (!part) return;
  if (part->device) cudaSetDevice(part->op->device);
  delete part;
}

extern "C" dg_status dg_partition_info(const dg_partition* part, int32_t p, int64_t* K_p,
                                       int64_t* G_p, int32_t* n_recv_peers,
                                       int32_t* n_send_peers, int64_t* n_recv, int64_t* n_send) {
  dgw::clear_error();
  dg_status st = check_part(part, p, "dg_partition_info");
  if (st) return st;
  int32_t rp = 0, sp = 0;
  int64_t rn = 0, sn = 0;
  for (const Pair& pr : part->pairs) {
    if (pr.dst == p) {
      ++rp;
      rn += static_cast<int64_t>(pr.dst_off.size());
    }
    if (pr.src == p) {
      ++sp;
      sn += static_cast<int64_t>(pr.src_off.size());
    }
  }
  if (K_p) *K_p = static_cast<int64_t>(part->own[p].size());
  if (G_p) *G_p = static_cast<int64_t>(part->ghost[p].size());
  if (n_recv_peers) *n_recv_peers = rp;
  if (n_send_peers) *n_send_peers = sp;
  if (n_recv) *n_recv = rn;
  if (n_send) *n_send = sn;
  return DG_OK;
}

extern "C" dg_status dg_partition_elements(const dg_partition* part, int32_t p, int64_t* gid) {
  dgw::clear_error();
  dg_status st = check_part(part, p, "dg_partition_elements");
  if (st) return st;
  if (!gid) return fail(DG_ERR_ARG, "dg_partition_elements: NULL gid");
  std::copy(part->own[p].begin(), part->own[p].end(), gid);
  return DG_OK;
}

extern "C" dg_status dg_partition_ghosts(const dg_partition* part, int32_t p, int64_t* gid) {
  dgw::clear_error();
  dg_status st = check_part(part, p, "dg_partition_ghosts");
  if (st) return st;
  if (!gid) return fail(DG_ERR_ARG, "dg_partition_ghosts: NULL gid");
  std::copy(part->ghost[p].begin(), part->ghost[p].end(), gid);
  return DG_OK;
}

extern "C" dg_status dg_partition_conn(const dg_partition* part, int32_t p, int32_t* conn) {
  dgw::clear_error();
  dg_status st = check_part(part, p, "dg_partition_conn");
  if (st) return st;
  if (!conn) return fail(DG_ERR_ARG, "dg_partition_conn: NULL conn");
  std::copy(part->conn[p].begin(), part->conn[p].end(), conn);
  return DG_OK;
}

extern "C" dg_status dg_partition_exchange_plan(const dg_partition* part, int32_t p,
                                                int32_t* send_peer, int64_t* send_count,
                                                int32_t* send_off, int32_t* recv_peer,
                                                int64_t* recv_count, int32_t* recv_off) {
  dgw::clear_error();
  dg_status st = check_part(part, p, "dg_partition_exchange_plan");
  if (st) return st;
  int64_t si = 0, so = 0, ri = 0, ro = 0;
  for (const Pair& pr : part->pairs) {  // (src, dst) order: peers ascending
    if (pr.src != p) continue;
    if (send_peer) send_peer[si] = pr.dst;
    if (send_count) send_count[si] = static_cast<int64_t>(pr.src_off.size());
    if (send_off) std::copy(pr.src_off.begin(), pr.src_off.end(), send_off + so);
    ++si;
    so += static_cast<int64_t>(pr.src_off.size());
  }
  for (const Pair& pr : part->pairs) {
    if (pr.dst != p) continue;
    if (recv_peer) recv_peer[ri] = pr.src;
    if (recv_count) recv_count[ri] = static_cast<int64_t>(pr.dst_off.size());
    if (recv_off) std::copy(pr.dst_off.begin(), pr.dst_off.end(), recv_off + ro);
    ++ri;
    ro += static_cast<int64_t>(pr.dst_off.size());
  }
  return DG_OK;
}

namespace {

dg_status transfer(dg_partition* part, void* q, int64_t q_stride, void* stream, bool to_part,
                   const char* where) {
  dgw::clear_error();
  dg_status st = check_device_part(part, where);
  if (st) return st;
  if (!q) return fail(DG_ERR_ARG, "%s: NULL fields", where);
  if (q_stride < part->op->K * part->op->Np)
    return fail(DG_ERR_ARG, "%s: field stride %lld < K * Np = %lld", where,
                static_cast<long long>(q_stride),
                static_cast<long long>(part->op->K * part->op->Np));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return part->op->precision == DG_FP32
             ? copy_fields<float>(*part, static_cast<float*>(q), q_stride, to_part, s, where)
             : copy_fields<double>(*part, static_cast<double*>(q), q_stride, to_part, s, where);
}

}  // namespace

extern "C" dg_status dg_partition_set_fields(dg_partition* part, const void* q, int64_t q_stride,
                                             void* stream) {
  // read only: the copy runs global -> part
  return transfer(part, const_cast<void*>(q), q_stride, stream, true, "dg_partition_set_fields");
}

extern "C" dg_status dg_partition_get_fields(dg_partition* part, void* q, int64_t q_stride,
                                             void* stream) {
  return transfer(part, q, q_stride, stream, false, "dg_partition_get_fields");
}

extern "C" dg_status dg_partition_exchange(dg_partition* part, void* stream) {
  dgw::clear_error();
  dg_status st = check_device_part(part, "dg_partition_exchange");
  if (st) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const cudaError_t err = part->op->precision == DG_FP32 ? exchange<float>(*part, s)
                                                         : exchange<double>(*part, s);
  if (err != cudaSuccess) return cuda_fail(err, "dg_partition_exchange");
  return DG_OK;
}

extern "C" dg_status dg_partition_step(dg_partition* part, double dt, int32_t nsteps,
                                       void* stream) {
  dgw::clear_error();
  const char* where = "dg_partition_step";
  dg_status st = check_device_part(part, where);
  if (st) return st;
  if (nsteps < 0) return fail(DG_ERR_ARG, "%s: nsteps = %d < 0", where, nsteps);
  if (!std::isfinite(dt)) return fail(DG_ERR_ARG, "%s: dt is not finite", where);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool fp32 = part->op->precision == DG_FP32;
  // per stage: the exchange on `stream`, then every part's stage launch on
  // its own stream once the exchange is done, and `stream` waits for them all
  for (int32_t n = 0; n < nsteps; ++n) {
    for (int i = 0; i < 5; ++i) {
      cudaError_t err = fp32 ? exchange<float>(*part, s) : exchange<double>(*part, s);
      if (err == cudaSuccess) err = cudaEventRecord(part->exchanged, s);
      if (err != cudaSuccess) return cuda_fail(err, "dg_partition_step: exchange");
      for (int p = 0; p < part->P; ++p) {
        dg_op* sub = part->sub[p];
        cudaStream_t ps = part->streams[p];
        void* qin = part->cur ? sub->d_qtmp : part->d_q[p];
        void* qout = part->cur ? part->d_q[p] : sub->d_qtmp;
        err = cudaStreamWaitEvent(ps, part->exchanged, 0);
        if (err == cudaSuccess) err = dgw::op_stage(sub, qin, qout, part->d_res[p], i, dt, ps);
        if (err == cudaSuccess) err = cudaEventRecord(part->part_done[p], ps);
        if (err == cudaSuccess) err = cudaStreamWaitEvent(s, part->part_done[p], 0);
        if (err != cudaSuccess) return cuda_fail(err, "dg_partition_step: stage launch");
        sub->launches.fetch_add(1, std::memory_order_relaxed);
      }
      part->cur ^= 1;
    }
  }
  return DG_OK;
}

extern "C" dg_status dg_partition_sync_check(dg_partition* part, void* stream) {
  dgw::clear_error();
  dg_status st = check_device_part(part, "dg_partition_sync_check");
  if (st) return st;
  for (dg_op* sub : part->sub)
    if ((st = dg_sync_check(sub, stream))) return st;
  return DG_OK;
}
