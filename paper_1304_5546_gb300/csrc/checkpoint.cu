// Checkpoint and resume of a solve (dg_checkpoint_save / dg_checkpoint_load).
//
// The state of a time-stepping solve between steps is the three fields, the
// time and the step count: the LSRK(5,4) residual needs no saving, because
// the first stage of a step overwrites it (a_1 = 0).  A checkpoint file is a
// fixed header followed by the K * Np values of each field in the
// operator's precision, without the padding of a device field buffer.  The
// header records the operator (order, K, precision, medium) and an FNV-1a
// hash of its node coordinates and permittivities, so that a checkpoint is
// never loaded into a different mesh, and an FNV-1a hash of the field
// bytes, so that a damaged file is refused.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

using dgw::fail;

namespace {

constexpr char kMagic[8] = {'D', 'G', 'W', 'C', 'K', 'P', 'T', '1'};
constexpr uint32_t kVersion = 1;

struct Header {
  char magic[8];
  uint32_t version;
  int32_t N;
  int64_t K;
  int32_t Np;
  int32_t precision;
  int32_t media;
  int32_t pad;
  double t;
  int64_t step;
  uint64_t mesh_hash;
  uint64_t data_hash;
  int64_t data_bytes;
};

uint64_t fnv1a(const void* data, size_t n, uint64_t h = 1469598103934665603ull) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

uint64_t mesh_hash(const dg_op* op) {
  uint64_t h = fnv1a(op->geo.x.data(), op->geo.x.size() * sizeof(double));
  h = fnv1a(op->geo.y.data(), op->geo.y.size() * sizeof(double), h);
  if (op->media()) h = fnv1a(op->eps.data(), op->eps.size() * sizeof(double), h);
  return h;
}

// fields of q (3 rows of K Np values at a stride of q_stride values) to or
// from the compact host array `buf`
dg_status copy_fields(const dg_op* op, void* q, int64_t q_stride, bool on_host,
                      std::vector<unsigned char>& buf, bool to_buf, const char* where) {
  const size_t row = static_cast<size_t>(op->K) * op->Np * op->elem_size;
  const size_t pitch = static_cast<size_t>(q_stride) * op->elem_size;
  if (on_host) {
    for (int f = 0; f < 3; ++f) {
      unsigned char* qf = static_cast<unsigned char*>(q) + f * pitch;
      if (to_buf)
        std::memcpy(buf.data() + f * row, qf, row);
      else
        std::memcpy(qf, buf.data() + f * row, row);
    }
    return DG_OK;
  }
  cudaError_t err = cudaSetDevice(op->device);
  if (err == cudaSuccess)
    err = to_buf ? cudaMemcpy2D(buf.data(), row, q, pitch, row, 3, cudaMemcpyDeviceToHost)
                 : cudaMemcpy2D(q, pitch, buf.data(), row, row, 3, cudaMemcpyHostToDevice);
  if (err != cudaSuccess)
    return fail(DG_ERR_CUDA, "%s: %s (%s)", where, cudaGetErrorName(err), cudaGetErrorString(err));
  return DG_OK;
}

dg_status check_args(const dg_op* op, const void* q, int64_t q_stride, int32_t flags,
                     const char* path, const char* where) {
  if (!op || !q || !path) return fail(DG_ERR_ARG, "%s: NULL argument", where);
  if (flags & ~DG_CKPT_HOST) return fail(DG_ERR_ARG, "%s: unknown flags 0x%x", where, flags);
  if (q_stride < op->K * op->Np)
    return fail(DG_ERR_ARG, "%s: field stride %lld < K * Np = %lld", where,
                static_cast<long long>(q_stride), static_cast<long long>(op->K * op->Np));
  if (!(flags & DG_CKPT_HOST) && !op->has_device)
    return fail(DG_ERR_NO_DEVICE, "%s: device fields with a host-only operator", where);
  return DG_OK;
}

}  // namespace

extern "C" dg_status dg_checkpoint_save(const dg_op* op, const void* q, int64_t q_stride,
                                        int32_t flags, double t, int64_t step, const char* path) {
  dgw::clear_error();
  const char* where = "dg_checkpoint_save";
  dg_status st = check_args(op, q, q_stride, flags, path, where);
  if (st) return st;
  std::vector<unsigned char> buf;
  try {
    buf.resize(3 * static_cast<size_t>(op->K) * op->Np * op->elem_size);
  } catch (const std::bad_alloc&) {
    return fail(DG_ERR_OOM, "%s: out of host memory", where);
  }
  if ((st = copy_fields(op, const_cast<void*>(q), q_stride, flags & DG_CKPT_HOST, buf, true, where)))
    return st;
  Header h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, kMagic, 8);
  h.version = kVersion;
  h.N = op->N;
  h.K = op->K;
  h.Np = op->Np;
  h.precision = op->precision;
  h.media = op->media() ? 1 : 0;
  h.t = t;
  h.step = step;
  h.mesh_hash = mesh_hash(op);
  h.data_hash = fnv1a(buf.data(), buf.size());
  h.data_bytes = static_cast<int64_t>(buf.size());
  // write to a temporary name, then rename: a crash leaves the old file
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) return fail(DG_ERR_IO, "%s: cannot open %s for writing", where, tmp.c_str());
  const bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1 &&
                  std::fwrite(buf.data(), 1, buf.size(), f) == buf.size();
  const bool closed = std::fclose(f) == 0;
  if (!ok || !closed) {
    std::remove(tmp.c_str());
    return fail(DG_ERR_IO, "%s: writing %s failed", where, tmp.c_str());
  }
  if (std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return fail(DG_ERR_IO, "%s: cannot rename %s to %s", where, tmp.c_str(), path);
  }
  return DG_OK;
}

extern "C" dg_status dg_checkpoint_load(const dg_op* op, const char* path, void* q,
                                        int64_t q_stride, int32_t flags, double* t,
                                        int64_t* step) {
  dgw::clear_error();
  const char* where = "dg_checkpoint_load";
  dg_status st = check_args(op, q, q_stride, flags, path, where);
  if (st) return st;
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(DG_ERR_IO, "%s: cannot open %s", where, path);
  Header h;
  if (std::fread(&h, sizeof(h), 1, f) != 1) {
    std::fclose(f);
    return fail(DG_ERR_IO, "%s: %s is too short for a header", where, path);
  }
  const size_t want = 3 * static_cast<size_t>(op->K) * op->Np * op->elem_size;
  const char* bad = nullptr;
  if (std::memcmp(h.magic, kMagic, 8) != 0 || h.version != kVersion)
    bad = "not a checkpoint of this format";
  else if (h.N != op->N || h.K != op->K || h.Np != op->Np || h.precision != op->precision ||
           h.media != (op->media() ? 1 : 0))
    bad = "written for another operator (order, size, precision or medium)";
  else if (h.data_bytes != static_cast<int64_t>(want))
    bad = "field size does not match";
  else if (h.mesh_hash != mesh_hash(op))
    bad = "written for another mesh";
  if (bad) {
    std::fclose(f);
    return fail(DG_ERR_ARG, "%s: %s: %s", where, path, bad);
  }
  std::vector<unsigned char> buf;
  try {
    buf.resize(want);
  } catch (const std::bad_alloc&) {
    std::fclose(f);
    return fail(DG_ERR_OOM, "%s: out of host memory", where);
  }
  const bool ok = std::fread(buf.data(), 1, want, f) == want;
  std::fclose(f);
  if (!ok) return fail(DG_ERR_IO, "%s: %s is truncated", where, path);
  if (fnv1a(buf.data(), buf.size()) != h.data_hash)
    return fail(DG_ERR_ARG, "%s: %s: field data damaged (hash mismatch)", where, path);
  if ((st = copy_fields(op, q, q_stride, flags & DG_CKPT_HOST, buf, false, where))) return st;
  if (t) *t = h.t;
  if (step) *step = h.step;
  return DG_OK;
}
