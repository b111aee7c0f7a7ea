// Pinned host staging buffers for asynchronous host-to-device and
// device-to-host copies (batches and the solve server).  Private to the
// library.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

namespace dgw {

// Pinned host buffers for asynchronous uploads; a buffer is reused once the
// event recorded after its copies has completed.
class Staging {
 public:
  ~Staging() { release(); }
  void* get(size_t bytes, size_t* idx) {
    for (size_t i = 0; i < bufs_.size(); ++i) {
      Buf& b = bufs_[i];
      if (b.busy && cudaEventQuery(b.ev) == cudaSuccess) b.busy = false;
      if (!b.busy && !b.held && b.cap >= bytes) {
        *idx = i;
        return b.p;
      }
    }
    Buf b;
    b.cap = std::max<size_t>(bytes, 1 << 16);
    if (cudaMallocHost(&b.p, b.cap) != cudaSuccess) return nullptr;
    if (cudaEventCreateWithFlags(&b.ev, cudaEventDisableTiming) != cudaSuccess) {
      cudaFreeHost(b.p);
      return nullptr;
    }
    bufs_.push_back(b);
    *idx = bufs_.size() - 1;
    return b.p;
  }
  // the copies from buffer idx are enqueued on `s`
  cudaError_t mark(size_t idx, cudaStream_t s) {
    bufs_[idx].busy = true;
    return cudaEventRecord(bufs_[idx].ev, s);
  }
  // a held buffer is not handed out again until unhold(), whatever its
  // event says (its contents are still to be read on the host)
  void hold(size_t idx) { bufs_[idx].held = true; }
  void unhold(size_t idx) { bufs_[idx].held = false; }
  // the event recorded by the last mark() of buffer idx
  cudaEvent_t event(size_t idx) const { return bufs_[idx].ev; }
  void* ptr(size_t idx) const { return bufs_[idx].p; }
  void release() {
    for (Buf& b : bufs_) {
      if (b.busy) cudaEventSynchronize(b.ev);
      cudaEventDestroy(b.ev);
      cudaFreeHost(b.p);
    }
    bufs_.clear();
  }

 private:
  struct Buf {
    void* p = nullptr;
    size_t cap = 0;
    cudaEvent_t ev = nullptr;
    bool busy = false;
    bool held = false;
  };
  std::vector<Buf> bufs_;
};

}  // namespace dgw
