// Per-context kernel tracing (crl_trace_start / crl_trace_stop): CUDA events
// around every launch of one kernel class, plus its algorithmic work.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

namespace crl {

// A named NVTX range on the host timeline of a profiler (nsys shows the
// kernels each range launched); without an attached tool a push / pop pair
// costs a few nanoseconds.
class NvtxRange {
 public:
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// NVTX names of the kernel classes CRL_TRACE_INSERT .. CRL_TRACE_AUX (index 0 unused).
inline const char* trace_class_name(int cls) {
  static const char* const names[] = {"crl", "insert", "relabel", "gemm", "energy", "adam", "aux"};
  return (cls >= 0 && cls <= 6) ? names[cls] : "crl";
}

struct Tracer {
  int cls = 0;
  int cap = 0;
  int n = 0;
  cudaEvent_t* ev = nullptr;  // 2 * cap events
  double work = 0.0;
};

// Set by each C-ABI entry point of a context for the duration of the call.
extern thread_local Tracer* g_tracer;

// RAII bracket around one launch of class `cls` with `work` algorithmic units
// (also an NVTX range named for the class).
class TraceLaunch {
 public:
  TraceLaunch(int cls, cudaStream_t st, double work) : nvtx_(trace_class_name(cls)), st_(st) {
    Tracer* t = g_tracer;
    if (t && t->cls == cls && t->n < t->cap) {
      t_ = t;
      cudaEventRecord(t->ev[2 * t->n], st);
      t->work += work;
    }
  }
  ~TraceLaunch() {
    if (t_) {
      cudaEventRecord(t_->ev[2 * t_->n + 1], st_);
      t_->n += 1;
    }
  }
  TraceLaunch(const TraceLaunch&) = delete;
  TraceLaunch& operator=(const TraceLaunch&) = delete;

 private:
  NvtxRange nvtx_;
  Tracer* t_ = nullptr;
  cudaStream_t st_;
};

}  // namespace crl
