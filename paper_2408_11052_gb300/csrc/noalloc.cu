// crl_infonce_forward_noalloc: the critic-loss forward without a caller-supplied
// workspace and without any device allocation.
//
// Who needs this: code that must not allocate device memory at the moment it
// evaluates the loss.  Examples are a host that fixes its device memory
// budget at start-up and forbids allocation afterwards (long-running or
// real-time loops, where cudaMalloc can stall on a device-wide
// synchronisation and fragments memory), and a plugin running inside a
// runtime that owns the device allocator (its pools and accounting would not
// see a cudaMalloc of ours).  Those callers still pass their inputs and
// outputs; the scratch lives here.
//
// The scratch is one fixed array in the library's device memory,
// kNoAllocScratchBytes long.  Every GPU that loads the library holds it until
// the process exits.  All calls share it: calls whose work overlaps on the GPU
// (different streams, or different host threads, without ordering between
// them) race on it and give wrong results.  Nothing in it needs to start at
// zero: the forward writes every scratch element before reading it.
//
// Host code cannot use the array's name as a device address (in host code it
// is a host-side stand-in), so the address is looked up with
// cudaGetSymbolAddress once per device, on that device's first call, and
// cached.  cudaDeviceReset destroys the array with the context; the cached
// address is then stale, so this entry point must not be used on a device
// after it has been reset.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "ctx.h"
#include "internal.h"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(4) << 20;  // 4 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch on the current device (one-time set-up per device).
int scratch_address(void** out, std::string* err) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    *err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    return CRL_E_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    *err = "device ordinal outside the 64 devices the allocation-free entry point supports";
    return CRL_E_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_scratch_addr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      *err = std::string("cudaGetSymbolAddress of the allocation-free scratch: ") + cudaGetErrorString(e);
      return CRL_E_CUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return CRL_OK;
}

}  // namespace

extern "C" int crl_infonce_forward_noalloc(const crl_loss_desc* d, const void* phi, const void* psi, int32_t B,
                                           int32_t R, void* loss4, void* row_lse, void* col_lse, void* stream) {
  using namespace crl;
  return guarded(nullptr, [&] {
    // the same descriptor checks and error codes as crl_infonce_forward
    const LossSpec ls = checked_loss(d);
    CRL_REQUIRE(phi && psi && loss4 && row_lse && col_lse && B >= 1 && R >= 1, CRL_E_INVALID_ARG, "bad argument");
    CRL_REQUIRE(ls.loss != CRL_LOSS_FB || B >= 2, CRL_E_SHAPE, "the forward-backward objective needs B >= 2");
    CRL_REQUIRE((d->dtype == CRL_PREC_FP32 || d->dtype == CRL_PREC_FP64) && d->path == CRL_PATH_PLAIN,
                CRL_E_UNSUPPORTED, "the allocation-free forward takes dtype FP32 or FP64 and path PLAIN");
    const size_t elem = d->dtype == CRL_PREC_FP64 ? sizeof(double) : sizeof(float);
    const size_t need = infonce_ws_bytes(ls, B, R, elem, d->path);
    CRL_REQUIRE(need <= kNoAllocScratchBytes, CRL_E_SHAPE,
                "batch " + std::to_string(B) + " x repr " + std::to_string(R) + " needs " + std::to_string(need) +
                    " bytes of scratch, above the fixed 4 MiB (4194304 bytes) of the allocation-free forward");
    void* ws = nullptr;
    std::string err;
    const int rc = scratch_address(&ws, &err);
    CRL_REQUIRE(rc == CRL_OK, rc, err);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (d->dtype == CRL_PREC_FP64)
      infonce_forward<double>(ls, static_cast<const double*>(phi), static_cast<const double*>(psi), B, R,
                              static_cast<double*>(loss4), static_cast<double*>(row_lse),
                              static_cast<double*>(col_lse), ws, d->path, nullptr, nullptr, st);
    else
      infonce_forward<float>(ls, static_cast<const float*>(phi), static_cast<const float*>(psi), B, R,
                             static_cast<float*>(loss4), static_cast<float*>(row_lse), static_cast<float*>(col_lse),
                             ws, d->path, nullptr, nullptr, st);
    check_launch("allocation-free infonce forward");
  });
}
