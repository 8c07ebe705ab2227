// Device helpers shared by the libcrl kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <utility>

namespace crl {

constexpr int kWarp = 32;

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum for blockDim.x a multiple of 32 (<= 1024).  Every thread gets the result.
template <typename T>
__device__ T block_sum(T v, T* smem /* >= 32 */) {
  const int lane = threadIdx.x % kWarp, wid = threadIdx.x / kWarp;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) smem[wid] = v;
  __syncthreads();
  const int nw = (blockDim.x + kWarp - 1) / kWarp;
  T r = (threadIdx.x < nw) ? smem[threadIdx.x] : T(0);
  if (wid == 0) r = warp_sum(r);
  if (threadIdx.x == 0) smem[0] = r;
  __syncthreads();
  r = smem[0];
  __syncthreads();
  return r;
}

__device__ __forceinline__ bool finite_val(float x) { return isfinite(x); }
__device__ __forceinline__ bool finite_val(double x) { return isfinite(x); }

__device__ __forceinline__ float dev_exp(float x) { return expf(x); }
__device__ __forceinline__ double dev_exp(double x) { return exp(x); }
__device__ __forceinline__ float dev_log(float x) { return logf(x); }
__device__ __forceinline__ double dev_log(double x) { return log(x); }
__device__ __forceinline__ float dev_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double dev_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float dev_tanh(float x) { return tanhf(x); }
__device__ __forceinline__ double dev_tanh(double x) { return tanh(x); }
__device__ __forceinline__ float dev_log1p(float x) { return log1pf(x); }
__device__ __forceinline__ double dev_log1p(double x) { return log1p(x); }

// softplus(x) = log(1 + e^x), overflow-free.
template <typename T>
__device__ __forceinline__ T softplus(T x) {
  return fmax(x, T(0)) + dev_log1p(dev_exp(-fabs(x)));
}

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }
inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// ---- multi-agent launches -------------------------------------------------------
// A launch over several independent problems (agents, networks) gives problem s
// the blocks [begin[s], begin[s + 1]) of a 1-D grid (begin: n + 1 entries).
// Returns s; lb = block index within the problem, nb = its block count.
__device__ __forceinline__ int segment_of(const int* __restrict__ begin, int n, int b, int& lb, int& nb) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (begin[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  lb = b - begin[lo];
  nb = begin[lo + 1] - begin[lo];
  return lo;
}

// ---- programmatic dependent launch ---------------------------------------------
// Every libcrl kernel is launched with programmatic stream serialisation
// allowed (launch_k), so it may start while its predecessor on the stream is
// still running.  Before its first global-memory access every kernel calls
// pdl_wait(), which returns once all prerequisite grids have completed and
// their writes are visible; pdl_trigger() then lets the next kernel of the
// stream be scheduled (it will in turn block in its own pdl_wait).  Kernels
// that allocate tensor memory trigger only after the allocation, so a waiting
// successor never holds TMEM that its predecessor still needs.
// Both instructions are no-ops for a kernel launched without the attribute.
// L2 prefetch of the line holding p (a hint; nothing waits for it).
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<uint64_t>(p)));
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_enter() {
  pdl_wait();
  pdl_trigger();
}

// Process-wide switches: crl_set_launch_overlap (1 = launch with the attribute)
// and crl_set_autotune (1 = grouped GEMMs time their tile widths on first use).
extern int g_launch_overlap;
extern int g_autotune;
extern int g_gemm_kernel;  // CRL_GEMM_*

template <typename... KArgs, typename... Args>
inline void launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                     Args&&... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = g_launch_overlap ? 1 : 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// The same with thread-block clusters of `cluster_x` consecutive blocks.
template <typename... KArgs, typename... Args>
inline void launch_k_cluster(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                             unsigned cluster_x, Args&&... args) {
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = g_launch_overlap ? 1 : 0;
  attr[1].id = cudaLaunchAttributeClusterDimension;
  attr[1].val.clusterDim.x = cluster_x;
  attr[1].val.clusterDim.y = 1;
  attr[1].val.clusterDim.z = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace crl
