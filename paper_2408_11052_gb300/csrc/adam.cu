// Adam update for the CRL networks (Kingma & Ba, 2015; bias-corrected, no
// weight decay).  arXiv 2408.11052 App. B.3 gives the learning rates (critic
// 3e-4, policy 6e-4) without naming the optimiser; Adam is the reading taken.
//
// The step number t is read from device memory (so the update can be replayed
// inside a CUDA graph while the counter advances) or passed by value.
#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "trace.h"

namespace crl {

namespace {

template <typename T>
__global__ void __launch_bounds__(256) adam_kernel(T* __restrict__ p, const T* __restrict__ g, T* __restrict__ m,
                                                  T* __restrict__ v, long long n, const int* __restrict__ t_dev,
                                                  int t_host, float lr, float b1, float b2, float eps) {
  pdl_enter();
  // Bias corrections in double (1 - b^t loses most of its digits in float for
  // small t), computed once per block.
  __shared__ double s_corr[2];
  if (threadIdx.x == 0) {
    const int t = t_dev ? *t_dev : t_host;
    s_corr[0] = (double)lr / (1.0 - pow((double)b1, (double)t));
    s_corr[1] = 1.0 / (1.0 - pow((double)b2, (double)t));
  }
  __syncthreads();
  const T step = T(s_corr[0]);
  const T ibc2 = T(s_corr[1]);
  const T tb1 = T(b1), tb2 = T(b2), one = T(1);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const T gi = g[i];
    const T mi = tb1 * m[i] + (one - tb1) * gi;
    const T vi = tb2 * v[i] + (one - tb2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= step * mi / (dev_sqrt(vi * ibc2) + T(eps));
  }
}

}  // namespace

template <typename T>
void adam_update(T* p, const T* g, T* m, T* v, int64_t n, const int* t_dev, int t_host, float lr, float b1, float b2,
                 float eps, cudaStream_t st) {
  if (n <= 0) return;
  const int blocks = (int)std::min<int64_t>(ceil_div(n, 256), 152 * 8);
  TraceLaunch tr(CRL_TRACE_ADAM, st, 7.0 * sizeof(T) * n);  // read p, g, m, v; write p, m, v
  launch_k(adam_kernel<T>, dim3(blocks), dim3(256), 0, st, p, g, m, v, n, t_dev, t_host, lr, b1, b2, eps);
}

template void adam_update<float>(float*, const float*, float*, float*, int64_t, const int*, int, float, float, float,
                                 float, cudaStream_t);
template void adam_update<double>(double*, const double*, double*, double*, int64_t, const int*, int, float, float,
                                  float, float, cudaStream_t);

}  // namespace crl
