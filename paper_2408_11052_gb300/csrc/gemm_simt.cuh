// Tiled SIMT GEMM for the FP32 and FP64 paths (CUDA cores, no tensor cores).
//
//   C(m, n) = epilogue(m, n, sum_k op(A(m, k), B(k, n)))
//
// A and B are read through small loader functors, so one kernel serves
// x W^T (forward), dY W (input gradient), dY^T X (weight gradient) and the
// energy matrices (op = product, squared difference or absolute difference).
// 64 x 64 output tile, 16-deep k slices staged in shared memory, 256 threads,
// 4 x 4 outputs per thread strided by 16 so that shared-memory reads are
// conflict free.
#pragma once

#include "common.cuh"
#include "internal.h"
#include "trace.h"

namespace crl {

enum class InnerOp { kMul, kSqDiff, kAbsDiff };

template <typename T, InnerOp OP>
__device__ __forceinline__ T inner(T a, T b) {
  if constexpr (OP == InnerOp::kMul) return a * b;
  else if constexpr (OP == InnerOp::kSqDiff) { const T d = a - b; return d * d; }
  else return fabs(a - b);
}

template <typename T, InnerOp OP, class LA, class LB, class EP>
__global__ void __launch_bounds__(256) gemm_tile_kernel(int M, int N, int K, LA la, LB lb, EP ep) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

  for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = tid + r * 256;
      int mm, kk;
      if constexpr (LA::kContigK) { kk = e % BK; mm = e / BK; }
      else { mm = e % BM; kk = e / BM; }
      const int m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < M && k < K) ? la(m, k) : T(0);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = tid + r * 256;
      int nn, kk;
      if constexpr (LB::kContigK) { kk = e % BK; nn = e / BK; }
      else { nn = e % BN; kk = e / BN; }
      const int n = n0 + nn, k = k0 + kk;
      Bs[kk][nn] = (n < N && k < K) ? lb(k, n) : T(0);
    }
    __syncthreads();
    // Padded k entries are zero on both sides, so they add 0 for every inner op.
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += inner<T, OP>(a[i], b[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
      if (m < M && n < N) ep(m, n, acc[i][j]);
    }
}

// Launch; traced as class `cls` (CRL_TRACE_*) with 2 M N K flops of work.
template <typename T, InnerOp OP = InnerOp::kMul, class LA, class LB, class EP>
void gemm(int M, int N, int K, const LA& la, const LB& lb, const EP& ep, cudaStream_t st, int cls = CRL_TRACE_GEMM) {
  if (M <= 0 || N <= 0) return;
  TraceLaunch tr(cls, st, 2.0 * M * N * K);
  dim3 grid(ceil_div(N, 64), ceil_div(M, 64));
  gemm_tile_kernel<T, OP, LA, LB, EP><<<grid, 256, 0, st>>>(M, N, K, la, lb, ep);
}

// ---- loaders ---------------------------------------------------------------
// A(m, k) = concat(x0[m][0:split], x1[m][0:K-split])[k]  (row-major, k contiguous)
template <typename T, typename T0, typename T1>
struct LoadRowsSplit {
  static constexpr bool kContigK = true;
  const T0* p0;
  const T1* p1;
  int ld0, ld1, split;
  __device__ T operator()(int m, int k) const {
    return k < split ? T(p0[(size_t)m * ld0 + k]) : T(p1[(size_t)m * ld1 + (k - split)]);
  }
};
// B(k, n) = X[k][n] split by columns (row-major X, n contiguous): weight gradient dY^T X.
template <typename T, typename T0, typename T1>
struct LoadColsSplit {
  static constexpr bool kContigK = false;
  const T0* p0;
  const T1* p1;
  int ld0, ld1, split;
  __device__ T operator()(int k, int n) const {
    return n < split ? T(p0[(size_t)k * ld0 + n]) : T(p1[(size_t)k * ld1 + (n - split)]);
  }
};
// B(k, n) = W[n][k]: the weight of x W^T (k contiguous).
template <typename T>
struct LoadNK {
  static constexpr bool kContigK = true;
  const T* p;
  int ld;
  __device__ T operator()(int k, int n) const { return p[(size_t)n * ld + k]; }
};
// B(k, n) = W[k][n] (n contiguous).
template <typename T>
struct LoadKN {
  static constexpr bool kContigK = false;
  const T* p;
  int ld;
  __device__ T operator()(int k, int n) const { return p[(size_t)k * ld + n]; }
};
// A(m, k) = X[k][m]: the transposed operand of dY^T X (m contiguous).
template <typename T>
struct LoadTrans {
  static constexpr bool kContigK = false;
  const T* p;
  int ld;
  __device__ T operator()(int m, int k) const { return p[(size_t)k * ld + m]; }
};
// A(m, k) = X[m][k] (k contiguous).
template <typename T>
struct LoadMK {
  static constexpr bool kContigK = true;
  const T* p;
  int ld;
  __device__ T operator()(int m, int k) const { return p[(size_t)m * ld + k]; }
};

// ---- epilogues -------------------------------------------------------------
// C = act(acc + bias[n])
template <typename T>
struct EpiBias {
  T* C;
  int ldc;
  const T* bias;
  int relu;
  __device__ void operator()(int m, int n, T acc) const {
    T v = acc + (bias ? bias[n] : T(0));
    if (relu) v = v > T(0) ? v : T(0);
    C[(size_t)m * ldc + n] = v;
  }
};
// C = alpha * acc
template <typename T>
struct EpiScale {
  T* C;
  int ldc;
  T alpha;
  __device__ void operator()(int m, int n, T acc) const { C[(size_t)m * ldc + n] = alpha * acc; }
};
// v = acc * [mask[m][n] > 0]; written to c0 (n < split) or c1 (n >= split), either may be null.
template <typename T>
struct EpiMaskSplit {
  T* c0;
  T* c1;
  int ld0, ld1, split;
  const T* mask;
  int ldm;
  __device__ void operator()(int m, int n, T acc) const {
    T v = acc;
    if (mask && !(mask[(size_t)m * ldm + n] > T(0))) v = T(0);
    if (n < split) {
      if (c0) c0[(size_t)m * ld0 + n] = v;
    } else if (c1) {
      c1[(size_t)m * ld1 + (n - split)] = v;
    }
  }
};
// C = alpha * acc - s[m] * X[m][n]
template <typename T>
struct EpiSubRowScaled {
  T* C;
  int ldc;
  T alpha;
  const T* s;
  const T* X;
  int ldx;
  __device__ void operator()(int m, int n, T acc) const {
    C[(size_t)m * ldc + n] = alpha * acc - s[m] * X[(size_t)m * ldx + n];
  }
};

}  // namespace crl
