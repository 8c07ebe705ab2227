// Tiled SIMT GEMM for the FP32 and FP64 paths (CUDA cores, no tensor cores).
//
//   C(m, n) = epilogue(m, n, sum_k op(A(m, k), B(k, n)))
//
// A and B are read through small loader functors, so one kernel serves
// x W^T (forward), dY W (input gradient), dY^T X (weight gradient) and the
// energy matrices (op = product, squared difference or absolute difference).
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

// Tile BM x BN (64 x 64 or 32 x 32), 32-deep k slices, 256 threads, each
// thread TM x TN outputs strided by 16 rows / columns (conflict-free shared
// reads).  The next slice is prefetched into registers while the current one
// is multiplied out of the other shared-memory buffer, so each slice costs one
// barrier and the global-load latency overlaps the arithmetic.
template <typename T, InnerOp OP, int BM, int BN, class LA, class LB, class EP>
__global__ void __launch_bounds__(256) gemm_tile_kernel(int M, int N, int K, LA la, LB lb, EP ep) {
  pdl_enter();
  constexpr int BK = 32;
  constexpr int TM = BM / 16, TN = BN / 16;
  constexpr int LDA = BM * BK / 256, LDB = BN * BK / 256;  // elements each thread loads per slice
  __shared__ T As[2][BK][BM + 1];
  __shared__ T Bs[2][BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

  T ra[LDA], rb[LDB];
  auto load = [&](int k0) {
#pragma unroll
    for (int r = 0; r < LDA; ++r) {
      const int e = tid + r * 256;
      int mm, kk;
      if constexpr (LA::kContigK) { kk = e % BK; mm = e / BK; }
      else { mm = e % BM; kk = e / BM; }
      const int m = m0 + mm, k = k0 + kk;
      ra[r] = (m < M && k < K) ? la(m, k) : T(0);
    }
#pragma unroll
    for (int r = 0; r < LDB; ++r) {
      const int e = tid + r * 256;
      int nn, kk;
      if constexpr (LB::kContigK) { kk = e % BK; nn = e / BK; }
      else { nn = e % BN; kk = e / BN; }
      const int n = n0 + nn, k = k0 + kk;
      rb[r] = (n < N && k < K) ? lb(k, n) : T(0);
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int r = 0; r < LDA; ++r) {
      const int e = tid + r * 256;
      int mm, kk;
      if constexpr (LA::kContigK) { kk = e % BK; mm = e / BK; }
      else { mm = e % BM; kk = e / BM; }
      As[buf][kk][mm] = ra[r];
    }
#pragma unroll
    for (int r = 0; r < LDB; ++r) {
      const int e = tid + r * 256;
      int nn, kk;
      if constexpr (LB::kContigK) { kk = e % BK; nn = e / BK; }
      else { nn = e % BN; kk = e / BN; }
      Bs[buf][kk][nn] = rb[r];
    }
  };

  load(0);
  store(0);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < K; k0 += BK) {
    const bool more = k0 + BK < K;
    if (more) load(k0 + BK);
    // Padded k entries are zero on both sides, so they add 0 for every inner op.
#pragma unroll 8
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[buf][kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[buf][kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] += inner<T, OP>(a[i], b[j]);
    }
    if (more) store(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
      if (m < M && n < N) ep(m, n, acc[i][j]);
    }
}

// Launch; traced as class `cls` (CRL_TRACE_*) with 2 M N K flops of work.  The
// 32 x 32 tile is used when 64 x 64 tiles would leave most of the 152 SMs idle.
template <typename T, InnerOp OP = InnerOp::kMul, class LA, class LB, class EP>
void gemm(int M, int N, int K, const LA& la, const LB& lb, const EP& ep, cudaStream_t st, int cls = CRL_TRACE_GEMM) {
  if (M <= 0 || N <= 0) return;
  TraceLaunch tr(cls, st, 2.0 * M * N * K);
  const long long tiles64 = (long long)ceil_div(N, 64) * ceil_div(M, 64);
  // FP64 always takes the 32 x 32 tile: its 64 x 64 double buffers exceed 48 KiB of static shared memory.
  if (sizeof(T) == 8 || tiles64 < 2 * 152) {
    dim3 grid(ceil_div(N, 32), ceil_div(M, 32));
    launch_k(gemm_tile_kernel<T, OP, 32, 32, LA, LB, EP>, dim3(grid), dim3(256), 0, st, M, N, K, la, lb, ep);
  } else if constexpr (sizeof(T) == 4) {
    dim3 grid(ceil_div(N, 64), ceil_div(M, 64));
    launch_k(gemm_tile_kernel<T, OP, 64, 64, LA, LB, EP>, dim3(grid), dim3(256), 0, st, M, N, K, la, lb, ep);
  }
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
