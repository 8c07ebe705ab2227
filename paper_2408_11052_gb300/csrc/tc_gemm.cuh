// BF16 tensor-core GEMM on tcgen05 with TMEM accumulators and TMA operand loads:
//
//   C(m, n) = epilogue(m, n, sum_k A[m][k] * B[n][k])      A, B: BF16, K-major
//
// One CTA computes a 128 x BN tile (BN in {64, 128, 256}); 128 threads:
//   warp 0 / lane 0 -- TMA producer: 64-wide K slices of A and B (as 64-row
//                      boxes: every tensor map has box {64, 64}) into a
//                      4-stage shared-memory ring (128-byte swizzle);
//   warp 1 / lane 0 -- MMA issuer: 4 x tcgen05.mma (K = 16 each) per slice
//                      into the FP32 accumulator in TMEM (128 lanes x BN cols);
//   all 4 warps     -- epilogue: warp w reads TMEM lanes 32w..32w+31 (rows)
//                      in chunks of 32 columns and hands them to the functor.
// Out-of-range rows and columns of the operands are zero-filled by TMA; the
// epilogue functor clips its stores to M x N.
#pragma once

#include "common.cuh"
#include "tc_common.cuh"

namespace crl {
namespace tc {

constexpr int kBM = 128;
constexpr int kBK = 64;
constexpr int kStages = 4;

template <int BN>
struct GemmSmem {
  static constexpr uint32_t kABytes = kBM * kBK * 2;   // 16 KiB
  static constexpr uint32_t kBBytes = BN * kBK * 2;    // BN * 128 B
  static constexpr uint32_t kStageBytes = kABytes + kBBytes;
  // operand ring + barriers (full[S], empty[S], done) + TMEM slot, plus 1 KiB for alignment
  static constexpr uint32_t kBytes = kStages * kStageBytes + 1024 + 256;
  static constexpr uint32_t kTmemCols = BN;
  static_assert(BN % 64 == 0 && BN <= 256, "BN must be 64, 128 or 256");
};

// nkA > 0: A has only nkA K-slices and slice kb of B multiplies slice kb % nkA of
// A -- B holds [W_hi | W_lo] along K and each A tile is used against both halves.
template <int BN, class Epi>
__global__ void __launch_bounds__(128, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M, int N,
                   int K, int nkA, Epi epi, unsigned* status) {
  using S = GemmSmem<BN>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align1024(smem_raw);
  uint8_t* sA = smem;
  uint8_t* sB = smem + kStages * S::kABytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * S::kStageBytes);
  uint64_t* empty = full + kStages;
  uint64_t* done = empty + kStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * BN;
  const int nk = (K + kBK - 1) / kBK;

  if (threadIdx.x == 0) {
    prefetch_tmap(&tmA);
    prefetch_tmap(&tmB);
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(tmem_slot, S::kTmemCols);
    tmem_relinquish();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // TMA producer
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % kStages;
      if (kb >= kStages && !mbar_wait(&empty[s], ((kb / kStages) & 1) ^ 1)) {
        atomicOr(status, CRL_STATUS_TIMEOUT);
        break;
      }
      mbar_arrive_expect_tx(&full[s], S::kStageBytes);
      // operands arrive as 64-row boxes (8 KiB each); stacked along rows they
      // form the same 128-byte-swizzled K-major tile as one tall box
      const int ka = nkA > 0 ? kb % nkA : kb;
#pragma unroll
      for (int r = 0; r < kBM / 64; ++r)
        tma_load_2d(sA + s * S::kABytes + r * 8192, &tmA, &full[s], ka * kBK, m0 + 64 * r);
#pragma unroll
      for (int r = 0; r < BN / 64; ++r)
        tma_load_2d(sB + s * S::kBBytes + r * 8192, &tmB, &full[s], kb * kBK, n0 + 64 * r);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    constexpr uint32_t idesc = idesc_bf16_f32(kBM, BN);
    bool ok = true;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % kStages;
      if (!mbar_wait(&full[s], (kb / kStages) & 1)) {
        atomicOr(status, CRL_STATUS_TIMEOUT);
        ok = false;
        break;
      }
      fence_after_sync();
      const uint64_t da = sdesc_kmajor_sw128(sA + s * S::kABytes);
      const uint64_t db = sdesc_kmajor_sw128(sB + s * S::kBBytes);
#pragma unroll
      for (int k = 0; k < kBK / 16; ++k) {
        // +32 bytes along K per 16-element step: +2 in the (addr >> 4) field
        mma_bf16(tmem, da + 2 * k, db + 2 * k, idesc, (kb > 0 || k > 0) ? 1u : 0u);
      }
      mma_commit(&empty[s]);
    }
    if (ok) mma_commit(done);
  }
  __syncwarp();

  // epilogue (tcgen05.ld is warp-collective: keep the decision warp-uniform)
  const bool ok = __all_sync(0xffffffffu, mbar_wait(done, 0) ? 1 : 0) != 0;
  fence_after_sync();
  if (ok) {
    const int row = m0 + warp * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int c = 0; c < BN; c += 32) {
      float v[32];
      tmem_ld32(lane_base + c, v);
      epi(row, n0 + c, v, M, N);
    }
  } else if (threadIdx.x == 0) {
    atomicOr(status, CRL_STATUS_TIMEOUT);
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, S::kTmemCols);
}

}  // namespace tc
}  // namespace crl
