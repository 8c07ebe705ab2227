// Grouped BF16 tensor-core GEMM on tcgen05 with TMEM accumulators and TMA
// operand loads.  One launch runs a list of independent problems
//
//   C_p(m, n) = epilogue_p(m, n, sum_k A_p[m][k] * B_p[n][k])      A, B: BF16, K-major
//
// (the same layer of several networks, or all weight gradients of a network),
// each split into 128 x BN tiles; CTA t finds its problem by a binary search of
// the tiles' prefix sums in the problem table.  The table (tensor maps,
// sizes, epilogue descriptor) lives in device memory and is never written
// while kernels run.
//
// One CTA computes one 128 x BN tile (BN in {64, 128, 256}); 128 threads:
//   warp 0 / lane 0 -- TMA producer: 64-wide K slices of A and B (as 64-row
//                      boxes: every tensor map has box {64, 64}) into a
//                      STAGES-deep shared-memory ring (128-byte swizzle);
//   warp 1 / lane 0 -- MMA issuer: 4 x tcgen05.mma (K = 16 each) per slice
//                      into the FP32 accumulator in TMEM (128 lanes x BN cols);
//   all 4 warps     -- epilogue: warp w reads TMEM lanes 32w..32w+31 (rows)
//                      in chunks of 32 columns and applies the problem's
//                      epilogue (vectorised row stores).
// Either operand may be stored MN-major instead (the weight gradients read the
// activations and output gradients as they are stored: the batch is K).
// Out-of-range rows and columns of the operands are zero-filled by TMA; the
// epilogue clips its stores to M x N.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"
#include "tc_common.cuh"

namespace crl {
namespace tc {

constexpr int kBM = 128;
constexpr int kBK = 64;

// What the FP32 accumulator tile of a problem becomes.
enum EpiKind : int {
  kEpiFwdHidden = 0,  // h = ReLU(acc + b) as BF16 hi / lo parts: h_hi [M][ld0] columns [0, N), h_lo = bf16(h -
                      // h_hi) at columns [c0, c0 + N) of the same rows
  kEpiFwdPreLN = 1,   // z = acc + b: FP32 [M][ld0] (LayerNorm follows)
  kEpiFwdOut = 2,     // y = acc + b: FP32 [M][ld0]
  kEpiBwdDX = 3,      // dz = acc * [mask > 0]: BF16 dz [M][ld0]
  kEpiBwdDXLN = 4,    // du = acc * [mask > 0]: FP32 [M][ld0]
  kEpiBwdDW = 5,      // dW [M][kin] (columns < kin), db [M] (column kin: the ones row)
  kEpiBwdDW0 = 6,     // split first layer: dW[m][c] = acc[2c] + acc[2c+1], db[m] = acc[2 kin]
  kEpiDX0 = 7,        // dx [M][nc] = acc columns [c0, c0 + nc)
  kEpiFwdOutEnergy = 8,  // output layer feeding the fused energy: y = acc + b FP32 [M][ld0], the BF16
                         // energy operand x = y * s [M][N] (out1), aux [M];
                         // s = 1 / |y| and aux = s for the cosine energy, else s = 1 and aux = |bf16(y)|^2.
                         // The tile must span the whole row (the launch picks BN >= N).
};

struct EpiDesc {
  int kind, ld0, ld1, kin, c0, nc, ldm, energy;
  const float* bias;
  const __nv_bfloat16* mask;  // [M][ldm], BF16 post-ReLU activation (> 0 where the unit is active)
  void* out0;
  void* out1;
  void* out2;
  float* aux;
};

struct GemmProblem {   // 128-byte aligned by its tensor maps
  CUtensorMap a, b;
  int M, N, K, nkA;   // nkA > 0: split-weight product (see tc_gemm_kernel)
  int a_mn, b_mn;     // operand stored MN-major ([K][M] / [K][N], the M / N index contiguous): its
                      // tensor map's inner dimension is M / N, boxes {64 MN, 64 K}
  int a_gap, a_skip;  // a_gap > 0 (K-major A): A's K slices from a_gap on sit a_skip 64-column blocks further
  int tiles_n, tile_begin;
  int ksplit;         // > 1: K is split over ksplit CTAs per output tile (one-tile kernel only)
  int ksplit_cap;     // the most splits the problem's buffers hold (the launch picks ksplit <= it)
  EpiDesc epi;
  float* part;        // split-K partial tiles [tile][ksplit][128][BN] (FP32)
  unsigned* tickets;  // split-K arrival count per output tile (zero between launches)
};
static_assert(alignof(GemmProblem) >= 64 && sizeof(GemmProblem) % 64 == 0, "problem tables hold aligned tensor maps");

// Ring depth STAGES: deep rings keep a whole 512-deep product in flight at
// once (latency-bound small problems); shallow ones leave room for two CTAs
// per SM, one's epilogue overlapping the other's main loop (large problems).
template <int BN, int STAGES>
struct GemmSmem {
  static constexpr uint32_t kABytes = kBM * kBK * 2;   // 16 KiB
  static constexpr uint32_t kBBytes = BN * kBK * 2;    // BN * 128 B
  static constexpr uint32_t kStageBytes = kABytes + kBBytes;
  static constexpr int kStages = STAGES;
  // operand ring + barriers (full[S], empty[S], done) + TMEM slot, plus 1 KiB for alignment
  static constexpr uint32_t kBytes = kStages * kStageBytes + 1024 + 256;
  static constexpr uint32_t kTmemCols = BN;
  static_assert(BN % 64 == 0 && BN <= 256, "BN must be 64, 128 or 256");
  static_assert(kBytes <= 227 * 1024, "shared memory per CTA");
};

// 32 BF16 values -> four 16-byte stores (dst 16-byte aligned)
__device__ __forceinline__ void store_bf16x32(__nv_bfloat16* dst, const float (&x)[32]) {
  uint32_t w[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const __nv_bfloat162 p = __floats2bfloat162_rn(x[2 * i], x[2 * i + 1]);
    w[i] = *reinterpret_cast<const uint32_t*>(&p);
  }
  uint4* d = reinterpret_cast<uint4*>(dst);
#pragma unroll
  for (int q = 0; q < 4; ++q) d[q] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
}
__device__ __forceinline__ void store_f32x32(float* dst, const float (&x)[32]) {
  float4* d = reinterpret_cast<float4*>(dst);
#pragma unroll
  for (int q = 0; q < 8; ++q) d[q] = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
}
__device__ __forceinline__ void load_bias32(const float* b, float (&x)[32]) {
  const float4* s = reinterpret_cast<const float4*>(b);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const float4 t = __ldg(s + q);
    x[4 * q] = t.x;
    x[4 * q + 1] = t.y;
    x[4 * q + 2] = t.z;
    x[4 * q + 3] = t.w;
  }
}
__device__ __forceinline__ void load_mask32(const __nv_bfloat16* m, bool (&on)[32]) {
  const uint4* s = reinterpret_cast<const uint4*>(m);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const uint4 t = s[q];
    const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const __nv_bfloat162 p = *reinterpret_cast<const __nv_bfloat162*>(&w[j]);
      on[8 * q + 2 * j] = __low2float(p) > 0.f;
      on[8 * q + 2 * j + 1] = __high2float(p) > 0.f;
    }
  }
}

// L2 prefetch of a tile's B operand (the weight side of every product here),
// issued before pdl_wait so that its DRAM reads overlap the predecessor's
// tail.  The predecessor never writes it: B holds weights (written by the
// Adam step of an earlier launch) or activations of an earlier layer.
template <int BN>
__device__ __forceinline__ void prefetch_b_tile(const CUtensorMap* tmB, int K, int N, int n0) {
  const int nk = (K + kBK - 1) / kBK;
  for (int kb = 0; kb < nk && kb < 64; ++kb)
#pragma unroll
    for (int r = 0; r < BN / 64; ++r)
      if (n0 + 64 * r < N) tma_prefetch_2d(tmB, kb * kBK, n0 + 64 * r);
}

// L2 prefetch of a tile's B operand in either storage order.
template <int BN>
__device__ __forceinline__ void prefetch_b(const GemmProblem* P, int n0) {
  if (!P->b_mn) {
    prefetch_b_tile<BN>(&P->b, P->K, P->N, n0);
    return;
  }
  const int nk = (P->K + kBK - 1) / kBK;
  for (int kb = 0; kb < nk && kb < 64; ++kb)
#pragma unroll
    for (int r = 0; r < BN / 64; ++r)
      if (n0 + 64 * r < P->N) tma_prefetch_2d(&P->b, n0 + 64 * r, kb * kBK);
}

// TMA loads of K slice kb: 128 rows of A from row m0 and NB 64-row boxes of B
// from row n0, each box landing 8 KiB after the previous.  K-major operands
// come as {64 K, 64 rows} boxes (the slice's 128-byte rows), MN-major ones as
// {64 MN, 64 K} boxes (64 K rows of 128 bytes per 64 M or N): in both cases a
// box is an 8 KiB 128-byte-swizzled block.
// The operand description of a problem, read into registers once per tile
// (the loads' asm statements would otherwise force a reread per slice).
struct SliceSrc {
  const CUtensorMap* a;
  const CUtensorMap* b;
  int a_mn, b_mn, nkA, a_gap, a_skip;
};
__device__ __forceinline__ SliceSrc slice_src(const GemmProblem* P) {
  return SliceSrc{&P->a, &P->b, P->a_mn, P->b_mn, P->nkA, P->a_gap, P->a_skip};
}
template <int NB>
__device__ __forceinline__ void load_slice(const SliceSrc& P, uint8_t* a_dst, uint8_t* b_dst, uint64_t* bar, int kb,
                                           int m0, int n0) {
  const CUtensorMap* tmA = P.a;
  const CUtensorMap* tmB = P.b;
  if (P.a_mn) {
#pragma unroll
    for (int r = 0; r < kBM / 64; ++r) tma_load_2d(a_dst + r * 8192, tmA, bar, m0 + 64 * r, kb * kBK);
  } else {
    const int ka = P.nkA > 0 ? kb % P.nkA : kb;
    const int kx = (P.a_gap > 0 && ka >= P.a_gap) ? ka + P.a_skip : ka;
#pragma unroll
    for (int r = 0; r < kBM / 64; ++r) tma_load_2d(a_dst + r * 8192, tmA, bar, kx * kBK, m0 + 64 * r);
  }
  if (P.b_mn) {
#pragma unroll
    for (int r = 0; r < NB; ++r) tma_load_2d(b_dst + r * 8192, tmB, bar, n0 + 64 * r, kb * kBK);
  } else {
#pragma unroll
    for (int r = 0; r < NB; ++r) tma_load_2d(b_dst + r * 8192, tmB, bar, kb * kBK, n0 + 64 * r);
  }
}

// Shared-memory descriptor of a slice's operand tile (K step 0) and the
// increment of its address field per K step of 16: K-major +32 bytes along the
// 128-byte rows, MN-major 16 K rows further (2 KiB; 64-element MN blocks 8 KiB
// apart).  The MMA issuer adds k * step: no per-MMA descriptor arithmetic.
__device__ __forceinline__ uint64_t slice_desc(const uint8_t* tile, bool mn) {
  return mn ? sdesc_mnmajor_sw128(tile, 8192) : sdesc_kmajor_sw128(tile);
}
__device__ __forceinline__ uint32_t slice_step(bool mn) { return mn ? 2048u >> 4 : 32u >> 4; }
// The instruction descriptor's operand-order bits (A: bit 15, B: bit 16; 1 = MN-major).
__device__ __forceinline__ uint32_t idesc_major(uint32_t idesc, const GemmProblem* P) {
  return idesc | ((P->a_mn ? 1u : 0u) << 15) | ((P->b_mn ? 1u : 0u) << 16);
}

// Epilogue of one 32-column chunk (columns col0 .. col0 + 31) of row `row`.
// The full-chunk paths use 16-byte accesses; they need 16-byte aligned rows:
// leading dimensions a multiple of 8 BF16 / 4 FP32 elements (hidden widths
// are multiples of 8; other widths are tested here) and 16-byte aligned base
// pointers (library buffers come from cudaMalloc; crl_bind_params rejects
// parameter and gradient arrays that are not 16-byte aligned).
__device__ __forceinline__ void epilogue_chunk(const EpiDesc& e, int row, int col0, float (&v)[32], int M, int N) {
  if (row >= M) return;
  const bool full = col0 + 32 <= N;
  using bf16 = __nv_bfloat16;
  switch (e.kind) {
    case kEpiFwdHidden: {
      bf16* h = static_cast<bf16*>(e.out0);
      if (full) {
        float b[32];
        load_bias32(e.bias + col0, b);
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = fmaxf(v[i] + b[i], 0.f);
        store_bf16x32(h + (size_t)row * e.ld0 + col0, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] -= __bfloat162float(__float2bfloat16_rn(v[i]));
        store_bf16x32(h + (size_t)row * e.ld0 + e.c0 + col0, v);
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          if (col0 + i >= N) break;
          const float x = fmaxf(v[i] + e.bias[col0 + i], 0.f);
          const bf16 o = __float2bfloat16_rn(x);
          h[(size_t)row * e.ld0 + col0 + i] = o;
          h[(size_t)row * e.ld0 + e.c0 + col0 + i] = __float2bfloat16_rn(x - __bfloat162float(o));
        }
      }
      break;
    }
    case kEpiFwdPreLN:
    case kEpiFwdOut: {
      float* z = static_cast<float*>(e.out0) + (size_t)row * e.ld0;
      if (full && (e.ld0 & 3) == 0) {
        float b[32];
        load_bias32(e.bias + col0, b);
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] += b[i];
        store_f32x32(z + col0, v);
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i)
          if (col0 + i < N) z[col0 + i] = v[i] + e.bias[col0 + i];
      }
      break;
    }
    case kEpiBwdDX:
    case kEpiBwdDXLN: {
      const bf16* mrow = e.mask + (size_t)row * e.ldm;
      if (full) {
        bool on[32];
        load_mask32(mrow + col0, on);
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = on[i] ? v[i] : 0.f;
        if (e.kind == kEpiBwdDXLN) store_f32x32(static_cast<float*>(e.out0) + (size_t)row * e.ld0 + col0, v);
        else store_bf16x32(static_cast<bf16*>(e.out0) + (size_t)row * e.ld0 + col0, v);
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int c = col0 + i;
          if (c >= N) break;
          const float x = __bfloat162float(mrow[c]) > 0.f ? v[i] : 0.f;
          if (e.kind == kEpiBwdDXLN) static_cast<float*>(e.out0)[(size_t)row * e.ld0 + c] = x;
          else static_cast<bf16*>(e.out0)[(size_t)row * e.ld0 + c] = __float2bfloat16_rn(x);
        }
      }
      break;
    }
    case kEpiBwdDW: {
      float* dW = static_cast<float*>(e.out0) + (size_t)row * e.kin;
      if (col0 + 32 <= e.kin && (e.kin & 3) == 0) {
        store_f32x32(dW + col0, v);
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int c = col0 + i;
          if (c >= N) break;
          if (c < e.kin) dW[c] = v[i];
          else static_cast<float*>(e.out1)[row] = v[i];
        }
      }
      break;
    }
    case kEpiBwdDW0: {
      float* dW = static_cast<float*>(e.out0) + (size_t)row * e.kin;
#pragma unroll
      for (int i = 0; i < 32; i += 2) {
        const int c = col0 + i;
        if (c < 2 * e.kin) dW[c / 2] = v[i] + v[i + 1];
        else if (c == 2 * e.kin) static_cast<float*>(e.out1)[row] = v[i];
      }
      break;
    }
    default: {  // kEpiDX0
      float* dx = static_cast<float*>(e.out0) + (size_t)row * e.nc;
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int c = col0 + i - e.c0;
        if (col0 + i < N && c >= 0 && c < e.nc) dx[c] = v[i];
      }
      break;
    }
  }
}

// The output layer feeding the fused energy (kEpiFwdOutEnergy): two passes over
// this thread's row in TMEM (the tile holds all N columns): FP32 output and the
// squared norm, then the scaled BF16 operand.
__device__ __forceinline__ void epilogue_energy(const EpiDesc& e, int row, uint32_t lane_base, int N, int M) {
  using bf16 = __nv_bfloat16;
  const bool live = row < M;
  const bool cosine = e.energy == CRL_ENERGY_COS;
  float q = 0.f;
#pragma unroll 1
  for (int c = 0; c < N; c += 32) {
    float v[32];
    tmem_ld32(lane_base + c, v);   // warp-collective: every lane, live or not
    if (!live) continue;
    float b[32];
    load_bias32(e.bias + c, b);
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      v[i] += b[i];
      const float r = cosine ? v[i] : __bfloat162float(__float2bfloat16_rn(v[i]));
      q += r * r;
    }
    store_f32x32(static_cast<float*>(e.out0) + (size_t)row * e.ld0 + c, v);
  }
  const float scale = cosine ? rsqrtf(q) : 1.f;
  if (live) e.aux[row] = cosine ? scale : q;
  bf16* X = static_cast<bf16*>(e.out1);
#pragma unroll 1
  for (int c = 0; c < N; c += 32) {
    float v[32];
    tmem_ld32(lane_base + c, v);
    if (!live) continue;
    float b[32];
    load_bias32(e.bias + c, b);
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = (v[i] + b[i]) * scale;
    store_bf16x32(X + (size_t)row * N + c, v);
  }
}

// nkA > 0: A has only nkA K-slices and slice kb of B multiplies slice kb % nkA of
// A -- B holds the weight pair along K ([W_hi | W_lo], or [W_hi | W_hi | W_lo]
// against A = [h_hi | h_lo]) and each A tile is used against several parts.
template <int BN, int STAGES>
__global__ void __launch_bounds__(128, 1)
    tc_gemm_kernel(const GemmProblem* __restrict__ probs, int nprob, unsigned* status) {
  using S = GemmSmem<BN, STAGES>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align1024(smem_raw);
  uint8_t* sA = smem;
  uint8_t* sB = smem + S::kStages * S::kABytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S::kStages * S::kStageBytes);
  uint64_t* empty = full + S::kStages;
  uint64_t* done = empty + S::kStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);

  // problem of this CTA: the last p with tile_begin <= blockIdx.x (the table is immutable)
  int lo = 0, hi = nprob - 1;
  const int t = blockIdx.x;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (probs[mid].tile_begin <= t) lo = mid;
    else hi = mid - 1;
  }
  const GemmProblem* P = probs + lo;
  // split-K: ksplit consecutive CTAs share one output tile, each a K range
  const int ksplit = P->ksplit > 1 ? P->ksplit : 1;
  const int lt = (t - P->tile_begin) / ksplit, split = (t - P->tile_begin) % ksplit;
  const int M = P->M, N = P->N, K = P->K, nkA = P->nkA;
  const int m0 = (lt / P->tiles_n) * kBM, n0 = (lt % P->tiles_n) * BN;
  const CUtensorMap* tmA = &P->a;
  const CUtensorMap* tmB = &P->b;

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int nk_all = (K + kBK - 1) / kBK;
  const int kb0 = split * nk_all / ksplit, nk = (split + 1) * nk_all / ksplit - kb0;

  if (threadIdx.x == 0) {
    tmap_acquire(tmA);
    tmap_acquire(tmB);
    prefetch_tmap(tmA);
    prefetch_tmap(tmB);
    prefetch_b<BN>(P, n0);
    for (int s = 0; s < S::kStages; ++s) {
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
  // operands come from the predecessor; the epilogue may overwrite what it read
  pdl_wait();
  pdl_trigger();
  const unsigned long long lim = wait_limit(status);

  if (warp == 0 && lane == 0) {
    // TMA producer
    const SliceSrc src = slice_src(P);
    int issued = 0;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % S::kStages;
      if (kb >= S::kStages && !mbar_wait(&empty[s], ((kb / S::kStages) & 1) ^ 1, lim)) {
        atomicOr(status, CRL_STATUS_TIMEOUT);
        break;
      }
      ++issued;
      mbar_arrive_expect_tx(&full[s], S::kStageBytes);
      // operands arrive as 64-row boxes (8 KiB each); stacked along rows they
      // form the same 128-byte-swizzled K-major tile as one tall box
      load_slice<BN / 64>(src, sA + s * S::kABytes, sB + s * S::kBBytes, &full[s], kb0 + kb, m0, n0);
    }
    // nothing may land in this CTA's shared memory after it exits
    drain_ring(full, S::kStages, issued);
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    const uint32_t idesc = idesc_major(idesc_bf16_f32(kBM, BN), P);
    const bool amn = P->a_mn != 0, bmn = P->b_mn != 0;
    const uint32_t sa = slice_step(amn), sb = slice_step(bmn);
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % S::kStages;
      if (!mbar_wait(&full[s], (kb / S::kStages) & 1, lim)) {
        atomicOr(status, CRL_STATUS_TIMEOUT);
        break;
      }
      fence_after_sync();
      const uint64_t da = slice_desc(sA + s * S::kABytes, amn), db = slice_desc(sB + s * S::kBBytes, bmn);
#pragma unroll
      for (int k = 0; k < kBK / 16; ++k)
        mma_bf16(tmem, da + sa * k, db + sb * k, idesc, (kb > 0 || k > 0) ? 1u : 0u);
      mma_commit(&empty[s]);
    }
    // always: `done` completes once every MMA issued here has (after a timeout
    // the accumulator is incomplete, and the status word says so)
    mma_commit(done);
  }
  __syncwarp();

  // epilogue (tcgen05.ld is warp-collective: keep the decision warp-uniform)
  const bool ok = __all_sync(0xffffffffu, mbar_wait(done, 0, lim) ? 1 : 0) != 0;
  fence_after_sync();
  if (ok && ksplit > 1) {
    // split-K: store this split's FP32 partial tile; the last CTA of the tile to
    // arrive adds the ksplit partials in split order (its own from TMEM) and
    // runs the epilogue, so the result does not depend on which CTA is last
    __shared__ int s_last;
    const EpiDesc e = P->epi;
    const int r = warp * 32 + lane, row = m0 + r;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    const int ncol = (N - n0 < BN) ? N - n0 : BN;
    float* part = P->part + (size_t)lt * ksplit * kBM * BN;
#pragma unroll 1
    for (int c = 0; c < ncol; c += 32) {
      float v[32];
      tmem_ld32(lane_base + c, v);
      store_f32x32(part + ((size_t)split * kBM + r) * BN + c, v);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(P->tickets + lt, 1u) == (unsigned)ksplit - 1u) ? 1 : 0;
    __syncthreads();
    if (s_last) {
      __threadfence();
#pragma unroll 1
      for (int c = 0; c < ncol; c += 32) {
        float v[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = 0.f;
        for (int q = 0; q < ksplit; ++q) {
          const float4* src = reinterpret_cast<const float4*>(part + ((size_t)q * kBM + r) * BN + c);
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const float4 x = __ldcg(src + i);
            v[4 * i] += x.x;
            v[4 * i + 1] += x.y;
            v[4 * i + 2] += x.z;
            v[4 * i + 3] += x.w;
          }
        }
        epilogue_chunk(e, row, n0 + c, v, M, N);
      }
      if (threadIdx.x == 0) P->tickets[lt] = 0u;
    }
  } else if (ok) {
    const EpiDesc e = P->epi;
    const int row = m0 + warp * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    const int ncol = (N - n0 < BN) ? N - n0 : BN;
    if (e.kind == kEpiFwdOutEnergy) {
      epilogue_energy(e, row, lane_base, ncol, M);
    } else {
#pragma unroll 1
      for (int c = 0; c < ncol; c += 32) {
        float v[32];
        tmem_ld32(lane_base + c, v);
        epilogue_chunk(e, row, n0 + c, v, M, N);
      }
    }
  } else if (threadIdx.x == 0) {
    atomicOr(status, CRL_STATUS_TIMEOUT);
  }
  // the accumulator is freed only after every MMA writing it has completed
  if (!ok && threadIdx.x == 0) mbar_wait(done, 0, kDrainLimitNs);
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, S::kTmemCols);
}

// The problem of tile t: the last p with tile_begin <= t (the table is immutable).
__device__ __forceinline__ const GemmProblem* find_problem(const GemmProblem* __restrict__ probs, int nprob, int t) {
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (probs[mid].tile_begin <= t) lo = mid;
    else hi = mid - 1;
  }
  return probs + lo;
}

// Persistent variant: gridDim.x CTAs (one per SM at most) walk the tiles
// t = blockIdx.x, blockIdx.x + gridDim.x, ... of the whole problem list.
// 192 threads:
//   warp 0 / lane 0 -- TMA producer over all of the CTA's tiles: the operand
//                      ring runs on across tile boundaries;
//   warp 1 / lane 0 -- MMA issuer: tile i accumulates into TMEM buffer i % 2
//                      (2 x BN columns), once the epilogue has released it;
//   warps 2..5      -- epilogue of tile i from buffer i % 2 while the MMAs of
//                      tile i + 1 fill the other one (warp w reads TMEM lanes
//                      32 (w % 4) ..).
// The epilogue is the same as the one-tile kernel's, so both give identical
// outputs.
template <int BN, int STAGES>
__global__ void __launch_bounds__(192, 1)
    tc_gemm_persistent_kernel(const GemmProblem* __restrict__ probs, int nprob, int total, unsigned* status) {
  using S = GemmSmem<BN, STAGES>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align1024(smem_raw);
  uint8_t* sA = smem;
  uint8_t* sB = smem + S::kStages * S::kABytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S::kStages * S::kStageBytes);
  uint64_t* empty = full + S::kStages;
  uint64_t* accf = empty + S::kStages;  // [2] accumulator buffer ready (MMA -> epilogue)
  uint64_t* acce = accf + 2;            // [2] accumulator buffer free (epilogue -> MMA), 4 arrivals
  uint64_t* drain = acce + 2;           // every MMA of this CTA has completed (teardown)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (threadIdx.x == 0) {
    if ((int)blockIdx.x < total) {   // the first tile's B operand
      const GemmProblem* P = find_problem(probs, nprob, blockIdx.x);
      tmap_acquire(&P->b);
      prefetch_b<BN>(P, (((int)blockIdx.x - P->tile_begin) % P->tiles_n) * BN);
    }
    for (int s = 0; s < S::kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], 4);
    }
    mbar_init(drain, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(tmem_slot, 2 * BN);
    tmem_relinquish();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  pdl_wait();
  pdl_trigger();
  const unsigned long long lim = wait_limit(status);

  if (warp == 0) {
    if (lane == 0) {
      // TMA producer; `it` counts K-slices over all tiles of this CTA
      int it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
        const GemmProblem* P = find_problem(probs, nprob, t);
        const int lt = t - P->tile_begin;
        const int m0 = (lt / P->tiles_n) * kBM, n0 = (lt % P->tiles_n) * BN;
        const int nk = (P->K + kBK - 1) / kBK;
        tmap_acquire(&P->a);
        tmap_acquire(&P->b);
        const SliceSrc src = slice_src(P);
        for (int kb = 0; kb < nk; ++kb, ++it) {
          const int s = it % S::kStages;
          if (it >= S::kStages && !mbar_wait(&empty[s], ((it / S::kStages) & 1) ^ 1, lim)) {
            atomicOr(status, CRL_STATUS_TIMEOUT);
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&full[s], S::kStageBytes);
          load_slice<BN / 64>(src, sA + s * S::kABytes, sB + s * S::kBBytes, &full[s], kb, m0, n0);
        }
      }
      // `it` slices were issued (a timed-out one was not): let them all land
      drain_ring(full, S::kStages, it);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer
      int it = 0, i = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < total && ok; t += gridDim.x, ++i) {
        const GemmProblem* P = find_problem(probs, nprob, t);
        const int nk = (P->K + kBK - 1) / kBK;
        const uint32_t idesc = idesc_major(idesc_bf16_f32(kBM, BN), P);
        const bool amn = P->a_mn != 0, bmn = P->b_mn != 0;
        const uint32_t sa = slice_step(amn), sb = slice_step(bmn);
        const int buf = i & 1, use = i >> 1;
        // the epilogue of tile i - 2 must have read this buffer out
        if (use > 0 && !mbar_wait(&acce[buf], (use - 1) & 1, lim)) {
          atomicOr(status, CRL_STATUS_TIMEOUT);
          break;
        }
        fence_after_sync();
        const uint32_t d = tmem + (uint32_t)(buf * BN);
        for (int kb = 0; kb < nk; ++kb, ++it) {
          const int s = it % S::kStages;
          if (!mbar_wait(&full[s], (it / S::kStages) & 1, lim)) {
            atomicOr(status, CRL_STATUS_TIMEOUT);
            ok = false;
            break;
          }
          fence_after_sync();
          const uint64_t da = slice_desc(sA + s * S::kABytes, amn), db = slice_desc(sB + s * S::kBBytes, bmn);
#pragma unroll
          for (int k = 0; k < kBK / 16; ++k) mma_bf16(d, da + sa * k, db + sb * k, idesc, (kb > 0 || k > 0) ? 1u : 0u);
          mma_commit(&empty[s]);
        }
        if (ok) mma_commit(&accf[buf]);
      }
      mma_commit(drain);   // completes once every MMA issued above has
    }
  } else {
    // epilogue warps (tcgen05.ld is warp-collective: decisions stay warp-uniform)
    const int eg = warp & 3;
    int i = 0;
    for (int t = blockIdx.x; t < total; t += gridDim.x, ++i) {
      const int buf = i & 1, use = i >> 1;
      const bool ok = __all_sync(0xffffffffu, mbar_wait(&accf[buf], use & 1, lim) ? 1 : 0) != 0;
      if (!ok) {
        if (lane == 0) atomicOr(status, CRL_STATUS_TIMEOUT);
        break;
      }
      fence_after_sync();
      const GemmProblem* P = find_problem(probs, nprob, t);
      const int lt = t - P->tile_begin;
      const int m0 = (lt / P->tiles_n) * kBM, n0 = (lt % P->tiles_n) * BN;
      const int M = P->M, N = P->N;
      const EpiDesc e = P->epi;
      const int row = m0 + eg * 32 + lane;
      const uint32_t lane_base = tmem + (uint32_t)(buf * BN) + ((uint32_t)(eg * 32) << 16);
      const int ncol = (N - n0 < BN) ? N - n0 : BN;
      if (e.kind == kEpiFwdOutEnergy) {
        epilogue_energy(e, row, lane_base, ncol, M);
      } else {
#pragma unroll 1
        for (int c = 0; c < ncol; c += 32) {
          float v[32];
          tmem_ld32(lane_base + c, v);
          epilogue_chunk(e, row, n0 + c, v, M, N);
        }
      }
      // release the buffer to the MMA issuer
      fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce[buf]);
    }
  }
  // no MMA may still write the accumulators when they are freed
  if (threadIdx.x == 0) mbar_wait(drain, 0, kDrainLimitNs);
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 2 * BN);
}

// CTA-pair variant: a cluster of two CTAs (on one TPC) computes 256 x BN
// tiles with tcgen05.mma.cta_group::2, walking the tiles t = cluster,
// cluster + clusters, ... like the persistent kernel.  Each CTA loads its own
// operands into its own ring: 128 rows of A (the pair's rows 128 r ..) and
// BN / 2 rows of B (columns BN / 2 r .. of the tile), so a pair moves half the
// operand bytes of two one-SM tiles of the same work.  The even CTA issues
// every MMA; its accumulator rows live in the even CTA's TMEM, the others in
// the odd CTA's.  No multicast: the CTAs exchange plain mbarrier arrivals.
//   warp 0 / lane 0 -- TMA producer of this CTA's ring;
//   warp 1 / lane 0 -- even CTA: MMA issuer (waits for its own slot and the
//                      odd CTA's `pfull` arrival); odd CTA: reports each
//                      landed slot to the even CTA's `pfull`;
//   warps 2..5      -- epilogue of this CTA's 128 rows from TMEM buffer i % 2;
//                      all eight warps release the buffer on the even CTA's `acce`;
//   warp 6 / lane 0 -- even CTA: passes each freed slot (`empty`) and each
//                      finished accumulator (`accf`) on to the odd CTA.
// The epilogue is the one-tile kernel's, so every kernel gives identical outputs
// where the MMA sums each K = 16 slice the same way.
template <int BN, int STAGES>
struct GemmPairSmem {
  static constexpr uint32_t kABytes = kBM * kBK * 2;         // 16 KiB: this CTA's 128 rows of A
  static constexpr uint32_t kBBytes = (BN / 2) * kBK * 2;    // this CTA's BN / 2 rows of B
  static constexpr uint32_t kStageBytes = kABytes + kBBytes;
  static constexpr int kStages = STAGES;
  // ring + barriers (full, empty, pfull [S]; accf, acce [2]; drain) + TMEM slot, plus 1 KiB for
  // alignment and one more B half behind the ring, so that the last slot's B rows plus BN / 2
  // rows stay inside this CTA's shared memory
  static constexpr uint32_t kBytes = kStages * kStageBytes + kBBytes + 1024 + 512;
  static constexpr uint32_t kTmemCols = 2 * BN;   // two accumulator buffers
  static_assert(BN == 128 || BN == 256, "pair tiles are 256 x 128 or 256 x 256");
  static_assert(kTmemCols <= 512, "TMEM columns");
  static_assert(kBytes <= 227 * 1024, "shared memory per CTA");
};

template <int BN, int STAGES>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(224, 1)
    tc_gemm_pair_kernel(const GemmProblem* __restrict__ probs, int nprob, int total, unsigned* status) {
  using S = GemmPairSmem<BN, STAGES>;
  constexpr int kPairM = 2 * kBM;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align1024(smem_raw);
  uint8_t* sA = smem;
  uint8_t* sB = smem + S::kStages * S::kABytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S::kStages * S::kStageBytes + S::kBBytes);
  uint64_t* empty = full + S::kStages;
  uint64_t* pfull = empty + S::kStages;  // even CTA: the odd CTA's slot has landed
  uint64_t* accf = pfull + S::kStages;   // [2] accumulator buffer ready
  uint64_t* acce = accf + 2;             // [2] even CTA: buffer read out by all 8 epilogue warps
  uint64_t* drain = acce + 2;            // every MMA of the pair has completed (teardown)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);

  const uint32_t rank = cluster_ctarank();
  const bool even = rank == 0;
  const int cl = blockIdx.x / 2, ncl = gridDim.x / 2;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (threadIdx.x == 0) {
    if (cl < total) {   // the first tile's B rows of this CTA
      const GemmProblem* P = find_problem(probs, nprob, cl);
      tmap_acquire(&P->b);
      prefetch_b<BN / 2>(P, ((cl - P->tile_begin) % P->tiles_n) * BN + (BN / 2) * rank);
    }
    for (int s = 0; s < S::kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      mbar_init(&pfull[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], 8);
    }
    mbar_init(drain, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc_pair(tmem_slot, S::kTmemCols);
    tmem_relinquish_pair();
  }
  fence_before_sync();
  cluster_sync();   // both CTAs' barriers are initialised before any remote arrival
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  pdl_wait();
  pdl_trigger();
  const unsigned long long lim = wait_limit(status);

  if (warp == 0) {
    if (lane == 0) {
      // TMA producer; `it` counts K-slices over all tiles of this pair
      int it = 0;
      bool ok = true;
      for (int t = cl; t < total && ok; t += ncl) {
        const GemmProblem* P = find_problem(probs, nprob, t);
        const int lt = t - P->tile_begin;
        const int m0 = (lt / P->tiles_n) * kPairM + kBM * (int)rank;
        const int n0 = (lt % P->tiles_n) * BN + (BN / 2) * (int)rank;
        const int nk = (P->K + kBK - 1) / kBK;
        tmap_acquire(&P->a);
        tmap_acquire(&P->b);
        const SliceSrc src = slice_src(P);
        for (int kb = 0; kb < nk; ++kb, ++it) {
          const int s = it % S::kStages;
          if (it >= S::kStages) {
            const bool got = even ? mbar_wait(&empty[s], ((it / S::kStages) & 1) ^ 1, lim)
                                  : mbar_wait_cluster(&empty[s], ((it / S::kStages) & 1) ^ 1, lim);
            if (!got) {
              atomicOr(status, CRL_STATUS_TIMEOUT);
              ok = false;
              break;
            }
          }
          mbar_arrive_expect_tx(&full[s], S::kStageBytes);
          load_slice<BN / 128>(src, sA + s * S::kABytes, sB + s * S::kBBytes, &full[s], kb, m0, n0);
        }
      }
      drain_ring(full, S::kStages, it);
    }
  } else if (warp == 1) {
    if (lane == 0 && even) {
      // MMA issuer of the pair
      int it = 0, i = 0;
      bool ok = true;
      for (int t = cl; t < total && ok; t += ncl, ++i) {
        const GemmProblem* P = find_problem(probs, nprob, t);
        const int nk = (P->K + kBK - 1) / kBK;
        const uint32_t idesc = idesc_major(idesc_bf16_f32(kPairM, BN), P);
        const bool amn = P->a_mn != 0, bmn = P->b_mn != 0;
        const uint32_t sa = slice_step(amn), sb = slice_step(bmn);
        const int buf = i & 1, use = i >> 1;
        // all eight epilogue warps must have read out this buffer (tile i - 2)
        if (use > 0 && !mbar_wait_cluster(&acce[buf], (use - 1) & 1, lim)) {
          atomicOr(status, CRL_STATUS_TIMEOUT);
          break;
        }
        fence_after_sync();
        const uint32_t d = tmem + (uint32_t)(buf * BN);
        for (int kb = 0; kb < nk; ++kb, ++it) {
          const int s = it % S::kStages;
          const uint32_t par = (it / S::kStages) & 1;
          if (!mbar_wait(&full[s], par, lim) || !mbar_wait_cluster(&pfull[s], par, lim)) {
            atomicOr(status, CRL_STATUS_TIMEOUT);
            ok = false;
            break;
          }
          fence_after_sync();
          const uint64_t da = slice_desc(sA + s * S::kABytes, amn), db = slice_desc(sB + s * S::kBBytes, bmn);
#pragma unroll
          for (int k = 0; k < kBK / 16; ++k)
            mma_bf16_pair(d, da + sa * k, db + sb * k, idesc, (kb > 0 || k > 0) ? 1u : 0u);
          mma_commit_pair(&empty[s]);
        }
        if (ok) mma_commit_pair(&accf[buf]);
      }
      mma_commit_pair(drain);   // completes once every MMA issued above has
    } else if (lane == 0) {
      // odd CTA: report each landed slot to the MMA issuer
      int it = 0;
      bool ok = true;
      for (int t = cl; t < total && ok; t += ncl) {
        const GemmProblem* P = find_problem(probs, nprob, t);
        const int nk = (P->K + kBK - 1) / kBK;
        for (int kb = 0; kb < nk; ++kb, ++it) {
          const int s = it % S::kStages;
          if (!mbar_wait(&full[s], (it / S::kStages) & 1, lim)) {
            atomicOr(status, CRL_STATUS_TIMEOUT);
            ok = false;
            break;
          }
          mbar_arrive_remote(mapa_shared(&pfull[s], 0));
        }
      }
    }
  } else if (warp == 6) {
    if (lane == 0 && even) {
      // relay of the even CTA: every completed MMA slice frees the odd CTA's
      // slot too, and every completed tile its accumulator rows (a thread of
      // its own, so that no cluster-scope release waits behind the producer's
      // copies or the epilogue's stores)
      int it = 0, i = 0;
      bool ok = true;
      for (int t = cl; t < total && ok; t += ncl, ++i) {
        const GemmProblem* P = find_problem(probs, nprob, t);
        const int nk = (P->K + kBK - 1) / kBK;
        for (int kb = 0; kb < nk; ++kb, ++it) {
          const int s = it % S::kStages;
          if (!mbar_wait(&empty[s], (it / S::kStages) & 1, lim)) {
            atomicOr(status, CRL_STATUS_TIMEOUT);
            ok = false;
            break;
          }
          mbar_arrive_remote(mapa_shared(&empty[s], 1));
        }
        if (!ok) break;
        const int buf = i & 1, use = i >> 1;
        if (!mbar_wait(&accf[buf], use & 1, lim)) {
          atomicOr(status, CRL_STATUS_TIMEOUT);
          break;
        }
        mbar_arrive_remote(mapa_shared(&accf[buf], 1));
      }
    }
  } else {
    // epilogue warps: this CTA's 128 rows of the pair's tile
    const int eg = warp & 3;
    int i = 0;
    for (int t = cl; t < total; t += ncl, ++i) {
      const int buf = i & 1, use = i >> 1;
      const bool got = even ? mbar_wait(&accf[buf], use & 1, lim) : mbar_wait_cluster(&accf[buf], use & 1, lim);
      const bool ok = __all_sync(0xffffffffu, got ? 1 : 0) != 0;
      if (!ok) {
        if (lane == 0) atomicOr(status, CRL_STATUS_TIMEOUT);
        break;
      }
      fence_after_sync();
      const GemmProblem* P = find_problem(probs, nprob, t);
      const int lt = t - P->tile_begin;
      const int m0 = (lt / P->tiles_n) * kPairM + kBM * (int)rank, n0 = (lt % P->tiles_n) * BN;
      const int M = P->M, N = P->N;
      const EpiDesc e = P->epi;
      const int row = m0 + eg * 32 + lane;
      const uint32_t lane_base = tmem + (uint32_t)(buf * BN) + ((uint32_t)(eg * 32) << 16);
      const int ncol = (N - n0 < BN) ? N - n0 : BN;
      if (e.kind == kEpiFwdOutEnergy) {
        epilogue_energy(e, row, lane_base, ncol, M);
      } else {
#pragma unroll 1
        for (int c = 0; c < ncol; c += 32) {
          float v[32];
          tmem_ld32(lane_base + c, v);
          epilogue_chunk(e, row, n0 + c, v, M, N);
        }
      }
      // release the buffer to the MMA issuer
      fence_before_sync();
      __syncwarp();
      if (lane == 0) {
        if (even) mbar_arrive(&acce[buf]);
        else mbar_arrive_remote(mapa_shared(&acce[buf], 0));
      }
    }
  }
  // teardown: no MMA may still write either CTA's accumulators when they are
  // freed, and no remote arrival may reach a CTA that has left
  fence_before_sync();
  __syncthreads();
  if (threadIdx.x == 0) {
    if (even) {
      mbar_wait(drain, 0, kDrainLimitNs);
      mbar_arrive_remote(mapa_shared(drain, 1));
    } else {
      mbar_wait_cluster(drain, 0, kDrainLimitNs);
    }
  }
  fence_before_sync();
  cluster_sync();
  fence_after_sync();
  if (warp == 0) tmem_dealloc_pair(tmem, S::kTmemCols);
}

}  // namespace tc
}  // namespace crl
