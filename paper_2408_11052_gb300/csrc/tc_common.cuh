// Blackwell (sm_103a) tensor-core primitives as inline PTX: mbarriers, TMA
// tile loads, TMEM allocation, tcgen05.mma (kind::f16, BF16 in / FP32 out),
// tcgen05.commit and tcgen05.ld.
//
// Every wait is bounded by a %globaltimer limit: a wait that gives up sets
// CRL_STATUS_TIMEOUT in the device status word and the kernel tears down
// instead of spinning forever.  Teardown first waits (bounded again) for the
// CTA's own tensor-memory copies and MMAs still in flight, then frees its TMEM.
// The limit is the word after the status word (0: the default 1 s), set per
// context with crl_set_wait_limit_ns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/crl.h"

namespace crl {
namespace tc {

constexpr unsigned long long kWaitLimitNs = 1000000000ull;   // default limit of a wait: 1 s
constexpr unsigned long long kDrainLimitNs = 1000000000ull;  // teardown: the CTA's own copies and MMAs
constexpr unsigned long long kPollBelowNs = 100000ull;       // shorter limits poll without suspending

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
  return reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

// ---- mbarrier ---------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Non-suspending test of phase `parity`.
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// The same two tests with cluster-scope acquire: for a barrier that another
// CTA of the cluster arrives on (its writes before the arrive become visible).
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_test_wait_cluster(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// One arrival on a barrier of another CTA of the cluster (`remote`: its
// mapa_shared address).  Relaxed: what such an arrival announces was written
// by the asynchronous proxy (TMA data, MMA results, TMEM reads) and had
// completed when this thread observed it; a cluster-scope release would add a
// memory barrier (measured as `membar` stalls) that orders nothing needed here.
__device__ __forceinline__ void mbar_arrive_remote(uint32_t remote) {
  asm volatile("mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [%0];" ::"r"(remote) : "memory");
}
// Wait for phase `parity` of `bar`; false if it did not complete within
// `limit` ns.  Limits below kPollBelowNs poll without suspending the thread, so
// that a short limit runs out even where the phase would complete within one
// suspension.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned long long limit) {
  if (limit < kPollBelowNs) {
    const unsigned long long t0 = globaltimer();
    while (!mbar_test_wait(bar, parity)) {
      if (globaltimer() - t0 >= limit) return false;
    }
    return true;
  }
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (!mbar_try_wait(bar, parity)) {
    if (globaltimer() - t0 > limit) return false;
  }
  return true;
}
// mbar_wait for a barrier that another CTA of the cluster arrives on (polls
// without suspending).
__device__ __forceinline__ bool mbar_wait_cluster(uint64_t* bar, uint32_t parity, unsigned long long limit) {
  if (mbar_test_wait_cluster(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (!mbar_test_wait_cluster(bar, parity)) {
    if (globaltimer() - t0 >= limit) return false;
  }
  return true;
}
// The wait limit of a launch: the word after its status word, 0 meaning the default.
__device__ __forceinline__ unsigned long long wait_limit(const unsigned* status) {
  const unsigned w = *reinterpret_cast<const volatile unsigned*>(status + 1);
  return w ? (unsigned long long)w : kWaitLimitNs;
}
// Teardown of a producer thread: wait for the last loads issued into each of
// the `stages` ring slots (`issued` loads in all, slot i % stages, phase i / stages).
__device__ __forceinline__ void drain_ring(uint64_t* full, int stages, int issued) {
  for (int s = 0; s < stages && s < issued; ++s) {
    const int last = s + stages * ((issued - 1 - s) / stages);
    mbar_wait(full + s, (uint32_t)((last / stages) & 1), kDrainLimitNs);
  }
}

// ---- TMA ----------------------------------------------------------------------
// 2-D tiled load of box {x: inner, y: outer} at coordinates (x, y) into shared
// memory, completing `bytes` on `bar`.  x * 2 bytes must be a multiple of 16.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// The shared::cluster address of `p` (this CTA's shared memory) in the CTA of rank `rank`.
__device__ __forceinline__ uint32_t mapa_shared(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}
// Bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned) from
// this CTA's shared memory to shared memory of another CTA of the cluster,
// completing the bytes on that CTA's barrier (dst and bar: mapa_shared addresses).
__device__ __forceinline__ void bulk_copy_to_peer(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "r"(smem_u32(src)), "r"(bytes), "r"(bar)
      : "memory");
}
// Named barrier `id` over `nthreads` threads (a multiple of 32) that also
// returns the AND of every participant's pred: a decision all of them share.
__device__ __forceinline__ bool named_barrier_and(uint32_t id, uint32_t nthreads, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"(pred ? 1u : 0u), "r"(id), "r"(nthreads)
      : "memory");
  return r != 0;
}
// Every thread of every CTA of the cluster (release / acquire).
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// A tensor map read from global memory (a device table written by a copy):
// order the tensor-map proxy's view of it after that write.
__device__ __forceinline__ void tmap_acquire(const CUtensorMap* m) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(m))
               : "memory");
}
__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}
// L2 prefetch of one box of a 2-D tensor map (a hint: it moves no data into
// shared memory and completes nothing; L2 is the coherence point of global
// memory, so a later load still sees every write made before it).
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap* map, int c0, int c1) {
  asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(c0), "r"(c1)
               : "memory");
}

// ---- TMEM ---------------------------------------------------------------------
// Executed by one full warp; writes the TMEM base address to *slot.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// CTA-pair forms (a cluster of two CTAs on one TPC; every tcgen05 instruction
// of such a kernel takes cta_group::2): one warp of EACH CTA of the pair
// executes the allocation (the same columns in both CTAs' TMEM), the
// relinquish and the deallocation.
__device__ __forceinline__ void tmem_alloc_pair(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish_pair() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// ---- descriptors ----------------------------------------------------------------
// Shared-memory matrix descriptor of a K-major operand tile stored with the
// 128-byte swizzle (the layout TMA writes with CU_TENSOR_MAP_SWIZZLE_128B):
// rows of 128 bytes (64 BF16 along K), 8-row groups 1024 bytes apart.  The
// tile must start on a 1024-byte boundary.  Advancing along K inside the
// 128-byte row is done by adding (bytes >> 4) to the start-address field.
__device__ __forceinline__ uint64_t sdesc_kmajor_sw128(const void* tile) {
  const uint64_t addr = smem_u32(tile);
  uint64_t d = (addr >> 4) & 0x3FFFull;      // bits  0-13: start address >> 4
  d |= 1ull << 16;                           // bits 16-29: leading byte offset (unused here) = 16 B
  d |= (uint64_t)(1024 >> 4) << 32;          // bits 32-45: stride byte offset = 1024 B
  d |= 1ull << 46;                           // bits 46-47: descriptor version 1
  d |= 2ull << 61;                           // bits 61-63: 128-byte swizzle
  return d;
}

// Shared-memory matrix descriptor of an MN-major operand tile with the
// 128-byte swizzle: rows of 128 bytes (64 BF16 along MN) for one K index,
// 8-K-row groups 1024 bytes apart (stride byte offset), and the next 64
// MN elements `lbo` bytes further (leading byte offset).  A K-major tile
// written by TMA with the 128-byte swizzle, [MN-chunk][rows][64], read with
// K = its rows and MN = its columns, is this layout with lbo = the chunk size.
__device__ __forceinline__ uint64_t sdesc_mnmajor_sw128(const void* tile, uint32_t lbo) {
  const uint64_t addr = smem_u32(tile);
  uint64_t d = (addr >> 4) & 0x3FFFull;      // bits  0-13: start address >> 4
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;  // bits 16-29: leading byte offset >> 4
  d |= (uint64_t)(1024 >> 4) << 32;          // bits 32-45: stride byte offset = 1024 B
  d |= 1ull << 46;                           // bits 46-47: descriptor version 1
  d |= 2ull << 61;                           // bits 61-63: 128-byte swizzle
  return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: BF16 A and B, FP32
// accumulator, both operands K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4)                             // D format: F32
         | (1u << 7)                           // A format: BF16
         | (1u << 10)                          // B format: BF16
         | (0u << 15) | (0u << 16)             // A, B K-major
         | ((uint32_t)(N >> 3) << 17)          // N / 8
         | ((uint32_t)(M >> 4) << 24);         // M / 16
}
// The same with B MN-major (bit 16).
__host__ __device__ constexpr uint32_t idesc_bf16_f32_bmn(int M, int N) { return idesc_bf16_f32(M, N) | (1u << 16); }

// D[tmem] (+)= A[smem] * B[smem]^T for one K = 16 slice.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// CTA-pair MMA, issued by one thread of the even CTA: D (M = 256 rows, the
// even CTA's TMEM lanes holding rows 0..127 and the odd CTA's rows 128..255,
// at the same TMEM address) (+)= A * B^T, where each CTA supplies its 128
// rows of A and its N / 2 rows of B at the same shared-memory offsets as the
// descriptors name in the issuing CTA.
__device__ __forceinline__ void mma_bf16_pair(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                              uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrive once on this CTA's `bar` when all previously issued CTA-pair MMAs of
// this thread complete (their writes to both CTAs' TMEM and their reads of
// both CTAs' shared memory).
__device__ __forceinline__ void mma_commit_pair(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// Arrive once on `bar` when all previously issued tcgen05 operations of this thread complete.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane (warp w reads lanes 32w..32w+31).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace tc
}  // namespace crl
