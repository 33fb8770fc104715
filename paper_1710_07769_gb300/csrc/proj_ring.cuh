// Shared pieces of the projection kernels: a ring of shared-memory slots that one
// producer warp fills with cp.async.bulk copies of factor tiles and 8 consumer warps
// drain in order, guarded by full/empty mbarriers.  full[s] completes when a copy has
// landed, empty[s] when all 8 consumer warps have passed the slot.  Every wait is
// bounded by %globaltimer; a wait that runs out sets the abort flag and the error word.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.cuh"

namespace cimmino {
namespace ring {

constexpr int T = kTile;
constexpr int kConsumers = 256;
constexpr int kProjThreads = kConsumers + 32;
constexpr uint32_t kWaitSpins = 1u << 30;
constexpr uint64_t kWaitNs = 2000000000ull;  // bounded waits give up after ~2 s

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait: try_wait suspends the thread in hardware until the phase completes (or
// its own time slice ends), so no sleep is added; give up after about two seconds.
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity) {
  if (mbar_try_wait(b, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t i = 0; i < kWaitSpins; ++i) {
    if (mbar_try_wait(b, parity)) return true;
    if (global_ns() - t0 > kWaitNs) return false;
  }
  return false;
}
// L2 policy for the factor stream: each tile is read once per pass and the stream is
// several times larger than L2, so its lines go first; the Gram copy, A, A^T and the
// vectors that every CG iteration re-reads keep their place in L2.
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}
// consumer-only barrier (8 warps) and whole-CTA barrier (consumers + producer)
__device__ __forceinline__ void csync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
__device__ __forceinline__ void allsync() { asm volatile("bar.sync 2, 288;" ::: "memory"); }

struct Ring {
  unsigned char *base;
  uint64_t *full;
  uint64_t *empty;
  uint32_t slots;
  uint32_t slot_bytes;
  int *abort;
};

// consumer side: wait for tile t, return its slot
__device__ __forceinline__ const void *slot_acquire(const Ring &R, uint32_t t, int32_t *err) {
  const uint32_t s = t % R.slots;
  if (!*(volatile int *)R.abort) {
    if (!mbar_wait(&R.full[s], (t / R.slots) & 1u)) {
      *(volatile int *)R.abort = 1;
      atomicOr(err, 1);
    }
  }
  return R.base + (size_t)s * R.slot_bytes;
}
__device__ __forceinline__ void slot_release(const Ring &R, uint32_t t) {
  __syncwarp();
  if ((threadIdx.x & 31) == 0) mbar_arrive(&R.empty[t % R.slots]);
}

// producer side: once the slot of tile t is free, copy `bytes` from src into it; t advances
__device__ __forceinline__ void slot_fill(const Ring &R, uint32_t &t, const void *src,
                                          uint32_t bytes, int32_t *err) {
  const uint32_t s = t % R.slots;
  if (!*(volatile int *)R.abort) {
    if (t >= R.slots && !mbar_wait(&R.empty[s], ((t / R.slots) - 1u) & 1u)) {
      *(volatile int *)R.abort = 1;
      atomicOr(err, 2);
    } else {
      mbar_expect_tx(&R.full[s], bytes);
      bulk_g2s(R.base + (size_t)s * R.slot_bytes, src, bytes, &R.full[s], l2_evict_first());
    }
  }
  ++t;
}

// set up the ring's mbarriers (one thread), before the CTA's first barrier
__device__ __forceinline__ void ring_init(const Ring &R) {
  for (uint32_t s = 0; s < R.slots; ++s) {
    mbar_init(&R.full[s], 1);
    mbar_init(&R.empty[s], kConsumers / 32);
  }
  *R.abort = 0;
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// the producer lane waits for its own copies still in flight before the CTA exits
__device__ __forceinline__ void ring_drain(const Ring &R, uint32_t t) {
  const uint32_t first = t > R.slots ? t - R.slots : 0u;
  for (uint32_t v = first; v < t; ++v) mbar_wait(&R.full[v % R.slots], (v / R.slots) & 1u);
}

}  // namespace ring
}  // namespace cimmino
