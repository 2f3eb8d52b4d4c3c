// Device helpers: ordered keys, mbarrier / bulk-copy PTX, bounded waits,
// warp-aggregated appends and the CTA radix select.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ebr {

// ------------------------------------------------------------ ranking keys
// A candidate is the 64-bit word  ord(score) << 32 | (0xFFFFFFFF - id):
// a larger word ranks first (higher score, then lower id) and words are
// unique because ids are.  ord() maps IEEE floats to unsigned integers with
// the same order; -0 is folded into +0 first.
__device__ __forceinline__ uint32_t ord_f32(float s) {
  s = s + 0.0f;
  uint32_t u = __float_as_uint(s);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float unord_f32(uint32_t o) {
  uint32_t u = (o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o;
  return __uint_as_float(u);
}
__device__ __forceinline__ uint64_t make_key(float s, uint32_t id) {
  return ((uint64_t)ord_f32(s) << 32) | (uint64_t)(0xFFFFFFFFu - id);
}
__device__ __forceinline__ uint32_t key_id(uint64_t k) { return 0xFFFFFFFFu - (uint32_t)k; }
__device__ __forceinline__ float key_score(uint64_t k) { return unord_f32((uint32_t)(k >> 32)); }

// ------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t cnt) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(cnt) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)),
               "r"(bytes)
               : "memory");
}
// 1-D bulk copy global -> shared (TMA engine), completion counted on mbarrier b.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(b))
      : "memory");
}
__device__ __forceinline__ uint32_t mbar_try_wait(uint64_t *b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok;
}
__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for phase `parity` of barrier b, giving up after timeout_ns.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *b, uint32_t parity,
                                                  uint64_t timeout_ns) {
  if (mbar_try_wait(b, parity)) return true;
  uint64_t t0 = global_timer_ns();
  while (!mbar_try_wait(b, parity)) {
    if (global_timer_ns() - t0 > timeout_ns) return false;
  }
  return true;
}

constexpr uint64_t kWaitTimeoutNs = 2000000000ull;  // 2 s

// ------------------------------------------------------- warp-aggregated append
// Lanes with pred reserve consecutive slots of *counter; returns the slot
// (undefined where !pred).  One atomic per warp.
__device__ __forceinline__ uint32_t warp_append(bool pred, uint32_t *counter) {
  const uint32_t mask = __activemask();
  const uint32_t ballot = __ballot_sync(mask, pred);
  if (!ballot) return 0;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(ballot) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(counter, (uint32_t)__popc(ballot));
  base = __shfl_sync(mask, base, leader);
  return base + __popc(ballot & ((1u << lane) - 1u));
}

// ------------------------------------------------------------ radix select
// Finds T such that exactly `need` of the n keys in buf are >= T (keys are
// unique).  8-bit digits from the top; stops as soon as the chosen digit's
// bucket is taken whole.  Collective over the CTA; hist holds 256 words and
// s_misc 4 words of shared memory.  Returns T to every thread.
template <int NT>
__device__ uint64_t cta_radix_select(const uint64_t *buf, uint32_t n, uint32_t need,
                                     uint32_t *hist, uint32_t *s_misc) {
  uint64_t prefix = 0;
  for (int shift = 56; shift >= 0; shift -= 8) {
    for (int i = threadIdx.x; i < 256; i += NT) hist[i] = 0;
    __syncthreads();
    const uint64_t hi_mask = (shift == 56) ? 0ull : (~0ull << (shift + 8));
    for (uint32_t i = threadIdx.x; i < n; i += NT) {
      uint64_t x = buf[i];
      if ((x & hi_mask) == prefix) atomicAdd(&hist[(x >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      // lane l owns bins 255-8l .. 248-8l (descending)
      const int lane = threadIdx.x;
      uint32_t c[8], tot = 0;
#pragma unroll
      for (int e = 0; e < 8; e++) {
        c[e] = hist[255 - 8 * lane - e];
        tot += c[e];
      }
      // exclusive prefix over lanes (counts of higher bins)
      uint32_t incl = tot;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      uint32_t above = incl - tot;
      if (above < need && need <= incl) {
        uint32_t acc = above;
#pragma unroll
        for (int e = 0; e < 8; e++) {
          if (acc < need && need <= acc + c[e]) {
            s_misc[0] = 255 - 8 * lane - e;  // digit
            s_misc[1] = need - acc;          // still needed inside the bucket
            s_misc[2] = (need - acc == c[e]) ? 1u : 0u;
          }
          acc += c[e];
        }
      }
    }
    __syncthreads();
    const uint32_t dg = s_misc[0];
    need = s_misc[1];
    const uint32_t whole = s_misc[2];
    prefix |= (uint64_t)dg << shift;
    __syncthreads();
    if (whole) break;
  }
  return prefix;
}

}  // namespace ebr
