// Device helpers: ordered keys, mbarrier / bulk-copy PTX, bounded waits,
// warp-aggregated appends and the CTA radix select.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

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
// Same, with an L2 cache-policy hint (e.g. evict-first for data read once).
__device__ __forceinline__ void bulk_g2s_hint(void *dst, const void *src, uint32_t bytes,
                                              uint64_t *b, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(b)), "l"(policy)
      : "memory");
}
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
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
// The same test, letting the hardware suspend the thread for up to
// suspend_ns (or until the phase completes, whichever comes first) instead
// of returning at once: a waiting warp then issues almost nothing.
__device__ __forceinline__ uint32_t mbar_try_wait_suspend(uint64_t *b, uint32_t parity,
                                                          uint32_t suspend_ns) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity), "r"(suspend_ns)
      : "memory");
  return ok;
}
// Wait for phase `parity` of barrier b, giving up after timeout_ns.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *b, uint32_t parity,
                                                  uint64_t timeout_ns) {
  if (mbar_try_wait(b, parity)) return true;
  uint64_t t0 = global_timer_ns();
  while (!mbar_try_wait_suspend(b, parity, 1000000u)) {
    if (global_timer_ns() - t0 > timeout_ns) return false;
  }
  return true;
}

constexpr uint64_t kWaitTimeoutNs = 2000000000ull;  // 2 s

// Plain arrive (release semantics) on an mbarrier.
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
// Programmatic dependent launch: pdl_wait blocks the calling thread until
// the grids it depends on have completed and their writes are visible (a
// no-op when the kernel was launched without the attribute); pdl_trigger lets
// the next kernel of the stream be scheduled before this one ends.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Barrier over a subset of the CTA's warps (hardware named barrier `id`).
__device__ __forceinline__ void named_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

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
struct CtaSync {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
// Two FP32 adds in one instruction (round to nearest even in each lane, as
// two scalar adds).
__device__ __forceinline__ float2 add_f32x2(float2 a, float2 b) {
  uint64_t ra, rb, rd;
  asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
  float2 d;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(rd));
  return d;
}

struct GroupSync {  // named barrier over the first `n` threads of the CTA
  int id, n;
  __device__ __forceinline__ void operator()() const { named_sync(id, n); }
};

// Generic form: `t` is the caller's index in its group of NT threads (the
// first warp of the group computes the digit), `sync` synchronises the group.
template <int NT, typename Sync>
__device__ uint64_t group_radix_select(const uint64_t *buf, uint32_t n, uint32_t need,
                                       uint32_t *hist, uint32_t *s_misc, int t, Sync sync) {
  uint64_t prefix = 0;
  for (int shift = 56; shift >= 0; shift -= 8) {
    for (int i = t; i < 256; i += NT) hist[i] = 0;
    sync();
    const uint64_t hi_mask = (shift == 56) ? 0ull : (~0ull << (shift + 8));
    for (uint32_t i = t; i < n; i += NT) {
      uint64_t x = buf[i];
      if ((x & hi_mask) == prefix) {
        // aggregate equal digits within the warp: one atomic per distinct digit
        const uint32_t dg = (uint32_t)(x >> shift) & 255u;
        const uint32_t peers = __match_any_sync(__activemask(), dg);
        if ((threadIdx.x & 31) == (uint32_t)(__ffs(peers) - 1))
          atomicAdd(&hist[dg], (uint32_t)__popc(peers));
      }
    }
    sync();
    if (t < 32) {
      // lane l owns bins 255-8l .. 248-8l (descending)
      const int lane = t;
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
    sync();
    const uint32_t dg = s_misc[0];
    need = s_misc[1];
    const uint32_t whole = s_misc[2];
    prefix |= (uint64_t)dg << shift;
    sync();
    if (whole) break;
  }
  return prefix;
}

template <int NT>
__device__ uint64_t cta_radix_select(const uint64_t *buf, uint32_t n, uint32_t need,
                                     uint32_t *hist, uint32_t *s_misc) {
  return group_radix_select<NT>(buf, n, need, hist, s_misc, threadIdx.x, CtaSync());
}

// ---------------------------------------------- histogram threshold (K-th bound)
// hist_c[256] counts candidates by the top 8 bits of ord(score), hist_f[65536]
// by the top 16 bits.  Every counted candidate is a distinct ad, so if at
// least K counted candidates have ord(score) >= T, the K-th best score
// overall is >= T and anything below T can be dropped.  Returns the largest
// such T of the form (coarse, fine) << 16, as a key threshold (T << 32), or 0.
// Counts only grow, so racy snapshots give a smaller, still valid, bound.
// Called by one full warp.
__device__ __forceinline__ uint64_t hist_threshold(const uint32_t *hist_c, const uint32_t *hist_f,
                                                   uint32_t K) {
  const int lane = threadIdx.x & 31;
  uint32_t c[8], tot = 0;
#pragma unroll
  for (int e = 0; e < 8; e++) {
    c[e] = __ldcg(hist_c + 255 - 8 * lane - e);
    tot += c[e];
  }
  uint32_t incl = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  int cb = -1;
  uint32_t above_c = 0;
  {
    uint32_t acc = incl - tot;
    int found = -1;
    uint32_t fa = 0;
#pragma unroll
    for (int e = 0; e < 8; e++) {
      if (found < 0 && acc < K && K <= acc + c[e]) {
        found = 255 - 8 * lane - e;
        fa = acc;
      }
      acc += c[e];
    }
    const uint32_t bal = __ballot_sync(0xffffffffu, found >= 0);
    if (!bal) return 0ull;
    const int src = __ffs(bal) - 1;
    cb = __shfl_sync(0xffffffffu, found, src);
    above_c = __shfl_sync(0xffffffffu, fa, src);
  }
  const uint32_t *hf = hist_f + (uint32_t)cb * 256u;
  tot = 0;
#pragma unroll
  for (int e = 0; e < 8; e++) {
    c[e] = __ldcg(hf + 255 - 8 * lane - e);
    tot += c[e];
  }
  incl = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  uint32_t acc = above_c + incl - tot;
  int found = -1;
#pragma unroll
  for (int e = 0; e < 8; e++) {
    if (found < 0 && acc < K && K <= acc + c[e]) found = 255 - 8 * lane - e;
    acc += c[e];
  }
  const uint32_t bal = __ballot_sync(0xffffffffu, found >= 0);
  if (!bal) return ((uint64_t)((uint32_t)cb << 24)) << 32;  // coarse bound only
  const int fb = __shfl_sync(0xffffffffu, found, __ffs(bal) - 1);
  return ((uint64_t)(((uint32_t)cb << 24) | ((uint32_t)fb << 16))) << 32;
}

// ------------------------------------------------- fixed-point wide terms
// The window accumulators hold each ad's wide term in 32-bit fixed point
// (shared-memory integer atomics run several times faster than FP32 or 64-bit
// ones on this part, and an integer sum does not depend on the order of the
// additions), in three exponent classes plus an FP32 remainder:
//   a weight w is turned into a term of class c in {0, 1, 2}, the first one
//   with |w| * 2^(F + c S) >= 2^kFixMinBits, and adds f = round(w * 2^(F + c S))
//   to accumulator c; a weight below all three classes is added in FP32.
// The ad's wide term is sum_c acc_c * 2^-(F + c S) + acc_fp32.  Every integer
// term has at least kFixMinBits significant bits, so its rounding error is
// below 2^-(kFixMinBits + 1) of the term: each ad's error is bounded by about
// 2^-19 of the sum of its own terms' magnitudes (plus the FP32 error of its
// smallest terms), whatever the range of w^ over the request.
// F is the largest power of two with max|w^| * 2^F <= min(2^28, 2^31 / (most
// keys of one ad)), and S <= 12 - ceil(log2(most keys of one ad)), so no
// class sum can overflow and a term packs into 30 bits:
//   packed = f << 2 | c, or the FP32 bits of w with the low two bits set to 3
//   (class 3, FP32), or 0 for a zero weight.
constexpr int kFixMinBits = 18;
__host__ __device__ __forceinline__ int fix_exponent(float wmax, uint32_t max_keys) {
  if (!(wmax > 0.f) || !(wmax < 3.0e38f)) return 0;
  const float mk = (float)(max_keys > 1u ? max_keys : 1u);
  const float lim = (2147483647.0f - mk) / mk;
  const float limit = lim < 268435456.0f ? lim : 268435456.0f;  // max |f| of class 0
  const float r = limit / wmax;
  uint32_t rb;
  memcpy(&rb, &r, 4);
  int e = (int)((rb >> 23) & 0xFFu) - 127;  // floor(log2 r), r normal
  if (e > 100) e = 100;
  if (e < -100) e = -100;
  return e;
}
__host__ __device__ __forceinline__ float pow2f(int e) {
  const uint32_t b = (uint32_t)(127 + e) << 23;
  float f;
  memcpy(&f, &b, 4);
  return f;
}
// S for an index whose ads hold at most max_keys keys (0: no classes 1 and 2)
inline int class_shift(uint32_t max_keys) {
  int lg = 0;
  while ((1u << lg) < std::max<uint32_t>(max_keys, 1u)) lg++;
  return std::max(0, std::min(10, 12 - lg));
}
// The packed term of weight v (see above); s0 = 2^F, s1 = 2^(F+S), s2 = 2^(F+2S).
__device__ __forceinline__ uint32_t pack_term(float v, float s0, float s1, float s2, bool cls12) {
  if (v == 0.f) return 0u;
  constexpr float kMin = (float)(1 << kFixMinBits);
  const float a = fabsf(v);
  float sc;
  uint32_t c;
  if (a * s0 >= kMin) {
    sc = s0;
    c = 0u;
  } else if (cls12 && a * s1 >= kMin) {
    sc = s1;
    c = 1u;
  } else if (cls12 && a * s2 >= kMin) {
    sc = s2;
    c = 2u;
  } else {
    return (__float_as_uint(v) & ~3u) | 3u;
  }
  return ((uint32_t)__float2int_rn(v * sc) << 2) | c;
}

// ------------------------------------------------------- embedding rows
// Scan element types: a 16-byte vector holds kVec elements, widened to float.
template <typename Elt> struct EltTraits;
template <> struct EltTraits<float> {
  static constexpr int kBytes = 4;
  static constexpr int kVec = 4;  // elements per 16-byte vector
  __device__ static __forceinline__ void load(const uint4 &v, float *f) {
    f[0] = __uint_as_float(v.x);
    f[1] = __uint_as_float(v.y);
    f[2] = __uint_as_float(v.z);
    f[3] = __uint_as_float(v.w);
  }
};
struct Bf16Tag {};
template <> struct EltTraits<Bf16Tag> {
  static constexpr int kBytes = 2;
  static constexpr int kVec = 8;
  __device__ static __forceinline__ void load(const uint4 &v, float *f) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; i++) {
      f[2 * i] = __uint_as_float(w[i] << 16);
      f[2 * i + 1] = __uint_as_float(w[i] & 0xFFFF0000u);
    }
  }
};
struct Fp8Tag {};
// Four E4M3 bytes (byte k of w is element k) -> FP32, with the hardware
// converters: each pair of bytes to an FP16 pair, then each FP16 to FP32.
// Both steps are exact: every E4M3 value is an FP16 value.  (The all-ones
// NaN codes, which the library's quantiser never writes, become NaN.)
__device__ __forceinline__ void e4m3x4_to_f32(uint32_t w, float *f) {
  uint32_t h01, h23;
  asm("{\n .reg .b16 lo, hi;\n mov.b32 {lo, hi}, %2;\n"
      " cvt.rn.f16x2.e4m3x2 %0, lo;\n cvt.rn.f16x2.e4m3x2 %1, hi;\n}"
      : "=r"(h01), "=r"(h23)
      : "r"(w));
  asm("{\n .reg .f16 x, y;\n mov.b32 {x, y}, %2;\n cvt.f32.f16 %0, x;\n cvt.f32.f16 %1, y;\n}"
      : "=f"(f[0]), "=f"(f[1])
      : "r"(h01));
  asm("{\n .reg .f16 x, y;\n mov.b32 {x, y}, %2;\n cvt.f32.f16 %0, x;\n cvt.f32.f16 %1, y;\n}"
      : "=f"(f[2]), "=f"(f[3])
      : "r"(h23));
}
template <> struct EltTraits<Fp8Tag> {
  static constexpr int kBytes = 1;
  static constexpr int kVec = 16;
  __device__ static __forceinline__ void load(const uint4 &v, float *f) {
    e4m3x4_to_f32(v.x, f);
    e4m3x4_to_f32(v.y, f + 4);
    e4m3x4_to_f32(v.z, f + 8);
    e4m3x4_to_f32(v.w, f + 12);
  }
};


}  // namespace ebr
