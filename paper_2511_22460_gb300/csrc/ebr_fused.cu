// Fused window-major scan for requests whose query covers the whole key space.
//
// The wide term of the HitMatch equation (Sec. 3.3) is accumulated per window
// of 256 consecutive ads -- the block granularity of Algorithm 1 (ads sharing
// ad >> 8) -- from the window-major view of the compressed inverted list, in
// shared memory, and added to the dual-tower inner product (Eq. 1) of the same
// ads as their embedding rows stream through; the K best survive in a per-CTA
// buffer (in shared memory, or in global memory when a large K would crowd
// out the index slots).  Neither the wide term nor the score vector is
// written to global memory.
//
// One persistent CTA per SM, three warp roles:
//   producers (2 warps, independent): one stages every window's
//       compressed-list segments (keys and value bytes of all nine size
//       groups) into a ring of index slots (two per decoder team when shared
//       memory allows), the other streams its embedding rows into a ring of
//       16 KB stages; all by TMA bulk copies (cp.async.bulk + mbarrier, L2
//       evict-first);
//   decoders (2 teams x 5 warps): each team takes every other window; warps
//       walk the window's blocks in chunks of 32 work units of one size group,
//       gather w^[key] and add it into one of four fixed-point accumulators
//       of 256 ads (one 32-bit integer atomic per real ad slot);
//   scorers (8 warps): one thread per row (two for 128-element rows) forms the
//       inner product with its permuted copy of h_u held in registers (each
//       thread reads the row's 16-byte chunks in its own order, so that
//       neighbouring rows hit other banks), adds the window's accumulator
//       (and the FP8 row scale), applies the filter and appends candidates;
//       a radix select trims the buffer to the K best.
// All hand-offs are mbarrier phases; every wait is bounded (2 s) and a CTA
// that times out flags the request and drains its copies.
#include <algorithm>
#include <cstring>
#include <type_traits>

#include "ebr_device.cuh"
#include "ebr_internal.cuh"

namespace ebr {

constexpr int kWin = 256;
constexpr int kDotWarps = 8, kTeamWarps = 5, kTeams = 2;
constexpr int kDotThreads = kDotWarps * 32;
constexpr int kTeamThreads = kTeamWarps * 32;
constexpr int kIdxWarp = kDotWarps + kTeams * kTeamWarps;  // index producer
constexpr int kEmbWarp = kIdxWarp + 1;                       // embedding producer
constexpr int kFusedThreads = (kEmbWarp + 1) * 32;           // 640 (20 warps)
constexpr int kAccBufs = 4;
constexpr int kMaxIdxSlots = 2 * kTeams;  // two per decoder team when they fit
constexpr int kStageBytes = 16384;
constexpr int kMaxStages = 12;
constexpr int kMinStages = 4;
constexpr int kChunksInFlight = 8;  // decoder chunks of 32 units per warp per round
constexpr int kMaxChunkTab = 512;  // chunk -> (group, chunk in group) table per team
static_assert(kWin % kDotThreads == 0, "scorer threads split the window evenly");
static_assert(kMaxIdxSlots % kTeams == 0, "window j uses slot j % slots, team j % kTeams");

struct FusedArgs {
  const void *emb;
  const float *scale;
  const float *h_u;
  const uint32_t *wq;  // dense over keys: packed fixed-point weight terms (pack_term)
  const uint32_t *wkey[kGroups];
  const uint8_t *wvals[kGroups];
  const uint32_t *win_ptr[kGroups];
  const uint64_t *filter;
  uint32_t n_ads, n_win, k, cap, stages, slot_bytes, idx_slots;
  uint64_t *cand_out;
  uint64_t *cand_g;   // if set: the CTAs' candidate buffers (cap entries each) live here, in
                      // global memory, instead of in shared memory
  Ctrl *ctrl;
  float *all_out;   // score-all mode
  float *wide_out;  // if set: the per-ad wide term is written here (FP32 rescoring needs it)
  uint32_t *hist;   // [kCandBins + 1] candidate-score histogram + top bin (zeroed per request)
  const int *fx_word;         // F of the packed terms (written with them)
  const float *wide_in;       // if set: the per-ad wide term, already summed (Algorithm 2
                              // scattered it); no window is decoded
  const uint32_t *route;      // if set: *route != 0 (decided on the device) ignores wide_in
                              // and decodes the windows with wq after all
  uint32_t max_keys;          // most keys of one ad
  int cls_shift;              // S: exponent step between the integer term classes
};

template <typename Elt, int D>
struct FusedShape {
  static constexpr int kRowBytes = D * EltTraits<Elt>::kBytes;
  static constexpr int kChunks = kRowBytes / 16;                 // 16-byte chunks per row
  static constexpr int kRowsPerStage =                           // rows per stage
      (kStageBytes / kRowBytes) < kWin ? (kStageBytes / kRowBytes) : kWin;
  static constexpr int kStagesPerWin = kWin / kRowsPerStage;
  static constexpr int kTPR = D > 64 ? D / 64 : 1;               // scorer threads per row
  static constexpr int kCPT = kChunks / kTPR;                    // chunks per scorer thread
  static constexpr int kRowsPerPass = kDotThreads / kTPR;
  static constexpr int kPasses = kWin / kRowsPerPass;
  static constexpr int kRowsPer128 = kRowBytes >= 128 ? 1 : 128 / kRowBytes;
  static constexpr int kHPT = kCPT * EltTraits<Elt>::kVec;       // h_u entries per thread
  static_assert(kRowsPerStage <= kWin && kWin % kRowsPerStage == 0, "stage split");
  static_assert(kRowsPerStage % (32 / kTPR) == 0, "a warp's rows lie in one stage");
  static_assert(kTPR >= 1 && kCPT >= 1 && kHPT <= 64, "row split");
};

__device__ __forceinline__ uint32_t unit_shift_f(uint32_t g) { return g >= 2 ? g - 2 : 0; }

struct SlotDesc {                // one window's staged segments
  uint32_t key_off[kGroups];     // byte offset of the window's first key in the slot
  uint32_t val_off[kGroups];     // byte offset of its first value byte
  uint32_t nblk[kGroups];        // blocks of the window in group g
  uint32_t window;
};

constexpr int kPrefetch = 4;  // producer reads window offsets this many windows ahead

// Candidate-score histogram shared by all CTAs (for a global K-th bound):
// bins are the top 11 bits of the order-preserving score key (sign, 8
// exponent bits, 2 mantissa bits).  CTAs count in shared memory and add
// their counts to the global histogram every kRefresh windows.
constexpr int kCandBins = 2048;
constexpr int kBinShift = 53;
constexpr int kRefresh = 2;

// Largest bin edge b << kBinShift with at least K candidates at or above it,
// scanning the global histogram down from its highest bin to bin b_lo (a
// bound already known); 0 if none.  Counts only grow, so racy snapshots give
// a smaller, still valid, bound.  One full warp.
__device__ __forceinline__ uint64_t hist_top_threshold(const uint32_t *gh, uint32_t b_lo,
                                                       uint32_t K) {
  const int lane = threadIdx.x & 31;
  const int top = (int)min(__ldcg(gh + kCandBins), (uint32_t)kCandBins - 1u);
  uint32_t run = 0;
  for (int hi = top; hi >= (int)b_lo; hi -= 32) {
    const int bin = hi - lane;
    const uint32_t c = bin >= (int)b_lo ? __ldcg(gh + bin) : 0u;
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    const uint32_t hit = __ballot_sync(0xffffffffu, run + incl >= K);
    if (hit) {
      const int src = __ffs(hit) - 1;
      return (uint64_t)(hi - src) << kBinShift;
    }
    run += __shfl_sync(0xffffffffu, incl, 31);
  }
  return 0ull;
}

__device__ __forceinline__ uint32_t lds_u32(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ uint4 lds_v4(uint32_t a) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(a));
  return v;
}
__device__ __forceinline__ void red_add_s32(uint32_t a, int v) {
  asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void red_add_f32(uint32_t a, float v) {
  asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}

struct AccBuf {         // one window's accumulators (see pack_term)
  int cls[3][kWin];     // integer term classes 0, 1, 2
  float fp[kWin];       // FP32 remainder
};

struct FusedSmem {
  AccBuf acc[kAccBufs];
  uint32_t wp[kPrefetch][kGroups];  // producer's ring of window offsets
  uint32_t ctab[kTeams][kMaxChunkTab];  // per team: group << 16 | chunk within the group
  // per team and size group of the current window: shared address of its
  // block keys (packed terms), of its value bytes, its units, and
  // unit shift | (value-load shift << 8)
  uint4 gtab[kTeams][kGroups];
  SlotDesc desc[kMaxIdxSlots];
  uint32_t hist[256];
  uint32_t chist[kCandBins];  // this CTA's candidates per score bin since the last flush
  uint32_t top_bin;           // highest bin this CTA has seen
  uint32_t misc[8];
  uint32_t wtot[2][kDotWarps];
  uint64_t full[kMaxStages], empty[kMaxStages], acc_full[kAccBufs], acc_empty[kAccBufs];
  uint64_t idx_full[kMaxIdxSlots], idx_empty[kMaxIdxSlots];
  unsigned long long thr;
  uint32_t n, abort;
  // group-uniform stop decisions: written by one thread before a barrier of
  // its group, read by all after it (a named barrier must never be skipped
  // by only part of its group)
  uint32_t stop_acc, stop_end, team_stop[kTeams];
};

// GC: the candidate buffers are in global memory (a.cand_g).
template <typename Elt, int D, bool ALL, bool GC>
__global__ void __maxnreg__(96) k_fused_window(FusedArgs a) {
  using Sh = FusedShape<Elt, D>;
  using Tr = EltTraits<Elt>;
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ FusedSmem sm;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t S = a.stages;
  uint8_t *stage0 = smem;
  uint8_t *slot0 = smem + (size_t)S * kStageBytes;
  float *s_h = reinterpret_cast<float *>(slot0 + (size_t)a.idx_slots * a.slot_bytes);
  uint64_t *cand = GC ? a.cand_g + (size_t)blockIdx.x * a.cap
                     : reinterpret_cast<uint64_t *>(s_h + D);

  // a contiguous, balanced range of windows per CTA: one sequential stream per SM
  const uint32_t w_begin = (uint32_t)(((uint64_t)a.n_win * blockIdx.x) / gridDim.x);
  const uint32_t w_end = (uint32_t)(((uint64_t)a.n_win * (blockIdx.x + 1)) / gridDim.x);
  const uint32_t my_wins = w_end - w_begin;

  pdl_trigger();  // the final selection may be scheduled behind this grid
  for (int i = tid; i < kAccBufs * 4 * kWin; i += kFusedThreads)
    reinterpret_cast<int *>(&sm.acc[0])[i] = 0;  // FP32 +0.0 has the same bits
  for (int i = tid; i < D; i += kFusedThreads) s_h[i] = a.h_u[i];
  for (int i = tid; i < kCandBins; i += kFusedThreads) sm.chist[i] = 0;
  if (tid == 0) {
    sm.n = 0;
    sm.abort = 0;
    sm.thr = 0ull;
    sm.top_bin = 0;
    for (uint32_t q = 0; q < S; q++) {
      mbar_init(&sm.full[q], 1);
      mbar_init(&sm.empty[q], Sh::kRowsPerStage * Sh::kTPR);  // every scorer visit of a row
    }
    for (int q = 0; q < kAccBufs; q++) {
      mbar_init(&sm.acc_full[q], kTeamThreads);
      mbar_init(&sm.acc_empty[q], kDotThreads);
    }
    for (int q = 0; q < kMaxIdxSlots; q++) {
      mbar_init(&sm.idx_full[q], 1);
      mbar_init(&sm.idx_empty[q], 1);
    }
    fence_mbar_init();
  }
  __syncthreads();

  if (warp == kEmbWarp) {
    // --------------------------------------------- embedding producer
    // Lane 0 streams every window's embedding rows into the stage ring.
    if (lane != 0) return;
    const uint64_t pol = l2_evict_first_policy();
    uint32_t seq = 0;  // stages issued
    bool stop = false;
    for (uint32_t j = 0; j < my_wins && !stop; j++) {
      const uint32_t w = w_begin + j;
      for (uint32_t q = 0; q < (uint32_t)Sh::kStagesPerWin; q++) {
        const uint32_t s = seq % S;
        if (seq >= S && !mbar_wait_bounded(&sm.empty[s], ((seq / S) - 1) & 1u, kWaitTimeoutNs)) {
          atomicOr(&a.ctrl->flags, DEVERR_TIMEOUT);
          sm.abort = 1;
          stop = true;
          break;
        }
        if (*((volatile uint32_t *)&sm.abort)) {
          stop = true;
          break;
        }
        const uint32_t row0 = w * kWin + q * Sh::kRowsPerStage;
        const uint32_t rows =
            row0 < a.n_ads ? min((uint32_t)Sh::kRowsPerStage, a.n_ads - row0) : 0u;
        if (rows) {
          mbar_arrive_expect_tx(&sm.full[s], rows * Sh::kRowBytes);
          bulk_g2s_hint(stage0 + (size_t)s * kStageBytes,
                        reinterpret_cast<const uint8_t *>(a.emb) + (uint64_t)row0 * Sh::kRowBytes,
                        rows * Sh::kRowBytes, &sm.full[s], pol);
        } else {
          mbar_arrive(&sm.full[s]);
        }
        seq++;
      }
    }
    if (stop)  // stopped early: wait (bounded) for the stage copies still in flight
      for (uint32_t q = (seq > S ? seq - S : 0); q < seq; q++)
        mbar_wait_bounded(&sm.full[q % S], (q / S) & 1u, kWaitTimeoutNs / 4);
    return;
  }

  // Everything below reads what the kernels before this one wrote (the
  // packed terms, their exponent, the route word): wait for them.  The
  // embedding producer above streams rows meanwhile.
  pdl_wait();
  // whether the wide term comes precomputed (no window decoding) in this launch
  const bool pre = a.wide_in != nullptr && !(a.route && *a.route);
  const int fx_e = *a.fx_word;
  // unit of each accumulator class: 2^-(F + c S)
  const float u0 = pow2f(-fx_e), u1 = pow2f(-fx_e - a.cls_shift),
              u2 = pow2f(-fx_e - 2 * a.cls_shift);

  if (warp == kIdxWarp) {
    // ------------------------------------------------- index producer
    // Lane g (< 9) stages window w's segment of size group g (its block keys
    // and value bytes) into index slot j % idx_slots as soon as the decoder
    // team that used the slot last has handed it back.
    const uint64_t pol = l2_evict_first_policy();
    const uint32_t NI = a.idx_slots;
    bool stop = false;
    if (lane < kGroups)
      for (uint32_t p = 0; p < (uint32_t)kPrefetch && p <= my_wins; p++)
        sm.wp[p][lane] = a.win_ptr[lane][w_begin + p];
    __syncwarp();
    // win_ptr[lane][w_begin + j - 1 + kPrefetch], loaded one iteration ago: it
    // is stored into the ring only now, so the load's latency is covered by a
    // whole iteration instead of stalling the one that issued it
    uint32_t pend_ptr = 0;
    bool pend = false;
    uint32_t issued = 0;
    for (uint32_t j = 0; j < my_wins && !stop; j++) {
      if (pend) sm.wp[(j - 1) % kPrefetch][lane] = pend_ptr;  // the slot of window j - 1
      __syncwarp();
      pend = lane < kGroups && j + kPrefetch <= my_wins;
      if (pend) pend_ptr = a.win_ptr[lane][w_begin + j + kPrefetch];
      const uint32_t w = w_begin + j;
      const uint32_t sl = j % NI, use = j / NI;
      if (use > 0) {
        bool ok = true;
        if (lane == 0) ok = mbar_wait_bounded(&sm.idx_empty[sl], (use - 1) & 1u, kWaitTimeoutNs);
        ok = __shfl_sync(0xffffffffu, ok, 0);
        const bool ab = __shfl_sync(0xffffffffu, *((volatile uint32_t *)&sm.abort) != 0, 0);
        if (!ok || ab) {
          if (lane == 0 && !ok) {
            atomicOr(&a.ctrl->flags, DEVERR_TIMEOUT);
            sm.abort = 1;
          }
          stop = true;
          break;
        }
      }
      // lane g (< 9): the segments of group g; 16-byte aligned, in group order
      // (all empty when the wide term comes precomputed)
      uint32_t lo = 0, hi = 0;
      if (lane < kGroups && !pre) {
        lo = sm.wp[j % kPrefetch][lane];
        hi = sm.wp[(j + 1) % kPrefetch][lane];
      }
      const uint32_t g = lane;
      uint64_t k0 = 0, k1 = 0, v0 = 0, v1 = 0;
      if (lane < kGroups && hi > lo) {
        k0 = ((uint64_t)lo * 4) & ~15ull;
        k1 = ((uint64_t)hi * 4 + 15) & ~15ull;
        v0 = ((uint64_t)lo << g) & ~15ull;
        v1 = (((uint64_t)hi << g) + 15) & ~15ull;
      }
      const uint32_t mine = (uint32_t)((k1 - k0) + (v1 - v0));
      uint32_t incl = mine;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      const uint32_t cursor = incl - mine;
      const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
      uint8_t *slot = slot0 + (size_t)sl * a.slot_bytes;
      if (lane < kGroups) {
        SlotDesc &dsc = sm.desc[sl];
        dsc.nblk[g] = hi - lo;
        // empty groups get in-slot offsets too: the decoders' predicated
        // reads may touch them (and discard what they read)
        dsc.key_off[g] = hi > lo ? cursor + (uint32_t)((uint64_t)lo * 4 - k0) : 0u;
        dsc.val_off[g] =
            hi > lo ? cursor + (uint32_t)(k1 - k0) + (uint32_t)(((uint64_t)lo << g) - v0) : 0u;
        if (lane == 0) dsc.window = w;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive_expect_tx(&sm.idx_full[sl], total);  // release: descriptor
      __syncwarp();
      if (lane < kGroups && hi > lo) {
        bulk_g2s_hint(slot + cursor, reinterpret_cast<const uint8_t *>(a.wkey[g]) + k0,
                      (uint32_t)(k1 - k0), &sm.idx_full[sl], pol);
        bulk_g2s_hint(slot + cursor + (uint32_t)(k1 - k0), a.wvals[g] + v0, (uint32_t)(v1 - v0),
                      &sm.idx_full[sl], pol);
      }
      issued = j + 1;
      if (!ALL && (j % kRefresh) == kRefresh - 1) {
        // raise this CTA's running threshold from the global candidate
        // histogram and the other CTAs' selections (off the scorers' path)
        const unsigned long long h =
            hist_top_threshold(a.hist, (uint32_t)(sm.thr >> kBinShift), a.k);
        if (lane == 0) {
          const unsigned long long g = *((volatile unsigned long long *)&a.ctrl->thr);
          atomicMax(&sm.thr, max(g, h));
        }
      }
      __syncwarp();
    }
    if (stop && lane == 0) {
      // stopped early: wait (bounded) for the index copies still in flight
      for (uint32_t j = issued > NI ? issued - NI : 0; j < issued; j++)
        mbar_wait_bounded(&sm.idx_full[j % NI], (j / NI) & 1u, kWaitTimeoutNs / 4);
    }
    return;
  }

  if (warp >= kDotWarps) {
    // ---------------------------------------------------------- decoders
    const int team = (warp - kDotWarps) / kTeamWarps;
    const int tw = (warp - kDotWarps) % kTeamWarps;  // warp within the team
    const int tt = tid - kDotThreads - team * kTeamThreads;
    for (uint32_t j = team; j < my_wins; j += kTeams) {
      const uint32_t b = j % kAccBufs, use = j / kAccBufs;
      const uint32_t sl = j % a.idx_slots, iuse = j / a.idx_slots;
      const uint8_t *slot = slot0 + (size_t)sl * a.slot_bytes;
      if (tt == 0) {
        uint32_t stop = *((volatile uint32_t *)&sm.abort);
        if (!stop && use > 0 &&
            !mbar_wait_bounded(&sm.acc_empty[b], (use - 1) & 1u, kWaitTimeoutNs))
          stop = 1;
        if (!stop && !mbar_wait_bounded(&sm.idx_full[sl], iuse & 1u, kWaitTimeoutNs)) stop = 1;
        if (stop && !*((volatile uint32_t *)&sm.abort)) {
          atomicOr(&a.ctrl->flags, DEVERR_TIMEOUT);
          sm.abort = 1;
        }
        sm.team_stop[team] = stop;
      }
      named_sync(2 + team, kTeamThreads);
      if (sm.team_stop[team]) break;
      if (use > 0) mbar_try_wait(&sm.acc_empty[b], (use - 1) & 1u);  // per-thread acquire
      mbar_try_wait(&sm.idx_full[sl], iuse & 1u);
      const SlotDesc &dsc = sm.desc[sl];
      // chunk prefix over the groups (chunks of 32 units never straddle groups)
      // and a chunk -> group table, one entry per thread, so the hot loop
      // below needs no search; per group the shared addresses and sizes the
      // hot loop reads with one 16-byte load
      uint32_t cpre[kGroups + 1];
      cpre[0] = 0;
#pragma unroll
      for (int g = 0; g < kGroups; g++)
        cpre[g + 1] = cpre[g] + (((dsc.nblk[g] << unit_shift_f(g)) + 31) >> 5);
      const uint32_t n_chunks = cpre[kGroups];
      uint32_t *tab = sm.ctab[team];
      for (uint32_t i = tt; i < n_chunks; i += kTeamThreads) {
        uint32_t g = 0;
#pragma unroll
        for (int t = 1; t < kGroups; t++) g += (i >= cpre[t]) ? 1u : 0u;
        uint32_t cb = 0;
#pragma unroll
        for (int t = 0; t < kGroups; t++) cb = (t == (int)g) ? cpre[t] : cb;
        tab[i] = (g << 16) | (i - cb);
      }
      if (tt < (uint32_t)kGroups) {
        const uint32_t g = tt, us = unit_shift_f(g);
        const uint32_t s_slot = smem_u32(slot);
        // a unit's value bytes start at byte (unit << vs) of the group's values:
        // one byte (g = 0), two (g = 1), or a 4-byte word (g >= 2)
        const uint32_t vs = g >= 2 ? 2u : g;
        sm.gtab[team][g] = make_uint4(s_slot + dsc.key_off[g], s_slot + dsc.val_off[g],
                                      dsc.nblk[g] << us, us | (vs << 8));
      }
      named_sync(2 + team, kTeamThreads);
      const uint32_t s_tab = smem_u32(tab), s_gtab = smem_u32(&sm.gtab[team][0]);
      const uint32_t s_acc = smem_u32(&sm.acc[b]);
      // Branch-free loads: every chunk's loads are independent of the
      // others', so the shared-memory reads and term gathers of a round
      // overlap; the additions then branch on the chunk's size group (uniform
      // across the warp), so a unit issues only the atomics its group can
      // need, into the accumulator of its term's class.
      for (uint32_t c0 = tw; c0 < n_chunks; c0 += kChunksInFlight * kTeamWarps) {
        uint32_t word[kChunksInFlight], key[kChunksInFlight], gq[kChunksInFlight];
        bool first[kChunksInFlight], valid[kChunksInFlight];
#pragma unroll
        for (int q = 0; q < kChunksInFlight; q++) {
          const uint32_t c = c0 + q * kTeamWarps;  // warp-uniform
          const bool cv = c < n_chunks;
          const uint32_t e = lds_u32(s_tab + 4 * (cv ? c : 0u));
          const uint32_t g = e >> 16;
          const uint4 gt = lds_v4(s_gtab + 16 * g);
          const uint32_t us = gt.w & 0xFFu, vs = gt.w >> 8;
          const uint32_t u = ((e & 0xFFFFu) << 5) + lane;
          const bool v = cv && u < gt.z;
          const uint32_t bk = v ? (u >> us) : 0u;
          key[q] = lds_u32(gt.x + 4 * bk);
          // the aligned 32-bit word holding this unit's 1, 2 or 4 value bytes
          const uint32_t va = gt.y + ((v ? u : 0u) << vs);
          const uint32_t w32 = lds_u32(va & ~3u);
          word[q] = (w32 >> ((va & 3u) << 3)) & (0xFFFFFFFFu >> (32u - (8u << vs)));
          gq[q] = cv ? g : 0xFFu;
          first[q] = (u & ((1u << us) - 1u)) == 0u;
          valid[q] = v;
        }
        uint32_t p[kChunksInFlight];
#pragma unroll
        for (int q = 0; q < kChunksInFlight; q++) p[q] = valid[q] ? __ldg(a.wq + key[q]) : 0u;
        uint32_t fl = 0;  // chunks whose term is FP32 (class 3)
#pragma unroll
        for (int q = 0; q < kChunksInFlight; q++) {
          const uint32_t g = gq[q];
          const uint32_t c = p[q] & 3u;
          const bool add = p[q] != 0u && c != 3u;
          fl |= (p[q] != 0u && c == 3u) ? (1u << q) : 0u;
          const int f = (int)p[q] >> 2;
          const uint32_t ac = s_acc + (c << 10);  // class c's 256 words
          if (g >= 2 && g < (uint32_t)kGroups) {
#pragma unroll
            for (int s2 = 0; s2 < 4; s2++) {
              const uint32_t l4 =
                  s2 == 0 ? (word[q] << 2) & 0x3FCu : (word[q] >> (8 * s2 - 2)) & 0x3FCu;
              if (add && ((s2 == 0 && first[q]) || l4 != 0u)) red_add_s32(ac + l4, f);
            }
          } else if (g == 1) {
            if (add) red_add_s32(ac + ((word[q] << 2) & 0x3FCu), f);  // slot 0 is real
            const uint32_t l4 = (word[q] >> 6) & 0x3FCu;
            if (add && l4 != 0u) red_add_s32(ac + l4, f);
          } else if (g == 0) {
            if (add) red_add_s32(ac + ((word[q] << 2) & 0x3FCu), f);
          }
        }
        if (__any_sync(0xffffffffu, fl != 0u)) {
          // weights too small for every integer class: FP32 additions
          const uint32_t af = s_acc + 3u * 1024u;
#pragma unroll
          for (int q = 0; q < kChunksInFlight; q++) {
            if (!((fl >> q) & 1u)) continue;
            const uint32_t g = gq[q];
            const float wv = __uint_as_float(p[q] & ~3u);
            const uint32_t ns = g >= 2 ? 4u : (g == 1 ? 2u : 1u);
            for (uint32_t s2 = 0; s2 < ns; s2++) {
              const uint32_t l = (word[q] >> (8 * s2)) & 255u;
              if ((s2 == 0 && (first[q] || g < 2)) || l != 0) red_add_f32(af + 4 * l, wv);
            }
          }
        }
      }
      named_sync(2 + team, kTeamThreads);  // every read of the slot and every addition done
      if (tt == 0) mbar_arrive(&sm.idx_empty[sl]);
      // fold the classes into one FP32 wide term per ad (in fp), and zero them
      for (uint32_t l = tt; l < (uint32_t)kWin; l += kTeamThreads) {
        AccBuf &ab = sm.acc[b];
        ab.fp[l] = ((float)ab.cls[0][l] * u0 + (float)ab.cls[1][l] * u1) +
                   ((float)ab.cls[2][l] * u2 + ab.fp[l]);
        ab.cls[0][l] = 0;
        ab.cls[1][l] = 0;
        ab.cls[2][l] = 0;
      }
      mbar_arrive(&sm.acc_full[b]);  // release: this thread's part of acc[b]
    }
    return;
  }

  // ------------------------------------------------------------ scorers
  const GroupSync gsync{1, kDotThreads};
  // this thread's row part and its rotated copy of h_u (constant for the kernel)
  const int qd = tid % Sh::kTPR;
  const int prow = tid / Sh::kTPR;              // row within a pass
  // 16-byte reads of neighbouring rows hit other banks: at step i a thread
  // reads chunk i ^ rot of its row part (rot < kCPT; threads with different
  // rot read different chunks)
  static_assert((Sh::kCPT & (Sh::kCPT - 1)) == 0, "chunks per thread: a power of two");
  const uint32_t rot = (tid / Sh::kRowsPer128) % Sh::kCPT;
  float hreg[Sh::kHPT];
#pragma unroll
  for (int i = 0; i < Sh::kCPT; i++) {
    const uint32_t c = qd * Sh::kCPT + (i ^ rot);
#pragma unroll
    for (int e = 0; e < Tr::kVec; e++) hreg[i * Tr::kVec + e] = s_h[c * Tr::kVec + e];
  }
  // Where the scorers wait for a window's wide terms: before its inner
  // products, or (FP32 tables) after them, so that the stages are read and
  // handed back while a decoder team finishes the window and the embedding
  // stream keeps moving.  Measured: the later wait is 3 % faster with FP32
  // rows (2M ads, d = 64); with FP8 rows (10M ads, d = 64) the two orders
  // take the same time, and the earlier one is kept there.
  constexpr bool kDotFirst = std::is_same<Elt, float>::value;
  // waits (thread 0, bounded) for window j's wide terms; true: stop scoring
  auto wait_wide = [&](uint32_t b, uint32_t apar) -> bool {
    if (tid == 0) {
      uint32_t stop = *((volatile uint32_t *)&sm.abort);
      if (!stop && !mbar_wait_bounded(&sm.acc_full[b], apar, kWaitTimeoutNs)) stop = 1;
      if (stop && !*((volatile uint32_t *)&sm.abort)) {
        atomicOr(&a.ctrl->flags, DEVERR_TIMEOUT);
        sm.abort = 1;
      }
      sm.stop_acc = stop;
    }
    gsync();
    if (sm.stop_acc) return true;
    mbar_try_wait(&sm.acc_full[b], apar);  // per-thread acquire
    return false;
  };
  for (uint32_t j = 0; j < my_wins; j++) {
    const uint32_t b = j % kAccBufs, apar = (j / kAccBufs) & 1u;
    const uint32_t w = w_begin + j;
    if (!kDotFirst && wait_wide(b, apar)) break;
    // per-row side inputs, loaded before the rows arrive so that their
    // latency overlaps the wait for the stage
    float pre_side[Sh::kPasses], pre_scale[Sh::kPasses];
    bool pre_keep[Sh::kPasses];
#pragma unroll
    for (int ps = 0; ps < Sh::kPasses; ps++) {
      const uint32_t ad = w * kWin + ps * Sh::kRowsPerPass + prow;
      const bool in = ad < a.n_ads && qd == 0;
      pre_side[ps] = in && pre ? __ldg(a.wide_in + ad) : 0.f;
      pre_scale[ps] = in && a.scale ? __ldg(a.scale + ad) : 1.f;
      pre_keep[ps] = !(in && a.filter) || ((__ldg(a.filter + (ad >> 6)) >> (ad & 63)) & 1ull);
    }
    // the inner products of the window's rows
    float dotv[Sh::kPasses];
    bool validv[Sh::kPasses];
#pragma unroll
    for (int ps = 0; ps < Sh::kPasses; ps++) {
      const uint32_t rw = ps * Sh::kRowsPerPass + prow;  // row within the window
      const uint32_t ad = w * kWin + rw;
      const uint32_t seq = j * Sh::kStagesPerWin + rw / Sh::kRowsPerStage;
      // Each warp's rows lie in one stage: wait for that stage only (not at
      // all once the CTA has given up), and hand it back right after reading
      // it, so the producer refills the ring while the rest of the window is
      // still being scored.
      bool staged = true;
      if (lane == 0)
        staged = (!kDotFirst || !*((volatile uint32_t *)&sm.abort)) &&
                 mbar_wait_bounded(&sm.full[seq % S], (seq / S) & 1u, kWaitTimeoutNs);
      staged = __shfl_sync(0xffffffffu, staged, 0);
      if (!staged && lane == 0 && (!kDotFirst || !*((volatile uint32_t *)&sm.abort))) {
        atomicOr(&a.ctrl->flags, DEVERR_TIMEOUT);
        sm.abort = 1;
      }
      if (staged) mbar_try_wait(&sm.full[seq % S], (seq / S) & 1u);  // per-thread acquire
      const bool valid = staged && ad < a.n_ads;
      const uint8_t *row = stage0 + (size_t)(seq % S) * kStageBytes +
                           (size_t)(rw % Sh::kRowsPerStage) * Sh::kRowBytes;
      float2 dot2 = make_float2(0.f, 0.f);
      if (valid) {
#pragma unroll
        for (int i = 0; i < Sh::kCPT; i++) {
          const uint32_t c = qd * Sh::kCPT + (i ^ rot);
          const uint4 v = *reinterpret_cast<const uint4 *>(row + c * 16);
          float f[Tr::kVec];
          Tr::load(v, f);
#pragma unroll
          for (int e = 0; e < Tr::kVec; e += 2)  // packed FP32 FMA: two lanes of the sum
            dot2 = __ffma2_rn(make_float2(hreg[i * Tr::kVec + e], hreg[i * Tr::kVec + e + 1]),
                              make_float2(f[e], f[e + 1]), dot2);
        }
      }
      mbar_arrive(&sm.empty[seq % S]);  // this thread is done with the stage
      float dot = dot2.x + dot2.y;
#pragma unroll
      for (int o = Sh::kTPR / 2; o >= 1; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
      dotv[ps] = dot;
      validv[ps] = valid;
    }
    if (kDotFirst && wait_wide(b, apar)) break;
    const float *acc = sm.acc[b].fp;  // the window's wide terms, folded by the decoders
#pragma unroll
    for (int ps = 0; ps < Sh::kPasses; ps++) {
      const uint32_t rw = ps * Sh::kRowsPerPass + prow;
      const uint32_t ad = w * kWin + rw;
      const bool leader = validv[ps] && qd == 0;
      float score = 0.f;
      if (leader) {
        const float wide = pre ? pre_side[ps] : acc[rw];
        score = dotv[ps];
        if (a.scale) score *= pre_scale[ps];
        score += wide;
        if (a.wide_out && !pre) a.wide_out[ad] = wide;
      }
      if (ALL) {
        if (leader) a.all_out[ad] = score;
      } else {
        bool keep = leader && pre_keep[ps];
        uint64_t kk = 0;
        if (keep) {
          kk = make_key(score, ad);
          keep = kk >= sm.thr;
        }
        const uint32_t pos = warp_append(keep, &sm.n);
        if (keep) {
          cand[pos] = kk;
          const uint32_t bin = (uint32_t)(kk >> kBinShift);
          atomicAdd(&sm.chist[bin], 1u);
          if (bin > sm.top_bin) atomicMax(&sm.top_bin, bin);
        }
      }
    }
    gsync();  // the window's accumulator is fully read; appends visible
    for (int i = tid; i < kWin; i += kDotThreads) sm.acc[b].fp[i] = 0.f;  // hand it back, zeroed
    mbar_arrive(&sm.acc_empty[b]);
    if (!ALL && sm.n + kWin > a.cap) {
      // trim the candidates to the K best: radix select, then a stable
      // in-place compaction in rounds of one entry per scorer thread
      const uint32_t n = sm.n;
      const uint64_t T =
          group_radix_select<kDotThreads>(cand, n, a.k, sm.hist, sm.misc, tid, gsync);
      uint32_t kept = 0;
      for (uint32_t b0 = 0, rnd = 0; b0 < n; b0 += kDotThreads, rnd++) {
        const uint32_t i = b0 + tid;
        const uint64_t x = i < n ? cand[i] : 0ull;
        const bool kp = i < n && x >= T;
        const uint32_t bal = __ballot_sync(0xffffffffu, kp);
        if (lane == 0) sm.wtot[rnd & 1][warp] = __popc(bal);
        gsync();
        uint32_t before = kept, round_total = 0;
#pragma unroll
        for (int q2 = 0; q2 < kDotWarps; q2++) {
          const uint32_t t2 = sm.wtot[rnd & 1][q2];
          before += (q2 < warp) ? t2 : 0u;
          round_total += t2;
        }
        if (kp) cand[before + __popc(bal & ((1u << lane) - 1u))] = x;
        kept += round_total;
      }
      gsync();
      if (tid == 0) {
        sm.n = kept;
        const unsigned long long g = atomicMax(&a.ctrl->thr, (unsigned long long)T);
        atomicMax(&sm.thr, max((unsigned long long)T, g));
      }
      gsync();
    } else if (!ALL && (j % kRefresh) == kRefresh - 1) {
      // add this CTA's counts to the global histogram (no appends run until
      // the next window's barrier); the index producer reads it back
      for (int i = tid; i < kCandBins; i += kDotThreads) {
        const uint32_t c = sm.chist[i];
        if (c) {
          atomicAdd(a.hist + i, c);
          sm.chist[i] = 0;
        }
      }
      if (tid == 0) atomicMax(a.hist + kCandBins, sm.top_bin);
    }
  }
  if (ALL) return;
  if (tid == 0) sm.stop_end = *((volatile uint32_t *)&sm.abort);
  gsync();
  if (sm.stop_end) return;
  const uint32_t n = sm.n;
  uint64_t T = 0;
  if (n > a.k) T = group_radix_select<kDotThreads>(cand, n, a.k, sm.hist, sm.misc, tid, gsync);
  for (int i = tid; i < kCandBins; i += kDotThreads) {  // last counts
    const uint32_t c = sm.chist[i];
    if (c) atomicAdd(a.hist + i, c);
  }
  if (tid == 0) atomicMax(a.hist + kCandBins, sm.top_bin);
  if (warp == 0) {
    const unsigned long long h =
        hist_top_threshold(a.hist, (uint32_t)(sm.thr >> kBinShift), a.k);
    if (lane == 0) {
      const unsigned long long g = *((volatile unsigned long long *)&a.ctrl->thr);
      sm.thr = max(max((unsigned long long)T, (unsigned long long)sm.thr), max(g, h));
      if (n > a.k) atomicMax(&a.ctrl->thr, (unsigned long long)T);
    }
  }
  gsync();
  const uint64_t fin = sm.thr;
  for (uint32_t b0 = 0; b0 < n; b0 += kDotThreads) {
    const uint32_t i = b0 + tid;
    const uint64_t x = i < n ? cand[i] : 0ull;
    const bool kp = i < n && x >= fin;
    const uint32_t pos = warp_append(kp, &a.ctrl->n_cand);
    if (kp) a.cand_out[pos] = x;
  }
}

// Shared memory the fused scan needs besides its stage ring (cap: entries of
// the candidate buffer held in shared memory, 0 when it is in global memory).
static size_t fused_fixed_bytes(const ebr_index *ix, uint32_t d, uint32_t cap, uint32_t slots,
                                uint32_t *slot_bytes) {
  *slot_bytes = (ix->max_win_bytes + 127) / 128 * 128;
  if (*slot_bytes == 0) *slot_bytes = 128;
  return (size_t)slots * *slot_bytes + (size_t)d * 4 + (size_t)cap * 8;
}

// dynamic part: what is left of 227 KB after the static part
constexpr size_t kFusedSmemBudget = 227 * 1024 - sizeof(FusedSmem) - 512;

static uint32_t fused_cap(uint32_t k) {
  // K plus slack for the appends between trims (a window adds at most 256)
  return (std::max<uint32_t>(k, 1) + 1024 + 255) / 256 * 256;
}

template <typename Elt, int D, bool ALL>
static int launch_fused_t(const ebr_index *ix, FusedArgs a, int max_grid, cudaStream_t st,
                          uint64_t *cta_cand, size_t cta_cand_entries) {
  a.cap = ALL ? 0 : fused_cap(a.k);
  int grid = ix->num_sms;
  if (max_grid > 0) grid = std::min(grid, max_grid);
  grid = std::min<int>(grid, (int)a.n_win);
  if (grid < 1) grid = 1;
  uint32_t slot_bytes = 0;
  // two index slots per decoder team (the next window's segments arrive while
  // the team decodes the current one) when that still leaves 8 stages; a
  // large candidate buffer (big K) moves to global memory to make room for
  // them, since after the first windows the running threshold lets few
  // candidates through and the buffer is rarely touched
  uint32_t slots = kMaxIdxSlots;
  size_t fixed = fused_fixed_bytes(ix, D, a.cap, slots, &slot_bytes);
  a.cand_g = nullptr;
  if (fixed + 8 * (size_t)kStageBytes > kFusedSmemBudget) {
    const size_t fixed_g = fused_fixed_bytes(ix, D, 0, slots, &slot_bytes);
    if (!ALL && cta_cand && (size_t)grid * a.cap <= cta_cand_entries &&
        fixed_g + 8 * (size_t)kStageBytes <= kFusedSmemBudget) {
      a.cand_g = cta_cand;
      fixed = fixed_g;
    } else {
      slots = kTeams;
      fixed = fused_fixed_bytes(ix, D, a.cap, slots, &slot_bytes);
    }
  }
  a.idx_slots = slots;
  if (fixed + kMinStages * (size_t)kStageBytes > kFusedSmemBudget) {
    set_error("fused scan: k = %u with %u-byte window segments needs too much shared memory",
              a.k, ix->max_win_bytes);
    return EBR_EINVAL;
  }
  uint32_t stages = kMinStages;
  while (stages < (uint32_t)kMaxStages &&
         fixed + (size_t)(stages + 1) * kStageBytes <= kFusedSmemBudget)
    stages++;
  a.stages = stages;
  a.slot_bytes = slot_bytes;
  const size_t smem = fixed + (size_t)stages * kStageBytes;
  auto kern = k_fused_window<Elt, D, ALL, false>;
  if constexpr (!ALL) {
    if (a.cand_g) kern = k_fused_window<Elt, D, false, true>;
  }
  EBR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int occ = 0;
  EBR_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kFusedThreads, smem));
  if (occ < 1) {
    set_error("fused scan: one CTA of %d threads with %zu bytes of shared memory does not fit an SM",
              kFusedThreads, smem);
    return EBR_ECUDA;
  }
  EBR_CUDA_TRY(launch_pdl(kern, grid, kFusedThreads, smem, st, a));
  return EBR_OK;
}

template <typename Elt, bool ALL>
static int launch_fused_d(const ebr_index *ix, const FusedArgs &a, int max_grid,
                          cudaStream_t st, uint64_t *cc, size_t ce) {
  switch (ix->d) {
    case 4: if constexpr (EltTraits<Elt>::kVec <= 4) return launch_fused_t<Elt, 4, ALL>(ix, a, max_grid, st, cc, ce); break;
    case 8: if constexpr (EltTraits<Elt>::kVec <= 8) return launch_fused_t<Elt, 8, ALL>(ix, a, max_grid, st, cc, ce); break;
    case 16: return launch_fused_t<Elt, 16, ALL>(ix, a, max_grid, st, cc, ce);
    case 32: return launch_fused_t<Elt, 32, ALL>(ix, a, max_grid, st, cc, ce);
    case 64: return launch_fused_t<Elt, 64, ALL>(ix, a, max_grid, st, cc, ce);
    case 128: return launch_fused_t<Elt, 128, ALL>(ix, a, max_grid, st, cc, ce);
  }
  set_error("embedding dimension %u unsupported for this dtype", ix->d);
  return EBR_EINVAL;
}

// Largest |w[i]| as FP32 bits (non-negative floats order like their bits);
// a non-finite weight is flagged.
__global__ void k_absmax(const float *__restrict__ w, uint32_t n, uint32_t *__restrict__ out,
                         uint32_t *__restrict__ flags) {
  uint32_t m = 0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    m = max(m, __float_as_uint(w[i]) & 0x7FFFFFFFu);
  for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) {
    if (m >= 0x7F800000u) atomicOr(flags, DEVERR_RANGE);
    atomicMax(out, m >= 0x7F800000u ? 0u : m);
  }
}

// Packs a dense w^ into the fixed-point terms the fused scan decodes
// (pack_term), with F from max |w^| (*wmax_bits) and the index's most keys of
// one ad; F goes to *fx_out.  With route set, does nothing unless *route
// chose the window-major decode (the device decided the traversal).
__global__ void k_pack(const float *__restrict__ w, uint32_t n,
                       const uint32_t *__restrict__ wmax_bits, uint32_t max_keys, int cls_shift,
                       const uint32_t *__restrict__ route, uint32_t *__restrict__ wq,
                       int *__restrict__ fx_out) {
  if (route && *route == 0u) return;
  const int F = fix_exponent(__uint_as_float(*wmax_bits), max_keys);
  if (blockIdx.x == 0 && threadIdx.x == 0) *fx_out = F;
  const float s0 = pow2f(F), s1 = pow2f(F + cls_shift), s2 = pow2f(F + 2 * cls_shift);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    wq[i] = pack_term(w[i], s0, s1, s2, cls_shift > 0);
}

// Whether the fused scan fits shared memory for top-k on this index; if not,
// dense queries take the key-major path (Algorithm 2) instead.
bool fused_fits(const ebr_index *ix, uint32_t k) {
  uint32_t slot_bytes = 0;
  return ix->max_win_chunks <= (uint32_t)kMaxChunkTab && ix->max_keys_per_ad <= 65536u &&
         fused_fixed_bytes(ix, ix->d, fused_cap(k), kTeams, &slot_bytes) +
                 kMinStages * (size_t)kStageBytes <=
             kFusedSmemBudget;
}

// Launches the fused scan over all windows.  all_out != nullptr: write every
// score instead of selecting.  Candidates go to cand_out (grid * k entries at
// most) with counters in ctrl.  The window decode reads packed terms from wq
// with F in ctrl->fx: when `packed` is false they are made here from the
// dense w_hat first (after max |w^| unless wmax_ready).  *n_launched counts
// this library's kernels launched.  cta_cand (cta_cand_entries entries), if
// given, may hold the CTAs' candidate buffers when they do not fit shared
// memory beside two index slots per decoder team.
int launch_fused(const ebr_index *ix, const float *h_u, const float *w_hat, uint32_t *wq,
                 bool packed, const uint64_t *filter, uint32_t k, uint64_t *cand_out,
                 Ctrl *ctrl, float *all_out, float *wide_out, uint32_t *hist, int max_grid,
                 cudaStream_t st, bool wmax_ready, const float *wide_in, const uint32_t *route,
                 int *n_launched, uint64_t *cta_cand, size_t cta_cand_entries) {
  FusedArgs a;
  memset(&a, 0, sizeof(a));
  int launched = 0;
  a.emb = ix->dtype == EBR_F32 ? ix->emb_f32.p : ix->emb_q.p;
  a.scale = ix->dtype == EBR_FP8E4M3 ? (const float *)ix->emb_scale.p : nullptr;
  a.h_u = h_u;
  a.wq = wq;
  for (int g = 0; g < kGroups; g++) {
    a.wkey[g] = ix->wkey[g];
    a.wvals[g] = ix->wvals[g];
    a.win_ptr[g] = ix->win_ptr[g];
  }
  a.filter = filter;
  a.n_ads = ix->n_ads;
  a.n_win = ix->n_win;
  a.k = std::max<uint32_t>(k, 1);
  a.cand_out = cand_out;
  a.ctrl = ctrl;
  a.all_out = all_out;
  a.wide_out = wide_out;
  a.hist = hist;
  a.max_keys = std::max<uint32_t>(ix->max_keys_per_ad, 1);
  a.cls_shift = class_shift(a.max_keys);
  a.fx_word = reinterpret_cast<const int *>(&ctrl->fx);
  a.wide_in = wide_in;
  a.route = route;
  const bool decodes = !wide_in || route;  // the windows may be decoded
  if (decodes && !packed) {
    if (!wmax_ready) {
      // max |w^| for the fixed-point scale (non-finite weights are flagged)
      EBR_CUDA_TRY(cudaMemsetAsync(&ctrl->pad, 0, sizeof(uint32_t), st));
      k_absmax<<<std::max<uint32_t>(1, std::min<uint32_t>(64, (ix->n_keys + 1023) / 1024)), 256,
                 0, st>>>(w_hat, ix->n_keys, &ctrl->pad, &ctrl->flags);
      EBR_CUDA_TRY(cudaGetLastError());
      launched++;
    }
    k_pack<<<std::max<uint32_t>(1, std::min<uint32_t>(1024, (ix->n_keys + 255) / 256)), 256, 0,
             st>>>(w_hat, ix->n_keys, &ctrl->pad, a.max_keys, a.cls_shift, route, wq,
                   reinterpret_cast<int *>(&ctrl->fx));
    EBR_CUDA_TRY(cudaGetLastError());
    launched++;
  }
  int rc;
  uint64_t *cc = cta_cand;
  const size_t ce = cta_cand_entries;
  if (all_out) {
    if (ix->dtype == EBR_F32) rc = launch_fused_d<float, true>(ix, a, max_grid, st, cc, ce);
    else if (ix->dtype == EBR_BF16) rc = launch_fused_d<Bf16Tag, true>(ix, a, max_grid, st, cc, ce);
    else rc = launch_fused_d<Fp8Tag, true>(ix, a, max_grid, st, cc, ce);
  } else {
    if (ix->dtype == EBR_F32) rc = launch_fused_d<float, false>(ix, a, max_grid, st, cc, ce);
    else if (ix->dtype == EBR_BF16) rc = launch_fused_d<Bf16Tag, false>(ix, a, max_grid, st, cc, ce);
    else rc = launch_fused_d<Fp8Tag, false>(ix, a, max_grid, st, cc, ce);
  }
  if (rc == EBR_OK) launched++;
  if (n_launched) *n_launched = launched;
  return rc;
}

}  // namespace ebr
