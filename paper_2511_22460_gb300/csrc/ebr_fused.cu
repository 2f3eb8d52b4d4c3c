// Fused window-major scan for requests whose query covers the whole key space.
//
// One CTA handles one window of 256 consecutive ads at a time (the block
// granularity of Algorithm 1: ads sharing ad >> 8).  For its window it
//   1. issues the streaming loads of the 256 embedding rows (kept in registers),
//   2. decodes every block of the window from the window-major view of the
//      compressed list -- all nine size groups -- and scatter-adds the block's
//      w^[key] into a 256-entry shared-memory accumulator (the wide term of
//      the HitMatch equation, Sec. 3.3, for these ads),
//   3. computes the inner products (Eq. 1), adds the accumulator and the FP8
//      row scale, applies the targeting filter and appends candidates to a
//      per-CTA buffer that a radix select trims to the K best,
// so the wide term never leaves shared memory and the score vector is never
// written.  Candidates surviving the running global threshold are appended to
// a global list for the final selection.
#include <algorithm>
#include <cstring>

#include "ebr_device.cuh"
#include "ebr_internal.cuh"

namespace ebr {

constexpr int kFusedThreads = 256;
constexpr int kFusedWarps = kFusedThreads / 32;
constexpr int kWin = 256;

struct FusedArgs {
  const void *emb;
  const float *scale;
  const float *h_u;
  const float *w_hat;  // dense over keys
  const uint32_t *wkey[kGroups];
  const uint8_t *wvals[kGroups];
  const uint32_t *win_ptr[kGroups];
  const uint64_t *filter;
  uint32_t n_ads, n_win, k, cap, stages;
  uint64_t *cand_out;
  Ctrl *ctrl;
  float *all_out;  // score-all mode
  float *wide_out; // if set: the per-ad wide term is written here (needed by FP32 rescoring)
  uint32_t *hist;  // [256 + 65536] candidate-score histogram (zeroed per request)
};

template <typename Elt, int D>
struct FusedShape {
  static constexpr int kRowBytes = D * EltTraits<Elt>::kBytes;
  static constexpr int kChunks = kRowBytes / 16;                 // 16-byte chunks per row
  static constexpr int kRowsPer128 = kRowBytes >= 128 ? 1 : 128 / kRowBytes;
  static constexpr int kStageBytes = kWin * kRowBytes;           // one window of rows
  static_assert(kChunks >= 1, "row width");
};

__device__ __forceinline__ uint32_t unit_shift_f(uint32_t g) { return g >= 2 ? g - 2 : 0; }

// Shared memory (dynamic): [stages x window rows][h_u, D floats][2 x cap candidates]
template <typename Elt, int D, bool ALL>
__global__ void __launch_bounds__(kFusedThreads, 2) k_fused_window(FusedArgs a) {
  using Sh = FusedShape<Elt, D>;
  using Tr = EltTraits<Elt>;
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ float s_acc[kWin];
  __shared__ uint32_t s_lo[kGroups], s_pre[kGroups + 1];
  __shared__ uint32_t s_hist[256];
  __shared__ uint32_t s_misc[8];
  __shared__ uint32_t s_n, s_n2, s_status, s_fail_j;
  __shared__ unsigned long long s_thr;
  __shared__ uint64_t s_bar[4];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t S = a.stages;
  uint8_t *stage0 = smem;
  float *s_h = reinterpret_cast<float *>(smem + (size_t)S * Sh::kStageBytes);
  uint64_t *cand = reinterpret_cast<uint64_t *>(s_h + D);
  uint64_t *cand2 = cand + a.cap;

  const uint32_t my_wins =
      blockIdx.x < a.n_win ? (a.n_win - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  auto issue = [&](uint32_t j) {  // window j of this CTA into stage j % S
    const uint32_t w = blockIdx.x + j * gridDim.x;
    const uint32_t row0 = w * kWin;
    const uint32_t rows = min((uint32_t)kWin, a.n_ads - row0);
    uint64_t *bar = &s_bar[j % S];
    mbar_arrive_expect_tx(bar, rows * Sh::kRowBytes);
    bulk_g2s(stage0 + (size_t)(j % S) * Sh::kStageBytes,
             reinterpret_cast<const uint8_t *>(a.emb) + (uint64_t)row0 * Sh::kRowBytes,
             rows * Sh::kRowBytes, bar);
  };
  s_acc[tid] = 0.f;
  for (int i = tid; i < D; i += kFusedThreads) s_h[i] = a.h_u[i];
  if (tid == 0) {
    s_n = 0;
    s_status = 0;
    s_thr = 0ull;
    for (uint32_t q = 0; q < S; q++) mbar_init(&s_bar[q], 1);
    fence_mbar_init();
    for (uint32_t j = 0; j < S && j < my_wins; j++) issue(j);
  }
  __syncthreads();

  for (uint32_t j = 0; j < my_wins; j++) {
    const uint32_t w = blockIdx.x + j * gridDim.x;
    const uint32_t row0 = w * kWin;
    const uint32_t rows = min((uint32_t)kWin, a.n_ads - row0);
    // ---- 1. wide term of window w from its blocks in all nine groups
    if (tid < kGroups) {
      const uint32_t lo = a.win_ptr[tid][w], hi = a.win_ptr[tid][w + 1];
      s_lo[tid] = lo;
      s_pre[tid + 1] = (hi - lo) << unit_shift_f(tid);
    }
    __syncthreads();
    if (tid == 0) {
      s_pre[0] = 0;
#pragma unroll
      for (int g = 0; g < kGroups; g++) s_pre[g + 1] += s_pre[g];
    }
    __syncthreads();
    uint32_t pre[kGroups + 1];
#pragma unroll
    for (int g = 0; g <= kGroups; g++) pre[g] = s_pre[g];
    const uint32_t total = pre[kGroups];
    constexpr int kB = 4;  // units per thread in flight
    for (uint32_t u0 = tid; u0 < total; u0 += kB * kFusedThreads) {
      uint32_t key[kB], word[kB], meta[kB];  // meta: group | first-word << 4 | valid << 5
#pragma unroll
      for (int q = 0; q < kB; q++) {
        const uint32_t u = u0 + q * kFusedThreads;
        key[q] = 0;
        word[q] = 0;
        meta[q] = 0;
        if (u < total) {
          uint32_t g = 0;
#pragma unroll
          for (int t = 1; t < kGroups; t++) g += (u >= pre[t]) ? 1u : 0u;
          const uint32_t us = unit_shift_f(g);
          const uint32_t vv = u - s_pre[g];
          const uint32_t b = s_lo[g] + (vv >> us);
          const uint32_t wi = vv & ((1u << us) - 1u);
          key[q] = __ldcs(a.wkey[g] + b);
          if (g >= 2)
            word[q] = __ldcs(reinterpret_cast<const uint32_t *>(a.wvals[g]) +
                             (((uint64_t)b << us) + wi));
          else if (g == 1)
            word[q] = __ldcs(reinterpret_cast<const unsigned short *>(a.wvals[1]) + b);
          else
            word[q] = __ldcs(reinterpret_cast<const unsigned char *>(a.wvals[0]) + b);
          meta[q] = g | ((wi == 0) ? 16u : 0u) | 32u;
        }
      }
      float wt[kB];
#pragma unroll
      for (int q = 0; q < kB; q++) wt[q] = (meta[q] & 32u) ? __ldg(a.w_hat + key[q]) : 0.f;
#pragma unroll
      for (int q = 0; q < kB; q++) {
        if (wt[q] == 0.f) continue;
        const uint32_t g = meta[q] & 15u;
        if (g >= 2) {
#pragma unroll
          for (int s2 = 0; s2 < 4; s2++) {
            const uint32_t l = (word[q] >> (8 * s2)) & 255u;
            if ((s2 == 0 && (meta[q] & 16u)) || l != 0) atomicAdd(&s_acc[l], wt[q]);
          }
        } else if (g == 1) {
          atomicAdd(&s_acc[word[q] & 255u], wt[q]);
          if (word[q] >> 8) atomicAdd(&s_acc[word[q] >> 8], wt[q]);
        } else {
          atomicAdd(&s_acc[word[q]], wt[q]);
        }
      }
    }
    // ---- 2. this window's rows (TMA) must have landed
    const uint32_t st = j % S, parity = (j / S) & 1u;
    if (tid == 0 && !mbar_wait_bounded(&s_bar[st], parity, kWaitTimeoutNs)) {
      s_status = 1;
      s_fail_j = j;
    }
    __syncthreads();  // also: accumulator complete
    if (s_status) break;
    mbar_try_wait(&s_bar[st], parity);  // per-thread acquire of the completed phase
    // ---- 3. one row per thread: inner product, wide add, filter, candidate
    {
      const uint32_t r = tid;
      const uint8_t *row = stage0 + (size_t)st * Sh::kStageBytes + (size_t)r * Sh::kRowBytes;
      const uint32_t rot = r / Sh::kRowsPer128;  // chunk rotation: conflict-free 16-byte reads
      float dot = 0.f;
      if (r < rows) {
#pragma unroll
        for (int c = 0; c < Sh::kChunks; c++) {
          const uint32_t cc = (c + rot) % Sh::kChunks;
          const uint4 v = *reinterpret_cast<const uint4 *>(row + cc * 16);
          float f[Tr::kVec];
          Tr::load(v, f);
          const float4 *hp = reinterpret_cast<const float4 *>(s_h + cc * Tr::kVec);
#pragma unroll
          for (int e4 = 0; e4 < Tr::kVec / 4; e4++) {
            const float4 hv = hp[e4];
            dot = fmaf(hv.x, f[4 * e4 + 0], dot);
            dot = fmaf(hv.y, f[4 * e4 + 1], dot);
            dot = fmaf(hv.z, f[4 * e4 + 2], dot);
            dot = fmaf(hv.w, f[4 * e4 + 3], dot);
          }
        }
      }
      const bool valid = r < rows;
      const uint32_t ad = row0 + r;
      float score = 0.f;
      if (valid) {
        score = dot;
        if (a.scale) score *= a.scale[ad];
        score += s_acc[r];
        if (a.wide_out) a.wide_out[ad] = s_acc[r];
      }
      if (ALL) {
        if (valid) a.all_out[ad] = score;
      } else {
        bool keep = valid;
        if (keep && a.filter) keep = (a.filter[ad >> 6] >> (ad & 63)) & 1ull;
        uint64_t kk = 0;
        if (keep) {
          kk = make_key(score, ad);
          keep = kk >= s_thr;
        }
        const uint32_t pos = warp_append(keep, &s_n);
        if (keep) {
          cand[pos] = kk;
          const uint32_t o = (uint32_t)(kk >> 32);
          atomicAdd(a.hist + 256 + (o >> 16), 1u);
          atomicAdd(a.hist + (o >> 24), 1u);
        }
      }
    }
    __syncthreads();  // stage and accumulator consumed
    if (tid == 0 && j + S < my_wins) issue(j + S);
    s_acc[tid] = 0.f;
    if (!ALL) {
      if (s_n + kWin > a.cap) {
        const uint32_t n = s_n;
        const uint64_t T = cta_radix_select<kFusedThreads>(cand, n, a.k, s_hist, s_misc);
        if (tid == 0) s_n2 = 0;
        __syncthreads();
        for (uint32_t b0 = 0; b0 < n; b0 += kFusedThreads) {
          const uint32_t i = b0 + tid;
          const uint64_t x = i < n ? cand[i] : 0ull;
          const bool kp = i < n && x >= T;
          const uint32_t pos = warp_append(kp, &s_n2);
          if (kp) cand2[pos] = x;
        }
        __syncthreads();
        uint64_t *t = cand;
        cand = cand2;
        cand2 = t;
        if (tid == 0) {
          s_n = s_n2;
          const unsigned long long g = atomicMax(&a.ctrl->thr, (unsigned long long)T);
          s_thr = max((unsigned long long)T, max(g, (unsigned long long)s_thr));
        }
      } else if (warp == 0 && (j & 3) == 3) {
        const unsigned long long h = hist_threshold(a.hist, a.hist + 256, a.k);
        if (lane == 0) {
          const unsigned long long g = *((volatile unsigned long long *)&a.ctrl->thr);
          s_thr = max(s_thr, max(g, h));
        }
      }
    }
    __syncthreads();
  }
  if (s_status) {
    // A window's rows never arrived: record it, drain the copies in flight, leave.
    if (tid == 0) {
      atomicOr(&a.ctrl->flags, DEVERR_TIMEOUT);
      for (uint32_t q = s_fail_j; q < s_fail_j + S && q < my_wins; q++)
        mbar_wait_bounded(&s_bar[q % S], (q / S) & 1u, kWaitTimeoutNs / 4);
    }
    return;
  }
  if (ALL) return;
  uint32_t n = s_n;
  uint64_t T = 0;
  if (n > a.k) T = cta_radix_select<kFusedThreads>(cand, n, a.k, s_hist, s_misc);
  if (warp == 0) {
    const unsigned long long h = hist_threshold(a.hist, a.hist + 256, a.k);
    if (lane == 0) {
      const unsigned long long g = *((volatile unsigned long long *)&a.ctrl->thr);
      s_thr = max(max((unsigned long long)T, (unsigned long long)s_thr), max(g, h));
      if (n > a.k) atomicMax(&a.ctrl->thr, (unsigned long long)T);
    }
  }
  __syncthreads();
  const uint64_t fin = s_thr;
  for (uint32_t b0 = 0; b0 < n; b0 += kFusedThreads) {
    const uint32_t i = b0 + tid;
    const uint64_t x = i < n ? cand[i] : 0ull;
    const bool kp = i < n && x >= fin;
    const uint32_t pos = warp_append(kp, &a.ctrl->n_cand);
    if (kp) a.cand_out[pos] = x;
  }
}

template <typename Elt, int D, bool ALL>
static int launch_fused_t(const ebr_index *ix, FusedArgs a, int max_grid, cudaStream_t st) {
  using Sh = FusedShape<Elt, D>;
  a.cap = ALL ? 0 : (a.k + std::max<uint32_t>(a.k, 2 * kWin) + 255) / 256 * 256;
  const size_t fixed = (size_t)D * 4 + (size_t)2 * a.cap * 8;
  // as many window stages as leave room for two CTAs per SM (at least one)
  const size_t budget = 110 * 1024;
  uint32_t stages = 1;
  while (stages < 4 && fixed + (size_t)(stages + 1) * Sh::kStageBytes <= budget) stages++;
  a.stages = stages;
  const size_t smem = fixed + (size_t)stages * Sh::kStageBytes;
  auto kern = k_fused_window<Elt, D, ALL>;
  EBR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int occ = 0;
  EBR_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kFusedThreads, smem));
  if (occ < 1) occ = 1;
  int grid = ix->num_sms * occ;
  if (max_grid > 0) grid = std::min(grid, max_grid);
  grid = std::min<int>(grid, (int)a.n_win);
  if (grid < 1) grid = 1;
  kern<<<grid, kFusedThreads, smem, st>>>(a);
  EBR_CUDA_TRY(cudaGetLastError());
  return EBR_OK;
}

template <typename Elt, bool ALL>
static int launch_fused_d(const ebr_index *ix, const FusedArgs &a, int max_grid,
                          cudaStream_t st) {
  switch (ix->d) {
    case 4: if constexpr (EltTraits<Elt>::kVec <= 4) return launch_fused_t<Elt, 4, ALL>(ix, a, max_grid, st); break;
    case 8: if constexpr (EltTraits<Elt>::kVec <= 8) return launch_fused_t<Elt, 8, ALL>(ix, a, max_grid, st); break;
    case 16: return launch_fused_t<Elt, 16, ALL>(ix, a, max_grid, st);
    case 32: return launch_fused_t<Elt, 32, ALL>(ix, a, max_grid, st);
    case 64: return launch_fused_t<Elt, 64, ALL>(ix, a, max_grid, st);
    case 128: return launch_fused_t<Elt, 128, ALL>(ix, a, max_grid, st);
  }
  set_error("embedding dimension %u unsupported for this dtype", ix->d);
  return EBR_EINVAL;
}

// Launches the fused scan over all windows.  all_out != nullptr: write every
// score instead of selecting.  Candidates go to cand_out (grid * k entries at
// most) with counters in ctrl.
int launch_fused(const ebr_index *ix, const float *h_u, const float *w_hat,
                 const uint64_t *filter, uint32_t k, uint64_t *cand_out, Ctrl *ctrl,
                 float *all_out, float *wide_out, uint32_t *hist, int max_grid,
                 cudaStream_t st) {
  FusedArgs a;
  memset(&a, 0, sizeof(a));
  a.emb = ix->dtype == EBR_F32 ? ix->emb_f32.p : ix->emb_q.p;
  a.scale = ix->dtype == EBR_FP8E4M3 ? (const float *)ix->emb_scale.p : nullptr;
  a.h_u = h_u;
  a.w_hat = w_hat;
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
  if (all_out) {
    if (ix->dtype == EBR_F32) return launch_fused_d<float, true>(ix, a, max_grid, st);
    if (ix->dtype == EBR_BF16) return launch_fused_d<Bf16Tag, true>(ix, a, max_grid, st);
    return launch_fused_d<Fp8Tag, true>(ix, a, max_grid, st);
  }
  if (ix->dtype == EBR_F32) return launch_fused_d<float, false>(ix, a, max_grid, st);
  if (ix->dtype == EBR_BF16) return launch_fused_d<Bf16Tag, false>(ix, a, max_grid, st);
  return launch_fused_d<Fp8Tag, false>(ix, a, max_grid, st);
}

}  // namespace ebr
