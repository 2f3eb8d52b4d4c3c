// Batched requests: the users x ads inner products on the tensor cores
// (tcgen05.mma fed by tensor TMA, accumulators in TMEM), plus the tensor-map
// plumbing they need.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "ebr_internal.cuh"
#include "ebr_umma.cuh"

namespace ebr {

// --------------------------------------------------------------- tensor maps
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
static std::mutex g_encode_mu;

static int get_encoder() {
  std::lock_guard<std::mutex> lk(g_encode_mu);
  if (g_encode) return EBR_OK;
  void *fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                   cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
    set_error("cuTensorMapEncodeTiled unavailable: %s", cudaGetErrorString(e));
    return EBR_ECUDA;
  }
  g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  return EBR_OK;
}

// Row-major [rows][cols] matrix of 2-byte (BF16) or 1-byte (FP8) elements
// viewed as a 2-D tensor, boxes of 128 bytes (or 64, a whole 64-byte row) x
// box_rows rows, swizzled to match (the UMMA K-major layouts).
int make_tmap_2d(CUtensorMap *map, const void *base, uint64_t rows, uint64_t cols,
                 uint32_t elt_bytes, uint32_t box_rows) {
  EBR_TRY(get_encoder());
  const uint64_t row_bytes = cols * elt_bytes;
  const uint32_t box_bytes = row_bytes >= 128 ? 128u : 64u;
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {row_bytes};
  cuuint32_t box[2] = {box_bytes / elt_bytes, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(map,
                        elt_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8,
                        2, const_cast<void *>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE,
                        box_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d) for %llu x %llu, box %u", (int)r,
              (unsigned long long)rows, (unsigned long long)cols, box_rows);
    return EBR_ECUDA;
  }
  return EBR_OK;
}
int make_tmap_bf16(CUtensorMap *map, const void *base, uint64_t rows, uint64_t cols,
                   uint32_t box_rows) {
  return make_tmap_2d(map, base, rows, cols, 2, box_rows);
}

// ------------------------------------------------------------ GEMM check
// out[i][b] = sum_t A[i][t] * U[b][t] for one 128-row tile per CTA: the
// tensor-core building block of the batched scan, exposed for testing (BF16,
// or FP8 E4M3 codes when F8).
template <bool F8>
__global__ void __launch_bounds__(128) k_gemm_tc(const __grid_constant__ CUtensorMap ma,
                                                 const __grid_constant__ CUtensorMap mu,
                                                 uint32_t n, uint32_t B, uint32_t d,
                                                 float *__restrict__ out,
                                                 uint32_t *__restrict__ flags) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ uint64_t bar_tma, bar_mma;
  __shared__ uint32_t tmem_base, ok;
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t row_bytes = d * (F8 ? 1u : 2u);
  const uint32_t tr = row_bytes >= 128 ? 128u : 64u;  // bytes per K-tile row
  const uint32_t kb_n = row_bytes / tr, tile_elems = tr / (F8 ? 1u : 2u);
  uint8_t *sa = smem;                          // kb_n x [128 rows x tr]
  uint8_t *su = smem + (size_t)kb_n * 128 * tr;  // kb_n x [B rows x tr]
  const int warp = threadIdx.x >> 5;
  uint32_t ncols = 32;
  while (ncols < B) ncols <<= 1;
  if (warp == 0) {
    tmem_alloc(&tmem_base, ncols);
    tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    mbar_init(&bar_tma, 1);
    mbar_init(&bar_mma, 1);
    fence_mbar_init();
    ok = 1;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t row0 = blockIdx.x * 128;
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(&bar_tma, kb_n * (128u * tr + B * tr));
    for (uint32_t kb = 0; kb < kb_n; kb++) {
      tma_load_2d(sa + kb * 128u * tr, &ma, (int)(kb * tile_elems), (int)row0, &bar_tma);
      tma_load_2d(su + (size_t)kb * B * tr, &mu, (int)(kb * tile_elems), 0, &bar_tma);
    }
    if (!mbar_wait_bounded(&bar_tma, 0, kWaitTimeoutNs)) {
      ok = 0;
      atomicOr(flags, DEVERR_TIMEOUT);
    } else {
      tc_fence_after();
      const uint32_t idesc = F8 ? idesc_e4m3_f32(128, B) : idesc_bf16_f32(128, B);
      const uint32_t spt = tr / 32;
      for (uint32_t k = 0; k < kb_n * spt; k++) {
        const uint32_t kb = k / spt, kk = k % spt;
        const uint32_t aa = smem_u32(sa + kb * 128u * tr + kk * 32);
        const uint32_t ua = smem_u32(su + (size_t)kb * B * tr + kk * 32);
        const uint64_t ad = tr == 128 ? sdesc_k_sw128(aa) : sdesc_k_sw64(aa);
        const uint64_t bd = tr == 128 ? sdesc_k_sw128(ua) : sdesc_k_sw64(ua);
        if (F8)
          umma_e4m3(tmem_base, ad, bd, idesc, k > 0 ? 1u : 0u);
        else
          umma_bf16(tmem_base, ad, bd, idesc, k > 0 ? 1u : 0u);
      }
      umma_commit(&bar_mma);
      if (!mbar_wait_bounded(&bar_mma, 0, kWaitTimeoutNs)) {
        ok = 0;
        atomicOr(flags, DEVERR_TIMEOUT);
      }
    }
  }
  __syncthreads();
  tc_fence_after();
  if (ok) {
    mbar_try_wait(&bar_mma, 0);
    const uint32_t row = row0 + warp * 32 + (threadIdx.x & 31);
    for (uint32_t c = 0; c < B / 32; c++) {
      uint32_t r[32];
      tmem_ld32(tmem_base + ((uint32_t)(warp * 32) << 16) + c * 32, r);
      tmem_ld_wait();
      if (row < n)
        for (int j = 0; j < 32; j++) out[(uint64_t)row * B + c * 32 + j] = __uint_as_float(r[j]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem_base, ncols);
}

static int debug_gemm(bool f8, const void *A, uint32_t n, const void *U, uint32_t B, uint32_t d,
                      float *out, void *stream) {
  if (!A || !U || !out || n == 0 || (d != 64 && d != 128) || B < 32 || B > 256 || B % 32) {
    set_error("ebr_debug_gemm: need d in {64, 128}, B a multiple of 32 in 32..256");
    return EBR_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const uint32_t eb = f8 ? 1u : 2u;
  CUtensorMap ma, mu;
  EBR_TRY(make_tmap_2d(&ma, A, n, d, eb, 128));
  EBR_TRY(make_tmap_2d(&mu, U, B, d, eb, B));
  uint32_t *flags = nullptr;
  EBR_CUDA_TRY(cudaMallocAsync((void **)&flags, 4, st));
  EBR_CUDA_TRY(cudaMemsetAsync(flags, 0, 4, st));
  const size_t smem = 1024 + (size_t)d * eb * (128 + B);
  auto kern = f8 ? k_gemm_tc<true> : k_gemm_tc<false>;
  EBR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<(n + 127) / 128, 128, smem, st>>>(ma, mu, n, B, d, out, flags);
  EBR_CUDA_TRY(cudaGetLastError());
  uint32_t hf = 0;
  EBR_CUDA_TRY(cudaMemcpyAsync(&hf, flags, 4, cudaMemcpyDeviceToHost, st));
  EBR_CUDA_TRY(cudaStreamSynchronize(st));
  cudaFreeAsync(flags, st);
  return check_device_flags(hf, f8 ? "ebr_debug_gemm_e4m3" : "ebr_debug_gemm_bf16");
}

}  // namespace ebr

using namespace ebr;

extern "C" int ebr_debug_gemm_bf16(const uint16_t *A, uint32_t n, const uint16_t *U, uint32_t B,
                                   uint32_t d, float *out, void *stream) {
  clear_error();
  return debug_gemm(false, A, n, U, B, d, out, stream);
}

extern "C" int ebr_debug_gemm_e4m3(const uint8_t *A, uint32_t n, const uint8_t *U, uint32_t B,
                                   uint32_t d, float *out, void *stream) {
  clear_error();
  return debug_gemm(true, A, n, U, B, d, out, stream);
}

namespace ebr {

// A wait nobody ends: the bounded-wait path must give up and flag it.
__global__ void k_wait_timeout(uint64_t timeout_ns, uint32_t *flags) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, 0, timeout_ns))
    atomicOr(flags, DEVERR_TIMEOUT);
  __syncthreads();
}

}  // namespace ebr

extern "C" int ebr_debug_wait_timeout(uint32_t timeout_us, void *stream) {
  using namespace ebr;
  clear_error();
  if (timeout_us == 0 || timeout_us > 1000000u) {
    set_error("ebr_debug_wait_timeout: timeout_us must be 1 .. 10^6");
    return EBR_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t *flags = nullptr;
  EBR_CUDA_TRY(cudaMallocAsync((void **)&flags, 4, st));
  EBR_CUDA_TRY(cudaMemsetAsync(flags, 0, 4, st));
  k_wait_timeout<<<1, 32, 0, st>>>((uint64_t)timeout_us * 1000ull, flags);
  EBR_CUDA_TRY(cudaGetLastError());
  uint32_t hf = 0;
  EBR_CUDA_TRY(cudaMemcpyAsync(&hf, flags, 4, cudaMemcpyDeviceToHost, st));
  EBR_CUDA_TRY(cudaStreamSynchronize(st));
  cudaFreeAsync(flags, st);
  return check_device_flags(hf, "ebr_debug_wait_timeout");
}

// =====================================================================
// Batched scan: B users against every ad, one pass over the inventory
// =====================================================================
// Per window of 256 ads (one persistent CTA per SM, contiguous windows):
//   producer warp   -- tensor TMA of the window's BF16/FP8 ad rows into a
//                      stage ring; the users' vectors are loaded once;
//   MMA warp        -- tcgen05.mma with the users as the M side and the
//                      window's ads as N = 256, in two M-tiles: the even
//                      users and the odd users (the user table is stored in
//                      that pair order), each replicated down the 128 TMEM
//                      lanes when the batch has fewer than 256 users;
//                      deep[user][ad] (Eq. 1) lands in TMEM, FP32;
//   list warps (2)  -- walk the window's blocks in the window-major view of
//                      the compressed list and lay out, per run of 32 ads, a
//                      key table T[r][i] = r-th key of ad i (the window's
//                      slice of L, transposed; short ads padded with a zero
//                      row of w^T);
//   epilogue (8)    -- thread = user pair (2u, 2u + 1) at TMEM lane L
//                      (u = L mod Bq/2), runs of 32 ads per warp:
//                      wide[i] += w^T[T[r][i]][2u .. 2u + 1] for every row r
//                      (32 independent coalesced 8-byte loads and 32 paired
//                      FP32 adds per row, accumulators in registers), added
//                      to both users' deep scores (TMEM columns c and
//                      256 + c), filtered, and each user's candidates above
//                      its running threshold go to this CTA's per-user buffer
//                      (top-m kept exactly).
// With Bq/2 user pairs per replica (32, 64 or 128), the 256/(Bq/2) warps
// that hold the same pairs split the window's ads, Bq/2 ads each.
namespace ebr {

constexpr int kBWin = 256;
constexpr int kEpiWarps = 8, kListWarps = 2;
constexpr int kEpiThreads = kEpiWarps * 32, kListThreads = kListWarps * 32;
constexpr int kMmaWarp = kEpiWarps + kListWarps, kProdWarpB = kMmaWarp + 1;
constexpr int kBatchThreads = (kProdWarpB + 1) * 32;  // 384
constexpr int kMaxUsers = 256;
static_assert(kBWin % (kListWarps * 32) == 0, "list threads split the window's ads evenly");
// List buffer: run_off[8], run_rows[8], fill[256], then the run tables.
constexpr uint32_t kListHdr = 8 + 8 + kBWin;
constexpr uint32_t kMaxBatchKeysPerAd = 64;  // longest key list the batched tables hold

// Row of user b in the batch's user table: even users first, then odd ones
// (the two M-tiles of the batched scan), `half` = Bq / 2 rows each.
__host__ __device__ __forceinline__ uint32_t user_row(uint32_t b, uint32_t half) {
  return (b & 1u) * half + (b >> 1);
}

struct CandEntry {
  unsigned long long key;  // approximate score | id
  float wide;              // the ad's wide term for this user (FP32 sum)
  uint32_t pad;
};

struct BatchArgs {
  CUtensorMap ta;  // ad rows, BF16 or FP8 [N][d], box {tile row, 128}
  CUtensorMap tu;  // users, same type [Bq][d] in pair order, box {tile row, Bq / 2}
  const uint32_t *wkey[kGroups];
  const uint8_t *wvals[kGroups];
  const uint32_t *win_ptr[kGroups];
  const uint16_t *ad_nkeys;    // [N] distinct keys of each ad
  const float *wT;             // [n_keys + 1][Bq] expanded weights, user-minor; last row 0
  const uint64_t *filters;     // [B][words] (rows of users without a filter are unused)
  const uint32_t *has_filter;  // [B]
  uint32_t n_ads, n_win, B, Bq, d, m, cap_u, list_cap, words;  // B: users (buffer stride)
  const uint32_t *B_dev;       // non-null: the active users (<= B) are read here at launch
  uint32_t zero_row;           // n_keys * Bq / 2: the zero row of wT, in user-pair units
  uint32_t sa, lb, tb;         // A stages, list buffers, TMEM buffers
  uint32_t tile_row, kb_n;     // bytes per K-tile row (128 or 64), K-tiles per row
  const float *ad_scale;       // FP8: [N] row scales of the ad table
  const float *user_scale;     // FP8: [Bq] row scales of the quantised users (pair order)
  CandEntry *cand;             // [grid][B][cap_u]
  uint32_t *cand_n;            // [grid][B]
  unsigned long long *cand_thr;  // [grid][B]
  Ctrl *ctrl;
};

struct BatchSmem {
  uint64_t a_full[2], a_empty[2], t_full[2], t_empty[2], l_full[2], l_empty[2], u_full;
  uint32_t tmem_base;
  uint32_t cnt_u[kMaxUsers];
  unsigned long long thr_u[kMaxUsers];
  uint32_t abort, stop_epi, stop_list, n_issued, n_mma;
};

__device__ __forceinline__ uint32_t ushift(uint32_t g) { return g >= 2 ? g - 2 : 0; }

// Walk the real slots of window w: f(ad_in_window, key).  `t`/`nt`: this
// thread's index in the walking group (whole warps).  The window's block
// range in each of the nine groups is read once (one lane per group) and the
// groups' work units are walked as one sequence, eight units per thread
// loaded before any is used, so loads stay in flight across group borders.
template <typename F>
__device__ __forceinline__ void walk_window(const BatchArgs &a, uint32_t w, int t, int nt, F f) {
  constexpr int kU = 8;
  const int lane = threadIdx.x & 31;
  uint32_t lo_l = 0, n_l = 0;
  if (lane < kGroups) {
    const uint32_t lo = __ldg(a.win_ptr[lane] + w), hi = __ldg(a.win_ptr[lane] + w + 1);
    lo_l = lo;
    n_l = (hi - lo) << ushift(lane);
  }
  uint32_t lo_g[kGroups], end_g[kGroups];  // first block, end of the group's units
  uint32_t total = 0;
#pragma unroll
  for (int g = 0; g < kGroups; g++) {
    lo_g[g] = __shfl_sync(0xffffffffu, lo_l, g);
    total += __shfl_sync(0xffffffffu, n_l, g);
    end_g[g] = total;
  }
#pragma unroll 1
  for (uint32_t u0 = t; u0 < total; u0 += kU * nt) {
    uint32_t key[kU], word[kU], gg[kU], first[kU];
#pragma unroll
    for (int e = 0; e < kU; e++) {
      const uint32_t U = u0 + e * nt;
      const bool v = U < total;
      uint32_t g = 0;
#pragma unroll
      for (int i = 0; i < kGroups - 1; i++) g += U >= end_g[i] ? 1u : 0u;
      uint32_t lo = lo_g[0], beg = 0;
#pragma unroll
      for (int i = 1; i < kGroups; i++)
        if (g == (uint32_t)i) {
          lo = lo_g[i];
          beg = end_g[i - 1];
        }
      const uint32_t us = ushift(g), u = U - beg;
      const uint32_t bk = lo + (v ? (u >> us) : 0u), wi = u & ((1u << us) - 1u);
      key[e] = v ? __ldg(a.wkey[g] + bk) : 0u;
      if (!v)
        word[e] = 0u;
      else if (g >= 2)
        word[e] = __ldg(reinterpret_cast<const uint32_t *>(a.wvals[g]) + (((uint64_t)bk << us) + wi));
      else if (g == 1)
        word[e] = __ldg(reinterpret_cast<const unsigned short *>(a.wvals[1]) + bk);
      else
        word[e] = __ldg(a.wvals[0] + bk);
      gg[e] = g;
      first[e] = (v && wi == 0) ? 1u : 0u;
    }
#pragma unroll
    for (int e = 0; e < kU; e++) {
      if (u0 + e * nt >= total) break;
      const uint32_t ns = gg[e] >= 2 ? 4u : (gg[e] == 1 ? 2u : 1u);
      for (uint32_t s = 0; s < ns; s++) {
        const uint32_t l = (word[e] >> (8 * s)) & 255u;
        if ((s == 0 && first[e]) || l != 0) f(l, key[e]);
      }
    }
  }
}

// Warp-level radix select: T with exactly `need` keys >= T among n (global).
__device__ uint64_t warp_radix_select(const CandEntry *buf, uint32_t n, uint32_t need,
                                      uint32_t *hist /* 256 words, this warp's */) {
  const int lane = threadIdx.x & 31;
  uint64_t prefix = 0;
  for (int shift = 56; shift >= 0; shift -= 8) {
    for (int i = lane; i < 256; i += 32) hist[i] = 0;
    __syncwarp();
    const uint64_t hi_mask = (shift == 56) ? 0ull : (~0ull << (shift + 8));
    for (uint32_t i = lane; i < n; i += 32) {
      const uint64_t x = buf[i].key;
      if ((x & hi_mask) == prefix) atomicAdd(&hist[(x >> shift) & 255u], 1u);
    }
    __syncwarp();
    uint32_t c[8], tot = 0;
#pragma unroll
    for (int e = 0; e < 8; e++) {
      c[e] = hist[255 - 8 * lane - e];
      tot += c[e];
    }
    uint32_t incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    uint32_t acc = incl - tot, dg = 0, nn = 0, whole = 0;
    bool found = false;
#pragma unroll
    for (int e = 0; e < 8; e++) {
      if (!found && acc < need && need <= acc + c[e]) {
        found = true;
        dg = 255 - 8 * lane - e;
        nn = need - acc;
        whole = (need - acc == c[e]) ? 1u : 0u;
      }
      acc += c[e];
    }
    const uint32_t bal = __ballot_sync(0xffffffffu, found);
    const int src = __ffs(bal) - 1;
    dg = __shfl_sync(0xffffffffu, dg, src);
    need = __shfl_sync(0xffffffffu, nn, src);
    whole = __shfl_sync(0xffffffffu, whole, src);
    prefix |= (uint64_t)dg << shift;
    __syncwarp();
    if (whole) break;
  }
  return prefix;
}

// Stable in-place compaction of buf[0..n) to the entries with key >= T;
// returns how many were kept.
__device__ uint32_t warp_compact(CandEntry *buf, uint32_t n, uint64_t T) {
  const int lane = threadIdx.x & 31;
  uint32_t kept = 0;
  for (uint32_t b0 = 0; b0 < n; b0 += 32) {
    const uint32_t i = b0 + lane;
    CandEntry e;
    e.key = 0;
    if (i < n) e = buf[i];
    const bool kp = i < n && e.key >= T;
    const uint32_t bal = __ballot_sync(0xffffffffu, kp);
    __syncwarp();
    if (kp) buf[kept + __popc(bal & ((1u << lane) - 1u))] = e;
    kept += __popc(bal);
    __syncwarp();
  }
  return kept;
}

// The same selection and compaction on a buffer of at most 32 * NPL entries,
// read once into registers: the eight digit passes then touch only the
// shared-memory histogram, and the survivors are written back in one sweep.
// Returns how many were kept; *T_out = the selected cut.
constexpr int kSelNpl = 28;  // entries per lane of the register form (896 per buffer)
template <int NPL>
__device__ uint32_t warp_trim_regs(CandEntry *buf, uint32_t n, uint32_t need, uint32_t *hist,
                                   uint64_t *T_out) {
  const int lane = threadIdx.x & 31;
  uint64_t x[NPL];
  float wd[NPL];
#pragma unroll
  for (int e = 0; e < NPL; e++) {
    const uint32_t i = lane + 32u * e;
    x[e] = 0ull;
    wd[e] = 0.f;
    if (i < n) {
      const CandEntry c = buf[i];
      x[e] = c.key;
      wd[e] = c.wide;
    }
  }
  uint64_t prefix = 0;
  for (int shift = 56; shift >= 0; shift -= 8) {
    for (int i = lane; i < 256; i += 32) hist[i] = 0;
    __syncwarp();
    const uint64_t hi_mask = (shift == 56) ? 0ull : (~0ull << (shift + 8));
#pragma unroll
    for (int e = 0; e < NPL; e++)
      if (lane + 32u * e < n && (x[e] & hi_mask) == prefix)
        atomicAdd(&hist[(x[e] >> shift) & 255u], 1u);
    __syncwarp();
    uint32_t c[8], tot = 0;
#pragma unroll
    for (int e = 0; e < 8; e++) {
      c[e] = hist[255 - 8 * lane - e];
      tot += c[e];
    }
    uint32_t incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    uint32_t acc = incl - tot, dg = 0, nn = 0, whole = 0;
    bool found = false;
#pragma unroll
    for (int e = 0; e < 8; e++) {
      if (!found && acc < need && need <= acc + c[e]) {
        found = true;
        dg = 255 - 8 * lane - e;
        nn = need - acc;
        whole = (need - acc == c[e]) ? 1u : 0u;
      }
      acc += c[e];
    }
    const uint32_t bal = __ballot_sync(0xffffffffu, found);
    const int src = __ffs(bal) - 1;
    dg = __shfl_sync(0xffffffffu, dg, src);
    need = __shfl_sync(0xffffffffu, nn, src);
    whole = __shfl_sync(0xffffffffu, whole, src);
    prefix |= (uint64_t)dg << shift;
    __syncwarp();
    if (whole) break;
  }
  uint32_t kept = 0;
#pragma unroll
  for (int e = 0; e < NPL; e++) {
    const bool kp = lane + 32u * e < n && x[e] >= prefix;
    const uint32_t bal = __ballot_sync(0xffffffffu, kp);
    if (kp) {
      CandEntry c;
      c.key = x[e];
      c.wide = wd[e];
      c.pad = 0;
      buf[kept + __popc(bal & ((1u << lane) - 1u))] = c;
    }
    kept += __popc(bal);
  }
  __syncwarp();
  *T_out = prefix;
  return kept;
}

// Exact top-`need` of a per-user buffer, in place; returns how many were kept.
__device__ __forceinline__ uint32_t warp_trim(CandEntry *buf, uint32_t n, uint32_t need,
                                              uint32_t *hist, uint64_t *T_out) {
  if (n <= 32u * kSelNpl) return warp_trim_regs<kSelNpl>(buf, n, need, hist, T_out);
  const uint64_t T = warp_radix_select(buf, n, need, hist);
  *T_out = T;
  return warp_compact(buf, n, T);
}

template <bool F8>
__global__ void __launch_bounds__(kBatchThreads, 1) k_batch_window(const __grid_constant__ BatchArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ BatchSmem sm;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t kb_n = a.kb_n, tr = a.tile_row;  // K-tiles per row, bytes per tile row
  const uint32_t tile_elems = tr / (F8 ? 1u : 2u);
  const uint32_t n_mt = 2;                        // M-tiles: even users, odd users
  const uint32_t u_tile = kb_n * 128u * tr;        // one M-tile: kb_n x [128 rows x tr]
  const uint32_t a_stage = kb_n * 256u * tr;       // kb_n x [256 ad rows x tr]
  uint8_t *su = smem;                              // n_mt user tiles
  uint8_t *sa = su + (size_t)n_mt * u_tile;        // sa ad stages
  uint32_t *lists = reinterpret_cast<uint32_t *>(sa + (size_t)a.sa * a_stage);
  const uint32_t list_words = kListHdr + a.list_cap;
  uint32_t *whist = lists + (size_t)a.lb * list_words;  // [8][256] radix histograms

  const uint32_t w_begin = (uint32_t)(((uint64_t)a.n_win * blockIdx.x) / gridDim.x);
  const uint32_t w_end = (uint32_t)(((uint64_t)a.n_win * (blockIdx.x + 1)) / gridDim.x);
  const uint32_t my_wins = w_end - w_begin;
  const uint32_t tcols = 256u * n_mt;  // TMEM columns per window
  const uint32_t ncols = 512;
  // active users: all B, or the count a device-side loop wrote for this wave
  // (the same for every thread; none: nothing to do, nothing allocated)
  const uint32_t nB = a.B_dev ? min(*a.B_dev, a.B) : a.B;
  if (nB == 0) return;

  for (uint32_t b = tid; b < a.B; b += kBatchThreads) {
    sm.cnt_u[b] = 0;
    sm.thr_u[b] = 0ull;
  }
  if (warp == kMmaWarp) {
    tmem_alloc(&sm.tmem_base, ncols);
    tmem_relinquish();
  }
  if (tid == 0) {
    sm.abort = 0;
    sm.stop_epi = 0;
    sm.n_issued = 0;
    sm.n_mma = 0;
    for (int q = 0; q < 2; q++) {
      mbar_init(&sm.a_full[q], 1);
      mbar_init(&sm.a_empty[q], 1);
      mbar_init(&sm.t_full[q], 1);
      mbar_init(&sm.t_empty[q], 1);
      mbar_init(&sm.l_full[q], kListThreads);
      mbar_init(&sm.l_empty[q], 1);
    }
    mbar_init(&sm.u_full, 1);
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sm.tmem_base;

  if (warp == kProdWarpB) {
    // ---------------------------------------------------------- producer
    if (lane == 0) {
      const uint64_t pol = l2_evict_first_policy();
      // users (stored in pair order: even users, then odd users): row r of
      // M-tile mt holds user 2 (r mod Bq/2) + mt (replicas when Bq < 256)
      const uint32_t box_u = a.Bq / 2;
      mbar_arrive_expect_tx(&sm.u_full, n_mt * u_tile);
      for (uint32_t mt = 0; mt < n_mt; mt++)
        for (uint32_t r0 = 0; r0 < 128; r0 += box_u)
          for (uint32_t kb = 0; kb < kb_n; kb++)
            tma_load_2d(su + mt * u_tile + kb * 128u * tr + r0 * tr, &a.tu,
                        (int)(kb * tile_elems), (int)(mt * box_u), &sm.u_full);
      for (uint32_t j = 0; j < my_wins; j++) {
        const uint32_t s = j % a.sa;
        if (j >= a.sa && !mbar_wait_bounded(&sm.a_empty[s], ((j / a.sa) - 1) & 1u, kWaitTimeoutNs)) {
          atomicOr(&a.ctrl->flags, DEVERR_TIMEOUT);
          sm.abort = 1;
          break;
        }
        if (*((volatile uint32_t *)&sm.abort)) break;
        const int row0 = (int)((w_begin + j) * kBWin);
        uint8_t *dst = sa + (size_t)s * a_stage;
        mbar_arrive_expect_tx(&sm.a_full[s], a_stage);
        for (uint32_t kb = 0; kb < kb_n; kb++)
          for (uint32_t h = 0; h < 2; h++)
            tma_load_2d_hint(dst + kb * 256u * tr + h * 128u * tr, &a.ta, (int)(kb * tile_elems),
                             row0 + (int)h * 128, &sm.a_full[s], pol);
        sm.n_issued = j + 1;
      }
    }
  } else if (warp == kMmaWarp) {
    // ---------------------------------------------------------- MMA issuer
    if (lane == 0) {
      bool ok = mbar_wait_bounded(&sm.u_full, 0, kWaitTimeoutNs);
      const uint32_t idesc = F8 ? idesc_e4m3_f32(128, 256) : idesc_bf16_f32(128, 256);
      const uint32_t spt = tr / 32;  // 32-byte K-steps per tile row
      for (uint32_t j = 0; ok && j < my_wins; j++) {
        const uint32_t s = j % a.sa, tb = j % a.tb;
        ok = mbar_wait_bounded(&sm.a_full[s], (j / a.sa) & 1u, kWaitTimeoutNs);
        if (ok && j >= a.tb) ok = mbar_wait_bounded(&sm.t_empty[tb], ((j / a.tb) - 1) & 1u, kWaitTimeoutNs);
        if (!ok || *((volatile uint32_t *)&sm.abort)) break;
        tc_fence_after();
        const uint8_t *as = sa + (size_t)s * a_stage;
        for (uint32_t mt = 0; mt < n_mt; mt++) {
          const uint32_t dcol = tmem + tb * tcols + mt * 256u;
          for (uint32_t k = 0; k < kb_n * spt; k++) {
            const uint32_t kb = k / spt, kk = k % spt;
            const uint32_t ua = smem_u32(su + mt * u_tile + kb * 128u * tr + kk * 32);
            const uint32_t aa = smem_u32(as + kb * 256u * tr + kk * 32);
            const uint64_t ud = tr == 128 ? sdesc_k_sw128(ua) : sdesc_k_sw64(ua);
            const uint64_t ad = tr == 128 ? sdesc_k_sw128(aa) : sdesc_k_sw64(aa);
            if (F8)
              umma_e4m3(dcol, ud, ad, idesc, k > 0 ? 1u : 0u);
            else
              umma_bf16(dcol, ud, ad, idesc, k > 0 ? 1u : 0u);
          }
        }
        umma_commit(&sm.a_empty[s]);
        umma_commit(&sm.t_full[tb]);
        sm.n_mma = j + 1;
      }
      if (!ok) {
        atomicOr(&a.ctrl->flags, DEVERR_TIMEOUT);
        sm.abort = 1;
      }
    }
  } else if (warp >= kEpiWarps) {
    // ---------------------------------------------------------- list builders
    // Per window: off[l] = first slot of ad l (exclusive scan of the ads' key
    // counts), then one walk of the window's blocks drops each key into its
    // ad's slot range.
    const int lt = tid - kEpiThreads;
    for (uint32_t j = 0; j < my_wins; j++) {
      const uint32_t lbuf = j % a.lb;
      if (lt == 0) {
        uint32_t stop = *((volatile uint32_t *)&sm.abort);
        if (!stop && j >= a.lb &&
            !mbar_wait_bounded(&sm.l_empty[lbuf], ((j / a.lb) - 1) & 1u, kWaitTimeoutNs)) {
          atomicOr(&a.ctrl->flags, DEVERR_TIMEOUT);
          sm.abort = 1;
          stop = 1;
        }
        sm.stop_list = stop;
      }
      named_sync(2, kListThreads);
      if (sm.stop_list) break;
      if (j >= a.lb) mbar_try_wait(&sm.l_empty[lbuf], ((j / a.lb) - 1) & 1u);
      uint32_t *run_off = lists + (size_t)lbuf * list_words;
      uint32_t *run_rows = run_off + 8;
      uint32_t *fill = run_off + 16;
      uint32_t *tab = run_off + kListHdr;
      const uint32_t w = w_begin + j;
      // rows of each run = most keys of its 32 ads; thread lt owns ads
      // lt, lt + kListThreads, ... (whole warps per run of 32 ads)
      constexpr int kPer = kBWin / kListThreads;
      uint32_t nk[kPer];
#pragma unroll
      for (int h = 0; h < kPer; h++) {
        const uint32_t al = lt + kListThreads * h;
        const uint32_t ad = w * kBWin + al;
        nk[h] = ad < a.n_ads ? (uint32_t)__ldg(a.ad_nkeys + ad) : 0u;
        fill[al] = 0;
        uint32_t mx = nk[h];
#pragma unroll
        for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) run_rows[al >> 5] = mx;
      }
      named_sync(2, kListThreads);
      uint32_t ro[kPer], rr[kPer];
      {
        uint32_t acc = 0;
        for (uint32_t r = 0; r < 8; r++) {
          const uint32_t rows = run_rows[r];
#pragma unroll
          for (int h = 0; h < kPer; h++)
            if (r == ((lt + kListThreads * h) >> 5)) {
              ro[h] = acc;
              rr[h] = rows;
            }
          if (lt == 0) run_off[r] = acc;
          acc += rows * 32u;
        }
      }
      // padding entries (rows nk .. rows-1) point at the zero row
#pragma unroll
      for (int h = 0; h < kPer; h++)
        for (uint32_t r = nk[h]; r < rr[h]; r++) {
          const uint32_t pos = ro[h] + r * 32u + (uint32_t)lane;
          if (pos < a.list_cap) tab[pos] = a.zero_row;
        }
      named_sync(2, kListThreads);
      walk_window(a, w, lt, kListThreads, [&](uint32_t l, uint32_t key) {
        const uint32_t rank = atomicAdd(&fill[l], 1u);
        const uint32_t pos = run_off[l >> 5] + rank * 32u + (l & 31u);
        if (rank < run_rows[l >> 5] && pos < a.list_cap) tab[pos] = key * (a.Bq / 2);
      });
      mbar_arrive(&sm.l_full[lbuf]);  // release: this thread's list writes
    }
  } else {
    // ---------------------------------------------------------- epilogue
    // Thread = user pair (2u, 2u + 1): M-tile 0 holds the even users and
    // M-tile 1 the odd ones, each replicated down the 128 lanes, so lane L
    // reads both users' deep scores (columns c and 256 + c) and gathers
    // both users' weights with one 8-byte load of the user-minor w^T.
    const GroupSync gsync{1, kEpiThreads};
    const uint32_t q = warp % 4;                  // TMEM lane quadrant of this warp
    uint32_t *hist = whist + warp * 256;
    const uint32_t U2 = a.Bq / 2;                 // user pairs (32, 64 or 128)
    const uint32_t pair = (32u * q + lane) % U2;
    const uint32_t ad_lo = ((warp / 4) * (128 / U2) + q / (U2 / 32)) * U2, n_ads_w = U2;
    const uint32_t tl = tmem + ((32u * q) << 16);
    const uint32_t user0 = 2 * pair, user1 = 2 * pair + 1;
    const bool ok0 = user0 < nB, ok1 = user1 < nB;
    // FP8: deep = TMEM x (user scale) x (the ad row's scale); user rows in pair order
    const float usc0 = F8 && ok0 ? a.user_scale[pair] : 1.f;
    const float usc1 = F8 && ok1 ? a.user_scale[U2 + pair] : 1.f;
    const bool filt0 = ok0 && a.has_filter[user0], filt1 = ok1 && a.has_filter[user1];
    const uint64_t *frow0 = a.filters + (uint64_t)(ok0 ? user0 : 0u) * a.words;
    const uint64_t *frow1 = a.filters + (uint64_t)(ok1 ? user1 : 0u) * a.words;
    const float2 *wcol = reinterpret_cast<const float2 *>(a.wT) + pair;
    CandEntry *ubuf0 = a.cand + ((uint64_t)blockIdx.x * a.B + (ok0 ? user0 : 0u)) * a.cap_u;
    CandEntry *ubuf1 = a.cand + ((uint64_t)blockIdx.x * a.B + (ok1 ? user1 : 0u)) * a.cap_u;
    // one (user, ad) score: filtered, thresholded, appended to the user's buffer
    auto offer = [&](uint32_t user, bool filt, const uint64_t *frow, CandEntry *ubuf,
                     unsigned long long thr, float deep, float wide, uint32_t ad) {
      const unsigned long long key = make_key(deep + wide, ad);
      if (key < thr) return;
      if (filt && !((__ldg(frow + (ad >> 6)) >> (ad & 63)) & 1ull)) return;
      const uint32_t pos = atomicAdd(&sm.cnt_u[user], 1u);
      if (pos < a.cap_u) {
        CandEntry ce;
        ce.key = key;
        ce.wide = wide;
        ce.pad = 0;
        ubuf[pos] = ce;
      } else {
        atomicOr(&a.ctrl->flags, DEVERR_OVERFLOW);
      }
    };
    for (uint32_t j = 0; j < my_wins; j++) {
      const uint32_t tb = j % a.tb, lbuf = j % a.lb;
      if (tid == 0) {
        uint32_t stop = *((volatile uint32_t *)&sm.abort);
        if (!stop && !mbar_wait_bounded(&sm.t_full[tb], (j / a.tb) & 1u, kWaitTimeoutNs)) stop = 1;
        if (!stop && !mbar_wait_bounded(&sm.l_full[lbuf], (j / a.lb) & 1u, kWaitTimeoutNs)) stop = 1;
        if (stop && !*((volatile uint32_t *)&sm.abort)) {
          atomicOr(&a.ctrl->flags, DEVERR_TIMEOUT);
          sm.abort = 1;
        }
        sm.stop_epi = stop;
      }
      gsync();
      if (sm.stop_epi) break;
      mbar_try_wait(&sm.t_full[tb], (j / a.tb) & 1u);
      mbar_try_wait(&sm.l_full[lbuf], (j / a.lb) & 1u);
      tc_fence_after();
      const uint32_t *run_off = lists + (size_t)lbuf * list_words;
      const uint32_t *tab = run_off + kListHdr;
      const uint32_t wbase = (w_begin + j) * kBWin;
      const unsigned long long thr0 = ok0 ? sm.thr_u[user0] : ~0ull;
      const unsigned long long thr1 = ok1 ? sm.thr_u[user1] : ~0ull;
      for (uint32_t c = 0; c < n_ads_w; c += 32) {
        const uint32_t a0 = ad_lo + c;  // first window-local ad of this run
        const uint32_t run = a0 >> 5;
        const uint32_t rows = run_off[8 + run];
        const uint4 *t4 = reinterpret_cast<const uint4 *>(tab + run_off[run]);
        float2 acc[32];
#pragma unroll
        for (int i = 0; i < 32; i++) acc[i] = make_float2(0.f, 0.f);
        for (uint32_t r = 0; r < rows; r++) {  // one row: 32 independent 8-byte loads
          float2 v[32];
#pragma unroll
          for (int i4 = 0; i4 < 8; i4++) {
            const uint4 k = t4[r * 8 + i4];
            v[4 * i4 + 0] = __ldg(wcol + k.x);
            v[4 * i4 + 1] = __ldg(wcol + k.y);
            v[4 * i4 + 2] = __ldg(wcol + k.z);
            v[4 * i4 + 3] = __ldg(wcol + k.w);
          }
#pragma unroll
          for (int i = 0; i < 32; i++) acc[i] = add_f32x2(acc[i], v[i]);
        }
        // lane i holds the row scale of the run's ad i (FP8)
        const uint32_t ad_l = wbase + a0 + lane;
        const float sa_l = F8 && ad_l < a.n_ads ? __ldg(a.ad_scale + ad_l) : 1.f;
#pragma unroll
        for (int h = 0; h < 2; h++) {
          uint32_t d0[16], d1[16];  // deep scores of 16 ads for both users, two TMEM loads
          tmem_ld16(tl + a0 + 16 * h, d0);
          tmem_ld16(tl + 256u + a0 + 16 * h, d1);
          tmem_ld_wait();
#pragma unroll
          for (int ii = 0; ii < 16; ii++) {
            const int i = 16 * h + ii;
            const float sa_i = F8 ? __shfl_sync(0xffffffffu, sa_l, i) : 1.f;
            const uint32_t ad = wbase + a0 + i;
            if (ad >= a.n_ads) continue;
            const float deep0 = F8 ? __uint_as_float(d0[ii]) * (sa_i * usc0) : __uint_as_float(d0[ii]);
            const float deep1 = F8 ? __uint_as_float(d1[ii]) * (sa_i * usc1) : __uint_as_float(d1[ii]);
            if (ok0) offer(user0, filt0, frow0, ubuf0, thr0, deep0, acc[i].x, ad);
            if (ok1) offer(user1, filt1, frow1, ubuf1, thr1, deep1, acc[i].y, ad);
          }
        }
      }
      tc_fence_before();
      gsync();
      if (tid == 0) {
        mbar_arrive(&sm.t_empty[tb]);
        mbar_arrive(&sm.l_empty[lbuf]);
      }
      // keep each user's buffer below capacity: exact top-m by radix select
      for (uint32_t b = warp; b < nB; b += kEpiWarps) {
        const uint32_t n = sm.cnt_u[b];
        if (n + kBWin <= a.cap_u) continue;
        CandEntry *buf = a.cand + ((uint64_t)blockIdx.x * a.B + b) * a.cap_u;
        const uint32_t nn = min(n, a.cap_u);
        uint64_t T;
        const uint32_t kept = warp_trim(buf, nn, a.m, hist, &T);
        if (lane == 0) {
          sm.cnt_u[b] = kept;
          sm.thr_u[b] = T;
        }
        __syncwarp();
      }
      gsync();
    }
    gsync();
    // final trim to at most m candidates per user (the merge reads grid * m)
    if (!sm.stop_epi) {
      for (uint32_t b = warp; b < nB; b += kEpiWarps) {
        const uint32_t n = min(sm.cnt_u[b], a.cap_u);
        if (n <= a.m) continue;
        CandEntry *buf = a.cand + ((uint64_t)blockIdx.x * a.B + b) * a.cap_u;
        uint64_t T;
        const uint32_t kept = warp_trim(buf, n, a.m, hist, &T);
        if (lane == 0) {
          sm.cnt_u[b] = kept;
          sm.thr_u[b] = T > sm.thr_u[b] ? T : sm.thr_u[b];
        }
        __syncwarp();
      }
    }
    gsync();
    for (uint32_t b = tid; b < a.B; b += kEpiThreads) {
      a.cand_n[(uint64_t)blockIdx.x * a.B + b] = min(sm.cnt_u[b], a.cap_u);
      a.cand_thr[(uint64_t)blockIdx.x * a.B + b] = sm.thr_u[b];
    }
  }
  // Drain before teardown (matters only after an abort): the last issued
  // tile loads must have landed and the last MMAs retired before the
  // shared memory and TMEM are released.
  __syncthreads();
  if (tid == 0) {
    const uint32_t ni = sm.n_issued, nm = sm.n_mma;
    bool ok = mbar_wait_bounded(&sm.u_full, 0, kWaitTimeoutNs);
    for (uint32_t j = ni > a.sa ? ni - a.sa : 0; ok && j < ni; j++)
      ok = mbar_wait_bounded(&sm.a_full[j % a.sa], (j / a.sa) & 1u, kWaitTimeoutNs);
    if (ok && nm) ok = mbar_wait_bounded(&sm.t_full[(nm - 1) % a.tb], ((nm - 1) / a.tb) & 1u, kWaitTimeoutNs);
    if (!ok) atomicOr(&a.ctrl->flags, DEVERR_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kMmaWarp) tmem_dealloc(tmem, ncols);
}

// Per user: the best R*K of the CTAs' candidate buffers (exact if no CTA's
// buffer threshold exceeds the selected cut), rescored in FP32, best K.
constexpr int kMergeThreads = 1024;
constexpr uint32_t kMergeCap = 32768;  // approximate candidates gathered per user

__global__ void __launch_bounds__(kMergeThreads) k_batch_merge(
    const CandEntry *__restrict__ cand, const uint32_t *__restrict__ cand_n,
    const unsigned long long *__restrict__ cand_thr, uint32_t grid, uint32_t B, uint32_t cap_u,
    const uint32_t *__restrict__ kscan, const uint32_t *__restrict__ kout, uint32_t kmax,
    const float *__restrict__ emb, uint32_t d, const float *__restrict__ h_u, uint32_t half,
    uint64_t *__restrict__ scratch /* [B][kMergeCap + 8192] */, uint32_t *__restrict__ out_ids,
    float *__restrict__ out_scores, uint32_t *__restrict__ status /* [B] */,
    const uint32_t *__restrict__ B_dev, const uint32_t *__restrict__ slot_dev,
    uint64_t out_slot_stride, uint32_t status_slot_stride) {
  extern __shared__ __align__(16) uint64_t s_v[];  // 8192 keys
  __shared__ uint32_t s_hist[256], s_misc[8], s_cnt;
  __shared__ uint32_t s_base[1024];
  __shared__ float s_h[128];
  const uint32_t b = blockIdx.x;
  // a device-side loop: only the wave's active users, results into its ring slot
  if (B_dev && b >= *B_dev) return;
  if (slot_dev) {
    const uint32_t slot = *slot_dev;
    out_ids += slot * out_slot_stride;
    out_scores += slot * out_slot_stride;
    status += (uint64_t)slot * status_slot_stride;
  }
  const uint32_t ks = kscan[b], ko = kout[b];
  uint64_t *keys = scratch + (uint64_t)b * (kMergeCap + 8192);  // gathered approximate keys
  uint32_t inexact = 0;
  // 1. gather this user's candidates into scratch (bounded by 8192: with the
  //    per-CTA thresholds far fewer survive; beyond that the request is flagged)
  if (threadIdx.x == 0) s_cnt = 0;
  const uint64_t hrow = user_row(b, half);  // the user table is in pair order
  for (uint32_t i = threadIdx.x; i < d; i += kMergeThreads) s_h[i] = h_u[hrow * d + i];
  __syncthreads();
  // count first, then copy (entries of all CTAs, in CTA order)
  uint32_t total = 0;
  for (uint32_t c0 = 0; c0 < grid; c0 += kMergeThreads) {
    const uint32_t c = c0 + threadIdx.x;
    const uint32_t n = c < grid ? cand_n[(uint64_t)c * B + b] : 0u;
    // block-wide exclusive scan of n (simple two-level)
    uint32_t incl = n;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) s_base[wp] = incl;
    __syncthreads();
    if (threadIdx.x < 32) {
      uint32_t x = s_base[threadIdx.x], in2 = x;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, in2, o);
        if (threadIdx.x >= o) in2 += v;
      }
      s_base[threadIdx.x] = in2 - x;
      if (threadIdx.x == 31) s_misc[4] = in2;
    }
    __syncthreads();
    const uint32_t start = total + s_base[wp] + incl - n;
    if (c < grid) {
      const CandEntry *src = cand + ((uint64_t)c * B + b) * cap_u;
      for (uint32_t i = 0; i < n; i++)
        if (start + i < kMergeCap) keys[start + i] = src[i].key;
    }
    total += s_misc[4];
    __syncthreads();
  }
  if (total > kMergeCap) {
    inexact = 1;
    total = kMergeCap;
  }
  // 2. the best ks of them by approximate score (T = 0: all of them)
  uint64_t T = 0;
  if (total > ks) T = cta_radix_select<kMergeThreads>(keys, total, ks, s_hist, s_misc);
  // Exactness: CTA c holds every one of its candidates with key >= its
  // threshold, so the union's best ks are the inventory's best ks when no
  // threshold lies above the selected cut T.
  for (uint32_t c = threadIdx.x; c < grid; c += kMergeThreads)
    if (cand_thr[(uint64_t)c * B + b] > T) inexact = 1;
  if (inexact) atomicOr(&status[b], 1u);
  // 3. FP32 rescoring of the survivors: gather (id, wide) into shared
  //    memory, then one warp per candidate (coalesced FP32 row read).
  if (threadIdx.x == 0) s_cnt = 0;
  __syncthreads();
  uint64_t *resc = keys + kMergeCap;
  for (uint32_t c = 0; c < grid; c++) {
    const uint32_t n = cand_n[(uint64_t)c * B + b];
    const CandEntry *src = cand + ((uint64_t)c * B + b) * cap_u;
    for (uint32_t i = threadIdx.x; i < n; i += kMergeThreads) {
      const CandEntry e = src[i];
      if (e.key < T || e.key == 0ull) continue;
      const uint32_t pos = atomicAdd(&s_cnt, 1u);
      if (pos < 8192) s_v[pos] = ((uint64_t)__float_as_uint(e.wide) << 32) | key_id(e.key);
    }
  }
  __syncthreads();
  const uint32_t nres = min(s_cnt, 8192u);
  {
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    for (uint32_t i = wp; i < nres; i += kMergeThreads / 32) {
      const uint64_t e = s_v[i];
      const uint32_t id = (uint32_t)e;
      const float *row = emb + (uint64_t)id * d;
      float dot = 0.f;
      for (uint32_t t = lane; t < d; t += 32) dot = fmaf(s_h[t], __ldg(row + t), dot);
      for (int o = 16; o; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
      if (lane == 0) resc[i] = make_key(dot + __uint_as_float((uint32_t)(e >> 32)), id);
    }
  }
  __syncthreads();
  // 4. best ko, sorted
  uint64_t T2 = 0;
  if (nres > ko) T2 = cta_radix_select<kMergeThreads>(resc, nres, ko, s_hist, s_misc);
  if (threadIdx.x == 0) s_cnt = 0;
  __syncthreads();
  const uint32_t take = min(nres, ko);
  uint32_t p2 = 1;
  while (p2 < take) p2 <<= 1;
  for (uint32_t i = threadIdx.x; i < nres; i += kMergeThreads) {
    const uint64_t x = resc[i];
    if (x >= T2) {
      const uint32_t pos = atomicAdd(&s_cnt, 1u);
      if (pos < p2) s_v[pos] = x;
    }
  }
  __syncthreads();
  for (uint32_t i = take + threadIdx.x; i < p2; i += kMergeThreads) s_v[i] = 0ull;
  // bitonic sort, descending
  for (uint32_t size = 2; size <= p2; size <<= 1)
    for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
      __syncthreads();
      for (uint32_t i = threadIdx.x; i < p2 / 2; i += kMergeThreads) {
        const uint32_t lo = 2 * i - (i & (stride - 1)), hi = lo + stride;
        const bool desc = (lo & size) == 0;
        const uint64_t x = s_v[lo], y = s_v[hi];
        if ((x < y) == desc) {
          s_v[lo] = y;
          s_v[hi] = x;
        }
      }
    }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < kmax; i += kMergeThreads) {
    const uint64_t x = i < take ? s_v[i] : 0ull;
    out_ids[(uint64_t)b * kmax + i] = i < take ? key_id(x) : 0xFFFFFFFFu;
    out_scores[(uint64_t)b * kmax + i] = i < take ? key_score(x) : -INFINITY;
  }
}

}  // namespace ebr

// =====================================================================
// Host side of the batched path
// =====================================================================
namespace ebr {

// Pointers of one request's inputs (device memory), gathered by
// k_stage_requests into the batch's contiguous arrays.
struct ReqSrc {
  const float *h_u;
  const uint32_t *vals;    // [n] user field values
  const uint64_t *filter;  // null: no filter
  const uint32_t *ptr;     // [f_u + 1] field offsets into vals; null: one value per field
  uint32_t n, base;        // values, and their first position in the batch's value array
};
constexpr uint32_t kStageWords = 8192;  // filter words per block of the gather

// Block (b, y): request b's user vector (to row user_row(b, half)), field
// values and field offsets (y == 0) and words [y * kStageWords, +kStageWords)
// of its filter.  With B_dev (a device-side loop launching Bq blocks), blocks
// past the wave's users zero their user row and stop.  With
// uptr set, the offsets are written (relative to the request's base, base[b]
// beside them) after a check that they start at 0, do not decrease and end
// at n; offsets that fail it are flagged and every field is left empty.
__global__ void __launch_bounds__(256) k_stage_requests(const ReqSrc *__restrict__ src,
                                                        uint32_t d, uint32_t fu, uint32_t words,
                                                        uint32_t half,
                                                        float *__restrict__ users,
                                                        uint32_t *__restrict__ vals,
                                                        uint32_t *__restrict__ uptr,
                                                        uint32_t *__restrict__ base,
                                                        uint64_t *__restrict__ filters,
                                                        uint32_t *__restrict__ flags,
                                                        const uint32_t *__restrict__ B_dev) {
  __shared__ uint32_t s_ok;
  const uint32_t b = blockIdx.x;
  if (B_dev && b >= *B_dev) {  // a device-side loop's wave has fewer users: zero the row
    if (blockIdx.y == 0)
      for (uint32_t t = threadIdx.x; t < d; t += blockDim.x)
        users[(size_t)user_row(b, half) * d + t] = 0.f;
    return;
  }
  const ReqSrc r = src[b];
  if (blockIdx.y == 0) {
    const size_t row = (size_t)user_row(b, half);
    for (uint32_t t = threadIdx.x; t < d; t += blockDim.x) users[row * d + t] = r.h_u[t];
    for (uint32_t t = threadIdx.x; t < r.n; t += blockDim.x) vals[(size_t)r.base + t] = r.vals[t];
    if (uptr) {
      if (threadIdx.x == 0) {
        uint32_t ok = 1;
        if (r.ptr) {
          uint32_t prev = 0;
          for (uint32_t i = 0; i <= fu; i++) {
            const uint32_t x = r.ptr[i];
            if ((i == 0 && x != 0) || x < prev || (i == fu && x != r.n)) ok = 0;
            prev = x;
          }
        }
        if (!ok) atomicOr(flags, DEVERR_BAD_USER);
        s_ok = ok;
        base[b] = r.base;
      }
      __syncthreads();
      for (uint32_t i = threadIdx.x; i <= fu; i += blockDim.x)
        uptr[(size_t)b * (fu + 1) + i] = !s_ok ? 0u : (r.ptr ? r.ptr[i] : i);
    }
  }
  if (r.filter) {
    const uint32_t w0 = blockIdx.y * kStageWords;
    const uint32_t w1 = min(words, w0 + kStageWords);
    for (uint32_t t = w0 + threadIdx.x; t < w1; t += blockDim.x)
      filters[(size_t)b * words + t] = r.filter[t];
  }
}

// Layout of the batch's user field values: request b's n[b] values start at
// base[b] (one value per field without user_ptr); returns the total.
static uint64_t user_vals_layout(const ebr_query *q, uint32_t B, uint32_t fu,
                                 std::vector<uint32_t> *n, std::vector<uint32_t> *base) {
  uint64_t t = 0;
  n->resize(B);
  base->resize(B);
  for (uint32_t b = 0; b < B; b++) {
    (*n)[b] = q[b].user_ptr ? q[b].n_user_vals : fu;
    (*base)[b] = (uint32_t)t;
    t += (*n)[b];
  }
  return t;
}

struct BatchPlan {
  uint32_t Bq, m, cap_u, sa, lb, tb, list_cap, tile_row, kb_n;
  size_t smem;
};

// Users of the M-tiles: the batch rounded up to 64, 128 or 256 (two tiles of
// Bq/2 user pairs' halves each).
static uint32_t users_pow2(uint32_t B) {
  uint32_t q = 64;
  while (q < B) q <<= 1;
  return q;
}

// Shared-memory layout of k_batch_window: the users' M-tiles, `sa` ad
// stages, `lb` per-ad key lists and the epilogue's per-warp score tiles.
// Preference: two list buffers (list building then overlaps the epilogue),
// then two ad stages.
static bool plan_smem(const ebr_index *ix, uint32_t B, BatchPlan *p) {
  p->Bq = users_pow2(B);
  p->list_cap = kBWin * ix->max_keys_per_ad;  // 8 runs x 32 ads x rows
  const uint32_t n_mt = 2;  // even and odd users: 512 TMEM columns per window
  p->tb = 1;
  const uint32_t row_bytes = ix->d * (ix->dtype == EBR_FP8E4M3 ? 1u : 2u);
  p->tile_row = row_bytes >= 128 ? 128u : 64u;
  p->kb_n = row_bytes / p->tile_row;
  const size_t u_bytes = (size_t)n_mt * p->kb_n * 128 * p->tile_row;
  const size_t a_stage = (size_t)p->kb_n * 256 * p->tile_row;
  const size_t list_bytes = ((size_t)kListHdr + p->list_cap) * 4;
  const size_t hist = (size_t)kEpiWarps * 256 * 4;
  const size_t budget = 220 * 1024;
  const uint32_t order[4][2] = {{2, 2}, {1, 2}, {2, 1}, {1, 1}};  // {sa, lb}
  for (const auto &o : order) {
    const size_t need = 1024 + u_bytes + o[0] * a_stage + o[1] * list_bytes + hist;
    if (need <= budget) {
      p->sa = o[0];
      p->lb = o[1];
      p->smem = need;
      return true;
    }
  }
  return false;
}

bool batch_index_ok(const ebr_index *ix, const ebr_cross *cross, uint32_t batch) {
  BatchPlan p;
  return (ix->dtype == EBR_BF16 || ix->dtype == EBR_FP8E4M3) && (ix->d == 64 || ix->d == 128) &&
         batch >= 2 && batch <= (uint32_t)kMaxUsers && cross && cross->n_keys == ix->n_keys &&
         ix->n_win > 0 && ix->ad_nkeys.p && ix->max_keys_per_ad > 0 &&
         ix->max_keys_per_ad <= kMaxBatchKeysPerAd &&
         (uint64_t)(ix->n_keys + 1) * users_pow2(batch) < (1ull << 32) &&
         plan_smem(ix, batch, &p);
}

bool batch_qualifies(const ebr_index *ix, const ebr_cross *cross, const ebr_query *q,
                     uint32_t batch) {
  if (!batch_index_ok(ix, cross, batch)) return false;
  for (uint32_t b = 0; b < batch; b++) {
    if (!q[b].user_vals || (q[b].flags & EBR_QF_KEY_MAJOR)) return false;
    if ((uint64_t)q[b].k * ix->rescore_mult > 8192) return false;
  }
  return true;
}

static bool plan_batch(const ebr_index *ix, uint32_t B, uint32_t kscan_max, int grid,
                       BatchPlan *p) {
  if (!plan_smem(ix, B, p)) return false;
  const uint32_t per_cta = (kscan_max + grid - 1) / grid;
  p->m = std::max<uint32_t>(64, (2 * per_cta + 32 + 31) / 32 * 32);
  p->cap_u = 4 * p->m + kBWin;  // a trim every 3m insertions at least
  return (uint64_t)grid * p->m <= kMergeCap;
}

// Device bytes of every buffer of one batched call (B users, scan depth up to
// kscan_max), in one place for the reservation below and the serving loop's
// memory budget.  The pinned host mirror holds [kscan B][kout B][has_filter B]
// [status B] words, then the request pointer table.
struct BatchSizes {
  BatchPlan pl;
  int grid;
  size_t users_f32, users_q, users_scale, user_vals, user_ptr, wT, filters, small, cand, cand_n,
      cand_thr, scratch, ctrl, req, host;
  size_t total() const {
    size_t t = 0;
    for (size_t b : {users_f32, users_q, users_scale, user_vals, user_ptr, wT, filters, small,
                     cand, cand_n, cand_thr, scratch, ctrl, req})
      t += (b + 255) / 256 * 256;
    return t;
  }
};

static size_t host_table_off(uint32_t B) { return ((size_t)4 * B * 4 + 15) / 16 * 16; }

static bool batch_sizes(const ebr_index *ix, const ebr_cross *cross, uint32_t B,
                        uint32_t kscan_max, uint64_t n_vals, BatchSizes *z) {
  if (n_vals == 0) n_vals = (uint64_t)B * cross->f_u;
  z->grid = std::max(1, std::min<int>(ix->num_sms, (int)ix->n_win));
  if (!plan_batch(ix, B, kscan_max, z->grid, &z->pl)) return false;
  const size_t Bp = z->pl.Bq, d = ix->d, words = (ix->n_ads + 63) / 64;
  z->users_f32 = Bp * d * 4;
  z->users_q = Bp * d * 2;  // BF16 or FP8 users
  z->users_scale = Bp * 4;
  z->user_vals = (size_t)n_vals * 4;
  z->user_ptr = (size_t)B * (cross->f_u + 2) * 4;  // offsets [B][f_u + 1], then base [B]
  z->wT = ((size_t)ix->n_keys + 1) * Bp * 4;
  z->filters = (size_t)B * words * 8;
  z->small = small_bytes(B);
  z->cand = (size_t)z->grid * B * z->pl.cap_u * sizeof(CandEntry);
  z->cand_n = (size_t)z->grid * B * 4;
  z->cand_thr = (size_t)z->grid * B * 8;
  z->scratch = (size_t)B * (kMergeCap + 8192) * 8;
  z->ctrl = sizeof(Ctrl);
  z->req = (size_t)B * sizeof(ReqSrc);
  // after the words: the pointer table (device requests) or the packed user
  // vectors and field values (host requests)
  z->host = host_table_off(B) + std::max(z->req, Bp * d * 4 + z->user_ptr + z->user_vals);
  return true;
}

size_t batch_ws_bytes(const ebr_index *ix, const ebr_cross *cross, uint32_t B,
                      uint32_t kscan_max, uint64_t n_vals) {
  BatchSizes z;
  return batch_sizes(ix, cross, B, kscan_max, n_vals, &z) ? z.total() : 0;
}

int batch_ws_reserve(const ebr_index *ix, const ebr_cross *cross, uint32_t B,
                     uint32_t kscan_max, uint64_t n_vals, BatchWs &w) {
  BatchSizes z;
  if (!batch_sizes(ix, cross, B, kscan_max, n_vals, &z)) {
    set_error("batched scan: per-window key tables (%u keys per ad) do not fit shared memory",
              ix->max_keys_per_ad);
    return EBR_EINVAL;
  }
  EBR_TRY(dev_reserve(w.users_f32, z.users_f32));
  EBR_TRY(dev_reserve(w.users_bf16, z.users_q));
  EBR_TRY(dev_reserve(w.users_scale, z.users_scale));
  EBR_TRY(dev_reserve(w.user_vals, z.user_vals));
  EBR_TRY(dev_reserve(w.user_ptr, z.user_ptr));
  EBR_TRY(dev_reserve(w.wT, z.wT));
  EBR_TRY(dev_reserve(w.filters, z.filters));
  EBR_TRY(dev_reserve(w.small, z.small));
  EBR_TRY(dev_reserve(w.cand, z.cand));
  EBR_TRY(dev_reserve(w.cand_n, z.cand_n));
  EBR_TRY(dev_reserve(w.cand_thr, z.cand_thr));
  EBR_TRY(dev_reserve(w.scratch, z.scratch));
  EBR_TRY(dev_reserve(w.ctrl, z.ctrl));
  EBR_TRY(dev_reserve(w.req, z.req));
  if (w.host_bytes < z.host) {
    if (w.host) cudaFreeHost(w.host);
    w.host = nullptr;
    w.host_bytes = 0;
    if (cudaMallocHost(&w.host, z.host) != cudaSuccess) {
      cudaGetLastError();
      set_error("batched scan: pinned host allocation of %zu bytes failed", z.host);
      return EBR_ENOMEM;
    }
    w.host_bytes = z.host;
  }
  return EBR_OK;
}

static int stage(void *dst, const void *src, size_t bytes, int io, cudaStream_t st) {
  if (!bytes) return EBR_OK;
  EBR_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes,
                               io == EBR_IO_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                               st));
  return EBR_OK;
}

// The window kernel's arguments for a batch of B users (B: the candidate
// buffers' user stride; B_dev: the active users, read on the device, or null).
static int fill_batch_args(ebr_index *ix, uint32_t B, const BatchPlan &pl, BatchWs &w,
                           const uint32_t *has_filter, Ctrl *ctrl, const uint32_t *B_dev,
                           BatchArgs *out) {
  const bool f8 = ix->dtype == EBR_FP8E4M3;
  const uint32_t eb = f8 ? 1u : 2u, d = ix->d, Bp = pl.Bq;
  if (!w.tmap_ready || w.tmap_for != ix->emb_q.p) {
    EBR_TRY(make_tmap_2d(reinterpret_cast<CUtensorMap *>(w.tmap_bytes), ix->emb_q.p, ix->n_ads, d,
                         eb, 128));
    w.tmap_ready = true;
    w.tmap_for = ix->emb_q.p;
  }
  BatchArgs &a = *out;
  memset(&a, 0, sizeof(a));
  memcpy(&a.ta, w.tmap_bytes, sizeof(CUtensorMap));
  EBR_TRY(make_tmap_2d(&a.tu, w.users_bf16.p, Bp, d, eb, Bp / 2));
  a.tile_row = pl.tile_row;
  a.kb_n = pl.kb_n;
  a.ad_scale = f8 ? (const float *)ix->emb_scale.p : nullptr;
  a.user_scale = f8 ? (const float *)w.users_scale.p : nullptr;
  for (int g = 0; g < kGroups; g++) {
    a.wkey[g] = ix->wkey[g];
    a.wvals[g] = ix->wvals[g];
    a.win_ptr[g] = ix->win_ptr[g];
  }
  a.ad_nkeys = (const uint16_t *)ix->ad_nkeys.p;
  a.wT = (const float *)w.wT.p;
  a.filters = (const uint64_t *)w.filters.p;
  a.has_filter = has_filter;
  a.n_ads = ix->n_ads;
  a.n_win = ix->n_win;
  a.B = B;
  a.B_dev = B_dev;
  a.Bq = Bp;
  a.d = d;
  a.m = pl.m;
  a.cap_u = pl.cap_u;
  a.list_cap = pl.list_cap;
  a.zero_row = ix->n_keys * (Bp / 2);  // in 8-byte pair units
  a.words = (ix->n_ads + 63) / 64;
  a.sa = pl.sa;
  a.lb = pl.lb;
  a.tb = pl.tb;
  a.cand = (CandEntry *)w.cand.p;
  a.cand_n = (uint32_t *)w.cand_n.p;
  a.cand_thr = (unsigned long long *)w.cand_thr.p;
  a.ctrl = ctrl;
  return EBR_OK;
}

// Stages the batch's requests into w, launches expansion, the window scan and
// the merge on st, and queues the copies of the per-user status and the
// control block to w's pinned mirror.  Nothing here waits for the device.
int batch_launch(ebr_index *ix, const ebr_cross *cross, const ebr_query *q, uint32_t B,
                 uint32_t *d_ids, float *d_scores, uint32_t kmax, int io, BatchWs &w,
                 cudaStream_t st) {
  const uint32_t d = ix->d, fu = cross->f_u, words = (ix->n_ads + 63) / 64;
  uint32_t kscan_max = 1;
  for (uint32_t b = 0; b < B; b++)
    kscan_max = std::max(kscan_max, std::min<uint32_t>(q[b].k * ix->rescore_mult, ix->n_ads));
  std::vector<uint32_t> nv, vbase;
  const uint64_t n_vals = user_vals_layout(q, B, fu, &nv, &vbase);
  bool multi = false;
  for (uint32_t b = 0; b < B; b++) multi |= q[b].user_ptr != nullptr;
  if (io == EBR_IO_HOST)  // offsets of host requests are checked here, before anything is queued
    for (uint32_t b = 0; b < B; b++) {
      const uint32_t *p = q[b].user_ptr;
      if (!p) continue;
      for (uint32_t i = 0; i <= fu; i++)
        if ((i == 0 && p[0] != 0) || (i > 0 && p[i] < p[i - 1]) || (i == fu && p[i] != nv[b])) {
          set_error("ebr_score_topk: request %u: user_ptr must start at 0, not decrease and end "
                    "at n_user_vals",
                    b);
          return EBR_EDATA;
        }
    }
  if (n_vals >= (1ull << 32)) {
    set_error("batched scan: %llu user values in one batch", (unsigned long long)n_vals);
    return EBR_EINVAL;
  }
  // profiling events (ebr_profile_enable): before staging, before the scan,
  // after the scan, after the merge
  std::array<cudaEvent_t, 5> ev{};
  const bool prof = ix->prof;
  if (prof) {
    if (!ix->prof_pool.empty()) {
      ev = ix->prof_pool.back();
      ix->prof_pool.pop_back();
    } else {
      for (auto &e : ev) EBR_CUDA_TRY(cudaEventCreate(&e));
    }
    EBR_CUDA_TRY(cudaEventRecord(ev[0], st));
  }
  EBR_TRY(batch_ws_reserve(ix, cross, B, kscan_max, n_vals, w));
  BatchSizes z;
  batch_sizes(ix, cross, B, kscan_max, n_vals, &z);
  const int grid = z.grid;
  const BatchPlan pl = z.pl;
  const uint32_t Bp = pl.Bq;
  // pinned host mirror: [kscan B][kout B][has_filter B] in, then [status B]
  // out, then the request table
  uint32_t *h_in = reinterpret_cast<uint32_t *>(w.host);
  for (uint32_t b = 0; b < B; b++) {
    h_in[b] = std::min<uint32_t>(q[b].k * ix->rescore_mult, ix->n_ads);
    h_in[B + b] = q[b].k;
    h_in[2 * B + b] = q[b].filter ? 1u : 0u;
  }
  uint32_t *kk = (uint32_t *)w.small.p;
  uint32_t *has_filter = kk + 2 * B;
  uint32_t *status = (uint32_t *)((char *)w.small.p + small_status_off(B));
  Ctrl *ctrl = (Ctrl *)w.ctrl.p;
  EBR_CUDA_TRY(cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), st));
  EBR_CUDA_TRY(cudaMemcpyAsync(kk, h_in, (size_t)3 * B * 4, cudaMemcpyHostToDevice, st));
  EBR_CUDA_TRY(cudaMemsetAsync(status, 0, B * 4, st));
  // request inputs: device-resident requests are gathered by one kernel
  // through a table of their pointers; host requests are packed into the
  // pinned mirror and copied in two transfers (filters one per request)
  // user vectors in pair order (user_row); rows of absent users stay zero
  if (Bp > B) EBR_CUDA_TRY(cudaMemsetAsync(w.users_f32.p, 0, (size_t)Bp * d * 4, st));
  bool any_filter = false;
  for (uint32_t b = 0; b < B; b++) any_filter |= q[b].filter != nullptr;
  uint32_t *d_uptr = multi ? (uint32_t *)w.user_ptr.p : nullptr;
  uint32_t *d_base = multi ? d_uptr + (size_t)B * (fu + 1) : nullptr;
  if (io == EBR_IO_HOST) {
    // [user vectors Bq x d, pair order][offsets B x (f_u + 1)][base B][values]
    float *hu = reinterpret_cast<float *>((char *)w.host + host_table_off(B));
    uint32_t *hp = reinterpret_cast<uint32_t *>(hu + (size_t)Bp * d);
    uint32_t *hv = hp + (size_t)B * (fu + 2);
    if (Bp > B) memset(hu, 0, (size_t)Bp * d * 4);
    for (uint32_t b = 0; b < B; b++) {
      memcpy(hu + (size_t)user_row(b, Bp / 2) * d, q[b].h_u, (size_t)d * 4);
      memcpy(hv + vbase[b], q[b].user_vals, (size_t)nv[b] * 4);
      if (!multi) continue;
      uint32_t *up = hp + (size_t)b * (fu + 1);
      for (uint32_t i = 0; i <= fu; i++) up[i] = q[b].user_ptr ? q[b].user_ptr[i] : i;
      hp[(size_t)B * (fu + 1) + b] = vbase[b];
    }
    EBR_CUDA_TRY(cudaMemcpyAsync(w.users_f32.p, hu, (size_t)Bp * d * 4, cudaMemcpyHostToDevice, st));
    if (multi)
      EBR_CUDA_TRY(cudaMemcpyAsync(d_uptr, hp, (size_t)B * (fu + 2) * 4, cudaMemcpyHostToDevice, st));
    EBR_CUDA_TRY(cudaMemcpyAsync(w.user_vals.p, hv, n_vals * 4, cudaMemcpyHostToDevice, st));
    for (uint32_t b = 0; b < B; b++)
      if (q[b].filter)
        EBR_TRY(stage((uint64_t *)w.filters.p + (size_t)b * words, q[b].filter, words * 8, io, st));
  } else {
    ReqSrc *tab = reinterpret_cast<ReqSrc *>((char *)w.host + host_table_off(B));
    for (uint32_t b = 0; b < B; b++)
      tab[b] = ReqSrc{q[b].h_u, q[b].user_vals, q[b].filter, q[b].user_ptr, nv[b], vbase[b]};
    EBR_CUDA_TRY(cudaMemcpyAsync(w.req.p, tab, (size_t)B * sizeof(ReqSrc), cudaMemcpyHostToDevice,
                                 st));
    const uint32_t ys = any_filter ? (words + kStageWords - 1) / kStageWords : 1u;
    k_stage_requests<<<dim3(B, ys), 256, 0, st>>>((const ReqSrc *)w.req.p, d, fu, words, Bp / 2,
                                                  (float *)w.users_f32.p,
                                                  (uint32_t *)w.user_vals.p, d_uptr, d_base,
                                                  (uint64_t *)w.filters.p, &ctrl->flags, nullptr);
    EBR_CUDA_TRY(cudaGetLastError());
    ix->launches += 1;
  }
  const bool f8 = ix->dtype == EBR_FP8E4M3;
  if (f8)  // users as FP8 with a scale per user (kind::f8f6f4 takes both operands in FP8)
    EBR_TRY(launch_quantize_rows_fp8((const float *)w.users_f32.p, Bp, d, (uint8_t *)w.users_bf16.p,
                                     (float *)w.users_scale.p, st));
  else
    EBR_TRY(launch_quantize((const float *)w.users_f32.p, (uint64_t)Bp * d, EBR_BF16,
                            w.users_bf16.p, st));
  EBR_TRY(expand_transposed(cross, (const uint32_t *)w.user_vals.p, d_uptr, d_base, B, Bp,
                            (float *)w.wT.p, &ctrl->flags, st));
  EBR_CUDA_TRY(cudaMemsetAsync((float *)w.wT.p + (size_t)ix->n_keys * Bp, 0, (size_t)Bp * 4, st));
  BatchArgs a;
  EBR_TRY(fill_batch_args(ix, B, pl, w, has_filter, ctrl, nullptr, &a));
  auto kern = f8 ? k_batch_window<true> : k_batch_window<false>;
  EBR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)pl.smem));
  if (prof) EBR_CUDA_TRY(cudaEventRecord(ev[1], st));
  kern<<<grid, kBatchThreads, pl.smem, st>>>(a);
  EBR_CUDA_TRY(cudaGetLastError());
  if (prof) EBR_CUDA_TRY(cudaEventRecord(ev[2], st));
  EBR_CUDA_TRY(cudaFuncSetAttribute(k_batch_merge, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    8192 * 8));
  k_batch_merge<<<B, kMergeThreads, 8192 * 8, st>>>(
      (const CandEntry *)w.cand.p, (const uint32_t *)w.cand_n.p,
      (const unsigned long long *)w.cand_thr.p, (uint32_t)grid, B, pl.cap_u, kk, kk + B, kmax,
      (const float *)ix->emb_f32.p, d, (const float *)w.users_f32.p, Bp / 2,
      (uint64_t *)w.scratch.p, d_ids, d_scores, status, nullptr, nullptr, 0, 0);
  EBR_CUDA_TRY(cudaGetLastError());
  if (prof) {
    EBR_CUDA_TRY(cudaEventRecord(ev[3], st));
    ix->bprof_pending.push_back(ev);
  }
  ix->launches += 4;
  ix->batched += B;
  // status and flags back to the pinned mirror
  uint32_t *h_status = h_in + 3 * B;
  EBR_CUDA_TRY(cudaMemcpyAsync(h_status, status, B * 4, cudaMemcpyDeviceToHost, st));
  return EBR_OK;
}

// Waits for a batch started by batch_launch, checks the device flags and
// recomputes on the single-request scan every user whose candidate buffers
// could not prove exactness (outputs rewritten in place on st).
int batch_finish(ebr_index *ix, const ebr_cross *cross, const ebr_query *q, uint32_t B,
                 uint32_t *d_ids, float *d_scores, uint32_t kmax, BatchWs &w, cudaStream_t st) {
  const uint32_t d = ix->d, fu = cross->f_u, words = (ix->n_ads + 63) / 64;
  Ctrl hc;
  EBR_CUDA_TRY(cudaMemcpyAsync(&hc, w.ctrl.p, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
  EBR_CUDA_TRY(cudaStreamSynchronize(st));
  EBR_TRY(check_device_flags(hc.flags, "ebr_score_topk (batched)"));
  const uint32_t *h_status = reinterpret_cast<const uint32_t *>(w.host) + 3 * B;
  std::vector<uint32_t> nv, vbase;
  user_vals_layout(q, B, fu, &nv, &vbase);
  for (uint32_t b = 0; b < B; b++) {
    if (!h_status[b]) continue;
    ebr_query dq = q[b];
    dq.h_u = (const float *)w.users_f32.p + (size_t)user_row(b, users_pow2(B) / 2) * d;
    dq.user_vals = (const uint32_t *)w.user_vals.p + vbase[b];
    // the checked offsets staged for the batch (device memory)
    dq.user_ptr = q[b].user_ptr ? (const uint32_t *)w.user_ptr.p + (size_t)b * (fu + 1) : nullptr;
    dq.n_user_vals = nv[b];
    dq.filter = q[b].filter ? (const uint64_t *)w.filters.p + (size_t)b * words : nullptr;
    EBR_TRY(ws_prepare_one(ix, ix->n_keys, 8192));
    EBR_TRY(query_one(ix, cross, dq, d_ids + (size_t)b * kmax, d_scores + (size_t)b * kmax, kmax,
                      st));
    ix->fallbacks += 1;
    EBR_CUDA_TRY(cudaMemcpyAsync(&hc, ix->ws.ctrl.p, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    EBR_CUDA_TRY(cudaStreamSynchronize(st));
    EBR_TRY(check_device_flags(hc.flags, "ebr_score_topk (single-request recompute)"));
  }
  return EBR_OK;
}

void batch_ws_free(BatchWs &w) {
  for (DevBuf *b : {&w.users_f32, &w.users_bf16, &w.users_scale, &w.user_vals, &w.user_ptr, &w.wT,
                    &w.filters, &w.small, &w.cand, &w.cand_n, &w.cand_thr, &w.scratch, &w.res,
                    &w.ctrl, &w.req})
    dev_free(*b);
  if (w.host) cudaFreeHost(w.host);
  w.host = nullptr;
  w.host_bytes = 0;
  w.tmap_ready = false;
}

int query_batch(ebr_index *ix, const ebr_cross *cross, const ebr_query *q, uint32_t B,
                uint32_t *out_ids, float *out_scores, uint32_t kmax, int io, cudaStream_t st) {
  BatchWs &w = ix->bws;
  uint32_t *d_ids = out_ids;
  float *d_scores = out_scores;
  if (io == EBR_IO_HOST) {
    EBR_TRY(dev_reserve(w.res, (size_t)B * kmax * 8 + 256));
    d_ids = (uint32_t *)w.res.p;
    d_scores = (float *)((char *)w.res.p + (((size_t)B * kmax * 4 + 255) / 256 * 256));
  }
  EBR_TRY(batch_launch(ix, cross, q, B, d_ids, d_scores, kmax, io, w, st));
  EBR_TRY(batch_finish(ix, cross, q, B, d_ids, d_scores, kmax, w, st));
  if (io == EBR_IO_HOST) {
    EBR_CUDA_TRY(cudaMemcpyAsync(out_ids, d_ids, (size_t)B * kmax * 4, cudaMemcpyDeviceToHost, st));
    EBR_CUDA_TRY(
        cudaMemcpyAsync(out_scores, d_scores, (size_t)B * kmax * 4, cudaMemcpyDeviceToHost, st));
    EBR_CUDA_TRY(cudaStreamSynchronize(st));
  }
  return EBR_OK;
}

// =====================================================================
// Device-resident serving loop
// =====================================================================
// Wave descriptor (one ring slot, written by the host, copied to `cur` by
// the fetch kernel): [B, pad x3][kscan Bmax][kout Bmax][has_filter Bmax]
// [ReqSrc Bmax, 16-byte aligned].
static size_t desc_src_off(uint32_t Bmax) { return (16 + (size_t)12 * Bmax + 15) / 16 * 16; }
static size_t desc_bytes_for(uint32_t Bmax) {
  return (desc_src_off(Bmax) + (size_t)Bmax * sizeof(ReqSrc) + 15) / 16 * 16;
}

struct LoopArgs {
  LoopShared *sh;              // mapped host words
  const uint8_t *desc;         // mapped [R][desc_bytes]
  uint32_t *flags_out;         // mapped [R]
  uint32_t *status_out;        // mapped [R][Bmax]
  uint8_t *cur;                // device copy of the current descriptor
  uint32_t *slot;
  unsigned long long *seq, *idle_ns;
  Ctrl *ctrl;
  uint32_t *status;            // [R][Bmax]
  uint32_t R, Bmax, desc_bytes;
  unsigned long long poll_ns, idle_exit_ns;
  cudaGraphConditionalHandle handle;  // the WHILE node's
  cudaGraphConditionalHandle sw;      // the SWITCH node's: which user-table width runs
  uint32_t nsw, bq[3];                // widths (users) of the switch's cases, ascending
};

__device__ __forceinline__ unsigned long long ld_acquire_sys(const volatile unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_sys(volatile unsigned long long *p,
                                               unsigned long long v) {
  asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// First node of the loop body.  Thread 0 waits, for at most poll_ns, for a
// wave the host posted whose result slot the host has freed, or for stop.
// A wave: its descriptor is copied into `cur`, its control block and status
// zeroed, and the SWITCH node that follows is told which user-table width
// (the narrowest that holds the wave's users) to run.  No wave: cur.B = 0
// (every later node of this iteration returns at once), and after
// idle_exit_ns without a wave, or on stop, the loop's condition is cleared
// so that this iteration is the last.
__global__ void __launch_bounds__(256) k_loop_fetch(LoopArgs a) {
  __shared__ uint32_t s_state, s_slot;
  if (threadIdx.x == 0) {
    const unsigned long long seq = *a.seq;
    const uint64_t t0 = global_timer_ns();
    uint32_t st = 0;  // 0: no wave, 1: a wave, 2: leave the loop
    for (;;) {
      if (a.sh->stop) {
        st = 2;
        break;
      }
      const unsigned long long posted = ld_acquire_sys(&a.sh->posted);
      if (posted > seq && seq < a.sh->freed + a.R) {
        st = 1;
        break;
      }
      if (global_timer_ns() - t0 >= a.poll_ns) break;
      __nanosleep(1000);
    }
    if (st == 0) {
      *a.idle_ns += global_timer_ns() - t0;
      if (*a.idle_ns >= a.idle_exit_ns) st = 2;
    } else if (st == 1) {
      *a.idle_ns = 0;
    }
    if (st == 2) cudaGraphSetConditional(a.handle, 0u);
    if (st == 1) {  // the narrowest user table that holds the wave
      const uint32_t B = reinterpret_cast<const volatile uint32_t *>(
          a.desc + (size_t)(seq % a.R) * a.desc_bytes)[0];
      uint32_t c = 0;
      while (c + 1 < a.nsw && B > a.bq[c]) c++;
      cudaGraphSetConditional(a.sw, c);
    }
    s_state = st;
    s_slot = (uint32_t)(seq % a.R);
    *a.slot = s_slot;
  }
  __syncthreads();
  if (s_state != 1) {
    if (threadIdx.x == 0) *reinterpret_cast<uint32_t *>(a.cur) = 0u;
    return;
  }
  const volatile uint32_t *src =
      reinterpret_cast<const volatile uint32_t *>(a.desc + (size_t)s_slot * a.desc_bytes);
  uint32_t *dst = reinterpret_cast<uint32_t *>(a.cur);
  for (uint32_t i = threadIdx.x; i < a.desc_bytes / 4; i += blockDim.x) dst[i] = src[i];
  for (uint32_t i = threadIdx.x; i < sizeof(Ctrl) / 4; i += blockDim.x)
    reinterpret_cast<uint32_t *>(a.ctrl)[i] = 0u;
  for (uint32_t i = threadIdx.x; i < a.Bmax; i += blockDim.x) a.status[s_slot * a.Bmax + i] = 0u;
}

// Last node of the loop body: a wave's flags and per-user status go to the
// mapped result words, then (system-scope release) done = waves finished.
__global__ void k_loop_publish(LoopArgs a) {
  const uint32_t B = *reinterpret_cast<const uint32_t *>(a.cur);
  if (B == 0) return;
  const uint32_t slot = *a.slot;
  for (uint32_t b = threadIdx.x; b < B; b += blockDim.x)
    a.status_out[slot * a.Bmax + b] = a.status[slot * a.Bmax + b];
  __syncthreads();
  if (threadIdx.x == 0) {
    a.flags_out[slot] = a.ctrl->flags;
    __threadfence_system();
    const unsigned long long seq = *a.seq + 1;
    *a.seq = seq;
    st_release_sys(&a.sh->done, seq);
  }
}

static void loop_dev_sizes(uint32_t R, uint32_t Bmax, uint32_t kmax, size_t *cur_b, size_t *st_b,
                           size_t *out_b, size_t *ctl_b) {
  *cur_b = (desc_bytes_for(Bmax) + 255) / 256 * 256;
  *st_b = ((size_t)R * Bmax * 4 + 255) / 256 * 256;
  *out_b = ((size_t)R * Bmax * kmax * 4 + 255) / 256 * 256;
  *ctl_b = (256 + sizeof(Ctrl) + 255) / 256 * 256;
}

size_t loop_dev_bytes(uint32_t Bmax, uint32_t kmax) {
  size_t cur_b, st_b, out_b, ctl_b;
  loop_dev_sizes(LoopBufs{}.R, Bmax, kmax, &cur_b, &st_b, &out_b, &ctl_b);
  return cur_b + st_b + 2 * out_b + ctl_b;
}

int loop_alloc(LoopBufs &L, uint32_t Bmax, uint32_t kmax) {
  L.Bmax = Bmax;
  L.kmax = kmax;
  L.desc_bytes = (uint32_t)desc_bytes_for(Bmax);
  const size_t sh_b = 256, desc_b = (size_t)L.R * L.desc_bytes, fl_b = (size_t)L.R * 4;
  const size_t host_b = sh_b + desc_b + fl_b + (size_t)L.R * Bmax * 4;
  if (cudaHostAlloc(&L.host, host_b, cudaHostAllocMapped) != cudaSuccess) {
    cudaGetLastError();
    L.host = nullptr;
    set_error("serving loop: mapped host allocation of %zu bytes failed", host_b);
    return EBR_ENOMEM;
  }
  memset(L.host, 0, host_b);
  void *dp = nullptr;
  EBR_CUDA_TRY(cudaHostGetDevicePointer(&dp, L.host, 0));
  if (dp != L.host) {  // every pointer below is used on both sides
    set_error("serving loop: mapped host memory has a different device address");
    return EBR_EINVAL;
  }
  uint8_t *h = (uint8_t *)L.host;
  L.sh = (LoopShared *)h;
  L.desc = h + sh_b;
  L.flags_out = (uint32_t *)(h + sh_b + desc_b);
  L.status_out = (uint32_t *)(h + sh_b + desc_b + fl_b);
  size_t cur_b, st_b, out_b, ctl_b;
  loop_dev_sizes(L.R, Bmax, kmax, &cur_b, &st_b, &out_b, &ctl_b);
  EBR_TRY(dev_alloc(L.dev, cur_b + st_b + 2 * out_b + ctl_b));
  uint8_t *d = (uint8_t *)L.dev.p;
  L.cur = d;
  L.status = (uint32_t *)(d + cur_b);
  L.out_ids = (uint32_t *)(d + cur_b + st_b);
  L.out_scores = (float *)(d + cur_b + st_b + out_b);
  uint8_t *c = d + cur_b + st_b + 2 * out_b;
  L.slot = (uint32_t *)c;
  L.seq = (unsigned long long *)(c + 8);
  L.idle_ns = (unsigned long long *)(c + 16);
  L.ctrl = (Ctrl *)(c + 256);
  EBR_CUDA_TRY(cudaMemset(L.dev.p, 0, L.dev.bytes));
  return EBR_OK;
}

void loop_free(LoopBufs &L) {
  if (L.exec) cudaGraphExecDestroy(L.exec);
  L.exec = nullptr;
  dev_free(L.dev);
  if (L.host) cudaFreeHost(L.host);
  L.host = nullptr;
}

int loop_fill(LoopBufs &L, uint64_t wave, const ebr_index *ix, const ebr_cross *cross,
              const ebr_query *q, uint32_t B) {
  if (B == 0 || B > L.Bmax) {
    set_error("serving loop: a wave of %u users (at most %u)", B, L.Bmax);
    return EBR_EINVAL;
  }
  uint8_t *p = L.desc + (size_t)(wave % L.R) * L.desc_bytes;
  uint32_t *w32 = (uint32_t *)p;
  w32[0] = B;
  uint32_t *ks = (uint32_t *)(p + 16), *ko = ks + L.Bmax, *hf = ko + L.Bmax;
  ReqSrc *src = (ReqSrc *)(p + desc_src_off(L.Bmax));
  uint32_t base = 0;
  for (uint32_t b = 0; b < B; b++) {
    ks[b] = std::min<uint32_t>(q[b].k * ix->rescore_mult, ix->n_ads);
    ko[b] = q[b].k;
    hf[b] = q[b].filter ? 1u : 0u;
    const uint32_t n = q[b].user_ptr ? q[b].n_user_vals : cross->f_u;
    src[b] = ReqSrc{q[b].h_u, q[b].user_vals, q[b].filter, q[b].user_ptr, n, base};
    base += n;
  }
  return EBR_OK;
}

// Builds the loop graph for index ix: a WHILE node whose body is
//   fetch -> SWITCH { one case per user-table width 64, 128, 256 (up to the
//   server's batch): staging, quantiser, expansion, window scan, merge }
//   -> publish,
// so a wave of a few users runs on the narrowest table that holds it.  The
// batch plan (candidate buffers, shared memory) is the same for every width.
int loop_build(ebr_index *ix, const ebr_cross *cross, uint32_t max_user_vals, BatchWs &w,
               LoopBufs &L, cudaStream_t st) {
  if (L.exec) {
    cudaGraphExecDestroy(L.exec);
    L.exec = nullptr;
  }
  const uint32_t Bmax = L.Bmax, d = ix->d, fu = cross->f_u, words = (ix->n_ads + 63) / 64;
  const uint32_t kscan_max = std::min<uint32_t>(L.kmax * ix->rescore_mult, ix->n_ads);
  EBR_TRY(batch_ws_reserve(ix, cross, Bmax, kscan_max, (uint64_t)Bmax * max_user_vals, w));
  BatchSizes z;
  batch_sizes(ix, cross, Bmax, kscan_max, (uint64_t)Bmax * max_user_vals, &z);
  const BatchPlan pl = z.pl;
  const bool f8 = ix->dtype == EBR_FP8E4M3;
  uint8_t *cur = L.cur;
  const uint32_t *B_dev = (const uint32_t *)cur;
  const uint32_t *ks = (const uint32_t *)(cur + 16), *ko = ks + Bmax, *hf = ko + Bmax;
  const ReqSrc *srcs = (const ReqSrc *)(cur + desc_src_off(Bmax));
  uint32_t *d_uptr = (uint32_t *)w.user_ptr.p;
  uint32_t *d_base = d_uptr + (size_t)Bmax * (fu + 1);
  auto kern = f8 ? k_batch_window<true> : k_batch_window<false>;
  EBR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)pl.smem));
  EBR_CUDA_TRY(cudaFuncSetAttribute(k_batch_merge, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    8192 * 8));
  LoopArgs la;
  memset(&la, 0, sizeof(la));
  la.nsw = 0;
  for (uint32_t q = 64; q <= pl.Bq; q <<= 1) la.bq[la.nsw++] = q;
  cudaGraph_t g = nullptr;
  EBR_CUDA_TRY(cudaGraphCreate(&g, 0));
  int rc = EBR_OK;
  const char *what = "conditional graph nodes";
  cudaError_t e = cudaGraphConditionalHandleCreate(&la.handle, g, 1u, cudaGraphCondAssignDefault);
  cudaGraphNodeParams wp = {}, sp = {};
  cudaGraphNode_t wnode, fnode, snode;
  if (e == cudaSuccess) {
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = la.handle;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    e = cudaGraphAddNode(&wnode, g, nullptr, nullptr, 0, &wp);
  }
  cudaGraph_t body = e == cudaSuccess ? wp.conditional.phGraph_out[0] : nullptr;
  if (e == cudaSuccess)
    e = cudaGraphConditionalHandleCreate(&la.sw, body, 0u, cudaGraphCondAssignDefault);
  la.sh = L.sh;
  la.desc = L.desc;
  la.flags_out = L.flags_out;
  la.status_out = L.status_out;
  la.cur = cur;
  la.slot = L.slot;
  la.seq = L.seq;
  la.idle_ns = L.idle_ns;
  la.ctrl = L.ctrl;
  la.status = L.status;
  la.R = L.R;
  la.Bmax = Bmax;
  la.desc_bytes = L.desc_bytes;
  la.poll_ns = L.poll_ns;
  la.idle_exit_ns = L.idle_exit_ns;
  // fetch
  if (e == cudaSuccess) {
    what = "capture of the fetch node";
    e = cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      k_loop_fetch<<<1, 256, 0, st>>>(la);
      cudaGraph_t cap = nullptr;
      e = cudaStreamEndCapture(st, &cap);
    }
    size_t nn = 1;
    if (e == cudaSuccess) e = cudaGraphGetNodes(body, &fnode, &nn);
    if (e == cudaSuccess && nn != 1) e = cudaErrorInvalidValue;
  }
  // the switch and its cases
  if (e == cudaSuccess) {
    what = "switch node";
    sp.type = cudaGraphNodeTypeConditional;
    sp.conditional.handle = la.sw;
    sp.conditional.type = cudaGraphCondTypeSwitch;
    sp.conditional.size = la.nsw;
    e = cudaGraphAddNode(&snode, body, &fnode, nullptr, 1, &sp);
  }
  for (uint32_t c = 0; e == cudaSuccess && rc == EBR_OK && c < la.nsw; c++) {
    what = "capture of a wave";
    BatchPlan pc = pl;
    pc.Bq = la.bq[c];
    const uint32_t Bp = pc.Bq;
    BatchArgs ba;
    rc = fill_batch_args(ix, Bmax, pc, w, hf, L.ctrl, B_dev, &ba);
    if (rc != EBR_OK) break;
    e = cudaStreamBeginCaptureToGraph(st, sp.conditional.phGraph_out[c], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) break;
    const uint32_t ys = (words + kStageWords - 1) / kStageWords;
    k_stage_requests<<<dim3(Bp, ys), 256, 0, st>>>(srcs, d, fu, words, Bp / 2,
                                                   (float *)w.users_f32.p,
                                                   (uint32_t *)w.user_vals.p, d_uptr, d_base,
                                                   (uint64_t *)w.filters.p, &L.ctrl->flags, B_dev);
    if (f8)
      rc = launch_quantize_rows_fp8((const float *)w.users_f32.p, Bp, d,
                                    (uint8_t *)w.users_bf16.p, (float *)w.users_scale.p, st);
    else
      rc = launch_quantize((const float *)w.users_f32.p, (uint64_t)Bp * d, EBR_BF16,
                           w.users_bf16.p, st);
    if (rc == EBR_OK)
      rc = expand_transposed(cross, (const uint32_t *)w.user_vals.p, d_uptr, d_base,
                             std::min(Bmax, Bp), Bp, (float *)w.wT.p, &L.ctrl->flags, st, B_dev);
    if (rc == EBR_OK) {
      cudaMemsetAsync((float *)w.wT.p + (size_t)ix->n_keys * Bp, 0, (size_t)Bp * 4, st);
      kern<<<z.grid, kBatchThreads, pl.smem, st>>>(ba);
      k_batch_merge<<<std::min(Bmax, Bp), kMergeThreads, 8192 * 8, st>>>(
          (const CandEntry *)w.cand.p, (const uint32_t *)w.cand_n.p,
          (const unsigned long long *)w.cand_thr.p, (uint32_t)z.grid, Bmax, pl.cap_u, ks, ko,
          L.kmax, (const float *)ix->emb_f32.p, d, (const float *)w.users_f32.p, Bp / 2,
          (uint64_t *)w.scratch.p, L.out_ids, L.out_scores, L.status, B_dev, L.slot,
          (uint64_t)Bmax * L.kmax, Bmax);
    }
    cudaGraph_t cap = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(st, &cap);
    if (e == cudaSuccess) e = e2;
  }
  // publish, after the switch
  if (e == cudaSuccess && rc == EBR_OK) {
    what = "capture of the publish node";
    e = cudaStreamBeginCaptureToGraph(st, body, &snode, nullptr, 1, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      k_loop_publish<<<1, 256, 0, st>>>(la);
      cudaGraph_t cap = nullptr;
      e = cudaStreamEndCapture(st, &cap);
    }
  }
  if (e == cudaSuccess && rc == EBR_OK) {
    what = "graph instantiation";
    e = cudaGraphInstantiate(&L.exec, g, 0);
  }
  cudaGraphDestroy(g);
  if (rc != EBR_OK) return rc;
  if (e != cudaSuccess) {
    L.exec = nullptr;
    cudaGetLastError();
    set_error("serving loop: %s: %s", what, cudaGetErrorString(e));
    return EBR_ECUDA;
  }
  return EBR_OK;
}

}  // namespace ebr
