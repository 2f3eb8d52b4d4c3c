// Device-wide primitives of the index builder and of Algorithm 2's long
// lists: an exclusive / inclusive scan over any type with an associative
// add, a stable least-significant-digit radix sort of 64-bit (or 8-bit)
// keys with optional 32-bit values, and the unique of a sorted array.
//
// The scan runs in three launches (tile sums; one CTA scans the tile sums;
// each tile scans itself from its offset), so no CTA ever waits on another.
// The radix sort takes 8-bit digits from the lowest bit up; each pass counts
// the digits of every tile of 2048 keys, scans the (digit, tile) counts, and
// scatters the tile's keys to their places.  The scatter is stable: a tile's
// keys are ranked in index order, round by round (256 keys per round, one
// per thread), within a warp by __match_any_sync on the digit and across
// warps by per-warp digit counts, so equal digits keep their order and the
// passes compose into a sort.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <utility>

#include "ebr_internal.cuh"

namespace ebr {
namespace prims {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;  // per thread: tiles of 4096
constexpr uint32_t kScanTile = kScanThreads * kScanItems;

// Block-wide exclusive scan of one value per thread (returns the thread's
// exclusive prefix, *total the block's sum).  s_warp: 32 entries of T.
template <typename T, typename Op>
__device__ __forceinline__ T block_exclusive(T v, Op op, T zero, T *s_warp, T *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y;
    // shuffle any trivially copyable T in 32-bit pieces
    static_assert(sizeof(T) % 4 == 0, "scan type size");
    uint32_t *pi = reinterpret_cast<uint32_t *>(&incl), *py = reinterpret_cast<uint32_t *>(&y);
#pragma unroll
    for (int k = 0; k < (int)(sizeof(T) / 4); k++) py[k] = __shfl_up_sync(0xffffffffu, pi[k], o);
    if (lane >= o) incl = op(y, incl);
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    T w = lane < nw ? s_warp[lane] : zero;
    T wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y;
      uint32_t *pi = reinterpret_cast<uint32_t *>(&wi), *py = reinterpret_cast<uint32_t *>(&y);
#pragma unroll
      for (int k = 0; k < (int)(sizeof(T) / 4); k++)
        py[k] = __shfl_up_sync(0xffffffffu, pi[k], o);
      if (lane >= o) wi = op(y, wi);
    }
    if (lane < nw) s_warp[lane] = wi;  // inclusive prefix of the warp sums
  }
  __syncthreads();
  const T before = warp > 0 ? s_warp[warp - 1] : zero;
  *total = s_warp[(blockDim.x >> 5) - 1];
  // exclusive = before + (incl - v): recompute as before + exclusive-in-warp
  T ex_in = zero;
  {
    T y;
    uint32_t *pi = reinterpret_cast<uint32_t *>(&incl), *py = reinterpret_cast<uint32_t *>(&y);
#pragma unroll
    for (int k = 0; k < (int)(sizeof(T) / 4); k++) py[k] = __shfl_up_sync(0xffffffffu, pi[k], 1);
    if (lane > 0) ex_in = y;
  }
  __syncthreads();  // s_warp may be reused by the caller
  return op(before, ex_in);
}

// Phase 1: the sum of each tile.
template <typename T, typename Op>
__global__ void __launch_bounds__(kScanThreads) k_scan_tile_sums(const T *__restrict__ in,
                                                                  uint64_t n, T *__restrict__ sums,
                                                                  Op op, T zero) {
  __shared__ T s_warp[32];
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
  T acc = zero;
#pragma unroll 4
  for (int i = 0; i < kScanItems; i++) {
    const uint64_t idx = base + (uint64_t)i * kScanThreads + threadIdx.x;
    if (idx < n) acc = op(acc, in[idx]);
  }
  T total;
  block_exclusive(acc, op, zero, s_warp, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// Phase 2: one CTA turns the tile sums into exclusive tile offsets (in
// place); *grand (if given) gets the total.
template <typename T, typename Op>
__global__ void __launch_bounds__(1024) k_scan_offsets(T *__restrict__ sums, uint32_t n_tiles,
                                                       Op op, T zero, T *__restrict__ grand) {
  __shared__ T s_warp[32];
  T carry = zero;
  for (uint32_t b0 = 0; b0 < n_tiles; b0 += 1024) {
    const uint32_t i = b0 + threadIdx.x;
    const T v = i < n_tiles ? sums[i] : zero;
    T total;
    const T ex = block_exclusive(v, op, zero, s_warp, &total);
    if (i < n_tiles) sums[i] = op(carry, ex);
    carry = op(carry, total);
  }
  if (grand && threadIdx.x == 0) *grand = carry;
}

// Phase 3: each tile scans itself from its offset (striped order: item i
// of the tile is element i * threads + thread, scanned per item row).
template <typename T, typename Op, bool INCLUSIVE>
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const T *in, uint64_t n,
                                                             const T *__restrict__ offs, T *out,
                                                             Op op, T zero) {  // in may be out
  __shared__ T s_warp[32];
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
  T carry = offs[blockIdx.x];
  for (int i = 0; i < kScanItems; i++) {
    const uint64_t idx = base + (uint64_t)i * kScanThreads + threadIdx.x;
    const T v = idx < n ? in[idx] : zero;
    T total;
    const T ex = block_exclusive(v, op, zero, s_warp, &total);
    if (idx < n) out[idx] = INCLUSIVE ? op(op(carry, ex), v) : op(carry, ex);
    carry = op(carry, total);
  }
}

struct AddU32 {
  __host__ __device__ __forceinline__ uint32_t operator()(uint32_t a, uint32_t b) const {
    return a + b;
  }
};

// Scratch (in elements of T) the scan of n elements needs: one per tile + 1.
inline size_t scan_scratch(uint64_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

// out = scan of in (n elements; in and out may be the same array).  tmp:
// scan_scratch(n) elements of T; *grand (device, optional): the total.
template <typename T, typename Op, bool INCLUSIVE>
int scan(const T *in, T *out, uint64_t n, Op op, T zero, T *tmp, T *grand, cudaStream_t st) {
  if (n == 0) {
    if (grand) EBR_CUDA_TRY(cudaMemsetAsync(grand, 0, sizeof(T), st));
    return EBR_OK;
  }
  const uint64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles > 0x7FFFFFFFull) {
    set_error("scan: %llu elements are too many", (unsigned long long)n);
    return EBR_EINVAL;
  }
  k_scan_tile_sums<T, Op><<<(unsigned)tiles, kScanThreads, 0, st>>>(in, n, tmp, op, zero);
  EBR_CUDA_TRY(cudaGetLastError());
  k_scan_offsets<T, Op><<<1, 1024, 0, st>>>(tmp, (uint32_t)tiles, op, zero, grand);
  EBR_CUDA_TRY(cudaGetLastError());
  k_scan_tiles<T, Op, INCLUSIVE><<<(unsigned)tiles, kScanThreads, 0, st>>>(in, n, tmp, out, op,
                                                                           zero);
  EBR_CUDA_TRY(cudaGetLastError());
  return EBR_OK;
}

// ------------------------------------------------------------- radix sort
constexpr int kSortThreads = 256;
constexpr int kSortRounds = 8;  // keys per thread per tile
constexpr uint32_t kSortTile = kSortThreads * kSortRounds;
constexpr int kSortWarps = kSortThreads / 32;

template <typename K>
__device__ __forceinline__ uint32_t digit_of(K k, int shift) {
  return (uint32_t)((uint64_t)k >> shift) & 255u;
}

// Digit counts of each tile, stored digit-major: counts[d * tiles + tile].
template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const K *__restrict__ keys,
                                                            uint64_t n, int shift, uint32_t tiles,
                                                            uint32_t *__restrict__ counts) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const uint64_t base = (uint64_t)blockIdx.x * kSortTile;
#pragma unroll
  for (int r = 0; r < kSortRounds; r++) {
    const uint64_t i = base + (uint64_t)r * kSortThreads + threadIdx.x;
    if (i < n) {
      const uint32_t d = digit_of(keys[i], shift);
      const uint32_t peers = __match_any_sync(__activemask(), d);
      if ((threadIdx.x & 31) == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&h[d], __popc(peers));
    }
  }
  __syncthreads();
  counts[(uint64_t)threadIdx.x * tiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of each tile's keys (and values) to offs[d * tiles + tile]
// + (rank of the key among the tile's keys of digit d, in index order).
template <typename K, bool VALS>
__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(
    const K *__restrict__ keys, const uint32_t *__restrict__ vals, uint64_t n, int shift,
    uint32_t tiles, const uint32_t *__restrict__ offs, K *__restrict__ keys_out,
    uint32_t *__restrict__ vals_out) {
  __shared__ uint32_t run[256];                // keys of each digit placed so far in this tile
  __shared__ uint32_t wcnt[kSortWarps][256];   // this round's count of each digit per warp
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  run[threadIdx.x] = offs[(uint64_t)threadIdx.x * tiles + blockIdx.x];
  for (int w = 0; w < kSortWarps; w++) wcnt[w][threadIdx.x] = 0;
  __syncthreads();
  const uint64_t base = (uint64_t)blockIdx.x * kSortTile;
  for (int r = 0; r < kSortRounds; r++) {
    const uint64_t i = base + (uint64_t)r * kSortThreads + threadIdx.x;
    const bool v = i < n;
    K k = 0;
    uint32_t val = 0, d = 0, peers = 0, rank = 0;
    if (v) {
      k = keys[i];
      if (VALS) val = vals[i];
      d = digit_of(k, shift);
    }
    // valid keys are a prefix of the round, so every warp's active lanes
    // are its first lanes; invalid lanes take part with a digit of their own
    const uint32_t dd = v ? d : 256u + lane;
    peers = __match_any_sync(0xffffffffu, dd);
    rank = __popc(peers & ((1u << lane) - 1u));
    const bool leader = v && rank == 0;
    if (leader) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    uint32_t pos = 0;
    if (v) {
      uint32_t before = 0;
      for (int w = 0; w < warp; w++) before += wcnt[w][d];
      pos = run[d] + before + rank;
    }
    __syncthreads();  // every thread has read run[] and wcnt[]
    if (v) {
      keys_out[pos] = k;
      if (VALS) vals_out[pos] = val;
    }
    if (leader) {
      // the last warp holding digit d this round advances run[d]
      uint32_t after = 0;
      for (int w = warp + 1; w < kSortWarps; w++) after += wcnt[w][d];
      if (after == 0) {
        uint32_t total = 0;
        for (int w = 0; w < kSortWarps; w++) total += wcnt[w][d];
        run[d] += total;
      }
    }
    __syncthreads();
    if (leader) wcnt[warp][d] = 0;
    __syncthreads();
  }
}

// Scratch (bytes) a radix sort of n keys needs: the (digit, tile) counts
// and the scan's tile sums.
inline size_t sort_scratch(uint64_t n) {
  const uint64_t tiles = (n + kSortTile - 1) / kSortTile;
  const uint64_t cnt = 256 * tiles;
  return (cnt + scan_scratch(cnt)) * 4 + 256;
}

// Sorts keys[0..n) (with vals, if given) by bits [0, end_bit), ping-ponging
// with keys_alt / vals_alt; *in_alt tells where the result ended.
template <typename K>
int radix_sort(K *keys, K *keys_alt, uint32_t *vals, uint32_t *vals_alt, uint64_t n, int end_bit,
               void *scratch, bool *in_alt, cudaStream_t st) {
  *in_alt = false;
  if (n <= 1) return EBR_OK;
  const uint64_t tiles64 = (n + kSortTile - 1) / kSortTile;
  if (tiles64 > 0x7FFFFFFFull / 256) {
    set_error("radix sort: %llu keys are too many", (unsigned long long)n);
    return EBR_EINVAL;
  }
  const uint32_t tiles = (uint32_t)tiles64;
  uint32_t *counts = reinterpret_cast<uint32_t *>(scratch);
  uint32_t *stmp = counts + (size_t)256 * tiles;
  K *src = keys, *dst = keys_alt;
  uint32_t *vsrc = vals, *vdst = vals_alt;
  for (int shift = 0; shift < end_bit; shift += 8) {
    k_sort_hist<K><<<tiles, kSortThreads, 0, st>>>(src, n, shift, tiles, counts);
    EBR_CUDA_TRY(cudaGetLastError());
    EBR_TRY((scan<uint32_t, AddU32, false>(counts, counts, (uint64_t)256 * tiles, AddU32(), 0u,
                                           stmp, nullptr, st)));
    if (vals)
      k_sort_scatter<K, true><<<tiles, kSortThreads, 0, st>>>(src, vsrc, n, shift, tiles, counts,
                                                              dst, vdst);
    else
      k_sort_scatter<K, false><<<tiles, kSortThreads, 0, st>>>(src, nullptr, n, shift, tiles,
                                                               counts, dst, nullptr);
    EBR_CUDA_TRY(cudaGetLastError());
    std::swap(src, dst);
    std::swap(vsrc, vdst);
    *in_alt = !*in_alt;
  }
  return EBR_OK;
}

// ------------------------------------------------------------------ unique
static __global__ void k_unique_flags(const uint64_t *__restrict__ x, uint64_t n,
                               uint32_t *__restrict__ f) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    f[i] = (i == 0 || x[i] != x[i - 1]) ? 1u : 0u;
}
static __global__ void k_unique_emit(const uint64_t *__restrict__ x, uint64_t n,
                              const uint32_t *__restrict__ pos, uint64_t *__restrict__ out) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    if (i == 0 || x[i] != x[i - 1]) out[pos[i]] = x[i];
}

// out = the distinct values of the sorted x[0..n), in order; *d_count
// (device) their number.  flags: n uint32 scratch; tmp: scan_scratch(n).
inline int unique_sorted(const uint64_t *x, uint64_t *out, uint64_t n, uint32_t *flags,
                         uint32_t *tmp, uint32_t *d_count, cudaStream_t st) {
  if (n == 0) {
    EBR_CUDA_TRY(cudaMemsetAsync(d_count, 0, 4, st));
    return EBR_OK;
  }
  const unsigned grid = (unsigned)std::min<uint64_t>((n + 255) / 256, 65535);
  k_unique_flags<<<grid, 256, 0, st>>>(x, n, flags);
  EBR_CUDA_TRY(cudaGetLastError());
  EBR_TRY((scan<uint32_t, AddU32, false>(flags, flags, n, AddU32(), 0u, tmp, d_count, st)));
  k_unique_emit<<<grid, 256, 0, st>>>(x, n, flags, out);
  EBR_CUDA_TRY(cudaGetLastError());
  return EBR_OK;
}

}  // namespace prims
}  // namespace ebr
