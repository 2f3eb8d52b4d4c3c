// Index construction (Algorithm 1, Sec. 3.4) on the GPU.
//
// Step 1 (Block Grouping): every (k, v) pair becomes the 64-bit word
// k << 32 | v, so sorting the words orders them by (k, h = v >> 8, l = v & 255);
// dropping repeated words turns each run of equal (k, h) into the set B[k, h].
// Step 2 (Logarithmic Categorization): a run of n ads is one block of group
// g = ceil(log2 n), padded with zero bytes to 2^g slots.
// Step 3 (Storage Layout): per group, header[g] (h of each block) and
// values[g] (the low bytes) in (k, h) order, and keys[g], the row pointer
// giving each key's first block (keys[g][k] = group-g blocks with key < k).
//
// The radix sort, the duplicate removal and the prefix sums are this
// library's own device primitives (ebr_prims.cuh); the grouping and storage
// steps are the kernels below.

#include <cstring>
#include <vector>

#include "ebr_internal.cuh"
#include "ebr_prims.cuh"

namespace ebr {
int launch_quantize(const float *x, uint64_t n, ebr_dtype dt, void *out, cudaStream_t st);
int launch_quantize_rows_fp8(const float *x, uint64_t n, uint32_t d, uint8_t *q, float *scale,
                             cudaStream_t st);

namespace {

__global__ void k_pack(const uint32_t *__restrict__ key, const uint32_t *__restrict__ ad,
                       uint64_t nnz, uint32_t n_keys, uint32_t n_ads,
                       uint64_t *__restrict__ out, uint32_t *__restrict__ flags) {
  uint32_t bad = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < nnz;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t k = key[i], a = ad[i];
    if (k >= n_keys) { bad |= DEVERR_BAD_BUILD_KEY; k = 0; }
    if (a >= n_ads) { bad |= DEVERR_BAD_AD; a = 0; }
    out[i] = ((uint64_t)k << 32) | a;
  }
  if (bad) atomicOr(flags, bad);
}

// keys per ad over the distinct (key, ad) pairs, and their maximum
__global__ void k_keys_per_ad(const uint64_t *__restrict__ x, uint32_t m, uint32_t *__restrict__ cnt) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
    atomicAdd(&cnt[(uint32_t)x[i]], 1u);
}
__global__ void k_u32_to_u16(const uint32_t *__restrict__ v, uint32_t n, uint16_t *__restrict__ out) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = (uint16_t)v[i];
}
__global__ void k_max_u32(const uint32_t *__restrict__ v, uint32_t n, unsigned int *__restrict__ out) {
  uint32_t mx = 0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    mx = max(mx, v[i]);
  atomicMax(out, mx);
}

// bs[i] = 1 where a new (k, h) run starts in the sorted, duplicate-free words.
__global__ void k_block_flags(const uint64_t *__restrict__ x, uint32_t m,
                              uint32_t *__restrict__ bs) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
    bs[i] = (i == 0 || (x[i] >> 8) != (x[i - 1] >> 8)) ? 1u : 0u;
}

// start[b] = first word of block b; start[nb] = m.
__global__ void k_block_start(const uint32_t *__restrict__ bs, const uint32_t *__restrict__ bid,
                              uint32_t m, uint32_t *__restrict__ start) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    if (bs[i]) start[bid[i] - 1] = i;
    if (i == m - 1) start[bid[i]] = m;
  }
}

__device__ __forceinline__ uint32_t ceil_log2(uint32_t n) {
  return n <= 1 ? 0u : 32u - __clz(n - 1);
}

// Per block: group, and counts per (group, key) and per group.
__global__ void k_block_info(const uint64_t *__restrict__ x, const uint32_t *__restrict__ start,
                             uint32_t nb, uint32_t n_keys, uint8_t *__restrict__ grp,
                             uint32_t *__restrict__ key_cnt /* [9][n_keys+1] */,
                             unsigned long long *__restrict__ gcount) {
  __shared__ unsigned int s_cnt[kGroups];
  if (threadIdx.x < kGroups) s_cnt[threadIdx.x] = 0;
  __syncthreads();
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
    uint32_t n = start[b + 1] - start[b];
    uint32_t g = ceil_log2(n);
    uint32_t k = (uint32_t)(x[start[b]] >> 32);
    grp[b] = (uint8_t)g;
    atomicAdd(&key_cnt[(uint64_t)g * (n_keys + 1) + k], 1u);
    atomicAdd(&s_cnt[g], 1u);
  }
  __syncthreads();
  if (threadIdx.x < kGroups && s_cnt[threadIdx.x])
    atomicAdd(&gcount[threadIdx.x], (unsigned long long)s_cnt[threadIdx.x]);
}

__global__ void k_iota(uint32_t *__restrict__ p, uint32_t n) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    p[i] = i;
}

struct EmitArgs {
  uint32_t *header[kGroups];
  uint8_t *values[kGroups];
  unsigned long long gstart[kGroups + 1];
};

// Blocks sorted (stably) by group: position p - gstart[g] is the block's rank
// inside its group, which preserves the (k, h) order.
__global__ void k_emit(const uint64_t *__restrict__ x, const uint32_t *__restrict__ start,
                       const uint32_t *__restrict__ perm, const uint8_t *__restrict__ grp_sorted,
                       uint32_t nb, EmitArgs args) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < nb; p += gridDim.x * blockDim.x) {
    uint32_t b = perm[p];
    uint32_t g = grp_sorted[p];
    uint64_t rank = p - args.gstart[g];
    uint32_t s0 = start[b], n = start[b + 1] - s0;
    args.header[g][rank] = (uint32_t)((x[s0] >> 8) & 0xFFFFFFu);
    uint8_t *dst = args.values[g] + (rank << g);
    for (uint32_t s = 0; s < n; s++) dst[s] = (uint8_t)(x[s0 + s] & 255u);
  }
}

// Window-major view of the same blocks: sort key (g, h, k) per block, with the
// block's position in the group-sorted order as payload.
__global__ void k_wm_keys(const uint64_t *__restrict__ x, const uint32_t *__restrict__ start,
                          const uint32_t *__restrict__ perm, const uint8_t *__restrict__ grp_sorted,
                          uint32_t nb, uint64_t *__restrict__ skey, uint32_t *__restrict__ sval) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < nb; p += gridDim.x * blockDim.x) {
    const uint64_t w0 = x[start[perm[p]]];
    const uint64_t h = (w0 >> 8) & 0xFFFFFFull, k = w0 >> 32;
    skey[p] = ((uint64_t)grp_sorted[p] << 56) | (h << 32) | k;
    sval[p] = p;
  }
}

struct WinPtrs {
  const uint32_t *p[kGroups];
};

struct WmArgs {
  const uint8_t *values[kGroups];
  uint32_t *wkey[kGroups];
  uint8_t *wvals[kGroups];
  uint32_t *wcnt;  // [9][n_win + 1]
  uint32_t n_win;
  unsigned long long gstart[kGroups + 1];
};

// q-th block in (g, h, k) order: store its key and copy its 2^g value bytes.
__global__ void k_wm_emit(const uint64_t *__restrict__ skey, const uint32_t *__restrict__ sval,
                          uint32_t nb, WmArgs a) {
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < nb; q += gridDim.x * blockDim.x) {
    const uint64_t sk = skey[q];
    const uint32_t g = (uint32_t)(sk >> 56), h = (uint32_t)((sk >> 32) & 0xFFFFFFu);
    const uint64_t rank = q - a.gstart[g], src = sval[q] - a.gstart[g];
    a.wkey[g][rank] = (uint32_t)sk;
    const uint8_t *from = a.values[g] + (src << g);
    uint8_t *to = a.wvals[g] + (rank << g);
    if (g >= 2) {
      for (uint32_t s = 0; s < (1u << g); s += 4)
        *reinterpret_cast<uint32_t *>(to + s) = *reinterpret_cast<const uint32_t *>(from + s);
    } else {
      for (uint32_t s = 0; s < (1u << g); s++) to[s] = from[s];
    }
    atomicAdd(&a.wcnt[(uint64_t)g * (a.n_win + 1) + h], 1u);
  }
}

// Bytes a window's segments of the window-major view occupy once each segment
// is widened to 16-byte boundaries (the staging size of the fused scan).
// Also: the most 32-unit work chunks any window has (a unit is one 4-slot
// word in groups >= 2, one block in groups 0 and 1).
__global__ void k_win_bytes(WinPtrs wp, uint32_t n_win, unsigned int *out_max) {
  uint32_t mx = 0, mc = 0, ms = 0;
  for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < n_win; w += gridDim.x * blockDim.x) {
    uint64_t total = 0, chunks = 0, slots = 0;
    for (int g = 0; g < kGroups; g++) {
      const uint64_t lo = wp.p[g][w], hi = wp.p[g][w + 1];
      if (hi == lo) continue;
      const uint64_t k0 = (lo * 4) & ~15ull, k1 = (hi * 4 + 15) & ~15ull;
      const uint64_t v0 = (lo << g) & ~15ull, v1 = ((hi << g) + 15) & ~15ull;
      total += (k1 - k0) + (v1 - v0);
      chunks += (((hi - lo) << (g >= 2 ? g - 2 : 0)) + 31) >> 5;
      slots += (hi - lo) << g;
    }
    mx = max(mx, (uint32_t)min(total, (uint64_t)0xFFFFFFFFu));
    mc = max(mc, (uint32_t)min(chunks, (uint64_t)0xFFFFFFFFu));
    ms = max(ms, (uint32_t)min(slots, (uint64_t)0xFFFFFFFFu));
  }
  atomicMax(out_max, mx);
  atomicMax(out_max + 1, mc);
  atomicMax(out_max + 2, ms);
}

inline int grid_for(uint64_t n, int threads = 256, int cap = 1 << 16) {
  uint64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > (uint64_t)cap) b = cap;
  return (int)b;
}

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace
}  // namespace ebr

using namespace ebr;

static int build_impl(const ebr_index_desc *desc, ebr_index *ix, cudaStream_t st) {
  const uint64_t nnz = desc->nnz;
  const uint32_t n_keys = desc->n_keys, n_ads = desc->n_ads;
  DevBuf d_key, d_ad, w0, w1, tmp, bs, bid, start, grp, grp2, perm, perm2, cnt, gcount, flags;
  DevBuf skey, skey2, sval, sval2, wcnt;
  std::vector<DevBuf *> temps = {&d_key, &d_ad, &w0, &w1, &tmp, &bs, &bid, &start,
                                 &grp, &grp2, &perm, &perm2, &cnt, &gcount, &flags,
                                 &skey, &skey2, &sval, &sval2, &wcnt};
  auto cleanup = [&]() {
    for (auto *b : temps) dev_free(*b);
  };
  int rc = EBR_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
#define BTRY(expr)                  \
  do {                              \
    rc = (expr);                    \
    if (rc != EBR_OK) goto fail;    \
  } while (0)
#define BCUDA(expr)                                                                       \
  do {                                                                                    \
    cudaError_t _e = (expr);                                                              \
    if (_e != cudaSuccess) {                                                              \
      set_error("%s: %s", #expr, cudaGetErrorString(_e));                                 \
      rc = EBR_ECUDA;                                                                     \
      goto fail;                                                                          \
    }                                                                                     \
  } while (0)
  {
    uint64_t m_host = 0;
    uint32_t nb = 0;
    unsigned long long gc[kGroups] = {0};
    uint32_t hflags = 0;
    uint32_t *d_num = nullptr;
    size_t need = 0;
    const uint32_t *pk = desc->post_key, *pa = desc->post_ad;
    int end_bit = 32;
    EmitArgs ea;
    size_t hdr_off[kGroups], val_off[kGroups], hdr_total = 0, val_total = 0;

    BCUDA(cudaEventCreate(&e0));
    BCUDA(cudaEventCreate(&e1));
    // Inputs may live on the host: bring them over first (not part of build_ms).
    if (nnz) {
      BTRY(dev_alloc(d_key, nnz * 4));
      BTRY(dev_alloc(d_ad, nnz * 4));
      BCUDA(cudaMemcpyAsync(d_key.p, pk, nnz * 4, cudaMemcpyDefault, st));
      BCUDA(cudaMemcpyAsync(d_ad.p, pa, nnz * 4, cudaMemcpyDefault, st));
    }
    BTRY(dev_alloc(w0, (nnz + 1) * 8));
    BTRY(dev_alloc(w1, (nnz + 1) * 8));
    BTRY(dev_alloc(flags, 64));
    BTRY(dev_alloc(gcount, kGroups * 8));
    BTRY(dev_alloc(cnt, (size_t)kGroups * (n_keys + 1) * 4));
    BCUDA(cudaMemsetAsync(flags.p, 0, 64, st));
    BCUDA(cudaMemsetAsync(gcount.p, 0, kGroups * 8, st));
    BCUDA(cudaMemsetAsync(cnt.p, 0, (size_t)kGroups * (n_keys + 1) * 4, st));
    BCUDA(cudaEventRecord(e0, st));
    if (nnz) {
      k_pack<<<grid_for(nnz), 256, 0, st>>>((const uint32_t *)d_key.p, (const uint32_t *)d_ad.p,
                                            nnz, n_keys, n_ads, (uint64_t *)w0.p,
                                            (uint32_t *)flags.p);
      BCUDA(cudaGetLastError());
    }
    // key bits needed: 32 + ceil(log2 n_keys)
    while (end_bit < 64 && ((uint64_t)1 << (end_bit - 32)) < n_keys) end_bit++;
    {
      // scratch of every primitive below: the sort's counts, the scans' tile
      // sums, the unique's flags, and a word for the unique count
      need = std::max<size_t>(prims::sort_scratch(nnz),
                              (nnz + prims::scan_scratch(nnz) + 64) * 4);
      need = std::max<size_t>(need, (prims::scan_scratch((uint64_t)n_keys + 1) + 64) * 4);
      BTRY(dev_alloc(tmp, need + 256));
      d_num = (uint32_t *)((char *)tmp.p + align_up(need, 16));
      bool in_alt = false;
      BTRY(prims::radix_sort<uint64_t>((uint64_t *)w0.p, (uint64_t *)w1.p, nullptr, nullptr, nnz,
                                       end_bit, tmp.p, &in_alt, st));
      uint64_t *sorted = in_alt ? (uint64_t *)w1.p : (uint64_t *)w0.p;
      uint64_t *other = in_alt ? (uint64_t *)w0.p : (uint64_t *)w1.p;
      uint32_t *uflags = (uint32_t *)tmp.p;
      BTRY(prims::unique_sorted(sorted, other, nnz, uflags, uflags + nnz, d_num, st));
      uint32_t m_i = 0;
      BCUDA(cudaMemcpyAsync(&m_i, d_num, 4, cudaMemcpyDeviceToHost, st));
      BCUDA(cudaMemcpyAsync(&hflags, flags.p, 4, cudaMemcpyDeviceToHost, st));
      BCUDA(cudaStreamSynchronize(st));
      if (hflags) {
        rc = check_device_flags(hflags, "ebr_build_index");
        goto fail;
      }
      m_host = (uint64_t)m_i;
      // swap roles so that w0 holds the unique words
      if (other != (uint64_t *)w0.p) std::swap(w0, w1);
    }
    const uint64_t *x = (const uint64_t *)w0.p;
    const uint32_t m = (uint32_t)m_host;
    ix->nnz_unique = m_host;
    if (m > 0) {
      // most keys any ad has (bounds the fused scan's exact accumulators)
      BTRY(dev_alloc(bs, (size_t)std::max<uint64_t>(m, n_ads) * 4));
      BCUDA(cudaMemsetAsync(bs.p, 0, (size_t)n_ads * 4, st));
      BCUDA(cudaMemsetAsync(flags.p, 0, 4, st));
      k_keys_per_ad<<<grid_for(m), 256, 0, st>>>(x, m, (uint32_t *)bs.p);
      k_max_u32<<<grid_for(n_ads), 256, 0, st>>>((const uint32_t *)bs.p, n_ads,
                                                (unsigned int *)flags.p);
      BCUDA(cudaMemcpyAsync(&ix->max_keys_per_ad, flags.p, 4, cudaMemcpyDeviceToHost, st));
      BCUDA(cudaStreamSynchronize(st));
      if (ix->max_keys_per_ad <= 65535) {  // per-ad slot counts of the batched scan
        BTRY(dev_alloc(ix->ad_nkeys, (size_t)n_ads * 2));
        k_u32_to_u16<<<grid_for(n_ads), 256, 0, st>>>((const uint32_t *)bs.p, n_ads,
                                                      (uint16_t *)ix->ad_nkeys.p);
        BCUDA(cudaGetLastError());
        BCUDA(cudaStreamSynchronize(st));
      }
      dev_free(bs);
      BTRY(dev_alloc(bs, (size_t)m * 4));
      BTRY(dev_alloc(bid, (size_t)m * 4));
      k_block_flags<<<grid_for(m), 256, 0, st>>>(x, m, (uint32_t *)bs.p);
      BCUDA(cudaGetLastError());
      BTRY((prims::scan<uint32_t, prims::AddU32, true>((const uint32_t *)bs.p, (uint32_t *)bid.p, m,
                                                       prims::AddU32(), 0u, (uint32_t *)tmp.p,
                                                       nullptr, st)));
      BCUDA(cudaMemcpyAsync(&nb, (uint32_t *)bid.p + (m - 1), 4, cudaMemcpyDeviceToHost, st));
      BCUDA(cudaStreamSynchronize(st));
      BTRY(dev_alloc(start, ((size_t)nb + 1) * 4));
      k_block_start<<<grid_for(m), 256, 0, st>>>((const uint32_t *)bs.p,
                                                 (const uint32_t *)bid.p, m,
                                                 (uint32_t *)start.p);
      BCUDA(cudaGetLastError());
      BTRY(dev_alloc(grp, nb));
      BTRY(dev_alloc(grp2, nb));
      BTRY(dev_alloc(perm, (size_t)nb * 4));
      BTRY(dev_alloc(perm2, (size_t)nb * 4));
      k_block_info<<<grid_for(nb), 256, 0, st>>>(x, (const uint32_t *)start.p, nb, n_keys,
                                                 (uint8_t *)grp.p, (uint32_t *)cnt.p,
                                                 (unsigned long long *)gcount.p);
      BCUDA(cudaGetLastError());
      k_iota<<<grid_for(nb), 256, 0, st>>>((uint32_t *)perm.p, nb);
      BCUDA(cudaGetLastError());
      {
        // blocks by size group, stably (one 8-bit pass: grp2 / perm2 hold the result)
        bool alt = false;
        BTRY(prims::radix_sort<uint8_t>((uint8_t *)grp.p, (uint8_t *)grp2.p, (uint32_t *)perm.p,
                                        (uint32_t *)perm2.p, nb, 8, tmp.p, &alt, st));
        if (!alt) {  // a single block: nothing moved
          BCUDA(cudaMemcpyAsync(grp2.p, grp.p, nb, cudaMemcpyDeviceToDevice, st));
          BCUDA(cudaMemcpyAsync(perm2.p, perm.p, (size_t)nb * 4, cudaMemcpyDeviceToDevice, st));
        }
      }
    }
    // per-key row pointers: exclusive scan of counts over n_keys + 1 entries
    BTRY(dev_alloc(ix->mem_keys, (size_t)kGroups * (n_keys + 1) * 4));
    for (int g = 0; g < kGroups; g++) {
      BTRY((prims::scan<uint32_t, prims::AddU32, false>(
          (const uint32_t *)cnt.p + (size_t)g * (n_keys + 1),
          (uint32_t *)ix->mem_keys.p + (size_t)g * (n_keys + 1), (uint64_t)n_keys + 1,
          prims::AddU32(), 0u, (uint32_t *)tmp.p, nullptr, st)));
      ix->keys[g] = (uint32_t *)ix->mem_keys.p + (size_t)g * (n_keys + 1);
    }
    BCUDA(cudaMemcpyAsync(gc, gcount.p, sizeof(gc), cudaMemcpyDeviceToHost, st));
    BCUDA(cudaStreamSynchronize(st));
    for (int g = 0; g < kGroups; g++) {
      ix->n_blocks[g] = gc[g];
      hdr_off[g] = hdr_total;
      val_off[g] = val_total;
      hdr_total += align_up(gc[g] * 4, 256);
      val_total += align_up(gc[g] << g, 256);
    }
    BTRY(dev_alloc(ix->mem_header, hdr_total + 256));
    BTRY(dev_alloc(ix->mem_values, val_total + 256));
    BCUDA(cudaMemsetAsync(ix->mem_values.p, 0, val_total + 256, st));
    ea.gstart[0] = 0;
    for (int g = 0; g < kGroups; g++) {
      ix->header[g] = (uint32_t *)((char *)ix->mem_header.p + hdr_off[g]);
      ix->values[g] = (uint8_t *)ix->mem_values.p + val_off[g];
      ea.header[g] = ix->header[g];
      ea.values[g] = ix->values[g];
      ea.gstart[g + 1] = ea.gstart[g] + gc[g];
    }
    if (nb) {
      k_emit<<<grid_for(nb), 256, 0, st>>>(x, (const uint32_t *)start.p,
                                           (const uint32_t *)perm2.p, (const uint8_t *)grp2.p,
                                           nb, ea);
      BCUDA(cudaGetLastError());
    }
    BCUDA(cudaEventRecord(e1, st));
    BCUDA(cudaEventSynchronize(e1));
    BCUDA(cudaEventElapsedTime(&ix->build_ms, e0, e1));

    // ---- window-major view of the same blocks (for the fused dense scan)
    {
      const uint32_t n_win = (n_ads + 255) / 256;
      ix->n_win = n_win;
      BCUDA(cudaEventRecord(e0, st));
      BTRY(dev_alloc(ix->mem_wkey, hdr_total + 256));
      BTRY(dev_alloc(ix->mem_wvals, val_total + 256));
      BTRY(dev_alloc(ix->mem_winptr, (size_t)kGroups * (n_win + 1) * 4));
      BTRY(dev_alloc(wcnt, (size_t)kGroups * (n_win + 1) * 4));
      BCUDA(cudaMemsetAsync(wcnt.p, 0, (size_t)kGroups * (n_win + 1) * 4, st));
      WmArgs wa;
      wa.wcnt = (uint32_t *)wcnt.p;
      wa.n_win = n_win;
      for (int g = 0; g < kGroups; g++) {
        ix->wkey[g] = (uint32_t *)((char *)ix->mem_wkey.p + hdr_off[g]);
        ix->wvals[g] = (uint8_t *)ix->mem_wvals.p + val_off[g];
        ix->win_ptr[g] = (uint32_t *)ix->mem_winptr.p + (size_t)g * (n_win + 1);
        wa.values[g] = ix->values[g];
        wa.wkey[g] = ix->wkey[g];
        wa.wvals[g] = ix->wvals[g];
        wa.gstart[g] = ea.gstart[g];
      }
      wa.gstart[kGroups] = ea.gstart[kGroups];
      if (nb) {
        BTRY(dev_alloc(skey, (size_t)nb * 8));
        BTRY(dev_alloc(skey2, (size_t)nb * 8));
        BTRY(dev_alloc(sval, (size_t)nb * 4));
        BTRY(dev_alloc(sval2, (size_t)nb * 4));
        k_wm_keys<<<grid_for(nb), 256, 0, st>>>(x, (const uint32_t *)start.p,
                                                (const uint32_t *)perm2.p,
                                                (const uint8_t *)grp2.p, nb, (uint64_t *)skey.p,
                                                (uint32_t *)sval.p);
        BCUDA(cudaGetLastError());
        BTRY(dev_reserve(tmp, std::max<size_t>(prims::sort_scratch(nb),
                                               (prims::scan_scratch((uint64_t)n_win + 1) + 64) * 4) +
                                  256));
        bool alt = false;
        BTRY(prims::radix_sort<uint64_t>((uint64_t *)skey.p, (uint64_t *)skey2.p,
                                         (uint32_t *)sval.p, (uint32_t *)sval2.p, nb, 60, tmp.p,
                                         &alt, st));
        if (!alt) {  // the result ended in the first buffers
          std::swap(skey, skey2);
          std::swap(sval, sval2);
        }
        k_wm_emit<<<grid_for(nb), 256, 0, st>>>((const uint64_t *)skey2.p,
                                                (const uint32_t *)sval2.p, nb, wa);
        BCUDA(cudaGetLastError());
      }
      BTRY(dev_reserve(tmp, (prims::scan_scratch((uint64_t)n_win + 1) + 64) * 4 + 256));
      for (int g = 0; g < kGroups; g++)
        BTRY((prims::scan<uint32_t, prims::AddU32, false>(
            (const uint32_t *)wcnt.p + (size_t)g * (n_win + 1), ix->win_ptr[g],
            (uint64_t)n_win + 1, prims::AddU32(), 0u, (uint32_t *)tmp.p, nullptr, st)));
      {
        WinPtrs wp;
        for (int g = 0; g < kGroups; g++) wp.p[g] = ix->win_ptr[g];
        BCUDA(cudaMemsetAsync(flags.p, 0, 12, st));
        k_win_bytes<<<grid_for(n_win), 256, 0, st>>>(wp, n_win, (unsigned int *)flags.p);
        BCUDA(cudaGetLastError());
        uint32_t mm[3] = {0, 0, 0};
        BCUDA(cudaMemcpyAsync(mm, flags.p, 12, cudaMemcpyDeviceToHost, st));
        BCUDA(cudaStreamSynchronize(st));
        ix->max_win_bytes = mm[0];
        ix->max_win_chunks = mm[1];
        ix->max_win_slots = mm[2];
      }
      BCUDA(cudaEventRecord(e1, st));
      BCUDA(cudaEventSynchronize(e1));
      BCUDA(cudaEventElapsedTime(&ix->wm_build_ms, e0, e1));
    }
  }
  cleanup();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return EBR_OK;
fail:
  cleanup();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return rc;
#undef BTRY
#undef BCUDA
}

static int upload_embeddings(const ebr_index_desc *desc, ebr_index *ix, cudaStream_t st) {
  const uint64_t n = (uint64_t)desc->n_ads * desc->d;
  EBR_TRY(dev_alloc(ix->emb_f32, n * 4));
  EBR_CUDA_TRY(cudaMemcpyAsync(ix->emb_f32.p, desc->emb_f32, n * 4, cudaMemcpyDefault, st));
  if (desc->emb_dtype == EBR_BF16) {
    EBR_TRY(dev_alloc(ix->emb_q, n * 2));
    EBR_TRY(launch_quantize((const float *)ix->emb_f32.p, n, EBR_BF16, ix->emb_q.p, st));
  } else if (desc->emb_dtype == EBR_FP8E4M3) {
    EBR_TRY(dev_alloc(ix->emb_q, n));
    EBR_TRY(dev_alloc(ix->emb_scale, (uint64_t)desc->n_ads * 4));
    EBR_TRY(launch_quantize_rows_fp8((const float *)ix->emb_f32.p, desc->n_ads, desc->d,
                                     (uint8_t *)ix->emb_q.p, (float *)ix->emb_scale.p, st));
  }
  EBR_CUDA_TRY(cudaStreamSynchronize(st));
  return EBR_OK;
}

extern "C" void ebr_index_free(ebr_index *ix) {
  if (!ix) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(ix->device);
  dev_free(ix->mem_keys);
  dev_free(ix->mem_header);
  dev_free(ix->mem_values);
  dev_free(ix->mem_wkey);
  dev_free(ix->mem_wvals);
  dev_free(ix->mem_winptr);
  dev_free(ix->ad_nkeys);
  dev_free(ix->emb_f32);
  dev_free(ix->emb_q);
  dev_free(ix->emb_scale);
  Workspace &w = ix->ws;
  for (DevBuf *b : {&w.wide, &w.w_dense, &w.lens, &w.scan, &w.work, &w.scan_tmp, &w.cand,
                    &w.ctrl, &w.io_in, &w.io_out, &w.route_stats})
    dev_free(*b);
  batch_ws_free(ix->bws);
  if (w.host_ctrl) cudaFreeHost(w.host_ctrl);
  for (auto *v : {&ix->prof_pending, &ix->prof_pool, &ix->bprof_pending})
    for (auto &ev : *v)
      for (cudaEvent_t e : ev) cudaEventDestroy(e);
  cudaSetDevice(prev);
  delete ix;
}

extern "C" int ebr_build_index(const ebr_index_desc *desc, ebr_index **out) {
  clear_error();
  if (!desc || !out) {
    set_error("ebr_build_index: null argument");
    return EBR_EINVAL;
  }
  *out = nullptr;
  const uint32_t d = desc->d;
  if (desc->n_ads == 0 || desc->n_keys == 0 || desc->n_keys == 0xFFFFFFFFu ||
      desc->nnz >= (1ULL << 31) || (desc->nnz && (!desc->post_key || !desc->post_ad)) ||
      !desc->emb_f32 || !(d == 4 || d == 8 || d == 16 || d == 32 || d == 64 || d == 128) ||
      (int)desc->emb_dtype < 0 || (int)desc->emb_dtype > 2) {
    set_error("ebr_build_index: invalid description (n_ads=%u n_keys=%u nnz=%llu d=%u dtype=%d)",
              desc->n_ads, desc->n_keys, (unsigned long long)desc->nnz, d,
              (int)desc->emb_dtype);
    return EBR_EINVAL;
  }
  int prev = 0;
  cudaGetDevice(&prev);
  EBR_CUDA_TRY(cudaSetDevice(desc->device));
  ebr_index *ix = new ebr_index();
  ix->device = desc->device;
  ix->n_ads = desc->n_ads;
  ix->n_keys = desc->n_keys;
  ix->d = d;
  ix->dtype = desc->emb_dtype;
  ix->rescore_mult = desc->rescore_mult ? desc->rescore_mult : 4;
  cudaDeviceGetAttribute(&ix->num_sms, cudaDevAttrMultiProcessorCount, desc->device);
  cudaStream_t st = (cudaStream_t)desc->stream;
  int rc = build_impl(desc, ix, st);
  if (rc == EBR_OK) rc = upload_embeddings(desc, ix, st);
  if (rc != EBR_OK) {
    std::string msg = ebr_last_error();
    ebr_index_free(ix);
    set_error("%s", msg.c_str());
    cudaSetDevice(prev);
    return rc;
  }
  cudaSetDevice(prev);
  *out = ix;
  return EBR_OK;
}

extern "C" int ebr_index_get_info(const ebr_index *ix, ebr_index_info *out) {
  clear_error();
  if (!ix || !out) {
    set_error("ebr_index_get_info: null argument");
    return EBR_EINVAL;
  }
  memset(out, 0, sizeof(*out));
  out->n_ads = ix->n_ads;
  out->n_keys = ix->n_keys;
  out->d = ix->d;
  out->emb_dtype = ix->dtype;
  out->rescore_mult = ix->rescore_mult;
  out->nnz_unique = ix->nnz_unique;
  uint64_t bytes = 0;
  for (int g = 0; g < kGroups; g++) {
    out->n_blocks[g] = ix->n_blocks[g];
    bytes += 4ull * (ix->n_keys + 1) + 4ull * ix->n_blocks[g] + (ix->n_blocks[g] << g);
  }
  out->index_bytes = bytes;
  uint64_t per = ix->dtype == EBR_F32 ? 4 : (ix->dtype == EBR_BF16 ? 2 : 1);
  out->emb_bytes = (uint64_t)ix->n_ads * ix->d * per + (ix->dtype == EBR_FP8E4M3 ? 4ull * ix->n_ads : 0);
  out->build_ms = ix->build_ms;
  out->window_view_ms = ix->wm_build_ms;
  out->window_view_bytes = bytes - 4ull * kGroups * (ix->n_keys + 1) + 4ull * kGroups * (ix->n_win + 1);
  out->n_windows = ix->n_win;
  out->max_keys_per_ad = ix->max_keys_per_ad;
  out->max_window_slots = ix->max_win_slots;
  out->max_window_chunks = ix->max_win_chunks;
  return EBR_OK;
}

extern "C" int ebr_index_export(const ebr_index *ix, uint32_t g, uint32_t *keys, uint32_t *header,
                                uint8_t *values) {
  clear_error();
  if (!ix || g >= (uint32_t)kGroups) {
    set_error("ebr_index_export: bad index or group");
    return EBR_EINVAL;
  }
  int prev = 0;
  cudaGetDevice(&prev);
  EBR_CUDA_TRY(cudaSetDevice(ix->device));
  if (keys) EBR_CUDA_TRY(cudaMemcpy(keys, ix->keys[g], (ix->n_keys + 1ull) * 4, cudaMemcpyDeviceToHost));
  if (header && ix->n_blocks[g])
    EBR_CUDA_TRY(cudaMemcpy(header, ix->header[g], ix->n_blocks[g] * 4, cudaMemcpyDeviceToHost));
  if (values && ix->n_blocks[g])
    EBR_CUDA_TRY(cudaMemcpy(values, ix->values[g], ix->n_blocks[g] << g, cudaMemcpyDeviceToHost));
  cudaSetDevice(prev);
  return EBR_OK;
}

extern "C" int ebr_index_export_emb(const ebr_index *ix, void *codes, float *scale) {
  clear_error();
  if (!ix) {
    set_error("ebr_index_export_emb: null index");
    return EBR_EINVAL;
  }
  int prev = 0;
  cudaGetDevice(&prev);
  EBR_CUDA_TRY(cudaSetDevice(ix->device));
  uint64_t n = (uint64_t)ix->n_ads * ix->d;
  if (codes) {
    if (ix->dtype == EBR_F32)
      EBR_CUDA_TRY(cudaMemcpy(codes, ix->emb_f32.p, n * 4, cudaMemcpyDeviceToHost));
    else
      EBR_CUDA_TRY(cudaMemcpy(codes, ix->emb_q.p, n * (ix->dtype == EBR_BF16 ? 2 : 1),
                              cudaMemcpyDeviceToHost));
  }
  if (scale && ix->dtype == EBR_FP8E4M3)
    EBR_CUDA_TRY(cudaMemcpy(scale, ix->emb_scale.p, ix->n_ads * 4ull, cudaMemcpyDeviceToHost));
  cudaSetDevice(prev);
  return EBR_OK;
}
