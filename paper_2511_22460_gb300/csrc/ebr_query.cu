// Query path: expansion of user features into (k, w^), the key-major wide
// scatter of Algorithm 2, the streaming inner product fused with the wide add
// and a per-CTA radix-select top-K, the final merge, and FP32 rescoring.

#include <algorithm>
#include <array>
#include <cstring>
#include <mutex>
#include <vector>

#include "ebr_device.cuh"
#include "ebr_internal.cuh"
#include "ebr_prims.cuh"

namespace ebr {

// =====================================================================
// Cross model and query expansion
// =====================================================================
// Metadata words (uint32) uploaded to the device, in this order:
//   key_off[f_a + 1], vocab_u[f_u], vocab_a[f_a], pair_ptr[f_a + 1]
//   (pairs grouped by ad field j), pair_of[n_pairs] (pair ids by j),
//   pair_user[n_pairs] (user field i of pair p), w_off_lo[n_pairs],
//   w_off_hi[n_pairs].
struct CrossView {
  uint32_t f_u, f_a, n_pairs, n_keys, hashed, hash_bits;
  const uint32_t *key_off, *vocab_u, *vocab_a, *pair_ptr, *pair_of, *pair_user, *w_lo, *w_hi;
  const float *table;
};

static CrossView cross_view(const ebr_cross *c) {
  CrossView v;
  v.f_u = c->f_u;
  v.f_a = c->f_a;
  v.n_pairs = c->n_pairs;
  v.n_keys = c->n_keys;
  v.hashed = c->kind == EBR_W_HASHED;
  v.hash_bits = c->hash_bits;
  const uint32_t *m = (const uint32_t *)c->meta.p;
  v.key_off = m;
  m += c->f_a + 1;
  v.vocab_u = m;
  m += c->f_u;
  v.vocab_a = m;
  m += c->f_a;
  v.pair_ptr = m;
  m += c->f_a + 1;
  v.pair_of = m;
  m += c->n_pairs;
  v.pair_user = m;
  m += c->n_pairs;
  v.w_lo = m;
  m += c->n_pairs;
  v.w_hi = m;
  v.table = (const float *)c->table.p;
  return v;
}

// SplitMix64 (Vigna): state += 0x9E3779B97F4A7C15, then two
// xor-shift-multiply rounds and a final xor-shift; the cross-weight hash is
// the first output for state x.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// w_hat[b][key_off[j] + v] = sum over pairs p = (i, j) of w_p(user[b][i], v).
// One thread per (request, key); the pairs of field j are summed in pair order.
// The pair lists of the ad fields (and, for one request, the request's user
// value of every pair) are staged in shared memory, so a thread's loop over
// the pairs of its key issues only the weight gathers, independently of
// each other.  With wmax set, the largest |w^| (FP32 bits) is max-reduced
// into it (non-finite sums are flagged).
// user_ptr != nullptr (batch 1 only): multi-valued user fields, field i
// holding users[user_ptr[i] .. user_ptr[i+1]); every value is one hit
// feature, so a pair (i, j) adds w_ij(u, v) for each u of field i.
// Packed terms (wq != nullptr, batch 1, single-valued user fields): each w^
// is also written as the fixed-point term the fused scan decodes (pack_term)
// with the exponent F given (chosen from the cross model's bound on |w^|,
// so it is known before w^ is); |w^| above wlimit, which the bound excludes,
// is flagged.
struct PackOut {
  uint32_t *wq;
  int *fx_out;
  int F, cls_shift;
  float wlimit;
};

__global__ void k_expand(CrossView cv, const uint32_t *__restrict__ users, uint32_t batch,
                         float *__restrict__ w_hat, uint32_t *__restrict__ flags,
                         uint32_t *__restrict__ wmax, const uint32_t *__restrict__ user_ptr,
                         uint32_t n_uv, PackOut po) {
  extern __shared__ uint32_t s_mem[];
  __shared__ uint32_t s_seq_ok;
  uint32_t *s_off = s_mem;                    // key_off[f_a + 1]
  uint32_t *s_ptr = s_off + cv.f_a + 1;       // pair_ptr[f_a + 1]
  uint32_t *s_of = s_ptr + cv.f_a + 1;        // pair_of[n_pairs]
  uint32_t *s_usr = s_of + cv.n_pairs;        // pair_user[n_pairs]
  uint32_t *s_u = s_usr + cv.n_pairs;         // batch 1: u of each pair, or ~0u if out of range
  uint32_t *s_up = s_u + cv.n_pairs;          // multi-valued: user_ptr[f_u + 1]
  const bool multi = user_ptr != nullptr && batch == 1;
  if (threadIdx.x == 0) s_seq_ok = 1;
  for (uint32_t j = threadIdx.x; j <= cv.f_a; j += blockDim.x) {
    s_off[j] = cv.key_off[j];
    s_ptr[j] = cv.pair_ptr[j];
  }
  if (multi) {
    __syncthreads();  // s_seq_ok initialised
    for (uint32_t i = threadIdx.x; i <= cv.f_u; i += blockDim.x) {
      const uint32_t x = user_ptr[i];
      s_up[i] = x;
      const bool ok = i == 0 ? x == 0 : (user_ptr[i - 1] <= x && (i < cv.f_u || x == n_uv));
      if (!ok) s_seq_ok = 0;
    }
  }
  for (uint32_t q = threadIdx.x; q < cv.n_pairs; q += blockDim.x) {
    s_of[q] = cv.pair_of[q];
    const uint32_t i = cv.pair_user[q];
    s_usr[q] = i;
    if (batch == 1 && !multi) {
      const uint32_t u = users[i];
      s_u[q] = u < cv.vocab_u[i] ? u : ~0u;
    }
  }
  __syncthreads();
  if (multi && !s_seq_ok) {  // malformed offsets: flag, every field treated as empty
    if (threadIdx.x == 0) atomicOr(flags, DEVERR_BAD_USER);
    for (uint32_t i = threadIdx.x; i <= cv.f_u; i += blockDim.x) s_up[i] = 0;
    __syncthreads();
  }
  const uint64_t total = (uint64_t)batch * cv.n_keys;
  uint32_t bad = 0, mx = 0;
  const bool pack = po.wq != nullptr && batch == 1 && !multi;
  pdl_trigger();  // the fused scan may start streaming its embedding rows
  const float s0 = pow2f(po.F), s1 = pow2f(po.F + po.cls_shift),
              s2 = pow2f(po.F + 2 * po.cls_shift);
  if (pack && blockIdx.x == 0 && threadIdx.x == 0) *po.fx_out = po.F;
  for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total;
       t += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t b = (uint32_t)(t / cv.n_keys), key = (uint32_t)(t % cv.n_keys);
    // field j: last j with key_off[j] <= key
    uint32_t lo = 0, hi = cv.f_a;  // invariant key_off[lo] <= key < key_off[hi]
    while (hi - lo > 1) {
      uint32_t mid = (lo + hi) >> 1;
      if (s_off[mid] <= key) lo = mid; else hi = mid;
    }
    const uint32_t j = lo, v = key - s_off[j];
    float acc = 0.f;
    const uint32_t q0 = s_ptr[j], q1 = s_ptr[j + 1];
    if (multi) {
      for (uint32_t q = q0; q < q1; q++) {
        const uint32_t p = s_of[q];
        const uint32_t i = s_usr[p];
        for (uint32_t r = s_up[i]; r < s_up[i + 1]; r++) {
          const uint32_t u = __ldg(users + r);
          if (u >= cv.vocab_u[i]) { bad |= DEVERR_BAD_USER; continue; }
          float w;
          if (cv.hashed) {
            uint64_t x = ((uint64_t)p << 40) | ((uint64_t)u << 20) | (uint64_t)v;
            w = __ldg(cv.table + (splitmix64(x) & ((1ull << cv.hash_bits) - 1ull)));
          } else {
            uint64_t off = ((uint64_t)cv.w_hi[p] << 32) | cv.w_lo[p];
            w = __ldg(cv.table + off + (uint64_t)u * cv.vocab_a[j] + v);
          }
          acc += w;
        }
      }
      w_hat[t] = acc;
      mx = max(mx, __float_as_uint(acc) & 0x7FFFFFFFu);
      continue;
    }
#pragma unroll 4
    for (uint32_t q = q0; q < q1; q++) {
      const uint32_t p = s_of[q];
      uint32_t u;
      if (batch == 1) {
        u = s_u[p];
      } else {
        const uint32_t i = s_usr[p];
        u = users[(uint64_t)b * cv.f_u + i];
        if (u >= cv.vocab_u[i]) u = ~0u;
      }
      if (u == ~0u) { bad |= DEVERR_BAD_USER; continue; }
      float w;
      if (cv.hashed) {
        uint64_t x = ((uint64_t)p << 40) | ((uint64_t)u << 20) | (uint64_t)v;
        w = __ldg(cv.table + (splitmix64(x) & ((1ull << cv.hash_bits) - 1ull)));
      } else {
        uint64_t off = ((uint64_t)cv.w_hi[p] << 32) | cv.w_lo[p];
        w = __ldg(cv.table + off + (uint64_t)u * cv.vocab_a[j] + v);
      }
      acc += w;
    }
    w_hat[t] = acc;
    if (pack) {
      if (!(fabsf(acc) <= po.wlimit)) bad |= DEVERR_RANGE;
      po.wq[t] = pack_term(acc, s0, s1, s2, po.cls_shift > 0);
    }
    mx = max(mx, __float_as_uint(acc) & 0x7FFFFFFFu);
  }
  if (bad) atomicOr(flags, bad);
  if (wmax && !pack) {  // packed terms need no max |w^| (their exponent is set)
    __shared__ uint32_t s_mx;
    if (threadIdx.x == 0) s_mx = 0;
    __syncthreads();
    for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(&s_mx, mx);
    __syncthreads();
    if (threadIdx.x == 0 && s_mx) {  // one global atomic per block
      if (s_mx >= 0x7F800000u) atomicOr(flags, DEVERR_RANGE);
      atomicMax(wmax, s_mx >= 0x7F800000u ? 0u : s_mx);
    }
  }
}

// =====================================================================
// Algorithm 2: key-major wide scatter with merge-based load balance
// =====================================================================
// Work unit: one 4-slot word of a block in groups g >= 2 (2^(g-2) units per
// block), one whole block in groups 0 and 1.  All nine groups are walked in
// one launch: entry p = g * n_q + i of the concatenated length array is
// query key i in group g (the per-group key lengths of Algorithm 2, scanned
// once across groups so that one grid balances all of them).
struct LenPair {
  unsigned long long units;
  unsigned int ne;
  unsigned int pad;
};
struct LenPairSum {
  __host__ __device__ __forceinline__ LenPair operator()(const LenPair &a, const LenPair &b) const {
    LenPair r;
    r.units = a.units + b.units;
    r.ne = a.ne + b.ne;
    r.pad = 0;
    return r;
  }
};

struct WorkEntry {
  unsigned long long seg_g;  // first unit (low 56 bits) | group << 56
  uint32_t blk0;             // first block of the key in its group
  float w;                   // w^ of the query entry
};

struct IndexView {
  const uint32_t *keys[kGroups];
  const uint32_t *header[kGroups];
  const uint8_t *values[kGroups];
  uint32_t n_keys, n_ads;
};

// Algorithm 2 work units of the whole index (every key's blocks).
static unsigned long long index_units(const ebr_index *ix) {
  unsigned long long u = 0;
  for (int g = 0; g < kGroups; g++) u += (unsigned long long)ix->n_blocks[g] << (g >= 2 ? g - 2 : 0);
  return u;
}

static IndexView index_view(const ebr_index *ix) {
  IndexView v;
  for (int g = 0; g < kGroups; g++) {
    v.keys[g] = ix->keys[g];
    v.header[g] = ix->header[g];
    v.values[g] = ix->values[g];
  }
  v.n_keys = ix->n_keys;
  v.n_ads = ix->n_ads;
  return v;
}

__device__ __forceinline__ uint32_t unit_shift(uint32_t g) { return g >= 2 ? g - 2 : 0; }

// A sparse key list summed into a dense w^ over the key space (repeated keys
// add), for the window-major traversal: the fused scan then decodes every
// window's blocks and skips the additions of keys whose w^ is zero.
__global__ void k_list_to_dense(const uint32_t *__restrict__ q_key, const float *__restrict__ q_w,
                                uint32_t n_q, uint32_t n_keys, float *__restrict__ w_dense,
                                uint32_t *__restrict__ flags) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_q; i += gridDim.x * blockDim.x) {
    const uint32_t key = q_key[i];
    if (key >= n_keys)
      atomicOr(flags, DEVERR_BAD_KEY);
    else if (q_w[i] != 0.0f)
      atomicAdd(&w_dense[key], q_w[i]);
  }
}

// k_length of Algorithm 2 for every (group, query entry), in work units.
// q_key == nullptr: dense query, entry i is key i.  Zero weights are dropped.
__global__ void k_wide_lens(IndexView ix, const uint32_t *__restrict__ q_key,
                            const float *__restrict__ q_w, uint32_t n_q, LenPair *__restrict__ lens,
                            uint32_t *__restrict__ flags) {
  const uint64_t total = (uint64_t)kGroups * n_q;
  for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p <= total;
       p += (uint64_t)gridDim.x * blockDim.x) {
    LenPair lp;
    lp.units = 0;
    lp.ne = 0;
    lp.pad = 0;
    if (p < total) {
      const uint32_t g = (uint32_t)(p / n_q), i = (uint32_t)(p % n_q);
      const uint32_t key = q_key ? q_key[i] : i;
      if (key >= ix.n_keys) {
        if (g == 0) atomicOr(flags, DEVERR_BAD_KEY);
      } else if (q_w[i] != 0.0f) {
        const uint32_t nb = ix.keys[g][key + 1] - ix.keys[g][key];
        lp.units = (unsigned long long)nb << unit_shift(g);
        lp.ne = nb ? 1u : 0u;
      }
    }
    lens[p] = lp;
  }
}

constexpr int kWideThreads = 256;
constexpr int kWideUPT = 8;                         // units per thread per tile
constexpr int kWideTile = kWideThreads * kWideUPT;  // units per tile

// Compact the non-empty (group, key) entries: entry e covers work units
// [seg_e, seg_e + units_e) of the whole query.  route_units != 0: choose the
// traversal of a sparse list on the device (ctrl->route): the window-major
// decode when the list's work units reach 1/kRouteRatio of the whole
// index's, where Algorithm 2's scatter costs more than decoding every window.
constexpr unsigned long long kRouteRatio = 8;

__global__ void k_wide_compact(IndexView ix, const uint32_t *__restrict__ q_key,
                               const float *__restrict__ q_w, uint32_t n_q,
                               const LenPair *__restrict__ lens, const LenPair *__restrict__ scan,
                               WorkEntry *__restrict__ work, Ctrl *__restrict__ ctrl,
                               unsigned long long route_units,
                               unsigned long long *__restrict__ route_stats) {
  const uint64_t total = (uint64_t)kGroups * n_q;
  for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p <= total;
       p += (uint64_t)gridDim.x * blockDim.x) {
    if (p == total) {
      ctrl->total_units = scan[p].units;
      ctrl->n_work = scan[p].ne;
      const uint32_t r = route_units && scan[p].units * kRouteRatio >= route_units ? 1u : 0u;
      ctrl->route = r;
      if (route_units && route_stats) {
        atomicAdd(&route_stats[0], 1ull);
        atomicAdd(&route_stats[1], (unsigned long long)r);
      }
      continue;
    }
    if (!lens[p].ne) continue;
    const uint32_t g = (uint32_t)(p / n_q), i = (uint32_t)(p % n_q);
    const uint32_t key = q_key ? q_key[i] : i;
    WorkEntry we;
    we.seg_g = scan[p].units | ((unsigned long long)g << 56);
    we.blk0 = ix.keys[g][key];
    we.w = q_w[i];
    work[scan[p].ne] = we;
  }
}

// Short lists: the three steps above (per-entry lengths, their exclusive
// scan, the compaction) in one CTA and one launch.  Thread t owns the
// contiguous entries [t * per, (t + 1) * per) of the group-major order
// p = g * n_q + i, so a block scan of the per-thread sums gives every entry's
// first unit and slot.  With route_units != 0 it also takes the traversal
// decision of k_wide_compact; for the window-major decode it sums the list
// into w_dense itself, reduces max |w^| into ctrl->pad (what the fused scan's
// fixed-point scale needs) and leaves no work for the scatter.
constexpr int kPlanThreads = 1024;
constexpr uint32_t kPlanMaxPer = 8;  // entries per thread (longer lists: the three kernels)
constexpr uint64_t kPlanMaxEntries = (uint64_t)kPlanThreads * kPlanMaxPer;
constexpr uint32_t kRouteWindow = 1u, kRouteSummed = 2u;  // ctrl->route bits

__device__ __forceinline__ unsigned long long plan_entry(const IndexView &ix,
                                                         const uint32_t *__restrict__ q_key,
                                                         const float *__restrict__ q_w,
                                                         uint32_t n_q, uint32_t p, uint32_t &key,
                                                         uint32_t &g, float &wv) {
  g = p / n_q;
  const uint32_t i = p - g * n_q;
  key = q_key[i];
  wv = q_w[i];
  if (key >= ix.n_keys || wv == 0.0f) return 0ull;
  return (unsigned long long)(ix.keys[g][key + 1] - ix.keys[g][key]) << unit_shift(g);
}

__global__ void __launch_bounds__(kPlanThreads) k_wide_plan(
    IndexView ix, const uint32_t *__restrict__ q_key, const float *__restrict__ q_w, uint32_t n_q,
    WorkEntry *__restrict__ work, Ctrl *__restrict__ ctrl, unsigned long long route_units,
    unsigned long long *__restrict__ route_stats, float *__restrict__ w_dense) {
  __shared__ unsigned long long s_u[32];
  __shared__ uint32_t s_n[32], s_m[32];
  __shared__ uint32_t s_route;
  const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t total = kGroups * n_q;
  const uint32_t per = (total + kPlanThreads - 1) / kPlanThreads;
  const uint32_t p0 = min(total, tid * per), p1 = min(total, p0 + per);
  // pass 1: this thread's units and non-empty entries
  unsigned long long su = 0;
  uint32_t sn = 0, bad = 0;
  for (uint32_t p = p0; p < p1; p++) {
    uint32_t key, g;
    float wv;
    const unsigned long long u = plan_entry(ix, q_key, q_w, n_q, p, key, g, wv);
    su += u;
    sn += u ? 1u : 0u;
    bad |= (g == 0 && key >= ix.n_keys) ? 1u : 0u;
  }
  if (bad) atomicOr(&ctrl->flags, DEVERR_BAD_KEY);
  // block exclusive scan of (units, entries)
  unsigned long long iu = su;
  uint32_t in = sn;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long tu = __shfl_up_sync(0xffffffffu, iu, o);
    const uint32_t tn = __shfl_up_sync(0xffffffffu, in, o);
    if (lane >= (uint32_t)o) {
      iu += tu;
      in += tn;
    }
  }
  if (lane == 31) {
    s_u[wid] = iu;
    s_n[wid] = in;
  }
  __syncthreads();
  if (wid == 0) {
    unsigned long long wu = s_u[lane];
    uint32_t wn = s_n[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long tu = __shfl_up_sync(0xffffffffu, wu, o);
      const uint32_t tn = __shfl_up_sync(0xffffffffu, wn, o);
      if (lane >= (uint32_t)o) {
        wu += tu;
        wn += tn;
      }
    }
    s_u[lane] = wu;  // inclusive over warps
    s_n[lane] = wn;
  }
  __syncthreads();
  const unsigned long long all_u = s_u[31];
  const uint32_t all_n = s_n[31];
  unsigned long long off_u = iu - su + (wid ? s_u[wid - 1] : 0ull);
  uint32_t off_n = in - sn + (wid ? s_n[wid - 1] : 0u);
  if (tid == 0) {
    const uint32_t r = route_units && all_u * kRouteRatio >= route_units ? kRouteWindow : 0u;
    s_route = r;
    if (route_units && route_stats) {
      atomicAdd(&route_stats[0], 1ull);
      atomicAdd(&route_stats[1], (unsigned long long)r);
    }
  }
  __syncthreads();
  if (s_route) {
    // window-major decode: the list summed into w_dense, then max |w^|
    for (uint32_t i = tid; i < n_q; i += kPlanThreads) {
      const uint32_t key = q_key[i];
      const float wv = q_w[i];
      if (key < ix.n_keys && wv != 0.0f) atomicAdd(&w_dense[key], wv);
    }
    __syncthreads();  // the block's atomics are visible to the block
    uint32_t m = 0;
    for (uint32_t i = tid; i < n_q; i += kPlanThreads) {
      const uint32_t key = q_key[i];
      if (key < ix.n_keys) m = max(m, __float_as_uint(__ldcg(w_dense + key)) & 0x7FFFFFFFu);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) s_m[wid] = m;
    __syncthreads();
    if (tid == 0) {
      uint32_t mm = 0;
      for (int q = 0; q < kPlanThreads / 32; q++) mm = max(mm, s_m[q]);
      if (mm >= 0x7F800000u) atomicOr(&ctrl->flags, DEVERR_RANGE);
      ctrl->pad = mm >= 0x7F800000u ? 0u : mm;
      ctrl->total_units = 0;
      ctrl->n_work = 0;
      ctrl->route = kRouteWindow | kRouteSummed;
    }
    return;
  }
  // pass 2: the non-empty entries, in order, at their first unit
  for (uint32_t p = p0; p < p1; p++) {
    uint32_t key, g;
    float wv;
    const unsigned long long u = plan_entry(ix, q_key, q_w, n_q, p, key, g, wv);
    if (!u) continue;
    WorkEntry we;
    we.seg_g = off_u | ((unsigned long long)g << 56);
    we.blk0 = ix.keys[g][key];
    we.w = wv;
    work[off_n] = we;
    off_u += u;
    off_n++;
  }
  if (tid == 0) {
    ctrl->total_units = all_u;
    ctrl->n_work = all_n;
    ctrl->route = 0;
  }
}

// Decode + scatter (Algorithm 2 inner loop): for each block (g, b) of a
// query key, ad = header << 8 | byte for every real slot (slot 0, or a
// non-zero byte), wide[ad] += w^.
//
// Load balance (merge-based, after the load-balancing search of the
// moderngpu library cited in Sec. 3.4): the units are split evenly over the
// CTAs; a CTA finds the entry holding its first unit with a 256-ary search
// over the entry offsets, then walks tile by tile, staging each tile's
// entries (at most one per unit) in shared memory, where every thread finds
// its unit's entry by binary search.
constexpr unsigned long long kSegMask = 0x00FFFFFFFFFFFFFFull;

__global__ void __launch_bounds__(kWideThreads) k_wide_scatter(
    IndexView ix, const WorkEntry *__restrict__ work, const Ctrl *__restrict__ ctrl,
    float *__restrict__ wide, const uint32_t *__restrict__ q_key, const float *__restrict__ q_w,
    uint32_t n_q, float *__restrict__ w_dense) {
  __shared__ unsigned long long s_seg[kWideTile + 1];
  __shared__ uint32_t s_blk[kWideTile + 1];
  __shared__ float s_w[kWideTile + 1];
  __shared__ uint32_t s_next;
  if (ctrl->route) {  // window-major decode chosen: only sum the list into a dense w^
    if (ctrl->route & kRouteSummed) return;  // k_wide_plan did
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_q;
         i += gridDim.x * blockDim.x) {
      const uint32_t key = q_key[i];  // keys >= n_keys were flagged by k_wide_lens
      if (key < ix.n_keys && q_w[i] != 0.0f) atomicAdd(&w_dense[key], q_w[i]);
    }
    return;
  }
  const unsigned long long total = ctrl->total_units;
  const uint32_t n_work = ctrl->n_work;
  const unsigned long long n_tiles = (total + kWideTile - 1) / kWideTile;
  const unsigned long long tpc = (n_tiles + gridDim.x - 1) / gridDim.x;
  const unsigned long long T0 = blockIdx.x * tpc;
  const unsigned long long T1 = min(n_tiles, T0 + tpc);
  if (T0 >= T1) return;
  // 256-ary search: last entry whose first unit is <= T0 * tile.
  const unsigned long long target = T0 * kWideTile;
  uint32_t lo = 0, hi = n_work;  // invariant: seg(lo) <= target, answer in [lo, hi)
  while (hi - lo > 1) {
    const uint32_t stride = (hi - lo + kWideThreads - 1) / kWideThreads;
    const uint32_t pos = lo + threadIdx.x * stride;
    const bool le = pos < hi && (work[pos].seg_g & kSegMask) <= target;
    const uint32_t cnt = __syncthreads_count(le);
    lo = lo + (cnt - 1) * stride;
    hi = min(hi, lo + stride);
  }
  uint32_t e_cur = lo;
  for (unsigned long long T = T0; T < T1; T++) {
    const unsigned long long t0 = T * kWideTile;
    const unsigned long long t1 = min(t0 + (unsigned long long)kWideTile, total);
    const uint32_t ne = min((uint32_t)kWideTile + 1, n_work - e_cur);
    for (uint32_t e = threadIdx.x; e < ne; e += kWideThreads) {
      const WorkEntry we = work[e_cur + e];
      s_seg[e] = we.seg_g;
      s_blk[e] = we.blk0;
      s_w[e] = we.w;
    }
    __syncthreads();
    for (unsigned long long t = t0 + threadIdx.x; t < t1; t += kWideThreads) {
      uint32_t a = 0, b2 = ne;  // last local entry whose first unit is <= t
      while (b2 - a > 1) {
        const uint32_t mid = (a + b2) >> 1;
        if ((s_seg[mid] & kSegMask) <= t) a = mid; else b2 = mid;
      }
      const unsigned long long sg = s_seg[a];
      const uint32_t g = (uint32_t)(sg >> 56);
      const uint32_t u = (uint32_t)(t - (sg & kSegMask));
      const uint32_t us = unit_shift(g);
      const uint32_t b = s_blk[a] + (u >> us);
      const float w = s_w[a];
      const uint32_t base = ix.header[g][b] << 8;
      if (g >= 2) {
        const uint32_t wi = u & ((1u << us) - 1u);
        const uint32_t word =
            reinterpret_cast<const uint32_t *>(ix.values[g])[((uint64_t)b << us) + wi];
#pragma unroll
        for (int q = 0; q < 4; q++) {
          const uint32_t l = (word >> (8 * q)) & 255u;
          if ((wi == 0 && q == 0) || l != 0) atomicAdd(&wide[base | l], w);
        }
      } else if (g == 1) {
        const uint16_t hw = reinterpret_cast<const uint16_t *>(ix.values[1])[b];
        atomicAdd(&wide[base | (hw & 255u)], w);
        if (hw >> 8) atomicAdd(&wide[base | (hw >> 8)], w);
      } else {
        atomicAdd(&wide[base | ix.values[0][b]], w);
      }
    }
    if (threadIdx.x == 0) {
      uint32_t a = 0, b2 = ne;  // entry holding unit t1 (first unit of the next tile)
      while (b2 - a > 1) {
        const uint32_t mid = (a + b2) >> 1;
        if ((s_seg[mid] & kSegMask) <= t1) a = mid; else b2 = mid;
      }
      s_next = a;
    }
    __syncthreads();
    e_cur += s_next;
    __syncthreads();
  }
}

// =====================================================================
// Streaming inner product + wide add + per-CTA top-K
// =====================================================================
enum { MODE_TOPK = 0, MODE_ALL = 1 };

constexpr int kScanThreads = 256;
constexpr int kScanWarps = kScanThreads / 32;

struct ScanArgs {
  const void *emb;          // [N][D] of Elt
  const float *scale;       // [N] (FP8) or nullptr
  const float *h_u;         // [D]
  const float *wide;        // [N] or nullptr
  const uint64_t *filter;   // bitmap or nullptr
  uint32_t n_ads;
  uint32_t k;               // candidates to keep
  uint32_t cap;             // candidate buffer capacity (per buffer)
  uint32_t stages;
  uint64_t *cand_out;       // [grid * k] global candidates
  Ctrl *ctrl;
  float *all_out;           // MODE_ALL: [N] scores
};

template <typename Elt, int D>
struct ScanShape {
  static constexpr int kRowBytes = D * EltTraits<Elt>::kBytes;
  static constexpr int kTileRows = (32768 / kRowBytes) < 256 ? (32768 / kRowBytes) : 256;
  static constexpr int kStageBytes = kTileRows * kRowBytes;
  static constexpr int kLPR = D / EltTraits<Elt>::kVec;  // lanes per row
  static constexpr int kRowsPerIter = 32 / kLPR;
  static constexpr int kRowsPerWarp = kTileRows / kScanWarps;
  static_assert(kLPR >= 1 && kLPR <= 32, "unsupported row width");
  static_assert(kRowsPerWarp % kRowsPerIter == 0, "tile split");
  static_assert(kRowsPerWarp <= 32, "one prefetched row per lane");
};

template <typename Elt, int D, int MODE>
__global__ void __launch_bounds__(kScanThreads) k_scan_topk(ScanArgs a) {
  using Sh = ScanShape<Elt, D>;
  using Tr = EltTraits<Elt>;
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ uint64_t s_bar[8];
  __shared__ uint32_t s_hist[256];
  __shared__ uint32_t s_misc[8];
  __shared__ uint32_t s_n, s_n2, s_status, s_fail_j;
  __shared__ unsigned long long s_thr;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t S = a.stages;
  uint8_t *stage0 = smem;
  uint64_t *cand = reinterpret_cast<uint64_t *>(smem + (size_t)S * Sh::kStageBytes);
  uint64_t *cand2 = cand + a.cap;

  const uint32_t n_tiles = (a.n_ads + Sh::kTileRows - 1) / Sh::kTileRows;
  const uint32_t my_tiles =
      blockIdx.x < n_tiles ? (n_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;

  if (tid == 0) {
    for (uint32_t s = 0; s < S; s++) mbar_init(&s_bar[s], 1);
    fence_mbar_init();
    s_n = 0;
    s_status = 0;
    s_thr = 0ull;
  }
  __syncthreads();
  auto issue = [&](uint32_t j) {  // tile j of this CTA into stage j % S
    const uint32_t tile = blockIdx.x + j * gridDim.x;
    const uint32_t row0 = tile * Sh::kTileRows;
    const uint32_t rows = min((uint32_t)Sh::kTileRows, a.n_ads - row0);
    const uint32_t bytes = rows * Sh::kRowBytes;
    uint64_t *bar = &s_bar[j % S];
    mbar_arrive_expect_tx(bar, bytes);
    bulk_g2s(stage0 + (size_t)(j % S) * Sh::kStageBytes,
             reinterpret_cast<const uint8_t *>(a.emb) + (uint64_t)row0 * Sh::kRowBytes, bytes,
             bar);
  };
  if (tid == 0)
    for (uint32_t j = 0; j < S && j < my_tiles; j++) issue(j);

  // this lane's slice of h_u
  float hreg[Tr::kVec];
  const int col = (lane % Sh::kLPR) * Tr::kVec;
#pragma unroll
  for (int e = 0; e < Tr::kVec; e++) hreg[e] = a.h_u[col + e];

  uint64_t thr = 0;
  for (uint32_t j = 0; j < my_tiles; j++) {
    const uint32_t s = j % S, parity = (j / S) & 1u;
    const uint32_t tile = blockIdx.x + j * gridDim.x;
    const uint32_t row0 = tile * Sh::kTileRows;
    const uint32_t rows = min((uint32_t)Sh::kTileRows, a.n_ads - row0);
    // Per-row side inputs of this warp's rows, one row per lane, fetched before
    // the wait so their latency overlaps the tile's arrival.
    float pre_w = 0.f, pre_s = 1.f;
    bool pre_f = true;
    {
      const uint32_t rl = warp * Sh::kRowsPerWarp + lane;
      if (lane < Sh::kRowsPerWarp && rl < rows) {
        const uint32_t ad = row0 + rl;
        if (a.wide) pre_w = a.wide[ad];
        if (a.scale) pre_s = a.scale[ad];
        if (a.filter) pre_f = (a.filter[ad >> 6] >> (ad & 63)) & 1ull;
      }
    }
    if (tid == 0) {
      if (!mbar_wait_bounded(&s_bar[s], parity, kWaitTimeoutNs)) {
        s_status = 1;
        s_fail_j = j;
      }
    }
    __syncthreads();
    if (s_status) break;
    mbar_try_wait(&s_bar[s], parity);  // per-thread acquire of the completed phase
    const uint8_t *st = stage0 + (size_t)s * Sh::kStageBytes;
    if (MODE == MODE_TOPK) {
      thr = s_thr;
    }
#pragma unroll 2
    for (int it = 0; it < Sh::kRowsPerWarp / Sh::kRowsPerIter; it++) {
      const uint32_t rw = it * Sh::kRowsPerIter + lane / Sh::kLPR;  // row within the warp's rows
      const uint32_t r = warp * Sh::kRowsPerWarp + rw;
      float dot = 0.f;
      if (r < rows) {
        const uint4 v = *reinterpret_cast<const uint4 *>(st + (size_t)r * Sh::kRowBytes +
                                                         (lane % Sh::kLPR) * 16);
        float f[Tr::kVec];
        Tr::load(v, f);
#pragma unroll
        for (int e = 0; e < Tr::kVec; e++) dot = fmaf(hreg[e], f[e], dot);
      }
#pragma unroll
      for (int o = Sh::kLPR / 2; o >= 1; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
      const float rw_w = __shfl_sync(0xffffffffu, pre_w, rw);
      const float rw_s = __shfl_sync(0xffffffffu, pre_s, rw);
      const bool rw_f = __shfl_sync(0xffffffffu, (int)pre_f, rw) != 0;
      const bool leader = (lane % Sh::kLPR) == 0 && r < rows;
      const uint32_t ad = row0 + r;
      float score = 0.f;
      if (leader) {
        score = dot;
        if (a.scale) score *= rw_s;
        if (a.wide) score += rw_w;
      }
      if (MODE == MODE_ALL) {
        if (leader) a.all_out[ad] = score;
      } else {
        bool keep = leader && rw_f;
        uint64_t key = 0;
        if (keep) {
          key = make_key(score, ad);
          keep = key >= thr;
        }
        const uint32_t pos = warp_append(keep, &s_n);
        if (keep) cand[pos] = key;
      }
    }
    __syncthreads();  // stage s fully consumed; candidate appends visible
    if (tid == 0 && j + S < my_tiles) issue(j + S);
    if (MODE == MODE_TOPK) {
      if (s_n + Sh::kTileRows > a.cap) {
        const uint32_t n = s_n;
        const uint64_t T = cta_radix_select<kScanThreads>(cand, n, a.k, s_hist, s_misc);
        if (tid == 0) s_n2 = 0;
        __syncthreads();
        for (uint32_t base = 0; base < n; base += kScanThreads) {
          const uint32_t i = base + tid;
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
          unsigned long long g = atomicMax(&a.ctrl->thr, (unsigned long long)T);
          s_thr = max((unsigned long long)T, max(g, (unsigned long long)s_thr));
        }
        __syncthreads();
      } else if (tid == 0 && (j & 7) == 7) {
        const unsigned long long g = *((volatile unsigned long long *)&a.ctrl->thr);
        if (g > s_thr) s_thr = g;
      }
    }
  }
  if (s_status) {
    // A stage never completed: record it, drain what is in flight, leave.
    if (tid == 0) {
      atomicOr(&a.ctrl->flags, DEVERR_TIMEOUT);
      // loads issued and not consumed: tiles s_fail_j .. s_fail_j + S - 1
      for (uint32_t q = s_fail_j; q < s_fail_j + S && q < my_tiles; q++)
        mbar_wait_bounded(&s_bar[q % S], (q / S) & 1u, kWaitTimeoutNs / 4);
    }
    return;
  }
  if (MODE == MODE_TOPK) {
    __syncthreads();
    uint32_t n = s_n;
    uint64_t T = 0;
    if (n > a.k) {
      T = cta_radix_select<kScanThreads>(cand, n, a.k, s_hist, s_misc);
    }
    if (tid == 0) {
      const unsigned long long g = *((volatile unsigned long long *)&a.ctrl->thr);
      s_thr = max(max((unsigned long long)T, (unsigned long long)s_thr), g);
      if (n > a.k) atomicMax(&a.ctrl->thr, (unsigned long long)T);
    }
    __syncthreads();
    const uint64_t fin = s_thr;
    for (uint32_t base = 0; base < n; base += kScanThreads) {
      const uint32_t i = base + tid;
      const uint64_t x = i < n ? cand[i] : 0ull;
      const bool kp = i < n && x >= fin;
      const uint32_t pos = warp_append(kp, &a.ctrl->n_cand);
      if (kp) a.cand_out[pos] = x;
    }
  }
}

// =====================================================================
// Final selection: top-K of the surviving candidates, sorted
// =====================================================================
constexpr int kFinalThreads = 1024;

__device__ void bitonic_sort_desc(uint64_t *v, uint32_t n_pow2) {
  for (uint32_t size = 2; size <= n_pow2; size <<= 1) {
    for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
      __syncthreads();
      for (uint32_t i = threadIdx.x; i < n_pow2 / 2; i += blockDim.x) {
        const uint32_t lo = 2 * i - (i & (stride - 1));
        const uint32_t hi = lo + stride;
        const bool desc = ((lo & size) == 0);
        const uint64_t x = v[lo], y = v[hi];
        if ((x < y) == desc) {
          v[lo] = y;
          v[hi] = x;
        }
      }
    }
  }
  __syncthreads();
}

// Selects the best min(k, n) keys among n (global memory) and writes k_out
// ids/scores sorted descending, padded with (0xFFFFFFFF, -inf), or the keys
// themselves in no particular order, padded with zero keys.  Dynamic shared memory: 8 * (pow2(min(k, n)) + buf_cap)
// bytes; when n <= buf_cap the keys are read from global memory once and the
// radix select runs on the shared copy, otherwise on the global keys.
// Waits (pdl_wait) for the kernel before it in the stream.
__global__ void __launch_bounds__(kFinalThreads) k_final_select(
    const uint64_t *__restrict__ keys, const Ctrl *__restrict__ ctrl, uint32_t n_fixed,
    uint32_t k, uint32_t k_out, uint32_t *__restrict__ out_ids, float *__restrict__ out_scores,
    uint64_t *__restrict__ out_keys, uint32_t buf_cap) {
  extern __shared__ __align__(16) uint64_t s_v[];
  __shared__ uint32_t s_hist[256];
  __shared__ uint32_t s_misc[8];
  __shared__ uint32_t s_cnt;
  pdl_wait();
  const uint32_t n = ctrl ? ctrl->n_cand : n_fixed;
  const uint32_t take = min(n, k);
  uint32_t p2 = 1;
  while (p2 < take) p2 <<= 1;
  const uint64_t *src = keys;
  if (n <= buf_cap) {  // one read of the keys, then everything in shared memory
    uint64_t *s_buf = s_v + p2;
    for (uint32_t i = threadIdx.x; i < n; i += kFinalThreads) s_buf[i] = keys[i];
    __syncthreads();
    src = s_buf;
  }
  uint64_t T = 0;
  if (n > k) T = cta_radix_select<kFinalThreads>(src, n, k, s_hist, s_misc);
  if (threadIdx.x == 0) s_cnt = 0;
  __syncthreads();
  for (uint32_t base = 0; base < n; base += kFinalThreads) {
    const uint32_t i = base + threadIdx.x;
    const uint64_t x = i < n ? src[i] : 0ull;
    const bool kp = i < n && x >= T;
    const uint32_t pos = warp_append(kp, &s_cnt);
    if (kp && pos < p2) s_v[pos] = x;
  }
  __syncthreads();
  for (uint32_t i = take + threadIdx.x; i < p2; i += kFinalThreads) s_v[i] = 0ull;
  if (out_keys) {  // keys for a later stage (FP32 rescoring): any order will do
    __syncthreads();
  } else {
    bitonic_sort_desc(s_v, p2);
  }
  for (uint32_t i = threadIdx.x; i < k_out; i += kFinalThreads) {
    if (out_keys) {
      out_keys[i] = i < take ? s_v[i] : 0ull;
    } else if (i < take) {
      out_ids[i] = key_id(s_v[i]);
      out_scores[i] = key_score(s_v[i]);
    } else {
      out_ids[i] = 0xFFFFFFFFu;
      out_scores[i] = -INFINITY;
    }
  }
}

// Shared-memory keys k_final_select buffers beyond its pow2(k) sort area.
constexpr uint32_t kFinalBufKeys = 16384;
constexpr size_t kFinalMaxSmem = (8192 + kFinalBufKeys) * 8;  // largest k is 8192
static size_t final_smem(uint32_t p2) { return ((size_t)p2 + kFinalBufKeys) * 8; }

// FP32 rescoring of candidate keys: s = <h_u, h_a (FP32 copy)> + wide[a].
// One warp per candidate; D <= 128.
__global__ void k_rescore(const uint64_t *__restrict__ cand, uint32_t n,
                          const float *__restrict__ emb, uint32_t d, const float *__restrict__ h_u,
                          const float *__restrict__ wide, uint64_t *__restrict__ out) {
  const int lane = threadIdx.x & 31;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t c = warp; c < n; c += nw) {
    const uint64_t key = cand[c];
    if (key == 0ull) {  // padding from the first selection
      if (lane == 0) out[c] = 0ull;
      continue;
    }
    const uint32_t ad = key_id(key);
    float dot = 0.f;
    for (uint32_t t = lane; t < d; t += 32) dot = fmaf(h_u[t], emb[(uint64_t)ad * d + t], dot);
    for (int o = 16; o; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
    if (lane == 0) out[c] = make_key(dot + (wide ? wide[ad] : 0.f), ad);
  }
}

// =====================================================================
// Host side
// =====================================================================
static uint32_t pow2_at_least(uint32_t x) {
  uint32_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

struct ScanPlan {
  int grid = 0;
  uint32_t stages = 0, cap = 0;
  size_t smem = 0;
};

template <typename Elt, int D>
static ScanPlan plan_scan(const ebr_index *ix, uint32_t k) {
  using Sh = ScanShape<Elt, D>;
  ScanPlan p;
  p.cap = k + std::max<uint32_t>(k, 2 * Sh::kTileRows);
  p.cap = (p.cap + 255) / 256 * 256;
  const size_t cand_bytes = (size_t)2 * p.cap * 8;
  const size_t budget = 200 * 1024;
  uint32_t st = 4;
  while (st > 2 && cand_bytes + (size_t)st * Sh::kStageBytes > budget) st--;
  p.stages = st;
  p.smem = cand_bytes + (size_t)st * Sh::kStageBytes;
  const uint32_t n_tiles = (ix->n_ads + Sh::kTileRows - 1) / Sh::kTileRows;
  p.grid = std::min<int>(ix->num_sms, (int)n_tiles);
  if (p.grid < 1) p.grid = 1;
  return p;
}

template <typename Elt, int D, int MODE>
static int launch_scan_t(const ebr_index *ix, ScanArgs a, cudaStream_t st) {
  ScanPlan p = plan_scan<Elt, D>(ix, std::max<uint32_t>(a.k, 1));
  a.cap = p.cap;
  a.stages = p.stages;
  auto kern = k_scan_topk<Elt, D, MODE>;
  EBR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)p.smem));
  kern<<<p.grid, kScanThreads, p.smem, st>>>(a);
  EBR_CUDA_TRY(cudaGetLastError());
  return EBR_OK;
}

template <typename Elt, int MODE>
static int launch_scan_d(const ebr_index *ix, const ScanArgs &a, cudaStream_t st) {
  switch (ix->d) {
    case 4: if constexpr (EltTraits<Elt>::kVec <= 4) return launch_scan_t<Elt, 4, MODE>(ix, a, st); break;
    case 8: if constexpr (EltTraits<Elt>::kVec <= 8) return launch_scan_t<Elt, 8, MODE>(ix, a, st); break;
    case 16: return launch_scan_t<Elt, 16, MODE>(ix, a, st);
    case 32: return launch_scan_t<Elt, 32, MODE>(ix, a, st);
    case 64: return launch_scan_t<Elt, 64, MODE>(ix, a, st);
    case 128: return launch_scan_t<Elt, 128, MODE>(ix, a, st);
  }
  set_error("embedding dimension %u unsupported for this dtype", ix->d);
  return EBR_EINVAL;
}

template <int MODE>
static int launch_scan(const ebr_index *ix, const ScanArgs &a, cudaStream_t st) {
  if (ix->dtype == EBR_F32) return launch_scan_d<float, MODE>(ix, a, st);
  if (ix->dtype == EBR_BF16) return launch_scan_d<Bf16Tag, MODE>(ix, a, st);
  return launch_scan_d<Fp8Tag, MODE>(ix, a, st);
}

// ----------------------------------------------------------- workspace
int ws_prepare_one(ebr_index *ix, uint32_t n_q, uint32_t kcap);
static int ws_prepare(ebr_index *ix, uint32_t n_q, uint32_t kcap) {
  return ws_prepare_one(ix, n_q, kcap);
}
int ws_prepare_one(ebr_index *ix, uint32_t n_q, uint32_t kcap) {
  Workspace &w = ix->ws;
  EBR_TRY(dev_reserve(w.wide, (size_t)ix->n_ads * 4));
  EBR_TRY(dev_reserve(w.w_dense, (size_t)ix->n_keys * 4));
  EBR_TRY(dev_reserve(w.wq, (size_t)ix->n_keys * 4));
  const size_t entries = (size_t)kGroups * n_q + 1;
  EBR_TRY(dev_reserve(w.lens, entries * sizeof(LenPair)));
  EBR_TRY(dev_reserve(w.scan, entries * sizeof(LenPair)));
  EBR_TRY(dev_reserve(w.work, entries * sizeof(WorkEntry)));
  EBR_TRY(dev_reserve(w.scan_tmp, prims::scan_scratch(entries) * sizeof(LenPair) + 256));
  EBR_TRY(dev_reserve(w.cand, ((size_t)ix->num_sms * kMaxCtasPerSm + 1) * kcap * 8 +
                                  2 * (size_t)kcap * 8));
  EBR_TRY(dev_reserve(w.ctrl, kCtrlBytes + kHistWords * 4));
  if (!w.route_stats.p) {  // lifetime counters, zeroed once
    EBR_TRY(dev_reserve(w.route_stats, 16));
    EBR_CUDA_TRY(cudaMemset(w.route_stats.p, 0, 16));
  }
  return EBR_OK;
}

static int launch_grid(uint64_t n, int threads, int cap) {
  uint64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > (uint64_t)cap) b = cap;
  return (int)b;
}

// Wide term of one request into ws.wide (zeroed first): Algorithm 2.
// w_dense != nullptr (a sparse list, zeroed w_dense): the traversal is chosen
// on the device; when it is the window-major decode, the list is summed into
// w_dense instead of being scattered.
// *planned (if given): whether the one-CTA plan ran, which also leaves max
// |w^| in ctrl->pad when it chose the window-major decode.
static int run_wide(ebr_index *ix, const uint32_t *q_key, const float *q_w, uint32_t n_q,
                    Ctrl *ctrl, cudaStream_t st, float *w_dense = nullptr,
                    bool *planned = nullptr) {
  Workspace &w = ix->ws;
  if (planned) *planned = false;
  EBR_CUDA_TRY(cudaMemsetAsync(w.wide.p, 0, (size_t)ix->n_ads * 4, st));
  if (n_q == 0) return EBR_OK;
  IndexView iv = index_view(ix);
  const uint64_t entries = (uint64_t)kGroups * n_q + 1;
  if (q_key && entries - 1 <= kPlanMaxEntries) {
    k_wide_plan<<<1, kPlanThreads, 0, st>>>(iv, q_key, q_w, n_q, (WorkEntry *)w.work.p, ctrl,
                                            w_dense ? index_units(ix) : 0ull,
                                            (unsigned long long *)w.route_stats.p, w_dense);
    EBR_CUDA_TRY(cudaGetLastError());
    k_wide_scatter<<<ix->num_sms * 8, kWideThreads, 0, st>>>(iv, (const WorkEntry *)w.work.p,
                                                             ctrl, (float *)w.wide.p, q_key, q_w,
                                                             n_q, w_dense);
    EBR_CUDA_TRY(cudaGetLastError());
    if (planned) *planned = true;
    return EBR_OK;
  }
  k_wide_lens<<<launch_grid(entries, 256, 65535), 256, 0, st>>>(
      iv, q_key, q_w, n_q, (LenPair *)w.lens.p, &ctrl->flags);
  EBR_CUDA_TRY(cudaGetLastError());
  EBR_TRY((prims::scan<LenPair, LenPairSum, false>((const LenPair *)w.lens.p, (LenPair *)w.scan.p,
                                                   entries, LenPairSum(), LenPair{0, 0, 0},
                                                   (LenPair *)w.scan_tmp.p, nullptr, st)));
  k_wide_compact<<<launch_grid(entries, 256, 65535), 256, 0, st>>>(
      iv, q_key, q_w, n_q, (const LenPair *)w.lens.p, (const LenPair *)w.scan.p,
      (WorkEntry *)w.work.p, ctrl, w_dense ? index_units(ix) : 0ull,
      (unsigned long long *)w.route_stats.p);
  EBR_CUDA_TRY(cudaGetLastError());
  k_wide_scatter<<<ix->num_sms * 8, kWideThreads, 0, st>>>(iv, (const WorkEntry *)w.work.p,
                                                           ctrl, (float *)w.wide.p, q_key, q_w,
                                                           n_q, w_dense);
  EBR_CUDA_TRY(cudaGetLastError());
  return EBR_OK;
}

// w_hat transposed: wT[key][b] for b < Bp (zero for padding users b >= batch).
// User b's field values are users[base[b] + uptr[b][i] .. base[b] +
// uptr[b][i+1]) for field i (MULTI; offsets already checked); without MULTI
// every field holds one value, users[b * f_u + i].  Pairs are summed in pair
// order and a field's values in their order, as in the single-request
// expansion, so both give the same FP32 w^.
template <bool MULTI>
__global__ void k_expand_T(CrossView cv, const uint32_t *__restrict__ users,
                           const uint32_t *__restrict__ uptr, const uint32_t *__restrict__ base,
                           uint32_t batch, uint32_t Bp, float *__restrict__ wT,
                           uint32_t *__restrict__ flags, const uint32_t *__restrict__ batch_dev) {
  extern __shared__ uint32_t s_off2[];
  if (batch_dev) {  // a device-side loop: this wave's users (none: nothing to expand)
    batch = min(*batch_dev, batch);
    if (batch == 0) return;
  }
  for (uint32_t j = threadIdx.x; j <= cv.f_a; j += blockDim.x) s_off2[j] = cv.key_off[j];
  __syncthreads();
  const uint64_t total = (uint64_t)cv.n_keys * Bp;
  uint32_t bad = 0;
  for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total;
       t += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t key = (uint32_t)(t / Bp), b = (uint32_t)(t % Bp);
    float acc = 0.f;
    if (b < batch) {
      uint32_t lo = 0, hi = cv.f_a;
      while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (s_off2[mid] <= key) lo = mid; else hi = mid;
      }
      const uint32_t j = lo, v = key - s_off2[j];
      const uint32_t *up = MULTI ? uptr + (uint64_t)b * (cv.f_u + 1) : nullptr;
      const uint32_t ub = MULTI ? __ldg(base + b) : b * cv.f_u;
      for (uint32_t q = cv.pair_ptr[j]; q < cv.pair_ptr[j + 1]; q++) {
        const uint32_t p = cv.pair_of[q];
        const uint32_t i = cv.pair_user[p];
        const uint32_t r0 = MULTI ? ub + __ldg(up + i) : ub + i;
        const uint32_t r1 = MULTI ? ub + __ldg(up + i + 1) : r0 + 1;
        for (uint32_t r = r0; r < r1; r++) {
          const uint32_t u = __ldg(users + r);
          if (u >= cv.vocab_u[i]) { bad |= DEVERR_BAD_USER; continue; }
          float w;
          if (cv.hashed) {
            const uint64_t x = ((uint64_t)p << 40) | ((uint64_t)u << 20) | (uint64_t)v;
            w = cv.table[splitmix64(x) & ((1ull << cv.hash_bits) - 1ull)];
          } else {
            const uint64_t off = ((uint64_t)cv.w_hi[p] << 32) | cv.w_lo[p];
            w = cv.table[off + (uint64_t)u * cv.vocab_a[j] + v];
          }
          acc += w;
        }
      }
    }
    wT[t] = acc;
  }
  if (bad) atomicOr(flags, bad);
}

int expand_transposed(const ebr_cross *c, const uint32_t *users, const uint32_t *uptr,
                      const uint32_t *base, uint32_t batch, uint32_t Bp, float *wT,
                      uint32_t *flags, cudaStream_t st, const uint32_t *batch_dev) {
  CrossView cv = cross_view(c);
  const uint64_t total = (uint64_t)cv.n_keys * Bp;
  uint64_t blocks = (total + 255) / 256;
  if (blocks > 65535) blocks = 65535;
  const size_t smem = (c->f_a + 1) * 4;
  if (uptr)
    k_expand_T<true><<<(int)blocks, 256, smem, st>>>(cv, users, uptr, base, batch, Bp, wT, flags,
                                                     batch_dev);
  else
    k_expand_T<false><<<(int)blocks, 256, smem, st>>>(cv, users, nullptr, nullptr, batch, Bp, wT,
                                                      flags, batch_dev);
  EBR_CUDA_TRY(cudaGetLastError());
  return EBR_OK;
}

static int expand_into(const ebr_cross *c, const uint32_t *users, uint32_t batch, float *w_hat,
                       uint32_t *flags, cudaStream_t st, uint32_t *wmax = nullptr,
                       const uint32_t *user_ptr = nullptr, uint32_t n_uv = 0,
                       PackOut po = PackOut{nullptr, nullptr, 0, 0, 0.f}) {
  CrossView cv = cross_view(c);
  const uint64_t total = (uint64_t)batch * cv.n_keys;
  const size_t smem =
      ((size_t)2 * (c->f_a + 1) + 3 * (size_t)c->n_pairs + (size_t)c->f_u + 1) * 4;
  if (user_ptr && batch != 1) {
    set_error("query expansion: multi-valued user fields are expanded one user at a time");
    return EBR_EINVAL;
  }
  if (smem > 48 * 1024)
    EBR_CUDA_TRY(cudaFuncSetAttribute(k_expand, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)std::min<size_t>(smem, 200 * 1024)));
  if (smem > 200 * 1024) {
    set_error("query expansion: %u cross pairs exceed the staging area", c->n_pairs);
    return EBR_EINVAL;
  }
  k_expand<<<launch_grid(total, 256, 65535), 256, smem, st>>>(cv, users, batch, w_hat, flags,
                                                              wmax, user_ptr, n_uv, po);
  EBR_CUDA_TRY(cudaGetLastError());
  return EBR_OK;
}

// One request, all pointers device-resident.  ids/scores get kmax entries.
// Profiling events of one request (recorded only when enabled).
struct ProfMarks {
  ebr_index *ix;
  std::array<cudaEvent_t, 5> ev;
  bool on;
  ProfMarks(ebr_index *x, cudaStream_t st) : ix(x), on(x->prof) {
    if (!on) return;
    if (!ix->prof_pool.empty()) {
      ev = ix->prof_pool.back();
      ix->prof_pool.pop_back();
    } else {
      for (auto &e : ev) cudaEventCreate(&e);
    }
    cudaEventRecord(ev[0], st);
  }
  void mark(int i, cudaStream_t st) {
    if (on) cudaEventRecord(ev[i], st);
  }
  void done() {
    if (on) ix->prof_pending.push_back(ev);
  }
};

// One request, all pointers device-resident.  ids/scores get kmax entries.
int query_one(const ebr_index *cix, const ebr_cross *cross, const ebr_query &q, uint32_t *ids,
              float *scores, uint32_t kmax, cudaStream_t st) {
  ebr_index *ix = const_cast<ebr_index *>(cix);
  Workspace &w = ix->ws;
  Ctrl *ctrl = (Ctrl *)w.ctrl.p;
  const bool quant = ix->dtype != EBR_F32;
  const uint32_t k = q.k;
  const uint32_t kscan = quant ? std::min<uint32_t>(k * ix->rescore_mult, ix->n_ads) : k;
  static bool attr_set = false;  // per process; the attribute applies to every device
  if (!attr_set) {
    EBR_CUDA_TRY(cudaFuncSetAttribute(k_final_select, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)kFinalMaxSmem));
    attr_set = true;
  }
  ProfMarks pm(ix, st);
  EBR_CUDA_TRY(cudaMemsetAsync(ctrl, 0, kCtrlBytes + kHistWords * 4, st));  // + histogram
  const uint32_t *q_key = q.q_key;
  const float *q_w = q.q_w;
  uint32_t n_q = q.n_q;
  bool packed = false;  // the expansion also wrote the fused scan's packed terms
  if (q.user_vals) {
    // single-valued user fields: the packed terms' exponent follows from the
    // cross model's bound on |w^|, so the expansion writes them directly;
    // otherwise the fused scan's launch packs w^ after its max |w^|
    PackOut po{nullptr, nullptr, 0, 0, 0.f};
    const float wb = cross->wbound * 1.001f;
    if (!q.user_ptr && wb < 3.0e38f && !(q.flags & EBR_QF_KEY_MAJOR)) {
      const uint32_t mk = std::max<uint32_t>(ix->max_keys_per_ad, 1);
      po = PackOut{(uint32_t *)w.wq.p, &ctrl->fx, fix_exponent(wb, mk), class_shift(mk), wb};
      packed = true;
    }
    EBR_TRY(expand_into(cross, q.user_vals, 1, (float *)w.w_dense.p, &ctrl->flags, st,
                        &ctrl->pad, q.user_ptr, q.n_user_vals, po));  // + max |w^|
    ix->launches += 1;
    q_key = nullptr;
    q_w = (const float *)w.w_dense.p;
    n_q = ix->n_keys;
  } else if (!q_key) {
    n_q = ix->n_keys;
  } else if ((q.flags & EBR_QF_WINDOW_MAJOR) && !(q.flags & EBR_QF_KEY_MAJOR) &&
             fused_fits(ix, kscan)) {
    EBR_CUDA_TRY(cudaMemsetAsync(w.w_dense.p, 0, (size_t)ix->n_keys * 4, st));
    if (n_q) {
      k_list_to_dense<<<launch_grid(n_q, 256, 1024), 256, 0, st>>>(
          q_key, q_w, n_q, ix->n_keys, (float *)w.w_dense.p, &ctrl->flags);
      EBR_CUDA_TRY(cudaGetLastError());
      ix->launches += 1;
    }
    q_key = nullptr;
    q_w = (const float *)w.w_dense.p;
    n_q = ix->n_keys;
  }
  pm.mark(1, st);
  const bool fused =
      q_key == nullptr && !(q.flags & EBR_QF_KEY_MAJOR) && fused_fits(ix, kscan);
  // the fused scan's per-CTA candidate buffers, when they go to global
  // memory: past the survivors' area (one CTA per SM, kscan each) and
  // before the tail the rescoring path selects into
  uint64_t *cta_cand = (uint64_t *)w.cand.p + (size_t)ix->num_sms * kscan;
  const size_t cand_used = (size_t)ix->num_sms * kscan +
                           2 * (size_t)pow2_at_least(std::max<uint32_t>(kscan, 1));
  const size_t cta_entries = w.cand.bytes / 8 > cand_used ? w.cand.bytes / 8 - cand_used : 0;
  // a sparse list with no traversal forced: chosen on the device by its work
  const bool auto_route = q_key != nullptr && n_q > 0 &&
                          !(q.flags & (EBR_QF_KEY_MAJOR | EBR_QF_WINDOW_MAJOR)) &&
                          fused_fits(ix, kscan);
  if (fused) {
    // dense query: wide term decoded window by window inside the scan
    pm.mark(2, st);
    const bool wmax_ready = q.user_vals != nullptr;  // the expansion reduced max |w^|
    int nl = 0;
    EBR_TRY(launch_fused(ix, q.h_u, q_w, (uint32_t *)w.wq.p, packed, q.filter, kscan,
                         (uint64_t *)w.cand.p, ctrl, nullptr, quant ? (float *)w.wide.p : nullptr,
                         ws_hist(w), ix->num_sms * kMaxCtasPerSm, st, wmax_ready,
                         nullptr, nullptr, &nl, cta_cand, cta_entries));
    ix->launches += nl;  // (k_absmax, k_pack) k_fused_window
  } else {
    float *w_dense = auto_route ? (float *)w.w_dense.p : nullptr;
    if (auto_route) EBR_CUDA_TRY(cudaMemsetAsync(w_dense, 0, (size_t)ix->n_keys * 4, st));
    bool planned = false;
    EBR_TRY(run_wide(ix, q_key, q_w, n_q, ctrl, st, w_dense, &planned));
    if (n_q) {
      // planned: k_wide_plan, k_wide_scatter; else k_wide_lens, the three
      // kernels of the scan of lens, k_wide_compact, k_wide_scatter
      ix->launches += planned ? 2 : 6;
    }
    pm.mark(2, st);
    if (fused_fits(ix, kscan)) {
      // the streaming scan of the fused kernel, adding the wide term that
      // Algorithm 2 has just scattered (no window decoding), or, when the
      // device chose the window-major decode, decoding w_dense's windows
      int nl = 0;
      EBR_TRY(launch_fused(ix, q.h_u, w_dense, (uint32_t *)w.wq.p, false, q.filter, kscan,
                           (uint64_t *)w.cand.p, ctrl, nullptr,
                           auto_route && quant ? (float *)w.wide.p : nullptr,
                           ws_hist(w), ix->num_sms * kMaxCtasPerSm, st,
                           !auto_route || planned, (const float *)w.wide.p,
                           auto_route ? &ctrl->route : nullptr, &nl, cta_cand, cta_entries));
      ix->launches += nl;  // (k_absmax, k_pack) k_fused_window

    } else {
      ScanArgs a;
      memset(&a, 0, sizeof(a));
      a.emb = quant ? ix->emb_q.p : ix->emb_f32.p;
      a.scale = ix->dtype == EBR_FP8E4M3 ? (const float *)ix->emb_scale.p : nullptr;
      a.h_u = q.h_u;
      a.wide = (const float *)w.wide.p;
      a.filter = q.filter;
      a.n_ads = ix->n_ads;
      a.k = kscan;
      a.cand_out = (uint64_t *)w.cand.p;
      a.ctrl = ctrl;
      EBR_TRY(launch_scan<MODE_TOPK>(ix, a, st));
      ix->launches += 1;
    }
  }
  pm.mark(3, st);
  const uint32_t p2 = pow2_at_least(std::max<uint32_t>(kscan, 1));
  if (!quant) {
    EBR_CUDA_TRY(launch_pdl(k_final_select, 1, kFinalThreads, final_smem(p2), st,
                            (const uint64_t *)w.cand.p, (const Ctrl *)ctrl, 0u, k, kmax, ids,
                            scores, (uint64_t *)nullptr, kFinalBufKeys));
    ix->launches += 1;
  } else {
    // R*K candidates -> FP32 rescoring -> K
    const uint64_t *ck = (const uint64_t *)w.cand.p;
    uint64_t *sel = (uint64_t *)w.cand.p + (w.cand.bytes / 8 - 2 * (size_t)p2);
    uint64_t *res = sel + p2;
    EBR_CUDA_TRY(launch_pdl(k_final_select, 1, kFinalThreads, final_smem(p2), st, ck,
                            (const Ctrl *)ctrl, 0u, kscan, kscan, (uint32_t *)nullptr,
                            (float *)nullptr, sel, kFinalBufKeys));
    k_rescore<<<launch_grid((uint64_t)kscan * 32, 256, 4096), 256, 0, st>>>(
        sel, kscan, (const float *)ix->emb_f32.p, ix->d, q.h_u, (const float *)w.wide.p, res);
    EBR_CUDA_TRY(cudaGetLastError());
    const uint32_t p2k = pow2_at_least(std::max<uint32_t>(std::min(k, kscan), 1));
    k_final_select<<<1, kFinalThreads, final_smem(p2k), st>>>(res, nullptr, kscan, k, kmax, ids,
                                                               scores, nullptr, kFinalBufKeys);
    EBR_CUDA_TRY(cudaGetLastError());
    ix->launches += 3;
  }
  pm.mark(4, st);
  pm.done();
  return EBR_OK;
}

}  // namespace ebr

namespace ebr {
// Largest |w| (FP32 bits) of each table segment: segment y covers
// table[off[y] .. off[y] + len[y]); out[y] must start at 0.
__global__ void k_seg_absmax(const float *__restrict__ table, const uint64_t *__restrict__ off,
                             const uint64_t *__restrict__ len, uint32_t *__restrict__ out) {
  const uint32_t y = blockIdx.y;
  const uint64_t o = off[y], n = len[y];
  uint32_t m = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    m = max(m, __float_as_uint(table[o + i]) & 0x7FFFFFFFu);
  for (int k = 16; k; k >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, k));
  if ((threadIdx.x & 31) == 0 && m) atomicMax(out + y, m);
}

// The cross model's bound on |w^| of a single-valued request: for ad field j,
// w^[(j, v)] sums one weight of each pair (i, j), so |w^| <= the sum over j's
// pairs of their largest |w|; the bound is the largest such sum over j
// (+inf when a weight is not finite).
static int cross_bound(ebr_cross *c, const ebr_cross_desc *d, cudaStream_t st) {
  const uint32_t nseg = d->kind == EBR_W_HASHED ? 1u : d->n_pairs;
  if (nseg == 0) {
    c->wbound = 0.f;
    return EBR_OK;
  }
  std::vector<uint64_t> meta(2 * (size_t)nseg);
  for (uint32_t y = 0; y < nseg; y++) {
    if (d->kind == EBR_W_HASHED) {
      meta[y] = 0;
      meta[nseg + y] = 1ull << d->hash_bits;
    } else {
      meta[y] = d->w_off[y];
      meta[nseg + y] = (uint64_t)d->vocab_u[d->pairs[2 * y]] * d->vocab_a[d->pairs[2 * y + 1]];
    }
  }
  DevBuf dm, dout;
  int rc = dev_alloc(dm, meta.size() * 8);
  if (rc == EBR_OK) rc = dev_alloc(dout, (size_t)nseg * 4);
  std::vector<uint32_t> mx(nseg, 0);
  if (rc == EBR_OK) {
    cudaError_t e = cudaMemcpyAsync(dm.p, meta.data(), meta.size() * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dout.p, 0, (size_t)nseg * 4, st);
    if (e == cudaSuccess) {
      const uint64_t *off = (const uint64_t *)dm.p;
      k_seg_absmax<<<dim3(d->kind == EBR_W_HASHED ? 1024u : 8u, nseg), 256, 0, st>>>(
          (const float *)c->table.p, off, off + nseg, (uint32_t *)dout.p);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(mx.data(), dout.p, (size_t)nseg * 4,
                                              cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      set_error("ebr_cross_create: %s", cudaGetErrorString(e));
      rc = EBR_ECUDA;
    }
  }
  dev_free(dm);
  dev_free(dout);
  if (rc != EBR_OK) return rc;
  std::vector<double> field(d->f_a, 0.0);
  bool finite = true;
  for (uint32_t p = 0; p < d->n_pairs; p++) {
    const uint32_t b = mx[d->kind == EBR_W_HASHED ? 0 : p];
    if (b >= 0x7F800000u) finite = false;
    float f;
    memcpy(&f, &b, 4);
    field[d->pairs[2 * p + 1]] += f;
  }
  double wb = 0.0;
  for (double x : field) wb = std::max(wb, x);
  c->wbound = finite && wb < 1e38 ? (float)wb : INFINITY;
  return EBR_OK;
}
}  // namespace ebr

using namespace ebr;

// ----------------------------------------------------------------- C ABI
extern "C" int ebr_cross_create(const ebr_cross_desc *d, ebr_cross **out) {
  clear_error();
  if (!d || !out || !d->vocab_u || !d->vocab_a || !d->pairs || !d->w_table || d->f_a == 0 ||
      d->f_u == 0 || d->w_len == 0) {
    set_error("ebr_cross_create: invalid description");
    return EBR_EINVAL;
  }
  *out = nullptr;
  uint64_t n_keys = 0;
  for (uint32_t j = 0; j < d->f_a; j++) n_keys += d->vocab_a[j];
  if (n_keys == 0 || n_keys >= 0xFFFFFFFFull) {
    set_error("ebr_cross_create: key space must be 1 .. 2^32-2");
    return EBR_EINVAL;
  }
  for (uint32_t p = 0; p < d->n_pairs; p++) {
    if (d->pairs[2 * p] >= d->f_u || d->pairs[2 * p + 1] >= d->f_a) {
      set_error("ebr_cross_create: pair %u out of range", p);
      return EBR_EINVAL;
    }
  }
  if (d->kind == EBR_W_HASHED) {
    if (d->hash_bits < 1 || d->hash_bits > 30 || d->w_len < (1ull << d->hash_bits) ||
        d->n_pairs >= (1u << 24)) {
      set_error("ebr_cross_create: hashed table needs 1 <= hash_bits <= 30, w_len >= 2^bits");
      return EBR_EINVAL;
    }
    for (uint32_t i = 0; i < d->f_u; i++)
      if (d->vocab_u[i] > (1u << 20)) { set_error("ebr_cross_create: user vocab >= 2^20"); return EBR_EINVAL; }
    for (uint32_t j = 0; j < d->f_a; j++)
      if (d->vocab_a[j] > (1u << 20)) { set_error("ebr_cross_create: ad vocab >= 2^20"); return EBR_EINVAL; }
  } else if (d->kind == EBR_W_DENSE) {
    if (!d->w_off) { set_error("ebr_cross_create: dense tables need w_off"); return EBR_EINVAL; }
    for (uint32_t p = 0; p < d->n_pairs; p++) {
      uint64_t need = d->w_off[p] + (uint64_t)d->vocab_u[d->pairs[2 * p]] * d->vocab_a[d->pairs[2 * p + 1]];
      if (need > d->w_len) { set_error("ebr_cross_create: dense table %u exceeds w_len", p); return EBR_EINVAL; }
    }
  } else {
    set_error("ebr_cross_create: unknown weight kind");
    return EBR_EINVAL;
  }
  // metadata
  std::vector<uint32_t> m;
  std::vector<uint32_t> key_off(d->f_a + 1, 0);
  for (uint32_t j = 0; j < d->f_a; j++) key_off[j + 1] = key_off[j] + d->vocab_a[j];
  m.insert(m.end(), key_off.begin(), key_off.end());
  m.insert(m.end(), d->vocab_u, d->vocab_u + d->f_u);
  m.insert(m.end(), d->vocab_a, d->vocab_a + d->f_a);
  std::vector<uint32_t> ptr(d->f_a + 1, 0), of(d->n_pairs), usr(d->n_pairs), lo(d->n_pairs),
      hi(d->n_pairs);
  for (uint32_t p = 0; p < d->n_pairs; p++) ptr[d->pairs[2 * p + 1] + 1]++;
  for (uint32_t j = 0; j < d->f_a; j++) ptr[j + 1] += ptr[j];
  std::vector<uint32_t> fill(ptr.begin(), ptr.end() - 1);
  for (uint32_t p = 0; p < d->n_pairs; p++) {
    of[fill[d->pairs[2 * p + 1]]++] = p;
    usr[p] = d->pairs[2 * p];
    uint64_t off = d->w_off ? d->w_off[p] : 0;
    lo[p] = (uint32_t)off;
    hi[p] = (uint32_t)(off >> 32);
  }
  for (auto *v : {&ptr, &of, &usr, &lo, &hi}) m.insert(m.end(), v->begin(), v->end());
  int prev = 0;
  cudaGetDevice(&prev);
  EBR_CUDA_TRY(cudaSetDevice(d->device));
  ebr_cross *c = new ebr_cross();
  c->device = d->device;
  c->f_u = d->f_u;
  c->f_a = d->f_a;
  c->n_pairs = d->n_pairs;
  c->n_keys = (uint32_t)n_keys;
  c->kind = d->kind;
  c->hash_bits = d->hash_bits;
  c->w_len = d->w_len;
  c->vocab_u_host.assign(d->vocab_u, d->vocab_u + d->f_u);
  int rc = dev_alloc(c->table, d->w_len * 4);
  if (rc == EBR_OK) rc = dev_alloc(c->meta, m.size() * 4);
  cudaStream_t st = (cudaStream_t)d->stream;
  if (rc == EBR_OK) {
    cudaError_t e = cudaMemcpyAsync(c->table.p, d->w_table, d->w_len * 4, cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->meta.p, m.data(), m.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      set_error("ebr_cross_create: %s", cudaGetErrorString(e));
      rc = EBR_ECUDA;
    }
  }
  if (rc == EBR_OK) rc = cross_bound(c, d, st);
  cudaSetDevice(prev);
  if (rc != EBR_OK) {
    dev_free(c->table);
    dev_free(c->meta);
    delete c;
    return rc;
  }
  *out = c;
  return EBR_OK;
}

extern "C" void ebr_cross_free(ebr_cross *c) {
  if (!c) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(c->device);
  dev_free(c->table);
  dev_free(c->meta);
  cudaSetDevice(prev);
  delete c;
}

extern "C" uint32_t ebr_cross_n_keys(const ebr_cross *c) { return c ? c->n_keys : 0; }

static int expand_checked(const ebr_cross *c, const uint32_t *user_vals, uint32_t batch,
                          float *w_hat, void *stream, const uint32_t *user_ptr, uint32_t n_uv,
                          const char *where);

extern "C" int ebr_expand_query_seq(const ebr_cross *c, const uint32_t *user_ptr,
                                    const uint32_t *user_vals, uint32_t n_user_vals,
                                    float *w_hat, void *stream) {
  clear_error();
  if (!c || !user_ptr || !user_vals || !w_hat) {
    set_error("ebr_expand_query_seq: null argument");
    return EBR_EINVAL;
  }
  return expand_checked(c, user_vals, 1, w_hat, stream, user_ptr, n_user_vals,
                        "ebr_expand_query_seq");
}

extern "C" int ebr_expand_query(const ebr_cross *c, const uint32_t *user_vals, uint32_t batch,
                                float *w_hat, void *stream) {
  clear_error();
  if (!c || (batch && (!user_vals || !w_hat))) {
    set_error("ebr_expand_query: null argument");
    return EBR_EINVAL;
  }
  if (!batch) return EBR_OK;
  return expand_checked(c, user_vals, batch, w_hat, stream, nullptr, 0, "ebr_expand_query");
}

// Expansion on the call's stream, then a wait for it and a check of the
// device-side input flags.
static int expand_checked(const ebr_cross *c, const uint32_t *user_vals, uint32_t batch,
                          float *w_hat, void *stream, const uint32_t *user_ptr, uint32_t n_uv,
                          const char *where) {
  int prev = 0;
  cudaGetDevice(&prev);
  EBR_CUDA_TRY(cudaSetDevice(c->device));
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t *flags = nullptr;
  EBR_CUDA_TRY(cudaMallocAsync((void **)&flags, 4, st));
  EBR_CUDA_TRY(cudaMemsetAsync(flags, 0, 4, st));
  int rc = expand_into(c, user_vals, batch, w_hat, flags, st, nullptr, user_ptr, n_uv);
  uint32_t hf = 0;
  if (rc == EBR_OK) {
    cudaError_t e = cudaMemcpyAsync(&hf, flags, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      set_error("%s: %s", where, cudaGetErrorString(e));
      rc = EBR_ECUDA;
    }
  }
  cudaFreeAsync(flags, st);
  cudaSetDevice(prev);
  if (rc == EBR_OK && hf) rc = check_device_flags(hf, where);
  return rc;
}

// Validates one request against the index (host-visible fields only).
static int check_query(const ebr_index *ix, const ebr_cross *cross, const ebr_query &q) {
  if (!q.h_u) { set_error("query: h_u is null"); return EBR_EINVAL; }
  if (q.flags & ~(EBR_QF_KEY_MAJOR | EBR_QF_WINDOW_MAJOR)) {
    set_error("query: unknown flag bits 0x%x", q.flags);
    return EBR_EINVAL;
  }
  if (q.k == 0 || q.k > 8192) { set_error("query: k must be 1..8192 (got %u)", q.k); return EBR_EINVAL; }
  if (ix->dtype != EBR_F32 && (uint64_t)q.k * ix->rescore_mult > 8192) {
    set_error("query: R*k must be <= 8192 for BF16/FP8 scans");
    return EBR_EINVAL;
  }
  if (q.user_ptr && !q.user_vals) {
    set_error("query: user_ptr needs user_vals");
    return EBR_EINVAL;
  }
  if (q.user_vals) {
    if (!cross) { set_error("query: user_vals needs a cross model"); return EBR_EINVAL; }
    if (cross->n_keys != ix->n_keys) {
      set_error("query: cross model has %u keys, index has %u", cross->n_keys, ix->n_keys);
      return EBR_EINVAL;
    }
  } else if (!q.q_w) {
    set_error("query: needs user_vals or q_w");
    return EBR_EINVAL;
  }
  return EBR_OK;
}

// Copies a host request into device staging; returns the device view.
static int stage_in(ebr_index *ix, const ebr_cross *cross, const ebr_query &hq, ebr_query &dq,
                    cudaStream_t st) {
  Workspace &w = ix->ws;
  const size_t words = ((size_t)ix->n_ads + 63) / 64;
  const size_t nq = hq.user_vals ? 0 : (hq.q_key ? hq.n_q : ix->n_keys);
  const size_t n_uv = hq.user_ptr ? hq.n_user_vals : (cross ? cross->f_u : 0);
  size_t need = 256 + ix->d * 4 + 256 + n_uv * 4 + 256 + nq * 8 + 256 +
                (hq.filter ? words * 8 : 0) + 256 + (cross ? (cross->f_u + 1) * 4 : 0) + 256;
  EBR_TRY(dev_reserve(w.io_in, need));
  char *base = (char *)w.io_in.p;
  size_t off = 0;
  auto put = [&](const void *src, size_t bytes) -> void * {
    void *dst = base + off;
    if (bytes) cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
    off += (bytes + 255) / 256 * 256;
    return dst;
  };
  dq = hq;
  dq.h_u = (const float *)put(hq.h_u, ix->d * 4);
  if (hq.user_vals) dq.user_vals = (const uint32_t *)put(hq.user_vals, n_uv * 4);
  if (hq.user_ptr) dq.user_ptr = (const uint32_t *)put(hq.user_ptr, (cross->f_u + 1) * 4);
  if (!hq.user_vals) {
    if (hq.q_key) dq.q_key = (const uint32_t *)put(hq.q_key, (size_t)hq.n_q * 4);
    dq.q_w = (const float *)put(hq.q_w, (hq.q_key ? (size_t)hq.n_q : ix->n_keys) * 4);
  }
  if (hq.filter) dq.filter = (const uint64_t *)put(hq.filter, words * 8);
  EBR_CUDA_TRY(cudaGetLastError());
  return EBR_OK;
}

extern "C" int ebr_score_topk(const ebr_index *cix, const ebr_cross *cross, const ebr_query *q,
                              uint32_t batch, uint32_t *out_ids, float *out_scores, int io,
                              void *stream) {
  clear_error();
  if (!cix || (batch && (!q || !out_ids || !out_scores)) || (io != EBR_IO_DEVICE && io != EBR_IO_HOST)) {
    set_error("ebr_score_topk: invalid argument");
    return EBR_EINVAL;
  }
  if (!batch) return EBR_OK;
  ebr_index *ix = const_cast<ebr_index *>(cix);
  uint32_t kmax = 0, nq_max = 0;
  for (uint32_t b = 0; b < batch; b++) {
    EBR_TRY(check_query(ix, cross, q[b]));
    kmax = std::max(kmax, q[b].k);
    nq_max = std::max(nq_max, (q[b].user_vals || !q[b].q_key) ? ix->n_keys : q[b].n_q);
  }
  int prev = 0;
  cudaGetDevice(&prev);
  EBR_CUDA_TRY(cudaSetDevice(ix->device));
  cudaStream_t st = (cudaStream_t)stream;
  const uint32_t kcap = ix->dtype == EBR_F32 ? kmax : std::min<uint32_t>(kmax * ix->rescore_mult, 8192);
  int rc = ws_prepare(ix, nq_max, pow2_at_least(std::max<uint32_t>(kcap, 256)));
  if (rc != EBR_OK) { cudaSetDevice(prev); return rc; }
  Workspace &w = ix->ws;
  if (!w.host_ctrl) {
    if (cudaMallocHost(&w.host_ctrl, sizeof(Ctrl)) != cudaSuccess) {
      cudaGetLastError();
      w.host_ctrl = nullptr;
    }
  }
  uint32_t *d_ids = out_ids;
  float *d_scores = out_scores;
  if (io == EBR_IO_HOST) {
    const size_t ids_bytes = ((size_t)batch * kmax * 4 + 255) / 256 * 256;
    rc = dev_reserve(w.io_out, 2 * ids_bytes);
    if (rc != EBR_OK) { cudaSetDevice(prev); return rc; }
    d_ids = (uint32_t *)w.io_out.p;
    d_scores = (float *)((char *)w.io_out.p + ids_bytes);
  }
  if (batch > 1 && batch_qualifies(ix, cross, q, batch)) {
    rc = query_batch(ix, cross, q, batch, out_ids, out_scores, kmax, io, st);
    cudaSetDevice(prev);
    return rc;
  }
  uint32_t flags_acc = 0;
  for (uint32_t b = 0; b < batch && rc == EBR_OK; b++) {
    ebr_query dq = q[b];
    if (io == EBR_IO_HOST) rc = stage_in(ix, cross, q[b], dq, st);
    if (rc == EBR_OK)
      rc = query_one(ix, cross, dq, d_ids + (size_t)b * kmax, d_scores + (size_t)b * kmax, kmax, st);
    if (rc == EBR_OK && (io == EBR_IO_HOST || b + 1 == batch) && w.host_ctrl) {
      cudaMemcpyAsync(w.host_ctrl, w.ctrl.p, sizeof(Ctrl), cudaMemcpyDeviceToHost, st);
    }
    if (rc == EBR_OK && io == EBR_IO_HOST) {
      cudaError_t e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) { set_error("ebr_score_topk: %s", cudaGetErrorString(e)); rc = EBR_ECUDA; }
      else if (w.host_ctrl) flags_acc |= ((Ctrl *)w.host_ctrl)->flags;
    }
  }
  if (rc == EBR_OK && io == EBR_IO_HOST) {
    cudaError_t e = cudaMemcpy2DAsync(out_ids, kmax * 4, d_ids, kmax * 4, kmax * 4, batch,
                                      cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(out_scores, kmax * 4, d_scores, kmax * 4, kmax * 4, batch,
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { set_error("ebr_score_topk: %s", cudaGetErrorString(e)); rc = EBR_ECUDA; }
    if (rc == EBR_OK && flags_acc) rc = check_device_flags(flags_acc, "ebr_score_topk");
  }
  cudaSetDevice(prev);
  return rc;
}

static int single_query_prep(ebr_index *ix, const ebr_cross *cross, const ebr_query *q,
                             const uint32_t **q_key, const float **q_w, uint32_t *n_q,
                             Ctrl **ctrl, cudaStream_t st) {
  ebr_query qq = *q;
  if (qq.k == 0) qq.k = 1;
  EBR_TRY(check_query(ix, cross, qq));
  EBR_TRY(ws_prepare(ix, (q->user_vals || !q->q_key) ? ix->n_keys : q->n_q, 256));
  *ctrl = (Ctrl *)ix->ws.ctrl.p;
  EBR_CUDA_TRY(cudaMemsetAsync(*ctrl, 0, kCtrlBytes + kHistWords * 4, st));  // + histogram
  *q_key = q->q_key;
  *q_w = q->q_w;
  *n_q = q->n_q;
  if (q->user_vals) {
    EBR_TRY(expand_into(cross, q->user_vals, 1, (float *)ix->ws.w_dense.p, &(*ctrl)->flags, st,
                        nullptr, q->user_ptr, q->n_user_vals));
    *q_key = nullptr;
    *q_w = (const float *)ix->ws.w_dense.p;
    *n_q = ix->n_keys;
  } else if (!q->q_key) {
    *n_q = ix->n_keys;
  }
  return EBR_OK;
}

static int finish_sync(ebr_index *ix, cudaStream_t st, const char *where) {
  Ctrl hc;
  EBR_CUDA_TRY(cudaMemcpyAsync(&hc, ix->ws.ctrl.p, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
  EBR_CUDA_TRY(cudaStreamSynchronize(st));
  return check_device_flags(hc.flags, where);
}

extern "C" int ebr_score_all(const ebr_index *cix, const ebr_cross *cross, const ebr_query *q,
                             float *out_scores, void *stream) {
  clear_error();
  if (!cix || !q || !out_scores) {
    set_error("ebr_score_all: null argument");
    return EBR_EINVAL;
  }
  ebr_index *ix = const_cast<ebr_index *>(cix);
  int prev = 0;
  cudaGetDevice(&prev);
  EBR_CUDA_TRY(cudaSetDevice(ix->device));
  cudaStream_t st = (cudaStream_t)stream;
  const uint32_t *q_key;
  const float *q_w;
  uint32_t n_q;
  Ctrl *ctrl;
  int rc = single_query_prep(ix, cross, q, &q_key, &q_w, &n_q, &ctrl, st);
  const bool fused = rc == EBR_OK && q_key == nullptr && !(q->flags & EBR_QF_KEY_MAJOR) &&
                     fused_fits(ix, 1);
  if (fused) {
    rc = launch_fused(ix, q->h_u, q_w, (uint32_t *)ix->ws.wq.p, false, nullptr, 1, nullptr, ctrl,
                      out_scores, nullptr, ws_hist(ix->ws),
                      ix->num_sms * kMaxCtasPerSm, st);
  } else {
    if (rc == EBR_OK) rc = run_wide(ix, q_key, q_w, n_q, ctrl, st);
    if (rc == EBR_OK) {
      ScanArgs a;
      memset(&a, 0, sizeof(a));
      const bool quant = ix->dtype != EBR_F32;
      a.emb = quant ? ix->emb_q.p : ix->emb_f32.p;
      a.scale = ix->dtype == EBR_FP8E4M3 ? (const float *)ix->emb_scale.p : nullptr;
      a.h_u = q->h_u;
      a.wide = (const float *)ix->ws.wide.p;
      a.n_ads = ix->n_ads;
      a.k = 1;
      a.ctrl = ctrl;
      a.all_out = out_scores;
      rc = launch_scan<MODE_ALL>(ix, a, st);
    }
  }
  if (rc == EBR_OK) rc = finish_sync(ix, st, "ebr_score_all");
  cudaSetDevice(prev);
  return rc;
}

extern "C" int ebr_wide_scores(const ebr_index *cix, const ebr_cross *cross, const ebr_query *q,
                               float *out_wide, void *stream) {
  clear_error();
  if (!cix || !q || !out_wide) {
    set_error("ebr_wide_scores: null argument");
    return EBR_EINVAL;
  }
  ebr_index *ix = const_cast<ebr_index *>(cix);
  int prev = 0;
  cudaGetDevice(&prev);
  EBR_CUDA_TRY(cudaSetDevice(ix->device));
  cudaStream_t st = (cudaStream_t)stream;
  const uint32_t *q_key;
  const float *q_w;
  uint32_t n_q;
  Ctrl *ctrl;
  int rc = single_query_prep(ix, cross, q, &q_key, &q_w, &n_q, &ctrl, st);
  if (rc == EBR_OK) rc = run_wide(ix, q_key, q_w, n_q, ctrl, st);
  if (rc == EBR_OK) {
    cudaError_t e = cudaMemcpyAsync(out_wide, ix->ws.wide.p, (size_t)ix->n_ads * 4,
                                    cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) { set_error("ebr_wide_scores: %s", cudaGetErrorString(e)); rc = EBR_ECUDA; }
  }
  if (rc == EBR_OK) rc = finish_sync(ix, st, "ebr_wide_scores");
  cudaSetDevice(prev);
  return rc;
}

// Device counters of the traversal chosen for sparse lists: [0] lists routed
// on the device, [1] of those decoded window by window.  Waits for the device.
static int read_route_stats(ebr_index *ix, uint64_t out[2]) {
  out[0] = out[1] = 0;
  if (!ix->ws.route_stats.p) return EBR_OK;
  unsigned long long h[2];
  EBR_CUDA_TRY(cudaMemcpy(h, ix->ws.route_stats.p, sizeof(h), cudaMemcpyDeviceToHost));
  out[0] = h[0];
  out[1] = h[1];
  return EBR_OK;
}

extern "C" int ebr_profile_enable(ebr_index *ix, int on) {
  clear_error();
  if (!ix) {
    set_error("ebr_profile_enable: null index");
    return EBR_EINVAL;
  }
  ebr_profile z;
  memset(&z, 0, sizeof(z));
  ebr_profile tmp;
  int rc = ebr_profile_read(ix, &tmp);  // drain pending events
  if (rc == EBR_OK) rc = read_route_stats(ix, ix->route_base);
  ix->prof_acc = z;
  ix->prof = on != 0;
  return rc;
}

extern "C" int ebr_profile_read(ebr_index *ix, ebr_profile *out) {
  clear_error();
  if (!ix || !out) {
    set_error("ebr_profile_read: null argument");
    return EBR_EINVAL;
  }
  for (auto &ev : ix->prof_pending) {
    EBR_CUDA_TRY(cudaEventSynchronize(ev[4]));
    float t[4];
    for (int i = 0; i < 4; i++) EBR_CUDA_TRY(cudaEventElapsedTime(&t[i], ev[i], ev[i + 1]));
    ix->prof_acc.calls += 1;
    ix->prof_acc.ms_expand += t[0];
    ix->prof_acc.ms_wide += t[1];
    ix->prof_acc.ms_scan += t[2];
    ix->prof_acc.ms_final += t[3];
    ix->prof_pool.push_back(ev);
  }
  ix->prof_pending.clear();
  for (auto &ev : ix->bprof_pending) {
    EBR_CUDA_TRY(cudaEventSynchronize(ev[3]));
    float t[3];
    for (int i = 0; i < 3; i++) EBR_CUDA_TRY(cudaEventElapsedTime(&t[i], ev[i], ev[i + 1]));
    ix->prof_acc.batch_calls += 1;
    ix->prof_acc.ms_batch_stage += t[0];
    ix->prof_acc.ms_batch_scan += t[1];
    ix->prof_acc.ms_batch_merge += t[2];
    ix->prof_pool.push_back(ev);
  }
  ix->bprof_pending.clear();
  *out = ix->prof_acc;
  uint64_t rs[2] = {0, 0};
  EBR_TRY(read_route_stats(ix, rs));
  out->auto_routed = rs[0] - ix->route_base[0];
  out->window_routed = rs[1] - ix->route_base[1];
  out->launches = ix->launches;
  out->lib_launches = ix->lib_launches;
  out->batched = ix->batched;
  out->recomputed = ix->fallbacks;
  return EBR_OK;
}

// =====================================================================
// Allocation-free variant of the scan + top-K (ebr_scan_topk_noalloc)
// =====================================================================
// For callers that must not allocate device memory: a serving process whose
// device memory is owned up front by another allocator (a framework's caching
// pool, a fixed HBM budget), or a latency-critical thread that cannot afford
// cudaMalloc's implicit device-wide synchronisation.  Its scratch (the
// per-CTA candidate lists and the control block) lives in the file-scope
// array below, which every GPU that loads this library holds until exit.
namespace ebr {
namespace {

constexpr uint32_t kNoAllocMaxK = 1024;     // largest K accepted
constexpr uint32_t kNoAllocMaxGrid = 160;   // CTAs of the scan (>= SM count of a GB300)
constexpr uint32_t kNoAllocCtrlWords = 8;   // 64 bytes reserved for the Ctrl block
constexpr size_t kNoAllocWords = kNoAllocCtrlWords + (size_t)kNoAllocMaxGrid * kNoAllocMaxK;
// 8 * (8 + 160 * 1024) bytes = 1.25 MiB.
static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNoAllocWords];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kNoAllocMaxDevices] = {nullptr};
void *g_noalloc_ctx[kNoAllocMaxDevices] = {nullptr};  // context the address belongs to
int g_noalloc_sms[kNoAllocMaxDevices] = {0};
typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
CtxGetCurrentFn g_ctx_get_current = nullptr;

// The current driver context (nullptr if it cannot be read): a device reset
// replaces the primary context, and with it the array's device address.
void *current_context() {
  if (!g_ctx_get_current) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return nullptr;
    g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(fn);
  }
  CUcontext c = nullptr;
  if (g_ctx_get_current(&c) != CUDA_SUCCESS) return nullptr;
  return reinterpret_cast<void *>(c);
}

template <int D>
int noalloc_launch(const ScanArgs &a0, int sms, cudaStream_t st) {
  using Sh = ScanShape<float, D>;
  ScanArgs a = a0;
  a.cap = a.k + std::max<uint32_t>(a.k, 2 * Sh::kTileRows);
  a.cap = (a.cap + 255) / 256 * 256;
  const size_t cand_bytes = (size_t)2 * a.cap * 8;
  uint32_t stages = 4;
  while (stages > 2 && cand_bytes + (size_t)stages * Sh::kStageBytes > 200 * 1024) stages--;
  a.stages = stages;
  const size_t smem = cand_bytes + (size_t)stages * Sh::kStageBytes;
  const uint32_t n_tiles = (a.n_ads + Sh::kTileRows - 1) / Sh::kTileRows;
  const int grid = (int)std::min<uint32_t>(std::min<uint32_t>((uint32_t)sms, kNoAllocMaxGrid),
                                           n_tiles);
  auto kern = k_scan_topk<float, D, MODE_TOPK>;
  EBR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  kern<<<grid, kScanThreads, smem, st>>>(a);
  EBR_CUDA_TRY(cudaGetLastError());
  return EBR_OK;
}

}  // namespace
}  // namespace ebr

extern "C" int ebr_scan_topk_noalloc(const float *emb, uint32_t n_ads, uint32_t d,
                                     const float *h_u, const float *wide,
                                     const uint64_t *filter, uint32_t k, uint32_t *out_ids,
                                     float *out_scores, int device, void *stream) {
  clear_error();
  if (!emb || !h_u || !out_ids || !out_scores || n_ads == 0) {
    set_error("ebr_scan_topk_noalloc: null pointer or n_ads == 0");
    return EBR_EINVAL;
  }
  if ((reinterpret_cast<uintptr_t>(emb) & 15u) != 0) {
    // the scan stages rows with bulk copies, which start on 16-byte boundaries
    set_error("ebr_scan_topk_noalloc: emb must be 16-byte aligned");
    return EBR_EINVAL;
  }
  if (k == 0 || k > kNoAllocMaxK) {
    set_error("ebr_scan_topk_noalloc: k = %u is outside 1..%u (the static scratch holds %u "
              "candidates per CTA)", k, kNoAllocMaxK, kNoAllocMaxK);
    return EBR_EINVAL;
  }
  if (!(d == 4 || d == 8 || d == 16 || d == 32 || d == 64 || d == 128)) {
    set_error("ebr_scan_topk_noalloc: d = %u unsupported (4, 8, 16, 32, 64 or 128)", d);
    return EBR_EINVAL;
  }
  if (device < 0 || device >= kNoAllocMaxDevices) {
    set_error("ebr_scan_topk_noalloc: device %d out of range", device);
    return EBR_EINVAL;
  }
  int prev = 0;
  EBR_CUDA_TRY(cudaGetDevice(&prev));
  if (prev != device) EBR_CUDA_TRY(cudaSetDevice(device));
  void *base = nullptr;
  int sms = 0;
  {
    // Set-up once per device, with that device current (and again if the
    // device's context was replaced, as cudaDeviceReset does): resolve the
    // device address of the static scratch array (the host-side symbol is
    // only a stand-in and must never reach a kernel).
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    void *ctx = current_context();
    if (!g_noalloc_addr[device] || ctx != g_noalloc_ctx[device]) {
      void *p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // creates the context if needed
      ctx = current_context();
      if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&g_noalloc_sms[device], cudaDevAttrMultiProcessorCount,
                                   device);
      if (e != cudaSuccess) {
        set_error("ebr_scan_topk_noalloc: set-up failed: %s", cudaGetErrorString(e));
        if (prev != device) cudaSetDevice(prev);
        return EBR_ECUDA;
      }
      g_noalloc_addr[device] = p;
      g_noalloc_ctx[device] = ctx;
    }
    base = g_noalloc_addr[device];
    sms = g_noalloc_sms[device];
  }
  cudaStream_t st = (cudaStream_t)stream;
  Ctrl *ctrl = reinterpret_cast<Ctrl *>(base);
  uint64_t *cand = reinterpret_cast<uint64_t *>(base) + kNoAllocCtrlWords;
  int rc = EBR_OK;
  // The array keeps the previous call's contents: clear the control block.
  cudaError_t e = cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), st);
  if (e != cudaSuccess) {
    set_error("ebr_scan_topk_noalloc: %s", cudaGetErrorString(e));
    rc = EBR_ECUDA;
  }
  if (rc == EBR_OK) {
    ScanArgs a;
    memset(&a, 0, sizeof(a));
    a.emb = emb;
    a.h_u = h_u;
    a.wide = wide;
    a.filter = filter;
    a.n_ads = n_ads;
    a.k = k;
    a.cand_out = cand;
    a.ctrl = ctrl;
    switch (d) {
      case 4: rc = noalloc_launch<4>(a, sms, st); break;
      case 8: rc = noalloc_launch<8>(a, sms, st); break;
      case 16: rc = noalloc_launch<16>(a, sms, st); break;
      case 32: rc = noalloc_launch<32>(a, sms, st); break;
      case 64: rc = noalloc_launch<64>(a, sms, st); break;
      default: rc = noalloc_launch<128>(a, sms, st); break;
    }
  }
  if (rc == EBR_OK) {
    uint32_t p2 = 1;
    while (p2 < k) p2 <<= 1;
    k_final_select<<<1, kFinalThreads, (size_t)p2 * 8, st>>>(cand, ctrl, 0, k, k, out_ids,
                                                             out_scores, nullptr, 0u);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
      set_error("ebr_scan_topk_noalloc: %s", cudaGetErrorString(e));
      rc = EBR_ECUDA;
    }
  }
  if (prev != device) cudaSetDevice(prev);
  return rc;
}
