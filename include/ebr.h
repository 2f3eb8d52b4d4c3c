/*
 * ebr.h -- C ABI of the GB300 embedding-based ad retrieval library.
 *
 * The library scores one request (or a batch) against every ad of an
 * inventory with the Wide & Deep retrieval score of the paper
 * "An Efficient Embedding Based Ad Retrieval with GPU-Powered Feature
 * Interaction" (arXiv 2511.22460):
 *
 *     s(u, a) = <h~_u, h~_a> + sum_m w_m x_m L[a, m]        (HitMatch eq., Sec. 3.3)
 *
 * and returns the K best ads.  The deep term is the dual-tower inner product
 * (Eq. 1, Sec. 3.1; IPNN dimensions are concatenated into h~, Sec. 3.2).  The
 * wide term is evaluated by walking the compressed inverted list of
 * Sec. 3.4 (Algorithm 1 builds it, Algorithm 2 queries it).
 *
 * Conventions for every entry point:
 *  - Return value: EBR_OK (0) or a negative EBR_E* code.  Nothing aborts or
 *    throws across this boundary.  After an error, ebr_last_error() returns a
 *    message for the calling thread.
 *  - Plain pointers only.  "device" means memory of the index's CUDA device;
 *    "host" means ordinary or pinned host memory.  Each argument says which
 *    it accepts.
 *  - Ownership: the caller owns every pointer it passes in and may free it
 *    once the call returns (stream-ordered calls: once the stream has
 *    drained).  The library owns the objects it creates (ebr_index,
 *    ebr_cross, ebr_server) and their device memory until the matching
 *    *_free / *_destroy.
 *  - stream: a cudaStream_t passed as void* (NULL = legacy default stream).
 *  - Calls that use one index's scratch memory (ebr_score_topk,
 *    ebr_score_all) must not overlap on the GPU: issue them on one stream, or
 *    synchronise between streams.
 */
#ifndef EBR_H
#define EBR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define EBR_OK 0
#define EBR_EINVAL (-1)    /* bad argument: shape, id >= N, key >= n_keys, K > limits ... */
#define EBR_ENOMEM (-2)    /* device allocation failed, or admission refused */
#define EBR_ECUDA (-3)     /* CUDA runtime error; see ebr_last_error() */
#define EBR_EAGAIN (-4)    /* ebr_poll: request still in flight */
#define EBR_ETIMEDOUT (-5) /* a bounded device or host wait ran out */
#define EBR_EDATA (-6)     /* a device-side check rejected input data (e.g. a query key >= n_keys) */

/* Message for the last failing call on this thread ("" if none). */
const char *ebr_last_error(void);
/* ABI version: 0xMMmmpp. */
int ebr_version(void);

typedef enum { EBR_F32 = 0, EBR_BF16 = 1, EBR_FP8E4M3 = 2 } ebr_dtype;

/* --------------------------------------------------------------- index */
typedef struct ebr_index ebr_index;

/*
 * Index description.  The feature->ad matrix L of Sec. 3.3 is given as its
 * non-zeros: (post_key[e], post_ad[e]) means ad post_ad[e] is in the posting
 * list of key post_key[e] (keys are feature indices, values are ad indices,
 * Sec. 3.4 and Algorithm 1's input).  Pairs may come in any order and may
 * repeat (a repeated pair counts once: a posting list is a set).
 */
typedef struct {
  uint32_t n_ads;            /* N, ad ids are 0 .. N-1 (N >= 1) */
  uint32_t n_keys;           /* number of feature keys, keys are 0 .. n_keys-1 (>= 1) */
  uint64_t nnz;              /* number of (key, ad) pairs, < 2^31 */
  const uint32_t *post_key;  /* [nnz] host or device */
  const uint32_t *post_ad;   /* [nnz] host or device */
  uint32_t d;                /* embedding dimension: 4, 8, 16, 32, 64 or 128 */
  ebr_dtype emb_dtype;       /* dtype the scan streams; BF16/FP8 keep an FP32 copy for rescoring */
  const float *emb_f32;      /* [N][d] row-major FP32 ad vectors h~_a, host or device */
  uint32_t rescore_mult;     /* R: BF16/FP8 scans keep R*K candidates for FP32 rescoring (0 -> 4) */
  int device;                /* CUDA device ordinal */
  void *stream;              /* stream for the build */
} ebr_index_desc;

/*
 * Besides the paper's key-major arrays, the index keeps a window-major view
 * of the same blocks (per group, ordered by (window h = ad >> 8, key k), each
 * with its key and its 2^g value bytes, plus per-window offsets).  Requests
 * whose query covers the whole key space (dense w^ or raw user features) walk
 * that view window by window inside the scan; sparse key lists walk the
 * key-major arrays with Algorithm 2.
 *
 * Build the compressed inverted list of Algorithm 1 (Block Grouping by
 * ad >> 8, Logarithmic Categorization into groups g = ceil(log2 n) = 0..8,
 * Block Compression to one 24-bit header per block plus one byte per ad,
 * struct-of-arrays storage with a per-key offset array; Sec. 3.4) on the GPU,
 * and upload (and, for BF16/FP8, quantise) the ad embeddings.
 * Returns EBR_EINVAL for bad sizes and EBR_EDATA if a key >= n_keys or an
 * ad >= n_ads is found.  Synchronous: returns after the build completes.
 */
int ebr_build_index(const ebr_index_desc *desc, ebr_index **out);
void ebr_index_free(ebr_index *ix);

typedef struct {
  uint32_t n_ads, n_keys, d;
  ebr_dtype emb_dtype;
  uint32_t rescore_mult;
  uint64_t nnz_unique;          /* distinct (key, ad) pairs */
  uint64_t n_blocks[9];         /* blocks per size group g */
  uint64_t index_bytes;         /* sum_g 4*(n_keys+1) + 4*n_blocks[g] + 2^g*n_blocks[g] */
  uint64_t emb_bytes;           /* bytes of the scanned embedding table (+ FP8 row scales) */
  float build_ms;               /* device time of the index build (Algorithm 1 only) */
  float window_view_ms;         /* device time of the window-major view (below) */
  uint64_t window_view_bytes;   /* its size: per-block keys + value bytes + window offsets */
  uint32_t n_windows;           /* windows of 256 consecutive ads: ceil(n_ads / 256) */
  uint32_t max_keys_per_ad;     /* most distinct keys of one ad */
  uint32_t max_window_slots;    /* most value slots (real + padding) in one window */
  uint32_t max_window_chunks;   /* most 32-slot work chunks in one window */
} ebr_index_info;
int ebr_index_get_info(const ebr_index *ix, ebr_index_info *out);

/*
 * Copy group g of the index to host buffers: keys[n_keys+1] (per-key block
 * offsets), header[n_blocks[g]] (ad >> 8 of each block), values[n_blocks[g] << g]
 * (ad & 255 of each slot; within a block ascending, padding slots are 0 and
 * only slot 0 may hold a real 0).  Any of the three may be NULL to skip it.
 */
int ebr_index_export(const ebr_index *ix, uint32_t g, uint32_t *keys, uint32_t *header,
                     uint8_t *values);

/*
 * Copy the scanned embedding table to host: codes[N*d] of the index dtype
 * (float, bfloat16 bits as uint16, or E4M3 bytes) and, for FP8, scale[N].
 */
int ebr_index_export_emb(const ebr_index *ix, void *codes, float *scale);

/* ------------------------------------------------- cross model / expansion */
typedef struct ebr_cross ebr_cross;
typedef enum { EBR_W_DENSE = 0, EBR_W_HASHED = 1 } ebr_wkind;

/*
 * Cross-feature model.  Feature key of ad field j with value v is
 * key_off[j] + v, key_off[j] = vocab_a[0] + ... + vocab_a[j-1].  A cross
 * pair p = (i, j) pairs user field i with ad field j; its weight for user
 * value u and ad value v is
 *   dense:  w_table[w_off[p] + u * vocab_a[j] + v]
 *   hashed: w_table[splitmix64((p << 40) | (u << 20) | v) & (2^hash_bits - 1)]
 * where splitmix64(x) is the first output of the SplitMix64 generator seeded
 * with x.  Hashed tables need vocabularies < 2^20 and n_pairs < 2^24.
 */
typedef struct {
  uint32_t f_u, f_a;
  const uint32_t *vocab_u;   /* host [f_u] */
  const uint32_t *vocab_a;   /* host [f_a] */
  uint32_t n_pairs;
  const uint32_t *pairs;     /* host [n_pairs][2] = (user field i, ad field j) */
  ebr_wkind kind;
  const float *w_table;      /* host or device, w_len floats; copied */
  uint64_t w_len;
  const uint64_t *w_off;     /* host [n_pairs], dense tables only (else NULL) */
  uint32_t hash_bits;        /* hashed tables: 1 .. 30 */
  int device;
  void *stream;
} ebr_cross_desc;
int ebr_cross_create(const ebr_cross_desc *desc, ebr_cross **out);
void ebr_cross_free(ebr_cross *c);
uint32_t ebr_cross_n_keys(const ebr_cross *c);

/*
 * Query expansion: the non-zero (k, w^) of a request (Algorithm 2's input,
 * w^ = w x of Sec. 3.4 with x = 1).  Cross features sharing an ad-field key
 * fold into one weight:  w_hat[b][key_off[j] + v] = sum over pairs (i, j) of
 * w_ij(user_vals[b][i], v).  Output is dense over all n_keys keys (0 for ad
 * fields in no pair).  user_vals: device [batch][f_u]; w_hat: device
 * [batch][n_keys].  A user value >= its vocabulary gives EBR_EDATA (checked on
 * device, reported after the stream drains) and a zero row.
 */
int ebr_expand_query(const ebr_cross *c, const uint32_t *user_vals, uint32_t batch,
                     float *w_hat, void *stream);
/*
 * The expansion of one user with multi-valued fields (history): field i
 * holds user_vals[user_ptr[i] .. user_ptr[i+1]), and every value is one hit
 * feature, so w_hat[key_off[j] + v] = sum over pairs (i, j) and values u of
 * field i of w_ij(u, v) (HitMatch equation, Sec. 3.3).  user_ptr: device
 * [f_u + 1], starting at 0, not decreasing, ending at n_user_vals;
 * user_vals: device [n_user_vals]; w_hat: device [n_keys].  Bad offsets or a
 * value outside its vocabulary give EBR_EDATA after the stream drains.
 */
int ebr_expand_query_seq(const ebr_cross *c, const uint32_t *user_ptr, const uint32_t *user_vals,
                         uint32_t n_user_vals, float *w_hat, void *stream);

/* ------------------------------------------------------------- queries */
/*
 * One request.  The wide term's query is either
 *   - raw user features: user_vals[f_u], expanded with the call's cross model;
 *   - multi-valued user features (a history per field): user_ptr[f_u + 1]
 *     and user_vals[n_user_vals], field i holding user_vals[user_ptr[i] ..
 *     user_ptr[i+1]) (none when equal); each (user value, ad value) of a
 *     cross pair is one hit feature with x = 1 (HitMatch equation, Sec. 3.3),
 *     so w^[key_off[j] + v] = sum over pairs (i, j) and values u of field i
 *     of w_ij(u, v).  user_ptr must start at 0, not decrease and end at
 *     n_user_vals; a violation or a value outside its vocabulary is an
 *     input error (EBR_EDATA; the offsets of host requests in a batch are
 *     checked on the host, the rest on the device).  A batch may mix such
 *     requests with single-valued ones;
 *   - a dense weight vector: q_key == NULL, q_w[n_keys] indexed by key;
 *   - a sparse list: q_key[n_q], q_w[n_q] (duplicates add, keys must be < n_keys).
 * filter: targeting bitmap, bit a of word a >> 6 keeps ad a (NULL keeps all).
 * k: 1 .. 8192 (with BF16/FP8 scans, R*k <= 8192).
 */
typedef struct {
  const float *h_u;            /* [d] */
  const uint32_t *user_vals;   /* [f_u] or NULL */
  uint32_t n_q;
  const uint32_t *q_key;       /* [n_q] or NULL */
  const float *q_w;            /* [n_q] or [n_keys] */
  const uint64_t *filter;      /* [ceil(N / 64)] or NULL */
  uint32_t k;
  uint32_t flags;              /* EBR_QF_* bits */
  const uint32_t *user_ptr;    /* [f_u + 1] or NULL (one value per field) */
  uint32_t n_user_vals;        /* values in user_vals when user_ptr is set */
} ebr_query;

/* Walk the key-major arrays with Algorithm 2 (global scatter into a per-ad
 * score buffer) even when the query is dense.  By default dense queries use
 * the fused window-major scan, and a sparse key list takes Algorithm 2 or
 * the window-major decode, chosen on the device by its share of the index's
 * work (the window-major decode from 1/8 of the index's work units on). */
#define EBR_QF_KEY_MAJOR 1u
/* For a sparse key list (q_key != NULL): sum the list into a dense w^ over the
 * key space (repeated keys add; a key >= n_keys fails the call with
 * EBR_EDATA, and so does a non-finite sum) and decode it window by window
 * inside the fused scan, as for a dense query; blocks of keys whose w^ is
 * zero add nothing.  Ignored for dense queries and when EBR_QF_KEY_MAJOR is
 * also set. */
#define EBR_QF_WINDOW_MAJOR 2u

#define EBR_IO_DEVICE 0   /* all query arrays and outputs are device pointers; stream-ordered */
#define EBR_IO_HOST 1     /* all query arrays and outputs are host pointers; the call copies them
                             in and out on `stream` and returns after the stream drained */

/*
 * Score every ad for each of `batch` requests and return its top K
 * (Eq. 1 + HitMatch equation; the top-K retrieval of Sec. 2/4.4).  Row b of
 * out_ids/out_scores ([batch][kmax], kmax = max_b q[b].k) holds request b's
 * best ads by score descending then id ascending; positions past the number
 * of eligible ads hold id 0xFFFFFFFF and score -inf.  The full score vector
 * is never written to device memory.  `cross` may be NULL when no request
 * uses user_vals.  `q` is a host array of `batch` structs.
 * Device-side input checks (a key >= n_keys, a user value outside its
 * vocabulary, a non-finite weight) fail the call with EBR_EDATA when it waits
 * for the device, i.e. with EBR_IO_HOST; with EBR_IO_DEVICE the call is
 * stream-ordered and does not wait, so such a request yields unspecified
 * results instead.
 */
int ebr_score_topk(const ebr_index *ix, const ebr_cross *cross, const ebr_query *q,
                   uint32_t batch, uint32_t *out_ids, float *out_scores, int io,
                   void *stream);

/*
 * Diagnostic: the full score vector of one request, out_scores[N] (device),
 * computed by the same kernels as ebr_score_topk's scan (with the index's
 * scan dtype) but written out instead of selected.  The filter is ignored.
 */
int ebr_score_all(const ebr_index *ix, const ebr_cross *cross, const ebr_query *q,
                  float *out_scores, void *stream);

/*
 * Diagnostic: only the wide (HitMatch) term of one request via Algorithm 2's
 * key-major walk: out_wide[N] (device) = sum over query entries (k, w^) of
 * w^ * L[a, k].
 */
int ebr_wide_scores(const ebr_index *ix, const ebr_cross *cross, const ebr_query *q,
                    float *out_wide, void *stream);

/*
 * Diagnostic: quantise n floats (device) with the library's converters:
 * dtype EBR_BF16 writes uint16 codes, EBR_FP8E4M3 writes E4M3 bytes of x
 * (saturating to +-448, no scaling).
 */
int ebr_quantize(const float *x, uint64_t n, ebr_dtype dtype, void *out, void *stream);

/*
 * Diagnostic: out[i][b] = sum_t A[i][t] * U[b][t] on the tensor cores
 * (tcgen05.mma, BF16 inputs, FP32 accumulation in TMEM, operands loaded by
 * tensor TMA) -- the deep term (Eq. 1) of a batch of users against ads, as the
 * batched scan computes it.  A: device [n][d] BF16 bits, U: device [B][d],
 * out: device [n][B] FP32.  d in {64, 128}; B a multiple of 32 in 32..256.
 * Synchronous.
 */
int ebr_debug_gemm_bf16(const uint16_t *A, uint32_t n, const uint16_t *U, uint32_t B, uint32_t d,
                        float *out, void *stream);
/*
 * The same for FP8 E4M3 codes (tcgen05.mma kind::f8f6f4, FP32 accumulation):
 * out[i][b] = sum_t e4m3(A[i][t]) * e4m3(U[b][t]), no scales -- the deep term
 * of the batched scan over an FP8 table before its per-row scales (Eq. 1).
 * A: device [n][d] codes, U: device [B][d] codes, out: device [n][B] FP32;
 * d in {64, 128}, B a multiple of 32 in 32..256.  Synchronous.
 */
int ebr_debug_gemm_e4m3(const uint8_t *A, uint32_t n, const uint8_t *U, uint32_t B, uint32_t d,
                        float *out, void *stream);

/*
 * Failure-detection check (no paper counterpart): launches one CTA whose
 * thread waits, with the library's bounded-wait routine, on an mbarrier that
 * nothing ever arrives on, giving up after timeout_us microseconds (1 .. 10^6).
 * Returns EBR_ETIMEDOUT when the wait ran out and was reported through the
 * device flag word, as every bounded wait in the library reports it; the CUDA
 * context stays usable.  Synchronous.
 */
int ebr_debug_wait_timeout(uint32_t timeout_us, void *stream);

/* ------------------------------------------------------- no-allocation form */
/*
 * Allocation-free scan + top-K.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc -- a serving process
 * whose device memory is owned up front by another allocator (a framework's
 * caching pool or a fixed HBM budget), or a latency-critical thread that
 * cannot afford cudaMalloc's implicit device-wide synchronisation.
 *
 * Computes s[a] = <h_u, emb[a]> (+ wide[a] when wide != NULL) for every ad
 * and returns the k best, like ebr_score_topk: out_ids/out_scores[k] by score
 * descending then id ascending, padded with (0xFFFFFFFF, -inf) past the
 * number of eligible ads.  All pointers are device pointers on `device`:
 * emb [n_ads][d] FP32 row-major, h_u [d], wide [n_ads] or NULL, filter
 * (bit a of word a >> 6 keeps ad a) or NULL.  d is 4, 8, 16, 32, 64 or 128;
 * 1 <= k <= 1024, larger k returns EBR_EINVAL.  emb must start on a 16-byte
 * boundary (its rows are staged by bulk copies); a misaligned emb returns
 * EBR_EINVAL before anything is launched.
 *
 * It allocates nothing: its scratch is a static device array of 1.25 MiB
 * (candidates of up to 160 CTAs x 1024, plus a 64-byte control block), held by
 * every GPU that loads this library until the process exits.  The first call
 * on a device looks up that array's device address (cudaGetSymbolAddress),
 * so make the first call on each device before any stream capture; the
 * lookup is repeated when the device's context has been replaced (after
 * cudaDeviceReset).  Every
 * call clears the control block and reuses the array, so calls whose work
 * overlaps on the GPU (different streams, or different host threads without
 * ordering) race and corrupt each other's results; order them on one stream.
 * Stream-ordered: returns before the GPU is done; device-side status is not
 * reported, so a scan whose bounded device waits ran out (2 s) can leave an
 * incomplete top-K in the outputs with no error returned.
 */
int ebr_scan_topk_noalloc(const float *emb, uint32_t n_ads, uint32_t d, const float *h_u,
                          const float *wide, const uint64_t *filter, uint32_t k,
                          uint32_t *out_ids, float *out_scores, int device, void *stream);

/* ------------------------------------------------------------ profiling */
/*
 * Per-stage device time of ebr_score_topk calls on one index, measured with
 * CUDA events recorded on the caller's stream around each stage:
 * query expansion, the wide term (Algorithm 2), the streaming scan with the
 * fused add + per-CTA top-K, and the final selection (+ FP32 rescoring).
 * ebr_profile_enable resets the counters; ebr_profile_read waits for the
 * recorded events and returns the sums.  Disabled by default.
 */
typedef struct {
  uint64_t calls;          /* requests profiled */
  uint64_t launches;       /* kernels of this library launched by those requests */
  uint64_t lib_launches;   /* device-library kernels launched: always 0 (none are used) */
  double ms_expand, ms_wide, ms_scan, ms_final;
  uint64_t batched;        /* requests served by the batched tensor-core scan */
  uint64_t recomputed;     /* of those, recomputed by the single-request scan because the
                              batched candidate buffers could not prove exactness */
  uint64_t batch_calls;    /* batched calls profiled */
  double ms_batch_stage;   /* staging + expansion into user-minor weights */
  double ms_batch_scan;    /* k_batch_window: tensor-core deep term + wide term + per-CTA top-m */
  double ms_batch_merge;   /* k_batch_merge: per-user merge, FP32 rescoring, final K */
  uint64_t auto_routed;    /* sparse key lists whose traversal the device chose */
  uint64_t window_routed;  /* of those, decoded window by window (the rest: Algorithm 2) */
} ebr_profile;
int ebr_profile_enable(ebr_index *ix, int on);
int ebr_profile_read(ebr_index *ix, ebr_profile *out);

/* ------------------------------------------------------------------ serving
 * Continuous-batching request loop over one index (the serving form of the
 * method's query, Algorithm 2 plus the dual-tower term of Eq. 1, for many
 * concurrent users; the paper itself gives no serving design).
 *
 * ebr_submit copies a host request into a device-resident slot (the copy
 * runs on the server's copy stream) and queues it.  By default (an index the
 * batched scan takes, host_driven = 0) the waves run in a device-resident
 * loop: one graph launch whose WHILE node, on the device, waits with a
 * bounded poll for the next wave a worker thread posted (up to max_batch
 * queued users; one wave at a time, the next formed while it runs), stages it from its slots, runs the
 * batched scan and merge and publishes the results; the loop leaves after
 * about 0.2 s without work and is relaunched on demand.  With host_driven =
 * 1 (and for FP32 indexes) the worker launches whatever is queued as one
 * batched scan as soon as one of two pipelines is free, so a batch is being
 * staged and launched while the previous one is still on the GPU.  ebr_poll
 * returns the result once it is visible on the host.
 *
 * Admission is by device memory: every slot holds a request's inputs (user
 * vector, user field values, targeting bitmap) in HBM, and the slots plus the
 * two pipelines' workspaces must fit `hbm_budget`.  A submit with no free
 * slot is refused with EBR_ENOMEM (the caller retries after polling).
 *
 * The index must not be used by other calls while a server runs on it.
 */
typedef struct ebr_server ebr_server;
typedef struct {
  uint64_t hbm_budget;        /* device bytes for slots + workspaces (0: half of the free memory) */
  uint32_t max_batch;         /* users per batched scan, 1..256 (0: 64) */
  uint32_t max_slots;         /* admitted requests at once, queued + running (0: 4 * max_batch) */
  uint32_t k_max;             /* largest K a request may ask for (0: 1000) */
  uint32_t queue_timeout_ms;  /* a request still queued after this long fails with EBR_ETIMEDOUT (0: never) */
  uint32_t max_user_vals;     /* user field values one request may carry, multi-valued (user_ptr)
                                 requests included; sizes every slot (0: 8 * f_u) */
  uint32_t host_driven;       /* 1: the worker thread launches every batch on two pipelines;
                                 0: the device-resident loop (indexes the batched scan takes) */
} ebr_server_cfg;

typedef struct {
  uint64_t submitted, admitted, rejected, completed, failed, batches, batched_requests;
  double p50_ms, p99_ms, mean_ms;   /* submit -> result visible, over up to the last 65536 requests */
  uint32_t max_batch, max_slots;    /* effective values after the HBM budget */
  uint64_t device_bytes;            /* device memory held by slots and workspaces */
  uint64_t slot_bytes;              /* device bytes of one request slot */
  double launch_ms, finish_ms;      /* worker host time staging+launching / waiting+publishing */
  uint64_t index_swaps;             /* indexes swapped in by ebr_server_swap_index */
  uint64_t loop_launches;           /* launches of the device-resident loop (it leaves when idle) */
} ebr_server_stats;

/*
 * cross: the cross model whose user field values the requests carry
 * (required: requests are given as raw user fields, expanded on the device).
 * Returns EBR_ENOMEM if not even one batch of one request fits the budget.
 */
int ebr_server_create(ebr_index *ix, const ebr_cross *cross, const ebr_server_cfg *cfg,
                      ebr_server **out);
/*
 * q: HOST pointers (h_u[d], user_vals[f_u], optional filter bitmap of
 * ceil(N/64) words); q->k in 1..k_max; q_key/q_w are not accepted here.
 * A multi-valued request (user_ptr[f_u + 1], user_vals[n_user_vals], as in
 * ebr_query) may carry up to the server's max_user_vals values; its offsets
 * and values are checked here (EBR_EINVAL), like the single-valued fields.
 * The request is copied before the call returns.  *ticket identifies it.
 */
int ebr_submit(ebr_server *s, const ebr_query *q, uint64_t *ticket);
/*
 * EBR_EAGAIN while pending; EBR_OK with ids[k], scores[k] (host) filled and
 * the ticket retired; the request's error code (ticket retired) if it
 * failed; EBR_EINVAL for an unknown or already retired ticket.
 */
int ebr_poll(ebr_server *s, uint64_t ticket, uint32_t *ids, float *scores);
int ebr_server_get_stats(ebr_server *s, ebr_server_stats *out);
/* Clears the counters and the latency record (e.g. after a warm-up). */
int ebr_server_reset_stats(ebr_server *s);
/*
 * Tickets of requests that finished (done or failed) since the previous
 * call, up to cap of them (the rest are kept for the next call); lets a
 * client poll only what is ready.
 */
int ebr_server_completed(ebr_server *s, uint64_t *tickets, uint32_t cap, uint32_t *n);
/*
 * Serve every request not yet launched from `next` instead (the production
 * mode of Sec. 3.4 and Sec. 4.3: the index is rebuilt from an updated
 * feature->ad map L with ebr_build_index, off the serving loop, then swapped
 * in without stopping it).  `next` must have the served index's n_ads,
 * n_keys, d, embedding dtype and device, and fit the server's cross model.
 * Batches already launched finish on the old index; no new batch starts
 * until they have, so the call blocks for at most about one batch.  When it
 * returns, the server no longer uses the old index and the caller may free
 * it; the server never owns an index.  Requests keep their tickets across a
 * swap.  Concurrent calls run one after another.  A call still waiting when
 * ebr_server_destroy runs returns EBR_EINVAL ("the server was destroyed"),
 * and destroy waits for it to return before freeing the server; a call made
 * after destroy has begun is a use after free.  Errors: EBR_EINVAL (null,
 * shape mismatch, server destroyed), EBR_ENOMEM (workspace of `next`).
 */
int ebr_server_swap_index(ebr_server *s, ebr_index *next);
/*
 * Stops the worker (requests still pending are dropped), waits for swap
 * calls in progress to return, and frees everything.
 */
int ebr_server_destroy(ebr_server *s);

#ifdef __cplusplus
}
#endif
#endif /* EBR_H */
