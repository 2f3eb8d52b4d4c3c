// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <array>
#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "ebr.h"
#include <cuda.h>

namespace ebr {

// ------------------------------------------------------------ error state
void set_error(const char *fmt, ...);
void clear_error();

#define EBR_CUDA_TRY(expr)                                                         \
  do {                                                                             \
    cudaError_t _e = (expr);                                                       \
    if (_e != cudaSuccess) {                                                       \
      ::ebr::set_error("%s failed at %s:%d: %s", #expr, __FILE__, __LINE__,         \
                       cudaGetErrorString(_e));                                    \
      return EBR_ECUDA;                                                            \
    }                                                                              \
  } while (0)

#define EBR_TRY(expr)             \
  do {                            \
    int _rc = (expr);             \
    if (_rc != EBR_OK) return _rc; \
  } while (0)

// Device error flags (bitwise OR of these lands in a device word).
enum : uint32_t {
  DEVERR_BAD_KEY = 1u,        // query key >= n_keys
  DEVERR_BAD_AD = 2u,         // ad id >= n_ads in build input
  DEVERR_BAD_USER = 4u,       // user value >= vocabulary
  DEVERR_TIMEOUT = 8u,        // a bounded wait ran out
  DEVERR_OVERFLOW = 16u,      // a capacity check failed
  DEVERR_BAD_BUILD_KEY = 32u, // key >= n_keys in build input
  DEVERR_RANGE = 64u,         // a non-finite query weight
};

int check_device_flags(uint32_t flags, const char *where);

// RAII-less device buffer helper (explicit free).
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
};
int dev_alloc(DevBuf &b, size_t bytes);
void dev_free(DevBuf &b);
int dev_reserve(DevBuf &b, size_t bytes);  // grow-only

// ---------------------------------------------------------- object layout
constexpr int kGroups = 9;

// Scratch used by one query call on one index.
struct Workspace {
  DevBuf wide;        // float [N] wide-score accumulator (Algorithm 2's score array)
  DevBuf w_dense;     // float [n_keys] expanded query (from user_vals)
  DevBuf wq;          // uint32 [n_keys] packed fixed-point terms of w_dense (fused scan)
  DevBuf lens;        // uint2 [9 * n_q + 1] (units, nonempty) per (group, query entry)
  DevBuf scan;        // uint2 [9 * n_q + 1] exclusive scan of lens
  DevBuf work;        // WorkEntry [9 * n_q] compacted non-empty (group, entry)
  DevBuf scan_tmp;    // tile sums of the scan of lens
  DevBuf cand;        // uint64 [G * KCAP] per-CTA candidates
  DevBuf ctrl;        // Ctrl block (counters, threshold, flags), then at kCtrlBytes the
                      // fused scan's candidate-score histogram (uint32 [kHistWords])
  DevBuf route_stats; // uint64 [2]: sparse lists routed on the device, of those window-major
  DevBuf io_in;       // staging for host inputs
  DevBuf io_out;      // staging for outputs
  void *host_ctrl = nullptr;  // pinned mirror of Ctrl
};

struct Ctrl {
  unsigned long long thr;    // global running K-th key
  unsigned int n_cand;       // candidates appended
  unsigned int flags;        // DEVERR_* bits
  unsigned long long total_units;  // Algorithm 2 work units
  unsigned int n_work;       // compacted work entries
  unsigned int pad;          // fused scan: max |w^| of the request (FP32 bits)
  unsigned int route;        // sparse list: 0 = Algorithm 2 scatter, 1 = window-major decode
  int fx;                    // F of the packed weight terms of the fused scan
};

// Scratch of the batched (tensor-core) path.
struct BatchWs {
  DevBuf users_f32, users_bf16, users_scale, user_vals, wT, filters;  // users_bf16: BF16 or FP8
  DevBuf user_ptr;  // multi-valued users: field offsets [B][f_u + 1], then base [B]
  DevBuf small;  // uint32 [kscan B][kout B][has_filter B], then status [B]
  DevBuf cand, cand_n, cand_thr, scratch;
  DevBuf res;    // device staging of host-bound results
  DevBuf ctrl;   // Ctrl of this batch
  DevBuf req;    // pointer table of device-resident requests (staging gather)
  void *host = nullptr;  // pinned mirror of `small`
  size_t host_bytes = 0;
  bool tmap_ready = false;
  const void *tmap_for = nullptr;
  alignas(64) unsigned char tmap_bytes[128];  // CUtensorMap of the BF16 table
};
void batch_ws_free(BatchWs &w);
// Layout of BatchWs::small for B users: [kscan B][kout B][has_filter B], then
// the per-user status words from a 128-byte boundary.
inline size_t small_status_off(uint32_t B) { return ((size_t)3 * B * 4 + 127) / 128 * 128; }
inline size_t small_bytes(uint32_t B) { return small_status_off(B) + (size_t)B * 4; }

// ------------------------------------------- device-resident serving loop
// One graph launch that runs waves of the batched scan back to back: a
// conditional WHILE node whose body fetches the next posted wave (a bounded
// wait on host-written words), stages it, scans it, merges it into a ring
// slot of results and publishes it; the loop leaves when told to stop or
// after idle_exit_ns without work (the host relaunches it on demand).
struct LoopShared {                     // pinned host memory mapped into the device
  volatile unsigned long long posted;   // host: waves posted
  volatile unsigned long long freed;    // host: waves whose results the host has taken
  volatile unsigned long long done;     // device: waves finished
  volatile uint32_t stop;               // host: leave the loop at the next poll
  uint32_t pad[9];
};
struct LoopBufs {
  uint32_t R = 4, Bmax = 0, kmax = 0, desc_bytes = 0;
  // waves posted and not yet taken back, at most (<= R): one, so that a
  // request that arrives while a wave runs waits for that wave only (with two,
  // p50 at 2 k req/s on 5M BF16 ads was 13.9 ms instead of 8.5 ms, at the
  // same throughput)
  uint32_t ahead = 1;
  void *host = nullptr;           // pinned, mapped: LoopShared, descriptors [R], flags [R], status [R][Bmax]
  LoopShared *sh = nullptr;
  uint8_t *desc = nullptr;        // [R][desc_bytes] wave descriptors (host-written)
  uint32_t *flags_out = nullptr;  // [R] device error flags of each wave (device-written)
  uint32_t *status_out = nullptr; // [R][Bmax] per-user "not proven exact" (device-written)
  DevBuf dev;                     // the device-side state below, one allocation
  uint8_t *cur = nullptr;         // the current wave's descriptor (device copy)
  uint32_t *slot = nullptr;       // its ring slot
  unsigned long long *seq = nullptr, *idle_ns = nullptr;
  uint32_t *status = nullptr;     // [R][Bmax] written by the merge
  uint32_t *out_ids = nullptr;    // [R][Bmax][kmax]
  float *out_scores = nullptr;    // [R][Bmax][kmax]
  Ctrl *ctrl = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t poll_ns = 2000000ull, idle_exit_ns = 200000000ull;
};
int loop_alloc(LoopBufs &L, uint32_t Bmax, uint32_t kmax);
size_t loop_dev_bytes(uint32_t Bmax, uint32_t kmax);  // the device memory loop_alloc takes
void loop_free(LoopBufs &L);
// (Re)builds L's graph for index ix; w is the loop's batch workspace.
int loop_build(ebr_index *ix, const ebr_cross *cross, uint32_t max_user_vals, BatchWs &w,
               LoopBufs &L, cudaStream_t st);
// Writes wave `wave`'s descriptor (ring slot wave % R) from B requests
// whose arrays are device pointers (user_ptr optional).
int loop_fill(LoopBufs &L, uint64_t wave, const ebr_index *ix, const ebr_cross *cross,
              const ebr_query *q, uint32_t B);

}  // namespace ebr

struct ebr_index {
  int device = 0;
  uint32_t n_ads = 0, n_keys = 0, d = 0;
  ebr_dtype dtype = EBR_F32;
  uint32_t rescore_mult = 4;
  uint64_t nnz_unique = 0;
  uint64_t n_blocks[ebr::kGroups] = {0};
  uint32_t *keys[ebr::kGroups] = {nullptr};
  uint32_t *header[ebr::kGroups] = {nullptr};
  uint8_t *values[ebr::kGroups] = {nullptr};
  ebr::DevBuf mem_keys, mem_header, mem_values;
  // Window-major view of the same blocks: per group, blocks ordered by
  // (window h, key k); wkey = key per block, wvals = its 2^g value bytes,
  // win_ptr[g][h] = first block of window h.
  uint32_t n_win = 0;
  uint32_t *wkey[ebr::kGroups] = {nullptr};
  uint8_t *wvals[ebr::kGroups] = {nullptr};
  uint32_t *win_ptr[ebr::kGroups] = {nullptr};
  ebr::DevBuf mem_wkey, mem_wvals, mem_winptr;
  float wm_build_ms = 0.f;
  uint32_t max_win_bytes = 0;   // largest 16-byte-widened window segment total
  uint32_t max_win_chunks = 0;  // most 32-unit work chunks in one window
  uint32_t max_keys_per_ad = 0; // most distinct keys any ad belongs to
  uint32_t max_win_slots = 0;   // most value slots (real + padding) in one window
  ebr::DevBuf ad_nkeys;         // uint16 [N]: distinct keys of each ad (empty if any > 65535)
  ebr::DevBuf emb_f32;    // float [N][d]
  ebr::DevBuf emb_q;      // bf16 / e4m3 [N][d]
  ebr::DevBuf emb_scale;  // float [N] (FP8)
  float build_ms = 0.f;
  int num_sms = 0;
  ebr::Workspace ws;
  ebr::BatchWs bws;
  // profiling (ebr_profile_enable)
  bool prof = false;
  std::vector<std::array<cudaEvent_t, 5>> prof_pending, prof_pool;
  std::vector<std::array<cudaEvent_t, 5>> bprof_pending;  // batched calls (same pool)
  ebr_profile prof_acc = {};
  uint64_t route_base[2] = {0, 0};  // route counters when profiling was (re)enabled
  uint64_t launches = 0, lib_launches = 0;  // counted on every call
  uint64_t batched = 0;    // requests served by the batched scan
  uint64_t fallbacks = 0;  // batched requests recomputed by the single-request scan
};

struct ebr_cross {
  int device = 0;
  // Bound on |w^| of any single-valued request: the largest, over ad fields j,
  // of the sum over j's pairs of the pair's largest |w| (+inf if a weight is
  // not finite); fixes the exponent of the packed terms before w^ is known.
  float wbound = 0.f;
  uint32_t f_u = 0, f_a = 0, n_pairs = 0, n_keys = 0;
  ebr_wkind kind = EBR_W_HASHED;
  uint32_t hash_bits = 24;
  ebr::DevBuf table;       // float [w_len]
  ebr::DevBuf meta;        // packed uint32 metadata (see ebr_query.cu)
  uint64_t w_len = 0;
  // host copies
  std::vector<uint32_t> vocab_u_host;  // user field vocabularies (request checks)
};

namespace ebr {
constexpr int kMaxCtasPerSm = 4;  // bound on scan CTAs per SM (candidate buffer sizing)
int launch_fused(const ebr_index *ix, const float *h_u, const float *w_hat, uint32_t *wq,
                 bool packed, const uint64_t *filter, uint32_t k, uint64_t *cand_out,
                 Ctrl *ctrl, float *all_out, float *wide_out, uint32_t *hist, int max_grid,
                 cudaStream_t st, bool wmax_ready = false, const float *wide_in = nullptr,
                 const uint32_t *route = nullptr, int *n_launched = nullptr,
                 uint64_t *cta_cand = nullptr, size_t cta_cand_entries = 0);
bool fused_fits(const ebr_index *ix, uint32_t k);
constexpr size_t kHistWords = 4096;  // candidate-score histogram of the fused scan (2048 bins + top bin)
constexpr size_t kCtrlBytes = 256;   // Ctrl block, then the histogram, in one buffer (one memset)
inline uint32_t *ws_hist(const Workspace &w) { return (uint32_t *)((char *)w.ctrl.p + kCtrlBytes); }

// Launches kern on st with programmatic stream serialization: it may start
// while the previous kernel of the stream is still running, and its threads
// that read that kernel's results call pdl_wait first.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}
// Launchers implemented in ebr_query.cu, used by the serving loop.
int query_one(const ebr_index *ix, const ebr_cross *cross, const ebr_query &q, uint32_t *ids,
              float *scores, uint32_t kmax, cudaStream_t st);
int ws_prepare_one(ebr_index *ix, uint32_t n_q, uint32_t kcap);
int launch_quantize(const float *x, uint64_t n, ebr_dtype dt, void *out, cudaStream_t st);
int launch_quantize_rows_fp8(const float *x, uint64_t n, uint32_t d, uint8_t *q, float *scale,
                             cudaStream_t st);
// Query expansion for a batch straight into user-minor layout wT[key][Bp].
// uptr/base null: users[b * f_u + i]; else user b's field i holds
// users[base[b] + uptr[b][i] .. base[b] + uptr[b][i + 1]) (checked offsets).
// batch_dev (optional): the users of this wave, read on the device (<= batch).
int expand_transposed(const ebr_cross *c, const uint32_t *users, const uint32_t *uptr,
                      const uint32_t *base, uint32_t batch, uint32_t Bp, float *wT,
                      uint32_t *flags, cudaStream_t st, const uint32_t *batch_dev = nullptr);
// Batched tensor-core path; returns EBR_EINVAL (nothing launched) when the
// batch does not qualify, so the caller can fall back to per-request scans.
bool batch_qualifies(const ebr_index *ix, const ebr_cross *cross, const ebr_query *q,
                     uint32_t batch);
// The index-level part of that test (dtype, dimension, key lists, sizes).
bool batch_index_ok(const ebr_index *ix, const ebr_cross *cross, uint32_t batch);
int query_batch(ebr_index *ix, const ebr_cross *cross, const ebr_query *q, uint32_t batch,
                uint32_t *out_ids, float *out_scores, uint32_t kmax, int io, cudaStream_t st);
// Device bytes of a batched call's workspace (0: the batch does not fit the
// kernel's shared memory), and its reservation (grow-only, with the pinned
// host mirror) for B users and scan depth up to kscan_max;
// n_vals: user field values of the whole batch (0: one per field).
size_t batch_ws_bytes(const ebr_index *ix, const ebr_cross *cross, uint32_t B,
                      uint32_t kscan_max, uint64_t n_vals);
int batch_ws_reserve(const ebr_index *ix, const ebr_cross *cross, uint32_t B,
                     uint32_t kscan_max, uint64_t n_vals, BatchWs &w);
// The same in two halves, for callers that keep several batches in flight:
// batch_launch queues everything on st (w must stay untouched until
// batch_finish returns); batch_finish waits, checks and recomputes.
int batch_launch(ebr_index *ix, const ebr_cross *cross, const ebr_query *q, uint32_t B,
                 uint32_t *d_ids, float *d_scores, uint32_t kmax, int io, BatchWs &w,
                 cudaStream_t st);
int batch_finish(ebr_index *ix, const ebr_cross *cross, const ebr_query *q, uint32_t B,
                 uint32_t *d_ids, float *d_scores, uint32_t kmax, BatchWs &w, cudaStream_t st);
}
