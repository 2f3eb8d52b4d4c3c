// Continuous-batching request loop (ebr_server_*, ebr_submit, ebr_poll).
//
// Requests arrive on any host thread and are copied into device-resident
// slots on a copy stream.  Two ways of running them:
//  - the device-resident loop (default for indexes the batched scan takes):
//    one graph launch whose conditional WHILE node runs waves back to back
//    on the device.  Each iteration waits (bounded, on host-written words in
//    mapped memory) for the next wave the worker thread posted, stages the
//    wave's requests from their slots, runs the batched scan and merge into
//    a ring slot of results and publishes it.  The worker thread only posts
//    waves (up to max_batch queued requests each; one running and one
//    waiting, as many as the host-driven form keeps in flight, so that a
//    request waits behind at most two waves) and takes finished ones back;
//    the loop leaves after a while without work and is relaunched on demand;
//  - host-driven pipelines: the worker thread keeps two pipelines (workspace
//    + stream each) and launches all queued requests (up to max_batch) as
//    one batched scan whenever one is free, finishing the oldest otherwise.
// Either way, requests that arrive while others are on the GPU join the
// next wave.  Admission is by device memory: the slots and the workspaces
// are allocated up front from the HBM budget, and a submit finding no free
// slot is refused.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ebr_internal.cuh"

namespace ebr {

namespace {

enum SlotState { kFree = 0, kQueued, kRunning, kDone, kFailed };

struct Slot {
  SlotState state = kFree;
  uint64_t ticket = 0;
  uint32_t k = 0;
  bool has_filter = false;
  double t_submit = 0.0;
  int rc = EBR_OK;
  std::string err;
  uint32_t n_uv = 0;       // user field values held (f_u when single-valued)
  bool has_ptr = false;    // multi-valued: field offsets in d_uptr
  float *d_hu = nullptr;
  uint32_t *d_uv = nullptr;    // [max_user_vals]
  uint32_t *d_uptr = nullptr;  // [f_u + 1]
  uint64_t *d_filter = nullptr;
  float *h_hu = nullptr;
  uint32_t *h_uv = nullptr;    // [max_user_vals], then the offsets [f_u + 1]
  uint64_t *h_filter = nullptr;
  uint32_t *h_ids = nullptr;
  float *h_scores = nullptr;
  cudaEvent_t copied = nullptr;
};

struct Pipe {
  BatchWs ws;
  cudaStream_t st = nullptr;
  DevBuf out;                  // ids [max_batch][k_max] then scores
  uint32_t *h_ids = nullptr;   // pinned copies of the outputs
  float *h_scores = nullptr;
  std::vector<int> slots;
  std::vector<ebr_query> qs;
  uint32_t kmax = 0;
  bool busy = false;
  bool single = false;  // ran on the single-request scan (already complete)
};

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

size_t round256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

}  // namespace ebr

using namespace ebr;

struct ebr_server {
  ebr_index *ix = nullptr;       // read and replaced by the worker thread only
  ebr_index *next_ix = nullptr;  // an index waiting to replace ix (under mu)
  bool swap_req = false;         // next_ix is set; no batch is launched until it is in
  std::condition_variable swap_cv;
  std::mutex swap_mu;            // one ebr_server_swap_index at a time
  uint32_t swappers = 0;         // swap calls inside the server (under mu); destroy waits for 0
  const ebr_cross *cross = nullptr;
  int device = 0;
  uint32_t d = 0;                // embedding dimension (the same for every index served)
  uint32_t max_batch = 64, max_slots = 256, k_max = 1000, timeout_ms = 0;
  uint32_t max_user_vals = 0;    // user field values one request may carry
  uint32_t words = 0;
  bool batched_ok = false;
  std::vector<Slot> slots;
  std::vector<int> free_slots;
  std::deque<int> queue;
  std::unordered_map<uint64_t, int> by_ticket;
  uint64_t next_ticket = 1;
  Pipe pipes[2];
  cudaStream_t copy_st = nullptr;
  DevBuf slot_mem;
  void *slot_host = nullptr;
  uint64_t device_bytes = 0, slot_bytes = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::thread worker;
  bool stop = false;
  ebr_server_stats st = {};
  std::vector<float> lat;  // ring of latencies (ms)
  uint64_t lat_n = 0;
  std::deque<uint64_t> finished;  // tickets not yet reported by ebr_server_completed
  // device-resident loop (loop_mode): one graph launch runs the waves
  bool loop_mode = false;
  LoopBufs loop;
  BatchWs loop_ws;
  cudaStream_t loop_st = nullptr, res_st = nullptr;
  cudaEvent_t loop_end = nullptr;
  bool loop_running = false;
  uint64_t loop_posted = 0, loop_done = 0;   // waves posted / taken back (worker thread only)
  std::vector<std::vector<int>> wave_slots;  // [R] slots of each wave in flight
  std::vector<std::vector<ebr_query>> wave_qs;
  uint32_t *h_wave_ids = nullptr;            // pinned [Bmax][k_max]
  float *h_wave_scores = nullptr;
};

namespace ebr {
namespace {

void fail_slots(ebr_server *s, const std::vector<int> &ids, int rc, const std::string &msg) {
  std::lock_guard<std::mutex> lk(s->mu);
  for (int i : ids) {
    Slot &sl = s->slots[i];
    sl.state = kFailed;
    sl.rc = rc;
    sl.err = msg;
    s->st.failed += 1;
    s->finished.push_back(sl.ticket);
  }
}

// Launch the queued requests `take` on pipe p (stream-ordered, no waiting);
// requests that cannot take the batched path run one by one, synchronously.
int pipe_launch(ebr_server *s, int p, const std::vector<int> &take) {
  Pipe &P = s->pipes[p];
  P.slots = take;
  P.qs.assign(take.size(), ebr_query{});
  P.kmax = 0;
  for (size_t i = 0; i < take.size(); i++) {
    Slot &sl = s->slots[take[i]];
    ebr_query &q = P.qs[i];
    q.h_u = sl.d_hu;
    q.user_vals = sl.d_uv;
    q.user_ptr = sl.has_ptr ? sl.d_uptr : nullptr;
    q.n_user_vals = sl.has_ptr ? sl.n_uv : 0;
    q.filter = sl.has_filter ? sl.d_filter : nullptr;
    q.k = sl.k;
    P.kmax = std::max(P.kmax, sl.k);
    EBR_CUDA_TRY(cudaStreamWaitEvent(P.st, sl.copied, 0));
  }
  const uint32_t B = (uint32_t)take.size();
  uint32_t *d_ids = (uint32_t *)P.out.p;
  float *d_scores = (float *)((char *)P.out.p + round256((size_t)s->max_batch * s->k_max * 4));
  if (s->batched_ok && batch_qualifies(s->ix, s->cross, P.qs.data(), B)) {
    EBR_TRY(batch_launch(s->ix, s->cross, P.qs.data(), B, d_ids, d_scores, P.kmax, EBR_IO_DEVICE,
                         P.ws, P.st));
    P.single = false;
    P.busy = true;
    return EBR_OK;
  }
  // one request (or an index the batched scan does not take): the
  // single-request scan, each checked before the next
  P.single = true;
  EBR_TRY(ws_prepare_one(s->ix, s->ix->n_keys, 8192));
  for (uint32_t b = 0; b < B; b++) {
    EBR_TRY(query_one(s->ix, s->cross, P.qs[b], d_ids + (size_t)b * P.kmax,
                      d_scores + (size_t)b * P.kmax, P.kmax, P.st));
    Ctrl hc;
    EBR_CUDA_TRY(cudaMemcpyAsync(&hc, s->ix->ws.ctrl.p, sizeof(Ctrl), cudaMemcpyDeviceToHost, P.st));
    EBR_CUDA_TRY(cudaStreamSynchronize(P.st));
    EBR_TRY(check_device_flags(hc.flags, "ebr_server (single-request scan)"));
  }
  P.busy = true;
  return EBR_OK;
}

int pipe_finish(ebr_server *s, int p) {
  Pipe &P = s->pipes[p];
  const uint32_t B = (uint32_t)P.slots.size();
  uint32_t *d_ids = (uint32_t *)P.out.p;
  float *d_scores = (float *)((char *)P.out.p + round256((size_t)s->max_batch * s->k_max * 4));
  if (!P.single)
    EBR_TRY(batch_finish(s->ix, s->cross, P.qs.data(), B, d_ids, d_scores, P.kmax, P.ws, P.st));
  EBR_CUDA_TRY(cudaMemcpyAsync(P.h_ids, d_ids, (size_t)B * P.kmax * 4, cudaMemcpyDeviceToHost, P.st));
  EBR_CUDA_TRY(
      cudaMemcpyAsync(P.h_scores, d_scores, (size_t)B * P.kmax * 4, cudaMemcpyDeviceToHost, P.st));
  EBR_CUDA_TRY(cudaStreamSynchronize(P.st));
  const double t = now_s();
  std::lock_guard<std::mutex> lk(s->mu);
  for (uint32_t b = 0; b < B; b++) {
    Slot &sl = s->slots[P.slots[b]];
    memcpy(sl.h_ids, P.h_ids + (size_t)b * P.kmax, sl.k * 4);
    memcpy(sl.h_scores, P.h_scores + (size_t)b * P.kmax, sl.k * 4);
    sl.state = kDone;
    s->finished.push_back(sl.ticket);
    const float ms = (float)((t - sl.t_submit) * 1e3);
    s->lat[s->lat_n % s->lat.size()] = ms;
    s->lat_n += 1;
    s->st.completed += 1;
  }
  s->st.batches += 1;
  s->st.batched_requests += B;
  return EBR_OK;
}

void shed_timed_out(ebr_server *s) {  // under s->mu
  if (!s->timeout_ms || s->queue.empty()) return;
  const double t = now_s();
  std::deque<int> keep;
  for (int i : s->queue) {
    Slot &sl = s->slots[i];
    if ((t - sl.t_submit) * 1e3 > s->timeout_ms) {
      sl.state = kFailed;
      sl.rc = EBR_ETIMEDOUT;
      sl.err = "ebr_server: request waited longer than queue_timeout_ms";
      s->st.failed += 1;
      s->finished.push_back(sl.ticket);
    } else {
      keep.push_back(i);
    }
  }
  s->queue.swap(keep);
}

void worker_main(ebr_server *s) {
  cudaSetDevice(s->device);
  std::deque<int> inflight;  // pipes in launch order
  for (;;) {
    int lp = -1;
    std::vector<int> take;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->stop) break;
      shed_timed_out(s);
      if (s->swap_req && inflight.empty()) {  // no batch uses the old index any more
        s->ix = s->next_ix;
        s->next_ix = nullptr;
        s->swap_req = false;
        s->st.index_swaps += 1;
        s->swap_cv.notify_all();
      }
      // while a swap waits, launched batches drain and nothing new starts
      for (int p = 0; p < 2 && lp < 0 && !s->swap_req; p++)
        if (!s->pipes[p].busy) lp = p;
      if (lp >= 0 && !s->queue.empty()) {
        while (!s->queue.empty() && take.size() < s->max_batch) {
          const int i = s->queue.front();
          s->queue.pop_front();
          s->slots[i].state = kRunning;
          take.push_back(i);
        }
      } else if (inflight.empty()) {
        s->cv.wait_for(lk, std::chrono::milliseconds(2));
        continue;
      }
    }
    if (!take.empty()) {
      const double tl0 = now_s();
      const int rc = pipe_launch(s, lp, take);
      {
        std::lock_guard<std::mutex> lk(s->mu);
        s->st.launch_ms += (now_s() - tl0) * 1e3;
      }
      if (rc != EBR_OK) {
        s->pipes[lp].busy = false;
        fail_slots(s, take, rc, ebr_last_error());
      } else {
        inflight.push_back(lp);
      }
      continue;
    }
    const int p = inflight.front();
    inflight.pop_front();
    const double tf0 = now_s();
    const int rc = pipe_finish(s, p);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->st.finish_ms += (now_s() - tf0) * 1e3;
    }
    if (rc != EBR_OK) fail_slots(s, s->pipes[p].slots, rc, ebr_last_error());
    s->pipes[p].busy = false;
  }
  while (!inflight.empty()) {  // let launched work drain before teardown
    cudaStreamSynchronize(s->pipes[inflight.front()].st);
    inflight.pop_front();
  }
}

// ------------------------------------------------- device-resident loop
// The worker posts waves (up to max_batch queued requests each) into the
// loop's descriptor ring and takes finished waves back; the device runs them
// back to back inside one graph launch, relaunched only after the loop left
// on its own for want of work.

// (Re)launches the loop graph unless it is running.
int loop_ensure_running(ebr_server *s) {
  if (s->loop_running) {
    const cudaError_t q = cudaEventQuery(s->loop_end);
    if (q == cudaErrorNotReady) return EBR_OK;
    s->loop_running = false;
    if (q != cudaSuccess) {
      set_error("ebr_server (device loop): %s", cudaGetErrorString(q));
      return EBR_ECUDA;
    }
  }
  EBR_CUDA_TRY(cudaMemsetAsync(s->loop.idle_ns, 0, sizeof(unsigned long long), s->loop_st));
  EBR_CUDA_TRY(cudaGraphLaunch(s->loop.exec, s->loop_st));
  EBR_CUDA_TRY(cudaEventRecord(s->loop_end, s->loop_st));
  s->loop_running = true;
  std::lock_guard<std::mutex> lk(s->mu);
  s->st.loop_launches += 1;
  return EBR_OK;
}

// Asks the running loop to leave and waits for it (its polls are bounded,
// so it leaves within one wave plus one poll period).
void loop_stop(ebr_server *s) {
  if (!s->loop_running) return;
  s->loop.sh->stop = 1u;
  cudaStreamSynchronize(s->loop_st);
  s->loop.sh->stop = 0u;
  s->loop_running = false;
}

int loop_post(ebr_server *s, const std::vector<int> &take) {
  LoopBufs &L = s->loop;
  const uint32_t r = (uint32_t)(s->loop_posted % L.R);
  std::vector<ebr_query> &qs = s->wave_qs[r];
  qs.assign(take.size(), ebr_query{});
  for (size_t i = 0; i < take.size(); i++) {
    Slot &sl = s->slots[take[i]];
    EBR_CUDA_TRY(cudaEventSynchronize(sl.copied));  // the slot's inputs are on the device
    ebr_query &q = qs[i];
    q.h_u = sl.d_hu;
    q.user_vals = sl.d_uv;
    q.user_ptr = sl.has_ptr ? sl.d_uptr : nullptr;
    q.n_user_vals = sl.has_ptr ? sl.n_uv : 0;
    q.filter = sl.has_filter ? sl.d_filter : nullptr;
    q.k = sl.k;
  }
  EBR_TRY(loop_fill(L, s->loop_posted, s->ix, s->cross, qs.data(), (uint32_t)take.size()));
  s->wave_slots[r] = take;
  std::atomic_thread_fence(std::memory_order_release);  // the descriptor before the count
  s->loop_posted += 1;
  L.sh->posted = s->loop_posted;
  return loop_ensure_running(s);
}

// A finished wave: error flags, the users whose exactness the merge could
// not prove recomputed on the single-request scan, results to the slots.
int loop_finish(ebr_server *s, uint32_t r) {
  LoopBufs &L = s->loop;
  const std::vector<int> &take = s->wave_slots[r];
  const uint32_t B = (uint32_t)take.size();
  std::atomic_thread_fence(std::memory_order_acquire);  // the count before the results
  const uint32_t flags = L.flags_out[r];
  EBR_TRY(check_device_flags(flags, "ebr_server (device loop)"));
  uint32_t *d_ids = L.out_ids + (size_t)r * L.Bmax * L.kmax;
  float *d_scores = L.out_scores + (size_t)r * L.Bmax * L.kmax;
  for (uint32_t b = 0; b < B; b++) {
    if (!L.status_out[(size_t)r * L.Bmax + b]) continue;
    EBR_TRY(ws_prepare_one(s->ix, s->ix->n_keys, 8192));
    EBR_TRY(query_one(s->ix, s->cross, s->wave_qs[r][b], d_ids + (size_t)b * L.kmax,
                      d_scores + (size_t)b * L.kmax, L.kmax, s->res_st));
    Ctrl hc;
    EBR_CUDA_TRY(cudaMemcpyAsync(&hc, s->ix->ws.ctrl.p, sizeof(Ctrl), cudaMemcpyDeviceToHost,
                                 s->res_st));
    EBR_CUDA_TRY(cudaStreamSynchronize(s->res_st));
    EBR_TRY(check_device_flags(hc.flags, "ebr_server (single-request recompute)"));
    s->ix->fallbacks += 1;
  }
  EBR_CUDA_TRY(cudaMemcpyAsync(s->h_wave_ids, d_ids, (size_t)B * L.kmax * 4,
                               cudaMemcpyDeviceToHost, s->res_st));
  EBR_CUDA_TRY(cudaMemcpyAsync(s->h_wave_scores, d_scores, (size_t)B * L.kmax * 4,
                               cudaMemcpyDeviceToHost, s->res_st));
  EBR_CUDA_TRY(cudaStreamSynchronize(s->res_st));
  s->ix->batched += B;
  s->ix->launches += 8;  // fetch, staging, quantiser, expansion, window scan, merge, publish (+ memset)
  const double t = now_s();
  std::lock_guard<std::mutex> lk(s->mu);
  for (uint32_t b = 0; b < B; b++) {
    Slot &sl = s->slots[take[b]];
    memcpy(sl.h_ids, s->h_wave_ids + (size_t)b * L.kmax, sl.k * 4);
    memcpy(sl.h_scores, s->h_wave_scores + (size_t)b * L.kmax, sl.k * 4);
    sl.state = kDone;
    s->finished.push_back(sl.ticket);
    const float ms = (float)((t - sl.t_submit) * 1e3);
    s->lat[s->lat_n % s->lat.size()] = ms;
    s->lat_n += 1;
    s->st.completed += 1;
  }
  s->st.batches += 1;
  s->st.batched_requests += B;
  return EBR_OK;
}

// Gives up on the waves in flight (the loop made no progress for
// kStallSeconds): stops the loop, fails their requests and moves the
// device's wave counter past them so that a relaunch does not run them.
constexpr double kStallSeconds = 10.0;
void loop_abandon(ebr_server *s, int rc, const char *why) {
  LoopBufs &L = s->loop;
  loop_stop(s);
  for (uint64_t w = s->loop_done; w < s->loop_posted; w++) {
    fail_slots(s, s->wave_slots[w % L.R], rc, why);
    s->wave_slots[w % L.R].clear();
  }
  const unsigned long long posted = s->loop_posted;
  cudaMemcpyAsync(L.seq, &posted, sizeof(posted), cudaMemcpyHostToDevice, s->loop_st);
  cudaStreamSynchronize(s->loop_st);
  s->loop_done = s->loop_posted;
  L.sh->done = posted;
  L.sh->freed = posted;
}

void worker_loop_main(ebr_server *s) {
  cudaSetDevice(s->device);
  LoopBufs &L = s->loop;
  double progress = now_s();  // last wave posted or taken back
  for (;;) {
    // waves the device finished
    const uint64_t done = L.sh->done;
    if (s->loop_done < done) progress = now_s();
    while (s->loop_done < done) {
      const uint32_t r = (uint32_t)(s->loop_done % L.R);
      const double tf0 = now_s();
      const int rc = loop_finish(s, r);
      if (rc != EBR_OK) fail_slots(s, s->wave_slots[r], rc, ebr_last_error());
      s->wave_slots[r].clear();
      s->loop_done += 1;
      std::atomic_thread_fence(std::memory_order_release);
      L.sh->freed = s->loop_done;  // the wave's result slot may be reused
      std::lock_guard<std::mutex> lk(s->mu);
      s->st.finish_ms += (now_s() - tf0) * 1e3;
    }
    const bool inflight = s->loop_posted > s->loop_done;
    std::vector<int> take;
    bool swap_now = false;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->stop && !inflight) break;
      shed_timed_out(s);
      if (s->swap_req && !inflight) {
        swap_now = true;
      } else if (!s->swap_req && !s->stop && !s->queue.empty() &&
                 s->loop_posted - s->loop_done < L.ahead) {
        while (!s->queue.empty() && take.size() < s->max_batch) {
          const int i = s->queue.front();
          s->queue.pop_front();
          s->slots[i].state = kRunning;
          take.push_back(i);
        }
      } else if (!inflight) {
        s->cv.wait_for(lk, std::chrono::milliseconds(2));
        continue;
      }
    }
    if (swap_now) {  // no wave uses the old index: leave the loop, rebuild it for the new one
      loop_stop(s);
      ebr_index *nx = nullptr;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        nx = s->next_ix;
      }
      const int rc = loop_build(nx, s->cross, s->max_user_vals, s->loop_ws, L, s->loop_st);
      std::lock_guard<std::mutex> lk(s->mu);
      if (rc == EBR_OK) {
        s->ix = nx;
        s->st.index_swaps += 1;
      } else {  // keep serving the old index: rebuild its graph
        loop_build(s->ix, s->cross, s->max_user_vals, s->loop_ws, L, s->loop_st);
      }
      s->next_ix = nullptr;
      s->swap_req = false;
      s->swap_cv.notify_all();
      continue;
    }
    if (!take.empty()) {
      const double tl0 = now_s();
      progress = tl0;
      const int rc = loop_post(s, take);
      if (rc != EBR_OK) fail_slots(s, take, rc, ebr_last_error());
      std::lock_guard<std::mutex> lk(s->mu);
      s->st.launch_ms += (now_s() - tl0) * 1e3;
      continue;
    }
    // waves on the device: keep the loop running and look again shortly
    if (loop_ensure_running(s) != EBR_OK) {  // the loop failed: its waves fail
      loop_abandon(s, EBR_ECUDA, ebr_last_error());
      continue;
    }
    if (now_s() - progress > kStallSeconds) {
      loop_abandon(s, EBR_ETIMEDOUT, "ebr_server: the device loop made no progress");
      progress = now_s();
      continue;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  loop_stop(s);
}

void server_free(ebr_server *s) {
  for (Pipe &P : s->pipes) {
    batch_ws_free(P.ws);
    dev_free(P.out);
    if (P.h_ids) cudaFreeHost(P.h_ids);
    if (P.h_scores) cudaFreeHost(P.h_scores);
    if (P.st) cudaStreamDestroy(P.st);
  }
  loop_free(s->loop);
  batch_ws_free(s->loop_ws);
  if (s->h_wave_ids) cudaFreeHost(s->h_wave_ids);
  if (s->h_wave_scores) cudaFreeHost(s->h_wave_scores);
  if (s->loop_end) cudaEventDestroy(s->loop_end);
  if (s->loop_st) cudaStreamDestroy(s->loop_st);
  if (s->res_st) cudaStreamDestroy(s->res_st);
  for (Slot &sl : s->slots)
    if (sl.copied) cudaEventDestroy(sl.copied);
  dev_free(s->slot_mem);
  if (s->slot_host) cudaFreeHost(s->slot_host);
  if (s->copy_st) cudaStreamDestroy(s->copy_st);
  delete s;
}

// Reserve every buffer a batch of B users with K up to kmax can touch, so
// that serving allocates nothing after creation.
int pipe_reserve(ebr_server *s, Pipe &P) {
  ebr_index *ix = s->ix;
  const uint32_t B = s->max_batch;
  const uint32_t kscan = std::min<uint32_t>(s->k_max * ix->rescore_mult, ix->n_ads);
  if (s->batched_ok)
    EBR_TRY(batch_ws_reserve(ix, s->cross, B, kscan, (uint64_t)B * s->max_user_vals, P.ws));
  const size_t ob = round256((size_t)B * s->k_max * 4);
  EBR_TRY(dev_reserve(P.out, 2 * ob));
  if (cudaMallocHost((void **)&P.h_ids, (size_t)B * s->k_max * 4) != cudaSuccess ||
      cudaMallocHost((void **)&P.h_scores, (size_t)B * s->k_max * 4) != cudaSuccess) {
    cudaGetLastError();
    set_error("ebr_server_create: pinned host allocation failed");
    return EBR_ENOMEM;
  }
  EBR_CUDA_TRY(cudaStreamCreateWithFlags(&P.st, cudaStreamNonBlocking));
  return EBR_OK;
}

}  // namespace
}  // namespace ebr

extern "C" int ebr_server_create(ebr_index *ix, const ebr_cross *cross, const ebr_server_cfg *cfg,
                                 ebr_server **out) {
  clear_error();
  if (!ix || !cross || !out) {
    set_error("ebr_server_create: null argument");
    return EBR_EINVAL;
  }
  if (cross->n_keys != ix->n_keys) {
    set_error("ebr_server_create: cross model has %u keys, index has %u", cross->n_keys,
              ix->n_keys);
    return EBR_EINVAL;
  }
  ebr_server_cfg c = cfg ? *cfg : ebr_server_cfg{};
  if (c.max_batch == 0) c.max_batch = 64;
  if (c.k_max == 0) c.k_max = 1000;
  if (c.max_batch > 256 || c.k_max > 8192 ||
      (ix->dtype != EBR_F32 && (uint64_t)c.k_max * ix->rescore_mult > 8192)) {
    set_error("ebr_server_create: max_batch must be <= 256 and k_max <= 8192 (R*k_max <= 8192 "
              "for BF16/FP8 indexes)");
    return EBR_EINVAL;
  }
  int prev = 0;
  cudaGetDevice(&prev);
  EBR_CUDA_TRY(cudaSetDevice(ix->device));
  ebr_server *s = new ebr_server();
  s->ix = ix;
  s->d = ix->d;
  s->cross = cross;
  s->device = ix->device;
  s->k_max = c.k_max;
  s->timeout_ms = c.queue_timeout_ms;
  s->words = (ix->n_ads + 63) / 64;
  // admission budget: slots + two pipelines must fit
  uint64_t budget = c.hbm_budget;
  if (budget == 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    budget = fr / 2;
  }
  s->max_user_vals = std::max(c.max_user_vals ? c.max_user_vals : 8 * cross->f_u, cross->f_u);
  const size_t uv_bytes = round256((size_t)(s->max_user_vals + cross->f_u + 1) * 4);
  s->slot_bytes = round256((size_t)s->words * 8) + round256((size_t)ix->d * 4) + uv_bytes;
  const uint32_t kscan = std::min<uint32_t>(c.k_max * ix->rescore_mult, ix->n_ads);
  s->batched_ok = c.max_batch >= 2 && batch_index_ok(ix, cross, std::min<uint32_t>(c.max_batch, 256)) &&
                  (uint64_t)c.k_max * ix->rescore_mult <= 8192;
  s->loop_mode = s->batched_ok && !c.host_driven;
  uint32_t mb = c.max_batch;
  // workspaces: the device loop's (one batch workspace and its result ring),
  // or two host-driven pipelines
  auto pipes_bytes = [&](uint32_t B) {
    const size_t ws = s->batched_ok ? batch_ws_bytes(ix, cross, std::max<uint32_t>(B, 2), kscan,
                                                     (uint64_t)std::max<uint32_t>(B, 2) *
                                                         s->max_user_vals)
                                    : 0;
    if (s->loop_mode) return ws + loop_dev_bytes(B, c.k_max);
    return 2 * (ws + 2 * round256((size_t)B * c.k_max * 4));
  };
  while (mb > 1 && pipes_bytes(mb) + (uint64_t)mb * s->slot_bytes > budget) mb >>= 1;
  if (pipes_bytes(mb) + (uint64_t)mb * s->slot_bytes > budget) {
    set_error("ebr_server_create: HBM budget of %llu bytes holds no batch (one request needs "
              "%llu)",
              (unsigned long long)budget,
              (unsigned long long)(pipes_bytes(1) + s->slot_bytes));
    delete s;
    cudaSetDevice(prev);
    return EBR_ENOMEM;
  }
  s->max_batch = mb;
  uint64_t n_slots = (budget - pipes_bytes(mb)) / s->slot_bytes;
  const uint32_t want = c.max_slots ? c.max_slots : 4 * mb;
  n_slots = std::min<uint64_t>(n_slots, want);
  s->max_slots = (uint32_t)std::max<uint64_t>(n_slots, 1);
  s->lat.assign(65536, 0.f);
  // slots: device memory and pinned host staging
  int rc = dev_alloc(s->slot_mem, (size_t)s->max_slots * s->slot_bytes);
  const size_t host_slot = round256((size_t)s->words * 8) + round256((size_t)ix->d * 4) +
                           uv_bytes + 2 * round256((size_t)c.k_max * 4);
  if (rc == EBR_OK && cudaMallocHost(&s->slot_host, (size_t)s->max_slots * host_slot) != cudaSuccess) {
    cudaGetLastError();
    set_error("ebr_server_create: pinned host allocation failed");
    rc = EBR_ENOMEM;
  }
  if (rc == EBR_OK && cudaStreamCreateWithFlags(&s->copy_st, cudaStreamNonBlocking) != cudaSuccess) {
    set_error("ebr_server_create: stream creation failed");
    rc = EBR_ECUDA;
  }
  if (rc == EBR_OK) {
    s->slots.resize(s->max_slots);
    for (uint32_t i = 0; i < s->max_slots; i++) {
      Slot &sl = s->slots[i];
      char *dp = (char *)s->slot_mem.p + (size_t)i * s->slot_bytes;
      sl.d_filter = (uint64_t *)dp;
      sl.d_hu = (float *)(dp + round256((size_t)s->words * 8));
      sl.d_uv = (uint32_t *)(dp + round256((size_t)s->words * 8) + round256((size_t)ix->d * 4));
      sl.d_uptr = sl.d_uv + s->max_user_vals;
      char *hp = (char *)s->slot_host + (size_t)i * host_slot;
      sl.h_filter = (uint64_t *)hp;
      hp += round256((size_t)s->words * 8);
      sl.h_hu = (float *)hp;
      hp += round256((size_t)ix->d * 4);
      sl.h_uv = (uint32_t *)hp;
      hp += uv_bytes;
      sl.h_ids = (uint32_t *)hp;
      hp += round256((size_t)c.k_max * 4);
      sl.h_scores = (float *)hp;
      if (cudaEventCreateWithFlags(&sl.copied, cudaEventDisableTiming) != cudaSuccess) {
        set_error("ebr_server_create: event creation failed");
        rc = EBR_ECUDA;
        break;
      }
      s->free_slots.push_back((int)(s->max_slots - 1 - i));
    }
  }
  if (!s->loop_mode) {
    for (int p = 0; p < 2 && rc == EBR_OK; p++) rc = pipe_reserve(s, s->pipes[p]);
  } else if (rc == EBR_OK) {
    rc = loop_alloc(s->loop, mb, c.k_max);
    s->wave_slots.resize(s->loop.R);
    s->wave_qs.resize(s->loop.R);
    if (rc == EBR_OK &&
        (cudaStreamCreateWithFlags(&s->loop_st, cudaStreamNonBlocking) != cudaSuccess ||
         cudaStreamCreateWithFlags(&s->res_st, cudaStreamNonBlocking) != cudaSuccess ||
         cudaEventCreateWithFlags(&s->loop_end, cudaEventDisableTiming) != cudaSuccess)) {
      set_error("ebr_server_create: stream creation failed");
      rc = EBR_ECUDA;
    }
    if (rc == EBR_OK &&
        (cudaMallocHost((void **)&s->h_wave_ids, (size_t)mb * c.k_max * 4) != cudaSuccess ||
         cudaMallocHost((void **)&s->h_wave_scores, (size_t)mb * c.k_max * 4) != cudaSuccess)) {
      cudaGetLastError();
      set_error("ebr_server_create: pinned host allocation failed");
      rc = EBR_ENOMEM;
    }
    if (rc == EBR_OK) rc = ws_prepare_one(ix, ix->n_keys, 8192);  // recomputes allocate nothing
    if (rc == EBR_OK) rc = loop_build(ix, cross, s->max_user_vals, s->loop_ws, s->loop, s->loop_st);
  }
  if (rc != EBR_OK) {
    server_free(s);
    cudaSetDevice(prev);
    return rc;
  }
  s->device_bytes = (uint64_t)s->max_slots * s->slot_bytes + pipes_bytes(mb);
  s->worker = std::thread(s->loop_mode ? worker_loop_main : worker_main, s);
  cudaSetDevice(prev);
  *out = s;
  return EBR_OK;
}

extern "C" int ebr_submit(ebr_server *s, const ebr_query *q, uint64_t *ticket) {
  clear_error();
  if (!s || !q || !ticket || !q->h_u || !q->user_vals) {
    set_error("ebr_submit: needs a server, h_u and user_vals (host pointers) and a ticket");
    return EBR_EINVAL;
  }
  if (q->k == 0 || q->k > s->k_max || q->q_key || q->q_w) {
    set_error("ebr_submit: k must be 1..%u; q_key/q_w are not accepted", s->k_max);
    return EBR_EINVAL;
  }
  const uint32_t fu = s->cross->f_u;
  const uint32_t n_uv = q->user_ptr ? q->n_user_vals : fu;
  if (q->user_ptr) {
    if (n_uv > s->max_user_vals) {
      set_error("ebr_submit: %u user field values exceed the server's max_user_vals of %u", n_uv,
                s->max_user_vals);
      return EBR_EINVAL;
    }
    for (uint32_t f = 0; f <= fu; f++)
      if ((f == 0 && q->user_ptr[0] != 0) || (f > 0 && q->user_ptr[f] < q->user_ptr[f - 1]) ||
          (f == fu && q->user_ptr[f] != n_uv)) {
        set_error("ebr_submit: user_ptr must start at 0, not decrease and end at n_user_vals");
        return EBR_EINVAL;
      }
  }
  for (uint32_t f = 0; f < fu; f++) {
    const uint32_t r0 = q->user_ptr ? q->user_ptr[f] : f, r1 = q->user_ptr ? q->user_ptr[f + 1] : f + 1;
    for (uint32_t r = r0; r < r1; r++)
      if (q->user_vals[r] >= s->cross->vocab_u_host[f]) {
        set_error("ebr_submit: user field %u value %u outside its vocabulary of %u", f,
                  q->user_vals[r], s->cross->vocab_u_host[f]);
        return EBR_EINVAL;
      }
  }
  int i = -1;
  uint64_t t = 0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->st.submitted += 1;
    if (s->free_slots.empty()) {
      s->st.rejected += 1;
      set_error("ebr_submit: admission refused, all %u device slots are in use", s->max_slots);
      return EBR_ENOMEM;
    }
    i = s->free_slots.back();
    s->free_slots.pop_back();
    t = s->next_ticket++;
  }
  Slot &sl = s->slots[i];
  sl.ticket = t;
  sl.k = q->k;
  sl.has_filter = q->filter != nullptr;
  sl.rc = EBR_OK;
  sl.err.clear();
  sl.t_submit = now_s();
  sl.n_uv = n_uv;
  sl.has_ptr = q->user_ptr != nullptr;
  memcpy(sl.h_hu, q->h_u, (size_t)s->d * 4);
  memcpy(sl.h_uv, q->user_vals, (size_t)n_uv * 4);
  if (sl.has_ptr) memcpy(sl.h_uv + s->max_user_vals, q->user_ptr, (size_t)(fu + 1) * 4);
  if (sl.has_filter) memcpy(sl.h_filter, q->filter, (size_t)s->words * 8);
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  cudaError_t e = cudaMemcpyAsync(sl.d_hu, sl.h_hu, (size_t)s->d * 4, cudaMemcpyHostToDevice,
                                  s->copy_st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(sl.d_uv, sl.h_uv, (size_t)n_uv * 4, cudaMemcpyHostToDevice, s->copy_st);
  if (e == cudaSuccess && sl.has_ptr)
    e = cudaMemcpyAsync(sl.d_uptr, sl.h_uv + s->max_user_vals, (size_t)(fu + 1) * 4,
                        cudaMemcpyHostToDevice, s->copy_st);
  if (e == cudaSuccess && sl.has_filter)
    e = cudaMemcpyAsync(sl.d_filter, sl.h_filter, (size_t)s->words * 8, cudaMemcpyHostToDevice,
                        s->copy_st);
  if (e == cudaSuccess) e = cudaEventRecord(sl.copied, s->copy_st);
  cudaSetDevice(prev);
  std::lock_guard<std::mutex> lk(s->mu);
  if (e != cudaSuccess) {
    sl.state = kFree;
    s->free_slots.push_back(i);
    set_error("ebr_submit: %s", cudaGetErrorString(e));
    return EBR_ECUDA;
  }
  sl.state = kQueued;
  s->by_ticket[t] = i;
  s->queue.push_back(i);
  s->st.admitted += 1;
  *ticket = t;
  s->cv.notify_one();
  return EBR_OK;
}

extern "C" int ebr_poll(ebr_server *s, uint64_t ticket, uint32_t *ids, float *scores) {
  clear_error();
  if (!s) {
    set_error("ebr_poll: null server");
    return EBR_EINVAL;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->by_ticket.find(ticket);
  if (it == s->by_ticket.end()) {
    set_error("ebr_poll: unknown or retired ticket %llu", (unsigned long long)ticket);
    return EBR_EINVAL;
  }
  Slot &sl = s->slots[it->second];
  if (sl.state == kQueued || sl.state == kRunning) return EBR_EAGAIN;
  int rc = EBR_OK;
  if (sl.state == kDone) {
    if (!ids || !scores) {
      set_error("ebr_poll: null output buffer");
      return EBR_EINVAL;
    }
    memcpy(ids, sl.h_ids, (size_t)sl.k * 4);
    memcpy(scores, sl.h_scores, (size_t)sl.k * 4);
  } else {
    rc = sl.rc;
    set_error("%s", sl.err.c_str());
  }
  sl.state = kFree;
  s->free_slots.push_back(it->second);
  s->by_ticket.erase(it);
  return rc;
}

extern "C" int ebr_server_get_stats(ebr_server *s, ebr_server_stats *out) {
  clear_error();
  if (!s || !out) {
    set_error("ebr_server_get_stats: null argument");
    return EBR_EINVAL;
  }
  std::vector<float> l;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->st;
    const size_t n = (size_t)std::min<uint64_t>(s->lat_n, s->lat.size());
    l.assign(s->lat.begin(), s->lat.begin() + n);
  }
  out->max_batch = s->max_batch;
  out->max_slots = s->max_slots;
  out->device_bytes = s->device_bytes;
  out->slot_bytes = s->slot_bytes;
  out->p50_ms = out->p99_ms = out->mean_ms = 0.0;
  if (!l.empty()) {
    double sum = 0;
    for (float x : l) sum += x;
    out->mean_ms = sum / l.size();
    std::sort(l.begin(), l.end());
    out->p50_ms = l[(size_t)(0.50 * (l.size() - 1) + 0.5)];
    out->p99_ms = l[(size_t)(0.99 * (l.size() - 1) + 0.5)];
  }
  return EBR_OK;
}

extern "C" int ebr_server_reset_stats(ebr_server *s) {
  clear_error();
  if (!s) {
    set_error("ebr_server_reset_stats: null server");
    return EBR_EINVAL;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  s->st = ebr_server_stats{};
  s->lat_n = 0;
  return EBR_OK;
}

extern "C" int ebr_server_completed(ebr_server *s, uint64_t *tickets, uint32_t cap, uint32_t *n) {
  clear_error();
  if (!s || !n || (cap && !tickets)) {
    set_error("ebr_server_completed: null argument");
    return EBR_EINVAL;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  uint32_t c = 0;
  while (c < cap && !s->finished.empty()) {
    tickets[c++] = s->finished.front();
    s->finished.pop_front();
  }
  *n = c;
  return EBR_OK;
}

extern "C" int ebr_server_swap_index(ebr_server *s, ebr_index *next) {
  clear_error();
  if (!s || !next) {
    set_error("ebr_server_swap_index: null argument");
    return EBR_EINVAL;
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      set_error("ebr_server_swap_index: the server was destroyed");
      return EBR_EINVAL;
    }
    s->swappers++;
  }
  // leaves the count (after swap_mu is released: declared before it) and
  // wakes a destroy that waits for the swap calls to return
  struct Leave {
    ebr_server *s;
    ~Leave() {
      std::lock_guard<std::mutex> lk(s->mu);
      s->swappers--;
      s->swap_cv.notify_all();
    }
  } leave{s};
  std::lock_guard<std::mutex> one_swap(s->swap_mu);  // concurrent swaps run one after another
  ebr_index *cur = nullptr;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {  // destroyed while this call waited for the previous swap
      set_error("ebr_server_swap_index: the server was destroyed");
      return EBR_EINVAL;
    }
    cur = s->ix;  // only a swap replaces it, and no other swap runs now
  }
  if (next == cur) return EBR_OK;
  if (next->n_ads != cur->n_ads || next->n_keys != cur->n_keys || next->d != cur->d ||
      next->dtype != cur->dtype || next->device != cur->device) {
    set_error("ebr_server_swap_index: the new index must have the served index's n_ads, "
              "n_keys, d, dtype and device (%u/%u/%u/%d vs %u/%u/%u/%d)",
              next->n_ads, next->n_keys, next->d, (int)next->dtype, cur->n_ads, cur->n_keys,
              cur->d, (int)cur->dtype);
    return EBR_EINVAL;
  }
  // the single-request workspace of the new index, reserved here so that the
  // serving loop still allocates nothing
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  int rc = ws_prepare_one(next, next->n_keys, 8192);
  cudaSetDevice(prev);
  if (rc != EBR_OK) return rc;
  std::unique_lock<std::mutex> lk(s->mu);
  s->next_ix = next;
  s->swap_req = true;
  s->cv.notify_all();
  s->swap_cv.wait(lk, [s] { return !s->swap_req || s->stop; });
  if (s->swap_req) {  // the server stopped first
    s->swap_req = false;
    s->next_ix = nullptr;
    set_error("ebr_server_swap_index: the server was destroyed");
    return EBR_EINVAL;
  }
  return EBR_OK;
}

extern "C" int ebr_server_destroy(ebr_server *s) {
  clear_error();
  if (!s) return EBR_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  s->swap_cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  {
    // swap calls still inside the server see `stop` and return; wait for them
    std::unique_lock<std::mutex> lk(s->mu);
    s->swap_cv.wait(lk, [s] { return s->swappers == 0; });
  }
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  if (s->copy_st) cudaStreamSynchronize(s->copy_st);
  server_free(s);
  cudaSetDevice(prev);
  return EBR_OK;
}
