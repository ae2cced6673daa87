// Serving loop: continuous batching of decode requests of mixed code length
// and constellation.
//
// Admission: a request is admitted when a slot is free and its device bytes
// (received symbols, hand-off record, outputs) fit the memory budget; its
// symbols go into a pinned host ring whose device mirror keeps every admitted
// request's received word resident until it completes. A worker thread
// launches the admitted requests as one uneven batch (grand_decode_mixed) on
// the first idle stream as soon as one is idle, so batches that arrive while
// others run overlap on the device. Completed batches are harvested by event
// query; results carry the arrival and completion times (CLOCK_MONOTONIC).
// Ring space is reclaimed in launch order; results are delivered in
// completion order. Every wait is bounded.
#include <errno.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.cuh"

namespace {

constexpr int kMaxStreams = 16;
constexpr int kResultWords = GRAND_N_MAX / 32;

int64_t now_ns() {
  timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (int64_t)ts.tv_sec * 1000000000ll + ts.tv_nsec;
}

int m_of(int M) {
  switch (M) {
    case 4: return 1;
    case 16: return 2;
    case 64: return 3;
    case 256: return 4;
    case 1024: return 5;
    case 4096: return 6;
    default: return 0;
  }
}

struct Req {
  uint64_t tag;
  int64_t arrival_ns;
  int32_t code, M, L, nw;
  int64_t vpos;   // virtual ring position of the first symbol
  int64_t bytes;  // device bytes charged to the budget
};

struct StreamBuf {
  cudaStream_t stream = nullptr;
  grand_frame_desc* d_desc = nullptr;
  grand_frame_desc* h_desc = nullptr;
  uint32_t* d_cw = nullptr;
  uint32_t* h_cw = nullptr;
  uint32_t* d_q = nullptr;
  uint32_t* h_q = nullptr;
  uint8_t* d_ab = nullptr;
  uint8_t* h_ab = nullptr;
  bool busy = false;
};

struct Batch {
  int stream;
  int64_t launch_ns;
  std::vector<Req> reqs;
  int64_t vend;   // ring released up to here once this and all earlier batches are done
  int64_t bytes;
  cudaEvent_t ev;
  bool done;
  int status;
};

}  // namespace

struct grand_server {
  grand_server_cfg cfg;
  std::vector<const grand_code*> codes;
  int device = 0;
  // ring of received symbols (complex64 as float2), virtual positions
  float2* h_ring = nullptr;
  float2* d_ring = nullptr;
  int64_t ring_cap = 0;   // symbols
  int64_t vhead = 0;      // next free virtual position
  int64_t vtail = 0;      // oldest live virtual position
  int64_t live_bytes = 0;
  int32_t live_slots = 0;
  std::vector<StreamBuf> sb;
  std::deque<Req> pending;
  std::deque<Batch> inflight;
  std::deque<grand_result> done;
  std::mutex mu;
  std::condition_variable cv;
  std::thread worker;
  std::atomic<bool> stop{false};
  grand_server_stats st{};
};

namespace {

int64_t request_bytes(int L, int N) { return 8ll * L + (int64_t)sizeof(grand::FrameRec) + 4ll * (N / 32) + 5; }

void free_server(grand_server* s) {
  for (StreamBuf& b : s->sb) {
    if (b.stream) cudaStreamSynchronize(b.stream);
    cudaFree(b.d_desc);
    cudaFree(b.d_cw);
    cudaFree(b.d_q);
    cudaFree(b.d_ab);
    cudaFreeHost(b.h_desc);
    cudaFreeHost(b.h_cw);
    cudaFreeHost(b.h_q);
    cudaFreeHost(b.h_ab);
    if (b.stream) cudaStreamDestroy(b.stream);
  }
  for (Batch& b : s->inflight) cudaEventDestroy(b.ev);
  cudaFree(s->d_ring);
  cudaFreeHost(s->h_ring);
  delete s;
}

// Launch the pending requests (at most max_batch) on stream `si`.
// Called by the worker without the lock held; `reqs` was taken under it.
int launch_batch(grand_server* s, int si, Batch& b) {
  StreamBuf& buf = s->sb[si];
  const int n = (int)b.reqs.size();
  for (int i = 0; i < n; ++i) {
    const Req& r = b.reqs[i];
    buf.h_desc[i].code = r.code;
    buf.h_desc[i].M = r.M;
    buf.h_desc[i].sym_offset = r.vpos % s->ring_cap;
    buf.h_desc[i].cw_offset = (int64_t)i * kResultWords;
  }
  // the symbols of the batch: contiguous in virtual positions, at most two
  // physical pieces (the ring wraps at most once inside a batch)
  const int64_t v0 = b.reqs.front().vpos;
  const int64_t v1 = b.reqs.back().vpos + b.reqs.back().L;
  int64_t v = v0;
  while (v < v1) {
    const int64_t p = v % s->ring_cap;
    const int64_t len = std::min(v1 - v, s->ring_cap - p);
    if (cudaMemcpyAsync(s->d_ring + p, s->h_ring + p, sizeof(float2) * len, cudaMemcpyHostToDevice, buf.stream) !=
        cudaSuccess)
      return GRAND_E_CUDA;
    v += len;
  }
  if (cudaMemcpyAsync(buf.d_desc, buf.h_desc, sizeof(grand_frame_desc) * n, cudaMemcpyHostToDevice, buf.stream) !=
      cudaSuccess)
    return GRAND_E_CUDA;
  int rc = grand_decode_mixed(s->codes.data(), (int)s->codes.size(), &s->cfg.params, buf.d_desc, n, s->d_ring,
                              s->ring_cap, s->cfg.N0, buf.d_cw, (int64_t)n * kResultWords, buf.d_q, buf.d_ab, nullptr,
                              buf.stream);
  if (rc != GRAND_OK) return rc;
  if (cudaMemcpyAsync(buf.h_cw, buf.d_cw, sizeof(uint32_t) * n * kResultWords, cudaMemcpyDeviceToHost, buf.stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(buf.h_q, buf.d_q, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, buf.stream) != cudaSuccess ||
      cudaMemcpyAsync(buf.h_ab, buf.d_ab, n, cudaMemcpyDeviceToHost, buf.stream) != cudaSuccess)
    return GRAND_E_CUDA;
  if (cudaEventRecord(b.ev, buf.stream) != cudaSuccess) return GRAND_E_CUDA;
  return GRAND_OK;
}

void worker_main(grand_server* s) {
  cudaSetDevice(s->device);
  while (!s->stop.load(std::memory_order_acquire)) {
    bool progressed = false;
    // 1. harvest completed batches (any order)
    std::vector<grand_result> out;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      for (Batch& b : s->inflight) {
        if (b.done) continue;
        const cudaError_t q = cudaEventQuery(b.ev);
        if (q == cudaErrorNotReady) continue;
        b.done = true;
        b.status = q == cudaSuccess ? b.status : GRAND_E_CUDA;
        StreamBuf& buf = s->sb[b.stream];
        const int64_t t = now_ns();
        for (size_t i = 0; i < b.reqs.size(); ++i) {
          grand_result r;
          memset(&r, 0, sizeof r);
          r.tag = b.reqs[i].tag;
          r.arrival_ns = b.reqs[i].arrival_ns;
          r.done_ns = t;
          if (b.status == GRAND_OK) {
            r.queries = buf.h_q[i];
            r.abandon = buf.h_ab[i];
            memcpy(r.cw, buf.h_cw + i * kResultWords, sizeof(uint32_t) * b.reqs[i].nw);
          } else {
            r.abandon = 4;  // the batch failed on the device
          }
          s->done.push_back(r);
        }
        s->st.completed += b.reqs.size();
        s->st.batch_service_ns += t - b.launch_ns;
        if (t - b.launch_ns > s->st.max_batch_service_ns) s->st.max_batch_service_ns = t - b.launch_ns;
        if (b.status != GRAND_OK) s->st.errors += 1;
        buf.busy = false;
        progressed = true;
      }
      // reclaim ring space and budget in launch order
      while (!s->inflight.empty() && s->inflight.front().done) {
        Batch& f = s->inflight.front();
        s->vtail = f.vend;
        s->live_bytes -= f.bytes;
        s->live_slots -= (int)f.reqs.size();
        cudaEventDestroy(f.ev);
        s->inflight.pop_front();
      }
    }
    (void)out;
    // 2. launch the pending requests on an idle stream
    for (;;) {
      Batch b;
      int si = -1;
      {
        std::unique_lock<std::mutex> lk(s->mu);
        if (s->pending.empty()) break;
        for (int i = 0; i < (int)s->sb.size(); ++i)
          if (!s->sb[i].busy) { si = i; break; }
        if (si < 0) break;
        const int maxb = s->cfg.max_batch;
        int64_t bytes = 0;
        while (!s->pending.empty() && (int)b.reqs.size() < maxb) {
          bytes += s->pending.front().bytes;
          b.reqs.push_back(s->pending.front());
          s->pending.pop_front();
        }
        b.stream = si;
        b.vend = b.reqs.back().vpos + b.reqs.back().L;
        b.bytes = bytes;
        b.done = false;
        b.status = GRAND_OK;
        s->sb[si].busy = true;
        s->st.batches += 1;
        s->st.batched_frames += b.reqs.size();
      }
      cudaEventCreateWithFlags(&b.ev, cudaEventDisableTiming);
      b.launch_ns = now_ns();
      b.status = launch_batch(s, si, b);
      const int64_t issued = now_ns() - b.launch_ns;
      if (b.status != GRAND_OK) cudaEventRecord(b.ev, s->sb[si].stream);
      {
        std::unique_lock<std::mutex> lk(s->mu);
        s->st.launch_ns += issued;
        if (issued > s->st.max_launch_ns) s->st.max_launch_ns = issued;
        s->inflight.push_back(std::move(b));
        const int64_t inflight = (int64_t)s->inflight.size();
        if (inflight > s->st.max_inflight_batches) s->st.max_inflight_batches = inflight;
      }
      progressed = true;
    }
    if (!progressed) {
      std::unique_lock<std::mutex> lk(s->mu);
      // nothing new: wait briefly for a submit, then poll the events again
      s->cv.wait_for(lk, std::chrono::microseconds(20));
    }
  }
}

}  // namespace

extern "C" int64_t grand_clock_ns(void) { return now_ns(); }

extern "C" int grand_server_create(const grand_server_cfg* cfg, grand_server** out) {
  if (!cfg || !out || !cfg->codes || cfg->n_codes < 1 || cfg->max_slots < 1 || cfg->max_device_bytes < 4096 ||
      cfg->n_streams < 1 || cfg->n_streams > kMaxStreams || cfg->max_batch < 0 || !(cfg->N0 > 0.0f))
    return GRAND_E_INVALID;
  if ((cfg->params.order != GRAND_ORDER_QAM_NNE && cfg->params.order != GRAND_ORDER_QAM_NEARER) ||
      cfg->params.membership != GRAND_MEMBERSHIP_AUTO || cfg->params.query_cap < 1 || cfg->params.S < 0 ||
      cfg->params.S > GRAND_S_MAX)
    return GRAND_E_INVALID;
  for (int i = 0; i < cfg->n_codes; ++i)
    if (!cfg->codes[i]) return GRAND_E_INVALID;
  *out = nullptr;
  grand_server* s = new (std::nothrow) grand_server();
  if (!s) return GRAND_E_NOMEM;
  s->cfg = *cfg;
  if (s->cfg.max_batch == 0 || s->cfg.max_batch > s->cfg.max_slots) s->cfg.max_batch = s->cfg.max_slots;
  s->codes.assign(cfg->codes, cfg->codes + cfg->n_codes);
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return GRAND_E_CUDA;
  }
  s->ring_cap = cfg->max_device_bytes / 8;
  if (cudaMallocHost((void**)&s->h_ring, sizeof(float2) * s->ring_cap) != cudaSuccess ||
      cudaMalloc((void**)&s->d_ring, sizeof(float2) * s->ring_cap) != cudaSuccess) {
    free_server(s);
    return GRAND_E_NOMEM;
  }
  s->sb.resize(cfg->n_streams);
  const size_t mb = (size_t)s->cfg.max_batch;
  for (StreamBuf& b : s->sb) {
    if (cudaStreamCreateWithFlags(&b.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc((void**)&b.d_desc, sizeof(grand_frame_desc) * mb) != cudaSuccess ||
        cudaMalloc((void**)&b.d_cw, sizeof(uint32_t) * mb * kResultWords) != cudaSuccess ||
        cudaMalloc((void**)&b.d_q, sizeof(uint32_t) * mb) != cudaSuccess ||
        cudaMalloc((void**)&b.d_ab, mb) != cudaSuccess ||
        cudaMallocHost((void**)&b.h_desc, sizeof(grand_frame_desc) * mb) != cudaSuccess ||
        cudaMallocHost((void**)&b.h_cw, sizeof(uint32_t) * mb * kResultWords) != cudaSuccess ||
        cudaMallocHost((void**)&b.h_q, sizeof(uint32_t) * mb) != cudaSuccess ||
        cudaMallocHost((void**)&b.h_ab, mb) != cudaSuccess) {
      free_server(s);
      return GRAND_E_NOMEM;
    }
  }
  s->worker = std::thread(worker_main, s);
  *out = s;
  return GRAND_OK;
}

extern "C" int grand_server_submit(grand_server* s, const grand_request* reqs, int n, int* n_admitted) {
  if (!s || (n > 0 && !reqs) || n < 0 || !n_admitted) return GRAND_E_INVALID;
  *n_admitted = 0;
  if (n == 0) return GRAND_OK;
  const int64_t t = now_ns();
  int admitted = 0;
  int rc = GRAND_OK;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    for (int i = 0; i < n; ++i) {
      const grand_request& q = reqs[i];
      const int m = m_of(q.M);
      if (q.code < 0 || q.code >= (int)s->codes.size() || !m || !q.symbols) {
        rc = GRAND_E_INVALID;
        break;
      }
      const int N = s->codes[q.code]->N;
      const int L = (N + 2 * m - 1) / (2 * m);
      const int64_t bytes = request_bytes(L, N);
      if (bytes > s->cfg.max_device_bytes || L > s->ring_cap) {  // could never be admitted
        rc = GRAND_E_INVALID;
        break;
      }
      // ring position: contiguous, skipping the tail end if it would wrap
      int64_t v = s->vhead;
      if (v % s->ring_cap + L > s->ring_cap) v += s->ring_cap - v % s->ring_cap;
      const bool fits = s->live_slots < s->cfg.max_slots && s->live_bytes + bytes <= s->cfg.max_device_bytes &&
                        v + L - s->vtail <= s->ring_cap;
      if (!fits) {
        rc = admitted ? GRAND_OK : GRAND_E_BUSY;
        s->st.rejected += n - i;
        break;
      }
      memcpy(s->h_ring + v % s->ring_cap, q.symbols, sizeof(float2) * L);
      Req r;
      r.tag = q.tag;
      r.arrival_ns = q.arrival_ns ? q.arrival_ns : t;
      r.code = q.code;
      r.M = q.M;
      r.L = L;
      r.nw = N / 32;
      r.vpos = v;
      r.bytes = bytes;
      s->pending.push_back(r);
      s->vhead = v + L;
      s->live_bytes += bytes;
      s->live_slots += 1;
      ++admitted;
    }
    s->st.admitted += admitted;
  }
  s->cv.notify_one();
  *n_admitted = admitted;
  return rc;
}

extern "C" int grand_server_poll(grand_server* s, grand_result* out, int max, int* n) {
  if (!s || !n || max < 0 || (max > 0 && !out)) return GRAND_E_INVALID;
  std::unique_lock<std::mutex> lk(s->mu);
  int k = 0;
  while (k < max && !s->done.empty()) {
    out[k++] = s->done.front();
    s->done.pop_front();
  }
  *n = k;
  return GRAND_OK;
}

extern "C" int grand_server_drain(grand_server* s, int64_t timeout_ns) {
  if (!s || timeout_ns < 0) return GRAND_E_INVALID;
  const int64_t deadline = now_ns() + timeout_ns;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->pending.empty() && s->inflight.empty()) return GRAND_OK;
    }
    if (now_ns() >= deadline) return GRAND_E_TIMEOUT;
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

extern "C" int grand_server_get_stats(grand_server* s, grand_server_stats* out) {
  if (!s || !out) return GRAND_E_INVALID;
  std::unique_lock<std::mutex> lk(s->mu);
  *out = s->st;
  out->live_slots = s->live_slots;
  out->live_bytes = s->live_bytes;
  out->pending = (int64_t)s->pending.size();
  out->inflight_batches = (int64_t)s->inflight.size();
  return GRAND_OK;
}

extern "C" int grand_server_destroy(grand_server* s) {
  if (!s) return GRAND_OK;
  grand_server_drain(s, 10ll * 1000000000ll);  // bounded: 10 s
  s->stop.store(true, std::memory_order_release);
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  free_server(s);
  return GRAND_OK;
}
