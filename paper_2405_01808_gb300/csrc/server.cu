// Serving loop: continuous batching of decode requests of mixed code length
// and constellation.
//
// Admission: a request is admitted when a slot is free and its device bytes
// (received symbols, hand-off record, outputs) fit the memory budget; its
// symbols go into a pinned host ring whose device mirror keeps every admitted
// request's received word resident until it completes. Submit reserves ring
// space under the lock and copies the symbols outside it; a request becomes
// launchable once its copy is done (launches take the ready prefix, so the
// ring stays contiguous in launch order).
//
// Two threads run the loop. The launcher takes the ready requests as one
// uneven batch as soon as a stream is idle and issues it (symbols to the
// device ring, descriptors, the decode on the server's resident code table,
// results back to pinned buffers, an event). The harvester polls the events
// of running batches, turns a finished batch into result records outside the
// lock and hands the stream back. Results carry the arrival and completion
// times (CLOCK_MONOTONIC). Ring space is reclaimed in launch order; results
// are delivered in completion order. Every wait is bounded.
//
// Long frames (resume_weight_step > 0): a batch searches each frame only up
// to resume_weight_step TEP weights beyond the preparation's; a frame with no
// codeword there is suspended and its cursor (the search state, see
// grand_decode_symbols_resumable) moves into a device-resident pool of long
// frames, so the batch completes and its other frames are reported at once.
// The launcher runs the pool's next weight window on a stream of its own
// whenever no pool launch is in flight; a frame leaves the pool when its
// search ends (decoded or abandoned), with the outputs an uninterrupted
// search gives. The carry (records, hard words, counters) is a device-side
// gather on the pool's stream; the batch's stream waits for it before its
// buffers are reused.
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

#include "host_util.cuh"
#include "internal.cuh"

namespace {

constexpr int kMaxStreams = 16;
constexpr int kResultWords = GRAND_N_MAX / 32;

int64_t now_ns() {
  timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (int64_t)ts.tv_sec * 1000000000ll + ts.tv_nsec;
}

struct Req {
  uint64_t tag;
  int64_t arrival_ns;
  int32_t code, M, L, nw;
  int64_t vpos;   // virtual ring position of the first symbol
  int64_t bytes;  // device bytes charged to the budget
  uint64_t seq;   // admission order
  bool ready;     // symbols copied into the ring
};

struct StreamBuf {
  cudaStream_t stream = nullptr;
  grand::FrameRec* d_cur = nullptr;   // per-frame cursors of the batch (long frames)
  int2* h_pairs = nullptr;            // (frame, pool slot) of the frames to carry
  int2* d_pairs = nullptr;
  cudaEvent_t carried = nullptr;      // the carry out of this stream's buffers is done
  bool wait_carry = false;            // the next batch waits for `carried`
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
  int64_t carried_bytes = 0;  // budget and slots of frames moved to the long-frame pool
  int32_t carried = 0;
};

// Completed results waiting for poll, in completion order.
struct Chunk {
  std::vector<grand_result> v;
  size_t off = 0;
};

}  // namespace

struct grand_server {
  grand_server_cfg cfg;
  std::vector<const grand_code*> codes;
  int device = 0;
  grand::CodeDev* d_table = nullptr;  // device copy of the codes' views
  int Lmax = 1, Wmax = 1;
  // ring of received symbols (complex64 as float2), virtual positions
  float2* h_ring = nullptr;
  float2* d_ring = nullptr;
  int64_t ring_cap = 0;   // symbols
  int64_t vhead = 0;      // next free virtual position
  int64_t vtail = 0;      // oldest live virtual position
  int64_t live_bytes = 0;
  int32_t live_slots = 0;
  uint64_t next_seq = 0;
  int running = 0;        // launched batches not yet harvested
  std::vector<StreamBuf> sb;
  std::deque<Req> pending;     // admitted, not launched (ring order)
  std::deque<Batch> inflight;  // launch order
  std::deque<Chunk> done;
  std::mutex mu;
  std::condition_variable cv_launch;   // ready requests, an idle stream, or stop
  std::condition_variable cv_harvest;  // a launched batch, or stop
  std::thread launcher, harvester;
  std::atomic<bool> stop{false};
  grand_server_stats st{};
  // long-frame pool (resume_weight_step > 0): cursor, hard word / decoded word,
  // queries and abandon flag per slot on the device, host mirrors, requests
  int32_t step = 0;
  int32_t pool_cap = 0;
  grand::FrameRec* d_pcur = nullptr;
  uint32_t* d_pcw = nullptr;
  uint32_t* d_pq = nullptr;
  uint8_t* d_pab = nullptr;
  uint32_t* h_pcw = nullptr;
  uint32_t* h_pq = nullptr;
  uint8_t* h_pab = nullptr;
  cudaStream_t pstream = nullptr;
  cudaEvent_t pev = nullptr;
  std::vector<Req> preq;          // request of each live slot
  std::vector<char> plive;
  std::vector<int32_t> pfree;     // free slots
  int32_t plive_n = 0;
  bool presume = false;           // a pool launch is in flight
  bool pissued = false;           // ... and its event is recorded (the harvester may look)
  bool pfailed = false;           // ... and it could not be issued
  std::vector<int32_t> psnap;     // live slots when it was launched
  int64_t presume_ns = 0;
};

namespace {

int64_t request_bytes(int L, int N) { return 8ll * L + (int64_t)sizeof(grand::FrameRec) + 4ll * (N / 32) + 5; }

void free_server(grand_server* s) {
  if (s->pstream) cudaStreamSynchronize(s->pstream);
  for (StreamBuf& b : s->sb) {
    if (b.stream) cudaStreamSynchronize(b.stream);
    cudaFree(b.d_cur);
    cudaFree(b.d_pairs);
    cudaFreeHost(b.h_pairs);
    if (b.carried) cudaEventDestroy(b.carried);
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
  cudaFree(s->d_pcur);
  cudaFree(s->d_pcw);
  cudaFree(s->d_pq);
  cudaFree(s->d_pab);
  cudaFreeHost(s->h_pcw);
  cudaFreeHost(s->h_pq);
  cudaFreeHost(s->h_pab);
  if (s->pev) cudaEventDestroy(s->pev);
  if (s->pstream) cudaStreamDestroy(s->pstream);
  cudaFree(s->d_table);
  cudaFree(s->d_ring);
  cudaFreeHost(s->h_ring);
  delete s;
}

// Move suspended frames of a finished batch into the long-frame pool: warp k
// copies pair k's cursor, hard word, query count and flag.
__global__ void k_carry(const int2* pairs, int n, const grand::FrameRec* cur, const uint32_t* cw, const uint32_t* q,
                        const uint8_t* ab, grand::FrameRec* pcur, uint32_t* pcw, uint32_t* pq, uint8_t* pab) {
  const int lane = threadIdx.x & 31;
  const int k = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  if (k >= n) return;
  const int f = pairs[k].x, slot = pairs[k].y;
  constexpr int kWords = (int)(sizeof(grand::FrameRec) / 4);
  const uint32_t* src = reinterpret_cast<const uint32_t*>(cur + f);
  uint32_t* dst = reinterpret_cast<uint32_t*>(pcur + slot);
  for (int w = lane; w < kWords; w += 32) dst[w] = src[w];
  pcw[(size_t)slot * kResultWords + lane] = cw[(size_t)f * kResultWords + lane];
  if (lane == 0) {
    pq[slot] = q[f];
    pab[slot] = ab[f];
  }
}

// Issue batch b on stream si (no lock held; b.reqs was taken under it).
int launch_batch(grand_server* s, int si, Batch& b) {
  grand::NvtxRange range("grand.server.batch");
  StreamBuf& buf = s->sb[si];
  const int n = (int)b.reqs.size();
  // the previous batch's long frames must have left this stream's buffers
  if (buf.wait_carry && cudaStreamWaitEvent(buf.stream, buf.carried, 0) != cudaSuccess) return GRAND_E_CUDA;
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
  int rc = grand::decode_mixed_resident(s->d_table, (int)s->codes.size(), s->Lmax, s->Wmax, &s->cfg.params,
                                        buf.d_desc, n, s->d_ring, s->ring_cap, buf.d_cw, (int64_t)n * kResultWords,
                                        buf.d_q, buf.d_ab, buf.stream, s->step, s->step > 0 ? buf.d_cur : nullptr);
  if (rc != GRAND_OK) return rc;
  if (cudaMemcpyAsync(buf.h_cw, buf.d_cw, sizeof(uint32_t) * n * kResultWords, cudaMemcpyDeviceToHost, buf.stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(buf.h_q, buf.d_q, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, buf.stream) != cudaSuccess ||
      cudaMemcpyAsync(buf.h_ab, buf.d_ab, n, cudaMemcpyDeviceToHost, buf.stream) != cudaSuccess)
    return GRAND_E_CUDA;
  if (cudaEventRecord(b.ev, buf.stream) != cudaSuccess) return GRAND_E_CUDA;
  return GRAND_OK;
}

// The next weight window of the long-frame pool's live slots [0, hi), on the
// pool's stream, and the read-back of their outputs (no lock held).
int launch_pool(grand_server* s, int32_t hi) {
  grand::NvtxRange range("grand.server.resume");
  int rc = grand::resume_resident(s->d_table, (int)s->codes.size(), s->Wmax, &s->cfg.params, s->d_pcur, hi, s->step,
                                  s->d_pcw, kResultWords, s->d_pq, s->d_pab, s->pstream);
  if (rc != GRAND_OK) return rc;
  if (cudaMemcpyAsync(s->h_pcw, s->d_pcw, sizeof(uint32_t) * hi * kResultWords, cudaMemcpyDeviceToHost, s->pstream) !=
          cudaSuccess ||
      cudaMemcpyAsync(s->h_pq, s->d_pq, sizeof(uint32_t) * hi, cudaMemcpyDeviceToHost, s->pstream) != cudaSuccess ||
      cudaMemcpyAsync(s->h_pab, s->d_pab, hi, cudaMemcpyDeviceToHost, s->pstream) != cudaSuccess)
    return GRAND_E_CUDA;
  return cudaEventRecord(s->pev, s->pstream) == cudaSuccess ? GRAND_OK : GRAND_E_CUDA;
}

void launcher_main(grand_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    Batch b;
    int si = -1;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      int32_t pool_hi = -1;
      while (!s->stop.load(std::memory_order_acquire)) {
        if (s->step > 0 && !s->presume && s->plive_n > 0) {  // the long frames' next window
          s->psnap.clear();
          for (int32_t k = 0; k < s->pool_cap; ++k)
            if (s->plive[k]) {
              s->psnap.push_back(k);
              pool_hi = k + 1;
            }
          s->presume = true;
          s->presume_ns = now_ns();
          s->st.resume_launches += 1;
          break;
        }
        if (!s->pending.empty() && s->pending.front().ready) {
          for (int i = 0; i < (int)s->sb.size(); ++i)
            if (!s->sb[i].busy) { si = i; break; }
          if (si >= 0) break;
        }
        s->cv_launch.wait_for(lk, std::chrono::milliseconds(1));  // bounded: re-check
      }
      if (pool_hi > 0) {
        lk.unlock();
        const int rc = launch_pool(s, pool_hi);
        if (rc != GRAND_OK) cudaEventRecord(s->pev, s->pstream);  // the harvester sees the failure
        {
          std::unique_lock<std::mutex> lk2(s->mu);
          s->running += 1;
          s->pfailed = rc != GRAND_OK;
          s->pissued = true;
        }
        s->cv_harvest.notify_one();
        continue;
      }
      if (si < 0) return;  // stop
      const int maxb = s->cfg.max_batch;
      int64_t bytes = 0;
      while (!s->pending.empty() && s->pending.front().ready && (int)b.reqs.size() < maxb) {
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
      s->running += 1;
      const int64_t inflight = (int64_t)s->inflight.size();
      if (inflight > s->st.max_inflight_batches) s->st.max_inflight_batches = inflight;
    }
    s->cv_harvest.notify_one();
  }
}

// A finished pool launch: report the slots of its snapshot whose search
// ended, free them; the others stay for the next window. Returns whether a
// launch was harvested.
bool harvest_pool(grand_server* s) {
  std::vector<int32_t> snap;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    if (!s->presume || !s->pissued) return false;
    snap = s->psnap;
  }
  const cudaError_t q = cudaEventQuery(s->pev);
  if (q == cudaErrorNotReady) return false;
  const int64_t t = now_ns();
  Chunk c;
  std::vector<int32_t> freed;
  {
    std::unique_lock<std::mutex> lk(s->mu);  // preq of live slots is read under the lock
    const bool failed = q != cudaSuccess || s->pfailed;
    for (int32_t k : snap) {
      if (!failed && s->h_pab[k] == GRAND_ABANDON_SUSPENDED) continue;
      c.v.emplace_back();
      grand_result& r = c.v.back();
      memset(&r, 0, sizeof r);
      r.tag = s->preq[k].tag;
      r.arrival_ns = s->preq[k].arrival_ns;
      r.done_ns = t;
      if (!failed) {
        r.queries = s->h_pq[k];
        r.abandon = s->h_pab[k];
        memcpy(r.cw, s->h_pcw + (size_t)k * kResultWords, sizeof(uint32_t) * s->preq[k].nw);
      } else {
        r.abandon = 4;
      }
      freed.push_back(k);
    }
    for (int32_t k : freed) {
      s->plive[k] = 0;
      s->plive_n -= 1;
      s->pfree.push_back(k);
      s->live_slots -= 1;
      s->live_bytes -= s->preq[k].bytes;
    }
    s->st.completed += (int64_t)freed.size();
    if (failed) s->st.errors += 1;
    if (!c.v.empty()) s->done.push_back(std::move(c));
    s->presume = false;
    s->pissued = false;
    s->running -= 1;
  }
  s->cv_launch.notify_one();
  return true;
}

void harvester_main(grand_server* s) {
  cudaSetDevice(s->device);
  std::vector<Batch*> running;
  for (;;) {
    running.clear();
    {
      std::unique_lock<std::mutex> lk(s->mu);
      while (!s->stop.load(std::memory_order_acquire) && s->running == 0)
        s->cv_harvest.wait_for(lk, std::chrono::milliseconds(1));  // bounded: re-check
      if (s->stop.load(std::memory_order_acquire)) return;
      // references into the deque stay valid: only finished batches are popped
      for (Batch& b : s->inflight)
        if (!b.done) running.push_back(&b);
    }
    bool any = false;
    for (Batch* b : running) {
      const cudaError_t q = cudaEventQuery(b->ev);
      if (q == cudaErrorNotReady) continue;
      any = true;
      const int64_t t = now_ns();
      const int status = q == cudaSuccess ? b->status : GRAND_E_CUDA;
      StreamBuf& buf = s->sb[b->stream];
      // frames the batch's weight window suspended go to the long-frame pool
      std::vector<int> carry;
      if (status == GRAND_OK && s->step > 0)
        for (size_t i = 0; i < b->reqs.size(); ++i)
          if (buf.h_ab[i] == GRAND_ABANDON_SUSPENDED) carry.push_back((int)i);
      Chunk c;
      c.v.reserve(b->reqs.size() - carry.size());
      size_t ci = 0;
      for (size_t i = 0; i < b->reqs.size(); ++i) {
        if (ci < carry.size() && carry[ci] == (int)i) {
          ++ci;
          continue;
        }
        c.v.emplace_back();
        grand_result& r = c.v.back();
        memset(&r, 0, sizeof r);
        r.tag = b->reqs[i].tag;
        r.arrival_ns = b->reqs[i].arrival_ns;
        r.done_ns = t;
        if (status == GRAND_OK) {
          r.queries = buf.h_q[i];
          r.abandon = buf.h_ab[i];
          memcpy(r.cw, buf.h_cw + i * kResultWords, sizeof(uint32_t) * b->reqs[i].nw);
        } else {
          r.abandon = 4;  // the batch failed on the device
        }
      }
      std::vector<int32_t> slots;
      if (!carry.empty()) {
        {
          std::unique_lock<std::mutex> lk(s->mu);
          for (size_t k = 0; k < carry.size(); ++k) {  // a carried request keeps its admission slot: never empty
            slots.push_back(s->pfree.back());
            s->pfree.pop_back();
          }
        }
        const int nc = (int)carry.size();
        for (int k = 0; k < nc; ++k) buf.h_pairs[k] = make_int2(carry[k], slots[k]);
        // on the pool's stream (ordered before any later pool launch); the
        // batch's stream waits for it before its buffers are reused
        cudaMemcpyAsync(buf.d_pairs, buf.h_pairs, sizeof(int2) * nc, cudaMemcpyHostToDevice, s->pstream);
        k_carry<<<(nc * 32 + 127) / 128, 128, 0, s->pstream>>>(buf.d_pairs, nc, buf.d_cur, buf.d_cw, buf.d_q, buf.d_ab,
                                                             s->d_pcur, s->d_pcw, s->d_pq, s->d_pab);
        cudaEventRecord(buf.carried, s->pstream);
      }
      {
        std::unique_lock<std::mutex> lk(s->mu);
        for (size_t k = 0; k < carry.size(); ++k) {
          const Req& r = b->reqs[carry[k]];
          s->preq[slots[k]] = r;
          s->plive[slots[k]] = 1;
          s->plive_n += 1;
          b->carried += 1;
          b->carried_bytes += r.bytes;
        }
        if (!carry.empty()) {
          buf.wait_carry = true;
          s->st.long_frames += (int64_t)carry.size();
        }
        s->done.push_back(std::move(c));
        b->done = true;
        b->status = status;
        s->running -= 1;
        s->st.completed += b->reqs.size() - carry.size();
        s->st.batch_service_ns += t - b->launch_ns;
        if (t - b->launch_ns > s->st.max_batch_service_ns) s->st.max_batch_service_ns = t - b->launch_ns;
        if (status != GRAND_OK) s->st.errors += 1;
        s->sb[b->stream].busy = false;
        // reclaim ring space and budget in launch order
        while (!s->inflight.empty() && s->inflight.front().done) {
          Batch& f = s->inflight.front();
          s->vtail = f.vend;
          s->live_bytes -= f.bytes - f.carried_bytes;
          s->live_slots -= (int)f.reqs.size() - f.carried;
          cudaEventDestroy(f.ev);
          s->inflight.pop_front();
        }
      }
      s->cv_launch.notify_one();
    }
    if (s->step > 0 && harvest_pool(s)) any = true;
    if (!any) std::this_thread::sleep_for(std::chrono::microseconds(5));
  }
}

}  // namespace

extern "C" int64_t grand_clock_ns(void) { return now_ns(); }

extern "C" int grand_server_create(const grand_server_cfg* cfg, grand_server** out) {
  if (!cfg || !out || !cfg->codes || cfg->n_codes < 1 || cfg->max_slots < 1 || cfg->max_device_bytes < 4096 ||
      cfg->n_streams < 1 || cfg->n_streams > kMaxStreams || cfg->max_batch < 0 || !(cfg->N0 > 0.0f))
    return GRAND_E_INVALID;
  if ((cfg->params.order != GRAND_ORDER_QAM_NNE && cfg->params.order != GRAND_ORDER_QAM_NEARER) ||
      (cfg->params.membership != GRAND_MEMBERSHIP_AUTO && cfg->params.membership != GRAND_MEMBERSHIP_HASH) ||
      cfg->params.query_cap < 1 || cfg->params.deadline_ns < 0 || cfg->params.S < 0 ||
      cfg->params.S > GRAND_S_MAX || cfg->resume_weight_step < 0)
    return GRAND_E_INVALID;
  if (cfg->resume_weight_step > 0 && cfg->params.tiles[1] > 0) return GRAND_E_UNSUPPORTED;
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
  {
    std::vector<grand::CodeDev> table(cfg->n_codes);
    for (int i = 0; i < cfg->n_codes; ++i) {
      table[i] = cfg->codes[i]->dev;
      s->Wmax = std::max(s->Wmax, table[i].W);
      s->Lmax = std::max(s->Lmax, (table[i].N + 1) / 2);  // QPSK bound
    }
    if (cudaMalloc((void**)&s->d_table, sizeof(grand::CodeDev) * cfg->n_codes) != cudaSuccess) {
      free_server(s);
      return GRAND_E_NOMEM;
    }
    if (cudaMemcpy(s->d_table, table.data(), sizeof(grand::CodeDev) * cfg->n_codes, cudaMemcpyHostToDevice) !=
        cudaSuccess) {
      free_server(s);
      return GRAND_E_CUDA;
    }
  }
  s->ring_cap = cfg->max_device_bytes / 8;
  if (cudaMallocHost((void**)&s->h_ring, sizeof(float2) * s->ring_cap) != cudaSuccess ||
      cudaMalloc((void**)&s->d_ring, sizeof(float2) * s->ring_cap) != cudaSuccess) {
    free_server(s);
    return GRAND_E_NOMEM;
  }
  s->sb.resize(cfg->n_streams);
  const size_t mb = (size_t)s->cfg.max_batch;
  s->step = cfg->resume_weight_step;
  if (s->step > 0) {
    // one pool slot per admission slot: a carried request keeps its slot
    s->pool_cap = s->cfg.max_slots;
    const size_t pc = (size_t)s->pool_cap;
    if (cudaStreamCreateWithFlags(&s->pstream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->pev, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc((void**)&s->d_pcur, sizeof(grand::FrameRec) * pc) != cudaSuccess ||
        cudaMalloc((void**)&s->d_pcw, sizeof(uint32_t) * pc * kResultWords) != cudaSuccess ||
        cudaMalloc((void**)&s->d_pq, sizeof(uint32_t) * pc) != cudaSuccess ||
        cudaMalloc((void**)&s->d_pab, pc) != cudaSuccess ||
        cudaMallocHost((void**)&s->h_pcw, sizeof(uint32_t) * pc * kResultWords) != cudaSuccess ||
        cudaMallocHost((void**)&s->h_pq, sizeof(uint32_t) * pc) != cudaSuccess ||
        cudaMallocHost((void**)&s->h_pab, pc) != cudaSuccess ||
        cudaMemset(s->d_pab, 0, pc) != cudaSuccess) {
      free_server(s);
      return GRAND_E_NOMEM;
    }
    s->preq.resize(pc);
    s->plive.assign(pc, 0);
    s->pfree.reserve(pc);
    for (int32_t k = s->pool_cap - 1; k >= 0; --k) s->pfree.push_back(k);
  }
  for (StreamBuf& b : s->sb) {
    if (s->step > 0 &&
        (cudaMalloc((void**)&b.d_cur, sizeof(grand::FrameRec) * mb) != cudaSuccess ||
         cudaMalloc((void**)&b.d_pairs, sizeof(int2) * mb) != cudaSuccess ||
         cudaMallocHost((void**)&b.h_pairs, sizeof(int2) * mb) != cudaSuccess ||
         cudaEventCreateWithFlags(&b.carried, cudaEventDisableTiming) != cudaSuccess)) {
      free_server(s);
      return GRAND_E_NOMEM;
    }
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
  // Grow the library's stream-ordered pool to the decode scratch of n_streams
  // full batches now, so that no batch waits on the pool growing later (the
  // pool keeps freed memory cached).
  {
    const size_t per_batch = 256 + sizeof(grand::FrameRec) * mb + 4096;
    void* warm = nullptr;
    if (grand::scratch_alloc(&warm, per_batch * s->sb.size(), s->sb[0].stream) == cudaSuccess)
      cudaFreeAsync(warm, s->sb[0].stream);
    cudaStreamSynchronize(s->sb[0].stream);
  }
  if (grand::preload_qam_kernels() != GRAND_OK) {
    free_server(s);
    return GRAND_E_CUDA;
  }
  s->launcher = std::thread(launcher_main, s);
  s->harvester = std::thread(harvester_main, s);
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
  uint64_t seq0 = 0;
  std::vector<int64_t> at;  // ring slot of each admitted request
  at.reserve(n);
  // 1. reserve ring space and budget (under the lock)
  {
    std::unique_lock<std::mutex> lk(s->mu);
    seq0 = s->next_seq;
    for (int i = 0; i < n; ++i) {
      const grand_request& q = reqs[i];
      const int m = grand::m_of(q.M);
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
      Req r;
      r.tag = q.tag;
      r.arrival_ns = q.arrival_ns ? q.arrival_ns : t;
      r.code = q.code;
      r.M = q.M;
      r.L = L;
      r.nw = N / 32;
      r.vpos = v;
      r.bytes = bytes;
      r.seq = s->next_seq++;
      r.ready = false;
      s->pending.push_back(r);
      at.push_back(v % s->ring_cap);
      s->vhead = v + L;
      s->live_bytes += bytes;
      s->live_slots += 1;
      ++admitted;
    }
    s->st.admitted += admitted;
  }
  // 2. copy the received symbols into the reserved slots (no lock: the slots
  //    are not launchable and cannot be reclaimed before they are marked ready)
  for (int i = 0; i < admitted; ++i) {
    const grand_request& q = reqs[i];
    const int m = grand::m_of(q.M);
    const int L = (s->codes[q.code]->N + 2 * m - 1) / (2 * m);
    memcpy(s->h_ring + at[i], q.symbols, sizeof(float2) * L);
  }
  // 3. mark them launchable
  if (admitted) {
    std::unique_lock<std::mutex> lk(s->mu);
    const uint64_t front = s->pending.front().seq;  // ours are still pending (not ready)
    for (int i = 0; i < admitted; ++i) s->pending[(size_t)(seq0 + i - front)].ready = true;
  }
  s->cv_launch.notify_one();
  *n_admitted = admitted;
  return rc;
}

extern "C" int grand_server_poll(grand_server* s, grand_result* out, int max, int* n) {
  if (!s || !n || max < 0 || (max > 0 && !out)) return GRAND_E_INVALID;
  // whole chunks are moved out under the lock and copied after it
  std::vector<Chunk> taken;
  int k = 0;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    while (k < max && !s->done.empty()) {
      Chunk& c = s->done.front();
      const size_t left = c.v.size() - c.off;
      if (left <= (size_t)(max - k)) {
        k += (int)left;
        taken.push_back(std::move(c));
        s->done.pop_front();
      } else {
        // the last, partial chunk: its prefix goes after the whole chunks
        memcpy(out + k, c.v.data() + c.off, sizeof(grand_result) * (size_t)(max - k));
        c.off += (size_t)(max - k);
        k = max;
      }
    }
  }
  // the whole chunks, in order, before the partial prefix
  int pos = 0;
  for (Chunk& c : taken) {
    const size_t left = c.v.size() - c.off;
    memcpy(out + pos, c.v.data() + c.off, sizeof(grand_result) * left);
    pos += (int)left;
  }
  *n = k;
  return GRAND_OK;
}

extern "C" int grand_server_drain(grand_server* s, int64_t timeout_ns) {
  if (!s || timeout_ns < 0) return GRAND_E_INVALID;
  const int64_t deadline = now_ns() + timeout_ns;
  for (;;) {
    {
      // live slots count every admitted request until its batch is reclaimed,
      // including a batch the launcher is issuing (then in neither queue)
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->live_slots == 0 && s->pending.empty() && s->inflight.empty()) return GRAND_OK;
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
  out->long_live = s->plive_n;
  return GRAND_OK;
}

extern "C" int grand_server_destroy(grand_server* s) {
  if (!s) return GRAND_OK;
  grand_server_drain(s, 10ll * 1000000000ll);  // bounded: 10 s
  s->stop.store(true, std::memory_order_release);
  {
    std::unique_lock<std::mutex> lk(s->mu);  // no waiter can miss the flag
  }
  s->cv_launch.notify_all();
  s->cv_harvest.notify_all();
  if (s->launcher.joinable()) s->launcher.join();
  if (s->harvester.joinable()) s->harvester.join();
  free_server(s);
  return GRAND_OK;
}
