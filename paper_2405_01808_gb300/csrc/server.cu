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
// Long frames (resume_weight_step > 0): a batch's search covers only the
// first resume_weight_step TEP weights beyond the preparation's. Frames left
// without a codeword there are suspended with their search state (a cursor,
// see grand_decode_symbols_resumable) in the batch's buffer set on the
// device; the harvester reports the batch's other frames at once, hands its
// stream back, and continues the suspended ones -- every remaining weight --
// on one of the server's continuation streams, from those cursors: a small
// gather on the batch's stream first moves the suspended frames' cursors and
// hard words into one of the server's continuation blocks (compact device
// arrays and pinned result buffers, preallocated), so the batch's buffer set
// is free again at once. When every block is in use (or a batch has more
// long frames than a block holds), the continuation runs in place instead and the batch keeps its
// buffer set until its last frame is reported (buffer sets outnumber streams:
// four per stream). Results are those of the uninterrupted search.
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

// Device and pinned host buffers of one batch (a batch holds its set until
// every frame of it is reported; its stream is freed earlier).
struct BufSet {
  grand::FrameRec* d_cur = nullptr;  // per-frame cursors (resume_weight_step > 0)
  int32_t* h_idx = nullptr;          // pinned: frames to gather into a continuation
  cudaEvent_t free_after = nullptr;  // the gather out of this set is done
  bool wait_free = false;            // the next batch on this set waits for free_after
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
  int set;        // buffer set
  int64_t launch_ns;
  std::vector<Req> reqs;
  int64_t vend;   // ring released up to here once this and all earlier batches have left the ring
  int64_t bytes;
  cudaEvent_t ev;
  bool done;       // every frame reported
  bool ring_done;  // the symbols are no longer read (the first launch finished)
  int status;
  // continuation of the suspended frames (resume_weight_step > 0)
  bool cont = false;               // the continuation is in flight (ev re-recorded on cstream)
  int cstream = -1;
  std::vector<int32_t> suspended;  // frames of the batch it continues
  int64_t left_bytes = 0;          // budget still held by them
};

// Buffers of one continuation job (capacity kBlockFrames frames): compact
// device copies of the suspended frames' cursors, words and counters, and the
// pinned host buffers receiving their results. Preallocated: a job allocates
// nothing (growing a memory pool under a running server stalls it).
constexpr int kBlockFrames = 4096;
struct ResultBlock {
  grand::FrameRec* d_cur = nullptr;
  uint32_t* d_cw = nullptr;
  uint32_t* d_q = nullptr;
  uint8_t* d_ab = nullptr;
  int32_t* d_idx = nullptr;
  uint32_t* h_cw = nullptr;
  uint32_t* h_q = nullptr;
  uint8_t* h_ab = nullptr;
  bool busy = false;
};

// Suspended frames of one batch continued from compact device copies of
// their cursors (the batch itself is done); request i is compact entry i.
struct LongJob {
  std::vector<Req> reqs;
  int block;
  int64_t bytes;
  cudaEvent_t ev;
  int status;
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
  std::vector<cudaStream_t> streams;
  std::vector<char> stream_busy;
  std::vector<BufSet> sets;
  int32_t step = 0;                    // resume_weight_step
  std::vector<cudaStream_t> cstreams;  // continuation streams of long frames
  int next_cstream = 0;
  std::vector<ResultBlock> blocks;     // result blocks of continuations
  std::deque<LongJob> jobs;            // continuations in flight (the harvester's)
  int64_t long_live = 0;               // frames being continued
  std::deque<Req> pending;     // admitted, not launched (ring order)
  std::deque<Batch> inflight;  // launch order
  std::deque<Chunk> done;
  std::mutex mu;
  std::condition_variable cv_launch;   // ready requests, an idle stream, or stop
  std::condition_variable cv_harvest;  // a launched batch, or stop
  std::thread launcher, harvester;
  std::atomic<bool> stop{false};
  grand_server_stats st{};
};

namespace {

int64_t request_bytes(int L, int N) { return 8ll * L + (int64_t)sizeof(grand::FrameRec) + 4ll * (N / 32) + 5; }

void free_server(grand_server* s) {
  for (cudaStream_t st : s->streams)
    if (st) cudaStreamSynchronize(st);
  for (cudaStream_t st : s->cstreams)
    if (st) cudaStreamSynchronize(st);
  for (ResultBlock& r : s->blocks) {
    cudaFree(r.d_cur);
    cudaFree(r.d_cw);
    cudaFree(r.d_q);
    cudaFree(r.d_ab);
    cudaFree(r.d_idx);
    cudaFreeHost(r.h_cw);
    cudaFreeHost(r.h_q);
    cudaFreeHost(r.h_ab);
  }
  for (LongJob& j : s->jobs) cudaEventDestroy(j.ev);
  for (BufSet& b : s->sets) {
    cudaFree(b.d_cur);
    cudaFreeHost(b.h_idx);
    if (b.free_after) cudaEventDestroy(b.free_after);
    cudaFree(b.d_desc);
    cudaFree(b.d_cw);
    cudaFree(b.d_q);
    cudaFree(b.d_ab);
    cudaFreeHost(b.h_desc);
    cudaFreeHost(b.h_cw);
    cudaFreeHost(b.h_q);
    cudaFreeHost(b.h_ab);
  }
  for (cudaStream_t st : s->streams)
    if (st) cudaStreamDestroy(st);
  for (cudaStream_t st : s->cstreams)
    if (st) cudaStreamDestroy(st);
  for (Batch& b : s->inflight) cudaEventDestroy(b.ev);
  cudaFree(s->d_table);
  cudaFree(s->d_ring);
  cudaFreeHost(s->h_ring);
  delete s;
}

// Issue batch b on its stream with its buffer set (no lock held; b.reqs was
// taken under it).
int launch_batch(grand_server* s, Batch& b) {
  grand::NvtxRange range("grand.server.batch");
  BufSet& buf = s->sets[b.set];
  const cudaStream_t stream = s->streams[b.stream];
  const int n = (int)b.reqs.size();
  // the previous batch's long frames must have been gathered out of this set
  if (buf.wait_free && cudaStreamWaitEvent(stream, buf.free_after, 0) != cudaSuccess) return GRAND_E_CUDA;
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
    if (cudaMemcpyAsync(s->d_ring + p, s->h_ring + p, sizeof(float2) * len, cudaMemcpyHostToDevice, stream) !=
        cudaSuccess)
      return GRAND_E_CUDA;
    v += len;
  }
  if (cudaMemcpyAsync(buf.d_desc, buf.h_desc, sizeof(grand_frame_desc) * n, cudaMemcpyHostToDevice, stream) !=
      cudaSuccess)
    return GRAND_E_CUDA;
  int rc = grand::decode_mixed_resident(s->d_table, (int)s->codes.size(), s->Lmax, s->Wmax, &s->cfg.params,
                                        buf.d_desc, n, s->d_ring, s->ring_cap, buf.d_cw, (int64_t)n * kResultWords,
                                        buf.d_q, buf.d_ab, stream, s->step, s->step > 0 ? buf.d_cur : nullptr);
  if (rc != GRAND_OK) return rc;
  if (cudaMemcpyAsync(buf.h_cw, buf.d_cw, sizeof(uint32_t) * n * kResultWords, cudaMemcpyDeviceToHost, stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(buf.h_q, buf.d_q, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaMemcpyAsync(buf.h_ab, buf.d_ab, n, cudaMemcpyDeviceToHost, stream) != cudaSuccess)
    return GRAND_E_CUDA;
  if (cudaEventRecord(b.ev, stream) != cudaSuccess) return GRAND_E_CUDA;
  return GRAND_OK;
}

// Gather k suspended frames (indices idx) of a buffer set into compact arrays.
__global__ void k_gather_long(const int32_t* idx, int k, const grand::FrameRec* cur, const uint32_t* cw,
                              const uint32_t* q, const uint8_t* ab, grand::FrameRec* ccur, uint32_t* ccw,
                              uint32_t* cq, uint8_t* cab) {
  const int lane = threadIdx.x & 31;
  const int i = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  if (i >= k) return;
  const int f = idx[i];
  constexpr int kWords = (int)(sizeof(grand::FrameRec) / 4);
  const uint32_t* src = reinterpret_cast<const uint32_t*>(cur + f);
  uint32_t* dst = reinterpret_cast<uint32_t*>(ccur + i);
  for (int w = lane; w < kWords; w += 32) dst[w] = src[w];
  ccw[(size_t)i * kResultWords + lane] = cw[(size_t)f * kResultWords + lane];
  if (lane == 0) {
    cq[i] = q[f];
    cab[i] = ab[f];
  }
}

// The suspended frames `susp` of batch b (its first launch finished) as a
// continuation job: gather their cursors and hard words out of the batch's
// set on the batch's stream (the set is reusable after that), then every
// remaining weight on a continuation stream, results into result block
// `block`. No lock held; returns a CUDA status.
int launch_job(grand_server* s, const Batch& b, const std::vector<int32_t>& susp, int block, int cstream,
               cudaEvent_t ev) {
  grand::NvtxRange range("grand.server.resume");
  BufSet& buf = s->sets[b.set];
  const cudaStream_t st = s->streams[b.stream];
  const cudaStream_t cs = s->cstreams[cstream];
  const int k = (int)susp.size();
  const ResultBlock& rb = s->blocks[block];
  const size_t cw_b = sizeof(uint32_t) * kResultWords * k, q_b = sizeof(uint32_t) * k, idx_b = sizeof(int32_t) * k;
  grand::FrameRec* ccur = rb.d_cur;
  uint32_t* ccw = rb.d_cw;
  uint32_t* cq = rb.d_q;
  int32_t* cidx = rb.d_idx;
  uint8_t* cab = rb.d_ab;
  for (int i = 0; i < k; ++i) buf.h_idx[i] = susp[i];
  if (cudaMemcpyAsync(cidx, buf.h_idx, idx_b, cudaMemcpyHostToDevice, st) != cudaSuccess) return GRAND_E_CUDA;
  k_gather_long<<<(k * 32 + 127) / 128, 128, 0, st>>>(cidx, k, buf.d_cur, buf.d_cw, buf.d_q, buf.d_ab, ccur, ccw, cq,
                                                      cab);
  if (cudaGetLastError() != cudaSuccess || cudaEventRecord(buf.free_after, st) != cudaSuccess ||
      cudaStreamWaitEvent(cs, buf.free_after, 0) != cudaSuccess)
    return GRAND_E_CUDA;
  int rc = grand::resume_resident(s->d_table, (int)s->codes.size(), s->Wmax, &s->cfg.params, ccur, k, 0, ccw,
                                  kResultWords, cq, cab, cs);
  if (rc != GRAND_OK) return rc;
  if (cudaMemcpyAsync(rb.h_cw, ccw, cw_b, cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
      cudaMemcpyAsync(rb.h_q, cq, q_b, cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
      cudaMemcpyAsync(rb.h_ab, cab, k, cudaMemcpyDeviceToHost, cs) != cudaSuccess)
    return GRAND_E_CUDA;
  return cudaEventRecord(ev, cs) == cudaSuccess ? GRAND_OK : GRAND_E_CUDA;
}

// The rest of batch b's suspended frames (every remaining weight) on a
// continuation stream, from the cursors in its buffer set, and the read-back
// of their outputs; b.ev is recorded again behind it. Called by the harvester
// once the batch's first launch has finished (no lock held).
int launch_continuation(grand_server* s, Batch& b) {
  grand::NvtxRange range("grand.server.resume");
  BufSet& buf = s->sets[b.set];
  const cudaStream_t cs = s->cstreams[b.cstream];
  const int n = (int)b.reqs.size();
  int rc = grand::resume_resident(s->d_table, (int)s->codes.size(), s->Wmax, &s->cfg.params, buf.d_cur, n, 0,
                                  buf.d_cw, kResultWords, buf.d_q, buf.d_ab, cs);
  if (rc != GRAND_OK) return rc;
  if (cudaMemcpyAsync(buf.h_cw, buf.d_cw, sizeof(uint32_t) * n * kResultWords, cudaMemcpyDeviceToHost, cs) !=
          cudaSuccess ||
      cudaMemcpyAsync(buf.h_q, buf.d_q, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
      cudaMemcpyAsync(buf.h_ab, buf.d_ab, n, cudaMemcpyDeviceToHost, cs) != cudaSuccess)
    return GRAND_E_CUDA;
  return cudaEventRecord(b.ev, cs) == cudaSuccess ? GRAND_OK : GRAND_E_CUDA;
}

void launcher_main(grand_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    Batch b;
    int si = -1;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      while (!s->stop.load(std::memory_order_acquire)) {
        if (!s->pending.empty() && s->pending.front().ready) {
          int set = -1;
          for (int i = 0; i < (int)s->streams.size(); ++i)
            if (!s->stream_busy[i]) { si = i; break; }
          for (int i = 0; i < (int)s->sets.size(); ++i)
            if (!s->sets[i].busy) { set = i; break; }
          if (si >= 0 && set >= 0) {
            b.set = set;
            break;
          }
          si = -1;
        }
        s->cv_launch.wait_for(lk, std::chrono::milliseconds(1));  // bounded: re-check
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
      b.ring_done = false;
      b.status = GRAND_OK;
      s->stream_busy[si] = 1;
      s->sets[b.set].busy = true;
      s->st.batches += 1;
      s->st.batched_frames += b.reqs.size();
    }
    cudaEventCreateWithFlags(&b.ev, cudaEventDisableTiming);
    b.launch_ns = now_ns();
    b.status = launch_batch(s, b);
    const int64_t issued = now_ns() - b.launch_ns;
    if (b.status != GRAND_OK) cudaEventRecord(b.ev, s->streams[si]);
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

// Finished continuation jobs: report their frames, free their result blocks.
// Harvester thread only (it alone adds and removes jobs). Returns whether one
// was harvested.
bool harvest_jobs(grand_server* s) {
  bool any = false;
  for (auto it = s->jobs.begin(); it != s->jobs.end();) {
    const cudaError_t q = cudaEventQuery(it->ev);
    if (q == cudaErrorNotReady) {
      ++it;
      continue;
    }
    any = true;
    const int64_t t = now_ns();
    const ResultBlock& rb = s->blocks[it->block];
    Chunk c;
    c.v.resize(it->reqs.size());
    for (size_t i = 0; i < it->reqs.size(); ++i) {
      grand_result& r = c.v[i];
      memset(&r, 0, sizeof r);
      r.tag = it->reqs[i].tag;
      r.arrival_ns = it->reqs[i].arrival_ns;
      r.done_ns = t;
      r.continued = 1;
      if (q == cudaSuccess) {
        r.queries = rb.h_q[i];
        r.abandon = rb.h_ab[i];
        memcpy(r.cw, rb.h_cw + i * kResultWords, sizeof(uint32_t) * it->reqs[i].nw);
      } else {
        r.abandon = 4;
      }
    }
    cudaEventDestroy(it->ev);
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->done.push_back(std::move(c));
      s->blocks[it->block].busy = false;
      const int k = (int)it->reqs.size();
      s->live_slots -= k;
      s->live_bytes -= it->bytes;
      s->long_live -= k;
      s->st.completed += k;
      if (q != cudaSuccess) s->st.errors += 1;
      s->running -= 1;
    }
    it = s->jobs.erase(it);
    s->cv_launch.notify_one();
  }
  return any;
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
      const BufSet& buf = s->sets[b->set];
      const bool first = !b->cont;  // the batch's first launch finished (else its continuation)
      const int n = (int)b->reqs.size();
      // frames suspended by the first launch's weight window continue
      std::vector<int32_t> susp;
      if (first && status == GRAND_OK && s->step > 0)
        for (int i = 0; i < n; ++i)
          if (buf.h_ab[i] == GRAND_ABANDON_SUSPENDED) susp.push_back(i);
      Chunk c;
      auto emit = [&](int i, bool failed) {
        c.v.emplace_back();
        grand_result& r = c.v.back();
        memset(&r, 0, sizeof r);
        r.tag = b->reqs[i].tag;
        r.arrival_ns = b->reqs[i].arrival_ns;
        r.done_ns = t;
        r.continued = first ? 0 : 1;
        if (!failed) {
          r.queries = buf.h_q[i];
          r.abandon = buf.h_ab[i];
          memcpy(r.cw, buf.h_cw + (size_t)i * kResultWords, sizeof(uint32_t) * b->reqs[i].nw);
        } else {
          r.abandon = 4;  // the batch failed on the device
        }
      };
      if (first) {
        c.v.reserve(n - susp.size());
        size_t k = 0;
        for (int i = 0; i < n; ++i) {
          if (k < susp.size() && susp[k] == i) {
            ++k;
            continue;
          }
          emit(i, status != GRAND_OK);
        }
      } else {
        for (int32_t i : b->suspended) emit(i, status != GRAND_OK);
      }
      bool continues = false;  // in place: the batch keeps its set
      bool job = false;        // as a continuation job: the batch is done
      LongJob lj;
      if (!susp.empty()) {
        b->suspended = susp;
        b->left_bytes = 0;
        for (int32_t i : susp) b->left_bytes += b->reqs[i].bytes;
        const int cstream = s->next_cstream;
        s->next_cstream = (s->next_cstream + 1) % (int)s->cstreams.size();
        int block = -1;
        if ((int)susp.size() <= kBlockFrames) {
          std::unique_lock<std::mutex> lk(s->mu);
          for (int i = 0; i < (int)s->blocks.size(); ++i)
            if (!s->blocks[i].busy) {
              block = i;
              s->blocks[i].busy = true;
              break;
            }
        }
        if (block >= 0 && cudaEventCreateWithFlags(&lj.ev, cudaEventDisableTiming) == cudaSuccess) {
          lj.block = block;
          lj.bytes = b->left_bytes;
          lj.status = GRAND_OK;
          for (int32_t i : susp) lj.reqs.push_back(b->reqs[i]);
          job = launch_job(s, *b, susp, block, cstream, lj.ev) == GRAND_OK;
          if (!job) cudaEventDestroy(lj.ev);
        }
        if (!job) {
          if (block >= 0) {
            std::unique_lock<std::mutex> lk(s->mu);
            s->blocks[block].busy = false;
          }
          b->cstream = cstream;
          b->cont = true;
          continues = launch_continuation(s, *b) == GRAND_OK;
          if (!continues) {  // report them as failed now
            b->cont = false;
            for (int32_t i : susp) emit(i, true);
          }
        }
      }
      {
        std::unique_lock<std::mutex> lk(s->mu);
        if (!c.v.empty()) s->done.push_back(std::move(c));
        if (first) {
          b->ring_done = true;
          s->stream_busy[b->stream] = 0;
          s->st.batch_service_ns += t - b->launch_ns;
          if (t - b->launch_ns > s->st.max_batch_service_ns) s->st.max_batch_service_ns = t - b->launch_ns;
        }
        if (status != GRAND_OK || (!susp.empty() && !continues && !job)) s->st.errors += 1;
        if (job) {  // the suspended frames left with the job: the batch is done, its set free after the gather
          s->st.long_frames += (int64_t)susp.size();
          s->st.resume_launches += 1;
          s->st.completed += n - (int64_t)susp.size();
          s->live_bytes -= b->bytes - b->left_bytes;
          s->live_slots -= n - (int)susp.size();
          s->long_live += (int64_t)susp.size();
          b->done = true;
          b->status = status;
          s->running -= 1;
          s->sets[b->set].wait_free = true;
          s->sets[b->set].busy = false;
          s->jobs.push_back(std::move(lj));
          s->running += 1;  // the job is harvested like a batch
        } else if (continues) {  // the frames reported now release their budget; the batch keeps its buffer set
          s->st.long_frames += (int64_t)susp.size();
          s->st.resume_launches += 1;
          s->long_live += (int64_t)susp.size();
          s->st.completed += n - (int64_t)susp.size();
          s->live_bytes -= b->bytes - b->left_bytes;
          s->live_slots -= n - (int)susp.size();
        } else {
          const int64_t nrep = first ? n : (int64_t)b->suspended.size();
          if (!first) s->long_live -= nrep;
          s->st.completed += nrep;
          s->live_bytes -= first ? b->bytes : b->left_bytes;
          s->live_slots -= (int)nrep;
          b->done = true;
          b->status = status;
          s->running -= 1;
          s->sets[b->set].busy = false;
        }
        // ring space goes back in launch order, as soon as a batch's symbols
        // are no longer read; batches leave the queue once fully reported
        for (Batch& f : s->inflight) {
          if (!f.ring_done) break;
          s->vtail = f.vend;
        }
        while (!s->inflight.empty() && s->inflight.front().done) {
          cudaEventDestroy(s->inflight.front().ev);
          s->inflight.pop_front();
        }
      }
      s->cv_launch.notify_one();
    }
    if (!s->jobs.empty() && harvest_jobs(s)) any = true;
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
      (cfg->params.membership != GRAND_MEMBERSHIP_AUTO && cfg->params.membership != GRAND_MEMBERSHIP_HASH &&
       cfg->params.membership != GRAND_MEMBERSHIP_SOLVE) ||
      cfg->params.query_cap < 1 || cfg->params.deadline_ns < 0 || cfg->params.S < 0 ||
      cfg->params.S > GRAND_S_MAX || cfg->resume_weight_step < 0)
    return GRAND_E_INVALID;
  if (cfg->resume_weight_step > 0 && (cfg->params.tiles[1] > 0 || cfg->params.membership == GRAND_MEMBERSHIP_SOLVE))
    return GRAND_E_UNSUPPORTED;
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
  s->step = cfg->resume_weight_step;
  const size_t mb = (size_t)s->cfg.max_batch;
  s->streams.assign(cfg->n_streams, nullptr);
  s->stream_busy.assign(cfg->n_streams, 0);
  for (cudaStream_t& st : s->streams)
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      free_server(s);
      return GRAND_E_CUDA;
    }
  if (s->step > 0) {
    s->cstreams.assign(cfg->n_streams, nullptr);
    for (cudaStream_t& st : s->cstreams)
      if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        free_server(s);
        return GRAND_E_CUDA;
      }
  }
  // a batch with long frames keeps its buffers after its stream is free again
  // (until its last frame is reported): with a long frame in most batches,
  // every set can be waiting on one, so there are four per stream
  s->sets.resize(s->step > 0 ? 4 * cfg->n_streams : cfg->n_streams);
  if (s->step > 0) {
    s->blocks.resize(4 * cfg->n_streams);
    const size_t bf = kBlockFrames;
    for (ResultBlock& r : s->blocks)
      if (cudaMalloc((void**)&r.d_cur, sizeof(grand::FrameRec) * bf) != cudaSuccess ||
          cudaMalloc((void**)&r.d_cw, sizeof(uint32_t) * bf * kResultWords) != cudaSuccess ||
          cudaMalloc((void**)&r.d_q, sizeof(uint32_t) * bf) != cudaSuccess ||
          cudaMalloc((void**)&r.d_ab, bf) != cudaSuccess ||
          cudaMalloc((void**)&r.d_idx, sizeof(int32_t) * bf) != cudaSuccess ||
          cudaMallocHost((void**)&r.h_cw, sizeof(uint32_t) * bf * kResultWords) != cudaSuccess ||
          cudaMallocHost((void**)&r.h_q, sizeof(uint32_t) * bf) != cudaSuccess ||
          cudaMallocHost((void**)&r.h_ab, bf) != cudaSuccess) {
        free_server(s);
        return GRAND_E_NOMEM;
      }
  }
  for (BufSet& b : s->sets) {
    if (s->step > 0 && (cudaMallocHost((void**)&b.h_idx, sizeof(int32_t) * mb) != cudaSuccess ||
                        cudaEventCreateWithFlags(&b.free_after, cudaEventDisableTiming) != cudaSuccess)) {
      free_server(s);
      return GRAND_E_NOMEM;
    }
    if ((s->step > 0 && cudaMalloc((void**)&b.d_cur, sizeof(grand::FrameRec) * mb) != cudaSuccess) ||
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
    if (grand::scratch_alloc(&warm, per_batch * s->sets.size(), s->streams[0]) == cudaSuccess)
      cudaFreeAsync(warm, s->streams[0]);
    cudaStreamSynchronize(s->streams[0]);
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
  out->long_live = s->long_live;
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
