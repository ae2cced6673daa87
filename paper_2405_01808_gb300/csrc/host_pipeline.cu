// Decoding frames held in host memory with the transfers overlapped
// (grand_decode_symbols_host). The batch is cut into chunks that alternate
// between two streams, each with its own device buffers; on a stream a chunk's
// received symbols are copied in, decoded by the fused call (demodulation,
// Def. III.1 / III.2, and the search of Alg. 2) and its results copied out. A
// chunk's copies on one stream run while the other stream's chunk is on the
// SMs, so only the first chunk's input copy and the last chunk's output copy
// stay exposed.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "host_util.cuh"
#include "internal.cuh"

namespace {

constexpr int kPipeStreams = 2;
constexpr int64_t kMinChunkFrames = 65536;  // keeps each chunk's search a full wave of warps

size_t round_up(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" int grand_decode_symbols_host(const grand_code* c, const grand_params* p, const void* h_symbols,
                                         int64_t n_frames, float N0, uint32_t* h_cw, uint32_t* h_queries,
                                         uint8_t* h_abandon, int64_t chunk_frames, void* stream) {
  if (!c || !p || n_frames < 0 || chunk_frames < 0 ||
      (n_frames > 0 && (!h_symbols || !h_cw || !h_queries || !h_abandon)))
    return GRAND_E_INVALID;
  if (!(N0 > 0.0f) || !isfinite(N0)) return GRAND_E_INVALID;
  size_t in_bytes = 0;  // received data per frame
  if (p->order == GRAND_ORDER_HAMMING) {
    if (p->M != 2) return GRAND_E_INVALID;
    in_bytes = sizeof(float) * (size_t)c->N;
  } else {
    const int m = grand::m_of(p->M);
    if (!m) return GRAND_E_INVALID;
    in_bytes = 2 * sizeof(float) * (size_t)((c->N + 2 * m - 1) / (2 * m));
  }
  // every argument check of the fused call, before any device work (a call
  // without frames validates and returns)
  int rc = grand_decode_symbols(c, p, nullptr, 0, N0, nullptr, nullptr, nullptr, nullptr, stream);
  if (rc != GRAND_OK || n_frames == 0) return rc;
  const size_t NW = (size_t)c->N / 32;
  int64_t chunk = chunk_frames > 0 ? chunk_frames : (n_frames + 3) / 4;
  if (chunk_frames == 0 && chunk < kMinChunkFrames) chunk = kMinChunkFrames;
  if (chunk > n_frames) chunk = n_frames;

  const size_t sym_b = round_up(in_bytes * (size_t)chunk), cw_b = round_up(4 * NW * (size_t)chunk),
               q_b = round_up(4 * (size_t)chunk), ab_b = round_up((size_t)chunk);
  cudaStream_t caller = (cudaStream_t)stream;
  cudaStream_t s[kPipeStreams] = {nullptr, nullptr};
  cudaEvent_t ev[kPipeStreams + 1] = {nullptr, nullptr, nullptr};
  char* dbuf[kPipeStreams] = {nullptr, nullptr};
  // the pipeline's streams start after the work already queued on the caller's
  for (int i = 0; i <= kPipeStreams && rc == GRAND_OK; ++i)
    if (cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) != cudaSuccess) rc = GRAND_E_CUDA;
  if (rc == GRAND_OK && cudaEventRecord(ev[kPipeStreams], caller) != cudaSuccess) rc = GRAND_E_CUDA;
  for (int i = 0; i < kPipeStreams && rc == GRAND_OK; ++i) {
    if (cudaStreamCreateWithFlags(&s[i], cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamWaitEvent(s[i], ev[kPipeStreams], 0) != cudaSuccess) {
      rc = GRAND_E_CUDA;
      break;
    }
    if (cudaMallocAsync((void**)&dbuf[i], sym_b + cw_b + q_b + ab_b, s[i]) != cudaSuccess) rc = GRAND_E_NOMEM;
  }
  const char* hs = static_cast<const char*>(h_symbols);
  for (int64_t k = 0, off = 0; rc == GRAND_OK && off < n_frames; ++k, off += chunk) {
    const int i = (int)(k % kPipeStreams);
    const int64_t nk = n_frames - off < chunk ? n_frames - off : chunk;
    char* d_sym = dbuf[i];
    uint32_t* d_cw = reinterpret_cast<uint32_t*>(dbuf[i] + sym_b);
    uint32_t* d_q = reinterpret_cast<uint32_t*>(dbuf[i] + sym_b + cw_b);
    uint8_t* d_ab = reinterpret_cast<uint8_t*>(dbuf[i] + sym_b + cw_b + q_b);
    // stream order on s[i]: this chunk's input copy follows the output copies
    // of the chunk that used the same buffers before
    if (cudaMemcpyAsync(d_sym, hs + (size_t)off * in_bytes, in_bytes * (size_t)nk, cudaMemcpyHostToDevice, s[i]) !=
        cudaSuccess) {
      rc = GRAND_E_CUDA;
      break;
    }
    rc = grand_decode_symbols(c, p, d_sym, nk, N0, d_cw, d_q, d_ab, nullptr, s[i]);
    if (rc != GRAND_OK) break;
    if (cudaMemcpyAsync(h_cw + (size_t)off * NW, d_cw, 4 * NW * (size_t)nk, cudaMemcpyDeviceToHost, s[i]) !=
            cudaSuccess ||
        cudaMemcpyAsync(h_queries + off, d_q, 4 * (size_t)nk, cudaMemcpyDeviceToHost, s[i]) != cudaSuccess ||
        cudaMemcpyAsync(h_abandon + off, d_ab, (size_t)nk, cudaMemcpyDeviceToHost, s[i]) != cudaSuccess)
      rc = GRAND_E_CUDA;
  }
  for (int i = 0; i < kPipeStreams; ++i) {
    if (!s[i]) continue;
    if (dbuf[i]) cudaFreeAsync(dbuf[i], s[i]);
    // the caller's stream continues after the pipeline (event-based timing on it
    // then covers the whole call)
    if (cudaEventRecord(ev[i], s[i]) != cudaSuccess || cudaStreamWaitEvent(caller, ev[i], 0) != cudaSuccess)
      rc = rc ? rc : GRAND_E_CUDA;
    if (cudaStreamSynchronize(s[i]) != cudaSuccess) rc = rc ? rc : GRAND_E_CUDA;
    cudaStreamDestroy(s[i]);
  }
  for (int i = 0; i <= kPipeStreams; ++i)
    if (ev[i]) cudaEventDestroy(ev[i]);
  return rc;
}
