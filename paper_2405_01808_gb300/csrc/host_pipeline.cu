// Decoding frames held in host memory with the transfers overlapped
// (grand_decode_symbols_host, grand_decode_mixed_host). The batch is cut into chunks that alternate
// between two streams, each with its own device buffers; on a stream a chunk's
// received symbols are copied in, decoded by the fused call (demodulation,
// Def. III.1 / III.2, and the search of Alg. 2) and its results copied out. A
// chunk's copies on one stream run while the other stream's chunk is on the
// SMs, so only the first chunk's input copy and the last chunk's output copy
// stay exposed.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <vector>

#include "host_util.cuh"
#include "internal.cuh"

namespace {

constexpr int kPipeStreams = 2;
constexpr int64_t kMinChunkFrames = 65536;  // keeps each chunk's search a full wave of warps

size_t round_up(size_t b) { return (b + 255) & ~(size_t)255; }

// A chunk's descriptors point into the whole batch's arrays; on the device
// they are made relative to the chunk's first symbol and output word.
__global__ void k_rebase_desc(grand_frame_desc* d, int64_t n, int64_t sym_lo, int64_t cw_lo) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    d[i].sym_offset -= sym_lo;
    d[i].cw_offset -= cw_lo;
  }
}

// The pipeline's streams, created once per host thread and device and kept:
// stream-ordered pool memory freed on a stream is reused by later allocations
// on the same stream, so the buffers and the decode scratch of one call are
// recycled by the next instead of growing the pool.
constexpr int kMaxDevices = 64;
struct ThreadStreams {
  cudaStream_t s[kMaxDevices][kPipeStreams] = {};
};
thread_local ThreadStreams t_streams;

// Streams and events of one pipelined call: the streams start after the work
// queued on the caller's stream; at the end the caller's stream is ordered
// after them and they are synchronised.
struct Pipe {
  cudaStream_t caller = nullptr;
  cudaStream_t s[kPipeStreams] = {nullptr, nullptr};
  cudaEvent_t ev[kPipeStreams + 1] = {nullptr, nullptr, nullptr};
  char* dbuf[kPipeStreams] = {nullptr, nullptr};

  int open(cudaStream_t c, size_t bytes_per_stream) {
    caller = c;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GRAND_E_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return GRAND_E_UNSUPPORTED;
    for (int i = 0; i <= kPipeStreams; ++i)
      if (cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) != cudaSuccess) return GRAND_E_CUDA;
    if (cudaEventRecord(ev[kPipeStreams], caller) != cudaSuccess) return GRAND_E_CUDA;
    for (int i = 0; i < kPipeStreams; ++i) {
      cudaStream_t& ts = t_streams.s[dev][i];
      if (!ts && cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking) != cudaSuccess) return GRAND_E_CUDA;
      s[i] = ts;
      if (cudaStreamWaitEvent(s[i], ev[kPipeStreams], 0) != cudaSuccess) return GRAND_E_CUDA;
      if (bytes_per_stream && grand::scratch_alloc((void**)&dbuf[i], bytes_per_stream, s[i]) != cudaSuccess)
        return GRAND_E_NOMEM;
    }
    return GRAND_OK;
  }

  int close(int rc) {
    for (int i = 0; i < kPipeStreams; ++i) {
      if (!s[i]) continue;
      if (dbuf[i]) cudaFreeAsync(dbuf[i], s[i]);
      // the caller's stream continues after the pipeline (event-based timing on
      // it then covers the whole call)
      if (cudaEventRecord(ev[i], s[i]) != cudaSuccess || cudaStreamWaitEvent(caller, ev[i], 0) != cudaSuccess)
        rc = rc ? rc : GRAND_E_CUDA;
      if (cudaStreamSynchronize(s[i]) != cudaSuccess) rc = rc ? rc : GRAND_E_CUDA;
    }
    for (int i = 0; i <= kPipeStreams; ++i)
      if (ev[i]) cudaEventDestroy(ev[i]);
    return rc;
  }
};

int64_t default_chunk(int64_t n_frames, int64_t chunk_frames) {
  int64_t chunk = chunk_frames > 0 ? chunk_frames : (n_frames + 3) / 4;
  if (chunk_frames == 0 && chunk < kMinChunkFrames) chunk = kMinChunkFrames;
  return chunk > n_frames ? n_frames : chunk;
}

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
  grand::NvtxRange range("grand.host_pipeline");
  const size_t NW = (size_t)c->N / 32;
  const int64_t chunk = default_chunk(n_frames, chunk_frames);
  const size_t sym_b = round_up(in_bytes * (size_t)chunk), cw_b = round_up(4 * NW * (size_t)chunk),
               q_b = round_up(4 * (size_t)chunk), ab_b = round_up((size_t)chunk);
  Pipe pipe;
  rc = pipe.open((cudaStream_t)stream, sym_b + cw_b + q_b + ab_b);
  const char* hs = static_cast<const char*>(h_symbols);
  for (int64_t k = 0, off = 0; rc == GRAND_OK && off < n_frames; ++k, off += chunk) {
    const int i = (int)(k % kPipeStreams);
    cudaStream_t si = pipe.s[i];
    const int64_t nk = n_frames - off < chunk ? n_frames - off : chunk;
    char* d_sym = pipe.dbuf[i];
    uint32_t* d_cw = reinterpret_cast<uint32_t*>(pipe.dbuf[i] + sym_b);
    uint32_t* d_q = reinterpret_cast<uint32_t*>(pipe.dbuf[i] + sym_b + cw_b);
    uint8_t* d_ab = reinterpret_cast<uint8_t*>(pipe.dbuf[i] + sym_b + cw_b + q_b);
    // stream order on s[i]: this chunk's input copy follows the output copies
    // of the chunk that used the same buffers before
    if (cudaMemcpyAsync(d_sym, hs + (size_t)off * in_bytes, in_bytes * (size_t)nk, cudaMemcpyHostToDevice, si) !=
        cudaSuccess) {
      rc = GRAND_E_CUDA;
      break;
    }
    rc = grand_decode_symbols(c, p, d_sym, nk, N0, d_cw, d_q, d_ab, nullptr, si);
    if (rc != GRAND_OK) break;
    if (cudaMemcpyAsync(h_cw + (size_t)off * NW, d_cw, 4 * NW * (size_t)nk, cudaMemcpyDeviceToHost, si) !=
            cudaSuccess ||
        cudaMemcpyAsync(h_queries + off, d_q, 4 * (size_t)nk, cudaMemcpyDeviceToHost, si) != cudaSuccess ||
        cudaMemcpyAsync(h_abandon + off, d_ab, (size_t)nk, cudaMemcpyDeviceToHost, si) != cudaSuccess)
      rc = GRAND_E_CUDA;
  }
  return pipe.close(rc);
}

namespace {

// One chunk of an uneven batch on stream st: frames [f0, f0 + nk) whose
// symbols are [sym_lo, sym_lo + n_sym) and output words [cw_lo, cw_lo + n_cw)
// of the whole arrays. Its buffers come from the stream-ordered pool and go
// back to it on the same stream, so the next chunk there reuses them. With
// `whole` the output array is copied in first (the chunk spans the whole
// arrays and may leave words that no frame owns).
int issue_mixed_chunk(const grand_code* const* codes, int n_codes, const grand_params* p,
                      const grand_frame_desc* h_desc, const float2* h_sym, float N0, uint32_t* h_cw,
                      uint32_t* h_queries, uint8_t* h_abandon, int64_t f0, int64_t nk, int64_t sym_lo, int64_t n_sym,
                      int64_t cw_lo, int64_t n_cw, bool whole, cudaStream_t st) {
  const size_t desc_b = round_up(sizeof(grand_frame_desc) * (size_t)nk), sym_b = round_up(8 * (size_t)n_sym),
               cw_b = round_up(4 * (size_t)n_cw), q_b = round_up(4 * (size_t)nk), ab_b = round_up((size_t)nk);
  char* buf = nullptr;
  if (grand::scratch_alloc((void**)&buf, desc_b + sym_b + cw_b + q_b + ab_b, st) != cudaSuccess) return GRAND_E_NOMEM;
  grand_frame_desc* d_desc = reinterpret_cast<grand_frame_desc*>(buf);
  float2* d_sym = reinterpret_cast<float2*>(buf + desc_b);
  uint32_t* d_cw = reinterpret_cast<uint32_t*>(buf + desc_b + sym_b);
  uint32_t* d_q = reinterpret_cast<uint32_t*>(buf + desc_b + sym_b + cw_b);
  uint8_t* d_ab = reinterpret_cast<uint8_t*>(buf + desc_b + sym_b + cw_b + q_b);
  int rc = GRAND_OK;
  do {
    if (cudaMemcpyAsync(d_desc, h_desc + f0, sizeof(grand_frame_desc) * (size_t)nk, cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(d_sym, h_sym + sym_lo, 8 * (size_t)n_sym, cudaMemcpyHostToDevice, st) != cudaSuccess) {
      rc = GRAND_E_CUDA;
      break;
    }
    if (sym_lo || cw_lo) {
      const int64_t blocks = (nk + 255) / 256;
      k_rebase_desc<<<(int)(blocks < 1024 ? blocks : 1024), 256, 0, st>>>(d_desc, nk, sym_lo, cw_lo);
      if (cudaGetLastError() != cudaSuccess) {
        rc = GRAND_E_CUDA;
        break;
      }
    }
    if (whole && cudaMemcpyAsync(d_cw, h_cw, 4 * (size_t)n_cw, cudaMemcpyHostToDevice, st) != cudaSuccess) {
      rc = GRAND_E_CUDA;
      break;
    }
    rc = grand_decode_mixed(codes, n_codes, p, d_desc, nk, d_sym, n_sym, N0, d_cw, n_cw, d_q, d_ab, nullptr, st);
    if (rc != GRAND_OK) break;
    if (cudaMemcpyAsync(h_cw + cw_lo, d_cw, 4 * (size_t)n_cw, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(h_queries + f0, d_q, 4 * (size_t)nk, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(h_abandon + f0, d_ab, (size_t)nk, cudaMemcpyDeviceToHost, st) != cudaSuccess)
      rc = GRAND_E_CUDA;
  } while (0);
  cudaFreeAsync(buf, st);
  return rc;
}

}  // namespace

extern "C" int grand_decode_mixed_host(const grand_code* const* codes, int n_codes, const grand_params* p,
                                        const grand_frame_desc* h_desc, int64_t n_frames, const void* h_symbols,
                                        int64_t n_symbols, float N0, uint32_t* h_cw, int64_t n_cw_words,
                                        uint32_t* h_queries, uint8_t* h_abandon, int64_t chunk_frames, void* stream) {
  if (!codes || n_codes < 1 || n_frames < 0 || n_symbols < 0 || n_cw_words < 0 || chunk_frames < 0 ||
      (n_frames > 0 && (!h_desc || !h_symbols || !h_cw || !h_queries || !h_abandon)))
    return GRAND_E_INVALID;
  for (int i = 0; i < n_codes; ++i)
    if (!codes[i]) return GRAND_E_INVALID;
  // every argument check of the device call, before any device work
  int rc = grand_decode_mixed(codes, n_codes, p, nullptr, 0, nullptr, 0, N0, nullptr, 0, nullptr, nullptr, nullptr,
                              stream);
  if (rc != GRAND_OK || n_frames == 0) return rc;
  grand::NvtxRange range("grand.host_pipeline.mixed");
  // symbols and output words of a frame, per (code, m); 0 for an invalid
  // descriptor (the device reports such a frame with abandon = 3)
  std::vector<int64_t> tabL((size_t)n_codes * 7, 0), tabNW((size_t)n_codes, 0);
  for (int i = 0; i < n_codes; ++i) {
    tabNW[(size_t)i] = codes[i]->N / 32;
    for (int m = 1; m <= 6; ++m) tabL[(size_t)i * 7 + m] = (codes[i]->N + 2 * m - 1) / (2 * m);
  }
  const int64_t chunk = default_chunk(n_frames, chunk_frames);
  const float2* hs = static_cast<const float2*>(h_symbols);
  Pipe pipe;
  rc = pipe.open((cudaStream_t)stream, 0);
  // Chunks are runs of consecutive frames, which needs the frames packed in
  // increasing, non-overlapping order inside the arrays. Each chunk's
  // descriptors are checked (branch-free: the constellations come in random
  // order) just before it is issued, so the check of one chunk overlaps the
  // device work of the previous ones. From the first chunk that breaks the
  // layout on, the remaining frames are decoded as one chunk over the whole
  // arrays, after the chunks already issued have finished.
  int64_t f0 = 0, end_sym = 0, end_cw = 0;
  bool packed = true;
  for (int k = 0; rc == GRAND_OK && f0 < n_frames; ++k) {
    const int64_t nk = n_frames - f0 < chunk ? n_frames - f0 : chunk;
    const int64_t sym_lo = h_desc[f0].sym_offset, cw_lo = h_desc[f0].cw_offset;
    int64_t es = end_sym, ec = end_cw;
    bool ok = true;
    for (int64_t f = f0; f < f0 + nk; ++f) {
      const grand_frame_desc& d = h_desc[f];
      const uint32_t uM = (uint32_t)d.M;
      const int tz = __builtin_ctz(uM | 0x10000u);
      const bool okM = (uM & (uM - 1u)) == 0 && uM >= 4u && uM <= 4096u && !(tz & 1);
      const bool okC = (uint32_t)d.code < (uint32_t)n_codes;
      const int ci = okC ? d.code : 0;
      const int64_t L = okC ? tabL[(size_t)ci * 7 + (okM ? tz >> 1 : 0)] : 0;
      const int64_t NW = (okC && okM) ? tabNW[(size_t)ci] : 0;
      ok &= !((d.sym_offset < es) | (d.cw_offset < ec));
      es = d.sym_offset + L;
      ec = d.cw_offset + NW;
    }
    if (!ok || es > n_symbols || ec > n_cw_words) {
      packed = false;
      break;
    }
    rc = issue_mixed_chunk(codes, n_codes, p, h_desc, hs, N0, h_cw, h_queries, h_abandon, f0, nk, sym_lo,
                           es - sym_lo, cw_lo, ec - cw_lo, false, pipe.s[k % kPipeStreams]);
    end_sym = es;
    end_cw = ec;
    f0 += nk;
  }
  if (rc == GRAND_OK && !packed) {
    for (int i = 0; i < kPipeStreams; ++i)  // the issued chunks' outputs are in h_cw before it is read
      if (cudaStreamSynchronize(pipe.s[i]) != cudaSuccess) rc = GRAND_E_CUDA;
    if (rc == GRAND_OK)
      rc = issue_mixed_chunk(codes, n_codes, p, h_desc, hs, N0, h_cw, h_queries, h_abandon, f0, n_frames - f0, 0,
                             n_symbols, 0, n_cw_words, true, pipe.s[0]);
  }
  return pipe.close(rc);
}
