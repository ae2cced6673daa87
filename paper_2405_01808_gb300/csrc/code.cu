// Host side of the library: version, status strings, the polar code helper
// (Def. II.1), the code object (column-packed H on the device) and the
// read-back of its deadline status word.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"

extern "C" int grand_version(void) { return GRAND_VERSION; }

extern "C" const char* grand_status_string(int s) {
  switch (s) {
    case GRAND_OK: return "ok";
    case GRAND_E_INVALID: return "invalid argument";
    case GRAND_E_RANK: return "parity-check matrix is not of full row rank";
    case GRAND_E_NOMEM: return "out of memory";
    case GRAND_E_CUDA: return "CUDA runtime error";
    case GRAND_E_TIMEOUT: return "bounded device wait ran out";
    case GRAND_E_BUSY: return "not admitted: no free slot or memory";
    case GRAND_E_UNSUPPORTED: return "outside the built limits";
    default: return "unknown status";
  }
}

static bool pow2_in_range(int N) { return N >= GRAND_N_MIN && N <= GRAND_N_MAX && (N & (N - 1)) == 0; }

// Polar code (Def. II.1). Entry (i, j) of G_N = F^{(x)n} is 1 exactly when the
// bits of j are a subset of those of i, so column f of G_N has ones at the
// rows j that contain f. Reliability: Bhattacharyya parameters of the BEC
// recursion (Arikan) -- child 2t gets 2z - z^2, child 2t+1 gets z^2.
extern "C" int grand_polar_H(int N, int K, double design_snr_db, uint32_t* H_out, int32_t* frozen_out) {
  if (!pow2_in_range(N) || K < 1 || K >= N || !H_out) return GRAND_E_INVALID;
  std::vector<double> z(1, exp(-(double)K / (double)N * pow(10.0, design_snr_db / 10.0)));
  while ((int)z.size() < N) {
    std::vector<double> nz(z.size() * 2);
    for (size_t t = 0; t < z.size(); ++t) {
      nz[2 * t] = 2.0 * z[t] - z[t] * z[t];
      nz[2 * t + 1] = z[t] * z[t];
    }
    z.swap(nz);
  }
  // the N-K least reliable indices; equal parameters: lower index first
  std::vector<int> idx(N);
  for (int i = 0; i < N; ++i) idx[i] = i;
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return z[a] > z[b]; });
  std::vector<int> frozen(idx.begin(), idx.begin() + (N - K));
  std::sort(frozen.begin(), frozen.end());
  const int words = N / 32;
  memset(H_out, 0, sizeof(uint32_t) * (size_t)(N - K) * words);
  for (int r = 0; r < N - K; ++r) {
    const int f = frozen[r];
    for (int j = 0; j < N; ++j)
      if ((j & f) == f) H_out[(size_t)r * words + (j >> 5)] |= 1u << (j & 31);
    if (frozen_out) frozen_out[r] = f;
  }
  return GRAND_OK;
}

// Row rank over GF(2) by Gaussian elimination on 64-bit words.
static int gf2_row_rank(const uint32_t* H, int R, int N) {
  const int W64 = N / 64 > 0 ? N / 64 : 1;
  std::vector<uint64_t> m((size_t)R * W64, 0);
  for (int r = 0; r < R; ++r)
    for (int j = 0; j < N; ++j)
      if ((H[(size_t)r * (N / 32) + (j >> 5)] >> (j & 31)) & 1u) m[(size_t)r * W64 + j / 64] |= 1ull << (j % 64);
  int rank = 0;
  for (int col = 0; col < N && rank < R; ++col) {
    const int w = col / 64;
    const uint64_t bit = 1ull << (col % 64);
    int piv = -1;
    for (int r = rank; r < R; ++r)
      if (m[(size_t)r * W64 + w] & bit) { piv = r; break; }
    if (piv < 0) continue;
    if (piv != rank)
      for (int k = 0; k < W64; ++k) std::swap(m[(size_t)piv * W64 + k], m[(size_t)rank * W64 + k]);
    for (int r = 0; r < R; ++r)
      if (r != rank && (m[(size_t)r * W64 + w] & bit))
        for (int k = 0; k < W64; ++k) m[(size_t)r * W64 + k] ^= m[(size_t)rank * W64 + k];
    ++rank;
  }
  return rank;
}

extern "C" int grand_code_create(const uint32_t* H, int N, int K, grand_code** out) {
  if (!H || !out || !pow2_in_range(N) || K < 1 || K >= N || N - K > 32 * grand::kWMax) return GRAND_E_INVALID;
  *out = nullptr;
  const int R = N - K;
  if (gf2_row_rank(H, R, N) != R) return GRAND_E_RANK;
  const int W = (R + 31) / 32;
  // column-packed copy: word w of column j holds rows 32w .. 32w+31; then the
  // per-column projections hf[j] (a fixed pseudo-random 32-bit word per row,
  // from the splitmix64 finaliser of the row index)
  // layout of the device copy: hcol [N*W], hf [N], prow [R], frozen [R] (u16, packed 2 per word),
  // hrow [R * N/32] (the rows as given)
  const size_t words = (size_t)N * W + N + R + (R + 1) / 2 + (size_t)R * (N / 32);
  std::vector<uint32_t> hcol(words, 0);
  uint32_t* hf = hcol.data() + (size_t)N * W;
  uint32_t* prow = hf + N;
  uint16_t* frozen = reinterpret_cast<uint16_t*>(prow + R);
  uint32_t* hrow = prow + R + (R + 1) / 2;
  memcpy(hrow, H, sizeof(uint32_t) * (size_t)R * (N / 32));
  bool polar = true;
  for (int r = 0; r < R; ++r) {
    uint64_t z = 0x9E3779B97F4A7C15ull * (uint64_t)(r + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const uint32_t pr = (uint32_t)z ^ (uint32_t)(z >> 32);
    prow[r] = pr;
    int first = -1;
    for (int j = 0; j < N; ++j)
      if ((H[(size_t)r * (N / 32) + (j >> 5)] >> (j & 31)) & 1u) {
        if (first < 0) first = j;
        hcol[(size_t)j * W + r / 32] |= 1u << (r % 32);
        hf[j] ^= pr;
      }
    // polar row: exactly the indices j that contain its first index f
    if (first < 0) {
      polar = false;
    } else {
      frozen[r] = (uint16_t)first;
      for (int j = 0; j < N && polar; ++j) {
        const bool bit = (H[(size_t)r * (N / 32) + (j >> 5)] >> (j & 31)) & 1u;
        if (bit != ((j & first) == first)) polar = false;
      }
    }
  }
  grand_code* c = (grand_code*)calloc(1, sizeof(grand_code));
  if (!c) return GRAND_E_NOMEM;
  c->N = N; c->K = K; c->R = R; c->W = W;
  if (cudaGetDevice(&c->device) != cudaSuccess) { free(c); return GRAND_E_CUDA; }
  if (cudaMalloc(&c->d_hcol, hcol.size() * sizeof(uint32_t)) != cudaSuccess) {
    free(c);
    return GRAND_E_NOMEM;
  }
  if (cudaMalloc(&c->d_dev, sizeof(grand::CodeDev)) != cudaSuccess) {
    cudaFree(c->d_hcol);
    free(c);
    return GRAND_E_NOMEM;
  }
  if (cudaMalloc(&c->d_status, 2 * sizeof(uint32_t)) != cudaSuccess) {
    cudaFree(c->d_hcol);
    cudaFree(c->d_dev);
    free(c);
    return GRAND_E_NOMEM;
  }
  c->dev.hcol = c->d_hcol;
  c->dev.hf = c->d_hcol + (size_t)N * W;
  c->dev.prow = c->dev.hf + N;
  c->dev.frozen = reinterpret_cast<const uint16_t*>(c->dev.prow + R);
  c->dev.hrow = c->dev.prow + R + (R + 1) / 2;
  c->dev.status = c->d_status;
  c->dev.N = N; c->dev.K = K; c->dev.R = R; c->dev.W = W;
  c->dev.polar = polar ? 1 : 0;
  if (cudaMemcpy(c->d_hcol, hcol.data(), hcol.size() * sizeof(uint32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->d_dev, &c->dev, sizeof(grand::CodeDev), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(c->d_status, 0, 2 * sizeof(uint32_t)) != cudaSuccess) {
    cudaFree(c->d_hcol);
    cudaFree(c->d_dev);
    cudaFree(c->d_status);
    free(c);
    return GRAND_E_CUDA;
  }
  *out = c;
  return GRAND_OK;
}

extern "C" int grand_code_destroy(grand_code* c) {
  if (!c) return GRAND_OK;
  cudaFree(c->d_hcol);
  cudaFree(c->d_dev);
  cudaFree(c->d_status);
  free(c);
  return GRAND_OK;
}

extern "C" int grand_code_info(const grand_code* c, int* N, int* K) {
  if (!c) return GRAND_E_INVALID;
  if (N) *N = c->N;
  if (K) *K = c->K;
  return GRAND_OK;
}

namespace {
// Take the code's status word with one atomic exchange (decodes on other
// streams may set it at any time) and leave the taken value in status[1].
__global__ void k_take_status(uint32_t* status) { status[1] = atomicExch(status, 0u); }
}  // namespace

// The watchdog's read-back: was a frame of a decode on this code cut at its
// deadline (grand_params.deadline_ns) since the last call?
extern "C" int grand_stream_status(const grand_code* c, void* stream) {
  if (!c) return GRAND_E_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaStreamSynchronize(st) != cudaSuccess) return GRAND_E_CUDA;
  k_take_status<<<1, 1, 0, st>>>(c->d_status);
  uint32_t h = 0;
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(&h, c->d_status + 1, sizeof h, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return GRAND_E_CUDA;
  return h ? GRAND_E_TIMEOUT : GRAND_OK;
}
