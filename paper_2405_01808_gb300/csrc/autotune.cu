// Launch-shape autotuner: times candidate `grand_params.tiles` (and, with
// GRAND_MEMBERSHIP_FASTEST, the two exact membership tests) on a sample batch
// with CUDA events and keeps the fastest; results do not depend on the
// choice, only the time does. Choices are cached in a text file keyed by the
// GPU name and the workload (code sizes, constellation, cut-off, cap).
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <initializer_list>
#include <functional>
#include <string>
#include <vector>

#include "internal.cuh"

namespace {

struct Candidate {
  int32_t tiles[4];
  int32_t membership;
};

// Launch shapes of one membership test.
void shapes(int S, int membership, std::vector<Candidate>& out) {
  if (membership == GRAND_MEMBERSHIP_HASH) {
    // hash join: warps per CTA (its shared-memory tables bound residency) x prep weights
    // (static arrays: the backing array of a braced list chosen by ?: would not
    // outlive the range-for's initialisation)
    static const int kWarpsS10[2] = {2, 4}, kWarpsS12[2] = {1, 2};
    const int* warps = S <= 10 ? kWarpsS10 : kWarpsS12;
    for (int i = 0; i < 2; ++i)
      for (int w0 : {1, 2, 3}) out.push_back({{warps[i], 0, w0, 0}, membership});
  } else if (S <= 10) {
    // warp search (warp pairs sharing a frame): prep weights x register budget
    for (int w0 : {1, 2, 3})
      for (int regs : {4, 6, 8}) out.push_back({{0, 0, w0, regs}, membership});
  } else {
    // warp search with a 7-rank B side: warp pairs or one warp per frame
    // (CTAs of 1, 2, 4 warps) x prep weights x register budget
    for (int warps : {0, 1, 2, 4})
      for (int w0 : {2, 3})
        for (int regs : {4, 6}) out.push_back({{warps, 0, w0, regs}, membership});
  }
}

// The candidates: the launch shapes of the params' membership test, or with
// GRAND_MEMBERSHIP_FASTEST those of both exact tests (the TEP-by-TEP split
// search and the hash join), whose outputs are identical.
std::vector<Candidate> candidates(int S, int membership) {
  std::vector<Candidate> out;
  if (membership == GRAND_MEMBERSHIP_FASTEST) {
    shapes(S, GRAND_MEMBERSHIP_AUTO, out);
    shapes(S, GRAND_MEMBERSHIP_HASH, out);
  } else {
    shapes(S, membership, out);
  }
  return out;
}

std::string device_name() {
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
  std::string n = prop.name;
  for (char& c : n)
    if (c == ' ' || c == '|') c = '_';
  return n;
}

// Cache lines: "key t0 t1 t2 t3 ms membership" (lines without the membership
// field keep the params' membership).
bool cache_lookup(const char* path, const std::string& key, int32_t tiles[4], int32_t* membership) {
  if (!path) return false;
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char line[512];
  bool found = false;
  while (fgets(line, sizeof line, f)) {
    char k[384];
    int t[4], mem = -1;
    float ms;
    const int n = sscanf(line, "%383s %d %d %d %d %f %d", k, &t[0], &t[1], &t[2], &t[3], &ms, &mem);
    if (n >= 6 && key == k) {
      for (int i = 0; i < 4; ++i) tiles[i] = t[i];
      if (n == 7 && (mem == GRAND_MEMBERSHIP_AUTO || mem == GRAND_MEMBERSHIP_HASH)) *membership = mem;
      found = true;  // the last entry for a key wins
    }
  }
  fclose(f);
  return found;
}

void cache_store(const char* path, const std::string& key, const int32_t tiles[4], float ms, int32_t membership) {
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %d %d %d %d %.4f %d\n", key.c_str(), tiles[0], tiles[1], tiles[2], tiles[3], ms, membership);
  fclose(f);
}

// Median of `reps` timed runs (after one untimed run) of `run`.
int time_runs(const std::function<int(cudaStream_t)>& run, cudaStream_t st, int reps, float* ms_out) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return GRAND_E_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return GRAND_E_CUDA;
  }
  int rc = run(st);
  std::vector<float> t;
  for (int r = 0; r < reps && rc == GRAND_OK; ++r) {
    cudaEventRecord(e0, st);
    rc = run(st);
    cudaEventRecord(e1, st);
    if (rc == GRAND_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = GRAND_E_CUDA;
    float ms = 0;
    if (rc == GRAND_OK) cudaEventElapsedTime(&ms, e0, e1);
    t.push_back(ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != GRAND_OK) return rc;
  std::sort(t.begin(), t.end());
  *ms_out = t[t.size() / 2];
  return GRAND_OK;
}

int tune(const std::string& key, grand_params* p, const char* cache_path, cudaStream_t st,
         const std::function<int(const grand_params*, cudaStream_t)>& run, grand_tune_result* res) {
  int32_t cached[4];
  int32_t cached_mem = p->membership == GRAND_MEMBERSHIP_FASTEST ? GRAND_MEMBERSHIP_AUTO : p->membership;
  if (cache_lookup(cache_path, key, cached, &cached_mem)) {
    for (int i = 0; i < 4; ++i) p->tiles[i] = cached[i];
    p->membership = cached_mem;
    if (res) {
      memset(res, 0, sizeof *res);
      res->from_cache = 1;
      res->membership = cached_mem;
    }
    return GRAND_OK;
  }
  float best = 1e30f;
  Candidate best_c{{0, 0, 0, 0}, p->membership};
  int tried = 0;
  for (const Candidate& c : candidates(p->S, p->membership)) {
    grand_params q = *p;
    for (int i = 0; i < 4; ++i) q.tiles[i] = c.tiles[i];
    q.membership = c.membership;
    q.deadline_ns = 0;  // time every candidate in full
    float ms = 0;
    const int rc = time_runs([&](cudaStream_t s) { return run(&q, s); }, st, 3, &ms);
    if (rc != GRAND_OK) return rc;
    ++tried;
    if (ms < best) {
      best = ms;
      best_c = c;
    }
  }
  for (int i = 0; i < 4; ++i) p->tiles[i] = best_c.tiles[i];
  p->membership = best_c.membership;
  cache_store(cache_path, key, p->tiles, best, p->membership);
  if (res) {
    res->best_ms = best;
    res->candidates = tried;
    res->from_cache = 0;
    res->membership = p->membership;
  }
  return GRAND_OK;
}

}  // namespace

extern "C" int grand_autotune(const grand_code* c, grand_params* p, const void* symbols, int64_t n_frames, float N0,
                              const char* cache_path, void* stream, grand_tune_result* res) {
  if (!c || !p || !symbols || n_frames < 1 ||
      (p->order != GRAND_ORDER_QAM_NNE && p->order != GRAND_ORDER_QAM_NEARER) ||
      (p->membership != GRAND_MEMBERSHIP_AUTO && p->membership != GRAND_MEMBERSHIP_HASH &&
       p->membership != GRAND_MEMBERSHIP_FASTEST))
    return GRAND_E_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  const int N = c->N, W = c->N / 32;
  uint32_t* cw = nullptr;
  uint32_t* q = nullptr;
  uint8_t* ab = nullptr;
  if (cudaMalloc(&cw, sizeof(uint32_t) * n_frames * W) != cudaSuccess) return GRAND_E_NOMEM;
  if (cudaMalloc(&q, sizeof(uint32_t) * n_frames) != cudaSuccess || cudaMalloc(&ab, n_frames) != cudaSuccess) {
    cudaFree(cw);
    cudaFree(q);
    return GRAND_E_NOMEM;
  }
  char key[384];
  snprintf(key, sizeof key, "%s|sym|N=%d|K=%d|M=%d|S=%d|cap=%lld|lik=%d|ord=%d|mem=%d", device_name().c_str(), N,
           c->K, p->M, p->S, (long long)p->query_cap, p->lik_variant, p->order, p->membership);
  const int rc = tune(
      key, p, cache_path, st,
      [&](const grand_params* pp, cudaStream_t s) {
        return grand_decode_symbols(c, pp, symbols, n_frames, N0, cw, q, ab, nullptr, s);
      },
      res);
  cudaFree(cw);
  cudaFree(q);
  cudaFree(ab);
  return rc;
}

extern "C" int grand_autotune_mixed(const grand_code* const* codes, int n_codes, grand_params* p,
                                    const grand_frame_desc* desc, int64_t n_frames, const void* symbols,
                                    int64_t n_symbols, float N0, int64_t n_cw_words, const char* cache_path,
                                    void* stream, grand_tune_result* res) {
  if (!codes || n_codes < 1 || !p || !desc || !symbols || n_frames < 1 || n_cw_words < 1) return GRAND_E_INVALID;
  if (p->membership != GRAND_MEMBERSHIP_AUTO && p->membership != GRAND_MEMBERSHIP_HASH &&
      p->membership != GRAND_MEMBERSHIP_FASTEST)
    return GRAND_E_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t* cw = nullptr;
  uint32_t* q = nullptr;
  uint8_t* ab = nullptr;
  if (cudaMalloc(&cw, sizeof(uint32_t) * n_cw_words) != cudaSuccess) return GRAND_E_NOMEM;
  if (cudaMalloc(&q, sizeof(uint32_t) * n_frames) != cudaSuccess || cudaMalloc(&ab, n_frames) != cudaSuccess) {
    cudaFree(cw);
    cudaFree(q);
    return GRAND_E_NOMEM;
  }
  std::string key = device_name() + "|mixed|codes=";
  for (int i = 0; i < n_codes; ++i) {
    if (!codes[i]) {
      cudaFree(cw);
      cudaFree(q);
      cudaFree(ab);
      return GRAND_E_INVALID;
    }
    key += std::to_string(codes[i]->N) + "/" + std::to_string(codes[i]->K) + (i + 1 < n_codes ? "," : "");
  }
  key += "|S=" + std::to_string(p->S) + "|cap=" + std::to_string((long long)p->query_cap) +
         "|lik=" + std::to_string(p->lik_variant) + "|ord=" + std::to_string(p->order) +
         "|mem=" + std::to_string(p->membership);
  const int rc = tune(
      key, p, cache_path, st,
      [&](const grand_params* pp, cudaStream_t s) {
        return grand_decode_mixed(codes, n_codes, pp, desc, n_frames, symbols, n_symbols, N0, cw, n_cw_words, q, ab,
                                  nullptr, s);
      },
      res);
  cudaFree(cw);
  cudaFree(q);
  cudaFree(ab);
  return rc;
}
