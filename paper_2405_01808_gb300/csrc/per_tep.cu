// Per-TEP decoding: one warp per frame demodulates it (Def. III.1 / III.2),
// selects the S' least reliable symbols (Alg. 2 Steps 2-3) and walks the
// valid TEPs in canonical order (Step 5), 32 altered-rank sets at a time: lane
// l takes one set of the current weight and steps through that set's
// alternatives in order, so the warp's lowest hitting lane holds the first hit.
//
// It serves what the split search of decode.cu does not: the five-point NNE
// order (up to four alternatives per symbol, no diagonal; the error model the
// paper contrasts with its own in Sec. II), and the two membership tests kept
// for comparison --
//   DELTA       z = s(y) xor the H columns the TEP flips (Alg. 2 Step 4),
//               filtered by a 32-bit projection and confirmed on all rows;
//   ROW_PARITY  the candidate y xor e multiplied by H row by row, each
//               syndrome bit the parity of (row AND word): the product of
//               Alg. 1 (pMult) evaluated for every TEP, stopping at the first
//               odd row.
// Results equal those of the split search (and of the CPU oracle) for every
// order; only the work per TEP differs.

#include <stdint.h>

#include "device_common.cuh"
#include "host_util.cuh"

namespace grand {
namespace {

constexpr unsigned kAll = 0xFFFFFFFFu;
constexpr int kAltMax = 4;  // alternatives per symbol (five-point NNE)
constexpr int kTepWarps = 4;

struct TepArgs {
  CodeDev code;
  const float2* symbols;
  int64_t n_frames;
  int m, side, L, Sp;
  int lik, order, rowparity;
  float q;
  uint32_t cap;
  uint32_t* cw;
  uint32_t* queries;
  uint8_t* abandon;
  unsigned int* next;            // frame work queue
  unsigned long long* counters;  // [0] TEPs tested, [1] frames past query 1, [2] their queries
  unsigned long long* t0;        // the call's clock start (deadline)
  long long deadline;            // grand_params.deadline_ns (0: none)
};

// Shared memory of one warp (words):
//   y[32] hard word, s0[kWMax] base syndrome, apos[kSMax][4] the (up to two)
//   bit positions of each alternative, aproj[kSMax][4] their projection,
//   sel[kSMax] selected symbols, kk[16] alternatives per rank (bytes),
//   key[L], info[L], and for the row test xs[N/32][32] (lane l's candidate
//   word in column l).
__host__ __device__ inline size_t tep_warp_bytes(int L, int NW, int rowparity) {
  size_t b = 4 * (32 + kWMax + 2 * kSMax * kAltMax + kSMax) + 16 + 8 * (size_t)L;
  if (rowparity) b += 4 * 32 * (size_t)NW;
  return (b + 15) & ~(size_t)15;
}

__device__ __forceinline__ void flip_lane(uint32_t* xs, int lane, uint32_t ap) {
  const uint32_t p0 = ap & 0xFFFFu, p1 = ap >> 16;
  if (p0 != kNoPos) xs[(p0 >> 5) * 32 + lane] ^= 1u << (p0 & 31);
  if (p1 != kNoPos) xs[(p1 >> 5) * 32 + lane] ^= 1u << (p1 & 31);
}

// H x = 0 for each live lane's candidate x (column `lane` of xs), by rows.
// Warp-collective: every lane calls it; the loop ends when no live lane has
// an all-even prefix of rows left.
__device__ bool row_parity_zero(const uint32_t* __restrict__ hrow, int R, int NW, const uint32_t* xs, int lane,
                                bool live) {
  bool zero = live;
  for (int r = 0; r < R; ++r) {
    if (!__any_sync(kAll, zero)) break;
    if (zero) {
      const uint32_t* h = hrow + (size_t)r * NW;
      uint32_t acc = 0;
      for (int w = 0; w < NW; ++w) acc ^= __ldg(h + w) & xs[w * 32 + lane];
      zero = (__popc(acc) & 1) == 0;
    }
  }
  return zero;
}

// Full syndrome of the TEP is zero: s0 xor the flipped H columns. The TEP is
// held packed: rank of position j in bits [4j, 4j+4) of pp, its alternative
// index in bits [2j, 2j+2) of dg.
__device__ bool delta_zero(const CodeDev& code, const uint32_t* s0, const uint32_t* apos, uint64_t pp, uint32_t dg,
                           int w) {
  for (int k = 0; k < code.W; ++k) {
    uint32_t v = s0[k];
    for (int j = 0; j < w; ++j) {
      const uint32_t ap = apos[(int)((pp >> (4 * j)) & 15u) * kAltMax + ((dg >> (2 * j)) & 3u)];
      const uint32_t p0 = ap & 0xFFFFu, p1 = ap >> 16;
      if (p0 != kNoPos) v ^= __ldg(code.hcol + (size_t)p0 * code.W + k);
      if (p1 != kNoPos) v ^= __ldg(code.hcol + (size_t)p1 * code.W + k);
    }
    if (v) return false;
  }
  return true;
}

__global__ void __launch_bounds__(32 * kTepWarps) k_per_tep(TepArgs a) {
  extern __shared__ __align__(16) char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const CodeDev& code = a.code;
  const int N = code.N, NW = N >> 5, L = a.L, Sp = a.Sp, m = a.m;
  char* base = smem_raw + (size_t)warp * tep_warp_bytes(L, NW, a.rowparity);
  uint32_t* y = reinterpret_cast<uint32_t*>(base);
  uint32_t* s0 = y + 32;
  uint32_t* apos = s0 + kWMax;
  uint32_t* aproj = apos + kSMax * kAltMax;
  int* sel = reinterpret_cast<int*>(aproj + kSMax * kAltMax);
  uint8_t* kk = reinterpret_cast<uint8_t*>(sel + kSMax);
  uint32_t* key = reinterpret_cast<uint32_t*>(kk + 16);
  uint32_t* info = key + L;
  uint32_t* xs = info + L;
  unsigned long long n_eval = 0, n_hard = 0, n_hard_q = 0;

  for (;;) {
    unsigned int fi = 0;
    if (lane == 0) fi = atomicAdd(a.next, 1u);
    fi = __shfl_sync(kAll, fi, 0);
    if ((int64_t)fi >= a.n_frames) break;
    const int64_t f = fi;

    // --- Step 1: demodulation and the hard word --------------------------
    if (lane < NW) y[lane] = 0u;
    __syncwarp();
    bool nonfinite = false;
    for (int i = lane; i < L; i += 32) {
      float2 sy = a.symbols[f * L + i];
      const bool nf = !(isfinite(sy.x) && isfinite(sy.y));
      if (nf) sy = make_float2(0.0f, 0.0f);
      nonfinite |= nf;
      const AxisDemod I = demod_axis_q(sy.x, a.q, a.side, a.lik);
      const AxisDemod Q = demod_axis_q(sy.y, a.q, a.side, a.lik);
      key[i] = (uint32_t)I.dq * (uint32_t)I.dq + (uint32_t)Q.dq * (uint32_t)Q.dq;
      info[i] = pack_info(I.level, Q.level, make_nmask(I, Q, nf));
      const uint32_t label = ((uint32_t)gray_code(I.level) << m) | (uint32_t)gray_code(Q.level);
      const uint32_t rl = __brev(label) >> (32 - 2 * m);  // bit k = label bit (2m-1-k)
      const int p0 = 2 * m * i, wd = p0 >> 5, sh = p0 & 31;
      if (wd < NW) atomicOr(&y[wd], rl << sh);
      if (sh && wd + 1 < NW) {
        const uint32_t hi = rl >> (32 - sh);
        if (hi) atomicOr(&y[wd + 1], hi);
      }
    }
    nonfinite = __any_sync(kAll, nonfinite);
    __syncwarp();
    if (nonfinite) {
      if (lane < NW) a.cw[f * NW + lane] = y[lane];
      if (lane == 0) {
        a.queries[f] = 0;
        a.abandon[f] = 2;
      }
      __syncwarp();
      continue;
    }
    if (a.deadline > 0) {
      int cut = 0;
      if (lane == 0) cut = past_deadline(a.t0, a.deadline);
      if (__shfl_sync(kAll, cut, 0)) {  // fetched after the deadline: the hard word, marked 5
        if (lane < NW) a.cw[f * NW + lane] = y[lane];
        if (lane == 0) {
          a.queries[f] = 0;
          a.abandon[f] = 5;
          atomicOr(code.status, 1u);
        }
        __syncwarp();
        continue;
      }
    }

    // --- base syndrome s0 = H y and its projection (delta test) ----------
    uint32_t f0 = 0;
    if (!a.rowparity) {
      uint32_t s[kWMax];
#pragma unroll
      for (int k = 0; k < kWMax; ++k) s[k] = 0u;
      for (int j = lane; j < N; j += 32) {
        if ((y[j >> 5] >> (j & 31)) & 1u) {
#pragma unroll
          for (int k = 0; k < kWMax; ++k)
            if (k < code.W) s[k] ^= __ldg(code.hcol + (size_t)j * code.W + k);
          f0 ^= __ldg(code.hf + j);
        }
      }
#pragma unroll
      for (int k = 0; k < kWMax; ++k) {
        if (k < code.W) {  // warp-uniform bound
          uint32_t v = s[k];
          for (int o = 16; o; o >>= 1) v ^= __shfl_xor_sync(kAll, v, o);
          if (lane == 0) s0[k] = v;
        }
      }
      for (int o = 16; o; o >>= 1) f0 ^= __shfl_xor_sync(kAll, f0, o);
    }

    // --- Steps 2-3: the S' least reliable symbols, by (key, index) -------
    for (int r = 0; r < Sp; ++r) {
      uint32_t bk = 0xFFFFFFFFu, bi = 0xFFFFFFFFu;
      for (int i = lane; i < L; i += 32) {
        const uint32_t k = key[i];
        if (k < bk) {
          bk = k;
          bi = (uint32_t)i;
        }
      }
      const uint32_t kmin = __reduce_min_sync(kAll, bk);
      const uint32_t imin = __reduce_min_sync(kAll, bk == kmin ? bi : 0xFFFFFFFFu);
      if (lane == 0) sel[r] = (int)imin;
      if (lane == (int)(imin & 31u)) key[imin] = 0xFFFFFFFFu;  // keys are < 2^31
      __syncwarp();
    }

    // --- Step 4: the alternatives of each rank, in their query order -----
    if (lane < Sp) {
      const int i = sel[lane];
      const uint32_t inf = info[i];
      const int lI = inf & 0xFF, lQ = (inf >> 8) & 0xFF;
      const uint32_t nm = (inf >> 16) & 0xFF;
      const bool exI = nm & 1u, exQ = nm & 2u;
      const int dI = (nm & 8u) ? 1 : -1, dQ = (nm & 16u) ? 1 : -1;
      const uint32_t pI = exI ? flip_pos_I(i, m, lI, dI, N) : kNoPos;
      const uint32_t pQ = exQ ? flip_pos_Q(i, m, lQ, dQ, N) : kNoPos;
      const uint32_t none = (uint32_t)kNoPos << 16;
      uint32_t list[kAltMax];
      int n = 0;
      if (a.order == GRAND_ORDER_QAM_NNE5) {
        // toward the received value on I, on Q; away from it on I, on Q
        if (exI) list[n++] = pI | none;
        if (exQ) list[n++] = pQ | none;
        if (lI - dI >= 0 && lI - dI < a.side) list[n++] = flip_pos_I(i, m, lI, -dI, N) | none;
        if (lQ - dQ >= 0 && lQ - dQ < a.side) list[n++] = flip_pos_Q(i, m, lQ, -dQ, N) | none;
      } else {
        // h, v, diag (Def. III.2); the nearer order puts v first where d_Q < d_I
        const bool swap = a.order == GRAND_ORDER_QAM_NEARER && (nm & 32u);
        const bool e1 = swap ? exQ : exI, e2 = swap ? exI : exQ;
        const uint32_t q1 = swap ? pQ : pI, q2 = swap ? pI : pQ;
        if (e1) list[n++] = q1 | none;
        if (e2) list[n++] = q2 | none;
        if (exI && exQ) list[n++] = pI | (pQ << 16);
      }
      for (int k = 0; k < kAltMax; ++k) {
        const uint32_t ap = k < n ? list[k] : ((uint32_t)kNoPos | none);
        const uint32_t p0 = ap & 0xFFFFu, p1 = ap >> 16;
        apos[lane * kAltMax + k] = ap;
        aproj[lane * kAltMax + k] =
            (p0 != kNoPos ? __ldg(code.hf + p0) : 0u) ^ (p1 != kNoPos ? __ldg(code.hf + p1) : 0u);
      }
      kk[lane] = (uint8_t)n;
    }
    __syncwarp();

    // --- Step 5: the canonical walk ----------------------------------------
    const uint32_t cap = a.cap;
    uint32_t cum = 0;  // valid TEPs of the batches already walked
    bool found = false;
    uint32_t hit_rank = 0;
    int hit_lane = -1, w_hit = 0;
    // the lane's TEP, packed: pp = ranks (4 bits per position, ascending),
    // dg = alternative indices (2 bits), km = alternatives - 1 (2 bits)
    uint64_t pp = 0;
    uint32_t dg = 0, km = 0;
    for (int w = 0; w <= Sp && !found && cum < cap; ++w) {
      const uint32_t nsets = binom16(Sp, w);
      for (uint32_t b0 = 0; b0 < nsets && !found && cum < cap;) {
        // m sets in this batch, P lanes per set: lane l takes part l % P of
        // set b0 + l / P (parts split the set's alternatives in order, so
        // lane order stays canonical order)
        const uint32_t m = min(32u, nsets - b0);
        const uint32_t P = 32u / m;
        const uint32_t si = b0 + (uint32_t)lane / P;
        const uint32_t part = (uint32_t)lane % P;
        const bool has_set = (uint32_t)lane < m * P;
        b0 += m;
        uint32_t nalpha = 0;
        pp = 0;
        km = 0;
        if (has_set) {
          // colex unranking: the largest rank first
          uint32_t t = si;
          nalpha = 1;
          for (int j = w; j >= 1; --j) {
            int p = j - 1;
            while (binom16(p + 1, j) <= t) ++p;
            t -= binom16(p, j);
            pp |= (uint64_t)p << (4 * (j - 1));
            const uint32_t k = kk[p];
            nalpha *= k;
            km |= ((k ? k : 1u) - 1u) << (2 * (j - 1));
          }
        }
        // this lane's part of the set's alternatives: [a0, a0 + n_lane)
        const uint32_t chunk = (nalpha + P - 1) / P;
        const uint32_t a0 = part * chunk;
        const uint32_t n_lane = a0 < nalpha ? min(chunk, nalpha - a0) : 0u;
        uint32_t incl = n_lane;
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t v = __shfl_up_sync(kAll, incl, o);
          if (lane >= o) incl += v;
        }
        const uint32_t batch = __shfl_sync(kAll, incl, 31);
        const uint32_t first = cum + (incl - n_lane) + 1;  // 1-based position of the lane's first TEP
        uint32_t n_here = 0;
        if (n_lane && first <= cap) n_here = min(n_lane, cap - first + 1);
        // alternative indices of the part's first TEP: a0 in mixed radix,
        // the smallest rank the least significant digit
        uint32_t z = f0;
        dg = 0;
        if (n_here) {
          uint32_t rest = a0;
          for (int j = 0; j < w; ++j) {
            const uint32_t k = ((km >> (2 * j)) & 3u) + 1u;
            const uint32_t d = rest % k;
            rest /= k;
            dg |= d << (2 * j);
            z ^= aproj[(int)((pp >> (4 * j)) & 15u) * kAltMax + d];
          }
        }
        if (a.rowparity) {
          for (int k = 0; k < NW; ++k) xs[k * 32 + lane] = y[k];
          if (n_here)
            for (int j = 0; j < w; ++j)
              flip_lane(xs, lane, apos[(int)((pp >> (4 * j)) & 15u) * kAltMax + ((dg >> (2 * j)) & 3u)]);
        }
        bool live = n_here > 0, hit = false;
        uint32_t ai = 0;
        for (;;) {
          bool h;
          if (a.rowparity)
            h = row_parity_zero(code.hrow, code.R, NW, xs, lane, live);
          else
            h = live && z == 0u && delta_zero(code, s0, apos, pp, dg, w);
          n_eval += live ? 1u : 0u;
          if (h) {
            hit = true;
            live = false;
          }
          if (live) {
            if (++ai >= n_here) {
              live = false;
            } else {
              // next alternative tuple: mixed-radix increment, smallest rank fastest
              for (int j = 0; j < w; ++j) {
                const int sh = 2 * j;
                const int r = (int)((pp >> (4 * j)) & 15u);
                const uint32_t d = (dg >> sh) & 3u;
                const uint32_t nd = d == ((km >> sh) & 3u) ? 0u : d + 1u;
                z ^= aproj[r * kAltMax + d] ^ aproj[r * kAltMax + nd];
                if (a.rowparity) {
                  flip_lane(xs, lane, apos[r * kAltMax + d]);
                  flip_lane(xs, lane, apos[r * kAltMax + nd]);
                }
                dg = (dg & ~(3u << sh)) | (nd << sh);
                if (nd) break;
              }
            }
          }
          const unsigned hm = __ballot_sync(kAll, hit);
          const unsigned lm = __ballot_sync(kAll, live);
          if (hm && !(lm & ((hm & (0u - hm)) - 1u))) break;  // nothing live below the lowest hit
          if (!lm) break;
        }
        const unsigned hm = __ballot_sync(kAll, hit);
        if (hm) {
          hit_lane = __ffs(hm) - 1;
          hit_rank = __shfl_sync(kAll, first + ai, hit_lane);
          w_hit = w;
          found = true;
        }
        cum += batch;
      }
    }

    // --- Return: x = y xor e of the first hit, else y ---------------------
    if (found && lane == hit_lane) {
      for (int j = 0; j < w_hit; ++j) {
        const uint32_t ap = apos[(int)((pp >> (4 * j)) & 15u) * kAltMax + ((dg >> (2 * j)) & 3u)];
        const uint32_t p0 = ap & 0xFFFFu, p1 = ap >> 16;
        if (p0 != kNoPos) y[p0 >> 5] ^= 1u << (p0 & 31);
        if (p1 != kNoPos) y[p1 >> 5] ^= 1u << (p1 & 31);
      }
    }
    __syncwarp();
    if (lane < NW) a.cw[f * NW + lane] = y[lane];
    if (lane == 0) {
      const uint32_t qn = found ? hit_rank : min(cum, cap);
      a.queries[f] = qn;
      a.abandon[f] = found ? 0 : 1;
      if (!(found && hit_rank == 1)) {
        n_hard += 1;
        n_hard_q += qn;
      }
    }
    __syncwarp();
  }
  for (int o = 16; o; o >>= 1) n_eval += __shfl_xor_sync(kAll, n_eval, o);
  if (lane == 0) {
    atomicAdd(a.counters + 0, n_eval);
    if (n_hard) {
      atomicAdd(a.counters + 1, n_hard);
      atomicAdd(a.counters + 2, n_hard_q);
    }
  }
}

}  // namespace

int run_per_tep(const grand_code* c, const grand_params* p, const void* symbols, int64_t n_frames, uint32_t* cw,
                uint32_t* queries, uint8_t* abandon, grand_stats* stats, cudaStream_t st) {
  if (n_frames == 0) {
    if (stats) *stats = grand_stats{};
    return GRAND_OK;
  }
  NvtxRange range("grand.per_tep");
  const int m = m_of(p->M);
  TepArgs a{};
  a.code = c->dev;
  a.symbols = static_cast<const float2*>(symbols);
  a.n_frames = n_frames;
  a.m = m;
  a.side = 1 << m;
  a.L = (c->N + 2 * m - 1) / (2 * m);
  a.Sp = p->S < a.L ? p->S : a.L;
  a.lik = p->lik_variant;
  a.order = p->order;
  a.rowparity = p->membership == GRAND_MEMBERSHIP_ROW_PARITY ? 1 : 0;
  a.q = make_qam_const().q[m];
  a.cap = (uint32_t)(p->query_cap < 0xFFFFFFFFll ? p->query_cap : 0xFFFFFFFFll);
  a.cw = cw;
  a.queries = queries;
  a.abandon = abandon;
  char* scratch = nullptr;
  if (scratch_alloc((void**)&scratch, 64, st) != cudaSuccess) return GRAND_E_NOMEM;
  a.next = reinterpret_cast<unsigned int*>(scratch);
  a.counters = reinterpret_cast<unsigned long long*>(scratch + 8);
  a.t0 = reinterpret_cast<unsigned long long*>(scratch + 32);
  a.deadline = p->deadline_ns;
  int rc = GRAND_OK;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  do {
    if (cudaMemsetAsync(scratch, 0, 64, st) != cudaSuccess) { rc = GRAND_E_CUDA; break; }
    const size_t smem = kTepWarps * tep_warp_bytes(a.L, c->N / 32, a.rowparity);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k_per_tep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
      rc = GRAND_E_CUDA;
      break;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_per_tep, 32 * kTepWarps, smem) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    const int64_t want = (n_frames + kTepWarps - 1) / kTepWarps;
    const int64_t full = (int64_t)sm_count() * per_sm;
    const int grid = (int)(want < full ? want : full);
    if (stats) {
      for (int i = 0; i < 2; ++i)
        if (cudaEventCreate(&ev[i]) != cudaSuccess) { rc = GRAND_E_CUDA; break; }
      if (rc) break;
      cudaEventRecord(ev[0], st);
    }
    k_per_tep<<<grid, 32 * kTepWarps, smem, st>>>(a);
    if (cudaGetLastError() != cudaSuccess) { rc = GRAND_E_CUDA; break; }
    if (stats) {
      cudaEventRecord(ev[1], st);
      unsigned long long h[3] = {0, 0, 0};
      if (cudaMemcpyAsync(h, a.counters, sizeof h, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess) {
        rc = GRAND_E_CUDA;
        break;
      }
      *stats = grand_stats{};
      stats->evaluated_checks = h[0];
      stats->hard_frames = h[1];
      stats->search_useful = h[2];
      stats->prep_ms = 0.0f;
      cudaEventElapsedTime(&stats->search_ms, ev[0], ev[1]);
    }
  } while (0);
  for (int i = 0; i < 2; ++i)
    if (ev[i]) cudaEventDestroy(ev[i]);
  cudaFreeAsync(scratch, st);
  return rc;
}

}  // namespace grand
