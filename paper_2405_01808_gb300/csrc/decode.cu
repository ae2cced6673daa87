// GRAND decoder kernels for sm_103a and the C ABI entry points.
//
// Stages of one decode call (Alg. 2 of the paper):
//   k_prep         one warp per frame: demodulation + likelihood + neighbours
//                  (Step 1), hard word y and base syndrome s0 = H y, selection
//                  of the S' least reliable symbols (Steps 2-3), the syndrome
//                  deltas of their alternatives (Step 4), and the first TEP
//                  weights in canonical order (Step 5). Most frames finish
//                  here; the others leave a hand-off record.
//   k_search_warp  the search of the rest of the TEP space (Step 5), one warp
//                  per frame from a work queue: the S' ranks are split into a
//                  low group A and a high group B, every valid alternative
//                  assignment of each group gets its partial syndrome, and a
//                  TEP (a, b) is a codeword iff
//                      s0 ^ D_A(a) == D_B(b)            (all syndrome words).
//                  The comparison is bit-sliced on a syndrome projection (32
//                  TEPs per 3-input logic op per projection bit), candidates
//                  are confirmed on every word and ranked in closed form.
//                  Sides of 5 ranks (S' <= 10) or 6 ranks (S' = 11, 12).
//   k_search_hash  the same decision by a hash join of the two sides
//                  (membership GRAND_MEMBERSHIP_HASH).
//   k_search       the split with one CTA per frame (explicit split in the
//                  launch shape): one projection compare per TEP.
//   k_ab           bit-level GRAND-AB (Sec. I), one warp per frame.
//   k_demod        the public demodulation call (per-symbol outputs).
// The five-point NNE order and the per-TEP membership tests are in per_tep.cu.
#include <stdio.h>

#include <mutex>
#include <type_traits>
#include <vector>

#include "device_common.cuh"
#include "host_util.cuh"

namespace grand {

constexpr unsigned kFull = 0xFFFFFFFFu;

// ---------------------------------------------------------------------------
// Launch-wide parameters
// ---------------------------------------------------------------------------

struct PrepArgs {
  // fused path: received symbols; else the demodulated arrays
  const float2* symbols;
  const uint16_t* hard_idx;
  const uint32_t* key;
  const uint8_t* nmask;
  const uint32_t* y_in;
  const grand_frame_desc* desc;  // NULL: uniform batch
  int64_t n_symbols;             // mixed: length of the flat symbol array
  int64_t n_cw_words;            // mixed: length of the flat output array
  const CodeDev* codes;          // device table
  int n_codes;
  int64_t n_frames;
  int M;                         // uniform batch
  int S;
  int lik;
  int nearer;                    // GRAND_ORDER_QAM_NEARER: swap h / v where d_Q < d_I
  int w0;
  int Lmax;
  int Wmax;
  int64_t cap;
  QamConst qc;
  uint32_t* cw;
  uint32_t* queries;
  uint8_t* abandon;
  FrameRec* recs;
  Scratch* scr;
  long long deadline;            // grand_params.deadline_ns (0: none)
};

struct SearchArgs {
  const FrameRec* recs;
  const CodeDev* codes;
  Scratch* scr;
  int64_t cap;
  int split;       // 0 = automatic (S'/2)
  int tabA, tabB;  // table capacities
  int max_tiles;
  int Wmax;
  int warp_kernel;  // 1 / 2: warp-per-frame flip-bit search, S' <= 10 / 12 (automatic split); 0: CTA kernel;
                    // 3 / 4: hash join (membership HASH) with 5- / 6-rank sides
  int warps;        // warps per CTA of the warp-per-frame kernels (0: their default)
  uint32_t* cw;
  uint32_t* queries;
  uint8_t* abandon;
  long long deadline;  // grand_params.deadline_ns (0: none)
  // Resumable search (weight windows). w_step > 0: a frame's search covers the
  // TEP weights w_done + 1 .. w_done + w_step only; a frame with no hit there
  // and weights left below the cap is suspended (abandon 6, queries = the
  // valid TEPs tested so far) and its record, with w_done advanced, is written
  // to cur_out[frame]. cur_in != NULL: the work queue runs over the n_cur
  // records of cur_in instead of the preparation's (record i writes its
  // outputs at index i, cw at i * cw_stride) and skips those whose abandon
  // flag is not 6; cur_out may equal cur_in.
  int w_step;
  FrameRec* cur_out;
  const FrameRec* cur_in;
  int64_t n_cur;
  int64_t cw_stride;
  int n_codes;  // entries of `codes` (a cursor naming another code is rejected)
  int sp_max;   // largest S' the launched kernel's tables hold
  int64_t max_entries;  // bound on the queue's length (the grid needs no more warps)
};

// CTAs of a persistent search launch: one wave (every SM full), or fewer when
// the queue cannot have more entries than that many CTAs' warps (a small
// batch then dispatches no CTAs that would only find the queue empty).
static inline int search_grid(int per_sm, int warps_per_cta, int64_t max_entries) {
  const int64_t full = (int64_t)sm_count() * per_sm;
  const int64_t need = max_entries > 0 ? (max_entries + warps_per_cta - 1) / warps_per_cta : full;
  return (int)(need < full ? (need > 0 ? need : 1) : full);
}

// Output slot of queue entry fi: the batch frame of a preparation record, or
// the cursor's own index when resuming (computed where needed, so that none of
// it stays live in registers during the search).
__device__ __forceinline__ uint32_t out_frame(const SearchArgs& a, unsigned fi, const FrameRec* rec) {
  return a.cur_in ? fi : rec->frame;
}
__device__ __forceinline__ int64_t out_cw_off(const SearchArgs& a, unsigned fi, const FrameRec* rec) {
  return a.cur_in ? (int64_t)fi * a.cw_stride : rec->cw_off;
}

// Cursor validation of the resume queue (outlined: it is not on the path of
// an ordinary decode): a cursor is read only if it describes a search the
// kernel can run -- a known code, 1 <= S' <= the kernel's bound, w_done < S',
// existing-alternative masks and flip positions inside the code; otherwise
// the entry gets abandon 3. Returns whether to search it.
__device__ __noinline__ bool resume_entry_ok(const SearchArgs& a, unsigned fi) {
  const FrameRec* rec = a.cur_in + fi;
  if (a.abandon[fi] != GRAND_ABANDON_SUSPENDED) return false;
  const int lane = threadIdx.x & 31;
  bool ok = rec->code < (unsigned)a.n_codes;
  const int sp = rec->sp;
  ok = ok && sp >= 1 && sp <= a.sp_max && rec->w_done < sp;
  if (ok) {
    const CodeDev& c = a.codes[rec->code];
    bool mine = true;
    if (lane < sp) {
      const uint16_t p0 = rec->pos[lane][0], p1 = rec->pos[lane][1];
      // the diagonal alternative exists exactly when both single-axis ones do
      const uint32_t e = rec->ex[lane];
      mine = (p0 == kNoPos || p0 < c.N) && (p1 == kNoPos || p1 < c.N) && (e & ~7u) == 0 &&
             ((e >> 2) & 1u) == (e & (e >> 1) & 1u);
    }
    ok = __all_sync(kFull, mine);
  }
  if (!ok) {
    __syncwarp();
    if (lane == 0) {
      a.abandon[fi] = 3;
      a.queries[fi] = 0;
    }
  }
  return ok;
}

// The record of queue entry fi, or NULL when there is nothing to search.
__device__ __forceinline__ const FrameRec* queue_entry(const SearchArgs& a, unsigned fi) {
  if (a.cur_in) return resume_entry_ok(a, fi) ? a.cur_in + fi : nullptr;
  return a.recs + fi;
}

// Suspend a frame (one warp): its record with w_done advanced to w_hi goes to
// its cursor slot; outputs say abandon 6 with the valid TEPs tested so far.
// The hard word stays in cw (the preparation wrote it).
__device__ __noinline__ void suspend_frame(const SearchArgs& a, unsigned fi, const FrameRec* rec, int w_hi,
                                           uint32_t tested) {
  const int lane = threadIdx.x & 31;
  static_assert(sizeof(FrameRec) % 4 == 0, "FrameRec words");
  constexpr int kWords = (int)(sizeof(FrameRec) / 4);
  const uint32_t frame = out_frame(a, fi, rec);
  FrameRec* cursor = a.cur_out ? a.cur_out + frame : nullptr;
  const uint32_t* src = reinterpret_cast<const uint32_t*>(rec);
  uint32_t* dst = reinterpret_cast<uint32_t*>(cursor);
  uint32_t v[(kWords + 31) / 32];
#pragma unroll
  for (int k = 0; k < (kWords + 31) / 32; ++k) v[k] = (lane + 32 * k < kWords) ? src[lane + 32 * k] : 0u;
  __syncwarp();  // every lane read the record before any lane writes (the cursor may be the record)
  if (dst) {
#pragma unroll
    for (int k = 0; k < (kWords + 31) / 32; ++k)
      if (lane + 32 * k < kWords) dst[lane + 32 * k] = v[k];
    __syncwarp();
    if (lane == 0) cursor->w_done = (uint8_t)w_hi;
  }
  if (lane == 0) {
    a.queries[frame] = tested;
    a.abandon[frame] = GRAND_ABANDON_SUSPENDED;
  }
}

// A hard frame fetched after the call's deadline (lane 0): it keeps what the
// preparation wrote (cw = the hard word, queries = the valid TEPs it tested
// without a hit) and is marked abandon 5; the code's status word records it.
__device__ __forceinline__ bool cut_at_deadline(const SearchArgs& a, const FrameRec* rec, uint32_t frame) {
  if (!past_deadline(&a.scr->t0, a.deadline)) return false;
  a.abandon[frame] = 5;
  atomicOr(a.codes[rec->code].status, 1u);
  return true;
}

// ---------------------------------------------------------------------------
// Per-frame preparation (one warp per frame)
// ---------------------------------------------------------------------------
struct PrepSmem {
  uint32_t* key;    // [Lmax]
  uint32_t* info;   // [Lmax]
  uint32_t* y;      // [32]
  uint32_t* delta;  // [kSMax][3][Wmax]
  uint32_t* dflt;   // [kSMax][3] projections of the deltas
  uint32_t* E;      // [kEStride^2]
  uint32_t* s0;     // [Wmax] base syndrome
  uint8_t* ex;      // [kSMax]
  uint16_t* pos;    // [kSMax][2]
};

__host__ __device__ inline size_t prep_warp_bytes(int Lmax, int Wmax) {
  size_t words = 2 * (size_t)Lmax + 32 + (size_t)kSMax * 3 * Wmax + kSMax * 3 + kEStride * kEStride + Wmax +
                 kSMax / 4 + 1 + kSMax;
  return ((words * 4) + 15) & ~(size_t)15;
}

__device__ inline PrepSmem prep_smem(char* base, int Lmax, int Wmax) {
  PrepSmem s;
  uint32_t* p = reinterpret_cast<uint32_t*>(base);
  s.key = p; p += Lmax;
  s.info = p; p += Lmax;
  s.y = p; p += 32;
  s.delta = p; p += kSMax * 3 * Wmax;
  s.dflt = p; p += kSMax * 3;
  s.E = p; p += kEStride * kEStride;
  s.s0 = p; p += Wmax;
  s.pos = reinterpret_cast<uint16_t*>(p); p += kSMax;
  s.ex = reinterpret_cast<uint8_t*>(p);
  return s;
}


// Full syndrome of the candidate `code` (2 bits per rank) is zero.
__device__ __forceinline__ bool syndrome_zero(const uint32_t* s0, const uint32_t* delta, int W, int Sp, uint32_t code) {
  uint32_t orr = 0;
  for (int w = 0; w < W; ++w) {
    uint32_t z = s0[w];
    for (int r = 0; r < Sp; ++r) {
      const uint32_t c = (code >> (2 * r)) & 3u;
      if (c) z ^= delta[((size_t)r * 3 + (c - 1)) * W + w];
    }
    orr |= z;
  }
  return orr == 0;
}

// Projection (see CodeDev::hf) of the candidate's syndrome.
__device__ __forceinline__ uint32_t projection(uint32_t f0, const uint32_t* dflt, int Sp, uint32_t code) {
  uint32_t z = f0;
  for (int r = 0; r < Sp; ++r) {
    const uint32_t c = (code >> (2 * r)) & 3u;
    if (c) z ^= dflt[r * 3 + (c - 1)];
  }
  return z;
}

constexpr int kPrepMaxW0 = 3;  // TEP weights the preparation can test in canonical order

// C(n, k) for 0 <= k <= 3 by integer arithmetic (0 when n < k): the lanes of
// the preparation's unranking hold different n, where a table read would be
// serialised.
__device__ __forceinline__ uint32_t binom_le3(int n, int k) {
  if (n < k) return 0u;
  const uint32_t m = (uint32_t)n;
  return k == 0 ? 1u : (k == 1 ? m : (k == 2 ? m * (m - 1) / 2u : m * (m - 1) * (m - 2) / 6u));
}

// Largest kernel dimension solve_frame ranks exhaustively (2^8 solutions).
constexpr int kSolveKerMax = 8;
// Resident CTAs per SM of the preparation with the elimination (syndromes of
// at most two words; the longer ones run 8 like the plain preparation).
constexpr int kPrepSolveBlocks = 10;

// 32 x 32 bit transpose across a warp: lane i holds row i on entry, lane j
// holds column j on return (bit i of it = bit j of row i).
__device__ __forceinline__ uint32_t warp_transpose_bits(uint32_t x) {
  const int lane = threadIdx.x & 31;
  constexpr uint32_t kMask[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int k = 16 >> s;
    const uint32_t m = kMask[s];
    const uint32_t y = __shfl_xor_sync(kFull, x, k);
    x = (lane & k) ? (((y >> k) & m) | (x & ~m)) : ((x & m) | ((y & m) << k));
  }
  return x;
}

// Column b of the slot system (see solve_frame): the syndrome delta of slot b
// (slot b & 1 of rank b >> 1) in the preparation's delta array.
__device__ __forceinline__ const uint32_t* slot_column(const PrepSmem& sm, int b, int W) {
  return sm.delta + ((b >> 1) * 3 + (b & 1)) * W;
}

// XOR of the slot columns over x (and s0 when with_s0) is zero on every
// syndrome word (lanes = words; x is the same in every lane).
__device__ __forceinline__ bool slot_sum_zero(const PrepSmem& sm, int W, uint32_t x, bool with_s0) {
  const int lane = threadIdx.x & 31;
  uint32_t acc = 0;
  if (lane < W) {
    acc = with_s0 ? sm.s0[lane] : 0u;
    for (uint32_t m = x; m; m &= m - 1u) acc ^= slot_column(sm, __ffs(m) - 1, W)[lane];
  }
  return !__any_sync(kFull, acc != 0u);
}

// The first hit among the solutions x0 + span(km[0..d)): every one is a
// valid TEP (only existing slots take part) and is ranked by its canonical
// position.
__device__ __forceinline__ void rank_solutions(const PrepSmem& sm, int Sp, uint32_t x0, const uint32_t (&km)[kSolveKerMax],
                                               int d, uint32_t& best_rank, uint32_t& best_code,
                                               unsigned long long& evaluated) {
  const int lane = threadIdx.x & 31;
  if (d == 0) {  // the usual case: one solution, ranked by every lane alike
    best_rank = tep_rank(sm.E, Sp, sm.ex, x0);
    best_code = x0;
    if (lane == 0) evaluated += 1;
    return;
  }
  uint32_t lr = 0xFFFFFFFFu, lc = 0;
  for (uint32_t c = (uint32_t)lane; c < (1u << d); c += 32) {
    uint32_t x = x0;
#pragma unroll
    for (int t = 0; t < kSolveKerMax; ++t)
      if ((c >> t) & 1u) x ^= km[t];
    const uint32_t rk = tep_rank(sm.E, Sp, sm.ex, x);
    if (rk < lr) { lr = rk; lc = x; }
  }
  if (lane == 0) evaluated += 1ull << d;
  const uint32_t br = __reduce_min_sync(kFull, lr);
  const unsigned who = __ballot_sync(kFull, lr == br);
  best_code = __shfl_sync(kFull, lc, __ffs(who) - 1);
  best_rank = br;
}

// GRAND_MEMBERSHIP_SOLVE: the frame's first codeword in canonical order by
// Gaussian elimination over GF(2) instead of a test per TEP. A valid TEP is a
// flip vector x over the existing slots (bit 2r: the first single-axis slot
// of rank r, bit 2r+1: the second; the diagonal is both), and H (y xor e) = 0
// reads XOR_{b in x} c_b = s0 with c_b the syndrome delta of slot b (zero for
// a flip beyond N): the codewords of the TEP space are the solutions x0 +
// ker of this system, and the first hit is the solution of smallest
// canonical rank.
//   Fast path: the system on one 32-bit word per column and for s0 -- the
// syndrome itself when it has one word (exact), else the 32-bit projections
// of the columns and of s0 -- transposed across the warp (lane r holds bit r
// of every column and of s0) and brought to reduced row echelon form, pivots
// in slot order (one ballot and one shuffle per slot). The projection is
// linear, so no projected solution means no solution. Otherwise the
// projected kernel vectors and x0 are checked on the full syndrome: when
// every kernel vector passes, the two kernels agree, and then x0 either
// passes (the solutions are x0 + that kernel) or no solution exists. A kernel vector that fails (the projection lost rank on
// the columns' span, about 2^(2S'-32) of frames) sends the frame to the
// exact path: the elimination on the full columns in shared memory.
// Returns 1 (best_rank and best_code set), 0 (no valid TEP gives a
// codeword: the frame abandons) or -1 (more than 2^kSolveKerMax solutions:
// the frame goes to the TEP search).
__device__ __forceinline__ int solve_frame(const PrepSmem& sm, int Sp, int W, uint32_t f0, uint32_t& best_rank,
                                           uint32_t& best_code, unsigned long long& evaluated) {
  const int lane = threadIdx.x & 31;
  const int nb = 2 * Sp;  // <= 24 < 31
  const bool on = lane < nb && ((sm.ex[lane >> 1] >> (lane & 1)) & 1u);
  uint32_t km[kSolveKerMax];
  {
    const bool one_word = W == 1;
    // lane b: the word of slot b, lane 31: that of s0; transposed so that
    // lane r holds bit r of every column (bit b: slot b, bit 31: s0)
    uint32_t row = on ? (one_word ? slot_column(sm, lane, 1)[0] : sm.dflt[(lane >> 1) * 3 + (lane & 1)])
                      : (lane == 31 ? (one_word ? sm.s0[0] : f0) : 0u);
    row = warp_transpose_bits(row);
    // reduced row echelon form over the existing slots, pivots in slot order
    const unsigned on_mask = __ballot_sync(kFull, on);
    bool used = false;  // this row holds a pivot
    int pc = 0;         // its slot
    uint32_t free_slots = 0;
    for (int b = 0; b < nb; ++b) {
      if (!((on_mask >> b) & 1u)) continue;  // an absent slot is no unknown
      const unsigned cand = __ballot_sync(kFull, !used && ((row >> b) & 1u));
      if (!cand) {
        free_slots |= 1u << b;
        continue;
      }
      const int pr = __ffs(cand) - 1;
      const uint32_t prow = __shfl_sync(kFull, row, pr);
      if (lane == pr) {
        used = true;
        pc = b;
      } else if ((row >> b) & 1u) {
        row ^= prow;
      }
    }
    // a row without pivot that still needs s0's bit: not even the word of s0 is reached
    if (__any_sync(kFull, !used && (row >> 31))) return 0;
    const uint32_t x0 = __reduce_or_sync(kFull, used && (row >> 31) ? 1u << pc : 0u);
    const int d = __popc(free_slots);
    bool kernels_agree = d <= kSolveKerMax;
    uint32_t fs = free_slots;
#pragma unroll
    for (int t = 0; t < kSolveKerMax; ++t) {
      km[t] = 0;
      if (t < d) {
        const int f = __ffs(fs) - 1;
        fs &= fs - 1u;
        km[t] = (1u << f) | __reduce_or_sync(kFull, used && ((row >> f) & 1u) ? 1u << pc : 0u);
        if (!one_word) kernels_agree = kernels_agree && slot_sum_zero(sm, W, km[t], false);
      }
    }
    if (kernels_agree) {
      if (!one_word && !slot_sum_zero(sm, W, x0, true)) return 0;
      rank_solutions(sm, Sp, x0, km, d, best_rank, best_code, evaluated);
      return 1;
    }
    if (one_word) return -1;  // exact already: the solution set is too large to rank
  }
  // exact path: lane b reduces column b in place (the delta slots), lane 31
  // reduces s0 (copied to the unused diagonal slot of rank 0)
  uint32_t* s0c = sm.delta + 2 * W;
  for (int w = lane; w < W; w += 32) s0c[w] = sm.s0[w];
  __syncwarp();
  const bool act = on || lane == 31;
  uint32_t* col = lane == 31 ? s0c : sm.delta + ((lane >> 1) * 3 + (lane & 1)) * W;
  uint32_t msk = on ? 1u << lane : 0u;
  bool pivot = false;
  for (int j = 0; j < nb; ++j) {
    int p = -1;
    if (lane == j && on) {
      for (int w = 0; w < W; ++w) {
        const uint32_t x = col[w];
        if (x) { p = 32 * w + __ffs(x) - 1; break; }
      }
      pivot = p >= 0;
    }
    p = __shfl_sync(kFull, p, j);
    if (p < 0) continue;  // slot j absent, or its column a sum of earlier ones
    const uint32_t pm = __shfl_sync(kFull, msk, j);
    const uint32_t* pc = slot_column(sm, j, W);
    if (act && lane > j && ((col[p >> 5] >> (p & 31)) & 1u)) {
      for (int w = 0; w < W; ++w) col[w] ^= pc[w];
      msk ^= pm;
    }
    __syncwarp();
  }
  uint32_t rest = 0;
  if (lane == 31)
    for (int w = 0; w < W; ++w) rest |= col[w];
  if (__shfl_sync(kFull, rest, 31) != 0u) return 0;  // s0 is not a sum of the slot columns
  const uint32_t x0 = __shfl_sync(kFull, msk, 31);
  uint32_t dep = __ballot_sync(kFull, on && !pivot);
  const int d = __popc(dep);
  if (d > kSolveKerMax) return -1;
#pragma unroll
  for (int t = 0; t < kSolveKerMax; ++t) {
    km[t] = 0;
    if (t < d) {
      km[t] = __shfl_sync(kFull, msk, __ffs(dep) - 1);
      dep &= dep - 1;
    }
  }
  rank_solutions(sm, Sp, x0, km, d, best_rank, best_code, evaluated);
  return 1;
}

// One frame of the preparation (one warp). Returns true when the frame needs
// the search stage; its hand-off record then went to a fresh slot of the
// batch's record array. WM: compile-time bound on the syndrome words
// (registers of the base syndrome).
template <int WM, bool kSolve>
__device__ __forceinline__ bool prep_frame(const PrepArgs& a, const int64_t f, const PrepSmem& sm,
                                           unsigned long long& evaluated) {
  const int lane = threadIdx.x & 31;
  {
    // --- frame parameters -------------------------------------------------
    int code_id = 0, M = a.M;
    int64_t sym_off = 0, cw_off = 0;
    bool bad_desc = false;
    if (a.desc) {
      const grand_frame_desc d = a.desc[f];
      code_id = d.code;
      M = d.M;
      sym_off = d.sym_offset;
      cw_off = d.cw_offset;
      bad_desc = code_id < 0 || code_id >= a.n_codes || !(M == 4 || M == 16 || M == 64 || M == 256 || M == 1024 || M == 4096) ||
                 sym_off < 0 || cw_off < 0;
      if (!bad_desc) {
        const int mm = (31 - __clz(M)) >> 1;
        const int NN = a.codes[code_id].N;
        const int LL = (NN + 2 * mm - 1) / (2 * mm);
        bad_desc = sym_off + LL > a.n_symbols || cw_off + (NN >> 5) > a.n_cw_words;
      }
    }
    if (bad_desc) {
      if (lane == 0) {
        a.queries[f] = 0;
        a.abandon[f] = 3;
      }
      return false;
    }
    const CodeDev code = a.codes[code_id];
    const int N = code.N, W = code.W, NW = N >> 5;
    const int m = (31 - __clz(M)) >> 1;
    const int side = 1 << m;
    const int L = (N + 2 * m - 1) / (2 * m);
    if (!a.desc) {
      sym_off = f * (int64_t)L;
      cw_off = f * (int64_t)NW;
    }
    const int Sp = a.S < L ? a.S : L;

    // --- Step 1: demodulation, hard word -----------------------------------
    if (lane < NW) sm.y[lane] = a.y_in && !a.symbols ? a.y_in[f * (int64_t)NW + lane] : 0u;
    __syncwarp();
    bool nonfinite = false;
    for (int i = lane; i < L; i += 32) {
      uint32_t key, info;
      if (a.symbols) {
        float2 sy = a.symbols[sym_off + i];
        const bool nf = !(isfinite(sy.x) && isfinite(sy.y));
        if (nf) sy = make_float2(0.0f, 0.0f);
        nonfinite |= nf;
        const AxisDemod I = demod_axis_q(sy.x, a.qc.q[m], side, a.lik);
        const AxisDemod Q = demod_axis_q(sy.y, a.qc.q[m], side, a.lik);
        key = (uint32_t)I.dq * (uint32_t)I.dq + (uint32_t)Q.dq * (uint32_t)Q.dq;
        info = pack_info(I.level, Q.level, make_nmask(I, Q, nf));
        // Gray label, MSB first, into the packed hard word
        const uint32_t label = ((uint32_t)gray_code(I.level) << m) | (uint32_t)gray_code(Q.level);
        const uint32_t rl = __brev(label) >> (32 - 2 * m);  // bit k = label bit (2m-1-k)
        const int p0 = 2 * m * i;
        const int wd = p0 >> 5, sh = p0 & 31;
        const uint32_t lo = rl << sh;
        const uint32_t hi = sh ? (rl >> (32 - sh)) : 0u;
        if (wd < NW) atomicOr(&sm.y[wd], lo);
        if (hi && wd + 1 < NW) atomicOr(&sm.y[wd + 1], hi);
      } else {
        const int64_t o = f * (int64_t)L + i;
        key = a.key[o];
        const uint32_t hidx = a.hard_idx[o];
        const uint32_t nm = a.nmask[o];
        nonfinite |= (nm & 128u) != 0;
        info = pack_info(hidx >> 8, hidx & 0xFF, nm);
      }
      sm.key[i] = key;
      sm.info[i] = info;
    }
    nonfinite = __any_sync(kFull, nonfinite);
    __syncwarp();
    if (nonfinite) {
      if (lane < NW) a.cw[cw_off + lane] = sm.y[lane];
      if (lane == 0) {
        a.queries[f] = 0;
        a.abandon[f] = 2;
      }
      __syncwarp();
      return false;
    }

    // --- base syndrome s0 = H y ---------------------------------------------
    uint32_t f0 = 0;  // projection of s0
    if (code.polar) {
      // H y = (y G_N) restricted to the frozen rows: superset sums of y by
      // butterfly stages (bits inside a word, then words across lanes)
      uint32_t x = lane < NW ? sm.y[lane] : 0u;
      x ^= (x >> 1) & 0x55555555u;
      x ^= (x >> 2) & 0x33333333u;
      x ^= (x >> 4) & 0x0F0F0F0Fu;
      x ^= (x >> 8) & 0x00FF00FFu;
      x ^= (x >> 16) & 0x0000FFFFu;
      for (int dw = 1; dw < 32; dw <<= 1) {
        const uint32_t o = __shfl_down_sync(kFull, x, dw);
        if (dw < NW && (lane & dw) == 0) x ^= o;
      }
#pragma unroll
      for (int w = 0; w < WM; ++w) {
        if (w < W) {
          const int r = 32 * w + lane;
          const int fr = r < code.R ? (int)__ldg(code.frozen + r) : 0;
          const uint32_t src = __shfl_sync(kFull, x, fr >> 5);
          const bool bit = r < code.R && ((src >> (fr & 31)) & 1u);
          const uint32_t word = __ballot_sync(kFull, bit);
          if (bit) f0 ^= __ldg(code.prow + r);
          if (lane == w) sm.s0[w] = word;
        }
      }
      for (int o = 16; o; o >>= 1) f0 ^= __shfl_xor_sync(kFull, f0, o);
    } else {
      // XOR of the H columns where y_j = 1
      uint32_t s0[WM];
#pragma unroll
      for (int w = 0; w < WM; ++w) s0[w] = 0;
      for (int j = lane; j < N; j += 32) {
        if ((sm.y[j >> 5] >> (j & 31)) & 1u) {
          const uint32_t* col = code.hcol + (size_t)j * W;
#pragma unroll
          for (int w = 0; w < WM; ++w)
            if (w < W) s0[w] ^= __ldg(col + w);
          f0 ^= __ldg(code.hf + j);
        }
      }
      for (int o = 16; o; o >>= 1) f0 ^= __shfl_xor_sync(kFull, f0, o);
#pragma unroll
      for (int w = 0; w < WM; ++w) {
        uint32_t v = s0[w];
        for (int o = 16; o; o >>= 1) v ^= __shfl_xor_sync(kFull, v, o);
        if (lane == w && w < W) sm.s0[w] = v;
      }
    }
    __syncwarp();

    // --- Steps 2-3: the S' least reliable symbols, by (key, index) ---------
    int my_sel = -1;
    if (L <= 32) {
      // one symbol per lane: S' rounds of the warp minimum of the keys; ties
      // go to the lowest index (the lowest lane of the ballot)
      uint32_t k_i = lane < L ? sm.key[lane] : 0xFFFFFFFFu;  // keys are < 2^31
      for (int r = 0; r < Sp; ++r) {
        const uint32_t kmin = __reduce_min_sync(kFull, k_i);
        const int win = __ffs(__ballot_sync(kFull, k_i == kmin)) - 1;
        if (lane == r) my_sel = win;
        if (lane == win) k_i = 0xFFFFFFFFu;
      }
    } else
    for (int r = 0; r < Sp; ++r) {
      uint32_t best_k = 0xFFFFFFFFu, best_i = 0xFFFFFFFFu;
      for (int i = lane; i < L; i += 32) {
        const uint32_t k = sm.key[i];
        if (k < best_k) { best_k = k; best_i = (uint32_t)i; }
      }
      const uint32_t kmin = __reduce_min_sync(kFull, best_k);
      const uint32_t imin = __reduce_min_sync(kFull, best_k == kmin ? best_i : 0xFFFFFFFFu);
      if (lane == (int)(imin & 31u)) sm.key[imin] = 0xFFFFFFFFu;  // keys are < 2^31
      if (lane == r) my_sel = (int)imin;
      __syncwarp();
    }

    // --- Step 4: alternatives and their syndrome deltas --------------------
    if (lane < Sp) {
      const int i = my_sel;
      const uint32_t info = sm.info[i];
      const int lI = info & 0xFF, lQ = (info >> 8) & 0xFF;
      const uint32_t nm = (info >> 16) & 0xFF;
      bool exI = nm & 1u, exQ = nm & 2u;
      const int dI = (nm & 8u) ? 1 : -1, dQ = (nm & 16u) ? 1 : -1;
      uint16_t pI = exI ? flip_pos_I(i, m, lI, dI, N) : kNoPos;
      uint16_t pQ = exQ ? flip_pos_Q(i, m, lQ, dQ, N) : kNoPos;
      if (a.nearer && (nm & 32u)) {
        // nearer axis first: the first single-axis slot takes the vertical
        // alternative (every later stage reads slots, not axes)
        const uint16_t tp = pI; pI = pQ; pQ = tp;
        const bool te = exI; exI = exQ; exQ = te;
      }
      sm.pos[2 * lane] = pI;
      sm.pos[2 * lane + 1] = pQ;
      sm.ex[lane] = (uint8_t)((exI ? 1 : 0) | (exQ ? 2 : 0) | (exI && exQ ? 4 : 0));
      uint32_t* dh = sm.delta + ((size_t)lane * 3 + 0) * W;
      for (int w = 0; w < W; ++w) {
        const uint32_t h = pI != kNoPos ? __ldg(code.hcol + (size_t)pI * W + w) : 0u;
        const uint32_t v = pQ != kNoPos ? __ldg(code.hcol + (size_t)pQ * W + w) : 0u;
        dh[w] = h;
        dh[W + w] = v;
        dh[2 * W + w] = h ^ v;
      }
      const uint32_t fh = pI != kNoPos ? __ldg(code.hf + pI) : 0u;
      const uint32_t fv = pQ != kNoPos ? __ldg(code.hf + pQ) : 0u;
      sm.dflt[3 * lane + 0] = fh;
      sm.dflt[3 * lane + 1] = fv;
      sm.dflt[3 * lane + 2] = fh ^ fv;
    }
    __syncwarp();
    esp_table_warp(sm.ex, Sp, sm.E);
    __syncwarp();
    const uint32_t total = esp_total(sm.E, Sp);

    // --- Step 5 (first part): small spaces completely, else light weights --
    uint32_t best_rank = 0xFFFFFFFFu, best_code = 0;
    int w_done = -1;
    {
      // every TEP of weight <= w0 in canonical order (all of them when S' <= w0)
      const int wmax = min(min(a.w0, kPrepMaxW0), Sp);
      for (int w = 0; w <= wmax && best_rank == 0xFFFFFFFFu; ++w) {
        const uint32_t nsets = binom16(Sp, w);
        for (uint32_t base = 0; base < nsets; base += 32) {
          const uint32_t cidx = base + lane;
          uint32_t hit_code = 0;
          bool hit = false;
          if (cidx < nsets) {
            // colex unranking of the altered rank set P[0] < ... < P[w-1]
            // (a single rank is its own index)
            int P[kPrepMaxW0] = {(int)cidx, 0, 0};
            if (w >= 2) {
              uint32_t rem = cidx;
              int p = Sp - 1;
#pragma unroll
              for (int jj = kPrepMaxW0; jj >= 1; --jj) {
                if (jj > w) continue;
                while (binom_le3(p, jj) > rem) --p;
                P[jj - 1] = p;
                rem -= binom_le3(p, jj);
                --p;
              }
            }
            // alternatives in base-3 order, least significant digit first
            int dig[kPrepMaxW0] = {0, 0, 0};
            uint32_t n_alpha = 1;
#pragma unroll
            for (int j = 0; j < kPrepMaxW0; ++j)
              if (j < w) n_alpha *= 3;
            for (uint32_t al = 0; al < n_alpha; ++al) {
              bool valid = true;
              uint32_t code_c = 0, z0 = f0;
#pragma unroll
              for (int j = 0; j < kPrepMaxW0; ++j) {
                if (j >= w) continue;
                if (!((sm.ex[P[j]] >> dig[j]) & 1u)) valid = false;
                code_c |= (uint32_t)(dig[j] + 1) << (2 * P[j]);
                z0 ^= sm.dflt[P[j] * 3 + dig[j]];
              }
              if (valid) {
                ++evaluated;
                if (z0 == 0 && syndrome_zero(sm.s0, sm.delta, W, Sp, code_c)) {
                  hit = true;
                  hit_code = code_c;
                  break;
                }
              }
#pragma unroll
              for (int j = 0; j < kPrepMaxW0; ++j) {  // odometer
                if (j >= w) break;
                if (++dig[j] < 3) break;
                dig[j] = 0;
              }
            }
          }
          const unsigned hb = __ballot_sync(kFull, hit);
          if (hb) {
            const int src = __ffs(hb) - 1;
            best_code = __shfl_sync(kFull, hit_code, src);
            best_rank = tep_rank(sm.E, Sp, sm.ex, best_code);
            break;
          }
        }
        w_done = w;
      }
    }
    // warp-wide best (only the full-space branch leaves lane-local values)
    {
      const uint32_t br = __reduce_min_sync(kFull, best_rank);
      const unsigned who = __ballot_sync(kFull, best_rank == br);
      best_code = __shfl_sync(kFull, best_code, __ffs(who) - 1);
      best_rank = br;
    }
    uint32_t done_count = 0;  // valid TEPs with at most w_done altered ranks
    for (int v = 0; v <= w_done; ++v) done_count += sm.E[Sp * kEStride + v];

    bool none = false;  // no valid TEP of the frame gives a codeword
    if constexpr (kSolve) {
      if (best_rank == 0xFFFFFFFFu && w_done < Sp && (uint64_t)done_count < (uint64_t)a.cap)
        none = solve_frame(sm, Sp, W, f0, best_rank, best_code, evaluated) == 0;
    }
    const bool resolved = best_rank != 0xFFFFFFFFu || none || w_done >= Sp || (uint64_t)done_count >= (uint64_t)a.cap;
    if (resolved) {
      uint32_t q;
      uint8_t ab;
      bool flip = false;
      if (best_rank != 0xFFFFFFFFu && (uint64_t)best_rank <= (uint64_t)a.cap) {
        q = best_rank;
        ab = 0;
        flip = true;
      } else {
        q = (uint32_t)((uint64_t)total < (uint64_t)a.cap ? total : a.cap);
        ab = 1;
      }
      if (flip && lane < Sp) {  // lane r flips the bits of rank r's alternative
        const uint32_t c = (best_code >> (2 * lane)) & 3u;
        if (c & 1u) { const uint16_t p = sm.pos[2 * lane]; if (p != kNoPos) atomicXor(&sm.y[p >> 5], 1u << (p & 31)); }
        if (c & 2u) { const uint16_t p = sm.pos[2 * lane + 1]; if (p != kNoPos) atomicXor(&sm.y[p >> 5], 1u << (p & 31)); }
      }
      __syncwarp();
      if (lane < NW) a.cw[cw_off + lane] = sm.y[lane];
      if (lane == 0) {
        a.queries[f] = q;
        a.abandon[f] = ab;
      }
    } else {
      // hand the frame to the search stage
      unsigned slot = 0;
      if (lane == 0) slot = atomicAdd(&a.scr->n_hard, 1u);
      slot = __shfl_sync(kFull, slot, 0);
      FrameRec* rec = a.recs + slot;
      if (lane < NW) a.cw[cw_off + lane] = sm.y[lane];
      if (lane < W) rec->s0[lane] = sm.s0[lane];
      if (lane < Sp) {
        rec->pos[lane][0] = sm.pos[2 * lane];
        rec->pos[lane][1] = sm.pos[2 * lane + 1];
        rec->ex[lane] = sm.ex[lane];
      }
      if (lane == 0) {
        a.queries[f] = done_count;  // what a frame cut at the deadline reports
        rec->f0 = f0;
        rec->frame = (uint32_t)f;
        rec->code = (uint16_t)code_id;
        rec->sp = (uint8_t)Sp;
        rec->w_done = (uint8_t)w_done;
        rec->cw_off = cw_off;
      }
      __syncwarp();
      return true;
    }
    __syncwarp();
  }
  return false;
}

// Resident CTAs per SM: 12 for syndromes of at most two words (the register
// bound then costs a few spilled words but the latency-bound preparation
// gains warps); 8 for the longer syndromes, whose per-lane arrays would spill
// heavily at 40 registers.
template <int WM, bool kSolve>
__global__ void __launch_bounds__(128, WM <= 2 ? (kSolve ? kPrepSolveBlocks : 12) : 8) k_prep(PrepArgs a) {
  extern __shared__ __align__(16) char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int warp_in_block = threadIdx.x >> 5;
  const int warps_per_block = blockDim.x >> 5;
  PrepSmem sm = prep_smem(smem_raw + warp_in_block * prep_warp_bytes(a.Lmax, a.Wmax), a.Lmax, a.Wmax);
  const int64_t gwarp = (int64_t)blockIdx.x * warps_per_block + warp_in_block;
  const int64_t nwarps = (int64_t)gridDim.x * warps_per_block;
  unsigned long long evaluated = 0;
  if (a.deadline > 0 && lane == 0) past_deadline(&a.scr->t0, a.deadline);  // start the call's clock
  for (int64_t f = gwarp; f < a.n_frames; f += nwarps) prep_frame<WM, kSolve>(a, f, sm, evaluated);
  // stats
  for (int o = 16; o; o >>= 1) evaluated += __shfl_xor_sync(kFull, evaluated, o);
  if (lane == 0 && evaluated) atomicAdd(&a.scr->evaluated, evaluated);
}

// ---------------------------------------------------------------------------
// Parallel search over the remaining TEP space (persistent CTAs)
// ---------------------------------------------------------------------------
constexpr int kRowsPerLane = 8;                 // A entries held per lane
constexpr int kTileRows = 32 * kRowsPerLane;    // A entries per tile
constexpr int kTileCols = 128;                  // B entries per tile
constexpr uint32_t kPadA = 0xA5A5A5A5u;
constexpr uint32_t kPadB = 0x5A5A5A5Au;

// 64 first-word compares: lane-held q[0..7] against 8 broadcast B words.
// One predicate-accumulating integer compare per pair; returns nonzero if any
// pair is equal.
__device__ __forceinline__ uint32_t any_equal_8x8(const uint32_t (&q)[kRowsPerLane], const uint4& z0,
                                                   const uint4& z1) {
  uint32_t f;
#define G_SETP(p, a, b) "setp.eq.u32 " p ", " a ", " b ";\n\t"
#define G_SETO(p, a, b) "setp.eq.or.u32 " p ", " a ", " b ", " p ";\n\t"
#define G_ROW_OR(b) G_SETO("p0", "%1", b) G_SETO("p1", "%2", b) G_SETO("p2", "%3", b) G_SETO("p3", "%4", b) \
  G_SETO("p0", "%5", b) G_SETO("p1", "%6", b) G_SETO("p2", "%7", b) G_SETO("p3", "%8", b)
  asm("{\n\t.reg .pred p0, p1, p2, p3;\n\t"
      G_SETP("p0", "%1", "%9") G_SETP("p1", "%2", "%9") G_SETP("p2", "%3", "%9") G_SETP("p3", "%4", "%9")
      G_SETO("p0", "%5", "%9") G_SETO("p1", "%6", "%9") G_SETO("p2", "%7", "%9") G_SETO("p3", "%8", "%9")
      G_ROW_OR("%10") G_ROW_OR("%11") G_ROW_OR("%12") G_ROW_OR("%13") G_ROW_OR("%14") G_ROW_OR("%15")
      G_ROW_OR("%16")
      "or.pred p0, p0, p1;\n\t"
      "or.pred p2, p2, p3;\n\t"
      "or.pred p0, p0, p2;\n\t"
      "selp.u32 %0, 1, 0, p0;\n\t}"
      : "=r"(f)
      : "r"(q[0]), "r"(q[1]), "r"(q[2]), "r"(q[3]), "r"(q[4]), "r"(q[5]), "r"(q[6]), "r"(q[7]), "r"(z0.x),
        "r"(z0.y), "r"(z0.z), "r"(z0.w), "r"(z1.x), "r"(z1.y), "r"(z1.z), "r"(z1.w));
#undef G_ROW_OR
#undef G_SETO
#undef G_SETP
  return f;
}

struct SearchSmem {
  uint32_t* Aq;      // [tabA + kTileRows] first word of s0 ^ D_A
  uint32_t* Bz;      // [tabB + kTileCols] first word of D_B
  uint16_t* Acode;   // [tabA]
  uint16_t* Bcode;   // [tabB]
  uint32_t* tiles;   // [max_tiles] (minw << 16) | (row block << 8) | column block
  uint32_t* delta;   // [kSMax][3][Wmax]
  uint32_t* dflt;    // [kSMax][3] projections of the deltas
  uint32_t* E;       // [kEStride^2]
  uint32_t* s0;      // [Wmax]
};

__host__ __device__ inline size_t search_smem_bytes(int tabA, int tabB, int max_tiles, int Wmax) {
  size_t b = 0;
  b += 4 * (size_t)(tabA + kTileRows);
  b += 4 * (size_t)(tabB + kTileCols);
  b += 2 * (size_t)tabA + 2 * (size_t)tabB;
  b = (b + 3) & ~(size_t)3;
  b += 4 * (size_t)max_tiles;
  b = (b + 15) & ~(size_t)15;
  b += 4 * (size_t)kSMax * 3 * Wmax + 4 * kSMax * 3 + 4 * kEStride * kEStride + 4 * (size_t)Wmax;
  return (b + 15) & ~(size_t)15;
}

__device__ inline SearchSmem search_smem(char* base, int tabA, int tabB, int max_tiles, int Wmax) {
  SearchSmem s;
  char* p = base;
  s.Aq = reinterpret_cast<uint32_t*>(p); p += 4 * (size_t)(tabA + kTileRows);
  s.Bz = reinterpret_cast<uint32_t*>(p); p += 4 * (size_t)(tabB + kTileCols);
  s.Acode = reinterpret_cast<uint16_t*>(p); p += 2 * (size_t)tabA;
  s.Bcode = reinterpret_cast<uint16_t*>(p); p += 2 * (size_t)tabB;
  p = base + (((size_t)(p - base) + 3) & ~(size_t)3);
  s.tiles = reinterpret_cast<uint32_t*>(p); p += 4 * (size_t)max_tiles;
  p = base + (((size_t)(p - base) + 15) & ~(size_t)15);
  s.delta = reinterpret_cast<uint32_t*>(p); p += 4 * (size_t)kSMax * 3 * Wmax;
  s.dflt = reinterpret_cast<uint32_t*>(p); p += 4 * kSMax * 3;
  s.E = reinterpret_cast<uint32_t*>(p); p += 4 * kEStride * kEStride;
  s.s0 = reinterpret_cast<uint32_t*>(p);
  return s;
}

// Build one side's table: every valid alternative assignment of the ranks
// [r0, r0 + n) (n <= 6) with the projection of its syndrome delta (XOR of the
// projected deltas, plus `seed`). Entries are grouped by the subset of
// altered ranks; subsets are ordered by size (the TEP weight), so the table
// is sorted by weight. A subset whose ranks have k_r existing alternatives
// contributes prod k_r entries (k_r is 1 or 3), decoded in base 3.
//   sub_off [2^n + 1]: first entry of each subset; cnt [n + 2]: entries per weight.
__device__ void build_side(const uint32_t* dflt, const uint8_t* ex, int r0, int n, uint32_t seed, uint32_t* outq,
                           uint16_t* outcode, unsigned* sub_off, unsigned* sub_size, unsigned* cnt) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int nsub = 1 << n;
  // subset sizes (prod k over its ranks), then each subset's offset in
  // (weight, subset) order: one thread per subset, no serial chain
  for (int sb = threadIdx.x; sb < nsub; sb += blockDim.x) {
    unsigned size = 1;
    for (int j = 0; j < n; ++j)
      if ((sb >> j) & 1) size *= (unsigned)__popc(ex[r0 + j] & 7u);
    sub_size[sb] = size;
  }
  __syncthreads();
  for (int sb = threadIdx.x; sb < nsub; sb += blockDim.x) {
    const int w = __popc(sb);
    unsigned off = 0;
    for (int t = 0; t < nsub; ++t) {
      const int wt = __popc(t);
      if (wt < w || (wt == w && t < sb)) off += sub_size[t];
    }
    sub_off[sb] = off;
  }
  for (int w = threadIdx.x; w <= kSideMax + 1; w += blockDim.x) {
    unsigned c = 0;
    for (int t = 0; t < nsub; ++t)
      if (__popc(t) == w) c += sub_size[t];
    cnt[w] = c;
  }
  __syncthreads();
  for (int sb = warp; sb < nsub; sb += nwarps) {
    const unsigned base = sub_off[sb];
    const unsigned size = sub_size[sb];
    for (unsigned c = lane; c < size; c += 32) {
      unsigned rem = c;
      uint32_t q = seed, code = 0;
      for (int j = 0; j < n; ++j) {
        if (!((sb >> j) & 1)) continue;
        const uint32_t exj = ex[r0 + j] & 7u;
        uint32_t alt;  // 1 h, 2 v, 3 diag
        if (exj == 7u) {
          alt = rem % 3u + 1u;
          rem /= 3u;
        } else {
          alt = (uint32_t)__ffs(exj);  // the single existing alternative
        }
        code |= alt << (2 * j);
        q ^= dflt[(r0 + j) * 3 + (alt - 1)];
      }
      outq[base + c] = q;
      outcode[base + c] = (uint16_t)code;
    }
  }
  __syncthreads();
}

// weight (number of altered ranks) of table entry i from the bucket counts
__device__ __forceinline__ int side_weight(const unsigned* cnt, unsigned i) {
  int w = 0;
  unsigned acc = cnt[0];
  while (i >= acc && w < kSideMax) acc += cnt[++w];
  return w;
}

// Full-syndrome check of a first-word match; records the canonical position.
__device__ __noinline__ void verify_hit(const SearchSmem& sm, const uint8_t* ex, int Sp, int W, int nAr, uint32_t acode,
                                        uint32_t bcode, unsigned long long* best, int* best_w) {
  const uint32_t c = acode | (bcode << (2 * nAr));
  uint32_t orr = 0;
  for (int w = 0; w < W; ++w) {
    uint32_t z = sm.s0[w];
    for (int r = 0; r < Sp; ++r) {
      const uint32_t d = (c >> (2 * r)) & 3u;
      if (d) z ^= sm.delta[((size_t)r * 3 + (d - 1)) * W + w];
    }
    orr |= z;
  }
  if (orr == 0) {
    const uint32_t rk = tep_rank(sm.E, Sp, ex, c);
    atomicMin(best, ((unsigned long long)rk << 32) | c);
    atomicMin(best_w, code_weight(c));
  }
}

// kMinBlocks sets the register budget (65536 / (256 * kMinBlocks) per thread).
template <int kMinBlocks>
__global__ void __launch_bounds__(256, kMinBlocks) k_search(SearchArgs a) {
  extern __shared__ __align__(16) char smem_raw[];
  __shared__ SearchSmem s_layout;  // pointers kept in shared memory, not registers
  if (threadIdx.x == 0) s_layout = search_smem(smem_raw, a.tabA, a.tabB, a.max_tiles, a.Wmax);
  __syncthreads();
  const SearchSmem& sm = s_layout;
  __shared__ unsigned s_frame;
  __shared__ int s_cut;
  __shared__ unsigned cntA[kSideMax + 2], cntB[kSideMax + 2];
  __shared__ unsigned subA[1 << kSideMax], subB[1 << kSideMax], sizeA[1 << kSideMax], sizeB[1 << kSideMax];
  __shared__ unsigned s_tile_cnt[2 * kSMax + 2];
  __shared__ unsigned s_n_tiles, s_tile_next;
  __shared__ unsigned long long s_best;  // (rank << 32) | code
  __shared__ int s_best_w;
  __shared__ FrameRec s_rec;
  __shared__ unsigned long long s_eval;
  __shared__ uint32_t s_qbuf[8][kTileRows];  // slow-path stash, one per warp (<= 8 warps)
  const int lane = threadIdx.x & 31;
  const int n_hard = (int)*(volatile unsigned*)&a.scr->n_hard;

  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned f = atomicAdd(&a.scr->next, 1u);
      s_frame = f;
      s_cut = a.deadline > 0 && f < (unsigned)n_hard && cut_at_deadline(a, a.recs + f, a.recs[f].frame);
    }
    __syncthreads();
    const unsigned fi = s_frame;
    if (fi >= (unsigned)n_hard) break;
    if (s_cut) {
      __syncthreads();  // everyone has read s_frame / s_cut before thread 0 rewrites them
      continue;
    }
    // --- load the frame ----------------------------------------------------
    if (threadIdx.x < sizeof(FrameRec) / 8)
      reinterpret_cast<unsigned long long*>(&s_rec)[threadIdx.x] =
          reinterpret_cast<const unsigned long long*>(a.recs + fi)[threadIdx.x];
    __syncthreads();
    const CodeDev code = a.codes[s_rec.code];
    const int W = code.W;
    const int Sp = s_rec.sp;
    const int split = (a.split > 0) ? min(Sp, max(Sp - kSideMax, min(a.split, kSideMax))) : (Sp >> 1);
    const int nAr = split, nBr = Sp - split;
    for (int t = threadIdx.x; t < Sp * 3 * W; t += blockDim.x) {
      const int r = t / (3 * W), rem = t % (3 * W), alt = rem / W, w = rem % W;
      const uint16_t pI = s_rec.pos[r][0], pQ = s_rec.pos[r][1];
      const uint32_t h = (alt != 1 && pI != kNoPos) ? __ldg(code.hcol + (size_t)pI * W + w) : 0u;
      const uint32_t v = (alt != 0 && pQ != kNoPos) ? __ldg(code.hcol + (size_t)pQ * W + w) : 0u;
      sm.delta[t] = h ^ v;  // alt 0: h, 1: v, 2: h ^ v
    }
    if (threadIdx.x < W) sm.s0[threadIdx.x] = s_rec.s0[threadIdx.x];
    if (threadIdx.x < 3 * Sp) {
      const int r = threadIdx.x / 3, alt = threadIdx.x % 3;
      const uint16_t pI = s_rec.pos[r][0], pQ = s_rec.pos[r][1];
      const uint32_t h = (alt != 1 && pI != kNoPos) ? __ldg(code.hf + pI) : 0u;
      const uint32_t v = (alt != 0 && pQ != kNoPos) ? __ldg(code.hf + pQ) : 0u;
      sm.dflt[threadIdx.x] = h ^ v;
    }
    if (threadIdx.x < 32) esp_table_warp(s_rec.ex, Sp, sm.E);
    if (threadIdx.x == 0) {
      s_best = ~0ull;
      s_best_w = 127;
      s_tile_next = 0;
      s_eval = 0;
    }
    __syncthreads();
    const uint32_t total = esp_total(sm.E, Sp);
    // heaviest weight class that still holds a position <= cap
    int w_cap = Sp;
    {
      uint64_t acc = 0;
      for (int v = 0; v <= Sp; ++v) {
        acc += sm.E[Sp * kEStride + v];
        if (acc >= (uint64_t)a.cap) { w_cap = v; break; }
      }
    }
    unsigned nA = 1, nB = 1;
    for (int r = 0; r < nAr; ++r) nA *= 1u + __popc(s_rec.ex[r] & 7u);
    for (int r = nAr; r < Sp; ++r) nB *= 1u + __popc(s_rec.ex[r] & 7u);
    build_side(sm.dflt, s_rec.ex, 0, nAr, s_rec.f0, sm.Aq, sm.Acode, subA, sizeA, cntA);
    build_side(sm.dflt, s_rec.ex, nAr, nBr, 0u, sm.Bz, sm.Bcode, subB, sizeB, cntB);
    // pads (never a real entry): rows to a full tile, columns to a full tile
    const unsigned nRB = (nA + kTileRows - 1) / kTileRows, nCB = (nB + kTileCols - 1) / kTileCols;
    for (unsigned i = nA + threadIdx.x; i < nRB * kTileRows; i += blockDim.x) sm.Aq[i] = kPadA;
    for (unsigned i = nB + threadIdx.x; i < nCB * kTileCols; i += blockDim.x) sm.Bz[i] = kPadB;
    // --- tile list ordered by the lightest TEP of each tile ----------------
    if (threadIdx.x < 2 * kSMax + 2) s_tile_cnt[threadIdx.x] = 0;
    __syncthreads();
    const int w_done = s_rec.w_done;
    const unsigned n_tiles_all = nRB * nCB;
    for (int pass = 0; pass < 2; ++pass) {
      for (unsigned t = threadIdx.x; t < n_tiles_all; t += blockDim.x) {
        const unsigned rb = t / nCB, cb = t % nCB;
        const int minw = side_weight(cntA, rb * kTileRows) + side_weight(cntB, cb * kTileCols);
        const int maxw = side_weight(cntA, min(nA, (rb + 1) * kTileRows) - 1) +
                         side_weight(cntB, min(nB, (cb + 1) * kTileCols) - 1);
        if (maxw <= w_done || minw > w_cap) continue;
        if (pass == 0) {
          atomicAdd(&s_tile_cnt[minw], 1u);
        } else {
          const unsigned slot = atomicAdd(&s_tile_cnt[minw], 1u);
          sm.tiles[slot] = ((unsigned)minw << 16) | (rb << 8) | cb;
        }
      }
      __syncthreads();
      if (pass == 0) {
        if (threadIdx.x < 32) {  // exclusive scan of the per-weight tile counts
          const unsigned c = threadIdx.x < 2 * kSMax + 2 ? s_tile_cnt[threadIdx.x] : 0u;
          unsigned incl = c;
          for (int o = 1; o < 32; o <<= 1) {
            const unsigned t = __shfl_up_sync(kFull, incl, o);
            if ((int)threadIdx.x >= o) incl += t;
          }
          if (threadIdx.x < 2 * kSMax + 2) s_tile_cnt[threadIdx.x] = incl - c;
          if (threadIdx.x == 31) s_n_tiles = incl;
        }
        __syncthreads();
      }
    }
    const unsigned n_tiles = s_n_tiles;

    // --- the tile loop (one warp per tile) ---------------------------------
    unsigned long long my_eval = 0;
    for (;;) {
      unsigned ti = 0;
      if (lane == 0) ti = atomicAdd(&s_tile_next, 1u);
      ti = __shfl_sync(kFull, ti, 0);
      if (ti >= n_tiles) break;
      const unsigned tile = sm.tiles[ti];
      const unsigned rb = (tile >> 8) & 0xFF, cb = tile & 0xFF;
      const unsigned row0 = rb * kTileRows, col0 = cb * kTileCols;
      if ((int)(tile >> 16) > *(volatile int*)&s_best_w) break;  // tiles are sorted by minw
      uint32_t q[kRowsPerLane];
#pragma unroll
      for (int t = 0; t < kRowsPerLane; ++t) q[t] = sm.Aq[row0 + lane + 32 * t];
      const uint4* zb = reinterpret_cast<const uint4*>(sm.Bz + col0);
      uint32_t any = 0;
#pragma unroll 2
      for (int g = 0; g < kTileCols / 8; ++g) any |= any_equal_8x8(q, zb[2 * g], zb[2 * g + 1]);
      if (lane == 0) my_eval += (unsigned long long)(min(nA - row0, (unsigned)kTileRows)) *
                                (unsigned long long)(min(nB - col0, (unsigned)kTileCols));
      if (__any_sync(kFull, any)) {
        // rare: locate the equal projections and verify every syndrome word
        uint32_t* qs = s_qbuf[threadIdx.x >> 5];
#pragma unroll
        for (int t = 0; t < kRowsPerLane; ++t) qs[lane + 32 * t] = q[t];
        __syncwarp();
        if (any) {
          for (int t = 0; t < kRowsPerLane; ++t) {
            const unsigned row = row0 + lane + 32 * t;
            const uint32_t qt = qs[lane + 32 * t];
            if (row >= nA) continue;
            for (int j = 0; j < kTileCols; ++j)
              if (sm.Bz[col0 + j] == qt && col0 + j < nB)
                verify_hit(sm, s_rec.ex, Sp, W, nAr, sm.Acode[row], sm.Bcode[col0 + j], &s_best, &s_best_w);
          }
        }
        __syncwarp();
      }
    }
    if (lane == 0 && my_eval) atomicAdd(&s_eval, my_eval);
    __syncthreads();
    // --- result ------------------------------------------------------------
    if (threadIdx.x == 0) {
      const unsigned f = s_rec.frame;
      const unsigned long long best = s_best;
      const uint32_t rk = (uint32_t)(best >> 32), c = (uint32_t)best;
      if (best != ~0ull && (uint64_t)rk <= (uint64_t)a.cap) {
        uint32_t* cw = a.cw + s_rec.cw_off;
        for (int r = 0; r < Sp; ++r) {
          const uint32_t d = (c >> (2 * r)) & 3u;
          if (d & 1u) { const uint16_t p = s_rec.pos[r][0]; if (p != kNoPos) cw[p >> 5] ^= 1u << (p & 31); }
          if (d & 2u) { const uint16_t p = s_rec.pos[r][1]; if (p != kNoPos) cw[p >> 5] ^= 1u << (p & 31); }
        }
        a.queries[f] = rk;
        a.abandon[f] = 0;
      } else {
        a.queries[f] = (uint32_t)((uint64_t)total < (uint64_t)a.cap ? total : (uint64_t)a.cap);
        a.abandon[f] = 1;
      }
      uint32_t done = 0;  // valid TEPs the preparation already tested
      for (int v = 0; v <= w_done; ++v) done += sm.E[Sp * kEStride + v];
      atomicAdd(&a.scr->evaluated, s_eval);
      atomicAdd(&a.scr->search_useful, (unsigned long long)(a.queries[f] - done));
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Meet-in-the-middle split of the TEP space: A x B sides. The warp search
// (k_search_warp, every S' <= 12) and the hash join (k_search_hash) own one
// frame per warp, with its tables in the warp's own slice of shared memory and
// a set-up that runs on warp shuffles and ballots, so no block-wide barrier
// exists and the set-up of one warp overlaps the compares of the others.
//
// The warp search compares a B entry with 32 A entries at once on a 20-bit
// projection of the syndrome (false matches 2^-20; candidates are verified on
// every syndrome word). Each A group of 32 entries keeps, per 5-bit slice k
// of the projection (bit-planes 5k..5k+4), the 32 words
//     T[k][v] = OR_{j<5} (plane_{5k+j} XOR (bit j of v ? ~0 : 0)),
// so a lane with B projection z gets
//     acc = T[0][z & 31] | T[1][(z >> 5) & 31] | T[2][(z >> 10) & 31],
// zero exactly at the A entries equal to z on 15 bits: three shared-memory
// reads and one logic op test 32 TEPs (the fourth slice only after a match).
// The 32 words of a slice sit in 32 distinct banks, so any pattern of lane
// reads is conflict-free; the kernel is bound by shared-memory bandwidth
// (0.375 B per TEP).
// ---------------------------------------------------------------------------
constexpr int kWarpSideMax = 5;                      // hash join: the small-table variant (S' <= 10)
constexpr int kPlanes = 20;                          // projection bits compared per TEP
constexpr int kGroupUnroll = 8;                      // groups per candidate check
constexpr int kQuarter = 4;                          // groups per fourth-slice decision
constexpr int kLutBits = 5;                          // projection bits per table (32 words)
constexpr int kLutSets = kPlanes / kLutBits;         // tables per group (the last one: second level)
constexpr int kLutWords = 1 << kLutBits;
constexpr int kLutStride = kLutSets * kLutWords + 1; // words per group (odd: conflict-free per-lane stores)

// Table sizes of one side for the kSide variant.
template <int kSide>
struct WarpDims {
  static constexpr int kTab = 1 << (2 * kSide);  // entries per side
  static constexpr int kGroups = kTab / 32;      // A groups of 32 entries
  static constexpr int kSub = 1 << kSide;        // rank subsets per side
  static constexpr int kRanks = 2 * kSide;       // S' bound
};

// The hash join's per-warp slice (sides of kSide ranks, weight-sorted tables).
struct WarpSlice {
  uint32_t* Bz;      // [kTab] projection of D_A, then of D_B, weight-sorted (kSide = 5 only)
  uint32_t* delta;   // [kRanks][3][Wmax] full syndrome deltas
  uint32_t* dflt;    // [kRanks][3] projections of the deltas
  uint32_t* E;       // [kEStride^2]
  uint32_t* s0;      // [Wmax]
  uint32_t* startA;  // [kSub + 1] first entry of the k-th subset of A in table order
  uint32_t* startB;  // [kSub + 1]
  uint32_t* cumA;    // [8] A entries of weight <= v
  uint32_t* cumB;    // [8]
  uint8_t* ordA;     // [kSub] subset at table position k
  uint8_t* ordB;     // [kSub]
  uint8_t* invA;     // [kSub] table position of subset sb
  uint8_t* invB;     // [kSub]
  uint8_t* ex;       // [16]
  uint16_t* pos;     // [kRanks][2]
};

template <int kSide>
__host__ __device__ inline size_t warp_slice_bytes(int Wmax) {
  using D = WarpDims<kSide>;
  const size_t bz = kSide == kWarpSideMax ? D::kTab : 0;
  size_t words = bz + 3 * D::kRanks * (size_t)Wmax + 3 * D::kRanks +
                 kEStride * kEStride + Wmax + 2 * (D::kSub + 1) + 8 + 8 + D::kSub + 4 + D::kRanks;
  return (words * 4 + 15) & ~(size_t)15;
}

template <int kSide>
__device__ inline WarpSlice warp_slice(char* base, int Wmax) {
  using D = WarpDims<kSide>;
  WarpSlice w;
  uint32_t* p = reinterpret_cast<uint32_t*>(base);
  w.Bz = p; p += kSide == kWarpSideMax ? D::kTab : 0;
  w.delta = p; p += 3 * D::kRanks * Wmax;
  w.dflt = p; p += 3 * D::kRanks;
  w.E = p; p += kEStride * kEStride;
  w.s0 = p; p += Wmax;
  w.startA = p; p += D::kSub + 1;
  w.startB = p; p += D::kSub + 1;
  w.cumA = p; p += 8;
  w.cumB = p; p += 8;
  w.ordA = reinterpret_cast<uint8_t*>(p); p += D::kSub / 4;
  w.ordB = reinterpret_cast<uint8_t*>(p); p += D::kSub / 4;
  w.invA = reinterpret_cast<uint8_t*>(p); p += D::kSub / 4;
  w.invB = reinterpret_cast<uint8_t*>(p); p += D::kSub / 4;
  w.ex = reinterpret_cast<uint8_t*>(p); p += 4;
  w.pos = reinterpret_cast<uint16_t*>(p);
  return w;
}

// Layout of one side's table, computed by one warp. Subsets of the side's n
// ranks are laid out by (size, colex order), i.e. by TEP weight; the k-th
// subset's entries start at start[k]; cum[v] = entries of weight <= v.
// Returns the number of entries.
__device__ inline unsigned warp_side_layout(const WarpSlice& sl, int r0, int n, uint32_t* start, uint8_t* ord,
                                            uint8_t* inv, uint32_t* cum) {
  const int lane = threadIdx.x & 31;
  const int nsub = 1 << n;  // <= 64: two subsets per lane
  for (int sb = lane; sb < nsub; sb += 32) {
    int w = 0, colex = 0;
    for (int j = 0; j < n; ++j)
      if ((sb >> j) & 1) {
        ++w;
        colex += (int)binom16(j, w);
      }
    int before = 0;
    for (int v = 0; v < w; ++v) before += (int)binom16(n, v);
    const int posk = before + colex;
    ord[posk] = (uint8_t)sb;
    inv[sb] = (uint8_t)posk;
  }
  __syncwarp();
  // entries of the subset at table position k, then an exclusive scan
  uint32_t kk = 0;  // 2 bits per rank of the side: its number of alternatives (1 or 3; 0 = none)
  for (int j = 0; j < n; ++j) kk |= (uint32_t)__popc(sl.ex[r0 + j] & 7u) << (2 * j);
  unsigned carry = 0;
  for (int k0 = 0; k0 < nsub; k0 += 32) {
    const int k = k0 + lane;
    unsigned size_k = 0;
    if (k < nsub) {
      const int sb = ord[k];
      size_k = 1;
      for (int j = 0; j < n; ++j)
        if ((sb >> j) & 1) size_k *= (kk >> (2 * j)) & 3u;
    }
    unsigned incl = size_k;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned t = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += t;
    }
    if (k < nsub) start[k] = carry + incl - size_k;
    carry += __shfl_sync(kFull, incl, 31);
  }
  const unsigned total = carry;
  if (lane == 0) start[nsub] = total;
  __syncwarp();
  // cumulative count per weight: subsets of weight <= v end at position
  // sum_{u<=v} C(n,u) (C(n,u+1) = C(n,u) (n-u) / (u+1))
  if (lane <= n) {
    int endk = 0, c = 1;
    for (int u = 0; u <= lane; ++u) {
      endk += c;
      c = c * (n - u) / (u + 1);
    }
    cum[lane] = start[endk];
  }
  for (int v = n + 1 + lane; v < 8; v += 32) cum[v] = total;
  __syncwarp();
  return total;
}

// Table entry e of a side: projection (seed ^ XOR of projected deltas) and the
// alternative code (2 bits per rank of the side). Within a subset's block the
// entries follow the doubling order of warp_fill_side: the highest rank's
// alternative is the least significant base-k digit.
__device__ __forceinline__ void warp_side_entry(const WarpSlice& sl, int r0, int n, const uint32_t* start,
                                                const uint8_t* ord, uint32_t seed, unsigned e, uint32_t& q,
                                                uint32_t& code) {
  const int nsub = 1 << n;
  int lo = 0, hi = nsub - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (start[mid] <= e) lo = mid; else hi = mid - 1;
  }
  const int sb = ord[lo];
  unsigned rem = e - start[lo];
  q = seed;
  code = 0;
  for (int j = n - 1; j >= 0; --j) {
    if (!((sb >> j) & 1)) continue;
    const uint32_t exj = sl.ex[r0 + j] & 7u;
    uint32_t alt;
    if (exj == 7u) {
      alt = rem % 3u + 1u;
      rem /= 3u;
    } else {
      alt = (uint32_t)__ffs(exj);  // the single existing alternative
    }
    code |= alt << (2 * j);
    q ^= sl.dflt[(r0 + j) * 3 + (alt - 1)];
  }
}

// Fill one side's weight-sorted table by doubling: the block of subset S is
// the block of S minus its highest rank j, each entry XORed with one of j's
// projected deltas (entry c = parent entry c / k_j, alternative c % k_j).
// Blocks are visited in table order, so parents (one rank lighter) are ready.
// Lane k first gathers the description of the k-th block (offsets, parent,
// neighbour mask, the three projected deltas of j); the walk over the blocks
// then reads it by shuffles instead of chains of shared-memory loads.
__device__ inline void warp_fill_side(const WarpSlice& sl, int r0, int n, const uint32_t* start, const uint8_t* ord,
                                      const uint8_t* inv, uint32_t seed, uint32_t* out) {
  const int lane = threadIdx.x & 31;
  const int nsub = 1 << n;
  uint32_t m_info = 0, m_off = 0, m_d0 = 0, m_d1 = 0, m_d2 = 0;
  if (lane < nsub) {
    const int sb = ord[lane];
    const unsigned base = start[lane], size = start[lane + 1] - base;
    uint32_t exj = 0;
    unsigned pbase = 0;
    if (sb) {
      const int j = 31 - __clz(sb);
      pbase = start[inv[sb & ~(1 << j)]];
      exj = sl.ex[r0 + j] & 7u;
      const uint32_t* dj = sl.dflt + (r0 + j) * 3;
      m_d0 = dj[0];
      m_d1 = dj[1];
      m_d2 = dj[2];
      if (exj != 7u && exj) m_d0 = dj[__ffs(exj) - 1];  // the single existing alternative
    }
    m_info = size | ((uint32_t)__popc(sb) << 16) | (exj << 24);
    m_off = base | (pbase << 16);
  }
  if (lane == 0) out[0] = seed;  // the empty subset is first
  __syncwarp();
  int prev_w = 0;
  for (int k = 1; k < nsub; ++k) {
    const uint32_t info = __shfl_sync(kFull, m_info, k);
    const uint32_t off = __shfl_sync(kFull, m_off, k);
    const uint32_t d0 = __shfl_sync(kFull, m_d0, k);
    const uint32_t d1 = __shfl_sync(kFull, m_d1, k);
    const uint32_t d2 = __shfl_sync(kFull, m_d2, k);
    const int w = (info >> 16) & 0xFF;
    if (w != prev_w) {  // the parents of this weight are complete
      __syncwarp();
      prev_w = w;
    }
    const unsigned size = info & 0xFFFFu;
    if (size == 0) continue;
    const unsigned base = off & 0xFFFFu, pbase = off >> 16;
    if ((info >> 24) == 7u) {
      for (unsigned c = lane; c < size; c += 32) {
        const unsigned pi = c / 3u, ai = c - 3u * pi;
        out[base + c] = out[pbase + pi] ^ (ai == 0 ? d0 : (ai == 1 ? d1 : d2));
      }
    } else {
      for (unsigned c = lane; c < size; c += 32) out[base + c] = out[pbase + c] ^ d0;
    }
  }
  __syncwarp();
}

// The compare of one lane's B entry z against the A groups' tables:
// block(g0) fixes the first group of a block of kGroupUnroll groups;
// first<U>() (slices 0..2) and second<U>() (slice 3) then read group g0 + U
// with immediate offsets; first_at / second_at read any group (candidates).
//
// 32-bit shared-memory read at a shared-window address plus an immediate.
template <int kOff>
__device__ __forceinline__ uint32_t lds_imm(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1+%2];" : "=r"(v) : "r"(addr), "n"(kOff) : "memory");
  return v;
}

struct LutCmp {
  uint32_t t[kLutSets];  // shared-window address of the word of slice k of z in group 0
  uint32_t b[kLutSets];  // the same in group g0 of the current block
  __device__ __forceinline__ void load(const uint32_t* tab, uint32_t z) {
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(tab);
#pragma unroll
    for (int k = 0; k < kLutSets; ++k)
      t[k] = base + 4u * (kLutWords * k + ((z >> (kLutBits * k)) & (kLutWords - 1u)));
  }
  __device__ __forceinline__ void block(int g) {
#pragma unroll
    for (int k = 0; k < kLutSets; ++k) b[k] = t[k] + 4u * kLutStride * (uint32_t)g;
  }
  template <int U>
  __device__ __forceinline__ uint32_t first() const {
    constexpr int o = 4 * kLutStride * U;
    return lds_imm<o>(b[0]) | lds_imm<o>(b[1]) | lds_imm<o>(b[2]);
  }
  template <int U>
  __device__ __forceinline__ uint32_t second() const {
    return lds_imm<4 * kLutStride * U>(b[3]);
  }
  __device__ __forceinline__ uint32_t first_at(int g) const {
    const uint32_t o = 4u * kLutStride * (uint32_t)g;
    return lds_imm<0>(t[0] + o) | lds_imm<0>(t[1] + o) | lds_imm<0>(t[2] + o);
  }
  __device__ __forceinline__ uint32_t second_at(int g) const {
    return lds_imm<0>(t[3] + 4u * kLutStride * (uint32_t)g);
  }
};

// f(std::integral_constant<int, U>) for U = I .. N-1, unrolled at compile time.
template <int I, int N, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    static_for<I + 1, N>(f);
  }
}

// ---------------------------------------------------------------------------
// Warp search on flip-bit tables (every S' <= 12).
//
// A TEP restricted to one side is a vector x of 2n flip bits: bit 2r selects
// the I-slot alternative of the side's r-th rank, bit 2r+1 the Q-slot one, and
// both together the diagonal one (which exists exactly when both single-axis
// ones do). x is then also the TEP's code in the canonical 2-bits-per-rank
// form, and its syndrome projection is linear in x:
//     proj(x) = seed ^ XOR_{b in x} H_b.
// A side's vectors are cut as x = 32 g + i: i (bits 0..4) within a group, g
// (the higher bits) the group. Within group g the projections are C_g ^ P_i,
// with P_i = XOR_{b < 5, b in i} H_b the same for every group, so
//   * the A side (at most 5 ranks: 32 groups) keeps one row of slice tables
//     per group, derived from the 20 bit-planes of P (one set of warp ballots)
//     inverted at the bits of C_g -- no per-group transposes and no table of
//     projections;
//   * the B side (at most 7 ranks: up to 512 groups) needs no table at all: the
//     lane holding within-group vector i of group h compares C'_h ^ P'_i.
// Vectors naming an alternative that does not exist are masked (existence is
// a per-bit property, within part and group part separately). Groups of both
// sides are visited in order of their lightest TEP weight (A groups as table
// rows, B groups two per chunk, one entry per lane each), which keeps the
// weight cut-offs of the canonical order.
// ---------------------------------------------------------------------------
constexpr int kFlipSideA = 5;   // ranks of the A side (table rows: 2^(2*5-5) = 32 groups)
constexpr int kFlipSideB = 7;   // ranks of the B side at most (S' <= 12)

// B groups of the largest split a launch handles (the size of its B-group list).
__host__ __device__ inline int flip_b_groups(int sp_max) {
  const int nA = sp_max >> 1 < kFlipSideA ? sp_max >> 1 : kFlipSideA;
  const int bits = 2 * (sp_max - nA) - 5;
  return bits > 0 ? 1 << bits : 1;
}

struct FlipSlice {
  uint32_t* lut;    // [32][kLutStride] tables of the A groups in visiting order
  uint2* bgrp;      // [flip_b_groups] B groups in visiting order: (C'_h, h << 16 | heaviest << 8 | lightest)
  uint32_t* dflt;   // [kSMax][3] projections of the deltas
  uint32_t* d0;     // [kSMax][3] first syndrome word of the deltas
  uint32_t* E;      // [kEStride^2]
  uint32_t* s0;     // [Wmax]
  uint8_t* ordA;    // [32] A group at visiting position t
  uint8_t* ex;      // [16]
  uint16_t* pos;    // [kSMax][2]
};

// (Of the full syndrome deltas only the first word is kept: the rare
// candidates of the projection compare are rejected on it, and a candidate
// that passes reads the code's columns for the other words.)
__host__ __device__ inline size_t flip_slice_bytes(int Wmax, int sp_max) {
  const size_t words = 32 * kLutStride + 2 * (size_t)flip_b_groups(sp_max) + 3 * kSMax + 3 * kSMax +
                       kEStride * kEStride + Wmax + 8 + 4 + kSMax;
  return (words * 4 + 15) & ~(size_t)15;
}

__device__ inline FlipSlice flip_slice(char* base, int Wmax, int sp_max) {
  FlipSlice w;
  uint32_t* p = reinterpret_cast<uint32_t*>(base);
  w.lut = p; p += 32 * kLutStride;  // even: the B-group list is 8-byte aligned
  w.bgrp = reinterpret_cast<uint2*>(p); p += 2 * flip_b_groups(sp_max);
  w.dflt = p; p += 3 * kSMax;
  w.d0 = p; p += 3 * kSMax;
  w.E = p; p += kEStride * kEStride;
  w.s0 = p; p += Wmax;
  w.ordA = reinterpret_cast<uint8_t*>(p); p += 8;
  w.ex = reinterpret_cast<uint8_t*>(p); p += 4;
  w.pos = reinterpret_cast<uint16_t*>(p);
  return w;
}

// Lightest TEP weight of the flip-bit group g (group bits start at bit 5).
__device__ __forceinline__ int group_min_weight(uint32_t g) { return code_weight(g << 5); }

// XOR of h[b] over the bits b of x (b < N).
template <int N>
__device__ __forceinline__ uint32_t xor_bits(uint32_t x, const uint32_t (&h)[N]) {
  uint32_t r = 0;
#pragma unroll
  for (int b = 0; b < N; ++b) r ^= ((x >> b) & 1u) ? h[b] : 0u;
  return r;
}

// Visiting order of the A side's valid groups (group existence bits ehi, at
// most 32 groups): by lightest weight, then by index. Writes ord[0..n) and
// returns n; lane w (w <= 5) gets in *cum the number of groups of lightest
// weight <= w.
__device__ __forceinline__ int order_groups_a(uint32_t ehi, uint8_t* ord, uint32_t* cum, bool write = true) {
  const int lane = threadIdx.x & 31;
  const bool valid = ((uint32_t)lane & ~ehi) == 0u;
  const int mw = group_min_weight((uint32_t)lane);
  int n = 0, my = 0;
  uint32_t c = 0;
  for (int w = 0; w <= 3; ++w) {
    const unsigned m = __ballot_sync(kFull, valid && mw == w);
    if (valid && mw == w) my = n + __popc(m & ((1u << lane) - 1u));
    n += __popc(m);
    if (lane == w) c = (uint32_t)n;
  }
  if (lane > 3) c = (uint32_t)n;
  if (valid && write) ord[my] = (uint8_t)lane;
  *cum = c;
  __syncwarp();
  return n;
}

// Visiting order of the B side's valid groups (group bits nbits <= 9,
// existence bits ehi): by lightest weight, then by index; each entry carries
// the group constant C'_h and the group's lightest and heaviest TEP weights
// (ewithin: the existence bits of the within-group part). Returns the count.
__device__ inline int order_groups_b(uint32_t ehi, int nbits, uint32_t ewithin, const uint32_t (&hhi)[9],
                                     uint2* out) {
  const int lane = threadIdx.x & 31;
  const int ng = 1 << nbits;
  int n = 0;
  for (int w = 0; w <= kFlipSideB - 2; ++w) {
    for (int h0 = 0; h0 < ng; h0 += 32) {
      const uint32_t h = (uint32_t)(h0 + lane);
      const bool take = (int)h < ng && (h & ~ehi) == 0u && group_min_weight(h) == w;
      const unsigned m = __ballot_sync(kFull, take);
      if (take) {
        const int at = n + __popc(m & ((1u << lane) - 1u));
        const uint32_t heavy = (uint32_t)code_weight((h << 5) | ewithin);
        out[at] = make_uint2(xor_bits<9>(h, hhi), (h << 16) | (heavy << 8) | (uint32_t)w);
      }
      n += __popc(m);
    }
  }
  __syncwarp();
  return n;
}

// State of the warp pair that shares one frame (pair mode: a CTA of two
// warps, one slice of shared memory).
struct PairShared {
  unsigned fi;            // the frame the pair works on
  int flag;               // a per-frame decision of warp 0 (cursor valid, deadline cut)
  int best_w;             // lightest hit weight found by either warp
  int nGB;                // valid B groups (ordered by warp 1)
  uint32_t best_rank[2];  // each warp's first hit
  uint32_t best_code[2];
};

// Block-wide barrier in pair mode, warp barrier otherwise.
template <bool kPair>
__device__ __forceinline__ void pair_sync() {
  if constexpr (kPair) __syncthreads(); else __syncwarp();
}

// The search of one frame. kPair: two warps of a CTA share the frame and its
// tables -- warp 0 writes the per-frame arrays and the A rows while warp 1
// orders the B groups, and the chunks then alternate between the warps (the
// lightest hit weight is shared, so either warp's hit tightens the other's
// cut-off); warp 0 reports the lower of the two first hits. Every barrier is
// reached by both warps.
template <bool kResume, bool kPair>
__device__ __forceinline__ void search_frame_flip(const SearchArgs& a, unsigned fi, const FrameRec* rec,
                                                  const FlipSlice& sl, unsigned long long& my_eval,
                                                  unsigned long long& my_useful, PairShared* ps) {
  const int lane = threadIdx.x & 31;
  const int wid = kPair ? (int)((threadIdx.x >> 5) & 1) : 0;
  const int Sp = rec->sp;
  const int w_done = rec->w_done;
  const CodeDev code = a.codes[rec->code];
  const int W = code.W;
  const uint32_t my_ex = lane < Sp ? (uint32_t)rec->ex[lane] : 0u;
  if (wid == 0) {
    if (lane < Sp) {
      sl.ex[lane] = (uint8_t)my_ex;
      sl.pos[2 * lane] = rec->pos[lane][0];
      sl.pos[2 * lane + 1] = rec->pos[lane][1];
    }
    if (lane < W) sl.s0[lane] = rec->s0[lane];
  }
  const uint32_t f0 = rec->f0;
  pair_sync<kPair>();
  if (wid == 0) {
    // projections and first syndrome words of rank r's alternatives (h, v,
    // diag): lane t = 3 r + alt
    for (int t = lane; t < 3 * Sp; t += 32) {
      const int r = t / 3, alt = t - 3 * (t / 3);
      const uint16_t pI = sl.pos[2 * r], pQ = sl.pos[2 * r + 1];
      const bool useI = alt != 1 && pI != kNoPos, useQ = alt != 0 && pQ != kNoPos;
      sl.dflt[t] = (useI ? __ldg(code.hf + pI) : 0u) ^ (useQ ? __ldg(code.hf + pQ) : 0u);
      sl.d0[t] = (useI ? __ldg(code.hcol + (size_t)pI * W) : 0u) ^ (useQ ? __ldg(code.hcol + (size_t)pQ * W) : 0u);
    }
    esp_table_warp(sl.ex, Sp, sl.E);
  }
  pair_sync<kPair>();
  // valid TEPs of weight <= v (lane v, a warp scan); the cap's weight class
  uint32_t cnt = lane <= Sp ? sl.E[Sp * kEStride + lane] : 0u;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(kFull, cnt, o);
    if (lane >= o) cnt += t;
  }
  const uint32_t total = __shfl_sync(kFull, cnt, Sp);
  const unsigned over = __ballot_sync(kFull, lane <= Sp && (uint64_t)cnt >= (uint64_t)a.cap);
  const int w_cap = over ? __ffs(over) - 1 : Sp;
  const int w_hi = kResume && a.w_step > 0 ? min(Sp, w_done + a.w_step) : Sp;
  const int w_lim = min(w_cap, w_hi);
  const int nAr = min(Sp >> 1, kFlipSideA), nBr = Sp - nAr;
  // existence bits of both sides' flip vectors (bit 2r: I slot, 2r+1: Q slot)
  const unsigned exh = __ballot_sync(kFull, lane < Sp && (my_ex & 1u));
  const unsigned exv = __ballot_sync(kFull, lane < Sp && (my_ex & 2u));
  uint32_t EA = 0, EB = 0;
#pragma unroll
  for (int r = 0; r < kFlipSideB; ++r) {
    if (r < kFlipSideA) EA |= (((exh >> r) & 1u) << (2 * r)) | (((exv >> r) & 1u) << (2 * r + 1));
    EB |= (((exh >> (nAr + r)) & 1u) << (2 * r)) | (((exv >> (nAr + r)) & 1u) << (2 * r + 1));
  }
  EA &= (1u << (2 * nAr)) - 1u;
  EB &= (1u << (2 * nBr)) - 1u;
  // flip projections H_b of both sides (b = 2r + slot; 0 where the flip does not exist)
  uint32_t HAlo[5], HAhi[5], HBlo[5], HBhi[9];
#pragma unroll
  for (int b = 0; b < 5; ++b) {
    HAlo[b] = ((EA >> b) & 1u) ? sl.dflt[(b >> 1) * 3 + (b & 1)] : 0u;
    HAhi[b] = ((EA >> (b + 5)) & 1u) ? sl.dflt[((b + 5) >> 1) * 3 + ((b + 5) & 1)] : 0u;
    HBlo[b] = ((EB >> b) & 1u) ? sl.dflt[(nAr + (b >> 1)) * 3 + (b & 1)] : 0u;
  }
#pragma unroll
  for (int b = 0; b < 9; ++b)
    HBhi[b] = ((EB >> (b + 5)) & 1u) ? sl.dflt[(nAr + ((b + 5) >> 1)) * 3 + ((b + 5) & 1)] : 0u;
  // visiting orders of the groups (pair mode: warp 0 writes the A order,
  // warp 1 the B list)
  uint32_t cumA_v;
  const int nGA = order_groups_a(EA >> 5, sl.ordA, &cumA_v, wid == 0);
  int nGB = 0;
  if (!kPair || wid == 1) nGB = order_groups_b(EB >> 5, max(0, 2 * nBr - 5), EB & 31u, HBhi, sl.bgrp);
  const uint32_t WA = __ballot_sync(kFull, ((uint32_t)lane & ~EA & 31u) == 0u);  // valid within-group A bits
  const uint32_t WB = __ballot_sync(kFull, ((uint32_t)lane & ~EB & 31u) == 0u);
  const bool lane_b_ok = (WB >> lane) & 1u;
  const int maxwA = code_weight(EA);
  // bit-planes of the within-group A projections: plane b bit i = bit b of P_i
  const uint32_t PA = xor_bits<5>((uint32_t)lane, HAlo);
  uint32_t pl[kPlanes];
#pragma unroll
  for (int b = 0; b < kPlanes; ++b) pl[b] = __ballot_sync(kFull, (PA >> b) & 1u);
  // table row t (lane t): A group g = ordA[t], planes inverted at the bits of
  // C_g = f0 ^ XOR_{b in g} H_{5+b}; rows past the valid groups never match
  if (wid == 0) {
    const int t = lane;
    uint32_t* row = sl.lut + t * kLutStride;
    if (t < nGA) {
      const uint32_t g = sl.ordA[t];
      const uint32_t cg = f0 ^ xor_bits<5>(g, HAhi);
      const uint32_t nwa = ~WA;
#pragma unroll
      for (int k = 0; k < kLutSets; ++k) {
        uint32_t q[kLutBits];
#pragma unroll
        for (int j = 0; j < kLutBits; ++j) q[j] = pl[kLutBits * k + j] ^ (0u - ((cg >> (kLutBits * k + j)) & 1u));
#pragma unroll
        for (int v = 0; v < kLutWords; ++v) {
          uint32_t w = nwa;
#pragma unroll
          for (int j = 0; j < kLutBits; ++j) w |= q[j] ^ (((v >> j) & 1) ? 0xFFFFFFFFu : 0u);
          row[kLutWords * k + v] = w;
        }
      }
    } else {
#pragma unroll
      for (int c = 0; c < kLutSets * kLutWords; ++c) row[c] = 0xFFFFFFFFu;
    }
  }
  // B side: this lane's within-group vector and its projection P'_lane
  const uint32_t PB = xor_bits<5>((uint32_t)lane, HBlo);
  if constexpr (kPair) {
    if (wid == 1 && lane == 0) ps->nGB = nGB;
    if (wid == 0 && lane == 0) ps->best_w = 127;
  }
  pair_sync<kPair>();
  if constexpr (kPair) nGB = ps->nGB;

  // --- chunks of two B groups in visiting order, A rows in visiting order ----
  constexpr int kB = 2;
  uint32_t best_rank = 0xFFFFFFFFu, best_code = 0;
  int best_w = 127;
  const int nCh = (nGB + 1) / 2;
  const unsigned wa_cnt = (unsigned)__popc(WA), wb_cnt = (unsigned)__popc(WB);
  for (int ch = wid; ch < nCh; ch += kPair ? 2 : 1) {
    const bool two = 2 * ch + 1 < nGB;
    const uint2 b0 = sl.bgrp[2 * ch];
    const uint2 b1 = two ? sl.bgrp[2 * ch + 1] : b0;
    const int wb = (int)(b0.y & 0xFFu);
    const int wb_hi = (int)max((b0.y >> 8) & 0xFFu, (b1.y >> 8) & 0xFFu);
    if constexpr (kPair) best_w = min(best_w, *(volatile int*)&ps->best_w);
    const int budget = min(best_w, w_lim) - wb;  // heaviest A weight still worth testing
    if (budget < 0) break;                      // later chunks are no lighter
    if (wb_hi + maxwA <= w_done) continue;      // every TEP here was tested before
    LutCmp cmp[kB];
    cmp[0].load(sl.lut, PB ^ b0.x);
    cmp[1].load(sl.lut, PB ^ b1.x);
    // A rows whose lightest weight is <= budget
    int g_end = (int)__shfl_sync(kFull, cumA_v, min(budget, 5));
    int g0 = 0;
    for (; g0 < g_end; g0 += kGroupUnroll) {
      uint32_t acc[kB][kGroupUnroll];
      uint32_t part[kB][kGroupUnroll / kQuarter];  // AND of the words of each quarter block
#pragma unroll
      for (int b = 0; b < kB; ++b) {
        cmp[b].block(g0);
        static_for<0, kGroupUnroll>([&](auto uc) {
          constexpr int u = decltype(uc)::value;
          acc[b][u] = cmp[b].template first<u>();
          if constexpr (u % kQuarter == 0) part[b][u / kQuarter] = acc[b][u];
          else part[b][u / kQuarter] &= acc[b][u];
        });
      }
      uint32_t all = 0xFFFFFFFFu;
#pragma unroll
      for (int b = 0; b < kB; ++b)
#pragma unroll
        for (int h = 0; h < kGroupUnroll / kQuarter; ++h) all &= part[b][h];
      if (!__any_sync(kFull, all != 0xFFFFFFFFu)) continue;
      // rare: a 15-bit match somewhere in the block; only the quarters with
      // a match in some lane read the fourth slice
      uint32_t cand[kB];
      uint32_t any_cand = 0;
#pragma unroll
      for (int b = 0; b < kB; ++b) {
        cand[b] = 0;
        static_for<0, kGroupUnroll / kQuarter>([&](auto hc) {
          constexpr int h = decltype(hc)::value;
          if (__any_sync(kFull, part[b][h] != 0xFFFFFFFFu)) {
            static_for<h * kQuarter, (h + 1) * kQuarter>([&](auto uc) {
              constexpr int u = decltype(uc)::value;
              cand[b] |= ~(acc[b][u] | cmp[b].template second<u>());
            });
          }
        });
        any_cand |= cand[b];
      }
      if (__any_sync(kFull, any_cand)) {
        // rare: verify this lane's candidates on every syndrome word
        uint32_t lr = 0xFFFFFFFFu, lc = 0;
#pragma unroll
        for (int b = 0; b < kB; ++b) {
          if (!cand[b] || !lane_b_ok || (b == 1 && !two)) continue;
          const uint32_t y = (((b == 0 ? b0.y : b1.y) >> 16) << 5) | (uint32_t)lane;
          for (int u = 0; u < kGroupUnroll; ++u) {
            uint32_t c = ~(cmp[b].first_at(g0 + u) | cmp[b].second_at(g0 + u));
            if (c == 0u || g0 + u >= nGA) continue;
            const uint32_t xg = (uint32_t)sl.ordA[g0 + u] << 5;
            while (c) {
              const int i = __ffs(c) - 1;
              c &= c - 1;
              const uint32_t cc = (xg | (uint32_t)i) | (y << (2 * nAr));
              if (kResume && code_weight(cc) > w_hi) continue;  // beyond this call's window
              // the full syndrome s0 ^ (the H columns the TEP flips), word by
              // word: the first from the kept deltas (a false match of the
              // projection fails there), the others from the code's columns
              uint32_t orr = sl.s0[0];
              for (int r = 0; r < Sp; ++r) {
                const uint32_t d = (cc >> (2 * r)) & 3u;
                if (d) orr ^= sl.d0[r * 3 + (d - 1)];
              }
              for (int w = 1; w < W && orr == 0; ++w) {
                uint32_t zz = sl.s0[w];
                for (int r = 0; r < Sp; ++r) {
                  const uint32_t d = (cc >> (2 * r)) & 3u;
                  const uint16_t pI = sl.pos[2 * r], pQ = sl.pos[2 * r + 1];
                  if ((d & 1u) && pI != kNoPos) zz ^= __ldg(code.hcol + (size_t)pI * W + w);
                  if ((d & 2u) && pQ != kNoPos) zz ^= __ldg(code.hcol + (size_t)pQ * W + w);
                }
                orr |= zz;
              }
              if (orr == 0) {
                const uint32_t rk = tep_rank(sl.E, Sp, sl.ex, cc);
                if (rk < lr) { lr = rk; lc = cc; }
              }
            }
          }
        }
        const uint32_t wr = __reduce_min_sync(kFull, lr);
        if (wr < best_rank) {
          const unsigned who = __ballot_sync(kFull, lr == wr);
          best_code = __shfl_sync(kFull, lc, __ffs(who) - 1);
          best_rank = wr;
          best_w = min(best_w, code_weight(best_code));
          if (kPair && lane == 0) atomicMin(&ps->best_w, best_w);
          const int nb = min(best_w, w_lim) - wb;
          g_end = nb < 0 ? 0 : min(g_end, (int)__shfl_sync(kFull, cumA_v, min(nb, 5)));
        }
      }
    }
    if (lane == 0)
      my_eval += (unsigned long long)min(g0, nGA) * wa_cnt * (unsigned long long)(wb_cnt * (two ? 2u : 1u));
  }
  if constexpr (kPair) {  // the lower of the two warps' first hits
    if (lane == 0) {
      ps->best_rank[wid] = best_rank;
      ps->best_code[wid] = best_code;
    }
    __syncthreads();
    if (wid == 1) return;
    if (ps->best_rank[1] < best_rank) {
      best_rank = ps->best_rank[1];
      best_code = ps->best_code[1];
    }
  }
  // --- result ---------------------------------------------------------------
  const bool hit = best_rank != 0xFFFFFFFFu && (uint64_t)best_rank <= (uint64_t)a.cap;
  if (kResume && !hit && w_hi < w_cap) {  // no codeword up to w_hi, weights left below the cap
    const uint32_t tested = __shfl_sync(kFull, cnt, w_hi), done = __shfl_sync(kFull, cnt, w_done);
    suspend_frame(a, fi, rec, w_hi, tested);
    if (lane == 0) my_useful += tested - done;
    __syncwarp();
    return;
  }
  const uint32_t done = __shfl_sync(kFull, cnt, w_done);
  if (lane == 0) {
    const unsigned f = out_frame(a, fi, rec);
    uint32_t q_out;
    if (hit) {
      uint32_t* cw = a.cw + out_cw_off(a, fi, rec);
      for (int r = 0; r < Sp; ++r) {
        const uint32_t d = (best_code >> (2 * r)) & 3u;
        if (d & 1u) { const uint16_t p = sl.pos[2 * r]; if (p != kNoPos) cw[p >> 5] ^= 1u << (p & 31); }
        if (d & 2u) { const uint16_t p = sl.pos[2 * r + 1]; if (p != kNoPos) cw[p >> 5] ^= 1u << (p & 31); }
      }
      q_out = best_rank;
      a.abandon[f] = 0;
    } else {
      q_out = (uint32_t)((uint64_t)total < (uint64_t)a.cap ? total : (uint64_t)a.cap);
      a.abandon[f] = 1;
    }
    a.queries[f] = q_out;
    my_useful += q_out - done;
  }
  __syncwarp();
}

// Persistent warp search: every warp (kPair: every pair of warps, one per
// CTA) pulls frames from the work queue and searches each in its own slice of
// shared memory. In pair mode the per-frame decisions are taken by thread 0 /
// warp 0 and read by both warps after a block barrier, so both reach every
// barrier.
template <int kMinBlocks, bool kResume, bool kPair>
__global__ void __launch_bounds__(128, kMinBlocks) k_search_warp(SearchArgs a) {
  extern __shared__ __align__(16) char smem_raw[];
  __shared__ PairShared ps;
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  const FlipSlice sl =
      flip_slice(smem_raw + (kPair ? 0 : wid) * flip_slice_bytes(a.Wmax, a.sp_max), a.Wmax, a.sp_max);
  const unsigned n_hard = kResume && a.cur_in ? (unsigned)a.n_cur : *(volatile unsigned*)&a.scr->n_hard;
  unsigned long long my_eval = 0, my_useful = 0;
  for (;;) {
    unsigned fi = 0;
    const FrameRec* rec = nullptr;
    if constexpr (kPair) {
      if (threadIdx.x == 0) ps.fi = atomicAdd(&a.scr->next, 1u);
      __syncthreads();
      fi = ps.fi;
      __syncthreads();
      if (fi >= n_hard) break;
      if (kResume && a.cur_in) {  // cursor validation by warp 0
        int ok = 0;
        if (wid == 0) ok = queue_entry(a, fi) != nullptr;
        if (threadIdx.x == 0) ps.flag = ok;
        __syncthreads();
        ok = ps.flag;
        __syncthreads();
        if (!ok) continue;
        rec = a.cur_in + fi;
      } else {
        rec = a.recs + fi;
      }
      if (a.deadline > 0) {
        if (threadIdx.x == 0) ps.flag = cut_at_deadline(a, rec, out_frame(a, fi, rec)) ? 1 : 0;
        __syncthreads();
        const int cut = ps.flag;
        __syncthreads();
        if (cut) continue;
      }
    } else {
      if (lane == 0) fi = atomicAdd(&a.scr->next, 1u);
      fi = __shfl_sync(kFull, fi, 0);
      if (fi >= n_hard) break;
      rec = kResume ? queue_entry(a, fi) : a.recs + fi;
      if (!rec) continue;
      if (a.deadline > 0) {
        int cut = 0;
        if (lane == 0) cut = cut_at_deadline(a, rec, out_frame(a, fi, rec));
        if (__shfl_sync(kFull, cut, 0)) continue;
      }
    }
    search_frame_flip<kResume, kPair>(a, fi, rec, sl, my_eval, my_useful, &ps);
  }
  if (lane == 0) {
    if (my_eval) atomicAdd(&a.scr->evaluated, my_eval);
    if (my_useful) atomicAdd(&a.scr->search_useful, my_useful);
  }
}

// ---------------------------------------------------------------------------
// Meet-in-the-middle hash join (membership GRAND_MEMBERSHIP_HASH; sides of 5
// ranks, S' <= 10, or 6 ranks, S' = 11, 12):
// the same A x B split, but instead of comparing every pair the warp inserts
// the A side's 32-bit syndrome projections (s0 ^ D_A) into a shared-memory
// hash table and looks every B projection up. Each pair whose projections are
// equal is confirmed on the full syndrome and ranked in closed form; the
// smallest rank is the canonical first hit. The decision equals that of the
// TEP-by-TEP test (every codeword TEP of the space is found), with O(|A| + |B|)
// work per frame instead of O(|A| |B|); no TEP is tested one by one, so this
// mode reports no TEP checks beyond the confirmed candidates.
// ---------------------------------------------------------------------------
// Table of one side of kSide ranks: 2 x 4^kSide slots (load factor <= 1/2).
// A slot packs the key's top (32 - kBits) bits with (A entry + 1) in the low
// kBits bits; 0 is empty.
template <int kSide>
struct HashDims {
  static constexpr int kBits = 2 * kSide + 1;
  static constexpr int kSlots = 1 << kBits;
  static constexpr uint32_t kLow = (1u << kBits) - 1u;
};
constexpr uint32_t kHashEmpty = 0u;

// Slot of a projection. The projections of one side form an affine subspace
// (XORs of a few deltas), so their low bits alone would fill one contiguous
// half of the table and make linear probing walk it; a multiplicative hash
// (the top bits of key * an odd constant) scatters them.
template <int kSide>
__device__ __forceinline__ uint32_t hash_slot(uint32_t key) {
  return (key * 0x9E3779B1u) >> (32 - HashDims<kSide>::kBits);
}

template <int kSide>
__host__ __device__ inline size_t hash_slice_bytes(int Wmax) {
  return warp_slice_bytes<kSide>(Wmax) + 4 * (size_t)HashDims<kSide>::kSlots;
}

template <int kSide, bool kResume>
__global__ void __launch_bounds__(128) k_search_hash(SearchArgs a) {
  using HD = HashDims<kSide>;
  extern __shared__ __align__(16) char smem_raw[];
  const int lane = threadIdx.x & 31;
  char* base = smem_raw + (threadIdx.x >> 5) * hash_slice_bytes<kSide>(a.Wmax);
  const WarpSlice sl = warp_slice<kSide>(base, a.Wmax);
  uint32_t* hslot = reinterpret_cast<uint32_t*>(base + warp_slice_bytes<kSide>(a.Wmax));
  const unsigned n_hard = kResume && a.cur_in ? (unsigned)a.n_cur : *(volatile unsigned*)&a.scr->n_hard;
  unsigned long long my_eval = 0, my_useful = 0;

  for (;;) {
    unsigned fi = 0;
    if (lane == 0) fi = atomicAdd(&a.scr->next, 1u);
    fi = __shfl_sync(kFull, fi, 0);
    if (fi >= n_hard) break;
    const FrameRec* rec = kResume ? queue_entry(a, fi) : a.recs + fi;
    if (!rec) continue;
    if (a.deadline > 0) {
      int cut = 0;
      if (lane == 0) cut = cut_at_deadline(a, rec, out_frame(a, fi, rec));
      if (__shfl_sync(kFull, cut, 0)) continue;
    }
    const int Sp = rec->sp;
    const int w_done = rec->w_done;
    const CodeDev code = a.codes[rec->code];
    const int W = code.W;
    if (lane < Sp) {
      sl.ex[lane] = rec->ex[lane];
      sl.pos[2 * lane] = rec->pos[lane][0];
      sl.pos[2 * lane + 1] = rec->pos[lane][1];
    }
    if (lane < W) sl.s0[lane] = rec->s0[lane];
    const uint32_t f0 = rec->f0;
    for (int t = lane; t < HD::kSlots; t += 32) hslot[t] = kHashEmpty;
    __syncwarp();
    for (int t = lane; t < Sp * 3 * W; t += 32) {
      const int r = t / (3 * W), rem = t % (3 * W), alt = rem / W, w = rem % W;
      const uint16_t pI = sl.pos[2 * r], pQ = sl.pos[2 * r + 1];
      const uint32_t h = (alt != 1 && pI != kNoPos) ? __ldg(code.hcol + (size_t)pI * W + w) : 0u;
      const uint32_t v = (alt != 0 && pQ != kNoPos) ? __ldg(code.hcol + (size_t)pQ * W + w) : 0u;
      sl.delta[t] = h ^ v;
    }
    for (int t = lane; t < 3 * Sp; t += 32) {
      const int r = t / 3, alt = t % 3;
      const uint16_t pI = sl.pos[2 * r], pQ = sl.pos[2 * r + 1];
      const uint32_t h = (alt != 1 && pI != kNoPos) ? __ldg(code.hf + pI) : 0u;
      const uint32_t v = (alt != 0 && pQ != kNoPos) ? __ldg(code.hf + pQ) : 0u;
      sl.dflt[t] = h ^ v;
    }
    esp_table_warp(sl.ex, Sp, sl.E);
    __syncwarp();
    const uint32_t total = esp_total(sl.E, Sp);
    const int nAr = Sp >> 1, nBr = Sp - nAr;
    const unsigned nA_all = warp_side_layout(sl, 0, nAr, sl.startA, sl.ordA, sl.invA, sl.cumA);
    const unsigned nB_all = warp_side_layout(sl, nAr, nBr, sl.startB, sl.ordB, sl.invB, sl.cumB);
    // weight window: w_done + 1 .. w_hi. With a step, only entries of weight
    // <= w_hi take part and a pair heavier than w_hi is not a hit; the cap's
    // weight class w_cap decides whether an empty window suspends the frame.
    int w_cap = Sp;
    if (kResume) {
      uint64_t acc = 0;
      for (int v = 0; v <= Sp; ++v) {
        acc += sl.E[Sp * kEStride + v];
        if (acc >= (uint64_t)a.cap) { w_cap = v; break; }
      }
    }
    const int w_hi = kResume && a.w_step > 0 ? min(Sp, w_done + a.w_step) : Sp;
    const unsigned nA = (!kResume || w_hi >= nAr) ? nA_all : sl.cumA[w_hi];
    const unsigned nB = (!kResume || w_hi >= nBr) ? nB_all : sl.cumB[w_hi];
    // A side: projections (with s0's) into the hash table -- by doubling into
    // the scalar buffer for 5-rank sides, from the table layout otherwise
    if constexpr (kSide == kWarpSideMax) warp_fill_side(sl, 0, nAr, sl.startA, sl.ordA, sl.invA, f0, sl.Bz);
    for (unsigned e = lane; e < nA; e += 32) {
      uint32_t key;
      if constexpr (kSide == kWarpSideMax) {
        key = sl.Bz[e];
      } else {
        uint32_t acode;
        warp_side_entry(sl, 0, nAr, sl.startA, sl.ordA, f0, e, key, acode);
      }
      const uint32_t packed = (key & ~HD::kLow) | (e + 1u);
      uint32_t h = hash_slot<kSide>(key);
      for (int probe = 0; probe < HD::kSlots; ++probe) {  // at most half full: ends at an empty slot
        if (atomicCAS(&hslot[h], kHashEmpty, packed) == kHashEmpty) break;
        h = (h + 1) & (HD::kSlots - 1);
      }
    }
    __syncwarp();
    // B side: one lookup per entry
    if constexpr (kSide == kWarpSideMax) warp_fill_side(sl, nAr, nBr, sl.startB, sl.ordB, sl.invB, 0u, sl.Bz);
    uint32_t lr = 0xFFFFFFFFu, lc = 0;
    // A slot whose top key bits equal the B projection's (the slot index came
    // from the whole key): a candidate pair, confirmed on every syndrome word
    // and ranked in closed form.
    auto confirm = [&](uint32_t slot, unsigned col, bool& have_b, uint32_t& bcode) {
      const uint32_t row = (slot & HD::kLow) - 1u;
      if (!have_b) {
        uint32_t bq;
        warp_side_entry(sl, nAr, nBr, sl.startB, sl.ordB, 0u, col, bq, bcode);
        have_b = true;
      }
      uint32_t aq, acode;
      warp_side_entry(sl, 0, nAr, sl.startA, sl.ordA, f0, row, aq, acode);
      const uint32_t cc = acode | (bcode << (2 * nAr));
      uint32_t orr = 0;
      for (int w = 0; w < W; ++w) {
        uint32_t zz = sl.s0[w];
        for (int r = 0; r < Sp; ++r) {
          const uint32_t d = (cc >> (2 * r)) & 3u;
          if (d) zz ^= sl.delta[((size_t)r * 3 + (d - 1)) * W + w];
        }
        orr |= zz;
      }
      ++my_eval;
      if (orr == 0 && (!kResume || code_weight(cc) <= w_hi)) {
        const uint32_t rk = tep_rank(sl.E, Sp, sl.ex, cc);
        if (rk < lr) {
          lr = rk;
          lc = cc;
        }
      }
    };
    if constexpr (kSide == kWarpSideMax) {
      // One probe per lane and step: a lane whose probe sequence ends (an
      // empty slot) starts its next entry at once (a read of the scalar B
      // table), so lanes with short sequences do not wait for the longest
      // one of the warp before moving on.
      unsigned col = lane;
      bool live = false, have_b = false;
      uint32_t zhi = 0, h = 0, bcode = 0;
      int probes = 0;
      for (;;) {
        if (!live && col < nB) {
          const uint32_t z = sl.Bz[col];
          have_b = false;
          bcode = 0;
          h = hash_slot<kSide>(z);
          zhi = z & ~HD::kLow;
          probes = 0;
          live = true;
        }
        if (!__any_sync(kFull, live)) break;
        if (live) {
          const uint32_t slot = hslot[h];
          // the table is at most half full, so every sequence meets an empty
          // slot; the probe count bounds it regardless
          if (slot == kHashEmpty || ++probes > HD::kSlots) {
            live = false;
            col += 32;
            continue;
          }
          if ((slot & ~HD::kLow) == zhi) confirm(slot, col, have_b, bcode);
          h = (h + 1) & (HD::kSlots - 1);
        }
      }
    } else {
      // sides of 6 ranks: an entry's projection comes from the table layout
      // (a search), so the warp starts its entries together
      for (unsigned col = lane; col < nB; col += 32) {
        uint32_t z, bcode = 0;
        warp_side_entry(sl, nAr, nBr, sl.startB, sl.ordB, 0u, col, z, bcode);
        bool have_b = true;
        uint32_t h = hash_slot<kSide>(z);
        const uint32_t zhi = z & ~HD::kLow;
        for (int probe = 0; probe < HD::kSlots; ++probe) {
          const uint32_t slot = hslot[h];
          if (slot == kHashEmpty) break;
          if ((slot & ~HD::kLow) == zhi) confirm(slot, col, have_b, bcode);
          h = (h + 1) & (HD::kSlots - 1);
        }
      }
    }
    const uint32_t best_rank = __reduce_min_sync(kFull, lr);
    const unsigned who = __ballot_sync(kFull, lr == best_rank);
    const uint32_t best_code = __shfl_sync(kFull, lc, __ffs(who) - 1);
    // --- result -------------------------------------------------------------
    const bool hit = best_rank != 0xFFFFFFFFu && (uint64_t)best_rank <= (uint64_t)a.cap;
    if (kResume && !hit && w_hi < w_cap) {  // no codeword up to w_hi, weights left below the cap
      uint32_t tested = 0, done = 0;
      for (int v = 0; v <= w_hi; ++v) tested += sl.E[Sp * kEStride + v];
      for (int v = 0; v <= w_done; ++v) done += sl.E[Sp * kEStride + v];
      suspend_frame(a, fi, rec, w_hi, tested);
      if (lane == 0) my_useful += tested - done;
      __syncwarp();
      continue;
    }
    if (lane == 0) {
      const unsigned f = out_frame(a, fi, rec);
      uint32_t q_out;
      if (hit) {
        uint32_t* cw = a.cw + out_cw_off(a, fi, rec);
        for (int r = 0; r < Sp; ++r) {
          const uint32_t d = (best_code >> (2 * r)) & 3u;
          if (d & 1u) { const uint16_t p = sl.pos[2 * r]; if (p != kNoPos) cw[p >> 5] ^= 1u << (p & 31); }
          if (d & 2u) { const uint16_t p = sl.pos[2 * r + 1]; if (p != kNoPos) cw[p >> 5] ^= 1u << (p & 31); }
        }
        q_out = best_rank;
        a.abandon[f] = 0;
      } else {
        q_out = (uint32_t)((uint64_t)total < (uint64_t)a.cap ? total : (uint64_t)a.cap);
        a.abandon[f] = 1;
      }
      a.queries[f] = q_out;
      uint32_t done = 0;
      for (int v = 0; v <= w_done; ++v) done += sl.E[Sp * kEStride + v];
      my_useful += q_out - done;
    }
    __syncwarp();
  }
  for (int o = 16; o; o >>= 1) my_eval += __shfl_xor_sync(kFull, my_eval, o);
  if (lane == 0) {
    if (my_eval) atomicAdd(&a.scr->evaluated, my_eval);
    if (my_useful) atomicAdd(&a.scr->search_useful, my_useful);
  }
}

// ---------------------------------------------------------------------------
// Bit-level GRAND-AB: TEPs of 0..max_weight flipped bits in colex order
// ---------------------------------------------------------------------------
struct AbArgs {
  const float* samples;   // fused: [n_frames][N] BPSK samples
  const uint32_t* y_in;   // else: packed hard words
  const uint8_t* nmask;   // optional: bit7 = non-finite sample
  CodeDev code;
  int64_t n_frames;
  int max_weight;
  int64_t cap;
  uint32_t* cw;
  uint32_t* queries;
  uint8_t* abandon;
  Scratch* scr;
  long long deadline;  // grand_params.deadline_ns (0: none)
};

__global__ void __launch_bounds__(128) k_ab(AbArgs a) {
  __shared__ uint32_t s_y[4][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t gwarp = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int N = a.code.N, W = a.code.W, NW = N >> 5;
  uint32_t* y = s_y[wib];
  unsigned long long evaluated = 0;
  for (int64_t f = gwarp; f < a.n_frames; f += nwarps) {
    bool nonfinite = false;
    if (a.samples) {
      for (int w = 0; w < NW; ++w) {
        float v = a.samples[f * N + 32 * w + lane];
        const bool nf = !isfinite(v);
        nonfinite |= nf;
        if (nf) v = 0.0f;
        const unsigned b = __ballot_sync(kFull, v < 0.0f);
        if (lane == 0) y[w] = b;
      }
    } else {
      if (lane < NW) y[lane] = a.y_in[f * NW + lane];
      if (a.nmask)
        for (int j = lane; j < N; j += 32) nonfinite |= (a.nmask[f * N + j] & 128u) != 0;
    }
    nonfinite = __any_sync(kFull, nonfinite);
    __syncwarp();
    if (nonfinite) {
      if (lane < NW) a.cw[f * NW + lane] = y[lane];
      if (lane == 0) { a.queries[f] = 0; a.abandon[f] = 2; }
      __syncwarp();
      continue;
    }
    if (a.deadline > 0) {
      int cut = 0;
      if (lane == 0) cut = past_deadline(&a.scr->t0, a.deadline);
      if (__shfl_sync(kFull, cut, 0)) {  // not searched: the hard word, marked 5
        if (lane < NW) a.cw[f * NW + lane] = y[lane];
        if (lane == 0) { a.queries[f] = 0; a.abandon[f] = 5; atomicOr(a.code.status, 1u); }
        __syncwarp();
        continue;
      }
    }
    uint32_t s0[kWMax];
    uint32_t f0 = 0;
#pragma unroll
    for (int w = 0; w < kWMax; ++w) s0[w] = 0;
    for (int j = lane; j < N; j += 32)
      if ((y[j >> 5] >> (j & 31)) & 1u) {
#pragma unroll
        for (int w = 0; w < kWMax; ++w)
          if (w < W) s0[w] ^= __ldg(a.code.hcol + (size_t)j * W + w);
        f0 ^= __ldg(a.code.hf + j);
      }
    for (int o = 16; o; o >>= 1) f0 ^= __shfl_xor_sync(kFull, f0, o);
#pragma unroll
    for (int w = 0; w < kWMax; ++w)
      if (w < W) {
        uint32_t v = s0[w];
        for (int o = 16; o; o >>= 1) v ^= __shfl_xor_sync(kFull, v, o);
        s0[w] = v;
      }
    // classes in order; position within the order = start(w) + colex + 1
    uint64_t start = 0;
    bool found = false;
    uint64_t hit_q = 0;
    int hit_p[GRAND_AB_WEIGHT_MAX] = {0, 0, 0, 0};
    int hit_w = 0;
    for (int w = 0; w <= a.max_weight && !found && start < (uint64_t)a.cap; ++w) {
      const uint64_t nsets = binom_big(N, w);
      const uint64_t limit = min(nsets, (uint64_t)a.cap - start);
      for (uint64_t base = 0; base < limit && !found; base += 32) {
        const uint64_t c = base + lane;
        bool hit = false;
        int P[GRAND_AB_WEIGHT_MAX] = {0, 0, 0, 0};
        if (c < limit) {
          ++evaluated;
          uint64_t rem = c;
          int hiP = N - 1;
          for (int j = w; j >= 1; --j) {
            // largest p <= hiP with C(p, j) <= rem (binary search)
            int lo = j - 1, hi = hiP;
            while (lo < hi) {
              const int mid = (lo + hi + 1) >> 1;
              if (binom_big(mid, j) <= rem) lo = mid; else hi = mid - 1;
            }
            P[j - 1] = lo;
            rem -= binom_big(lo, j);
            hiP = lo - 1;
          }
          uint32_t z0 = f0;
          for (int j = 0; j < w; ++j) z0 ^= __ldg(a.code.hf + P[j]);
          if (z0 == 0) {
            uint32_t orr = 0;
            for (int ww = 0; ww < W; ++ww) {
              uint32_t z = s0[ww];
              for (int j = 0; j < w; ++j) z ^= __ldg(a.code.hcol + (size_t)P[j] * W + ww);
              orr |= z;
            }
            hit = orr == 0;
          }
        }
        const unsigned hb = __ballot_sync(kFull, hit);
        if (hb) {
          const int src = __ffs(hb) - 1;
          found = true;
          hit_w = w;
          hit_q = start + base + src + 1;
          for (int j = 0; j < GRAND_AB_WEIGHT_MAX; ++j) hit_p[j] = __shfl_sync(kFull, P[j], src);
        }
      }
      start += nsets;
    }
    if (found && lane == 0)
      for (int j = 0; j < hit_w; ++j) y[hit_p[j] >> 5] ^= 1u << (hit_p[j] & 31);
    __syncwarp();
    if (lane < NW) a.cw[f * NW + lane] = y[lane];
    if (lane == 0) {
      uint64_t total = 0;
      for (int w = 0; w <= a.max_weight; ++w) total += binom_big(N, w);
      a.queries[f] = (uint32_t)(found ? hit_q : min(total, (uint64_t)a.cap));
      a.abandon[f] = found ? 0 : 1;
    }
    __syncwarp();
  }
  for (int o = 16; o; o >>= 1) evaluated += __shfl_xor_sync(kFull, evaluated, o);
  if (lane == 0 && evaluated && a.scr) atomicAdd(&a.scr->evaluated, evaluated);
}

// ---------------------------------------------------------------------------
// Bit-level GRAND-AB on a code whose syndrome fits one word (N - K <= 32) and
// N <= 64, weights <= 3: the TEPs split into a pair and a single.
//
// A TEP of weight 3, positions p1 < p2 < p3, is a codeword iff
//     s0 ^ h_p1 ^ h_p2 == h_p3          (h_j = column j of H, s0 = H y).
// Its colex rank is C(p3,3) + c with c = C(p2,2) + p1 the colex rank of the
// pair, so the first hit in canonical order is the hit of smallest p3 and,
// among those, of smallest c. Each lane takes one pair per step (pairs in
// colex order) and compares its target s0 ^ h_p1 ^ h_p2 with 32 columns at
// once: the columns of a 32-position group are held as R bit-planes
// (plane[b] bit i = bit b of h_{32 g + i}), and OR_b(plane[b] ^ -(t_b)) has a
// zero at every column equal to t -- 3 logic ops per syndrome bit for 32
// TEPs. Weights 1 and 2 use the same compare (a single against s0, a column
// p2 against s0 ^ h_p2). A step whose pairs all have p2 >= the best p3 so far
// cannot improve it, which ends the weight-3 walk of a decoded frame early.
// The planes depend only on the code: a CTA builds them once and keeps them
// in registers for all its frames. Ranks fit 32 bits for N <= 1024.
// ---------------------------------------------------------------------------
// Columns of group g equal to t (bit i: column 32 g + i). g must be a
// compile-time constant after unrolling (the planes stay in registers).
template <int kNG, int kR>
__device__ __forceinline__ uint32_t ab_match(const uint32_t (&plane)[kNG][kR], int g, uint32_t t) {
  uint32_t acc = 0;
#pragma unroll
  for (int b = 0; b < kR; ++b) acc |= plane[g][b] ^ (0u - ((t >> b) & 1u));
  return ~acc;
}

// Word w of a frame's words held uniformly by every lane, picked without
// dynamic register indexing.
template <int kNG>
__device__ __forceinline__ uint32_t pick_word(const uint32_t (&v)[kNG], int w) {
  uint32_t r = v[0];
#pragma unroll
  for (int i = 1; i < kNG; ++i)
    if (w == i) r = v[i];
  return r;
}

template <int kNG, int kR>
__global__ void __launch_bounds__(128) k_ab_split(AbArgs a) {
  __shared__ uint32_t s_h[4][32 * kNG];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t gwarp = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  constexpr int N = 32 * kNG;
  uint32_t* h = s_h[wib];
  // columns and their bit-planes (code constants; syndrome bits >= kR are 0)
  uint32_t plane[kNG][kR];
#pragma unroll
  for (int g = 0; g < kNG; ++g) {
    const uint32_t col = __ldg(a.code.hcol + 32 * g + lane);
    h[32 * g + lane] = col;
#pragma unroll
    for (int b = 0; b < kR; ++b) plane[g][b] = __ballot_sync(kFull, (col >> b) & 1u);
  }
  __syncwarp();
  const uint32_t c2N = (uint32_t)(N * (N - 1) / 2);
  uint64_t total = 0;
  for (int w = 0; w <= a.max_weight; ++w) total += binom_big(N, w);
  const uint64_t cap = (uint64_t)a.cap;
  unsigned long long evaluated = 0;
  for (int64_t f = gwarp; f < a.n_frames; f += nwarps) {
    bool nonfinite = false;
    uint32_t ywords[kNG];
    if (a.samples) {
#pragma unroll
      for (int w = 0; w < kNG; ++w) {
        float v = a.samples[f * N + 32 * w + lane];
        const bool nf = !isfinite(v);
        nonfinite |= nf;
        if (nf) v = 0.0f;
        ywords[w] = __ballot_sync(kFull, v < 0.0f);
      }
    } else {
#pragma unroll
      for (int w = 0; w < kNG; ++w) ywords[w] = __ldg(a.y_in + f * kNG + w);
      if (a.nmask)
        for (int j = lane; j < N; j += 32) nonfinite |= (a.nmask[f * N + j] & 128u) != 0;
    }
    nonfinite = __any_sync(kFull, nonfinite);
    if (nonfinite) {
      if (lane < kNG) a.cw[f * kNG + lane] = pick_word<kNG>(ywords, lane);
      if (lane == 0) { a.queries[f] = 0; a.abandon[f] = 2; }
      continue;
    }
    if (a.deadline > 0) {
      int cut = 0;
      if (lane == 0) cut = past_deadline(&a.scr->t0, a.deadline);
      if (__shfl_sync(kFull, cut, 0)) {  // not searched: the hard word, marked 5
        if (lane < kNG) a.cw[f * kNG + lane] = pick_word<kNG>(ywords, lane);
        if (lane == 0) { a.queries[f] = 0; a.abandon[f] = 5; atomicOr(a.code.status, 1u); }
        continue;
      }
    }
    // base syndrome s0 = H y: XOR of the columns at the one-bits of y
    uint32_t part = 0;
#pragma unroll
    for (int w = 0; w < kNG; ++w)
      if ((ywords[w] >> lane) & 1u) part ^= h[32 * w + lane];
    const uint32_t s0 = __reduce_xor_sync(kFull, part);
    // first hit: weight and colex rank within the weight (positions p[0..w-1])
    int hit_w = -1;
    uint32_t hit_rank = 0;
    if (s0 == 0) {
      hit_w = 0;
      evaluated += (lane == 0);
    }
    if (hit_w < 0 && a.max_weight >= 1 && cap > 1) {
      uint32_t best = 0xFFFFFFFFu;
#pragma unroll
      for (int g = 0; g < kNG; ++g) {
        const uint32_t m = ab_match<kNG, kR>(plane, g, s0);
        if (m) best = min(best, (uint32_t)(32 * g + __ffs(m) - 1));
      }
      evaluated += (lane == 0) ? N : 0;
      if (best != 0xFFFFFFFFu) { hit_w = 1; hit_rank = best; }
    }
    if (hit_w < 0 && a.max_weight >= 2 && cap > 1 + (uint64_t)N) {
      // lane = p2 (per group step), matches p1 < p2
      uint32_t best = 0xFFFFFFFFu;
#pragma unroll
      for (int s = 0; s < kNG; ++s) {
        const int p2 = 32 * s + lane;
        const uint32_t t = s0 ^ h[p2];
#pragma unroll
        for (int g = 0; g <= s; ++g) {
          uint32_t m = ab_match<kNG, kR>(plane, g, t);
          if (g == s) m &= (1u << lane) - 1u;  // p1 < p2
          if (m) best = min(best, (uint32_t)(p2 * (p2 - 1) / 2 + 32 * g + __ffs(m) - 1));
        }
        evaluated += (uint32_t)p2;
      }
      best = __reduce_min_sync(kFull, best);
      if (best != 0xFFFFFFFFu) { hit_w = 2; hit_rank = best; }
    }
    if (hit_w < 0 && a.max_weight >= 3 && cap > 1 + (uint64_t)N + c2N) {
      // kPairs pairs per lane and step (independent compares in flight: the
      // step count, which sets an abandoned frame's latency, drops by kPairs)
      constexpr int kPairs = 4;
      uint32_t best = 0xFFFFFFFFu;  // colex rank of the best triple so far
      int best_p3 = N;
      for (uint32_t base = 0; base < c2N; base += 32 * kPairs) {
        // smallest p2 of this step's pairs: pairs are in colex order
        int p2 = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)base)) * 0.5f);
        while ((uint32_t)(p2 * (p2 - 1) / 2) > base) --p2;
        while ((uint32_t)((p2 + 1) * p2 / 2) <= base) ++p2;
        if (p2 >= best_p3 - 1) break;  // every later pair needs p3 > p2 >= best_p3 - 1
#pragma unroll
        for (int k = 0; k < kPairs; ++k) {
          const uint32_t c = base + 32 * k + lane;
          if (c < c2N) {
            int q2 = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)c)) * 0.5f);
            while ((uint32_t)(q2 * (q2 - 1) / 2) > c) --q2;
            while ((uint32_t)((q2 + 1) * q2 / 2) <= c) ++q2;
            const int q1 = (int)(c - (uint32_t)(q2 * (q2 - 1) / 2));
            const uint32_t t = s0 ^ h[q1] ^ h[q2];
#pragma unroll
            for (int g = 0; g < kNG; ++g) {
              if (32 * g + 31 <= q2) continue;  // every p3 of the group is <= p2
              uint32_t m = ab_match<kNG, kR>(plane, g, t);
              if (32 * g <= q2) m &= ~((2u << (q2 - 32 * g)) - 1u);  // p3 > p2
              if (m) {
                const uint32_t p3 = 32 * g + __ffs(m) - 1;
                best = min(best, (uint32_t)(p3 * (p3 - 1) * (p3 - 2) / 6) + c);
                break;
              }
            }
            evaluated += (uint32_t)(N - 1 - q2);
          }
        }
        best = __reduce_min_sync(kFull, best);
        if (best != 0xFFFFFFFFu) {
          int p3 = 2;
          while ((uint32_t)((p3 + 1) * p3 * (p3 - 1) / 6) <= best) ++p3;
          best_p3 = p3;
        }
      }
      if (best != 0xFFFFFFFFu) { hit_w = 3; hit_rank = best; }
    }
    // query position of the hit (1-based) and the decoded word
    uint64_t q = 0;
    if (hit_w >= 0) {
      uint64_t start = 0;
      for (int w = 0; w < hit_w; ++w) start += binom_big(N, w);
      q = start + hit_rank + 1;
    }
    const bool decoded = hit_w >= 0 && q <= cap;
    if (lane < kNG) {
      uint32_t word = pick_word<kNG>(ywords, lane);
      if (decoded) {
        // unrank the hit's positions (colex, largest first)
        uint32_t rem = hit_rank;
        for (int j = hit_w; j >= 1; --j) {
          int pj = j - 1;
          while (binom_big(pj + 1, j) <= rem) ++pj;
          rem -= (uint32_t)binom_big(pj, j);
          if ((pj >> 5) == lane) word ^= 1u << (pj & 31);
        }
      }
      a.cw[f * kNG + lane] = word;
    }
    if (lane == 0) {
      a.queries[f] = (uint32_t)(decoded ? q : min(total, cap));
      a.abandon[f] = decoded ? 0 : 1;
    }
  }
  for (int o = 16; o; o >>= 1) evaluated += __shfl_xor_sync(kFull, evaluated, o);
  if (lane == 0 && evaluated && a.scr) atomicAdd(&a.scr->evaluated, evaluated);
}

// ---------------------------------------------------------------------------
// Public demodulation: one thread per symbol
// ---------------------------------------------------------------------------
struct DemodArgs {
  const float2* symbols;
  int64_t n_sym;
  int L, m, side, N, NW, lik;
  float q, inv_d;
  uint16_t* hard_idx;
  uint32_t* key;
  uint8_t* nmask;
  float* rel;
  uint32_t* y;
  uint64_t Lmagic;  // ceil(2^64 / L): frame of symbol s = high word of s * Lmagic (exact for s < 2^64 / L)
};

// One symbol of the public demodulation call (outputs that are NULL are
// skipped); rl = the symbol's Gray label bits in transmission order (bit k =
// label bit 2m-1-k), for the hard word. kM = log2(sqrt(M)) is a template
// argument so that the level arithmetic folds into constants.
// Square root by the SFU's approximate instruction (relative error about
// 2^-22, far inside the 1e-5 tolerance of the reported likelihood).
__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

template <int kM, int kLit>
__device__ __forceinline__ void demod_one(const DemodArgs& a, float2 v, uint16_t& hidx, uint32_t& key, uint8_t& nmask,
                                          float& rel, uint32_t& rl) {
  const bool nf = !(isfinite(v.x) && isfinite(v.y));
  if (nf) v = make_float2(0.0f, 0.0f);
  const AxisDemod I = demod_axis_q(v.x, a.q, 1 << kM, kLit);
  const AxisDemod Q = demod_axis_q(v.y, a.q, 1 << kM, kLit);
  hidx = (uint16_t)((I.level << 8) | Q.level);
  key = (uint32_t)I.dq * (uint32_t)I.dq + (uint32_t)Q.dq * (uint32_t)Q.dq;
  nmask = (uint8_t)make_nmask(I, Q, nf);
  if (a.rel) {
    const float dI = axis_dist_f32(v.x, a.inv_d, I.amp, I.outside, kLit);
    const float dQ = axis_dist_f32(v.y, a.inv_d, Q.amp, Q.outside, kLit);
    rel = sqrt_approx(dI * dI + dQ * dQ);
  }
  const uint32_t label = ((uint32_t)gray_code(I.level) << kM) | (uint32_t)gray_code(Q.level);
  rl = __brev(label) >> (32 - 2 * kM);
}

// OR `bits` (at most 24) into the packed hard word yf at bit position p0;
// words at or beyond NW (bits >= N: padding) are dropped.
__device__ __forceinline__ void or_bits(uint32_t* yf, int NW, int p0, uint32_t bits) {
  const int wd = p0 >> 5, sh = p0 & 31;
  const uint32_t lo = bits << sh, hi = sh ? (bits >> (32 - sh)) : 0u;
  if (wd < NW && lo) atomicOr(yf + wd, lo);
  if (hi && wd + 1 < NW) atomicOr(yf + wd + 1, hi);
}

// Two symbols per thread: 16-byte loads, paired stores (every pointer aligned
// for its pair type, checked by the host); otherwise one symbol per thread.
// The frame of a symbol is found once per thread and then advanced by the
// grid stride (a quotient and remainder of the stride by L, no division per
// step); the pair's label bits go into the hard word with one OR when both
// symbols belong to the same frame. kLit: the likelihood reading (selects
// fold into constants).
template <bool kPaired, int kM, int kLit>
__global__ void __launch_bounds__(256, 8) k_demod(DemodArgs a) {
  constexpr int b2 = 2 * kM;
  const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
  if constexpr (!kPaired) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < a.n_sym; s += gstride) {
      uint16_t h0;
      uint32_t k0, rl0;
      uint8_t m0;
      float r0 = 0.0f;
      demod_one<kM, kLit>(a, a.symbols[s], h0, k0, m0, r0, rl0);
      if (a.hard_idx) a.hard_idx[s] = h0;
      if (a.key) a.key[s] = k0;
      if (a.nmask) a.nmask[s] = m0;
      if (a.rel) a.rel[s] = r0;
      if (a.y) {
        const int64_t f = (int64_t)__umul64hi((uint64_t)s, a.Lmagic);
        const int i = (int)(s - f * a.L);
        or_bits(a.y + f * a.NW, a.NW, b2 * i, rl0);
      }
    }
    return;
  }
  const int64_t n_pairs = a.n_sym >> 1;
  const float4* sym4 = reinterpret_cast<const float4*>(a.symbols);
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // frame f and symbol i of this thread's first pair, and the symbol stride
  // 2 * gstride = dq frames + dr symbols
  int64_t f = (int64_t)__umul64hi((uint64_t)(2 * t0), a.Lmagic);
  int i = (int)(2 * t0 - f * a.L);
  const int64_t dq = (int64_t)__umul64hi((uint64_t)(2 * gstride), a.Lmagic);
  const int dr = (int)(2 * gstride - dq * a.L);
  for (int64_t t = t0; t <= n_pairs; t += gstride) {
    const int64_t s = 2 * t;
    if (t < n_pairs) {
      const float4 v = sym4[t];
      uint16_t h0, h1;
      uint32_t k0, k1, rl0, rl1;
      uint8_t m0, m1;
      float r0 = 0.0f, r1 = 0.0f;
      demod_one<kM, kLit>(a, make_float2(v.x, v.y), h0, k0, m0, r0, rl0);
      demod_one<kM, kLit>(a, make_float2(v.z, v.w), h1, k1, m1, r1, rl1);
      if (a.hard_idx) reinterpret_cast<ushort2*>(a.hard_idx)[t] = make_ushort2(h0, h1);
      if (a.key) reinterpret_cast<uint2*>(a.key)[t] = make_uint2(k0, k1);
      if (a.nmask) reinterpret_cast<uchar2*>(a.nmask)[t] = make_uchar2(m0, m1);
      if (a.rel) reinterpret_cast<float2*>(a.rel)[t] = make_float2(r0, r1);
      if (a.y) {
        uint32_t* yf = a.y + f * a.NW;
        if (i + 1 < a.L) {
          or_bits(yf, a.NW, b2 * i, rl0 | (rl1 << b2));
        } else {  // the pair straddles two frames
          or_bits(yf, a.NW, b2 * i, rl0);
          or_bits(yf + a.NW, a.NW, 0, rl1);
        }
      }
    } else if (s < a.n_sym) {  // odd count: the last symbol
      uint16_t h0;
      uint32_t k0, rl0;
      uint8_t m0;
      float r0 = 0.0f;
      demod_one<kM, kLit>(a, a.symbols[s], h0, k0, m0, r0, rl0);
      if (a.hard_idx) a.hard_idx[s] = h0;
      if (a.key) a.key[s] = k0;
      if (a.nmask) a.nmask[s] = m0;
      if (a.rel) a.rel[s] = r0;
      if (a.y) or_bits(a.y + f * a.NW, a.NW, b2 * i, rl0);
    }
    // advance to the next pair of this thread
    f += dq;
    i += dr;
    if (i >= a.L) {
      i -= a.L;
      f += 1;
    }
  }
}

// BPSK hard decisions: one warp per 32 samples
__global__ void __launch_bounds__(256) k_demod_bpsk(const float* r, int64_t n_words, uint32_t* y, uint8_t* nmask) {
  const int lane = threadIdx.x & 31;
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < n_words;
       w += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    float v = r[32 * w + lane];
    const bool nf = !isfinite(v);
    if (nf) v = 0.0f;
    const unsigned b = __ballot_sync(kFull, v < 0.0f);
    if (lane == 0 && y) y[w] = b;
    if (nmask) nmask[32 * w + lane] = nf ? 128 : 0;
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

template <int kM>
static void launch_demod_m(const DemodArgs& a, bool paired, int grid, cudaStream_t st) {
  if (a.lik == GRAND_LIK_LITERAL) {
    if (paired)
      k_demod<true, kM, 1><<<grid, 256, 0, st>>>(a);
    else
      k_demod<false, kM, 1><<<grid, 256, 0, st>>>(a);
  } else {
    if (paired)
      k_demod<true, kM, 0><<<grid, 256, 0, st>>>(a);
    else
      k_demod<false, kM, 0><<<grid, 256, 0, st>>>(a);
  }
}

// m = log2(sqrt(M)) in 1..6 (validated by the caller).
static void launch_demod(const DemodArgs& a, bool paired, int grid, cudaStream_t st) {
  switch (a.m) {
    case 1: launch_demod_m<1>(a, paired, grid, st); break;
    case 2: launch_demod_m<2>(a, paired, grid, st); break;
    case 3: launch_demod_m<3>(a, paired, grid, st); break;
    case 4: launch_demod_m<4>(a, paired, grid, st); break;
    case 5: launch_demod_m<5>(a, paired, grid, st); break;
    default: launch_demod_m<6>(a, paired, grid, st); break;
  }
}

typedef void (*PrepKernel)(PrepArgs);
static PrepKernel prep_kernel_for(int Wmax, bool solve = false) {
  if (solve) {
    if (Wmax <= 1) return k_prep<1, true>;
    if (Wmax <= 2) return k_prep<2, true>;
    if (Wmax <= 4) return k_prep<4, true>;
    if (Wmax <= 8) return k_prep<8, true>;
    return k_prep<16, true>;
  }
  if (Wmax <= 1) return k_prep<1, false>;
  if (Wmax <= 2) return k_prep<2, false>;
  if (Wmax <= 4) return k_prep<4, false>;
  if (Wmax <= 8) return k_prep<8, false>;
  return k_prep<16, false>;
}




// Resident CTAs per SM of a kernel for one launch shape on the current
// device, with its dynamic shared-memory limit raised to the request: both
// runtime queries are made once per (kernel, device, shape) and cached, so a
// launch costs no attribute or occupancy call after the first.
static int resident_ctas(const void* kern, int threads, size_t smem) {
  struct Entry {
    const void* kern;
    int dev, threads;
    size_t smem;
    int per_sm;
  };
  // a fixed table (no heap allocation on any launch path); when it is full
  // the queries are simply made every time
  constexpr int kEntries = 512;
  static std::mutex mu;
  static Entry cache[kEntries];
  static int used = 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  std::lock_guard<std::mutex> lock(mu);
  size_t most = smem;  // the attribute is a per-kernel maximum: never lower it
  for (int i = 0; i < used; ++i) {
    const Entry& e = cache[i];
    if (e.kern != kern || e.dev != dev) continue;
    if (e.threads == threads && e.smem == smem) return e.per_sm;
    if (e.smem > most) most = e.smem;
  }
  if (most > 48 * 1024 &&
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most) != cudaSuccess)
    return -1;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess) return -1;
  if (per_sm < 1) per_sm = 1;
  if (used < kEntries) cache[used++] = Entry{kern, dev, threads, smem, per_sm};
  return per_sm;
}

// Persistent launch of the search kernel: one wave of CTAs (as many as fit
// on every SM) pulling frames from the work queue. variant: register budget
// (4, 6 or 8 CTAs of 256 threads per SM; 0 = 4).
template <int B>
static int launch_search_t(const SearchArgs& s, int threads, size_t smem, cudaStream_t st) {
  const int per_sm = resident_ctas((const void*)k_search<B>, threads, smem);
  if (per_sm < 0) return GRAND_E_CUDA;
  k_search<B><<<search_grid(per_sm, 1, s.max_entries), threads, smem, st>>>(s);
  return cudaGetLastError() == cudaSuccess ? GRAND_OK : GRAND_E_CUDA;
}

// warps = 0: pair mode (CTAs of two warps sharing each frame); else CTAs of
// `warps` warps, one frame per warp.
template <int B>
static int launch_search_warp_t(const SearchArgs& s, int warps, cudaStream_t st) {
  const bool res = s.w_step > 0 || s.cur_in;
  const bool pair = warps == 0;
  const size_t smem = flip_slice_bytes(s.Wmax, s.sp_max) * (pair ? 1 : warps);
  auto kern = pair ? (res ? k_search_warp<B, true, true> : k_search_warp<B, false, true>)
                   : (res ? k_search_warp<B, true, false> : k_search_warp<B, false, false>);
  const int threads = pair ? 64 : 32 * warps;
  const int per_sm = resident_ctas((const void*)kern, threads, smem);
  if (per_sm < 0) return GRAND_E_CUDA;
  kern<<<search_grid(per_sm, pair ? 1 : warps, s.max_entries), threads, smem, st>>>(s);
  return cudaGetLastError() == cudaSuccess ? GRAND_OK : GRAND_E_CUDA;
}

template <int kSide>
static int launch_search_hash_t(const SearchArgs& s, int warps, cudaStream_t st) {
  const size_t hsmem = hash_slice_bytes<kSide>(s.Wmax) * warps;
  auto kern = (s.w_step > 0 || s.cur_in) ? k_search_hash<kSide, true> : k_search_hash<kSide, false>;
  const int per_sm = resident_ctas((const void*)kern, 32 * warps, hsmem);
  if (per_sm < 0) return GRAND_E_CUDA;
  kern<<<search_grid(per_sm, warps, s.max_entries), 32 * warps, hsmem, st>>>(s);
  return cudaGetLastError() == cudaSuccess ? GRAND_OK : GRAND_E_CUDA;
}

static int launch_search(const SearchArgs& s, int threads, size_t smem, int variant, cudaStream_t st) {
  // the warp-per-frame kernels are compiled for CTAs of at most 4 warps
  const int req_warps = s.warps > 4 ? 4 : s.warps;
  if (s.warp_kernel == 1 || s.warp_kernel == 2) {  // flip-bit warp search; warps per CTA from the tiles
    const int warps = req_warps > 0 ? req_warps : 0;   // automatic: warp pairs sharing a frame
    switch (variant) {  // default: 128 registers
      case 6: return launch_search_warp_t<6>(s, warps, st);
      case 8: return launch_search_warp_t<8>(s, warps, st);
      default: return launch_search_warp_t<4>(s, warps, st);
    }
  }
  if (s.warp_kernel == 3 || s.warp_kernel == 4) {  // hash join; warps per CTA from the tiles
    return s.warp_kernel == 3 ? launch_search_hash_t<kWarpSideMax>(s, req_warps > 0 ? req_warps : 4, st)
                              : launch_search_hash_t<kWarpSideMax + 1>(s, req_warps > 0 ? req_warps : 1, st);
  }
  switch (variant) {
    case 6: return launch_search_t<6>(s, threads, smem, st);
    case 8: return launch_search_t<8>(s, threads, smem, st);
    default: return launch_search_t<4>(s, threads, smem, st);
  }
}

// Load every kernel the symbol-level decode can launch (with lazy module
// loading a kernel is otherwise loaded at its first launch, which puts a
// one-time stall of milliseconds into the first batch that needs it).
int preload_qam_kernels() {
  const void* kernels[] = {
      (const void*)k_prep<1, false>, (const void*)k_prep<2, false>, (const void*)k_prep<4, false>,
      (const void*)k_prep<8, false>, (const void*)k_prep<16, false>, (const void*)k_prep<1, true>,
      (const void*)k_prep<2, true>, (const void*)k_prep<4, true>, (const void*)k_prep<8, true>,
      (const void*)k_prep<16, true>,
      (const void*)k_search_warp<4, false, false>, (const void*)k_search_warp<6, false, false>,
      (const void*)k_search_warp<8, false, false>, (const void*)k_search_warp<4, true, false>,
      (const void*)k_search_warp<6, true, false>, (const void*)k_search_warp<8, true, false>,
      (const void*)k_search_warp<4, false, true>, (const void*)k_search_warp<6, false, true>,
      (const void*)k_search_warp<8, false, true>, (const void*)k_search_warp<4, true, true>,
      (const void*)k_search_warp<6, true, true>, (const void*)k_search_warp<8, true, true>,
      (const void*)k_search_hash<kWarpSideMax, false>, (const void*)k_search_hash<kWarpSideMax + 1, false>,
      (const void*)k_search_hash<kWarpSideMax, true>, (const void*)k_search_hash<kWarpSideMax + 1, true>,
      (const void*)k_search<4>, (const void*)k_search<6>, (const void*)k_search<8>};
  for (const void* k : kernels) {
    cudaFuncAttributes attr;
    if (cudaFuncGetAttributes(&attr, k) != cudaSuccess) return GRAND_E_CUDA;
  }
  return GRAND_OK;
}

#define CU(x)                                   \
  do {                                          \
    if ((x) != cudaSuccess) return GRAND_E_CUDA; \
  } while (0)

// The search stage of a symbol-level decode (Alg. 2 Step 5 for the frames
// the preparation handed on): the kernel and its launch shape follow from the
// params and the call's largest S' and syndrome length. Every symbol-level
// call (direct, mixed, plans, the fixed-scratch variant) launches it here, so
// they run the same kernel for the same params.
// Options of a resumable search (weight windows and cursors; see SearchArgs).
struct ResumeOpt {
  int w_step = 0;
  FrameRec* cur_out = nullptr;
  const FrameRec* cur_in = nullptr;
  int64_t n_cur = 0;
  int64_t cw_stride = 0;
  int n_codes = 1;
  int64_t max_entries = 0;  // bound on the search queue (0: unknown)
};

static int launch_qam_search(const grand_params* p, int Smax, int w0, int Wmax, const CodeDev* d_codes,
                             const FrameRec* recs, Scratch* scr, uint32_t* cw, uint32_t* queries, uint8_t* abandon,
                             cudaStream_t st, const ResumeOpt& ro = ResumeOpt()) {
  if (Smax <= w0) return GRAND_OK;  // the preparation finished every frame
  SearchArgs s{};
  s.w_step = ro.w_step;
  s.cur_out = ro.cur_out;
  s.cur_in = ro.cur_in;
  s.n_cur = ro.n_cur;
  s.cw_stride = ro.cw_stride;
  s.n_codes = ro.n_codes;
  s.sp_max = Smax;
  s.max_entries = ro.cur_in ? ro.n_cur : ro.max_entries;
  s.recs = recs;
  s.codes = d_codes;
  s.scr = scr;
  s.cap = p->query_cap;
  s.split = p->tiles[1];
  // table capacities for the largest split the call can produce
  s.tabA = kTableMax;
  s.tabB = kTableMax;
  if (s.split <= 0) {
    s.tabA = 1 << (2 * (Smax / 2));
    s.tabB = 1 << (2 * (Smax - Smax / 2));
  }
  s.max_tiles = ((s.tabA + kTileRows - 1) / kTileRows) * ((s.tabB + kTileCols - 1) / kTileCols);
  s.Wmax = Wmax;
  // warp-per-frame flip-bit search (or the hash join with 5- or 6-rank
  // sides); an explicit split selects the CTA kernel
  s.warp_kernel = s.split > 0 ? 0 : (Smax <= 2 * kWarpSideMax ? 1 : 2);
  if (p->membership == GRAND_MEMBERSHIP_HASH && s.split <= 0) s.warp_kernel = Smax <= 2 * kWarpSideMax ? 3 : 4;
  s.warps = p->tiles[0] > 0 ? (p->tiles[0] > 8 ? 8 : p->tiles[0]) : 0;
  s.cw = cw;
  s.queries = queries;
  s.abandon = abandon;
  s.deadline = p->deadline_ns;
  const int threads = p->tiles[0] > 0 ? 32 * (p->tiles[0] > 8 ? 8 : p->tiles[0]) : 256;
  const size_t smem = search_smem_bytes(s.tabA, s.tabB, s.max_tiles, Wmax);
  NvtxRange r_search("grand.search");
  return launch_search(s, threads, smem, p->tiles[3], st);
}

// Common body of the symbol-level decode calls.
static int run_qam(const CodeDev* d_codes, int n_codes, int Lmax, int Wmax, const grand_params* p,
                   const PrepArgs& proto, int64_t n_frames, grand_stats* stats, cudaStream_t st,
                   const ResumeOpt& ro = ResumeOpt()) {
  if (n_frames == 0) {
    if (stats) *stats = grand_stats{};
    return GRAND_OK;
  }
  NvtxRange range("grand.decode");
  const int w0 = p->tiles[2] > 0 ? (p->tiles[2] > 3 ? 3 : p->tiles[2]) : 2;
  const int Smax = p->S < Lmax ? p->S : Lmax;
  // scratch: header + one record per frame (worst case: every frame hard)
  const size_t rec_bytes = sizeof(FrameRec) * (size_t)n_frames;
  char* scratch = nullptr;
  if (scratch_alloc((void**)&scratch, 256 + rec_bytes, st) != cudaSuccess) return GRAND_E_NOMEM;
  Scratch* scr = reinterpret_cast<Scratch*>(scratch);
  FrameRec* recs = reinterpret_cast<FrameRec*>(scratch + 256);
  int rc = GRAND_OK;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  do {
    if (cudaMemsetAsync(scr, 0, sizeof(Scratch), st) != cudaSuccess) { rc = GRAND_E_CUDA; break; }
    PrepArgs a = proto;
    a.nearer = p->order == GRAND_ORDER_QAM_NEARER ? 1 : 0;
    a.recs = recs;
    a.scr = scr;
    a.deadline = p->deadline_ns;
    a.Lmax = Lmax;
    a.Wmax = Wmax;
    const bool solve = p->membership == GRAND_MEMBERSHIP_SOLVE;
    a.w0 = solve ? 1 : w0;  // weights <= 1 filter the frames the elimination then solves
    const int warps = 4;
    const size_t prep_smem = prep_warp_bytes(Lmax, Wmax) * warps;
    const int64_t want = (n_frames + warps - 1) / warps;
    const int grid = (int)(want < (int64_t)sm_count() * 64 ? want : (int64_t)sm_count() * 64);
    auto kp = prep_kernel_for(Wmax, solve);
    if (prep_smem > 48 * 1024 && resident_ctas((const void*)kp, 32 * warps, prep_smem) < 0) {  // raises the limit
      rc = GRAND_E_CUDA;
      break;
    }
    if (stats) {
      for (int i = 0; i < 3; ++i)
        if (cudaEventCreate(&ev[i]) != cudaSuccess) { rc = GRAND_E_CUDA; break; }
      if (rc) break;
      cudaEventRecord(ev[0], st);
    }
    {
      NvtxRange r_prep("grand.prep");
      kp<<<grid, 32 * warps, prep_smem, st>>>(a);
    }
    if (stats) cudaEventRecord(ev[1], st);
    if (cudaGetLastError() != cudaSuccess) { rc = GRAND_E_CUDA; break; }

    ResumeOpt ro2 = ro;
    ro2.n_codes = n_codes;
    ro2.max_entries = n_frames;  // at most every frame is handed on
    // with the elimination, only frames whose solution set is too large to
    // rank are handed on (none on the measured workloads): one CTA per SM
    // keeps that launch short
    if (solve) ro2.max_entries = n_frames < (int64_t)sm_count() ? n_frames : (int64_t)sm_count();
    if (launch_qam_search(p, Smax, a.w0, Wmax, d_codes, recs, scr, proto.cw, proto.queries, proto.abandon, st, ro2) !=
        GRAND_OK) {
      rc = GRAND_E_CUDA;
      break;
    }
    if (stats) {
      cudaEventRecord(ev[2], st);
      Scratch h{};
      if (cudaMemcpyAsync(&h, scr, sizeof(Scratch), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess) {
        rc = GRAND_E_CUDA;
        break;
      }
      stats->evaluated_checks = h.evaluated;
      stats->hard_frames = h.n_hard;
      stats->search_useful = h.search_useful;
      cudaEventElapsedTime(&stats->prep_ms, ev[0], ev[1]);
      cudaEventElapsedTime(&stats->search_ms, ev[1], ev[2]);
    }
  } while (0);
  for (int i = 0; i < 3; ++i)
    if (ev[i]) cudaEventDestroy(ev[i]);
  cudaFreeAsync(scratch, st);
  return rc;
}

static int check_params(const grand_params* p) {
  if (!p) return GRAND_E_INVALID;
  if (p->query_cap < 1 || p->deadline_ns < 0) return GRAND_E_INVALID;
  if (p->lik_variant != GRAND_LIK_THRESHOLD && p->lik_variant != GRAND_LIK_LITERAL) return GRAND_E_INVALID;
  if (p->membership < GRAND_MEMBERSHIP_AUTO || p->membership > GRAND_MEMBERSHIP_SOLVE ||
      p->membership == GRAND_MEMBERSHIP_FASTEST)
    return GRAND_E_INVALID;
  if (p->order == GRAND_ORDER_QAM_NNE5 &&
      (p->membership == GRAND_MEMBERSHIP_HASH || p->membership == GRAND_MEMBERSHIP_SOLVE))
    return GRAND_E_UNSUPPORTED;
  // the bit-level TEP set (weights <= max_weight) is not a coordinate space
  if (p->order == GRAND_ORDER_HAMMING && p->membership == GRAND_MEMBERSHIP_SOLVE) return GRAND_E_UNSUPPORTED;
  if (p->order == GRAND_ORDER_QAM_NNE || p->order == GRAND_ORDER_QAM_NEARER || p->order == GRAND_ORDER_QAM_NNE5) {
    if (p->S < 0) return GRAND_E_INVALID;
    if (p->S > (p->order == GRAND_ORDER_QAM_NNE5 ? GRAND_S_MAX_NNE5 : kSMax)) return GRAND_E_UNSUPPORTED;
  } else if (p->order == GRAND_ORDER_HAMMING) {
    if (p->max_weight < 0) return GRAND_E_INVALID;
    if (p->max_weight > GRAND_AB_WEIGHT_MAX) return GRAND_E_UNSUPPORTED;
  } else {
    return GRAND_E_INVALID;
  }
  for (int i = 0; i < 4; ++i)
    if (p->tiles[i] < 0) return GRAND_E_INVALID;
  return GRAND_OK;
}

static int run_ab(const grand_code* c, const grand_params* p, const float* samples, const uint32_t* y,
                  const uint8_t* nmask, int64_t n_frames, uint32_t* cw, uint32_t* queries, uint8_t* abandon,
                  grand_stats* stats, cudaStream_t st) {
  // positions must fit the 32-bit query counter
  uint64_t total = 0;
  for (int w = 0; w <= p->max_weight; ++w) {
    uint64_t b = 1;
    for (int i = 1; i <= w; ++i) b = b * (uint64_t)(c->N - w + i) / (uint64_t)i;
    total += b;
  }
  if ((total < (uint64_t)p->query_cap ? total : (uint64_t)p->query_cap) > 0xFFFFFFFFull) return GRAND_E_UNSUPPORTED;
  if (n_frames == 0) {
    if (stats) *stats = grand_stats{};
    return GRAND_OK;
  }
  // the counters (statistics) and the deadline's clock stamp are the only
  // scratch of the bit-level search: without either, none is allocated
  Scratch* scr = nullptr;
  const bool need_scr = stats != nullptr || p->deadline_ns > 0;
  if (need_scr && scratch_alloc((void**)&scr, sizeof(Scratch), st) != cudaSuccess) return GRAND_E_NOMEM;
  int rc = GRAND_OK;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  do {
    if (need_scr && cudaMemsetAsync(scr, 0, sizeof(Scratch), st) != cudaSuccess) { rc = GRAND_E_CUDA; break; }
    if (stats) {
      if (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess) { rc = GRAND_E_CUDA; break; }
      cudaEventRecord(ev[0], st);
    }
    AbArgs a{};
    a.samples = samples;
    a.y_in = y;
    a.nmask = nmask;
    a.code = c->dev;
    a.n_frames = n_frames;
    a.max_weight = p->max_weight;
    a.cap = p->query_cap;
    a.cw = cw;
    a.queries = queries;
    a.abandon = abandon;
    a.scr = scr;
    a.deadline = p->deadline_ns;
    const int64_t want = (n_frames + 3) / 4;
    if (p->max_weight <= 3 && c->W == 1 && (c->N == 32 || c->N == 64)) {
      // pair x single split with the columns as bit-planes in registers
      const int grid = (int)(want < (int64_t)sm_count() * 16 ? want : (int64_t)sm_count() * 16);
      if (c->N == 32) {
        if (c->R <= 16) k_ab_split<1, 16><<<grid, 128, 0, st>>>(a);
        else k_ab_split<1, 32><<<grid, 128, 0, st>>>(a);
      } else {
        if (c->R <= 16) k_ab_split<2, 16><<<grid, 128, 0, st>>>(a);
        else k_ab_split<2, 32><<<grid, 128, 0, st>>>(a);
      }
    } else {
      const int grid = (int)(want < (int64_t)sm_count() * 64 ? want : (int64_t)sm_count() * 64);
      k_ab<<<grid, 128, 0, st>>>(a);
    }
    if (cudaGetLastError() != cudaSuccess) { rc = GRAND_E_CUDA; break; }
    if (stats) {
      cudaEventRecord(ev[1], st);
      Scratch h{};
      if (cudaMemcpyAsync(&h, scr, sizeof(Scratch), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess) {
        rc = GRAND_E_CUDA;
        break;
      }
      stats->evaluated_checks = h.evaluated;
      stats->hard_frames = 0;
      stats->search_useful = 0;
      stats->prep_ms = 0.0f;
      cudaEventElapsedTime(&stats->search_ms, ev[0], ev[1]);  // the one search kernel
    }
  } while (0);
  for (int i = 0; i < 2; ++i)
    if (ev[i]) cudaEventDestroy(ev[i]);
  if (scr) cudaFreeAsync(scr, st);
  return rc;
}

}  // namespace grand

using namespace grand;

extern "C" int grand_demod(const void* symbols, int64_t n_frames, int L, int M, float N0, int lik_variant,
                           uint16_t* hard_idx, uint32_t* key, uint8_t* nmask, float* rel, uint32_t* y, int N,
                           void* stream) {
  if ((!symbols && n_frames > 0) || n_frames < 0 || !(N0 > 0.0f) || !isfinite(N0)) return GRAND_E_INVALID;
  if (N < GRAND_N_MIN || N > GRAND_N_MAX || (N & (N - 1))) return GRAND_E_INVALID;
  if (lik_variant != GRAND_LIK_THRESHOLD && lik_variant != GRAND_LIK_LITERAL) return GRAND_E_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  if (M == 2) {
    if (L != N) return GRAND_E_INVALID;
    if (n_frames == 0) return GRAND_OK;
    const int64_t n_words = n_frames * (N / 32);
    const int64_t blocks = (n_words * 32 + 255) / 256;
    k_demod_bpsk<<<(int)(blocks < 65535 * 8 ? blocks : 65535 * 8), 256, 0, st>>>((const float*)symbols, n_words, y,
                                                                                  nmask);
    return cudaGetLastError() == cudaSuccess ? GRAND_OK : GRAND_E_CUDA;
  }
  const int m = m_of(M);
  if (!m || L != (N + 2 * m - 1) / (2 * m)) return GRAND_E_INVALID;
  if (n_frames == 0) return GRAND_OK;
  const QamConst qc = make_qam_const();
  DemodArgs a{};
  a.symbols = (const float2*)symbols;
  a.n_sym = n_frames * L;
  a.L = L;
  a.m = m;
  a.side = 1 << m;
  a.N = N;
  a.NW = N / 32;
  a.lik = lik_variant;
  a.q = qc.q[m];
  a.inv_d = qc.inv_d[m];
  a.hard_idx = hard_idx;
  a.key = key;
  a.nmask = nmask;
  a.rel = rel;
  a.y = y;
  a.Lmagic = UINT64_MAX / (uint64_t)L + 1;  // L >= 3 for the supported N and M
  if (y && cudaMemsetAsync(y, 0, sizeof(uint32_t) * (size_t)n_frames * (N / 32), st) != cudaSuccess)
    return GRAND_E_CUDA;
  auto aligned = [](const void* p, uintptr_t b) { return ((uintptr_t)p % b) == 0; };
  const bool paired = aligned(a.symbols, 16) && aligned(a.hard_idx, 4) && aligned(a.key, 8) &&
                      aligned(a.nmask, 2) && aligned(a.rel, 8);
  const int64_t per_thread = paired ? 2 : 1;
  const int64_t blocks = ((a.n_sym + per_thread - 1) / per_thread + 255) / 256;
  const int grid = (int)(blocks < (int64_t)sm_count() * 32 ? blocks : (int64_t)sm_count() * 32);
  launch_demod(a, paired, grid, st);
  return cudaGetLastError() == cudaSuccess ? GRAND_OK : GRAND_E_CUDA;
}

extern "C" int grand_decode_batch(const grand_code* c, const grand_params* p, const uint16_t* hard_idx,
                                  const uint32_t* key, const uint8_t* nmask, const uint32_t* y, int64_t n_frames,
                                  uint32_t* cw, uint32_t* queries, uint8_t* abandon, grand_stats* stats,
                                  void* stream) {
  if (!c || n_frames < 0 || (n_frames > 0 && (!cw || !queries || !abandon || !y))) return GRAND_E_INVALID;
  int rc = check_params(p);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if (p->order == GRAND_ORDER_HAMMING) return run_ab(c, p, nullptr, y, nmask, n_frames, cw, queries, abandon, stats, st);
  if (p->order == GRAND_ORDER_QAM_NNE5 || p->membership == GRAND_MEMBERSHIP_DELTA ||
      p->membership == GRAND_MEMBERSHIP_ROW_PARITY)
    return GRAND_E_UNSUPPORTED;
  const int m = m_of(p->M);
  if (!m || (n_frames > 0 && (!hard_idx || !key || !nmask))) return GRAND_E_INVALID;
  if (n_frames > 0xFFFFFFFFll) return GRAND_E_UNSUPPORTED;
  const int L = (c->N + 2 * m - 1) / (2 * m);
  PrepArgs a{};
  a.hard_idx = hard_idx;
  a.key = key;
  a.nmask = nmask;
  a.y_in = y;
  a.codes = c->d_dev;
  a.n_codes = 1;
  a.n_frames = n_frames;
  a.M = p->M;
  a.S = p->S;
  a.lik = p->lik_variant;
  a.cap = p->query_cap;
  a.qc = make_qam_const();
  a.cw = cw;
  a.queries = queries;
  a.abandon = abandon;
  return run_qam(c->d_dev, 1, L, c->W, p, a, n_frames, stats, st);
}

extern "C" int grand_decode_symbols(const grand_code* c, const grand_params* p, const void* symbols, int64_t n_frames,
                                    float N0, uint32_t* cw, uint32_t* queries, uint8_t* abandon, grand_stats* stats,
                                    void* stream) {
  if (!c || n_frames < 0 || (n_frames > 0 && (!symbols || !cw || !queries || !abandon))) return GRAND_E_INVALID;
  if (!(N0 > 0.0f) || !isfinite(N0)) return GRAND_E_INVALID;
  int rc = check_params(p);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if (p->order == GRAND_ORDER_HAMMING) {
    if (p->M != 2) return GRAND_E_INVALID;
    return run_ab(c, p, (const float*)symbols, nullptr, nullptr, n_frames, cw, queries, abandon, stats, st);
  }
  const int m = m_of(p->M);
  if (!m) return GRAND_E_INVALID;
  if (n_frames > 0xFFFFFFFFll) return GRAND_E_UNSUPPORTED;
  if (p->order == GRAND_ORDER_QAM_NNE5 || p->membership == GRAND_MEMBERSHIP_DELTA ||
      p->membership == GRAND_MEMBERSHIP_ROW_PARITY)
    return run_per_tep(c, p, symbols, n_frames, cw, queries, abandon, stats, st);
  const int L = (c->N + 2 * m - 1) / (2 * m);
  PrepArgs a{};
  a.symbols = (const float2*)symbols;
  a.codes = c->d_dev;
  a.n_codes = 1;
  a.n_frames = n_frames;
  a.M = p->M;
  a.S = p->S;
  a.lik = p->lik_variant;
  a.cap = p->query_cap;
  a.qc = make_qam_const();
  a.cw = cw;
  a.queries = queries;
  a.abandon = abandon;
  return run_qam(c->d_dev, 1, L, c->W, p, a, n_frames, stats, st);
}

namespace grand {

// Checks shared by the resumable calls: the split search (automatic split) of
// the symbol-level orders, with a membership test that supports weight windows.
static int check_resumable(const grand_params* p) {
  int rc = check_params(p);
  if (rc) return rc;
  if (p->order != GRAND_ORDER_QAM_NNE && p->order != GRAND_ORDER_QAM_NEARER) return GRAND_E_UNSUPPORTED;
  if (p->membership != GRAND_MEMBERSHIP_AUTO && p->membership != GRAND_MEMBERSHIP_HASH) return GRAND_E_UNSUPPORTED;
  if (p->tiles[1] > 0) return GRAND_E_UNSUPPORTED;  // the CTA-per-frame search has no weight windows
  return GRAND_OK;
}

}  // namespace grand

extern "C" int grand_decode_symbols_resumable(const grand_code* c, const grand_params* p, const void* symbols,
                                              int64_t n_frames, float N0, int32_t weight_step, void* cursors,
                                              uint32_t* cw, uint32_t* queries, uint8_t* abandon, void* stream) {
  using namespace grand;
  static_assert(sizeof(FrameRec) == GRAND_CURSOR_BYTES, "cursor size");
  if (!c || n_frames < 0 || (n_frames > 0 && (!symbols || !cw || !queries || !abandon || !cursors)))
    return GRAND_E_INVALID;
  if (!(N0 > 0.0f) || !isfinite(N0) || weight_step < 1) return GRAND_E_INVALID;
  int rc = check_resumable(p);
  if (rc) return rc;
  const int m = m_of(p->M);
  if (!m) return GRAND_E_INVALID;
  if (n_frames > 0xFFFFFFFFll) return GRAND_E_UNSUPPORTED;
  const int L = (c->N + 2 * m - 1) / (2 * m);
  PrepArgs a{};
  a.symbols = (const float2*)symbols;
  a.codes = c->d_dev;
  a.n_codes = 1;
  a.n_frames = n_frames;
  a.M = p->M;
  a.S = p->S;
  a.lik = p->lik_variant;
  a.cap = p->query_cap;
  a.qc = make_qam_const();
  a.cw = cw;
  a.queries = queries;
  a.abandon = abandon;
  ResumeOpt ro;
  ro.w_step = weight_step;
  ro.cur_out = static_cast<FrameRec*>(cursors);
  return run_qam(c->d_dev, 1, L, c->W, p, a, n_frames, nullptr, (cudaStream_t)stream, ro);
}

extern "C" int grand_decode_resume(const grand_code* c, const grand_params* p, void* cursors, int64_t n,
                                   int32_t weight_step, uint32_t* cw, int64_t cw_stride_words, uint32_t* queries,
                                   uint8_t* abandon, void* stream) {
  using namespace grand;
  if (!c || n < 0 || (n > 0 && (!cursors || !cw || !queries || !abandon))) return GRAND_E_INVALID;
  if (weight_step < 0 || cw_stride_words < c->N / 32) return GRAND_E_INVALID;
  int rc = check_resumable(p);
  if (rc) return rc;
  if (n > 0xFFFFFFFFll) return GRAND_E_UNSUPPORTED;
  return resume_resident(c->d_dev, 1, c->W, p, static_cast<FrameRec*>(cursors), n, weight_step, cw,
                         cw_stride_words, queries, abandon, (cudaStream_t)stream);
}

namespace grand {

// Code table of an uneven batch: device views plus the batch-wide bounds.
static int code_table(const grand_code* const* codes, int n_codes, std::vector<CodeDev>& table, int& Lmax, int& Wmax) {
  Wmax = 1;
  Lmax = 1;
  table.resize(n_codes);
  for (int i = 0; i < n_codes; ++i) {
    if (!codes[i]) return GRAND_E_INVALID;
    table[i] = codes[i]->dev;
    Wmax = table[i].W > Wmax ? table[i].W : Wmax;
    const int L = (table[i].N + 1) / 2;  // QPSK bound
    Lmax = L > Lmax ? L : Lmax;
  }
  return GRAND_OK;
}

static int check_mixed_args(const grand_code* const* codes, int n_codes, const grand_params* p,
                            const grand_frame_desc* desc, int64_t n_frames, const void* symbols, int64_t n_symbols,
                            float N0, uint32_t* cw, int64_t n_cw_words, uint32_t* queries, uint8_t* abandon) {
  if (!codes || n_codes < 1 || n_codes > 65535 || n_frames < 0 || n_symbols < 0 || n_cw_words < 0 ||
      (n_frames > 0 && (!desc || !symbols || !cw || !queries || !abandon)))
    return GRAND_E_INVALID;
  if (!(N0 > 0.0f) || !isfinite(N0)) return GRAND_E_INVALID;
  int rc = check_params(p);
  if (rc) return rc;
  if ((p->order != GRAND_ORDER_QAM_NNE && p->order != GRAND_ORDER_QAM_NEARER) ||
      (p->membership != GRAND_MEMBERSHIP_AUTO && p->membership != GRAND_MEMBERSHIP_HASH &&
       p->membership != GRAND_MEMBERSHIP_SOLVE))
    return GRAND_E_INVALID;
  if (n_frames > 0xFFFFFFFFll) return GRAND_E_UNSUPPORTED;
  return GRAND_OK;
}

// The uneven-batch launch sequence on a device-resident code table.
static int mixed_impl(const CodeDev* d_table, int n_codes, int Lmax, int Wmax, const grand_params* p,
                      const grand_frame_desc* desc, int64_t n_frames, const void* symbols, int64_t n_symbols,
                      uint32_t* cw, int64_t n_cw_words, uint32_t* queries, uint8_t* abandon, grand_stats* stats,
                      cudaStream_t st, const ResumeOpt& ro = ResumeOpt()) {
  PrepArgs a{};
  a.symbols = (const float2*)symbols;
  a.desc = desc;
  a.n_symbols = n_symbols;
  a.n_cw_words = n_cw_words;
  a.codes = d_table;
  a.n_codes = n_codes;
  a.n_frames = n_frames;
  a.M = 0;
  a.S = p->S;
  a.lik = p->lik_variant;
  a.cap = p->query_cap;
  a.qc = make_qam_const();
  a.cw = cw;
  a.queries = queries;
  a.abandon = abandon;
  return run_qam(d_table, n_codes, Lmax, Wmax, p, a, n_frames, stats, st, ro);
}

int decode_mixed_resident(const CodeDev* d_table, int n_codes, int Lmax, int Wmax, const grand_params* p,
                          const grand_frame_desc* desc, int64_t n_frames, const void* symbols, int64_t n_symbols,
                          uint32_t* cw, int64_t n_cw_words, uint32_t* queries, uint8_t* abandon, cudaStream_t st,
                          int w_step, FrameRec* cursors) {
  ResumeOpt ro;
  ro.w_step = w_step;
  ro.cur_out = cursors;
  return mixed_impl(d_table, n_codes, Lmax, Wmax, p, desc, n_frames, symbols, n_symbols, cw, n_cw_words, queries,
                    abandon, nullptr, st, ro);
}

// The search over suspended cursors (grand_decode_resume, the serving loop's
// long frames): one search launch with cursor i's outputs at index i.
int resume_resident(const CodeDev* d_table, int n_codes, int Wmax, const grand_params* p, FrameRec* cursors,
                    int64_t n, int w_step, uint32_t* cw, int64_t cw_stride, uint32_t* queries, uint8_t* abandon,
                    cudaStream_t st) {
  if (n == 0) return GRAND_OK;
  Scratch* scr = nullptr;
  if (scratch_alloc((void**)&scr, sizeof(Scratch), st) != cudaSuccess) return GRAND_E_NOMEM;
  int rc = GRAND_OK;
  if (cudaMemsetAsync(scr, 0, sizeof(Scratch), st) != cudaSuccess) rc = GRAND_E_CUDA;
  if (rc == GRAND_OK) {
    ResumeOpt ro;
    ro.w_step = w_step;
    ro.cur_out = cursors;
    ro.cur_in = cursors;
    ro.n_cur = n;
    ro.cw_stride = cw_stride;
    ro.n_codes = n_codes;
    const int Smax = p->S < kSMax ? p->S : kSMax;
    // w0 = 0: every cursor goes to the search (the preparation is not run)
    NvtxRange range("grand.resume");
    if (launch_qam_search(p, Smax, 0, Wmax, d_table, nullptr, scr, cw, queries, abandon, st, ro) != GRAND_OK)
      rc = GRAND_E_CUDA;
  }
  cudaFreeAsync(scr, st);
  return rc;
}

}  // namespace grand

extern "C" int grand_decode_mixed(const grand_code* const* codes, int n_codes, const grand_params* p,
                                  const grand_frame_desc* desc, int64_t n_frames, const void* symbols,
                                  int64_t n_symbols, float N0, uint32_t* cw, int64_t n_cw_words, uint32_t* queries,
                                  uint8_t* abandon, grand_stats* stats, void* stream) {
  int rc = check_mixed_args(codes, n_codes, p, desc, n_frames, symbols, n_symbols, N0, cw, n_cw_words, queries,
                            abandon);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  int Wmax = 1, Lmax = 1;
  std::vector<CodeDev> table;
  rc = code_table(codes, n_codes, table, Lmax, Wmax);
  if (rc) return rc;
  CodeDev* d_table = nullptr;
  if (scratch_alloc((void**)&d_table, sizeof(CodeDev) * n_codes, st) != cudaSuccess) return GRAND_E_NOMEM;
  // pageable source: the copy is staged before the call returns
  if (cudaMemcpyAsync(d_table, table.data(), sizeof(CodeDev) * n_codes, cudaMemcpyHostToDevice, st) != cudaSuccess) {
    cudaFreeAsync(d_table, st);
    return GRAND_E_CUDA;
  }
  rc = mixed_impl(d_table, n_codes, Lmax, Wmax, p, desc, n_frames, symbols, n_symbols, cw, n_cw_words, queries,
                  abandon, stats, st);
  // the table must outlive the kernels: stream-ordered free
  cudaFreeAsync(d_table, st);
  return rc;
}

// ---------------------------------------------------------------------------
// Plans: one decode call captured into a CUDA graph for repeated launches on
// fixed buffers (the launch sequence -- counter reset, preparation, search,
// with the stream-ordered scratch as graph memory nodes -- replays with one
// cudaGraphLaunch).
// ---------------------------------------------------------------------------
struct grand_plan {
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  grand::CodeDev* d_table;  // uneven batches: code table owned by the plan
};

namespace grand {

template <typename F>
static int capture_plan(F&& body, grand_plan** out) {
  cudaStream_t cap = nullptr;
  if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return GRAND_E_CUDA;
  int rc = body(cap);  // one eager run: module load, attributes, pool warm-up
  if (rc == GRAND_OK && cudaStreamSynchronize(cap) != cudaSuccess) rc = GRAND_E_CUDA;
  grand_plan* plan = nullptr;
  if (rc == GRAND_OK) {
    plan = (grand_plan*)calloc(1, sizeof(grand_plan));
    if (!plan) rc = GRAND_E_NOMEM;
  }
  if (rc == GRAND_OK) {
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      rc = GRAND_E_CUDA;
    } else {
      const int brc = body(cap);
      cudaGraph_t g = nullptr;
      const cudaError_t e = cudaStreamEndCapture(cap, &g);
      if (brc != GRAND_OK || e != cudaSuccess || !g) {
        rc = brc != GRAND_OK ? brc : GRAND_E_CUDA;
        if (g) cudaGraphDestroy(g);
      } else {
        plan->graph = g;
        if (cudaGraphInstantiate(&plan->exec, g, 0) != cudaSuccess) rc = GRAND_E_CUDA;
      }
    }
  }
  cudaStreamDestroy(cap);
  if (rc != GRAND_OK) {
    if (plan) {
      if (plan->exec) cudaGraphExecDestroy(plan->exec);
      if (plan->graph) cudaGraphDestroy(plan->graph);
      free(plan);
    }
    return rc;
  }
  *out = plan;
  return GRAND_OK;
}

}  // namespace grand

extern "C" int grand_plan_symbols(const grand_code* c, const grand_params* p, const void* symbols, int64_t n_frames,
                                  float N0, uint32_t* cw, uint32_t* queries, uint8_t* abandon, grand_plan** out) {
  if (!out || n_frames < 1) return GRAND_E_INVALID;
  *out = nullptr;
  return capture_plan(
      [&](cudaStream_t st) {
        return grand_decode_symbols(c, p, symbols, n_frames, N0, cw, queries, abandon, nullptr, st);
      },
      out);
}

extern "C" int grand_plan_mixed(const grand_code* const* codes, int n_codes, const grand_params* p,
                                const grand_frame_desc* desc, int64_t n_frames, const void* symbols, int64_t n_symbols,
                                float N0, uint32_t* cw, int64_t n_cw_words, uint32_t* queries, uint8_t* abandon,
                                grand_plan** out) {
  if (!out || n_frames < 1) return GRAND_E_INVALID;
  *out = nullptr;
  int rc = check_mixed_args(codes, n_codes, p, desc, n_frames, symbols, n_symbols, N0, cw, n_cw_words, queries,
                            abandon);
  if (rc) return rc;
  int Wmax = 1, Lmax = 1;
  std::vector<CodeDev> table;
  rc = code_table(codes, n_codes, table, Lmax, Wmax);
  if (rc) return rc;
  CodeDev* d_table = nullptr;
  if (cudaMalloc((void**)&d_table, sizeof(CodeDev) * n_codes) != cudaSuccess) return GRAND_E_NOMEM;
  if (cudaMemcpy(d_table, table.data(), sizeof(CodeDev) * n_codes, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(d_table);
    return GRAND_E_CUDA;
  }
  rc = capture_plan(
      [&](cudaStream_t st) {
        return mixed_impl(d_table, n_codes, Lmax, Wmax, p, desc, n_frames, symbols, n_symbols, cw, n_cw_words,
                          queries, abandon, nullptr, st);
      },
      out);
  if (rc != GRAND_OK) {
    cudaFree(d_table);
    return rc;
  }
  (*out)->d_table = d_table;
  return GRAND_OK;
}

extern "C" int grand_plan_launch(grand_plan* plan, void* stream) {
  if (!plan || !plan->exec) return GRAND_E_INVALID;
  return cudaGraphLaunch(plan->exec, (cudaStream_t)stream) == cudaSuccess ? GRAND_OK : GRAND_E_CUDA;
}

extern "C" int grand_plan_destroy(grand_plan* plan) {
  if (!plan) return GRAND_OK;
  if (plan->exec) cudaGraphExecDestroy(plan->exec);
  if (plan->graph) cudaGraphDestroy(plan->graph);
  if (plan->d_table) cudaFree(plan->d_table);
  free(plan);
  return GRAND_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of grand_decode_symbols.
//
// The regular call takes its scratch (a header plus one hand-off record per
// frame between the preparation and the search kernel) from the library's
// stream-ordered pool.
// This variant takes it from one fixed array in device memory instead, so a
// caller that must not allocate after start-up can still decode. The array is
// part of the library's device code: every GPU that loads the library holds
// it (kNoAllocScratchBytes, about 2.4 MB) until the process exits.
// ---------------------------------------------------------------------------
namespace grand {

constexpr int64_t kNoAllocMaxFrames = GRAND_NOALLOC_MAX_FRAMES;
constexpr size_t kNoAllocHeader = 256;
constexpr size_t kNoAllocScratchBytes = kNoAllocHeader + sizeof(FrameRec) * (size_t)kNoAllocMaxFrames;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kNoAllocMaxDevices = 64;
static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[kNoAllocMaxDevices];

// Device address of the array on the current device. In host code the name
// g_noalloc_scratch is only a host-side handle, so the address is looked up
// once per device (with that device current) and cached.
static int noalloc_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GRAND_E_CUDA;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return GRAND_E_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return GRAND_E_CUDA;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return GRAND_OK;
}

}  // namespace grand

extern "C" int grand_decode_symbols_noalloc(const grand_code* c, const grand_params* p, const void* symbols,
                                            int64_t n_frames, float N0, uint32_t* cw, uint32_t* queries,
                                            uint8_t* abandon, void* stream) {
  if (!c || n_frames < 0 || (n_frames > 0 && (!symbols || !cw || !queries || !abandon))) return GRAND_E_INVALID;
  if (!(N0 > 0.0f) || !isfinite(N0)) return GRAND_E_INVALID;
  int rc = check_params(p);
  if (rc) return rc;
  if (p->order != GRAND_ORDER_QAM_NNE || p->membership != GRAND_MEMBERSHIP_AUTO) return GRAND_E_INVALID;
  const int m = m_of(p->M);
  if (!m) return GRAND_E_INVALID;
  if (n_frames > kNoAllocMaxFrames) return GRAND_E_UNSUPPORTED;
  void* base = nullptr;
  rc = noalloc_scratch(&base);  // first call on a device: symbol lookup
  if (rc) return rc;
  if (n_frames == 0) return GRAND_OK;
  cudaStream_t st = (cudaStream_t)stream;
  Scratch* scr = reinterpret_cast<Scratch*>(base);
  FrameRec* recs = reinterpret_cast<FrameRec*>(static_cast<char*>(base) + kNoAllocHeader);
  // the array keeps the previous call's contents: reset the counters
  if (cudaMemsetAsync(scr, 0, sizeof(Scratch), st) != cudaSuccess) return GRAND_E_CUDA;
  const int L = (c->N + 2 * m - 1) / (2 * m);
  PrepArgs a{};
  a.symbols = (const float2*)symbols;
  a.codes = c->d_dev;
  a.n_codes = 1;
  a.n_frames = n_frames;
  a.M = p->M;
  a.S = p->S;
  a.lik = p->lik_variant;
  a.cap = p->query_cap;
  a.qc = make_qam_const();
  a.cw = cw;
  a.queries = queries;
  a.abandon = abandon;
  a.recs = recs;
  a.scr = scr;
  a.deadline = p->deadline_ns;
  a.Lmax = L;
  a.Wmax = c->W;
  a.w0 = p->tiles[2] > 0 ? (p->tiles[2] > 3 ? 3 : p->tiles[2]) : 2;
  const int warps = 4;
  const size_t prep_smem = prep_warp_bytes(L, c->W) * warps;
  auto kp = prep_kernel_for(c->W);
  if (prep_smem > 48 * 1024 && resident_ctas((const void*)kp, 32 * warps, prep_smem) < 0) return GRAND_E_CUDA;
  const int64_t want = (n_frames + warps - 1) / warps;
  const int grid = (int)(want < (int64_t)sm_count() * 64 ? want : (int64_t)sm_count() * 64);
  kp<<<grid, 32 * warps, prep_smem, st>>>(a);
  if (cudaGetLastError() != cudaSuccess) return GRAND_E_CUDA;
  const int Smax = p->S < L ? p->S : L;
  if (launch_qam_search(p, Smax, a.w0, c->W, c->d_dev, recs, scr, cw, queries, abandon, st) != GRAND_OK)
    return GRAND_E_CUDA;
  return GRAND_OK;
}
