/*
 * grand_oracle.c -- plain, slow CPU reference of GRAND with the M-QAM likelihood
 * order of arXiv 2405.01808 ("GRAND Massive Parallel Decoding Framework for Low
 * Latency in Beyond 5G").
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library. The decoding library
 * (the CUDA path) shares no code, header, table or helper with it.
 *
 * Everything here is written for obviousness, not speed:
 *   - the code is built from the Kronecker definition (Def. II.1) and the
 *     Bhattacharyya recursion,
 *   - every received symbol is demodulated per Def. III.1 / III.2,
 *   - test error patterns are enumerated one at a time in the canonical order,
 *   - every query recomputes the full syndrome H (y xor e) by a dense GF(2)
 *     matrix-vector product (Alg. 2, Step 5) -- no incremental syndromes.
 *
 * Readings of the paper (it is silent or ambiguous on these; each is also
 * listed in the project's design notes):
 *   R1 distance to the decision threshold (Def. III.1): in Q8.8 units of the
 *      odd-integer lattice, d = 256 - |256 A - a_q| when the received value lies
 *      on the constellation side of its hard point, d = 256 + |256 A - a_q|
 *      when it lies outside the outermost level (no neighbour that way).
 *      The LITERAL variant always uses 256 - |256 A - a_q|, clamped at 0.
 *   R2 neighbour direction (Def. III.2): -Sign(A - a); on a tie (A == a) the
 *      direction is toward the lower level, except at the lowest level where
 *      it is upward. A neighbour exists iff its level is on the constellation.
 *      The diagonal exists iff both the horizontal and vertical ones do.
 *   R3 canonical TEP order over the S' = min(S, L) least reliable symbols
 *      (Alg. 2 Steps 2-5): by number of altered symbols w, then the colex
 *      order of the altered rank set, then the alternatives read as a base-3
 *      number whose least significant digit is the smallest altered rank
 *      (h = 0, v = 1, diag = 2). Invalid TEPs (an alternative that does not
 *      exist) are skipped and not counted.
 *   R4 queries = 1-based position of the first hit among valid TEPs. When no
 *      hit occurs within the first `cap` valid TEPs, or the valid TEPs run
 *      out, the output is the hard word, queries = min(cap, #valid) and
 *      abandon = 1. A frame with a non-finite received value is not searched:
 *      abandon = 2, queries = 0, output = hard word (its non-finite
 *      coordinates read as 0).
 *   R5 bit-level GRAND-AB (Sec. I): hard bit = [r < 0]; TEPs are the bit sets
 *      of weight 0..max_weight in (weight, colex) order over bit indices.
 *   R6 order variant "nearer axis first": as R3, but the horizontal and
 *      vertical alternatives of a symbol swap places when the vertical
 *      distance to the threshold is strictly smaller (d_Q < d_I), so the
 *      single-axis alternative of the less reliable axis is queried first.
 *   R7 order variant "five-point NNE" (the nearest-neighbour error channel
 *      the paper compares against in Sec. II): up to four alternatives per
 *      symbol, the neighbouring levels on either side of each axis (toward
 *      the received point on I, toward it on Q, away from it on I, away on
 *      Q, in that order), no diagonal; a neighbour exists iff its level is
 *      on the constellation. Symbols are sorted by the same key, and the
 *      TEPs follow R3 with base-4 alternative digits.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_MAX_S 16
#define ORACLE_MAX_N 1024

/* ------------------------------------------------------------------------- */
/* Code construction (Def. II.1)                                              */
/* ------------------------------------------------------------------------- */

/* G_N = F^{(x)n} with F = [[1,0],[1,1]], built by repeated Kronecker products:
 * G_{2k} = [[G_k, 0], [G_k, G_k]]. G is N*N bytes, row-major. */
void oracle_polar_G(int N, uint8_t* G) {
  memset(G, 0, (size_t)N * N);
  G[0] = 1;
  for (int k = 1; k < N; k *= 2) {
    for (int i = 0; i < k; ++i) {
      for (int j = 0; j < k; ++j) {
        uint8_t g = G[(size_t)i * N + j];
        /* F[1][0] = 1: lower-left block */
        G[(size_t)(i + k) * N + j] = g;
        /* F[1][1] = 1: lower-right block */
        G[(size_t)(i + k) * N + (j + k)] = g;
        /* F[0][1] = 0: upper-right block stays zero */
      }
    }
  }
}

/* Bhattacharyya parameters of the N synthetic channels (Arikan's construction,
 * cited in Sec. II): start from z = exp(-R * 10^(snr_db/10)) and apply the
 * binary-erasure recursion n times; index 2t takes 2z - z^2, index 2t+1 takes
 * z^2. */
void oracle_bhattacharyya(int N, double rate, double design_snr_db, double* z) {
  double* tmp = (double*)malloc(sizeof(double) * (size_t)N);
  z[0] = exp(-rate * pow(10.0, design_snr_db / 10.0));
  for (int len = 1; len < N; len *= 2) {
    for (int t = 0; t < len; ++t) {
      double zt = z[t];
      tmp[2 * t] = 2.0 * zt - zt * zt;
      tmp[2 * t + 1] = zt * zt;
    }
    memcpy(z, tmp, sizeof(double) * (size_t)(2 * len));
  }
  free(tmp);
}

/* Frozen set F: the N-K indices with the largest Bhattacharyya parameter
 * (least reliable); among equal values the lower index counts as less
 * reliable. Written ascending into frozen[0..N-K-1]. Returns 0 or -1. */
int oracle_frozen_set(int N, int K, double design_snr_db, int32_t* frozen) {
  if (N < 2 || N > ORACLE_MAX_N || (N & (N - 1)) || K < 0 || K >= N) return -1;
  double* z = (double*)malloc(sizeof(double) * (size_t)N);
  uint8_t* taken = (uint8_t*)calloc((size_t)N, 1);
  oracle_bhattacharyya(N, (double)K / (double)N, design_snr_db, z);
  for (int c = 0; c < N - K; ++c) {
    int best = -1;
    for (int i = 0; i < N; ++i) {
      if (taken[i]) continue;
      if (best < 0 || z[i] > z[best]) best = i; /* strict >: lower index wins ties */
    }
    taken[best] = 1;
  }
  int r = 0;
  for (int i = 0; i < N; ++i)
    if (taken[i]) frozen[r++] = i;
  free(z);
  free(taken);
  return 0;
}

/* Parity-check matrix H ((N-K) x N bytes): row r is column frozen[r] of G_N.
 * Since G_N G_N = I over GF(2), every information row of G_N is orthogonal to
 * these columns, i.e. G_I H^T = 0 (Def. II.1). */
void oracle_parity_H(int N, int K, const int32_t* frozen, uint8_t* H) {
  uint8_t* G = (uint8_t*)malloc((size_t)N * N);
  oracle_polar_G(N, G);
  for (int r = 0; r < N - K; ++r)
    for (int j = 0; j < N; ++j) H[(size_t)r * N + j] = G[(size_t)j * N + frozen[r]];
  free(G);
}

/* ------------------------------------------------------------------------- */
/* Square M-QAM (Def. II.2, Eq. 2) and demodulation (Def. III.1, III.2)       */
/* ------------------------------------------------------------------------- */

/* d = sqrt(3 m E_b / (M - 1)) with E_b = 1 and M = 2^(2m) (Eq. 2). */
double oracle_qam_d(int M) {
  int bits = 0;
  while ((1 << bits) < M) ++bits;
  int m = bits / 2;
  return sqrt(3.0 * (double)m / (double)(M - 1));
}

/* The fixed-point scale shared by both sides: 256 / d rounded once to float. */
float oracle_qam_qscale(int M) { return (float)(256.0 / oracle_qam_d(M)); }

typedef struct {
  int level;     /* hard level l in [0, sqrtM) */
  int32_t dq;    /* Q8.8 distance to the decision threshold (R1), >= 0 */
  int exists;    /* neighbour level l + dir is on the constellation (R2) */
  int dir;       /* +1 or -1 */
  double dist64; /* the same distance without quantisation, FP64 */
} axis_t;

/* One axis of Def. III.1 / III.2. `a` is the received coordinate in
 * transmitted units, q = 256/d (float), dscale = d (double). */
static axis_t demod_axis(float a, float q, double dscale, int sqrtM, int literal) {
  axis_t r;
  /* quantise: fp32 product rounded to nearest-even, clamped to int16 */
  float x = a * q;
  if (x > 32767.0f) x = 32767.0f;
  if (x < -32768.0f) x = -32768.0f;
  int32_t aq = (int32_t)nearbyintf(x);
  /* hard decision: decision thresholds at even multiples of 256 (the
   * midpoints between odd-integer levels); a value on a threshold goes up */
  int32_t t = aq + 256 * sqrtM;
  int l = (t < 0) ? 0 : (int)(t / 512);
  if (l > sqrtM - 1) l = sqrtM - 1;
  int A = 2 * l - (sqrtM - 1); /* odd-integer amplitude */
  int32_t delta = 256 * A - aq; /* A - a in Q8.8 */
  int32_t mag = delta < 0 ? -delta : delta;
  int outside = (l == 0 && delta > 0) || (l == sqrtM - 1 && delta < 0);
  int32_t d;
  if (literal) d = 256 - mag;
  else d = outside ? 256 + mag : 256 - mag;
  if (d < 0) d = 0;
  if (d > 32767) d = 32767;
  /* Def. III.2: the neighbour is at s - 2 Sign(A - a) */
  int dir;
  if (delta > 0) dir = -1;
  else if (delta < 0) dir = +1;
  else dir = (l == 0) ? +1 : -1;
  int nl = l + dir;
  r.level = l;
  r.dq = d;
  r.dir = dir;
  r.exists = (nl >= 0 && nl < sqrtM);
  /* FP64 distance of Def. III.1, from the unquantised value */
  double xa = (double)a / dscale;
  double m64 = fabs((double)A - xa);
  if (literal) r.dist64 = 1.0 - m64;
  else r.dist64 = outside ? 1.0 + m64 : 1.0 - m64;
  return r;
}

static int gray(int l) { return l ^ (l >> 1); }

typedef struct {
  axis_t I, Q;
  uint32_t key;  /* dI^2 + dQ^2 */
  double rel;    /* FP64 likelihood sqrt(d1^2 + d2^2) (Def. III.1) */
  int nonfinite;
} sym_t;

static sym_t demod_symbol(float a, float b, float q, double dscale, int sqrtM, int literal) {
  sym_t s;
  s.nonfinite = !(isfinite(a) && isfinite(b));
  if (s.nonfinite) { a = 0.0f; b = 0.0f; }
  s.I = demod_axis(a, q, dscale, sqrtM, literal);
  s.Q = demod_axis(b, q, dscale, sqrtM, literal);
  s.key = (uint32_t)s.I.dq * (uint32_t)s.I.dq + (uint32_t)s.Q.dq * (uint32_t)s.Q.dq;
  s.rel = sqrt(s.I.dist64 * s.I.dist64 + s.Q.dist64 * s.Q.dist64);
  return s;
}

/* Packed per-symbol outputs (shared layout with the public demod call):
 *   hard_idx = (I level << 8) | Q level
 *   nmask bit0 = horizontal neighbour exists, bit1 = vertical, bit2 = diagonal,
 *         bit3 = I direction is +1, bit4 = Q direction is +1,
 *         bit5 = d_Q < d_I (the vertical alternative is the nearer one),
 *         bit7 = non-finite received value. */
static uint8_t pack_nmask(const sym_t* s) {
  uint8_t m = 0;
  if (s->I.exists) m |= 1;
  if (s->Q.exists) m |= 2;
  if (s->I.exists && s->Q.exists) m |= 4;
  if (s->I.dir > 0) m |= 8;
  if (s->Q.dir > 0) m |= 16;
  if (s->Q.dq < s->I.dq) m |= 32; /* vertical alternative nearer (R6) */
  if (s->nonfinite) m |= 128;
  return m;
}

static int log2i(int x) {
  int b = 0;
  while ((1 << b) < x) ++b;
  return b;
}

/* Place the 2m-bit label of symbol i (I label first, MSB first) into bits[],
 * dropping positions >= N (padding, Alg. 2 input L = ceil(N/2m)). */
static void put_label(uint8_t* bits, int N, int i, int m, int gI, int gQ) {
  int label = (gI << m) | gQ;
  int nb = 2 * m;
  for (int k = 0; k < nb; ++k) {
    int pos = nb * i + k;
    if (pos < N) bits[pos] = (uint8_t)((label >> (nb - 1 - k)) & 1);
  }
}

/* Demodulate F frames of L symbols (interleaved float pairs). Any output
 * pointer may be NULL. y_words: F x (N/32) packed hard words. */
void oracle_demod(const float* sym, int64_t F, int L, int M, int N, int literal, uint16_t* hard_idx,
                  uint32_t* key, uint8_t* nmask, double* rel, uint32_t* y_words) {
  int sqrtM = 1 << (log2i(M) / 2);
  int m = log2i(M) / 2;
  float q = oracle_qam_qscale(M);
  double dscale = oracle_qam_d(M);
  uint8_t bits[ORACLE_MAX_N];
  for (int64_t f = 0; f < F; ++f) {
    memset(bits, 0, sizeof bits);
    for (int i = 0; i < L; ++i) {
      const float* p = sym + 2 * ((size_t)f * L + i);
      sym_t s = demod_symbol(p[0], p[1], q, dscale, sqrtM, literal);
      size_t o = (size_t)f * L + i;
      if (hard_idx) hard_idx[o] = (uint16_t)((s.I.level << 8) | s.Q.level);
      if (key) key[o] = s.key;
      if (nmask) nmask[o] = pack_nmask(&s);
      if (rel) rel[o] = s.rel;
      put_label(bits, N, i, m, gray(s.I.level), gray(s.Q.level));
    }
    if (y_words) {
      int W = N / 32;
      for (int w = 0; w < W; ++w) {
        uint32_t v = 0;
        for (int b = 0; b < 32; ++b) v |= (uint32_t)bits[32 * w + b] << b;
        y_words[(size_t)f * W + w] = v;
      }
    }
  }
}

/* ------------------------------------------------------------------------- */
/* Canonical TEP order (R3) and the GF(2) membership test (Alg. 2 Step 5)     */
/* ------------------------------------------------------------------------- */

/* Advance the sorted set p[0] < ... < p[w-1] < n to its successor in colex
 * order (sets compared by their largest element first). Returns 0 after the
 * last set. */
static int colex_next(int* p, int w, int n) {
  for (int j = 0; j < w; ++j) {
    int limit = (j + 1 < w) ? p[j + 1] : n;
    if (p[j] + 1 < limit) {
      p[j] += 1;
      for (int i = 0; i < j; ++i) p[i] = i;
      return 1;
    }
  }
  return 0;
}

/* Syndrome test: 1 iff H x = 0 over GF(2). H rows are packed into 64-bit
 * words (bit j of the row at word j/64, bit j%64), x likewise. */
static int syndrome_is_zero(const uint64_t* Hrows, int R, int NW, const uint64_t* x) {
  for (int r = 0; r < R; ++r) {
    int parity = 0;
    for (int w = 0; w < NW; ++w) parity ^= __builtin_popcountll(Hrows[(size_t)r * NW + w] & x[w]) & 1;
    if (parity) return 0;
  }
  return 1;
}

static void pack64(const uint8_t* bits, int N, uint64_t* x) {
  int NW = (N + 63) / 64;
  for (int w = 0; w < NW; ++w) x[w] = 0;
  for (int j = 0; j < N; ++j)
    if (bits[j]) x[j / 64] |= (uint64_t)1 << (j % 64);
}

/* Visit the valid TEPs over S' ranks in canonical order (R3), with n_alt
 * alternatives per symbol (3 for the paper's order, 4 for R7). Bit c-1 of
 * exists[r] says whether alternative c of rank r exists. For each valid TEP
 * the callback gets its per-rank alternative codes alt[r] in {0 = unchanged,
 * 1 .. n_alt}; it returns nonzero to stop. Returns the number of valid TEPs
 * visited (including the one that stopped the walk). */
typedef int (*tep_visit_fn)(void* ctx, const int* alt, int64_t count);

static int64_t walk_teps(int Sp, int n_alt, const uint8_t* exists, tep_visit_fn visit, void* ctx) {
  int64_t count = 0;
  int p[ORACLE_MAX_S];
  int alt[ORACLE_MAX_S];
  for (int w = 0; w <= Sp; ++w) {
    for (int i = 0; i < w; ++i) p[i] = i; /* first set in colex order */
    int more = 1;
    while (more) {
      int64_t n_alpha = 1;
      for (int i = 0; i < w; ++i) n_alpha *= n_alt;
      for (int64_t alpha = 0; alpha < n_alpha; ++alpha) {
        for (int r = 0; r < Sp; ++r) alt[r] = 0;
        int valid = 1;
        int64_t rest = alpha;
        for (int j = 0; j < w; ++j) { /* digit j belongs to the j-th smallest rank */
          int code = (int)(rest % n_alt) + 1; /* e.g. 1 = h, 2 = v, 3 = diag */
          rest /= n_alt;
          alt[p[j]] = code;
          if (!((exists[p[j]] >> (code - 1)) & 1)) valid = 0;
        }
        if (!valid) continue;
        ++count;
        if (visit(ctx, alt, count)) return count;
      }
      more = (w > 0) ? colex_next(p, w, Sp) : 0;
    }
  }
  return count;
}

/* ------------------------------------------------------------------------- */
/* Symbol-level GRAND with the likelihood order (Alg. 2)                      */
/* ------------------------------------------------------------------------- */

typedef struct {
  /* code */
  const uint64_t* Hrows;
  int N, R, NW;
  /* frame */
  int m;
  int Sp;
  int sym_of_rank[ORACLE_MAX_S];
  int alt_label[ORACLE_MAX_S][5]; /* label after alternative code c (c=0: hard) */
  const uint8_t* ybits;
  int64_t cap;
  /* result */
  int hit;
  uint8_t xbits[ORACLE_MAX_N];
} qam_ctx;

static int qam_visit(void* vctx, const int* alt, int64_t count) {
  qam_ctx* c = (qam_ctx*)vctx;
  /* candidate x = y xor e, with e from the altered symbols' labels */
  memcpy(c->xbits, c->ybits, (size_t)c->N);
  for (int r = 0; r < c->Sp; ++r) {
    if (!alt[r]) continue;
    put_label(c->xbits, c->N, c->sym_of_rank[r], c->m, c->alt_label[r][alt[r]] >> c->m,
              c->alt_label[r][alt[r]] & ((1 << c->m) - 1));
  }
  uint64_t x[ORACLE_MAX_N / 64];
  pack64(c->xbits, c->N, x);
  if (syndrome_is_zero(c->Hrows, c->R, c->NW, x)) {
    c->hit = 1;
    return 1;
  }
  return count >= c->cap;
}

typedef struct {
  const uint8_t* exists;
  uint32_t* out;
  int64_t max;
} list_ctx;

static int list_visit(void* vctx, const int* alt, int64_t count) {
  list_ctx* c = (list_ctx*)vctx;
  (void)alt;
  if (count > c->max) return 1;
  return 0;
}

/* Decode one frame. H is (R x N) bytes. Writes cw_words (N/32), queries,
 * abandon. Returns the number of valid TEPs of the frame (Prod (1+k_i)). */
#define ORDER_NNE 1       /* Def. III.2: h, v, diag */
#define ORDER_NNE_DSORT 2 /* R6 */
#define ORDER_NNE5 3      /* R7 */

static void decode_qam_frame(const uint64_t* Hrows, int N, int R, const float* sym, int L, int M,
                             int S, int64_t cap, int literal, int order, uint32_t* cw_words,
                             int64_t* queries, uint8_t* abandon) {
  int sqrtM = 1 << (log2i(M) / 2);
  int m = log2i(M) / 2;
  float q = oracle_qam_qscale(M);
  double dscale = oracle_qam_d(M);
  sym_t* s = (sym_t*)malloc(sizeof(sym_t) * (size_t)L);
  uint8_t ybits[ORACLE_MAX_N];
  memset(ybits, 0, sizeof ybits);
  int nonfinite = 0;
  /* Alg. 2 Step 1: likelihood and neighbours of every symbol */
  for (int i = 0; i < L; ++i) {
    s[i] = demod_symbol(sym[2 * i], sym[2 * i + 1], q, dscale, sqrtM, literal);
    nonfinite |= s[i].nonfinite;
    put_label(ybits, N, i, m, gray(s[i].I.level), gray(s[i].Q.level));
  }
  int W = N / 32;
  if (nonfinite) {
    for (int w = 0; w < W; ++w) {
      uint32_t v = 0;
      for (int b = 0; b < 32; ++b) v |= (uint32_t)ybits[32 * w + b] << b;
      cw_words[w] = v;
    }
    *queries = 0;
    *abandon = 2;
    free(s);
    return;
  }
  /* Alg. 2 Step 2: order symbols by (key ascending, index ascending) -- a
   * plain selection of the minimum, S' times (Step 3 keeps only these). */
  int Sp = S < L ? S : L;
  qam_ctx c;
  memset(&c, 0, sizeof c);
  uint8_t* used = (uint8_t*)calloc((size_t)L, 1);
  uint8_t exists[ORACLE_MAX_S];
  for (int r = 0; r < Sp; ++r) {
    int best = -1;
    for (int i = 0; i < L; ++i) {
      if (used[i]) continue;
      if (best < 0 || s[i].key < s[best].key) best = i; /* ties: lower index first */
    }
    used[best] = 1;
    c.sym_of_rank[r] = best;
    const sym_t* t = &s[best];
    int lI = t->I.level, lQ = t->Q.level;
    int nI = lI + t->I.dir, nQ = lQ + t->Q.dir;
    /* Def. III.2: horizontal s_d1, vertical s_d2, diagonal s_d1d2 */
    int lab_h = t->I.exists ? ((gray(nI) << m) | gray(lQ)) : 0;
    int lab_v = t->Q.exists ? ((gray(lI) << m) | gray(nQ)) : 0;
    int ex_h = t->I.exists, ex_v = t->Q.exists;
    c.alt_label[r][0] = (gray(lI) << m) | gray(lQ);
    if (order == ORDER_NNE5) {
      /* R7: the other neighbouring level of each axis, away from r */
      int aI = lI - t->I.dir, aQ = lQ - t->Q.dir;
      int ex_aI = aI >= 0 && aI < sqrtM, ex_aQ = aQ >= 0 && aQ < sqrtM;
      c.alt_label[r][1] = lab_h;
      c.alt_label[r][2] = lab_v;
      c.alt_label[r][3] = ex_aI ? ((gray(aI) << m) | gray(lQ)) : 0;
      c.alt_label[r][4] = ex_aQ ? ((gray(lI) << m) | gray(aQ)) : 0;
      exists[r] = (uint8_t)(ex_h | (ex_v << 1) | (ex_aI << 2) | (ex_aQ << 3));
      continue;
    }
    if (order == ORDER_NNE_DSORT && t->Q.dq < t->I.dq) { /* R6: nearer axis first */
      int tl = lab_h; lab_h = lab_v; lab_v = tl;
      int te = ex_h; ex_h = ex_v; ex_v = te;
    }
    c.alt_label[r][1] = lab_h;
    c.alt_label[r][2] = lab_v;
    c.alt_label[r][3] = (t->I.exists && t->Q.exists) ? ((gray(nI) << m) | gray(nQ)) : 0;
    exists[r] = (uint8_t)((ex_h ? 1 : 0) | (ex_v ? 2 : 0) | ((ex_h && ex_v) ? 4 : 0));
  }
  free(used);
  c.Hrows = Hrows;
  c.N = N;
  c.R = R;
  c.NW = (N + 63) / 64;
  c.m = m;
  c.Sp = Sp;
  c.ybits = ybits;
  c.cap = cap;
  /* Alg. 2 Steps 4-5: query the TEPs in canonical order until a codeword */
  int64_t n = walk_teps(Sp, order == ORDER_NNE5 ? 4 : 3, exists, qam_visit, &c);
  const uint8_t* out = c.hit ? c.xbits : ybits;
  for (int w = 0; w < W; ++w) {
    uint32_t v = 0;
    for (int b = 0; b < 32; ++b) v |= (uint32_t)out[32 * w + b] << b;
    cw_words[w] = v;
  }
  *queries = n;
  *abandon = c.hit ? 0 : 1;
  free(s);
}

/* ------------------------------------------------------------------------- */
/* Bit-level GRAND-AB (Sec. I; hard decision, ascending Hamming weight)       */
/* ------------------------------------------------------------------------- */

static void decode_ab_frame(const uint64_t* Hrows, int N, int R, const float* r, int max_weight,
                            int64_t cap, uint32_t* cw_words, int64_t* queries, uint8_t* abandon) {
  uint8_t ybits[ORACLE_MAX_N], xbits[ORACLE_MAX_N];
  int NW = (N + 63) / 64;
  uint64_t x[ORACLE_MAX_N / 64];
  int nonfinite = 0;
  for (int j = 0; j < N; ++j) {
    float v = r[j];
    if (!isfinite(v)) { nonfinite = 1; v = 0.0f; }
    ybits[j] = (uint8_t)(v < 0.0f);
  }
  int W = N / 32;
  int64_t count = 0;
  int hit = 0;
  if (!nonfinite) {
    int p[ORACLE_MAX_N];
    for (int w = 0; w <= max_weight && w <= N && !hit && count < cap; ++w) {
      for (int i = 0; i < w; ++i) p[i] = i;
      int more = 1;
      while (more) {
        memcpy(xbits, ybits, (size_t)N);
        for (int i = 0; i < w; ++i) xbits[p[i]] ^= 1;
        ++count;
        pack64(xbits, N, x);
        if (syndrome_is_zero(Hrows, R, NW, x)) { hit = 1; break; }
        if (count >= cap) break;
        more = (w > 0) ? colex_next(p, w, N) : 0;
      }
    }
  }
  const uint8_t* out = hit ? xbits : ybits;
  for (int w = 0; w < W; ++w) {
    uint32_t v = 0;
    for (int b = 0; b < 32; ++b) v |= (uint32_t)out[32 * w + b] << b;
    cw_words[w] = v;
  }
  *queries = nonfinite ? 0 : count;
  *abandon = nonfinite ? 2 : (hit ? 0 : 1);
}

/* ------------------------------------------------------------------------- */
/* Batch entry points (frames split across threads; each frame is sequential) */
/* ------------------------------------------------------------------------- */

static uint64_t* pack_H_rows(const uint8_t* H, int R, int N) {
  int NW = (N + 63) / 64;
  uint64_t* Hr = (uint64_t*)calloc((size_t)R * NW, sizeof(uint64_t));
  for (int r = 0; r < R; ++r)
    for (int j = 0; j < N; ++j)
      if (H[(size_t)r * N + j]) Hr[(size_t)r * NW + j / 64] |= (uint64_t)1 << (j % 64);
  return Hr;
}

typedef struct {
  const uint64_t* Hrows;
  int N, R, L, M, S, max_weight, literal, order, bit_level;
  int64_t cap;
  const float* sym;
  int64_t F;
  uint32_t* cw;
  int64_t* queries;
  uint8_t* abandon;
  int tid, nthreads;
} job_t;

static void* run_job(void* vjob) {
  job_t* j = (job_t*)vjob;
  int W = j->N / 32;
  for (int64_t f = j->tid; f < j->F; f += j->nthreads) {
    if (j->bit_level)
      decode_ab_frame(j->Hrows, j->N, j->R, j->sym + (size_t)f * j->N, j->max_weight, j->cap,
                      j->cw + (size_t)f * W, &j->queries[f], &j->abandon[f]);
    else
      decode_qam_frame(j->Hrows, j->N, j->R, j->sym + 2 * (size_t)f * j->L, j->L, j->M, j->S, j->cap,
                       j->literal, j->order, j->cw + (size_t)f * W, &j->queries[f], &j->abandon[f]);
  }
  return NULL;
}

static int run_batch(job_t proto, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  pthread_t th[256];
  job_t jobs[256];
  for (int t = 0; t < nthreads; ++t) {
    jobs[t] = proto;
    jobs[t].tid = t;
    jobs[t].nthreads = nthreads;
  }
  if (nthreads == 1) {
    run_job(&jobs[0]);
    return 0;
  }
  for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, run_job, &jobs[t]);
  for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
  return 0;
}

/* Symbol-level decode of F frames of L complex symbols (float pairs), with
 * the TEP order `order` (ORDER_NNE, ORDER_NNE_DSORT or ORDER_NNE5). */
int oracle_decode_qam_order(const uint8_t* H, int N, int K, const float* sym, int64_t F, int L, int M,
                            int S, int64_t cap, int literal, int order, int nthreads, uint32_t* cw,
                            int64_t* queries, uint8_t* abandon) {
  if (S < 0 || S > ORACLE_MAX_S || cap < 1 || N > ORACLE_MAX_N || N % 32) return -1;
  if (order != ORDER_NNE && order != ORDER_NNE_DSORT && order != ORDER_NNE5) return -1;
  job_t p;
  memset(&p, 0, sizeof p);
  p.R = N - K;
  p.Hrows = pack_H_rows(H, p.R, N);
  p.N = N; p.L = L; p.M = M; p.S = S; p.cap = cap; p.literal = literal; p.order = order;
  p.bit_level = 0;
  p.sym = sym; p.F = F; p.cw = cw; p.queries = queries; p.abandon = abandon;
  run_batch(p, nthreads);
  free((void*)p.Hrows);
  return 0;
}

/* The same with the paper's order (Def. III.2). */
int oracle_decode_qam(const uint8_t* H, int N, int K, const float* sym, int64_t F, int L, int M, int S,
                      int64_t cap, int literal, int nthreads, uint32_t* cw, int64_t* queries,
                      uint8_t* abandon) {
  return oracle_decode_qam_order(H, N, K, sym, F, L, M, S, cap, literal, ORDER_NNE, nthreads, cw,
                                 queries, abandon);
}

/* Bit-level GRAND-AB decode of F frames of N real BPSK samples. */
int oracle_decode_ab(const uint8_t* H, int N, int K, const float* r, int64_t F, int max_weight,
                     int64_t cap, int nthreads, uint32_t* cw, int64_t* queries, uint8_t* abandon) {
  if (max_weight < 0 || cap < 1 || N > ORACLE_MAX_N || N % 32) return -1;
  job_t p;
  memset(&p, 0, sizeof p);
  p.R = N - K;
  p.Hrows = pack_H_rows(H, p.R, N);
  p.N = N; p.L = N; p.max_weight = max_weight; p.cap = cap; p.bit_level = 1;
  p.sym = r; p.F = F; p.cw = cw; p.queries = queries; p.abandon = abandon;
  run_batch(p, nthreads);
  free((void*)p.Hrows);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Introspection for the tests                                                */
/* ------------------------------------------------------------------------- */

typedef struct {
  int Sp;
  int bits; /* bits per rank in the packed code */
  uint32_t* out;
  int64_t max;
} codes_ctx;

static int codes_visit(void* vctx, const int* alt, int64_t count) {
  codes_ctx* c = (codes_ctx*)vctx;
  if (count > c->max) return 1;
  uint32_t code = 0;
  for (int r = 0; r < c->Sp; ++r) code |= (uint32_t)alt[r] << (c->bits * r);
  c->out[count - 1] = code;
  return 0;
}

/* Write the valid TEPs over Sp ranks in canonical order as packed codes
 * (2 bits per rank: 0 unchanged, 1 h, 2 v, 3 diag; rank r at bits 2r..2r+1).
 * Returns the total number of valid TEPs (even if larger than max_out). */
int64_t oracle_tep_order(int Sp, const uint8_t* exists, uint32_t* out, int64_t max_out) {
  if (Sp < 0 || Sp > ORACLE_MAX_S) return -1;
  codes_ctx c = {Sp, 2, out, max_out};
  int64_t total = walk_teps(Sp, 3, exists, codes_visit, &c);
  if (total > max_out) {
    /* the walk stopped early; count the rest without recording */
    list_ctx l = {exists, NULL, INT64_MAX};
    total = walk_teps(Sp, 3, exists, list_visit, &l);
  }
  return total;
}

/* The same for n_alt alternatives per symbol (3 or 4), packed with 3 bits
 * per rank (Sp <= 10). */
int64_t oracle_tep_order_n(int Sp, int n_alt, const uint8_t* exists, uint32_t* out, int64_t max_out) {
  if (Sp < 0 || Sp > 10 || n_alt < 1 || n_alt > 4) return -1;
  codes_ctx c = {Sp, 3, out, max_out};
  int64_t total = walk_teps(Sp, n_alt, exists, codes_visit, &c);
  if (total > max_out) {
    list_ctx l = {exists, NULL, INT64_MAX};
    total = walk_teps(Sp, n_alt, exists, list_visit, &l);
  }
  return total;
}

/* Indices of the Sp least reliable symbols of one frame, ascending (Step 2-3). */
int oracle_select(const uint32_t* key, int L, int S, int32_t* ranks_out) {
  int Sp = S < L ? S : L;
  uint8_t* used = (uint8_t*)calloc((size_t)L, 1);
  for (int r = 0; r < Sp; ++r) {
    int best = -1;
    for (int i = 0; i < L; ++i) {
      if (used[i]) continue;
      if (best < 0 || key[i] < key[best]) best = i;
    }
    used[best] = 1;
    ranks_out[r] = best;
  }
  free(used);
  return Sp;
}
