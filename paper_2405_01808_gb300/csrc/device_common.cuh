// Device helpers shared by the decoder kernels: fixed-point demodulation
// (Def. III.1 / III.2), Gray labels, binomials and the TEP rank function of the
// canonical order.
#pragma once

#include <stdint.h>

#include "internal.cuh"

namespace grand {

// ---------------------------------------------------------------------------
// Binomial coefficients C(n, k), n, k <= 16, generated at compile time.
// ---------------------------------------------------------------------------
struct BinomTable {
  uint32_t v[17][17];
};

constexpr BinomTable make_binom() {
  BinomTable t{};
  for (int n = 0; n <= 16; ++n) {
    t.v[n][0] = 1;
    for (int k = 1; k <= n; ++k) t.v[n][k] = t.v[n - 1][k - 1] + (k <= n - 1 ? t.v[n - 1][k] : 0);
  }
  return t;
}

__constant__ const BinomTable c_binom = make_binom();

__device__ __forceinline__ uint32_t binom16(int n, int k) {
  return (k < 0 || n < 0 || k > n) ? 0u : c_binom.v[n][k];
}

// ---------------------------------------------------------------------------
// The call's deadline (grand_params.deadline_ns). The budget runs from the
// first look at the device clock by any warp of the call (stored in *t0, zero
// before the call); a warp that looks after budget nanoseconds sees true.
// Called by one lane; the caller broadcasts the answer to its warp.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool past_deadline(unsigned long long* t0, long long budget) {
  if (budget <= 0 || !t0) return false;
  const unsigned long long now = global_ns();
  unsigned long long start = *(volatile unsigned long long*)t0;
  if (start == 0) {
    start = atomicCAS(t0, 0ull, now);
    if (start == 0) start = now;
  }
  // another warp may have stamped a later time than this warp's reading
  return now > start && now - start > (unsigned long long)budget;
}

// C(n, k) for n up to 1024, k up to 4 (bit-level orders), 64-bit: the falling
// factorial over k!, with constant divisors (no division loop).
__device__ __forceinline__ uint64_t binom_big(int n, int k) {
  if (k < 0 || n < k) return 0;
  const uint64_t m = (uint64_t)n;
  switch (k) {
    case 0: return 1;
    case 1: return m;
    case 2: return m * (m - 1) / 2;
    case 3: return m * (m - 1) * (m - 2) / 6;
    case 4: return m * (m - 1) * (m - 2) * (m - 3) / 24;
    default: {
      uint64_t r = 1;
      for (int i = 1; i <= k; ++i) r = r * (uint64_t)(n - k + i) / (uint64_t)i;
      return r;
    }
  }
}

// ---------------------------------------------------------------------------
// Demodulation of one axis in Q8.8 units of the odd-integer grid.
//   a_q = round_half_even(fp32(a * 256/d)), clamped to int16
//   level l = floor((a_q + 256 sqrtM) / 512) clamped; amplitude A = 2l - (sqrtM-1)
//   distance to the nearest decision threshold (Def. III.1 read with the
//   "beyond the outermost level" case as 1 + |A - a|; LITERAL: 1 - |A - a|)
//   neighbour direction -Sign(A - a) (Def. III.2); tie -> lower level except
//   at the lowest level.
// ---------------------------------------------------------------------------
struct AxisDemod {
  int level;
  int dq;
  int dir;
  bool exists;
  bool outside;
  int amp;
};

__device__ __forceinline__ AxisDemod demod_axis_q(float a, float q, int side, int literal) {
  AxisDemod r;
  float x = __fmul_rn(a, q);
  x = fminf(fmaxf(x, -32768.0f), 32767.0f);
  const int aq = __float2int_rn(x);
  const int t = aq + 256 * side;
  int l = t < 0 ? 0 : (t >> 9);
  l = l > side - 1 ? side - 1 : l;
  const int A = 2 * l - (side - 1);
  const int delta = 256 * A - aq;
  const int mag = delta < 0 ? -delta : delta;
  const bool outside = (l == 0 && delta > 0) || (l == side - 1 && delta < 0);
  int d = literal ? 256 - mag : (outside ? 256 + mag : 256 - mag);
  d = d < 0 ? 0 : (d > 32767 ? 32767 : d);
  const int dir = delta > 0 ? -1 : (delta < 0 ? 1 : (l == 0 ? 1 : -1));
  const int nl = l + dir;
  r.level = l;
  r.dq = d;
  r.dir = dir;
  r.exists = nl >= 0 && nl < side;
  r.outside = outside;
  r.amp = A;
  return r;
}

// FP32 likelihood distance of one axis from the unquantised value.
__device__ __forceinline__ float axis_dist_f32(float a, float inv_d, int amp, bool outside, int literal) {
  const float x = __fmul_rn(a, inv_d);
  const float m = fabsf((float)amp - x);
  return literal ? 1.0f - m : (outside ? 1.0f + m : 1.0f - m);
}

__device__ __forceinline__ int gray_code(int l) { return l ^ (l >> 1); }

// Packed per-symbol summary used inside the kernels:
//   bits 0..7 I level, 8..15 Q level, 16..23 nmask (see grand.h)
__device__ __forceinline__ uint32_t pack_info(int lI, int lQ, uint32_t nmask) {
  return (uint32_t)lI | ((uint32_t)lQ << 8) | (nmask << 16);
}

__device__ __forceinline__ uint32_t make_nmask(const AxisDemod& I, const AxisDemod& Q, bool nonfinite) {
  uint32_t m = 0;
  if (I.exists) m |= 1u;
  if (Q.exists) m |= 2u;
  if (I.exists && Q.exists) m |= 4u;
  if (I.dir > 0) m |= 8u;
  if (Q.dir > 0) m |= 16u;
  if (Q.dq < I.dq) m |= 32u;  // the vertical alternative is the nearer one
  if (nonfinite) m |= 128u;
  return m;
}

// Frame bit positions flipped by the horizontal / vertical alternative of a
// symbol (a neighbouring level differs from the hard level in exactly one bit
// of the binary-reflected Gray label: bit ctz(max(l, l')) of the m-bit label).
// Labels are MSB first: I label bits occupy [2m i, 2m i + m), Q label bits
// [2m i + m, 2m i + 2m). Returns kNoPos if the position is beyond N.
__device__ __forceinline__ uint16_t flip_pos_I(int i, int m, int l, int dir, int N) {
  const int hi = l > l + dir ? l : l + dir;
  const int b = __ffs(hi) - 1;
  const int p = 2 * m * i + (m - 1 - b);
  return p < N ? (uint16_t)p : kNoPos;
}
__device__ __forceinline__ uint16_t flip_pos_Q(int i, int m, int l, int dir, int N) {
  const int hi = l > l + dir ? l : l + dir;
  const int b = __ffs(hi) - 1;
  const int p = 2 * m * i + (2 * m - 1 - b);
  return p < N ? (uint16_t)p : kNoPos;
}

// ---------------------------------------------------------------------------
// Canonical order bookkeeping.
//   k_r = number of existing alternatives of rank r (0, 1 or 3)
//   E[x][v] = e_v(k_0, ..., k_{x-1}) (elementary symmetric polynomials):
//   the number of valid TEPs that alter exactly v of the ranks 0..x-1.
// ---------------------------------------------------------------------------
constexpr int kEStride = kSMax + 1;

// One full warp: lane v carries e_v along x (E[x+1][v] = E[x][v] + k_x E[x][v-1]).
__device__ inline void esp_table_warp(const uint8_t* ex, int Sp, uint32_t* E) {
  const int v = threadIdx.x & 31;
  uint32_t e = (v == 0) ? 1u : 0u;
  if (v <= Sp) E[v] = e;
  for (int x = 0; x < Sp; ++x) {
    const uint32_t k = __popc(ex[x] & 7u);
    uint32_t up = __shfl_up_sync(0xFFFFFFFFu, e, 1);
    if (v == 0) up = 0;
    e += k * up;
    if (v <= Sp) E[(x + 1) * kEStride + v] = e;
  }
}

__device__ __forceinline__ uint32_t esp_total(const uint32_t* E, int Sp) {
  uint32_t t = 0;
  for (int v = 0; v <= Sp; ++v) t += E[Sp * kEStride + v];
  return t;
}

// 1-based position of a valid TEP among the valid TEPs in canonical order.
// code: 2 bits per rank (0 unchanged, 1 h, 2 v, 3 diag).
//   = (valid TEPs with fewer altered ranks)
//   + sum_i (prod_{j>i} k_{p_j}) * E[p_i][i]      (altered sets before P in colex)
//   + sum_j less_j * prod_{i<j} k_{p_i}          (alternatives before alpha)
//   + 1
__device__ inline uint32_t tep_rank(const uint32_t* E, int Sp, const uint8_t* ex, uint32_t code) {
  int P[kSMax];
  int w = 0;
  for (int r = 0; r < Sp; ++r)
    if ((code >> (2 * r)) & 3u) P[w++] = r;
  uint32_t cnt = 0;
  for (int v = 0; v < w; ++v) cnt += E[Sp * kEStride + v];
  uint32_t mult = 1;
  for (int i = w; i >= 1; --i) {
    cnt += mult * E[P[i - 1] * kEStride + i];
    mult *= (uint32_t)__popc(ex[P[i - 1]] & 7u);
  }
  uint32_t low = 1;
  for (int j = 0; j < w; ++j) {
    const uint32_t c = (code >> (2 * P[j])) & 3u;
    const uint32_t e = ex[P[j]] & 7u;
    cnt += (uint32_t)__popc(e & ((1u << (c - 1)) - 1u)) * low;
    low *= (uint32_t)__popc(e);
  }
  return cnt + 1;
}

__device__ __forceinline__ int code_weight(uint32_t code) {
  return __popc((code | (code >> 1)) & 0x55555555u);
}

}  // namespace grand
