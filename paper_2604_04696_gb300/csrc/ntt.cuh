// Negacyclic NTT, its inverse and the gadget digit decomposition (Dcp) on one
// CTA, for the ciphertext-tree kernels of ColTor and ExpandQuery (GPIR paper
// Sec. 2.4.1 for the NTT, Sec. 2.5.1 for the Inverse NTT -> Dcp -> Forward
// NTT -> multiply-accumulate chain they share).
//
// Transform: A_s = sum_j a_j psi^((2s+1) j) mod q, psi = g^((q-1)/2N) with g
// the smallest generator of Z_q^* (the NTT form RowSel's data is in), slots in
// natural order. The butterfly networks are the merged-twist Cooley-Tukey
// (forward, natural -> bit-reversed) and Gentleman-Sande (inverse,
// bit-reversed -> natural) networks of Longa and Naehrig ("Speeding up the
// Number Theoretic Transform for Faster Ideal Lattice-Based Cryptography",
// CANS 2016), with twiddles psi^brv(k) and psi^-brv(k).
//
// Arithmetic: Harvey's lazy butterflies ("Faster arithmetic for
// number-theoretic transforms", J. Symb. Comp. 2014) with Shoup products:
// a * w mod q for a fixed w is a*w - floor(a * w' / 2^32) * q with
// w' = floor(w 2^32 / q), a value in [0, 2q) for any 32-bit a. Inverse values
// stay in [0, 2q) (one conditional subtraction per butterfly). Forward values
// are reduced below 8q once per radix round and grow by at most 2q per level,
// so they stay below 14q; q < 2^28 keeps 14q < 2^32. A conditional
// subtraction x >= c ? x - c : x is min(x, x - c) on unsigned values.
//
// GPU mapping. A polynomial of one limb belongs to a CTA of HALF threads
// (the kernels run one CTA per limb of a tree node, the limbs of a node in one
// thread-block cluster). Thread b of the group owns the 8 points
// b + (N/8) e, e = 0..7, in registers on both ends of a transform, so the
// transforms chain with the coefficient-wise Dcp and the slot-wise
// multiply-accumulate without a trip through memory:
//   - forward: the first radix-8 round (levels 0-2) works on exactly the
//     owned coefficients; the last radix-8 round works on 8 consecutive
//     bit-reversed positions 8i+k, and with i = brv(b) those hold the owned
//     slots b + (N/8) brv3(k), so no bit-reversal pass is needed;
//   - inverse: the mirror image (first round on the owned slots at positions
//     8 brv(b) + k, last round on the owned coefficients).
// Middle rounds go through shared memory: one load of 8 values, three levels
// of butterflies in registers, one store, one barrier. N is a template
// parameter, so every round's geometry is a compile-time constant.
//
// Shared-memory layout: position x lives at word pad(x) = x + (x >> 7) of a
// buffer of padn(N) = N + N/128 words. Every set of every round has the form
// base + k u with base = i 2^R u + o, o < u, and for those
// pad(base + k u) = pad(base) + k u + (k u >> 7): one address per set, the
// rest are immediate offsets. With the thread-to-set map of the 64i + o + 8k
// round below, every access of every round at N = 4096 is free of bank
// conflicts (the pad word per 128 spreads the bit-reversed sets 8 brv(b) + k
// over all banks).
#pragma once

#include <stdint.h>

#include "common.cuh"
#include "internal.h"

namespace gpir {
namespace ntt {

constexpr int HALF = 512;                 // threads per limb polynomial (N/8 at N = 4096)
constexpr uint32_t MAX_N = 4096;
constexpr uint32_t MIN_N = 16;
constexpr int MIN_LOGN = 4, MAX_LOGN = 12;
constexpr uint32_t MAX_LIMBS = 2;
constexpr int LOG_BASE = 22;              // gadget base z = 2^22 (the paper's)

struct Limb {
  const uint2 *fw;        // [N]  (psi^brv(k), Shoup quotient)
  const uint2 *iv;        // [N]  (psi^-brv(k), Shoup quotient)
  const uint2 *fw_last;   // [N/8][8]: the twiddles of the last forward round of thread b, in thread order
  const uint2 *iv_first;  // [N/8][8]: the twiddles of the first inverse round of thread b, in thread order
  const uint2 *mono;      // [2N] (psi^-e, Shoup quotient): slot s of NTT(X^-m) is psi^-((2s+1) m mod 2N)
  uint32_t q, n_inv, n_inv_s, pad;
  uint64_t mu;            // floor(2^64 / q)
};

struct Ring {
  uint32_t L, N, logn, ell;
  uint64_t Q;             // prod q_l (< 2^56)
  uint64_t half_Q;        // floor(Q / 2)
  uint64_t offset;        // O = sum_{k < ell-1} 2^21 2^(22 k): y = x + O has the balanced digits as plain digits
  uint32_t q0_inv, q0_inv_s;   // q0^-1 mod q1 and its Shoup quotient (L = 2)
  Limb limb[MAX_LIMBS];
};

__host__ __device__ constexpr uint32_t padn(uint32_t n) { return n + (n >> 7); }
__device__ __forceinline__ uint32_t pad(uint32_t x) { return x + (x >> 7); }
__device__ __forceinline__ uint32_t brev(uint32_t x, uint32_t bits) { return bits ? __brev(x) >> (32 - bits) : 0u; }

__device__ __forceinline__ uint32_t csub(uint32_t x, uint32_t c) { return min(x, x - c); }
__device__ __forceinline__ uint32_t shoup_lazy(uint32_t a, uint32_t w, uint32_t ws, uint32_t q) {
  return a * w - __umulhi(a, ws) * q;
}
__device__ __forceinline__ uint32_t shoup(uint32_t a, uint32_t w, uint32_t ws, uint32_t q) {
  return csub(shoup_lazy(a, w, ws, q), q);
}
__device__ __forceinline__ uint32_t add_mod(uint32_t a, uint32_t b, uint32_t q) { return csub(a + b, q); }
__device__ __forceinline__ uint32_t sub_mod(uint32_t a, uint32_t b, uint32_t q) { return csub(a - b + q, q); }

// Cooley-Tukey butterfly with no reduction of its own: t = w y mod q lies in
// [0, 2q) for any 32-bit y (Shoup), so x < B gives outputs below B + 2q. Each
// forward round first brings its values below 8q (fwd_entry), so after its at
// most three levels they stay below 14q < 2^32 (q < 2^28): one conditional
// subtraction per value and round instead of one per butterfly.
__device__ __forceinline__ void ct(uint32_t &x, uint32_t &y, uint32_t w, uint32_t ws, uint32_t q) {
  const uint32_t t = shoup_lazy(y, w, ws, q);
  const uint32_t u = x;
  x = u + t;
  y = u - t + 2 * q;
}
// Start of a forward round: values below 16q (14q from the previous round,
// q for the input coefficients) are brought below 8q.
template <int K>
__device__ __forceinline__ void fwd_entry(uint32_t (&v)[8], uint32_t q) {
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = csub(v[k], 8 * q);
}
// Gentleman-Sande butterfly, inputs and outputs in [0, 2q).
__device__ __forceinline__ void gs(uint32_t &x, uint32_t &y, uint32_t w, uint32_t ws, uint32_t q) {
  const uint32_t u = csub(x + y, 2 * q);
  const uint32_t t = x - y + 2 * q;
  x = u;
  y = shoup_lazy(t, w, ws, q);
}

__device__ __forceinline__ uint4 ld4(const uint2 *p) { return __ldg(reinterpret_cast<const uint4 *>(p)); }
__device__ __forceinline__ uint2 ld2(const uint2 *p) { return __ldg(p); }

// Forward round of R levels starting at level l0 (M0 = 2^l0 groups) on the set
// of group i: v[k] holds position i * 2^R u + o + k u, u = N / (2^R M0).
// Level r pairs k with k + 2^(R-1-r) and uses twiddle 2^r M0 + 2^r i + (k >> (R-r)).
template <int R, uint32_t M0>
__device__ __forceinline__ void fwd_round(uint32_t (&v)[8], const uint2 *fw, uint32_t i, uint32_t q) {
  fwd_entry<(1 << R)>(v, q);
  if constexpr (R == 3) {
    const uint2 a = ld2(fw + i + M0);
    ct(v[0], v[4], a.x, a.y, q); ct(v[1], v[5], a.x, a.y, q); ct(v[2], v[6], a.x, a.y, q); ct(v[3], v[7], a.x, a.y, q);
    const uint4 b = ld4(fw + 2 * i + 2 * M0);
    ct(v[0], v[2], b.x, b.y, q); ct(v[1], v[3], b.x, b.y, q); ct(v[4], v[6], b.z, b.w, q); ct(v[5], v[7], b.z, b.w, q);
    const uint4 c = ld4(fw + 4 * i + 4 * M0), d = ld4(fw + 4 * i + 4 * M0 + 2);
    ct(v[0], v[1], c.x, c.y, q); ct(v[2], v[3], c.z, c.w, q); ct(v[4], v[5], d.x, d.y, q); ct(v[6], v[7], d.z, d.w, q);
  } else if constexpr (R == 2) {
    const uint2 a = ld2(fw + i + M0);
    ct(v[0], v[2], a.x, a.y, q); ct(v[1], v[3], a.x, a.y, q);
    const uint4 b = ld4(fw + 2 * i + 2 * M0);
    ct(v[0], v[1], b.x, b.y, q); ct(v[2], v[3], b.z, b.w, q);
  } else {
    const uint2 a = ld2(fw + i + M0);
    ct(v[0], v[1], a.x, a.y, q);
  }
}

// Inverse round of R levels starting at t0: v[k] holds position
// i * 2^R t0 + o + k t0. Level r pairs k with k + 2^r and uses twiddle
// H0 / 2^r + 2^(R-1-r) i + (k >> (r+1)), H0 = N / (2 t0).
template <int R, uint32_t H0>
__device__ __forceinline__ void inv_round(uint32_t (&v)[8], const uint2 *iv, uint32_t i, uint32_t q) {
  if constexpr (R == 3) {
    const uint4 a = ld4(iv + 4 * i + H0), b = ld4(iv + 4 * i + H0 + 2);
    gs(v[0], v[1], a.x, a.y, q); gs(v[2], v[3], a.z, a.w, q); gs(v[4], v[5], b.x, b.y, q); gs(v[6], v[7], b.z, b.w, q);
    const uint4 c = ld4(iv + 2 * i + H0 / 2);
    gs(v[0], v[2], c.x, c.y, q); gs(v[1], v[3], c.x, c.y, q); gs(v[4], v[6], c.z, c.w, q); gs(v[5], v[7], c.z, c.w, q);
    const uint2 d = ld2(iv + i + H0 / 4);
    gs(v[0], v[4], d.x, d.y, q); gs(v[1], v[5], d.x, d.y, q); gs(v[2], v[6], d.x, d.y, q); gs(v[3], v[7], d.x, d.y, q);
  } else if constexpr (R == 2) {
    const uint4 a = ld4(iv + 2 * i + H0);
    gs(v[0], v[1], a.x, a.y, q); gs(v[2], v[3], a.z, a.w, q);
    const uint2 c = ld2(iv + i + H0 / 2);
    gs(v[0], v[2], c.x, c.y, q); gs(v[1], v[3], c.x, c.y, q);
  } else {
    const uint2 a = ld2(iv + i + H0);
    gs(v[0], v[1], a.x, a.y, q);
  }
}

// The bit-reversed rounds (the last forward round and the first inverse round,
// set i = brv(b)) touch 7/8 of the twiddle table, scattered over the threads of
// a warp. Their twiddles are also stored per thread, in thread order (64 bytes
// each, see ring_tables.cu), so that these loads are contiguous across a warp:
//   fw_last[b]  = W[N/8 + i], W[N/4 + 2i], W[N/4 + 2i + 1], -, W[N/2 + 4i + 0..3]
//   iv_first[b] = V[N/2 + 4i + 0..3], V[N/4 + 2i], V[N/4 + 2i + 1], V[N/8 + i], -
__device__ __forceinline__ void fwd_round_last(uint32_t (&v)[8], const uint2 *t, uint32_t q) {
  fwd_entry<8>(v, q);
  const uint4 a = ld4(t), b = ld4(t + 2);
  ct(v[0], v[4], a.x, a.y, q); ct(v[1], v[5], a.x, a.y, q); ct(v[2], v[6], a.x, a.y, q); ct(v[3], v[7], a.x, a.y, q);
  ct(v[0], v[2], a.z, a.w, q); ct(v[1], v[3], a.z, a.w, q); ct(v[4], v[6], b.x, b.y, q); ct(v[5], v[7], b.x, b.y, q);
  const uint4 c = ld4(t + 4), d = ld4(t + 6);
  ct(v[0], v[1], c.x, c.y, q); ct(v[2], v[3], c.z, c.w, q); ct(v[4], v[5], d.x, d.y, q); ct(v[6], v[7], d.z, d.w, q);
}
__device__ __forceinline__ void inv_round_first(uint32_t (&v)[8], const uint2 *t, uint32_t q) {
  const uint4 a = ld4(t), b = ld4(t + 2);
  gs(v[0], v[1], a.x, a.y, q); gs(v[2], v[3], a.z, a.w, q); gs(v[4], v[5], b.x, b.y, q); gs(v[6], v[7], b.z, b.w, q);
  const uint4 c = ld4(t + 4), d = ld4(t + 6);
  gs(v[0], v[2], c.x, c.y, q); gs(v[1], v[3], c.x, c.y, q); gs(v[4], v[6], c.z, c.w, q); gs(v[5], v[7], c.z, c.w, q);
  gs(v[0], v[4], d.x, d.y, q); gs(v[1], v[5], d.x, d.y, q); gs(v[2], v[6], d.x, d.y, q); gs(v[3], v[7], d.x, d.y, q);
}

// Levels of the next middle round when LEFT levels remain (4 -> 2 + 2, so that
// no round is a lone radix-2 when it can be avoided).
template <int LEFT>
__host__ __device__ constexpr int middle_levels() { return LEFT == 4 ? 2 : (LEFT < 3 ? LEFT : 3); }

// Thread-to-set map of a middle round (run by the threads b < N/8, each
// taking sets b, b + N/8, ...): set sb -> (group i, offset o), INNER = the
// offset range (u forward, t0 inverse). The radix-8 round whose sets are
// 64i + o + 8k (INNER = 8) takes i = warp + (N/256) ((sb >> 3) & 3), which
// spreads a warp over 4 groups 16 apart; every other round maps
// sb = i INNER + o.
template <int R, uint32_t INNER, uint32_t N>
__device__ __forceinline__ void set_of(uint32_t sb, uint32_t &i, uint32_t &o) {
  if constexpr (R == 3 && INNER == 8 && N >= 256) {
    o = sb & 7;
    i = (sb >> 5) + (N >> 8) * ((sb >> 3) & 3);
  } else {
    i = sb / INNER;
    o = sb % INNER;
  }
}

template <int LOGN, int R, int LVL>
__device__ __forceinline__ void fwd_middle(uint32_t *buf, const Limb &T, uint32_t b) {
  constexpr uint32_t N = 1u << LOGN, S = N >> 3, M0 = 1u << LVL, U = N >> (LVL + R);
#pragma unroll
  for (uint32_t t = 0; t < (N >> R) / S; ++t) {
    uint32_t i, o;
    set_of<R, U, N>(b + t * S, i, o);
    uint32_t *p = buf + pad((i << R) * U + o);
    uint32_t v[8];
#pragma unroll
    for (uint32_t k = 0; k < (1u << R); ++k) v[k] = p[k * U + ((k * U) >> 7)];
    fwd_round<R, M0>(v, T.fw, i, T.q);
#pragma unroll
    for (uint32_t k = 0; k < (1u << R); ++k) p[k * U + ((k * U) >> 7)] = v[k];
  }
}

template <int LOGN, int R, int G>
__device__ __forceinline__ void inv_middle(uint32_t *buf, const Limb &T, uint32_t b) {
  constexpr uint32_t N = 1u << LOGN, S = N >> 3, T0 = 1u << G;
#pragma unroll
  for (uint32_t t = 0; t < (N >> R) / S; ++t) {
    uint32_t i, o;
    set_of<R, T0, N>(b + t * S, i, o);
    uint32_t *p = buf + pad((i << R) * T0 + o);
    uint32_t v[8];
#pragma unroll
    for (uint32_t k = 0; k < (1u << R); ++k) v[k] = p[k * T0 + ((k * T0) >> 7)];
    inv_round<R, N / (2 * T0)>(v, T.iv, i, T.q);
#pragma unroll
    for (uint32_t k = 0; k < (1u << R); ++k) p[k * T0 + ((k * T0) >> 7)] = v[k];
  }
}

template <int LOGN, int LVL, int P>
__device__ __forceinline__ void fwd_middles(uint32_t *const (&buf)[P], const Limb &T, uint32_t b, bool act) {
  constexpr int END = LOGN >= 6 ? LOGN - 3 : LOGN;
  if constexpr (LVL < END) {
    constexpr int R = middle_levels<END - LVL>();
    if (act) {
#pragma unroll
      for (int p = 0; p < P; ++p) fwd_middle<LOGN, R, LVL>(buf[p], T, b);
    }
    __syncthreads();
    fwd_middles<LOGN, LVL + R, P>(buf, T, b, act);
  }
}

template <int LOGN, int G, int P>
__device__ __forceinline__ void inv_middles(uint32_t *const (&buf)[P], const Limb &T, uint32_t b, bool act) {
  constexpr int END = LOGN >= 6 ? LOGN - 3 : LOGN;
  if constexpr (G < END) {
    constexpr int R = middle_levels<END - G>();
    if (act) {
#pragma unroll
      for (int p = 0; p < P; ++p) inv_middle<LOGN, R, G>(buf[p], T, b);
    }
    __syncthreads();
    inv_middles<LOGN, G + R, P>(buf, T, b, act);
  }
}

// Forward NTT of P polynomials of one limb (one padded buffer of padn(N) words
// each). In: v[p][k] = coefficient b + (N/8) k, values < 16q. Out: v[p][e] =
// slot b + (N/8) e, values in [0, 14q) (lazy: congruent mod q, not reduced). Every thread of the CTA must call it
// (it holds __syncthreads); act = b < N/8. The buffers are free again once
// the next barrier of the CTA has passed.
template <int LOGN, int P>
__device__ __forceinline__ void forward(uint32_t (&v)[P][8], uint32_t *const (&buf)[P], const Limb &T, uint32_t b,
                                        bool act) {
  constexpr uint32_t N = 1u << LOGN, S = N >> 3;
  if (act) {
    const uint32_t base = pad(b);
#pragma unroll
    for (int p = 0; p < P; ++p) {
      fwd_round<3, 1>(v[p], T.fw, 0, T.q);
#pragma unroll
      for (uint32_t k = 0; k < 8; ++k) buf[p][base + k * S + ((k * S) >> 7)] = v[p][k];
    }
  }
  __syncthreads();
  fwd_middles<LOGN, 3, P>(buf, T, b, act);
  if (!act) return;
  if constexpr (LOGN >= 6) {
    const uint32_t i = brev(b, LOGN - 3);
    const uint32_t base = pad(8 * i);
#pragma unroll
    for (int p = 0; p < P; ++p) {
      uint32_t w[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) w[k] = buf[p][base + k];
      fwd_round_last(w, T.fw_last + 8 * b, T.q);
      // position 8i + k holds slot (N/8) brv3(k) + b
      v[p][0] = w[0]; v[p][1] = w[4]; v[p][2] = w[2]; v[p][3] = w[6];
      v[p][4] = w[1]; v[p][5] = w[5]; v[p][6] = w[3]; v[p][7] = w[7];
    }
  } else {
#pragma unroll
    for (int p = 0; p < P; ++p)
#pragma unroll
      for (uint32_t e = 0; e < 8; ++e) v[p][e] = buf[p][pad(brev(b + e * S, LOGN))];
  }
}

// Inverse NTT of P polynomials of one limb. In: v[p][e] = slot b + (N/8) e,
// values < 2q. Out: the canonical coefficients in buf[p] (natural order,
// padded layout), visible to the whole CTA on return.
template <int LOGN, int P>
__device__ __forceinline__ void inverse(uint32_t (&v)[P][8], uint32_t *const (&buf)[P], const Limb &T, uint32_t b,
                                        bool act) {
  constexpr uint32_t N = 1u << LOGN, S = N >> 3;
  if (act) {
    const uint32_t i = brev(b, LOGN - 3);
    const uint32_t base = pad(8 * i);
#pragma unroll
    for (int p = 0; p < P; ++p) {
      // position 8i + k holds slot (N/8) brv3(k) + b
      uint32_t w[8] = {v[p][0], v[p][4], v[p][2], v[p][6], v[p][1], v[p][5], v[p][3], v[p][7]};
      if constexpr (LOGN >= 6) inv_round_first(w, T.iv_first + 8 * b, T.q);
      else inv_round<3, (N >> 1)>(w, T.iv, i, T.q);
#pragma unroll
      for (int k = 0; k < 8; ++k) buf[p][base + k] = w[k];
    }
  }
  __syncthreads();
  inv_middles<LOGN, 3, P>(buf, T, b, act);
  if (act) {
    const uint32_t base = pad(b);
#pragma unroll
    for (int p = 0; p < P; ++p) {
      uint32_t w[8];
#pragma unroll
      for (uint32_t k = 0; k < 8; ++k) w[k] = buf[p][base + k * S + ((k * S) >> 7)];
      if constexpr (LOGN >= 6) inv_round<3, 4>(w, T.iv, 0, T.q);
#pragma unroll
      for (uint32_t k = 0; k < 8; ++k)
        buf[p][base + k * S + ((k * S) >> 7)] = shoup(w[k], T.n_inv, T.n_inv_s, T.q);
    }
  }
  __syncthreads();
}

// Dcp, first half: y = x + O for the centred CRT value x in (-Q/2, Q/2] of one
// coefficient with residues (r0 mod q0, r1 mod q1) (Garner for L = 2), where
// O = sum_{k < ell-1} (z/2) z^k. The balanced base-z digits of x are then
// plain fields of y: d_k = ((y >> 22k) mod z) - z/2 for k < ell - 1, and the
// top digit is y >> 22 (ell - 1) (arithmetic shift).
__device__ __forceinline__ int64_t dcp_offset_value(const Ring &R, uint32_t r0, uint32_t r1) {
  uint64_t x;
  if (R.L == 1) {
    x = r0;
  } else {
    const uint32_t q1 = R.limb[1].q;
    const uint32_t k = shoup(sub_mod(r1, csub(r0, q1), q1), R.q0_inv, R.q0_inv_s, q1);   // q0 < 2 q1
    x = (uint64_t)r0 + (uint64_t)R.limb[0].q * k;
  }
  const int64_t xc = x > R.half_Q ? (int64_t)(x - R.Q) : (int64_t)x;
  return xc + (int64_t)R.offset;
}

// Dcp, second half: digit i of y, reduced mod q (|d| < q).
__device__ __forceinline__ uint32_t dcp_digit(int64_t y, uint32_t i, uint32_t ell, uint32_t q) {
  constexpr int32_t z = 1 << LOG_BASE;
  int32_t d;
  if (i + 1 == ell) {
    d = (int32_t)(y >> (LOG_BASE * i));
  } else {
    d = (int32_t)(((uint64_t)y >> (LOG_BASE * i)) & (uint64_t)(z - 1)) - z / 2;
  }
  return (uint32_t)d + (d < 0 ? q : 0u);
}

__device__ __forceinline__ void prefetch_l1(const void *p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// Thread-block cluster helpers: the two limb CTAs of a tree node exchange
// coefficient residues through distributed shared memory.
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// Shared-memory address of the same offset in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t peer_addr(const void *local, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(local)), "r"(rank));
  return r;
}
__device__ __forceinline__ uint32_t ld_peer(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

}  // namespace ntt

// Host side (ring_tables.cu): twiddle tables on the current device, built once
// per (device, N, primes) and kept for the process.
int ring_tables(const gpir_params_t *params, ntt::Ring *out);

}  // namespace gpir
