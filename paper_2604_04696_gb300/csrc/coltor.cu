// ColTor: the column tournament that follows RowSel (GPIR paper Sec. 2.2,
// "ColTor"), with the external product of Sec. 2.5.1.
//
// For every client, log2(D1) stages halve the client's D1 ciphertexts: stage s
// pairs the stage inputs (2k, 2k+1) and keeps
//     ct_{2k} + RGSW_s [x] (ct_{2k+1} - ct_{2k}).
// The external product of an RGSW ciphertext (2 ell rows of two polynomials)
// with a ciphertext (c_0, c_1), everything in the NTT domain:
//   1. inverse NTT of c_0 and c_1, limb by limb;
//   2. Dcp: every coefficient is rebuilt from its limbs (CRT) as x in [0, Q),
//      centred to (-Q/2, Q/2], and split into balanced base-2^22 digits
//      x = sum_{i<ell} d_i 2^(22 i), d_i in [-2^21, 2^21) (the last digit takes
//      the rest);
//   3. forward NTT of the 2 ell digit polynomials (digits reduced mod q_l);
//   4. out_r = sum_{p, i} NTT(d_{p,i}) (.) rgsw[p ell + i][r], r in {0, 1}.
//
// GPU mapping (stage-level kernel, as the paper's Sec. 4.1.2 argues for): one
// CTA per tree node does the whole node in shared memory, so the 2 ell digit
// polynomials never leave the SM. The NTT is the negacyclic Cooley-Tukey /
// Gentleman-Sande butterfly network with psi powers in bit-reversed order
// (Longa and Naehrig, "Speeding up the Number Theoretic Transform for Faster
// Ideal Lattice-Based Cryptography", CANS 2016), with an explicit bit-reversal
// pass so that both transforms take and return natural slot order:
//     A_s = sum_j a_j psi^((2s+1) j) mod q,  psi = g^((q-1)/2N),
// g the smallest generator of Z_q^* (the same NTT form RowSel's data is in).
// Twiddle products use Shoup's precomputed quotients; data products use the
// Barrett reduction of the RowSel kernels.

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace gpir {
namespace {

constexpr int CT_THREADS = 512;                   // per tree node
constexpr uint32_t CT_MAX_N = 4096;
constexpr uint32_t CT_MAX_LIMBS = 2;
constexpr int CT_LOG_BASE = 22;                   // gadget base z = 2^22 (the paper's)

// Per limb: psi^brv(k), psi^-brv(k) and their Shoup quotients floor(w 2^32 / q).
struct NttLimb {
  const uint32_t *fw, *fw_s, *iv, *iv_s;
  uint32_t q, n_inv, n_inv_s, pad;
  uint64_t mu;                                    // floor(2^64 / q) for Barrett
};

struct ColTorParams {
  uint32_t L, N, logn, ell, nodes_per_client, d_in;
  uint64_t Q;                                     // prod q_l (< 2^56)
  uint32_t q0_inv_mod_q1;                         // CRT (L = 2)
  uint32_t pad;
  const uint32_t *in;                             // [B][d_in][2][L][N]
  const uint32_t *rgsw;                           // [B][stages][2 ell][2][L][N]
  uint32_t stage, stages;
  uint32_t *out;                                  // [B][d_in / 2][2][L][N]
  NttLimb limb[CT_MAX_LIMBS];
};

__device__ __forceinline__ uint32_t add_mod(uint32_t a, uint32_t b, uint32_t q) {
  const uint32_t s = a + b;
  return s >= q ? s - q : s;
}
__device__ __forceinline__ uint32_t sub_mod(uint32_t a, uint32_t b, uint32_t q) {
  return a >= b ? a - b : a + q - b;
}
// a * w mod q with w' = floor(w 2^32 / q) (Shoup): result in [0, q).
__device__ __forceinline__ uint32_t mul_shoup(uint32_t a, uint32_t w, uint32_t ws, uint32_t q) {
  const uint32_t t = __umulhi(a, ws);
  uint32_t r = a * w - t * q;
  return r >= q ? r - q : r;
}
__device__ __forceinline__ uint32_t mul_mod(uint32_t a, uint32_t b, uint32_t q, uint64_t mu) {
  return reduce64((uint64_t)a * b, q, mu);
}

// Forward NTT of one limb in shared memory, natural order in and out.
__device__ void ntt_forward(uint32_t *a, const NttLimb &T, uint32_t N, uint32_t logn) {
  const uint32_t q = T.q;
  for (uint32_t m = 1, t = N >> 1; m < N; m <<= 1, t >>= 1) {
    for (uint32_t b = threadIdx.x; b < (N >> 1); b += CT_THREADS) {
      const uint32_t i = b / t, j = 2 * i * t + (b % t);
      const uint32_t w = __ldg(&T.fw[m + i]), ws = __ldg(&T.fw_s[m + i]);
      const uint32_t u = a[j], v = mul_shoup(a[j + t], w, ws, q);
      a[j] = add_mod(u, v, q);
      a[j + t] = sub_mod(u, v, q);
    }
    __syncthreads();
  }
  // bit-reversed -> natural order
  for (uint32_t k = threadIdx.x; k < N; k += CT_THREADS) {
    const uint32_t r = __brev(k) >> (32 - logn);
    if (k < r) {
      const uint32_t x = a[k];
      a[k] = a[r];
      a[r] = x;
    }
  }
  __syncthreads();
}

// Inverse NTT of one limb in shared memory, natural order in and out.
__device__ void ntt_inverse(uint32_t *a, const NttLimb &T, uint32_t N, uint32_t logn) {
  const uint32_t q = T.q;
  for (uint32_t k = threadIdx.x; k < N; k += CT_THREADS) {
    const uint32_t r = __brev(k) >> (32 - logn);
    if (k < r) {
      const uint32_t x = a[k];
      a[k] = a[r];
      a[r] = x;
    }
  }
  __syncthreads();
  for (uint32_t h = N >> 1, t = 1; h >= 1; h >>= 1, t <<= 1) {
    for (uint32_t b = threadIdx.x; b < (N >> 1); b += CT_THREADS) {
      const uint32_t i = b / t, j = 2 * i * t + (b % t);
      const uint32_t w = __ldg(&T.iv[h + i]), ws = __ldg(&T.iv_s[h + i]);
      const uint32_t u = a[j], v = a[j + t];
      a[j] = add_mod(u, v, q);
      a[j + t] = mul_shoup(sub_mod(u, v, q), w, ws, q);
    }
    __syncthreads();
  }
  for (uint32_t k = threadIdx.x; k < N; k += CT_THREADS) a[k] = mul_shoup(a[k], T.n_inv, T.n_inv_s, q);
  __syncthreads();
}

// Digit i of the balanced base-2^22 decomposition of the centred CRT value of
// coefficient j (limbs r[0..L-1]), as a signed integer.
__device__ __forceinline__ int64_t centred_value(const ColTorParams &p, uint32_t r0, uint32_t r1) {
  uint64_t x;
  if (p.L == 1) {
    x = r0;
  } else {
    // Garner: x = r0 + q0 * ((r1 - r0) * q0^-1 mod q1), in [0, q0 q1)
    const NttLimb &T1 = p.limb[1];
    const uint32_t d = sub_mod(r1, r0 % T1.q, T1.q);
    const uint32_t k = mul_mod(d, p.q0_inv_mod_q1, T1.q, T1.mu);
    x = (uint64_t)r0 + (uint64_t)p.limb[0].q * k;
  }
  return x > (p.Q >> 1) ? (int64_t)x - (int64_t)p.Q : (int64_t)x;
}

__device__ __forceinline__ int64_t digit_of(int64_t x, uint32_t i, uint32_t ell) {
  constexpr int64_t z = (int64_t)1 << CT_LOG_BASE;
  for (uint32_t k = 0;; ++k) {
    if (k + 1 == ell) return x;                   // the last digit takes the rest
    int64_t r = x & (z - 1);
    if (r >= z / 2) r -= z;
    if (k == i) return r;
    x = (x - r) >> CT_LOG_BASE;                   // exact: x - r is a multiple of z
  }
}

// One tree node per CTA: node (client c, k) of the stage.
template <int L>
__global__ void __launch_bounds__(CT_THREADS) coltor_stage_kernel(const __grid_constant__ ColTorParams p) {
  extern __shared__ __align__(16) uint32_t sm[];
  const uint32_t N = p.N;
  uint32_t *coef = sm;                             // [2][L][N]: hi - lo, then its coefficients
  uint32_t *work = sm + 2 * L * N;                 // [L][N]: one digit polynomial
  constexpr int PPT = CT_MAX_N / CT_THREADS;       // points per thread (at most)

  const uint32_t c = blockIdx.x / p.nodes_per_client, k = blockIdx.x % p.nodes_per_client;
  const size_t ct_words = (size_t)2 * L * N;
  const uint32_t *lo = p.in + ((size_t)c * p.d_in + 2 * k) * ct_words;
  const uint32_t *hi = lo + ct_words;
  const uint32_t *rgsw = p.rgsw + ((size_t)c * p.stages + p.stage) * (2 * p.ell) * ct_words;

  // 1. d = hi - lo, then inverse NTT of its 2 L limb polynomials
  for (uint32_t x = threadIdx.x; x < 2 * L * N; x += CT_THREADS) {
    const uint32_t l = (x / N) % L;
    coef[x] = sub_mod(__ldg(&hi[x]), __ldg(&lo[x]), p.limb[l].q);
  }
  __syncthreads();
  for (int pl = 0; pl < 2 * L; ++pl) ntt_inverse(coef + pl * N, p.limb[pl % L], N, p.logn);

  uint32_t acc[2][L][PPT];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int l = 0; l < L; ++l)
#pragma unroll
      for (int e = 0; e < PPT; ++e) acc[r][l][e] = 0;

  // 2-4. per polynomial p and digit i: Dcp, forward NTT, multiply-accumulate
  for (uint32_t pp = 0; pp < 2; ++pp) {
    for (uint32_t i = 0; i < p.ell; ++i) {
      for (uint32_t j = threadIdx.x; j < N; j += CT_THREADS) {
        const uint32_t r0 = coef[(pp * L + 0) * N + j];
        const uint32_t r1 = L > 1 ? coef[(pp * L + (L - 1)) * N + j] : 0u;
        const int64_t d = digit_of(centred_value(p, r0, r1), i, p.ell);
#pragma unroll
        for (int l = 0; l < L; ++l) {
          const int64_t q = p.limb[l].q;
          work[l * N + j] = (uint32_t)(d < 0 ? d + q : d);
        }
      }
      __syncthreads();
#pragma unroll
      for (int l = 0; l < L; ++l) ntt_forward(work + l * N, p.limb[l], N, p.logn);
      const uint32_t *row = rgsw + (size_t)(pp * p.ell + i) * ct_words;
#pragma unroll
      for (int e = 0; e < PPT; ++e) {
        const uint32_t j = threadIdx.x + e * CT_THREADS;
        if (j < N) {
#pragma unroll
          for (int l = 0; l < L; ++l) {
            const NttLimb &T = p.limb[l];
            const uint32_t dv = work[l * N + j];
#pragma unroll
            for (int r = 0; r < 2; ++r)
              acc[r][l][e] = add_mod(acc[r][l][e], mul_mod(dv, __ldg(&row[((size_t)r * L + l) * N + j]), T.q, T.mu), T.q);
          }
        }
      }
      __syncthreads();   // work is rewritten by the next digit
    }
  }

  // 5. out = lo + RGSW [x] d
  uint32_t *out = p.out + ((size_t)c * p.nodes_per_client + k) * ct_words;
#pragma unroll
  for (int e = 0; e < PPT; ++e) {
    const uint32_t j = threadIdx.x + e * CT_THREADS;
    if (j < N) {
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int l = 0; l < L; ++l) {
          const size_t x = ((size_t)r * L + l) * N + j;
          out[x] = add_mod(__ldg(&lo[x]), acc[r][l][e], p.limb[l].q);
        }
    }
  }
}

// ---- host side ----------------------------------------------------------------

uint64_t pow_mod(uint64_t b, uint64_t e, uint64_t q) {
  uint64_t r = 1;
  b %= q;
  while (e) {
    if (e & 1) r = (unsigned __int128)r * b % q;
    b = (unsigned __int128)b * b % q;
    e >>= 1;
  }
  return r;
}

// Smallest generator of Z_q^* (q prime).
uint64_t smallest_generator(uint64_t q) {
  std::vector<uint64_t> f;
  uint64_t n = q - 1;
  for (uint64_t d = 2; d * d <= n; ++d)
    if (n % d == 0) {
      f.push_back(d);
      while (n % d == 0) n /= d;
    }
  if (n > 1) f.push_back(n);
  for (uint64_t g = 2;; ++g) {
    bool ok = true;
    for (uint64_t x : f)
      if (pow_mod(g, (q - 1) / x, q) == 1) {
        ok = false;
        break;
      }
    if (ok) return g;
  }
}

uint32_t bit_reverse(uint32_t k, uint32_t bits) {
  uint32_t r = 0;
  for (uint32_t i = 0; i < bits; ++i) r |= ((k >> i) & 1u) << (bits - 1 - i);
  return r;
}

struct DeviceTables {
  uint32_t *mem = nullptr;                          // 4 tables per limb, N words each
  NttLimb limb[CT_MAX_LIMBS];
};

std::mutex g_ct_mu;
std::map<std::tuple<int, uint32_t, uint32_t, uint32_t>, DeviceTables> g_tables;   // (device, N, q0, q1)
std::map<std::pair<int, cudaStream_t>, std::pair<uint32_t *, size_t>> g_ct_ws;

int get_tables(int dev, const gpir_params &prm, DeviceTables **out) {
  const uint32_t N = prm.n, L = prm.num_limbs;
  const auto key = std::make_tuple(dev, N, prm.primes[0], L > 1 ? prm.primes[1] : 0u);
  auto it = g_tables.find(key);
  if (it != g_tables.end()) {
    *out = &it->second;
    return GPIR_OK;
  }
  uint32_t logn = 0;
  while ((1u << logn) < N) ++logn;
  std::vector<uint32_t> host((size_t)4 * L * N);
  DeviceTables t;
  for (uint32_t l = 0; l < L; ++l) {
    const uint64_t q = prm.primes[l];
    const uint64_t psi = pow_mod(smallest_generator(q), (q - 1) / (2 * N), q);
    const uint64_t psi_inv = pow_mod(psi, q - 2, q);
    uint32_t *fw = host.data() + (size_t)(4 * l + 0) * N, *fws = fw + N, *iv = fws + N, *ivs = iv + N;
    for (uint32_t k = 0; k < N; ++k) {
      const uint32_t e = bit_reverse(k, logn);
      const uint64_t w = pow_mod(psi, e, q), wi = pow_mod(psi_inv, e, q);
      fw[k] = (uint32_t)w;
      fws[k] = (uint32_t)((w << 32) / q);
      iv[k] = (uint32_t)wi;
      ivs[k] = (uint32_t)((wi << 32) / q);
    }
    const uint64_t ninv = pow_mod(N, q - 2, q);
    t.limb[l].q = (uint32_t)q;
    t.limb[l].n_inv = (uint32_t)ninv;
    t.limb[l].n_inv_s = (uint32_t)((ninv << 32) / q);
    t.limb[l].pad = 0;
    t.limb[l].mu = ~0ull / q;
  }
  cudaError_t e = cudaMalloc(&t.mem, host.size() * 4);
  if (e != cudaSuccess) return set_cuda_error(e);
  e = cudaMemcpy(t.mem, host.data(), host.size() * 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(t.mem);
    return set_cuda_error(e);
  }
  for (uint32_t l = 0; l < L; ++l) {
    const uint32_t *base = t.mem + (size_t)4 * l * N;
    t.limb[l].fw = base;
    t.limb[l].fw_s = base + N;
    t.limb[l].iv = base + 2 * N;
    t.limb[l].iv_s = base + 3 * N;
  }
  auto r = g_tables.emplace(key, t);
  *out = &r.first->second;
  return GPIR_OK;
}

int get_workspace(int dev, cudaStream_t s, size_t words, uint32_t **out) {
  auto &w = g_ct_ws[std::make_pair(dev, s)];
  if (w.second < words) {
    if (w.first) {
      cudaStreamSynchronize(s);
      cudaFree(w.first);
      w.first = nullptr;
      w.second = 0;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) return GPIR_EINVAL;
    cudaError_t e = cudaMalloc(&w.first, words * 4);
    if (e != cudaSuccess) {
      w.first = nullptr;
      return set_cuda_error(e);
    }
    w.second = words;
  }
  *out = w.first;
  return GPIR_OK;
}

}  // namespace
}  // namespace gpir

extern "C" int gpir_coltor_gadget_digits(const gpir_params_t *params) {
  if (!params) return GPIR_EINVAL;
  unsigned __int128 Q = 1;
  for (uint32_t l = 0; l < params->num_limbs; ++l) Q *= params->primes[l];
  uint32_t bits = 0;
  for (unsigned __int128 v = Q - 1; v; v >>= 1) ++bits;
  return (int)((bits + gpir::CT_LOG_BASE - 1) / gpir::CT_LOG_BASE);
}

extern "C" int gpir_coltor(const gpir_params_t *params, uint32_t batch, uint32_t d1, const uint32_t *ct_dev,
                           const uint32_t *rgsw_dev, uint32_t *out_dev, void *stream) {
  using namespace gpir;
  if (!params || !ct_dev || !rgsw_dev || !out_dev || batch == 0 || d1 < 2 || (d1 & (d1 - 1)) != 0)
    return GPIR_EINVAL;
  const uint32_t L = params->num_limbs, N = params->n;
  if (L > CT_MAX_LIMBS || N > CT_MAX_N) return GPIR_ENOTSUP;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_cuda_error(e);
  std::lock_guard<std::mutex> lk(g_ct_mu);
  DeviceTables *tab = nullptr;
  int rc = get_tables(dev, *params, &tab);
  if (rc != GPIR_OK) return rc;
  uint32_t logn = 0;
  while ((1u << logn) < N) ++logn;
  uint32_t stages = 0;
  while ((1u << stages) < d1) ++stages;
  const size_t ct_words = (size_t)2 * L * N;
  // ping-pong buffers for the intermediate stages: d1/2 and d1/4 ciphertexts per client
  uint32_t *ws = nullptr;
  const size_t half = (size_t)batch * (d1 / 2) * ct_words;
  if (stages > 1) {
    rc = get_workspace(dev, s, half + half / 2, &ws);
    if (rc != GPIR_OK) return rc;
  }
  ColTorParams p;
  memset(&p, 0, sizeof(p));
  p.L = L;
  p.N = N;
  p.logn = logn;
  p.ell = (uint32_t)gpir_coltor_gadget_digits(params);
  p.Q = 1;
  for (uint32_t l = 0; l < L; ++l) p.Q *= params->primes[l];
  p.q0_inv_mod_q1 = L > 1 ? (uint32_t)pow_mod(params->primes[0] % params->primes[1], params->primes[1] - 2,
                                               params->primes[1])
                          : 0u;
  p.rgsw = rgsw_dev;
  p.stages = stages;
  for (uint32_t l = 0; l < L; ++l) p.limb[l] = tab->limb[l];
  const size_t smem = (size_t)(2 * L + L) * N * 4;
  static bool attr_done[2] = {false, false};
  if (!attr_done[L - 1]) {
    e = L == 1 ? cudaFuncSetAttribute(coltor_stage_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(3 * CT_MAX_N * 4))
               : cudaFuncSetAttribute(coltor_stage_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(6 * CT_MAX_N * 4));
    if (e != cudaSuccess) return set_cuda_error(e);
    attr_done[L - 1] = true;
  }
  const uint32_t *in = ct_dev;
  uint32_t d_in = d1;
  for (uint32_t st = 0; st < stages; ++st) {
    uint32_t *dst = (st + 1 == stages) ? out_dev : (st % 2 == 0 ? ws : ws + half);
    p.in = in;
    p.out = dst;
    p.d_in = d_in;
    p.stage = st;
    p.nodes_per_client = d_in / 2;
    const unsigned grid = batch * (d_in / 2);
    const int tr = trace_begin("coltor_stage", s);
    if (L == 1)
      coltor_stage_kernel<1><<<grid, CT_THREADS, smem, s>>>(p);
    else
      coltor_stage_kernel<2><<<grid, CT_THREADS, smem, s>>>(p);
    trace_end(tr, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_cuda_error(e);
    in = dst;
    d_in /= 2;
  }
  return GPIR_OK;
}
