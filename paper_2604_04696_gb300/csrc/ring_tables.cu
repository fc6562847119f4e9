// Twiddle and monomial tables of the negacyclic NTT (see ntt.cuh), built on the
// host once per (device, N, primes) and kept on the device for the process.

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "internal.h"
#include "ntt.cuh"

namespace gpir {
namespace {

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

uint32_t shoup_quotient(uint64_t w, uint64_t q) { return (uint32_t)((w << 32) / q); }

std::mutex g_mu;
std::map<std::tuple<int, uint32_t, uint32_t, uint32_t, uint32_t>, ntt::Ring> g_rings;

}  // namespace

static int ring_tables_impl(const gpir_params_t *params, ntt::Ring *out);

// The tables of one parameter set; GPIR_ENOMEM if host memory runs out (no
// exception leaves this function: it is called from the C ABI).
int ring_tables(const gpir_params_t *params, ntt::Ring *out) {
  try {
    return ring_tables_impl(params, out);
  } catch (...) {
    return GPIR_ENOMEM;
  }
}

static int ring_tables_impl(const gpir_params_t *params, ntt::Ring *out) {
  const uint32_t N = params->n, L = params->num_limbs;
  if (L < 1 || L > ntt::MAX_LIMBS || N < ntt::MIN_N || N > ntt::MAX_N) return GPIR_ENOTSUP;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_cuda_error(e);
  std::lock_guard<std::mutex> lk(g_mu);
  const auto key = std::make_tuple(dev, N, L, params->primes[0], L > 1 ? params->primes[1] : 0u);
  auto it = g_rings.find(key);
  if (it != g_rings.end()) {
    *out = it->second;
    return GPIR_OK;
  }
  uint32_t logn = 0;
  while ((1u << logn) < N) ++logn;
  // uint2 entries: fw [N], iv [N], mono [2N], fw_last [N/8][8], iv_first [N/8][8]
  const size_t per_limb = (size_t)6 * N;
  std::vector<uint2> host(per_limb * L);
  ntt::Ring R;
  memset(&R, 0, sizeof(R));
  R.L = L;
  R.N = N;
  R.logn = logn;
  R.Q = 1;
  for (uint32_t l = 0; l < L; ++l) {
    const uint64_t q = params->primes[l];
    R.Q *= q;
    const uint64_t psi = pow_mod(smallest_generator(q), (q - 1) / (2 * N), q);
    const uint64_t psi_inv = pow_mod(psi, q - 2, q);
    uint2 *fw = host.data() + per_limb * l, *iv = fw + N, *mono = iv + N;
    for (uint32_t k = 0; k < N; ++k) {
      const uint32_t r = bit_reverse(k, logn);
      const uint64_t w = pow_mod(psi, r, q), wi = pow_mod(psi_inv, r, q);
      fw[k] = make_uint2((uint32_t)w, shoup_quotient(w, q));
      iv[k] = make_uint2((uint32_t)wi, shoup_quotient(wi, q));
    }
    uint64_t m = 1;
    for (uint32_t k = 0; k < 2 * N; ++k) {
      mono[k] = make_uint2((uint32_t)m, shoup_quotient(m, q));
      m = m * psi_inv % q;
    }
    // per-thread copies for the bit-reversed rounds (ntt.cuh): thread b, set i = brv(b)
    uint2 *fwl = mono + 2 * N, *ivf = fwl + N;
    const uint32_t S = N / 8;
    for (uint32_t b = 0; b < S; ++b) {
      const uint32_t i = bit_reverse(b, logn - 3);
      uint2 *f = fwl + 8 * b, *v = ivf + 8 * b;
      f[0] = fw[S + i];
      f[1] = fw[2 * S + 2 * i];
      f[2] = fw[2 * S + 2 * i + 1];
      f[3] = make_uint2(0, 0);
      for (uint32_t k = 0; k < 4; ++k) f[4 + k] = fw[4 * S + 4 * i + k];
      for (uint32_t k = 0; k < 4; ++k) v[k] = iv[4 * S + 4 * i + k];
      v[4] = iv[2 * S + 2 * i];
      v[5] = iv[2 * S + 2 * i + 1];
      v[6] = iv[S + i];
      v[7] = make_uint2(0, 0);
    }
    const uint64_t ninv = pow_mod(N, q - 2, q);
    R.limb[l].q = (uint32_t)q;
    R.limb[l].n_inv = (uint32_t)ninv;
    R.limb[l].n_inv_s = shoup_quotient(ninv, q);
    R.limb[l].mu = ~0ull / q;
  }
  if (L == 2) {
    const uint64_t q1 = params->primes[1];
    const uint64_t inv = pow_mod(params->primes[0] % q1, q1 - 2, q1);
    R.q0_inv = (uint32_t)inv;
    R.q0_inv_s = shoup_quotient(inv, q1);
  }
  {
    unsigned __int128 Q = R.Q;
    uint32_t bits = 0;
    for (unsigned __int128 v = Q - 1; v; v >>= 1) ++bits;
    R.ell = (bits + ntt::LOG_BASE - 1) / ntt::LOG_BASE;
  }
  R.half_Q = R.Q / 2;
  R.offset = 0;
  for (uint32_t k = 0; k + 1 < R.ell; ++k) R.offset += (1ull << (ntt::LOG_BASE - 1)) << (ntt::LOG_BASE * k);
  uint2 *mem = nullptr;
  e = dev_malloc(reinterpret_cast<void **>(&mem), host.size() * sizeof(uint2));
  if (e != cudaSuccess) return set_cuda_error(e);
  e = cudaMemcpy(mem, host.data(), host.size() * sizeof(uint2), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(mem);
    return set_cuda_error(e);
  }
  for (uint32_t l = 0; l < L; ++l) {
    const uint2 *base = mem + per_limb * l;
    R.limb[l].fw = base;
    R.limb[l].iv = base + N;
    R.limb[l].mono = base + 2 * N;
    R.limb[l].fw_last = base + 4 * N;
    R.limb[l].iv_first = base + 5 * N;
  }
  g_rings.emplace(key, R);
  *out = R;
  return GPIR_OK;
}

}  // namespace gpir
