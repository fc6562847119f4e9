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
// GPU mapping: stage-level kernels (Sec. 4.1.2): each tree node is done on
// chip, so the 2 ell digit polynomials never leave the SMs; one launch per
// stage. Thread b of a CTA (ntt::HALF threads, one limb) owns slots /
// coefficients b + (N/8) e (see ntt.cuh). Two cluster shapes, chosen per stage
// (Sec. 4.4):
//   - coltor_limb_kernel: one cluster of L CTAs per node, CTA l on limb l for
//     both input polynomials (2 inverse NTTs sharing their rounds, then the
//     2 ell digit transforms); used while the nodes fill the GPU;
//   - coltor_split_kernel: one cluster of 2L CTAs per node, CTA (p, l) on
//     polynomial p and limb l: the two polynomials go through separate inverse
//     NTTs, Dcps and forward NTTs and meet only in the final sum, so the split
//     doubles the parallelism of a stage without repeating any transform; used
//     for the late stages with few nodes.
// The exchanges go through distributed shared memory: the CRT of the Dcp reads
// the other limb's residues, and (split kernel) the polynomial-1 CTA hands its
// reduced partial sums to the polynomial-0 CTA. Shared memory per CTA: the
// limb's coefficients (padded), the Dcp offset values y = x + O of the owned
// coefficients of the current polynomial (one CRT per coefficient, after which
// each digit is a shift and a mask, see ntt.cuh), and two work buffers for the
// digit transforms, used in turn so that one digit's last round and the next
// digit's first round need no barrier between them: 98.8 KB (limb kernel) or
// 82.3 KB (split kernel) at N = 4096, two CTAs per SM, so that their phases
// (transform-bound, load-bound) overlap. The multiply-accumulate keeps 64-bit
// sums in registers: each of the at most 2 ell <= 6 terms is below
// 14q * q < 2^60 (the forward transform's lazy range times a key residue), so
// the sum stays below 2^63 and one Barrett reduction per output finishes it.

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <map>
#include <mutex>

#include "common.cuh"
#include "internal.h"
#include "ntt.cuh"

namespace gpir {
namespace {

struct ColTorParams {
  ntt::Ring ring;
  const uint32_t *in;                             // [B][d_in][2][L][N]
  const uint32_t *rgsw;                           // [B][stages][2 ell][2][L][N]
  uint32_t *out;                                  // [B][d_in / 2][2][L][N]
  uint32_t d_in, nodes_per_client, stage, stages;
};

template <int L, int LOGN>
__global__ void __launch_bounds__(ntt::HALF, 2) coltor_limb_kernel(const __grid_constant__ ColTorParams p) {
  using namespace ntt;
  constexpr uint32_t N = 1u << LOGN, S = N >> 3, PN = padn(N);
  extern __shared__ __align__(16) uint32_t sm[];
  const Ring &R = p.ring;
  const uint32_t ell = R.ell;
  const uint32_t h = L > 1 ? cluster_rank() : 0u;  // this CTA's limb
  const uint32_t b = threadIdx.x;
  const bool act = b < S;
  const Limb &T = R.limb[h];
  const uint32_t q = T.q;
  uint32_t *res = sm;                                             // [2][PN]: coefficients, limb h
  int64_t *ybuf = reinterpret_cast<int64_t *>(sm + 2 * PN);       // [N]: Dcp offset values
  uint32_t *work = sm + 2 * PN + 2 * N;                           // [2][PN]: two digit buffers

  const uint32_t node = blockIdx.x / L;
  const uint32_t c = node / p.nodes_per_client, k = node % p.nodes_per_client;
  const size_t ctw = (size_t)2 * L * N;
  const uint32_t *lo = p.in + ((size_t)c * p.d_in + 2 * k) * ctw;
  const uint32_t *hi = lo + ctw;
  const uint32_t *rgsw = p.rgsw + ((size_t)c * p.stages + p.stage) * (2 * ell) * ctw;

  // 1. hi - lo on the owned slots of limb h, then the inverse NTT of both polynomials
  {
    uint32_t v[2][8];
    if (act) {
#pragma unroll
      for (int pp = 0; pp < 2; ++pp)
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const size_t x = (size_t)(pp * L + h) * N + b + e * S;
          v[pp][e] = sub_mod(__ldg(hi + x), __ldg(lo + x), q);
        }
    }
    uint32_t *const bufs[2] = {res, res + PN};
    inverse<LOGN, 2>(v, bufs, T, b, act);
  }
  if constexpr (L > 1) {
    cluster_arrive();   // the other limb's residues are complete and visible after this pair
    cluster_wait();
  }
  const uint32_t peer = L > 1 ? peer_addr(res, h ^ 1u) : 0u;

  // 2-4. per polynomial: Dcp offset values of the owned coefficients (CRT over
  // both limbs), then per digit: digit residues, forward NTT, multiply-accumulate
  uint64_t acc[2][8];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int e = 0; e < 8; ++e) acc[r][e] = 0;
  uint32_t ping = 0;
  for (uint32_t pp = 0; pp < 2; ++pp) {
    if (act) {
#pragma unroll
      for (uint32_t kk = 0; kk < 8; ++kk) {
        const uint32_t j = pad(b) + kk * S + ((kk * S) >> 7);
        const uint32_t own = res[pp * PN + j];
        uint32_t r0 = own, r1 = 0u;
        if constexpr (L > 1) {
          const uint32_t other = ld_peer(peer + 4 * (pp * PN + j));
          r0 = h == 0 ? own : other;
          r1 = h == 0 ? other : own;
        }
        ybuf[b + kk * S] = dcp_offset_value(R, r0, r1);   // read back by this thread only
      }
    }
    if constexpr (L > 1) {
      if (pp == 1) cluster_arrive();   // done reading the other CTA's shared memory
    }
    for (uint32_t i = 0; i < ell; ++i) {
      uint32_t d[1][8];
      if (act) {
#pragma unroll
        for (uint32_t kk = 0; kk < 8; ++kk) d[0][kk] = dcp_digit(ybuf[b + kk * S], i, ell, q);
      }
      if (act && (b & 31) < 16) {   // the 16 key-row lines this warp multiplies with after the transform
        const uint32_t l = b & 31;
        prefetch_l1(rgsw + (size_t)(pp * ell + i) * ctw + (size_t)h * N + (b & ~31u) + (l >> 3) * (size_t)L * N + (l & 7) * S);
      }
      {
        uint32_t *const bufs[1] = {work + ping * PN};
        forward<LOGN, 1>(d, bufs, T, b, act);
      }
      ping ^= 1;
      if (act) {
        const uint32_t *row = rgsw + (size_t)(pp * ell + i) * ctw + (size_t)h * N + b;
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
          for (int e = 0; e < 8; ++e) acc[r][e] += (uint64_t)d[0][e] * __ldg(row + (size_t)r * L * N + e * S);
      }
    }
  }

  // 5. out = lo + RGSW [x] (hi - lo), limb h
  if (act) {
    uint32_t *out = p.out + ((size_t)c * p.nodes_per_client + k) * ctw;
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const size_t x = (size_t)(r * L + h) * N + b + e * S;
        out[x] = add_mod(__ldg(lo + x), reduce64(acc[r][e], q, T.mu), q);
      }
  }
  if constexpr (L > 1) cluster_wait();   // the other CTA has finished reading this CTA's residues
}

template <int LOGN>
constexpr size_t coltor_limb_smem() {
  constexpr uint32_t N = 1u << LOGN, PN = ntt::padn(N);
  return (size_t)(4 * PN + 2 * N) * 4;
}

template <int L, int LOGN>
__global__ void __launch_bounds__(ntt::HALF, 2) coltor_split_kernel(const __grid_constant__ ColTorParams p) {
  using namespace ntt;
  constexpr uint32_t N = 1u << LOGN, S = N >> 3, PN = padn(N);
  extern __shared__ __align__(16) uint32_t sm[];
  const Ring &R = p.ring;
  const uint32_t ell = R.ell;
  const uint32_t rank = cluster_rank();
  const uint32_t h = rank % L, pp = rank / L;       // this CTA's limb and input polynomial
  const uint32_t b = threadIdx.x;
  const bool act = b < S;
  const Limb &T = R.limb[h];
  const uint32_t q = T.q;
  uint32_t *res = sm;                                             // [PN]: coefficients of polynomial pp, limb h
  int64_t *ybuf = reinterpret_cast<int64_t *>(sm + PN + (PN & 1)); // [N]: Dcp offset values, then partial sums
  uint32_t *work = sm + PN + (PN & 1) + 2 * N;                    // [2][PN]: two digit buffers

  const uint32_t node = blockIdx.x / (2 * L);
  const uint32_t c = node / p.nodes_per_client, k = node % p.nodes_per_client;
  const size_t ctw = (size_t)2 * L * N;
  const uint32_t *lo = p.in + ((size_t)c * p.d_in + 2 * k) * ctw;
  const uint32_t *hi = lo + ctw;
  const uint32_t *rgsw = p.rgsw + ((size_t)c * p.stages + p.stage) * (2 * ell) * ctw;

  // 1. hi - lo on the owned slots of (pp, h), then its inverse NTT
  {
    uint32_t v[1][8];
    if (act) {
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const size_t x = (size_t)(pp * L + h) * N + b + e * S;
        v[0][e] = sub_mod(__ldg(hi + x), __ldg(lo + x), q);
      }
    }
    uint32_t *const bufs[1] = {res};
    inverse<LOGN, 1>(v, bufs, T, b, act);
  }
  cluster_arrive();   // every CTA's residues are complete and visible after this pair
  cluster_wait();

  // 2a. Dcp offset values of the owned coefficients of polynomial pp (CRT over the limbs)
  if (act) {
    const uint32_t peer = L > 1 ? peer_addr(res, (h ^ 1u) + L * pp) : 0u;
#pragma unroll
    for (uint32_t kk = 0; kk < 8; ++kk) {
      const uint32_t j = pad(b) + kk * S + ((kk * S) >> 7);
      const uint32_t own = res[j];
      uint32_t r0 = own, r1 = 0u;
      if constexpr (L > 1) {
        const uint32_t other = ld_peer(peer + 4 * j);
        r0 = h == 0 ? own : other;
        r1 = h == 0 ? other : own;
      }
      ybuf[b + kk * S] = dcp_offset_value(R, r0, r1);   // read back by this thread only
    }
  }
  cluster_arrive();   // done reading the other limb's residues

  // 2b-4. per digit: digit residues, forward NTT, multiply-accumulate with RGSW rows pp ell + i
  uint64_t acc[2][8];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int e = 0; e < 8; ++e) acc[r][e] = 0;
  uint32_t ping = 0;
  for (uint32_t i = 0; i < ell; ++i) {
    uint32_t d[1][8];
    if (act) {
#pragma unroll
      for (uint32_t kk = 0; kk < 8; ++kk) d[0][kk] = dcp_digit(ybuf[b + kk * S], i, ell, q);
    }
    if (act && (b & 31) < 16) {   // the 16 RGSW-row lines this warp multiplies with after the transform
      const uint32_t l = b & 31;
      prefetch_l1(rgsw + (size_t)(pp * ell + i) * ctw + (size_t)h * N + (b & ~31u) + (l >> 3) * (size_t)L * N +
                  (l & 7) * S);
    }
    {
      uint32_t *const bufs[1] = {work + ping * PN};
      forward<LOGN, 1>(d, bufs, T, b, act);
    }
    ping ^= 1;
    if (act) {
      const uint32_t *row = rgsw + (size_t)(pp * ell + i) * ctw + (size_t)h * N + b;
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int e = 0; e < 8; ++e) acc[r][e] += (uint64_t)d[0][e] * __ldg(row + (size_t)r * L * N + e * S);
    }
  }

  // 5. out = lo + (partial of polynomial 0) + (partial of polynomial 1), limb h: the
  // polynomial-1 CTA leaves its reduced partial sums (2N words) in its shared
  // memory, the polynomial-0 CTA adds them. They go where y was: every thread
  // read its last y values before the first barrier of the last transform.
  uint32_t *part = reinterpret_cast<uint32_t *>(ybuf);
  if (pp == 1 && act) {
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int e = 0; e < 8; ++e) part[(r * 8 + e) * S + b] = reduce64(acc[r][e], q, T.mu);
  }
  cluster_wait();     // pairs the arrive after step 2a
  cluster_arrive();   // the partial sums are written
  cluster_wait();
  if (pp == 0 && act) {
    const uint32_t peer = peer_addr(part, h + L);
    uint32_t *out = p.out + ((size_t)c * p.nodes_per_client + k) * ctw;
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const size_t x = (size_t)(r * L + h) * N + b + e * S;
        const uint32_t other = ld_peer(peer + 4 * ((r * 8 + e) * S + b));
        out[x] = add_mod(add_mod(__ldg(lo + x), reduce64(acc[r][e], q, T.mu), q), other, q);
      }
  }
  cluster_arrive();   // the polynomial-0 CTA has read the partial sums
  cluster_wait();
}

template <int LOGN>
constexpr size_t coltor_split_smem() {
  constexpr uint32_t N = 1u << LOGN, PN = ntt::padn(N);
  return (size_t)(PN + (PN & 1) + 2 * N + 2 * PN) * 4;
}

std::mutex g_ct_mu;
std::map<std::pair<int, cudaStream_t>, std::pair<uint32_t *, size_t>> g_ct_ws;

int get_workspace(int dev, cudaStream_t s, size_t words, uint32_t **out) {
  auto &w = g_ct_ws[std::make_pair(dev, s)];
  if (w.second < words) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) return GPIR_EINVAL;
    if (w.first) {
      cudaStreamSynchronize(s);
      cudaFree(w.first);
      w.first = nullptr;
      w.second = 0;
    }
    cudaError_t e = dev_malloc(reinterpret_cast<void **>(&w.first), words * 4);
    if (e != cudaSuccess) {
      w.first = nullptr;
      return set_cuda_error(e);
    }
    w.second = words;
  }
  *out = w.first;
  return GPIR_OK;
}

bool g_attr_done[64][2][ntt::MAX_LIMBS][ntt::MAX_LOGN + 1] = {};

// One stage. split: one cluster of 2L CTAs per node (polynomial x limb), else
// one cluster of L CTAs per node (limb).
template <int L, int LOGN>
int launch_stage(const ColTorParams &p, unsigned nodes, bool split, int dev, cudaStream_t s) {
  if (dev < 0 || dev >= 64) return GPIR_EINVAL;
  const size_t smem = split ? coltor_split_smem<LOGN>() : coltor_limb_smem<LOGN>();
  void (*kern)(ColTorParams) = split ? coltor_split_kernel<L, LOGN> : coltor_limb_kernel<L, LOGN>;
  if (!g_attr_done[dev][split][L - 1][LOGN]) {
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return set_cuda_error(e);
    g_attr_done[dev][split][L - 1][LOGN] = true;
  }
  const unsigned cl = split ? 2 * L : L;
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(nodes * cl);
  cfg.blockDim = dim3(ntt::HALF);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, p);
  return e == cudaSuccess ? GPIR_OK : set_cuda_error(e);
}

template <int L>
int launch_stage_n(const ColTorParams &p, unsigned nodes, bool split, int dev, cudaStream_t s) {
  switch (p.ring.logn) {
    case 4: return launch_stage<L, 4>(p, nodes, split, dev, s);
    case 5: return launch_stage<L, 5>(p, nodes, split, dev, s);
    case 6: return launch_stage<L, 6>(p, nodes, split, dev, s);
    case 7: return launch_stage<L, 7>(p, nodes, split, dev, s);
    case 8: return launch_stage<L, 8>(p, nodes, split, dev, s);
    case 9: return launch_stage<L, 9>(p, nodes, split, dev, s);
    case 10: return launch_stage<L, 10>(p, nodes, split, dev, s);
    case 11: return launch_stage<L, 11>(p, nodes, split, dev, s);
    case 12: return launch_stage<L, 12>(p, nodes, split, dev, s);
    default: return GPIR_ENOTSUP;
  }
}

}  // namespace
}  // namespace gpir

extern "C" int gpir_coltor_gadget_digits(const gpir_params_t *params) {
  if (!params) return GPIR_EINVAL;
  unsigned __int128 Q = 1;
  for (uint32_t l = 0; l < params->num_limbs; ++l) Q *= params->primes[l];
  uint32_t bits = 0;
  for (unsigned __int128 v = Q - 1; v; v >>= 1) ++bits;
  return (int)((bits + gpir::ntt::LOG_BASE - 1) / gpir::ntt::LOG_BASE);
}

extern "C" int gpir_coltor(const gpir_params_t *params, uint32_t batch, uint32_t d1, const uint32_t *ct_dev,
                           const uint32_t *rgsw_dev, uint32_t *out_dev, void *stream) {
  using namespace gpir;
  // every argument is checked here, on the host, before any CUDA call
  if (!params || !ct_dev || !rgsw_dev || !out_dev || batch == 0 || d1 < 2 || (d1 & (d1 - 1)) != 0)
    return GPIR_EINVAL;
  if (params->num_limbs < 1 || params->num_limbs > ntt::MAX_LIMBS || params->n < ntt::MIN_N || params->n > ntt::MAX_N)
    return GPIR_ENOTSUP;
  {
    const size_t ctw = (size_t)2 * params->num_limbs * params->n * 4;
    const uintptr_t i0 = (uintptr_t)ct_dev, i1 = i0 + (size_t)batch * d1 * ctw;
    const uintptr_t o0 = (uintptr_t)out_dev, o1 = o0 + batch * ctw;
    if (i0 < o1 && o0 < i1) return GPIR_EINVAL;   // the last stage reads ct_dev's results while writing out_dev
  }
  ntt::Ring ring;
  int rc = ring_tables(params, &ring);
  if (rc != GPIR_OK) return rc;
  const uint32_t L = ring.L, N = ring.N;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_cuda_error(e);
  std::lock_guard<std::mutex> lk(g_ct_mu);
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
  p.ring = ring;
  p.rgsw = rgsw_dev;
  p.stages = stages;
  const uint32_t *in = ct_dev;
  uint32_t d_in = d1;
  for (uint32_t st = 0; st < stages; ++st) {
    uint32_t *dst = (st + 1 == stages) ? out_dev : (st % 2 == 0 ? ws : ws + half);
    p.in = in;
    p.out = dst;
    p.d_in = d_in;
    p.stage = st;
    p.nodes_per_client = d_in / 2;
    const unsigned nodes = batch * (d_in / 2);
    // stage-aware choice (Sec. 4.4): the polynomial x limb split when its 2L
    // CTAs per node fit one wave (two CTAs per SM), the limb split otherwise.
    // Measured at N = 4096, L = 2: the split wins the 32-node stage (0.022 vs
    // 0.033 ms), ties at 64 nodes and loses from 128 nodes up.
    const bool split = (uint64_t)nodes * 2 * L <= 2ull * (uint64_t)sm_count();
    const int tr = trace_begin(split ? "coltor_stage_split" : "coltor_stage", s);
    rc = L == 1 ? launch_stage_n<1>(p, nodes, split, dev, s) : launch_stage_n<2>(p, nodes, split, dev, s);
    trace_end(tr, s);
    if (rc != GPIR_OK) return rc;
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_cuda_error(e);
    in = dst;
    d_in /= 2;
  }
  return GPIR_OK;
}
