// ExpandQuery: the query-expansion tree before RowSel (GPIR paper Sec. 2.2,
// "ExpandQuery"), with the homomorphic substitution Subs of Sec. 2.5.1.
//
// For every client, J stages turn its query ciphertext into 2^J ciphertexts
// (the first n_out are kept). Node k of stage j takes ciphertext c = list[k]
// and writes
//     list[k]       = c + t
//     list[k + 2^j] = X^(-2^j) (c - t),     t = Subs(c, N/2^j + 1, evk_j).
// Subs(ct = (a, b), k): the automorphism tau_k (X -> X^k) of both polynomials,
// then key switching with Dcp on tau_k(a) only:
//     t = ( sum_i NTT(d_i) (.) evk[i][0],  tau_k(b) + sum_i NTT(d_i) (.) evk[i][1] ),
// d_i the balanced base-2^22 digits of the centred CRT value of tau_k(a)'s
// coefficients (inverse NTT first, forward NTT of each digit polynomial after).
//
// In the NTT domain tau_k is a permutation of the slots: slot s of tau_k(A)
// is A[s'] with 2s'+1 = (2s+1) k mod 2N, so the kernel gathers tau_k(a) and
// tau_k(b) while it loads them. The slot values of X^(-2^j) are
// psi^-((2s+1) 2^j mod 2N), read from a table.
//
// GPU mapping: stage-level kernels (Sec. 4.1.2), one launch per stage, the
// cluster shape chosen per stage (Sec. 4.4):
//   - expand_stage_kernel: one thread-block cluster of L CTAs per tree node,
//     CTA l on limb l, the CRT of the Dcp reading the other limb's residues
//     through distributed shared memory (see ntt.cuh and coltor.cu); about
//     81 KB of shared memory per CTA at N = 4096;
//   - expand_split_kernel: for stages with few nodes, L ell CTAs per node
//     (limb x digit), each repeating the inverse NTT and doing one digit.
// The tree runs in place in the output array: stage j reads list[k], k < 2^j,
// and writes list[k] and list[k + 2^j]; each CTA reads only its limb of
// list[k], and every such read comes before the barrier that precedes the
// writes of that limb. Only
// the outputs with index < n_out are computed at any stage (an intermediate
// list[k] feeds final outputs k, k + 2^(j+1), ..., so k < n_out is exactly the
// condition for it to be needed).

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "common.cuh"
#include "internal.h"
#include "ntt.cuh"

namespace gpir {
namespace {

struct ExpandParams {
  ntt::Ring ring;
  const uint32_t *query;                          // [B][2][L][N] (read by stage 0)
  const uint32_t *evk;                            // [B][J][ell][2][L][N]
  uint32_t *out;                                  // [B][n_out][2][L][N]
  uint32_t n_out, J, stage, nodes;                // nodes = min(2^stage, n_out) per client
  uint32_t ksub;                                  // N / 2^stage + 1
};

template <int L, int LOGN>
__global__ void __launch_bounds__(ntt::HALF, 2) expand_stage_kernel(const __grid_constant__ ExpandParams p) {
  using namespace ntt;
  constexpr uint32_t N = 1u << LOGN, S = N >> 3, PN = padn(N), MASK2N = 2 * N - 1;
  extern __shared__ __align__(16) uint32_t sm[];
  const Ring &R = p.ring;
  const uint32_t ell = R.ell;
  const uint32_t h = L > 1 ? cluster_rank() : 0u;  // this CTA's limb
  const uint32_t b = threadIdx.x;
  const bool act = b < S;
  const Limb &T = R.limb[h];
  const uint32_t q = T.q;
  uint32_t *res = sm;                                             // [PN]: coefficients of tau(a), limb h
  int64_t *ybuf = reinterpret_cast<int64_t *>(sm + PN + (PN & 1)); // [N]: Dcp offset values
  uint32_t *work = sm + PN + (PN & 1) + 2 * N;                    // [2][PN]: two digit buffers

  const uint32_t node = blockIdx.x / L;
  const uint32_t c = node / p.nodes, k = node % p.nodes;
  const size_t ctw = (size_t)2 * L * N;
  // Plain loads: at stages >= 1 this CTA overwrites (its limb of) its input at the end.
  const uint32_t *in = p.stage == 0 ? p.query + (size_t)c * ctw : p.out + ((size_t)c * p.n_out + k) * ctw;
  uint32_t *out0 = p.out + ((size_t)c * p.n_out + k) * ctw;
  const uint32_t k1 = k + (1u << p.stage);
  const bool has1 = k1 < p.n_out;
  uint32_t *out1 = p.out + ((size_t)c * p.n_out + k1) * ctw;
  const uint32_t *evk = p.evk + ((size_t)c * p.J + p.stage) * ell * ctw;

  // 1. tau(a) on the owned slots of limb h (a gather), then its inverse NTT
  {
    uint32_t v[1][8];
    if (act) {
#pragma unroll
      for (uint32_t e = 0; e < 8; ++e) {
        const uint32_t s = b + e * S;
        const uint32_t src = ((((2 * s + 1) * p.ksub) & MASK2N) - 1) >> 1;
        v[0][e] = in[(size_t)h * N + src];
      }
    }
    uint32_t *const bufs[1] = {res};
    inverse<LOGN, 1>(v, bufs, T, b, act);
  }
  if constexpr (L > 1) {
    cluster_arrive();   // the other limb's residues are complete and visible after this pair
    cluster_wait();
  }

  // 2a. Dcp offset values of the owned coefficients (CRT over both limbs)
  if (act) {
    const uint32_t peer = L > 1 ? peer_addr(res, h ^ 1u) : 0u;
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
  if constexpr (L > 1) cluster_arrive();   // done reading the other CTA's shared memory

  // 2b. per digit: digit residues, forward NTT, multiply-accumulate with the key rows
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
    if (act && (b & 31) < 16) {   // the 16 key-row lines this warp multiplies with after the transform
      const uint32_t l = b & 31;
      prefetch_l1(evk + (size_t)i * ctw + (size_t)h * N + (b & ~31u) + (l >> 3) * (size_t)L * N + (l & 7) * S);
    }
    {
      uint32_t *const bufs[1] = {work + ping * PN};
      forward<LOGN, 1>(d, bufs, T, b, act);
    }
    ping ^= 1;
    if (act) {
      const uint32_t *row = evk + (size_t)i * ctw + (size_t)h * N + b;
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int e = 0; e < 8; ++e) acc[r][e] += (uint64_t)d[0][e] * __ldg(row + (size_t)r * L * N + e * S);
    }
  }

  // 3. t = (a', tau(b) + b'); out0 = c + t, out1 = X^(-2^j) (c - t), limb h
  uint32_t ta[8], tb[8], ca[8], cb[8];
  if (act) {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      ta[e] = reduce64(acc[0][e], q, T.mu);
      tb[e] = reduce64(acc[1][e], q, T.mu);
    }
#pragma unroll
    for (uint32_t e = 0; e < 8; ++e) {
      const uint32_t s = b + e * S;
      const uint32_t src = ((((2 * s + 1) * p.ksub) & MASK2N) - 1) >> 1;
      tb[e] = add_mod(tb[e], in[(size_t)(L + h) * N + src], q);
      ca[e] = in[(size_t)h * N + s];
      cb[e] = in[(size_t)(L + h) * N + s];
    }
  }
  __syncthreads();   // every read of (limb h of) list[k] by this CTA precedes the writes below
  if (act) {
#pragma unroll
    for (uint32_t e = 0; e < 8; ++e) {
      const uint32_t s = b + e * S;
      out0[(size_t)h * N + s] = add_mod(ca[e], ta[e], q);
      out0[(size_t)(L + h) * N + s] = add_mod(cb[e], tb[e], q);
      if (has1) {
        const uint2 m = __ldg(T.mono + (((2 * s + 1) << p.stage) & MASK2N));
        out1[(size_t)h * N + s] = shoup(sub_mod(ca[e], ta[e], q), m.x, m.y, q);
        out1[(size_t)(L + h) * N + s] = shoup(sub_mod(cb[e], tb[e], q), m.x, m.y, q);
      }
    }
  }
  if constexpr (L > 1) cluster_wait();   // the other CTA has finished reading this CTA's residues
}

template <int LOGN>
constexpr size_t expand_smem() {
  constexpr uint32_t N = 1u << LOGN, PN = ntt::padn(N);
  return (size_t)(PN + (PN & 1) + 2 * N + 2 * PN) * 4;
}

// The same node for the stages with few nodes (the early ones): one cluster of
// L ell CTAs, CTA (l, g) on limb l and digit g. Every CTA takes the inverse
// NTT of tau(a) (repeated across g: free while the GPU is not full), then one
// digit's forward NTT and multiply-accumulate; the digit-0 CTA of each limb
// adds the other digits' reduced partial sums (read through distributed shared
// memory) and writes the node's outputs.
template <int L, int LOGN>
__global__ void __launch_bounds__(ntt::HALF, 2) expand_split_kernel(const __grid_constant__ ExpandParams p) {
  using namespace ntt;
  constexpr uint32_t N = 1u << LOGN, S = N >> 3, PN = padn(N), MASK2N = 2 * N - 1;
  extern __shared__ __align__(16) uint32_t sm[];
  const Ring &R = p.ring;
  const uint32_t ell = R.ell;
  const uint32_t rank = cluster_rank();
  const uint32_t h = rank % L, g = rank / L;       // this CTA's limb and digit
  const uint32_t b = threadIdx.x;
  const bool act = b < S;
  const Limb &T = R.limb[h];
  const uint32_t q = T.q;
  uint32_t *res = sm;                                             // [PN]: coefficients of tau(a), limb h
  int64_t *ybuf = reinterpret_cast<int64_t *>(sm + PN + (PN & 1)); // [N]: Dcp offset values, then partial sums
  uint32_t *work = sm + PN + (PN & 1) + 2 * N;                    // [PN]: the digit transform

  const uint32_t node = blockIdx.x / (L * ell);
  const uint32_t c = node / p.nodes, k = node % p.nodes;
  const size_t ctw = (size_t)2 * L * N;
  // Plain loads: at stages >= 1 the digit-0 CTAs overwrite the input at the end.
  const uint32_t *in = p.stage == 0 ? p.query + (size_t)c * ctw : p.out + ((size_t)c * p.n_out + k) * ctw;
  uint32_t *out0 = p.out + ((size_t)c * p.n_out + k) * ctw;
  const uint32_t k1 = k + (1u << p.stage);
  const bool has1 = k1 < p.n_out;
  uint32_t *out1 = p.out + ((size_t)c * p.n_out + k1) * ctw;
  const uint32_t *row = p.evk + ((size_t)c * p.J + p.stage) * ell * ctw + (size_t)g * ctw + (size_t)h * N;

  // 1. tau(a) on the owned slots of limb h, then its inverse NTT
  {
    uint32_t v[1][8];
    if (act) {
#pragma unroll
      for (uint32_t e = 0; e < 8; ++e) {
        const uint32_t s = b + e * S;
        const uint32_t src = ((((2 * s + 1) * p.ksub) & MASK2N) - 1) >> 1;
        v[0][e] = in[(size_t)h * N + src];
      }
    }
    uint32_t *const bufs[1] = {res};
    inverse<LOGN, 1>(v, bufs, T, b, act);
  }
  cluster_arrive();   // every CTA's residues are complete and visible after this pair
  cluster_wait();

  // 2. digit g of the owned coefficients (CRT over the limbs), forward NTT,
  // multiply-accumulate with key row g
  uint32_t d[1][8];
  if (act) {
    const uint32_t peer = L > 1 ? peer_addr(res, (h ^ 1u) + L * g) : 0u;
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
      d[0][kk] = dcp_digit(dcp_offset_value(R, r0, r1), g, ell, q);
    }
    if ((b & 31) < 16) {
      const uint32_t l = b & 31;
      prefetch_l1(row + (b & ~31u) + (l >> 3) * (size_t)L * N + (l & 7) * S);
    }
  }
  cluster_arrive();   // done reading the other limb's residues
  {
    uint32_t *const bufs[1] = {work};
    forward<LOGN, 1>(d, bufs, T, b, act);
  }
  uint32_t part[2][8];
  if (act) {
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int e = 0; e < 8; ++e)
        part[r][e] = reduce64((uint64_t)d[0][e] * __ldg(row + (size_t)r * L * N + b + e * S), q, T.mu);
  }
  uint32_t *pbuf = reinterpret_cast<uint32_t *>(ybuf);   // 2N words, unused by this kernel until now
  if (g > 0 && act) {
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int e = 0; e < 8; ++e) pbuf[(r * 8 + e) * S + b] = part[r][e];
  }
  cluster_wait();     // pairs the arrive after step 2
  cluster_arrive();   // the partial sums are written
  cluster_wait();

  // 3. digit-0 CTAs: t = (a', tau(b) + b'); out0 = c + t, out1 = X^(-2^j) (c - t), limb h
  if (g == 0) {
    uint32_t tb[8], ca[8], cb[8];
    if (act) {
      for (uint32_t gg = 1; gg < ell; ++gg) {
        const uint32_t peer = peer_addr(pbuf, h + L * gg);
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
          for (int e = 0; e < 8; ++e) part[r][e] = add_mod(part[r][e], ld_peer(peer + 4 * ((r * 8 + e) * S + b)), q);
      }
#pragma unroll
      for (uint32_t e = 0; e < 8; ++e) {
        const uint32_t s = b + e * S;
        const uint32_t src = ((((2 * s + 1) * p.ksub) & MASK2N) - 1) >> 1;
        tb[e] = add_mod(part[1][e], in[(size_t)(L + h) * N + src], q);
        ca[e] = in[(size_t)h * N + s];
        cb[e] = in[(size_t)(L + h) * N + s];
      }
    }
    __syncthreads();   // every read of (limb h of) list[k] by this CTA precedes the writes below
    if (act) {
#pragma unroll
      for (uint32_t e = 0; e < 8; ++e) {
        const uint32_t s = b + e * S;
        out0[(size_t)h * N + s] = add_mod(ca[e], part[0][e], q);
        out0[(size_t)(L + h) * N + s] = add_mod(cb[e], tb[e], q);
        if (has1) {
          const uint2 m = __ldg(T.mono + (((2 * s + 1) << p.stage) & MASK2N));
          out1[(size_t)h * N + s] = shoup(sub_mod(ca[e], part[0][e], q), m.x, m.y, q);
          out1[(size_t)(L + h) * N + s] = shoup(sub_mod(cb[e], tb[e], q), m.x, m.y, q);
        }
      }
    }
  }
  cluster_arrive();   // the digit-0 CTAs have read the partial sums
  cluster_wait();
}

template <int LOGN>
constexpr size_t expand_split_smem() {
  constexpr uint32_t N = 1u << LOGN, PN = ntt::padn(N);
  return (size_t)(PN + (PN & 1) + 2 * N + PN) * 4;
}

bool g_ex_attr_done[64][2][ntt::MAX_LIMBS][ntt::MAX_LOGN + 1] = {};
std::mutex g_ex_mu;

// One stage. split: one cluster of L ell CTAs per node (limb x digit), else one
// cluster of L CTAs per node (limb).
template <int L, int LOGN>
int launch_stage(const ExpandParams &p, unsigned nodes, bool split, int dev, cudaStream_t s) {
  if (dev < 0 || dev >= 64) return GPIR_EINVAL;
  const size_t smem = split ? expand_split_smem<LOGN>() : expand_smem<LOGN>();
  void (*kern)(ExpandParams) = split ? expand_split_kernel<L, LOGN> : expand_stage_kernel<L, LOGN>;
  {
    std::lock_guard<std::mutex> lk(g_ex_mu);
    if (!g_ex_attr_done[dev][split][L - 1][LOGN]) {
      const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return set_cuda_error(e);
      g_ex_attr_done[dev][split][L - 1][LOGN] = true;
    }
  }
  const unsigned cl = split ? L * p.ring.ell : L;
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
int launch_stage_n(const ExpandParams &p, unsigned nodes, bool split, int dev, cudaStream_t s) {
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

extern "C" int gpir_expand_query(const gpir_params_t *params, uint32_t batch, uint32_t stages, uint32_t n_out,
                                 const uint32_t *query_dev, const uint32_t *evk_dev, uint32_t *out_dev,
                                 void *stream) {
  using namespace gpir;
  // every argument is checked here, on the host, before any CUDA call
  if (!params || !query_dev || !out_dev || batch == 0 || n_out == 0) return GPIR_EINVAL;
  if (stages > 0 && !evk_dev) return GPIR_EINVAL;
  if (params->num_limbs < 1 || params->num_limbs > ntt::MAX_LIMBS || params->n < ntt::MIN_N || params->n > ntt::MAX_N)
    return GPIR_ENOTSUP;
  uint32_t logn = 0;
  while ((1u << logn) < params->n) ++logn;
  // tau_k with k = N / 2^j + 1 is an automorphism (k odd) only for j < log2 N
  if (stages > logn || n_out > (1u << stages)) return GPIR_EINVAL;
  {
    const size_t ctw = (size_t)2 * params->num_limbs * params->n * 4;
    const uintptr_t q0 = (uintptr_t)query_dev, q1 = q0 + batch * ctw;
    const uintptr_t o0 = (uintptr_t)out_dev, o1 = o0 + (size_t)batch * n_out * ctw;
    if (q0 < o1 && o0 < q1) return GPIR_EINVAL;   // the tree runs in place in out_dev
  }
  ntt::Ring ring;
  int rc = ring_tables(params, &ring);
  if (rc != GPIR_OK) return rc;
  const uint32_t L = ring.L, N = ring.N;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t ct_words = (size_t)2 * L * N;
  if (stages == 0) {
    const cudaError_t e =
        cudaMemcpyAsync(out_dev, query_dev, (size_t)batch * ct_words * 4, cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? GPIR_OK : set_cuda_error(e);
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_cuda_error(e);
  ExpandParams p;
  memset(&p, 0, sizeof(p));
  p.ring = ring;
  p.query = query_dev;
  p.evk = evk_dev;
  p.out = out_dev;
  p.n_out = n_out;
  p.J = stages;
  for (uint32_t st = 0; st < stages; ++st) {
    p.stage = st;
    p.nodes = (1u << st) < n_out ? (1u << st) : n_out;
    p.ksub = (N >> st) + 1;
    const unsigned nodes = batch * p.nodes;
    // stage-aware choice (Sec. 4.4): the limb x digit split (which repeats the
    // inverse NTT per digit) when its L ell CTAs per node fit one CTA per SM,
    // the limb split otherwise. Measured at N = 4096, L = 2: the split is about
    // 10% faster per stage up to 16 nodes and slower from 32 nodes up.
    const bool split = (uint64_t)nodes * L * ring.ell <= (uint64_t)sm_count() && ring.ell <= 4;
    const int tr = trace_begin(split ? "expand_stage_split" : "expand_stage", s);
    rc = L == 1 ? launch_stage_n<1>(p, nodes, split, dev, s) : launch_stage_n<2>(p, nodes, split, dev, s);
    trace_end(tr, s);
    if (rc != GPIR_OK) return rc;
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_cuda_error(e);
  }
  return GPIR_OK;
}
