// RowSel on CUDA cores: exact 32x32->64-bit integer multiply-accumulate.
//
// GPIR paper, Sec. 2.3 / Sec. 5.1: RowSel is one GEMM per NTT point p = (limb
// l, slot t): out[p][m][n] = sum_k ct[p][m][k] * db[p][k][n] mod q_l, with
// m = (client c, polynomial r), k = DB row i, n = DB column j.
//
// Layout choice. The inputs stay in the paper's p-major layout (every
// polynomial's N slots contiguous). Instead of transposing them (Sec. 5.2),
// a warp's 32 lanes own 32 consecutive slots of one limb, so every global
// access is one 128-byte row segment, and each lane runs the small GEMMs of
// its own slot with a register tile of MT x NT 64-bit accumulators. A CTA
// covers MB = WM*MT rows and NB = WN*NT columns for 32 slots; TMA moves
// [MB x KC x 32-slot] ciphertext tiles and [KC x NB x 32-slot] database tiles
// into shared memory through an mbarrier ring of STAGES buffers, and zero-fills
// everything outside the tensors, so ragged D0 / D1 / batch tails need no
// special code on the load side.
//
// Arithmetic. A product of two residues below 2^28 is below 2^56, so a
// 64-bit accumulator holds any 256 of them; every 256 rows the accumulators
// are reduced mod q (Barrett), and once more at the end. mad.wide.u32 does one
// product-and-add per instruction.
#include <cuda.h>
#include <stdint.h>

#include "common.cuh"

namespace gpir {
namespace {

struct CcParams {
  uint32_t M, d0, d1, L, N;
  uint32_t m_blocks, n_blocks, slot_blocks_per_limb;
  unsigned int *err;
  LimbTable limbs;
};

template <int MT_, int NT_, int WM_, int WN_, int KC_, int STAGES_, int MINB_ = 1>
struct CcCfg {
  static constexpr int MT = MT_, NT = NT_, WM = WM_, WN = WN_, KC = KC_, STAGES = STAGES_, MINB = MINB_;
  static constexpr int MB = WM * MT, NB = WN * NT, THREADS = WM * WN * 32;
  static_assert(MB % 2 == 0, "a row block holds whole ciphertexts (2 polynomials)");
  static_assert(256 % KC == 0, "reduction period must be a whole number of chunks");
  static constexpr int CT_WORDS = MB * KC * 32;   // [MB/2][KC][2][32]
  static constexpr int DB_WORDS = KC * NB * 32;   // [KC][NB][32]
  static constexpr uint32_t STAGE_BYTES = (CT_WORDS + DB_WORDS) * 4u;
  static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + STAGES * 8 + 128;
  static_assert(SMEM <= 232448, "exceeds the 227 KB opt-in shared memory per CTA");
};

template <class C>
__global__ void __launch_bounds__(C::THREADS, C::MINB)
    rowsel_cc_kernel(const __grid_constant__ CUtensorMap ct_map, const __grid_constant__ CUtensorMap db_map,
                     uint32_t *__restrict__ out, const CcParams p) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  uint32_t *ct_s = reinterpret_cast<uint32_t *>(smem);
  uint32_t *db_s = ct_s + C::STAGES * C::CT_WORDS;
  uint64_t *full = reinterpret_cast<uint64_t *>(db_s + C::STAGES * C::DB_WORDS);

  uint32_t bid = blockIdx.x;
  const uint32_t nblk = bid % p.n_blocks;
  bid /= p.n_blocks;
  const uint32_t mblk = bid % p.m_blocks;
  const uint32_t sblk = bid / p.m_blocks;
  const uint32_t l = sblk / p.slot_blocks_per_limb;
  const uint32_t t0 = (sblk % p.slot_blocks_per_limb) * 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wm = warp / C::WN, wn = warp % C::WN;
  const int nK = (int)((p.d0 + C::KC - 1) / C::KC);

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) mbar_init(&full[s], 1);
    fence_mbar_init();
  }
  __syncthreads();

  auto issue = [&](int kc) {
    const int s = kc % C::STAGES;
    mbar_arrive_expect_tx(&full[s], C::STAGE_BYTES);
    tma_load_5d(ct_s + s * C::CT_WORDS, &ct_map, &full[s], (int)t0, (int)l, 0, kc * C::KC, (int)mblk * (C::MB / 2));
    tma_load_4d(db_s + s * C::DB_WORDS, &db_map, &full[s], (int)t0, (int)l, (int)nblk * C::NB, kc * C::KC);
  };
  if (threadIdx.x == 0) {
    tma_prefetch_desc(&ct_map);
    tma_prefetch_desc(&db_map);
    for (int kc = 0; kc < C::STAGES - 1 && kc < nK; ++kc) issue(kc);
  }

  const uint32_t q = p.limbs.m[l].q;
  const uint64_t mu = p.limbs.m[l].mu;
  uint64_t acc[C::MT][C::NT];
#pragma unroll
  for (int i = 0; i < C::MT; ++i)
#pragma unroll
    for (int j = 0; j < C::NT; ++j) acc[i][j] = 0;

  bool ok = true;
  for (int kc = 0; kc < nK; ++kc) {
    const int s = kc % C::STAGES;
    if (threadIdx.x == 0 && kc + C::STAGES - 1 < nK) issue(kc + C::STAGES - 1);
    if (ok) ok = mbar_wait_bounded(&full[s], (uint32_t)(kc / C::STAGES) & 1u, p.err, kErrTmaWait);
    const uint32_t *cs = ct_s + s * C::CT_WORDS;
    const uint32_t *ds = db_s + s * C::DB_WORDS;
#pragma unroll
    for (int kk = 0; kk < C::KC; ++kk) {
      uint32_t a[C::MT], b[C::NT];
#pragma unroll
      for (int i = 0; i < C::MT; ++i) {
        const int ml = wm * C::MT + i;
        a[i] = cs[(((ml >> 1) * C::KC + kk) * 2 + (ml & 1)) * 32 + lane];
      }
#pragma unroll
      for (int j = 0; j < C::NT; ++j) b[j] = ds[(kk * C::NB + wn * C::NT + j) * 32 + lane];
#pragma unroll
      for (int i = 0; i < C::MT; ++i)
#pragma unroll
        for (int j = 0; j < C::NT; ++j) acc[i][j] += (uint64_t)a[i] * b[j];
    }
    if (((kc + 1) * C::KC) % 256 == 0) {
#pragma unroll
      for (int i = 0; i < C::MT; ++i)
#pragma unroll
        for (int j = 0; j < C::NT; ++j) acc[i][j] = reduce64(acc[i][j], q, mu);
    }
    __syncthreads();
  }
  if (!ok) {
    // A TMA wait expired: drain what may still be in flight (bounded), skip stores.
    if (threadIdx.x == 0)
      for (int kc = (nK > C::STAGES ? nK - C::STAGES : 0); kc < nK; ++kc)
        mbar_wait_bounded(&full[kc % C::STAGES], (uint32_t)(kc / C::STAGES) & 1u, nullptr, 0);
    return;
  }

  const uint32_t t = t0 + lane;
  if (t >= p.N) return;
#pragma unroll
  for (int i = 0; i < C::MT; ++i) {
    const uint32_t m = mblk * C::MB + wm * C::MT + i;
    if (m >= p.M) continue;
    const uint32_t c = m >> 1, r = m & 1;
#pragma unroll
    for (int j = 0; j < C::NT; ++j) {
      const uint32_t n = nblk * C::NB + wn * C::NT + j;
      if (n >= p.d1) continue;
      const size_t idx = ((((size_t)c * p.d1 + n) * 2 + r) * p.L + l) * p.N + t;
      out[idx] = reduce64(acc[i][j], q, mu);
    }
  }
}

template <class C>
int launch_cc(const gpir_db *db, uint32_t batch, const uint32_t *ct, uint32_t *out, cudaStream_t stream) {
  const uint32_t N = db->params.n, L = db->params.num_limbs, d0 = db->d0, d1 = db->d1;
  const uint32_t M = 2 * batch;
  CUtensorMap ct_map, db_map;
  {
    const uint64_t dims[5] = {N, L, 2, d0, batch};
    const uint64_t str[4] = {(uint64_t)N * 4, (uint64_t)L * N * 4, (uint64_t)2 * L * N * 4, (uint64_t)d0 * 2 * L * N * 4};
    const uint32_t box[5] = {32, 1, 2, (uint32_t)C::KC, (uint32_t)(C::MB / 2)};
    int rc = encode_tiled_u32(&ct_map, ct, 5, dims, str, box);
    if (rc) return rc;
  }
  {
    const uint64_t dims[4] = {N, L, d1, d0};
    const uint64_t str[3] = {(uint64_t)N * 4, (uint64_t)L * N * 4, (uint64_t)d1 * L * N * 4};
    const uint32_t box[4] = {32, 1, (uint32_t)C::NB, (uint32_t)C::KC};
    int rc = encode_tiled_u32(&db_map, db->db_pmajor, 4, dims, str, box);
    if (rc) return rc;
  }
  CcParams p;
  p.M = M;
  p.d0 = d0;
  p.d1 = d1;
  p.L = L;
  p.N = N;
  p.m_blocks = (M + C::MB - 1) / C::MB;
  p.n_blocks = (d1 + C::NB - 1) / C::NB;
  p.slot_blocks_per_limb = (N + 31) / 32;
  p.err = device_error_word();
  p.limbs = db->params.limbs;
  const uint64_t grid = (uint64_t)p.m_blocks * p.n_blocks * p.slot_blocks_per_limb * L;
  if (grid == 0 || grid > 0x7fffffffull) return GPIR_EINVAL;
  static bool attr_done = false;  // per instantiation
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(rowsel_cc_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess) return set_cuda_error(e);
    attr_done = true;
  }
  const int tr = trace_begin("rowsel_cc", stream);
  rowsel_cc_kernel<C><<<(unsigned)grid, C::THREADS, C::SMEM, stream>>>(ct_map, db_map, out, p);
  trace_end(tr, stream);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GPIR_OK : set_cuda_error(e);
}

// Variant table: register tile (MT x NT), warp grid (WM x WN), k chunk, stages.
using V0 = CcCfg<2, 8, 1, 8, 8, 3>;   // MB=2  NB=64 : one client
using V1 = CcCfg<4, 8, 2, 4, 8, 3>;   // MB=8  NB=32
using V2 = CcCfg<8, 8, 2, 4, 8, 3>;   // MB=16 NB=32
using V3 = CcCfg<8, 8, 4, 2, 8, 3>;   // MB=32 NB=16
using V4 = CcCfg<4, 4, 2, 4, 8, 4>;   // MB=8  NB=16 : small shapes
using V5 = CcCfg<8, 4, 4, 2, 16, 2>;  // MB=32 NB=8
using V6 = CcCfg<4, 4, 4, 4, 8, 3, 2>;   // MB=16 NB=16, 16 warps, 2 CTAs/SM
using V7 = CcCfg<4, 8, 4, 4, 8, 3>;      // MB=16 NB=32, 16 warps
using V8 = CcCfg<8, 4, 4, 4, 8, 3>;      // MB=32 NB=16, 16 warps
using V9 = CcCfg<4, 4, 2, 4, 8, 3, 3>;   // MB=8  NB=16, 8 warps, 3 CTAs/SM

}  // namespace

int rowsel_cc_num_variants() { return 10; }

int rowsel_cc_default_variant(uint32_t batch, uint32_t d0, uint32_t d1) {
  (void)d0;
  if (batch <= 1) return 0;
  if (batch <= 4) return 1;
  if (d1 <= 16) return 3;
  return 2;
}

int rowsel_cc_launch(const gpir_db *db, uint32_t batch, const uint32_t *ct, uint32_t *out, int variant,
                     cudaStream_t stream) {
  switch (variant) {
    case 0: return launch_cc<V0>(db, batch, ct, out, stream);
    case 1: return launch_cc<V1>(db, batch, ct, out, stream);
    case 2: return launch_cc<V2>(db, batch, ct, out, stream);
    case 3: return launch_cc<V3>(db, batch, ct, out, stream);
    case 4: return launch_cc<V4>(db, batch, ct, out, stream);
    case 5: return launch_cc<V5>(db, batch, ct, out, stream);
    case 6: return launch_cc<V6>(db, batch, ct, out, stream);
    case 7: return launch_cc<V7>(db, batch, ct, out, stream);
    case 8: return launch_cc<V8>(db, batch, ct, out, stream);
    case 9: return launch_cc<V9>(db, batch, ct, out, stream);
    default: return GPIR_EINVAL;
  }
}

}  // namespace gpir
