// RowSel on the INT8 tensor cores: exact byte-limb products with mma.sync.
//
// Per NTT point p = (limb, slot) RowSel is the GEMM of Sec. 2.3 / Sec. 5.1 of
// the GPIR paper, out[p][m][n] = sum_k ct[p][m][k] * db[p][k][n] mod q.
//
// Byte limbs. Each residue (< 2^28) is its 4 unsigned bytes, x = sum_u x_u
// 2^(8u) (the top byte is <= 15). Then x*y = sum_s 2^(8s) C_s with
// C_s = sum_{u+v=s} x_u y_v (s = 0..6). The tensor core forms, exactly in
// int32, A_s = sum_k sum_{u+v=s} a_u[m][k] b_v[k][n] with one
// mma.sync.m16n8k32.u8.u8.s32 per digit pair (u, v) into accumulator set s.
// Bound: C_2 has the largest per-row sum, three full byte pairs, 3*255^2 =
// 195075 (C_3: 2*255*15 + 2*255^2 = 137700), so up to 11008 rows fit below
// 2^31; accumulators are folded into residues every KFOLD = 8192 rows. The epilogue reduces sum_s A_s * (2^(8s) mod q) (< 2^62)
// with one Barrett reduction.
//
// Why legacy mma.sync: on sm_103a ptxas rejects tcgen05.mma .kind::i8, so the
// warp-level IMMA is the only INT8 tensor-core instruction. Its measured rate
// on GB300 is about 151 TOPS, i.e. < 4.7e12 modular MACs/s after the 16-way
// byte split: this path is compute-bound far below HBM speed, so its data
// staging is kept simple.
//
// Data movement. Like the CUDA-core path the p-major inputs are read in place:
// TMA boxes cover 32 consecutive slots (one 128-byte row segment per (m, k) or
// (k, n) row) with the 128-byte swizzle, so that a warp reading one slot's
// column of the box spreads over 8 bank groups instead of one. Each warp owns
// two of the block's 32 slots and runs the m16 x n8 tile of both, K in steps
// of 32 (one MMA k-step per stage).
#include <cuda.h>
#include <stdint.h>

#include "common.cuh"

namespace gpir {
namespace {

constexpr int MB = 16, NB = 8, KC = 32;      // rows (m), columns (n), k per stage
constexpr int WARPS = 16, THREADS = WARPS * 32;
constexpr int STAGES = 2;
constexpr int CT_BYTES = MB * KC * 128;      // [MB/2][KC][2][32 slots] u32, 128 B per row
constexpr int DB_BYTES = KC * NB * 128;      // [KC][NB][32 slots]
constexpr int STAGE_BYTES = CT_BYTES + DB_BYTES;
constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + 1024 + 64;
constexpr int KFOLD = 8192;                  // rows per int32 accumulation (bound above)

struct ImmaParams {
  uint32_t M, d0, d1, L, N;
  uint32_t m_blocks, n_blocks, slot_blocks_per_limb;
  unsigned int *err;
  LimbTable limbs;
  uint32_t cs[GPIR_MAX_LIMBS][7];            // 2^(8s) mod q_l
};

// Word for (box row R, slot s) in a 128-byte-swizzled box: chunk s/4 moves to
// chunk (s/4) ^ (R % 8).
__device__ __forceinline__ uint32_t sw_word(const uint32_t *base, uint32_t R, uint32_t s) {
  return base[R * 32 + ((((s >> 2) ^ (R & 7)) << 2) | (s & 3))];
}

// Byte u of each of x0..x3, packed little-endian.
__device__ __forceinline__ uint32_t pack_byte(uint32_t x0, uint32_t x1, uint32_t x2, uint32_t x3, uint32_t u) {
  const uint32_t sel = u | ((u + 4) << 4);
  return __byte_perm(__byte_perm(x0, x1, sel), __byte_perm(x2, x3, sel), 0x5410);
}

__device__ __forceinline__ void imma(int (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                     uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k32.row.col.s32.u8.u8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__global__ void __launch_bounds__(THREADS, 1)
    rowsel_imma_kernel(const __grid_constant__ CUtensorMap ct_map, const __grid_constant__ CUtensorMap db_map,
                       uint32_t *__restrict__ out, const ImmaParams p) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE_BYTES);

  uint32_t bid = blockIdx.x;
  const uint32_t nblk = bid % p.n_blocks;
  bid /= p.n_blocks;
  const uint32_t mblk = bid % p.m_blocks;
  const uint32_t sblk = bid / p.m_blocks;
  const uint32_t l = sblk / p.slot_blocks_per_limb;
  const uint32_t t0 = (sblk % p.slot_blocks_per_limb) * 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t g = lane >> 2, tig = lane & 3;
  const int nK = (int)((p.d0 + KC - 1) / KC);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) mbar_init(&full[s], 1);
    fence_mbar_init();
  }
  __syncthreads();
  auto issue = [&](int kc) {
    const int s = kc % STAGES;
    uint8_t *base = smem + s * STAGE_BYTES;
    mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
    tma_load_5d(base, &ct_map, &full[s], (int)t0, (int)l, 0, kc * KC, (int)mblk * (MB / 2));
    tma_load_4d(base + CT_BYTES, &db_map, &full[s], (int)t0, (int)l, (int)nblk * NB, kc * KC);
  };
  if (threadIdx.x == 0) {
    tma_prefetch_desc(&ct_map);
    tma_prefetch_desc(&db_map);
    for (int kc = 0; kc < STAGES - 1 && kc < nK; ++kc) issue(kc);
  }

  const uint32_t q = p.limbs.m[l].q;
  const uint64_t mu = p.limbs.m[l].mu;
  int acc[2][7][4];
  uint32_t res[2][4];
#pragma unroll
  for (int w = 0; w < 2; ++w) {
#pragma unroll
    for (int s = 0; s < 7; ++s)
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[w][s][i] = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) res[w][i] = 0;
  }

  // Fold the int32 digit-pair accumulators into running residues.
  auto fold = [&]() {
#pragma unroll
    for (int w = 0; w < 2; ++w) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        uint64_t v = 0;
#pragma unroll
        for (int s = 0; s < 7; ++s) v += (uint64_t)(uint32_t)acc[w][s][i] * p.cs[l][s];
        uint32_t r = reduce64(v, q, mu) + res[w][i];
        res[w][i] = r >= q ? r - q : r;
#pragma unroll
        for (int s = 0; s < 7; ++s) acc[w][s][i] = 0;
      }
    }
  };

  bool ok = true;
  for (int kc = 0; kc < nK; ++kc) {
    const int st = kc % STAGES;
    if (threadIdx.x == 0 && kc + STAGES - 1 < nK) issue(kc + STAGES - 1);
    if (ok) ok = mbar_wait_bounded(&full[st], (uint32_t)(kc / STAGES) & 1u, p.err, kErrTmaWait);
    const uint32_t *cs = reinterpret_cast<const uint32_t *>(smem + st * STAGE_BYTES);
    const uint32_t *ds = reinterpret_cast<const uint32_t *>(smem + st * STAGE_BYTES + CT_BYTES);
#pragma unroll
    for (int w = 0; w < 2; ++w) {
      const uint32_t sl = (uint32_t)warp + 16u * w;    // slot within the 32-slot box
      // A fragment rows g and g+8 (m), k = tig*4 + {0..3} and +16; B fragment
      // column g (n), the same k.
      uint32_t ra[4][4], rb[2][4];
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const uint32_t m = g + ((h & 1) ? 8u : 0u);
        const uint32_t kb = tig * 4 + ((h & 2) ? 16u : 0u);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const uint32_t k = kb + e;
          ra[h][e] = sw_word(cs, ((m >> 1) * KC + k) * 2 + (m & 1), sl);
        }
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const uint32_t k = tig * 4 + (h ? 16u : 0u) + e;
          rb[h][e] = sw_word(ds, k * NB + g, sl);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint32_t a0 = pack_byte(ra[0][0], ra[0][1], ra[0][2], ra[0][3], u);
        const uint32_t a1 = pack_byte(ra[1][0], ra[1][1], ra[1][2], ra[1][3], u);
        const uint32_t a2 = pack_byte(ra[2][0], ra[2][1], ra[2][2], ra[2][3], u);
        const uint32_t a3 = pack_byte(ra[3][0], ra[3][1], ra[3][2], ra[3][3], u);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const uint32_t b0 = pack_byte(rb[0][0], rb[0][1], rb[0][2], rb[0][3], v);
          const uint32_t b1 = pack_byte(rb[1][0], rb[1][1], rb[1][2], rb[1][3], v);
          imma(acc[w][u + v], a0, a1, a2, a3, b0, b1);
        }
      }
    }
    if (((kc + 1) * KC) % KFOLD == 0) fold();
    __syncthreads();
  }
  if (!ok) {
    if (threadIdx.x == 0)
      for (int kc = (nK > STAGES ? nK - STAGES : 0); kc < nK; ++kc)
        mbar_wait_bounded(&full[kc % STAGES], (uint32_t)(kc / STAGES) & 1u, nullptr, 0);
    return;
  }
  if ((nK * KC) % KFOLD != 0) fold();

#pragma unroll
  for (int w = 0; w < 2; ++w) {
    const uint32_t t = t0 + (uint32_t)warp + 16u * w;
    if (t >= p.N) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint32_t m = mblk * MB + g + ((i & 2) ? 8u : 0u);
      const uint32_t n = nblk * NB + tig * 2 + (i & 1);
      if (m >= p.M || n >= p.d1) continue;
      const uint32_t c = m >> 1, r = m & 1;
      out[((((size_t)c * p.d1 + n) * 2 + r) * p.L + l) * p.N + t] = res[w][i];
    }
  }
}

}  // namespace

int rowsel_imma_num_variants() { return 1; }
int rowsel_imma_default_variant(uint32_t, uint32_t, uint32_t) { return 0; }

int rowsel_imma_launch(const gpir_db *db, uint32_t batch, const uint32_t *ct, uint32_t *out, int variant,
                       cudaStream_t stream) {
  (void)variant;
  const uint32_t N = db->params.n, L = db->params.num_limbs, d0 = db->d0, d1 = db->d1;
  const uint32_t M = 2 * batch;
  CUtensorMap ct_map, db_map;
  {
    const uint64_t dims[5] = {N, L, 2, d0, batch};
    const uint64_t str[4] = {(uint64_t)N * 4, (uint64_t)L * N * 4, (uint64_t)2 * L * N * 4,
                             (uint64_t)d0 * 2 * L * N * 4};
    const uint32_t box[5] = {32, 1, 2, (uint32_t)KC, (uint32_t)(MB / 2)};
    int rc = encode_tiled(&ct_map, CU_TENSOR_MAP_DATA_TYPE_UINT32, ct, 5, dims, str, box,
                          CU_TENSOR_MAP_SWIZZLE_128B);
    if (rc) return rc;
  }
  {
    const uint64_t dims[4] = {N, L, d1, d0};
    const uint64_t str[3] = {(uint64_t)N * 4, (uint64_t)L * N * 4, (uint64_t)d1 * L * N * 4};
    const uint32_t box[4] = {32, 1, (uint32_t)NB, (uint32_t)KC};
    int rc = encode_tiled(&db_map, CU_TENSOR_MAP_DATA_TYPE_UINT32, db->db_pmajor, 4, dims, str, box,
                          CU_TENSOR_MAP_SWIZZLE_128B);
    if (rc) return rc;
  }
  ImmaParams p;
  p.M = M;
  p.d0 = d0;
  p.d1 = d1;
  p.L = L;
  p.N = N;
  p.m_blocks = (M + MB - 1) / MB;
  p.n_blocks = (d1 + NB - 1) / NB;
  p.slot_blocks_per_limb = (N + 31) / 32;
  p.err = device_error_word();
  p.limbs = db->params.limbs;
  for (uint32_t li = 0; li < L; ++li) {
    const uint64_t q = db->params.primes[li];
    uint64_t pw = 1;
    for (int s = 0; s < 7; ++s) {
      p.cs[li][s] = (uint32_t)(pw % q);
      pw = (pw << 8) % q;
    }
  }
  const uint64_t grid = (uint64_t)p.m_blocks * p.n_blocks * p.slot_blocks_per_limb * L;
  if (grid == 0 || grid > 0x7fffffffull) return GPIR_EINVAL;
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(rowsel_imma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
    if (e != cudaSuccess) return set_cuda_error(e);
    attr_done = true;
  }
  const int tr = trace_begin("rowsel_imma", stream);
  rowsel_imma_kernel<<<(unsigned)grid, THREADS, SMEM, stream>>>(ct_map, db_map, out, p);
  trace_end(tr, stream);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GPIR_OK : set_cuda_error(e);
}

}  // namespace gpir
