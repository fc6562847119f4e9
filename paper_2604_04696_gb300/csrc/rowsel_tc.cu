// RowSel on the 5th-generation tensor cores (tcgen05, fp16 operands, fp32
// accumulators in tensor memory), exact.
//
// What is computed: the per-point modular GEMM of Sec. 2.3 / Sec. 5.1 of the
// GPIR paper, out[p][m][n] = sum_k ct[p][m][k] * db[p][k][n] mod q, with
// p = (limb, slot), m = (client, polynomial), k = DB row, n = DB column.
//
// Exactness. Each residue x < 2^28 is written in balanced base-256 digits,
//     x = d0 + d1 2^8 + d2 2^16 + d3 2^24,  d0,d1,d2 in [-128, 127], d3 in [0, 16]
// (byte u of x + 0x808080, minus 128 for u < 3). Every digit is exactly an fp16.
// A digit product has |d e| <= 2^14, so a sum of at most 256 of them has
// magnitude <= 2^22 < 2^24 and is exact in the fp32 accumulator: every partial
// sum is an integer representable in fp32, so no rounding can occur. Hence
// the tensor core computes, exactly, for each digit pair (u, v),
//     D_uv[m][n] = sum_{k in group} a_u[m][k] * b_v[k][n]        (|D| <= 2^22)
// and  x*y = sum_{u,v} a_u b_v 2^(8(u+v)), so
//     out = sum_groups sum_{u,v} D_uv * (2^(8(u+v)) mod q)   (mod q),
// computed in 64-bit integers in the epilogue. The K dimension is processed in
// groups of 256 rows (two-pass kernel) or 512 rows (fused, pair and cluster
// kernels, |D| <= 2^23, still exact), each group accumulating in its own
// tensor-memory buffer.
//
// GEMM shape. One MMA instruction computes all 16 digit pairs at once: the A
// operand stacks the 4 digits of 32 ciphertext rows (M' = 128 rows, ordered
// m_hi*32 + u*8 + m_lo with m = 8 m_hi + m_lo), the B operand stacks the 4
// digits of 64 DB columns (N' = 256 rows, ordered n*4 + v); tcgen05.mma
// .kind::f16 M=128 N=256 K=16, fp16 in, fp32 out. A TMEM lane quarter then
// holds 8 rows m with all 4 digits u, so the epilogue sums over u with two
// warp shuffles and over v within the thread.
//
// Data movement. The DB is stored once, at upload, as per-slot digit tiles
// already in the shared-memory image the MMA reads (K-major, 128-byte
// swizzle): [slot][n-block][k-chunk] x (256 rows x 64 k) fp16. Per batch the
// p-major ciphertexts are split into the same image for the A operand,
// reading 8 slots (one 32-byte sector) per row, in one of four forms:
//   - fused (default): persistent CTAs whose ingest warps write the A tiles
//     into an L2-sized ring in global memory while their GEMM warps stream A
//     and B tiles with bulk copies into shared-memory stages, one thread issues
//     the MMAs, epilogue warps drain tensor memory (double-buffered) and a
//     store warp writes the p-major output;
//   - SM pair: the fused kernel on 2-CTA clusters with cta_group::2 MMAs
//     (M = 256) that share one database tile between the two SMs;
//   - two-pass: an ingest kernel writes every A tile to HBM, then a persistent
//     GEMM kernel reads them (also the multi-job form);
//   - cluster: 8-CTA clusters, one CTA per slot of a group, exchange the digit
//     rows through distributed shared memory, so no A tile leaves the cluster.
#include <cuda.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>

#include "common.cuh"
#include "tcgen05.cuh"

namespace gpir {
namespace {

constexpr int KCHUNK = 64;             // k per pipeline stage (one 128-byte swizzle row of fp16)
constexpr int KGROUP_CHUNKS = 4;       // 4 x 64 = 256 rows per exact fp32 group
constexpr int MROWS = 32;              // ciphertext rows (m) per tile -> 128 digit rows
constexpr int NCOLS = 64;              // DB columns per tile -> 256 digit rows
constexpr int A_TILE_BYTES = 128 * KCHUNK * 2;   // 16 KB
constexpr int B_TILE_BYTES = 256 * KCHUNK * 2;   // 32 KB
constexpr int STAGES = 4;
constexpr int STAGE_BYTES = A_TILE_BYTES + B_TILE_BYTES;
constexpr int EPI_WARPS = 16;          // 4 per TMEM lane quarter, 2 column chunks each
constexpr int GEMM_THREADS = 64 + 32 * EPI_WARPS;   // warp 0 producer, warp 1 MMA, then epilogue
constexpr size_t GEMM_SMEM = (size_t)STAGES * STAGE_BYTES + 1024 + 256;
constexpr uint32_t TMEM_COLS = 512;    // two 128 x 256 fp32 accumulators

struct TcLimb {
  uint32_t q;
  uint32_t pad;
  uint64_t mu;        // floor(2^64 / q)
  uint64_t off;       // multiple of q, >= 2^55: makes signed sums non-negative
  int64_t kfix;       // 0x4B400000 * sum_{u,v} c[u+v] (see the epilogue)
  int32_t c[8];       // 2^(8s) mod q, s = 0..6 (c[7] unused)
  uint64_t off58;     // multiple of q, >= 2^58 (fused kernel: up to 8 groups summed before reducing)
};

constexpr int MAX_JOBS = 8;            // RowSel problems per launch (inline job table)

// One RowSel problem of a launch. Units of all jobs are numbered into one
// index space [0, units): job j owns [unit_begin, unit_begin + slots*mblk*nblk),
// ordered m-block fastest, then n-block, then slot.
struct TcJob {
  const uint16_t *a_tiles;              // [slot][mblk][kch] x 16 KB
  const uint16_t *b_tiles;              // [slot][nblk][kch] x 32 KB
  uint32_t *out;
  uint32_t M, d0, d1, mblk, nblk, kch;
  uint64_t unit_begin;
};

struct TcParams {
  uint32_t L, N, njobs, pad;
  uint64_t units;
  unsigned int *err;
  TcJob job[MAX_JOBS];
  TcLimb limb[GPIR_MAX_LIMBS];
};

struct UnitRef {
  uint32_t j, mb, nb;
  uint64_t slot;
};

__device__ __forceinline__ UnitRef decode_unit(const TcParams &p, uint64_t u) {
  uint32_t j = 0;
  while (j + 1 < p.njobs && u >= p.job[j + 1].unit_begin) ++j;
  const TcJob &jb = p.job[j];
  uint64_t x = u - jb.unit_begin;
  UnitRef r;
  r.j = j;
  r.mb = (uint32_t)(x % jb.mblk);
  x /= jb.mblk;
  r.nb = (uint32_t)(x % jb.nblk);
  r.slot = x / jb.nblk;
  return r;
}

// ---- digit helpers -----------------------------------------------------------

// fp16 bit pattern of the balanced digit u (0..3) of x (< 2^28).
__device__ __forceinline__ uint32_t digit_f16_bits(uint32_t x, int u) {
  const uint32_t b = x + 0x808080u;
  const uint32_t byte = (b >> (8 * u)) & 0xFFu;
  // 2^23 + byte as an fp32 bit pattern, minus (2^23 + 128) (or 2^23 for the top digit)
  const float f = __int_as_float(0x4B000000 | byte) - (u < 3 ? 8388736.0f : 8388608.0f);
  return (uint32_t)__half_as_ushort(__float2half_rn(f));   // exact: |digit| <= 128 fits fp16
}

// ---- ingest: p-major ciphertexts -> A-operand digit tiles --------------------

struct IngestJob {
  uint4 *a_tiles;
  uint32_t M, d0, mblk, kch;
  uint32_t block_begin;                 // first CTA of this job
};

struct IngestParams {
  uint32_t L, N, gpl, groups8, njobs;   // gpl: 8-slot groups per limb
  unsigned int *err;
  IngestJob job[MAX_JOBS];
  CUtensorMap ct_map[MAX_JOBS];         // p-major ct [B][D0][2][L][N], box (8 slots, 1, 2, 64 k, 16 clients)
};

// One CTA: 8 consecutive slots of one limb x one m-block (32 rows = 16
// clients x 2 polynomials) x one k-chunk (64 k). One TMA box brings the raw
// residues ([16 clients][64 k][2][8 slots], 64 KB, zero-filled outside the
// tensor) into shared memory; threads split them into digits and build the 8
// slots' A tiles in shared memory, each followed by a 16-byte pad so the 8
// lanes of a store phase (8 different slots) hit 8 different bank groups;
// the tiles then leave with coalesced 16-byte stores.
constexpr int INGEST_THREADS = 512;
constexpr int TILE_PAD = 1025;                       // uint4 per staged tile incl. pad
constexpr int RAW_BYTES = 16 * KCHUNK * 2 * 8 * 4;   // 64 KB raw box
constexpr size_t INGEST_SMEM = 1024 + RAW_BYTES + 8 * TILE_PAD * 16 + 64;
__global__ void __launch_bounds__(INGEST_THREADS) tc_ingest_kernel(const __grid_constant__ IngestParams p) {
  extern __shared__ __align__(1024) uint8_t ing_raw[];
  uint8_t *base = (uint8_t *)(((uintptr_t)ing_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t *raw = reinterpret_cast<const uint32_t *>(base);
  uint4 *tiles = reinterpret_cast<uint4 *>(base + RAW_BYTES);    // [8 slots][128 rows x 8 chunks + pad]
  uint64_t *bar = reinterpret_cast<uint64_t *>(base + RAW_BYTES + 8 * TILE_PAD * 16);
  uint32_t jj = 0;
  while (jj + 1 < p.njobs && blockIdx.x >= p.job[jj + 1].block_begin) ++jj;
  const IngestJob &jb = p.job[jj];
  uint32_t bid = blockIdx.x - jb.block_begin;
  const uint32_t g8 = bid % p.groups8;
  bid /= p.groups8;
  const uint32_t kc = bid % jb.kch;
  const uint32_t mb = bid / jb.kch;
  const uint32_t l = g8 / p.gpl, t0 = (g8 % p.gpl) * 8;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(bar, RAW_BYTES);
    tma_load_5d(base, &p.ct_map[jj], bar, (int)t0, (int)l, 0, (int)(kc * KCHUNK), (int)(mb * (MROWS / 2)));
  }
  const bool ok = mbar_wait_bounded(bar, 0, p.err, kErrTmaWait);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int s = lane & 7, msub = lane >> 3;
  if (ok) {
    // Each warp owns 64 / 16 = 4 (m-quad, k-octet) tasks.
#pragma unroll
    for (int tt = 0; tt < 64 / (INGEST_THREADS / 32); ++tt) {
      const int task = warp + tt * (INGEST_THREADS / 32);
      const int m_local = (task >> 3) * 4 + msub;
      const int k_oct = task & 7;
      const int c = m_local >> 1, r = m_local & 1;
      uint32_t v[8];
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) v[kk] = raw[((c * KCHUNK + k_oct * 8 + kk) * 2 + r) * 8 + s];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        uint4 w;
        w.x = digit_f16_bits(v[0], u) | (digit_f16_bits(v[1], u) << 16);
        w.y = digit_f16_bits(v[2], u) | (digit_f16_bits(v[3], u) << 16);
        w.z = digit_f16_bits(v[4], u) | (digit_f16_bits(v[5], u) << 16);
        w.w = digit_f16_bits(v[6], u) | (digit_f16_bits(v[7], u) << 16);
        const int row = (m_local >> 3) * 32 + u * 8 + (m_local & 7);
        tiles[s * TILE_PAD + row * 8 + (k_oct ^ (row & 7))] = w;
      }
    }
  }
  __syncthreads();
  if (!ok) {
    if (threadIdx.x == 0) mbar_wait_bounded(bar, 0, nullptr, 0);   // let a late copy land first
    return;
  }
  for (int idx = threadIdx.x; idx < 8 * 1024; idx += INGEST_THREADS) {
    const int ss = idx >> 10;
    const uint32_t t = t0 + ss;
    if (t >= p.N) continue;
    const uint64_t sl = (uint64_t)l * p.N + t;
    jb.a_tiles[((sl * jb.mblk + mb) * jb.kch + kc) * 1024 + (idx & 1023)] = tiles[ss * TILE_PAD + (idx & 1023)];
  }
}

// ---- DB packing (once per upload): p-major DB -> B-operand digit tiles -------

struct PackParams {
  uint32_t d0, d1, L, N, nblk, kch;
  const uint32_t *db;
  uint4 *b_tiles;
};

// One thread per (slot, n-block, k-chunk, digit row, k octet); slots fastest so
// the reads of the p-major DB are coalesced.
__global__ void tc_pack_db_kernel(const PackParams p, uint64_t total) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t x = i;
    const uint32_t slot = (uint32_t)(x % ((uint64_t)p.L * p.N));
    x /= (uint64_t)p.L * p.N;
    const uint32_t k_oct = (uint32_t)(x % 8);
    x /= 8;
    const uint32_t row = (uint32_t)(x % 256);
    x /= 256;
    const uint32_t kc = (uint32_t)(x % p.kch);
    const uint32_t nb = (uint32_t)(x / p.kch);
    const uint32_t n = nb * NCOLS + row / 4, v = row % 4;
    const uint32_t l = slot / p.N, t = slot % p.N;
    uint32_t bits[8];
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      const uint32_t k = kc * KCHUNK + k_oct * 8 + kk;
      const uint32_t val =
          (n < p.d1 && k < p.d0) ? p.db[(((uint64_t)k * p.d1 + n) * p.L + l) * p.N + t] : 0u;
      bits[kk] = digit_f16_bits(val, (int)v);
    }
    uint4 w;
    w.x = bits[0] | (bits[1] << 16);
    w.y = bits[2] | (bits[3] << 16);
    w.z = bits[4] | (bits[5] << 16);
    w.w = bits[6] | (bits[7] << 16);
    p.b_tiles[(((uint64_t)slot * p.nblk + nb) * p.kch + kc) * 2048 + row * 8 + (k_oct ^ (row & 7))] = w;
  }
}

// ---- persistent GEMM ---------------------------------------------------------

__global__ void __launch_bounds__(GEMM_THREADS, 1) tc_gemm_kernel(const __grid_constant__ TcParams p) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE_BYTES);
  uint64_t *empty = full + STAGES;
  uint64_t *acc_full = empty + STAGES;
  uint64_t *acc_empty = acc_full + 2;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_empty + 2);
  volatile uint32_t *abort_flag = tmem_slot + 1;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], EPI_WARPS);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;


  // A bounded wait that also gives up when another role already gave up.
  auto wait = [&](uint64_t *bar, uint32_t parity, unsigned int code) -> bool {
    if (mbar_try_wait(bar, parity)) return true;
    uint64_t t0 = globaltimer_ns();
    for (uint32_t n = 1;; ++n) {
      if (mbar_try_wait(bar, parity)) return true;
      if ((n & 63u) == 0) {
        if (*abort_flag) return false;
        if (globaltimer_ns() - t0 > kWaitLimitNs) {
          atomicCAS(p.err, 0u, code);
          *abort_flag = 1;
          return false;
        }
      }
    }
  };

  if (warp == 0) {
    // ---------------- producer ----------------
    if (lane == 0) {
      uint32_t st = 0, ph = 0;
      bool ok = true;
      for (uint64_t u = blockIdx.x; u < p.units && ok; u += gridDim.x) {
        const UnitRef ur = decode_unit(p, u);
        const TcJob &jb = p.job[ur.j];
        const uint8_t *a_src =
            (const uint8_t *)jb.a_tiles + ((ur.slot * jb.mblk + ur.mb) * jb.kch) * (uint64_t)A_TILE_BYTES;
        const uint8_t *b_src =
            (const uint8_t *)jb.b_tiles + ((ur.slot * jb.nblk + ur.nb) * jb.kch) * (uint64_t)B_TILE_BYTES;
        for (uint32_t kc = 0; kc < jb.kch; ++kc) {
          if (!(ok = wait(&empty[st], ph ^ 1u, kErrTmaWait))) break;
          uint8_t *sa = smem + st * STAGE_BYTES;
          mbar_arrive_expect_tx(&full[st], STAGE_BYTES);
          bulk_g2s(sa, a_src + (uint64_t)kc * A_TILE_BYTES, A_TILE_BYTES, &full[st]);
          bulk_g2s(sa + A_TILE_BYTES, b_src + (uint64_t)kc * B_TILE_BYTES, B_TILE_BYTES, &full[st]);
          if (++st == STAGES) {
            st = 0;
            ph ^= 1u;
          }
        }
      }
      if (!ok) {
        // let copies already issued land before the CTA can exit (bounded)
        for (int s = 0; s < STAGES; ++s) mbar_wait_bounded(&empty[s], ph ^ 1u, nullptr, 0);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      uint32_t st = 0, ph = 0, buf = 0;
      uint32_t aph[2] = {0, 0};
      bool ok = true;
      for (uint64_t u = blockIdx.x; u < p.units && ok; u += gridDim.x) {
        const uint32_t kch = p.job[decode_unit(p, u).j].kch;
        const uint32_t kgroups = (kch + KGROUP_CHUNKS - 1) / KGROUP_CHUNKS;
        for (uint32_t g = 0; g < kgroups && ok; ++g) {
          if (!(ok = wait(&acc_empty[buf], aph[buf] ^ 1u, kErrMmaWait))) break;
          tc_fence_after();
          const uint32_t tmem_d = tmem_base + buf * 256;
          const uint32_t c0 = g * KGROUP_CHUNKS;
          const uint32_t c1 = min(kch, c0 + KGROUP_CHUNKS);
          for (uint32_t kc = c0; kc < c1; ++kc) {
            if (!(ok = wait(&full[st], ph, kErrTmaWait))) break;
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + st * STAGE_BYTES);
            const uint32_t sb = sa + A_TILE_BYTES;
#pragma unroll
            for (int k16 = 0; k16 < KCHUNK / 16; ++k16) {
              mma_f16(tmem_d, sw128_desc(sa + k16 * 32), sw128_desc(sb + k16 * 32),
                       (kc > c0 || k16 > 0) ? 1u : 0u);
            }
            mma_commit(&empty[st]);      // frees the smem stage once these MMAs have read it
            if (++st == STAGES) {
              st = 0;
              ph ^= 1u;
            }
          }
          if (!ok) break;
          mma_commit(&acc_full[buf]);    // accumulator group complete
          aph[buf] ^= 1u;
          buf ^= 1u;
        }
      }
      if (!ok) {
        for (int b = 0; b < 2; ++b) mbar_wait_bounded(&acc_full[b], aph[b], nullptr, 0);
      }
    }
  } else {
    // ---------------- epilogue (warps 2 .. 2+EPI_WARPS-1) ----------------
    // Warp w reads TMEM lane quarter w % 4 (hardware rule); the four warps of
    // a quarter split the 8 column chunks of the 256-column accumulator.
    constexpr int CHUNKS = 8 / (EPI_WARPS / 4);
    const uint32_t quarter = warp & 3;
    const int jbase = ((warp - 2) >> 2) * CHUNKS;
    const int u = lane >> 3, m_lo = lane & 7;
    const int m_local = quarter * 8 + m_lo;
    uint32_t buf = 0;
    uint32_t aph[2] = {0, 0};
    bool ok = true;
    for (uint64_t un = blockIdx.x; un < p.units && ok; un += gridDim.x) {
      const UnitRef ur = decode_unit(p, un);
      const TcJob &jb = p.job[ur.j];
      const uint32_t mb = ur.mb, nb = ur.nb;
      const uint32_t kgroups = (jb.kch + KGROUP_CHUNKS - 1) / KGROUP_CHUNKS;
      const uint32_t l = (uint32_t)(ur.slot / p.N), t = (uint32_t)(ur.slot % p.N);
      const TcLimb &lm = p.limb[l];
      const int32_t c0 = lm.c[u], c1 = lm.c[u + 1], c2 = lm.c[u + 2], c3 = lm.c[u + 3];
      // fp32 D + 1.5*2^23 has bit pattern 0x4B400000 + D for |D| <= 2^22, so
      // sum_{u,v} bits_uv c_{u+v} - lm.kfix = sum_{u,v} D_uv c_{u+v} exactly
      // (|bits * c| < 2^58.3: the 16-term sum stays below 2^63).
      const bool odd = (u & 1) != 0, high = (u & 2) != 0;
      uint32_t res[2 * CHUNKS];
#pragma unroll
      for (int i = 0; i < 2 * CHUNKS; ++i) res[i] = 0;
      for (uint32_t g = 0; g < kgroups; ++g) {
        if (!(ok = wait(&acc_full[buf], aph[buf], kErrMmaWait))) break;
        tc_fence_after();
        const uint32_t taddr = tmem_base + ((quarter * 32u) << 16) + buf * 256 + jbase * 32;
#pragma unroll
        for (int j = 0; j < CHUNKS; ++j) {
          uint32_t d[32];
          tmem_ld32(taddr + j * 32, d);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            int64_t P[4];
#pragma unroll
            for (int w = 0; w < 4; ++w) {
              const int n8 = h * 4 + w;
              const int32_t b0 = __float_as_int(__uint_as_float(d[n8 * 4 + 0]) + 12582912.0f);
              const int32_t b1 = __float_as_int(__uint_as_float(d[n8 * 4 + 1]) + 12582912.0f);
              const int32_t b2 = __float_as_int(__uint_as_float(d[n8 * 4 + 2]) + 12582912.0f);
              const int32_t b3 = __float_as_int(__uint_as_float(d[n8 * 4 + 3]) + 12582912.0f);
              P[w] = (int64_t)b0 * c0 + (int64_t)b1 * c1 + (int64_t)b2 * c2 + (int64_t)b3 * c3;
            }
            // Reduce-scatter over the 4 digit lanes u (lane bits 3-4): lane u
            // ends with the sum over u' of P_u'[w = u], i.e. output n8 = 4h + u.
            int64_t k0 = odd ? P[1] : P[0], k1 = odd ? P[3] : P[2];
            const int64_t s0 = odd ? P[0] : P[1], s1 = odd ? P[2] : P[3];
            k0 += __shfl_xor_sync(0xffffffffu, s0, 8);
            k1 += __shfl_xor_sync(0xffffffffu, s1, 8);
            int64_t keep = high ? k1 : k0;
            const int64_t send = high ? k0 : k1;
            keep += __shfl_xor_sync(0xffffffffu, send, 16);
            const uint32_t rr = reduce64((uint64_t)(keep - lm.kfix + (int64_t)lm.off), lm.q, lm.mu);
            uint32_t &acc = res[j * 2 + h];
            acc += rr;
            acc = acc >= lm.q ? acc - lm.q : acc;
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[buf]);
        aph[buf] ^= 1u;
        buf ^= 1u;
      }
      if (!ok) break;
      const uint32_t m = mb * MROWS + m_local;
      if (m < jb.M) {
        const uint32_t c = m >> 1, rr = m & 1;
#pragma unroll
        for (int j = 0; j < CHUNKS; ++j) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const uint32_t n = nb * NCOLS + (jbase + j) * 8 + h * 4 + u;
            if (n < jb.d1) jb.out[((((uint64_t)c * jb.d1 + n) * 2 + rr) * p.L + l) * p.N + t] = res[j * 2 + h];
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                 : "memory");
  }
}

// ---- fused persistent kernel: ingest warps + GEMM warps in one launch ------
//
// The ciphertexts still arrive p-major, but their digit tiles never go to HBM.
// Work is cut into entries E = (8-slot group g, m-block mb). In every CTA,
// eight ingest warps claim ingest tasks (E, k-chunk) in increasing order from
// a global counter: one TMA box brings the raw residues of 8 slots x 32 rows x
// 64 k, the warps split them into digit tiles and store them into a ring of R
// entries in global memory (sized to stay in L2), then count the task into
// ready[E % R]. The GEMM warps claim units (E, slot, n-block) in increasing
// order from a second counter; the producer waits until ready[E % R] shows
// every k-chunk of entry E before bulk-copying its tiles, and an epilogue
// thread counts the unit into consumed[E % R] once its MMAs have read them.
// An ingest task for E first waits until the previous occupant E - R of its
// ring entry is fully consumed. Because both sides claim in increasing E and
// only running CTAs hold claims, the smallest unfinished entry can always
// progress (its only dependency lies R entries back): no deadlock, whatever
// number of CTAs is resident. Counters are monotonic and zeroed before the
// launch. Unit ids travel producer -> MMA thread -> epilogue through shared
// memory with the stage and accumulator barriers. All waits are bounded.
//
// SM-pair form (PAIR = true, clusters of 2 CTAs, cta_group::2). A pair unit
// (E2, slot, n-block) covers the two m-blocks of entries 2 E2 (even CTA) and
// 2 E2 + 1 (odd CTA) against ONE database tile: each CTA bulk-copies its own
// A tile (16 KB per k-chunk) and half of the B tile (16 KB, B rows 128 r ..
// 128 r + 127 for CTA rank r), and the even CTA's MMA thread issues M = 256,
// N = 256 MMAs that read both CTAs' shared memory and write both CTAs' tensor
// memory. Per SM that is 32 KB of operands per k-chunk instead of 48 KB, for
// the same tensor work. Protocol on top of the single-CTA form:
//   - the even CTA's producer claims units and hands each to the odd CTA's
//     producer through a 4-slot mailbox (remote store + release arrive);
//   - the odd CTA's warp 1 relays "my operands of stage st have landed" to the
//     even CTA's pfull[st] (a relaxed remote arrive: it carries no data of the
//     relaying thread, and a cluster-scope release would wait for the SM's
//     outstanding ring stores);
//   - MMA commits arrive on empty[st] and acc_full[b] in both CTAs
//     (multicast), and the odd CTA's epilogue warps also arrive on the even
//     CTA's acc_empty[b] (count 16 there; relaxed too, after their
//     tensor-memory loads have completed);
//   - each CTA's epilogue, store warp and ring accounting work on its own
//     entry 2 E2 + rank, exactly as in the single-CTA form.
// Both CTAs walk the same unit sequence, so their stage and accumulator
// phases stay aligned. The lookahead compares entries with claimed pair
// units (two entries each), and the deadlock argument carries over: the
// smallest unfinished pair unit depends only on ring entries R back and on
// claims already made. Needs an even number of m-blocks.

constexpr int F_EPI_WARPS = 8;
// Exact fp32 group of the fused kernel: 512 rows, so |D| <= 512 * 2^14 = 2^23,
// converted exactly with cvt.rni (the magic-number conversion of the two-pass
// kernel needs |D| < 2^22). Each output sums 16 terms |D| * c < 2^51 per
// group, so up to 8 groups (< 2^58) are accumulated in 64 bits before one
// Barrett reduction.
constexpr int F_KGROUP_CHUNKS = 8;
constexpr int F_FLUSH_GROUPS = 8;
constexpr int F_INGEST_WARPS = 8;
constexpr int F_STORE_WARP = 2 + F_EPI_WARPS + F_INGEST_WARPS;                // output store warp
constexpr int FUSED_THREADS = 32 * (F_STORE_WARP + 1);                        // 608
constexpr int FSTAGES = 3;                                     // operand stages (48 KB each)
constexpr int F_RAW_BYTES = 16 * KCHUNK * 2 * 8 * 4;           // raw box: 16 clients x 2 x 64 k x 8 slots
constexpr int F_OUT_BYTES = MROWS * NCOLS * 4;                 // one unit's 32 x 64 output block
constexpr size_t FUSED_SMEM = 1024 + (size_t)FSTAGES * STAGE_BYTES + F_RAW_BYTES + F_OUT_BYTES + 256;
static_assert(FUSED_SMEM <= 232448, "fused kernel shared memory exceeds 227 KB");
constexpr int P_STAGES = 4;                                    // pair form: operand stages (32 KB each)
constexpr int P_STAGE_BYTES = A_TILE_BYTES + B_TILE_BYTES / 2;
constexpr int P_MAIL = 4;                                      // pair form: claimed units in flight to the odd CTA
constexpr size_t PAIR_SMEM = 1024 + (size_t)P_STAGES * P_STAGE_BYTES + F_RAW_BYTES + F_OUT_BYTES + 512;
static_assert(PAIR_SMEM <= 232448, "pair kernel shared memory exceeds 227 KB");

constexpr uint64_t kNoUnit = ~0ull;

// L2 eviction priorities of the fused kernel's streams (tile-variant bits).
enum FusedHint : uint32_t {
  kHintCtEvictFirst = 1,     // raw ciphertext TMA boxes: read once
  kHintDbEvictFirst = 2,     // database digit tiles
  kHintRingEvictLast = 4,    // digit-ring stores: keep until overwritten
};

struct FusedParams {
  uint32_t L, N, M, d0, d1, mblk, nblk, kch;
  uint32_t R, gpl;                      // ring entries; 8-slot groups per limb
  uint32_t hints;                       // FusedHint bits: L2 eviction priorities
  uint32_t spg;                         // valid slots per group
  uint32_t lookahead;                   // ingest runs at most this many entries past the claims (0: ring-bound)
  uint64_t n_entries, upe, n_units, n_tasks;
  const uint16_t *b_tiles;
  uint32_t *out;
  uint8_t *ring;                        // [R][8 slots][kch] x 16 KB
  uint32_t *ready, *consumed;           // [R] each
  unsigned long long *ctr;              // [0] next unit, [1] next ingest task
  unsigned int *err;
  unsigned long long *prof;             // wait-cycle counters (traced instantiation only)
  CUtensorMap ct_map;                   // box (8 slots, 1, 2, 64 k, 16 clients)
  TcLimb limb[GPIR_MAX_LIMBS];
};


// Two fp16 digits u of x0, x1 (x' = x + 0x808080 precomputed) packed as
// f16x2: PRMT/LOP3 build the halves 0x6400 | byte (= 1024 + byte exactly),
// one HADD2 subtracts 1024 + 128 (1024 for the top digit) from both.
__device__ __forceinline__ uint32_t digits2_f16(uint32_t xp0, uint32_t xp1, int u) {
  const uint32_t t = (__byte_perm(xp0, xp1, (uint32_t)(u | (u << 4) | ((u + 4) << 8) | ((u + 4) << 12))) &
                      0x00FF00FFu) | 0x64006400u;
  const __half2 magic = u < 3 ? __half2half2(__ushort_as_half((unsigned short)0xE480))    // -1152
                              : __half2half2(__ushort_as_half((unsigned short)0xE400));   // -1024
  __half2 h = __hadd2(*reinterpret_cast<const __half2 *>(&t), magic);
  return *reinterpret_cast<uint32_t *>(&h);
}

// Wait-cycle counters of the fused kernel (summed over CTAs; one thread per
// role counts), compiled in only for the traced instantiation and read
// through gpir_trace_counters.
enum FusedCounter {
  kPWaitReady = 0,    // producer waits for the ingest (ring entry not ready)
  kPWaitEmpty,        // producer waits for a free smem stage (MMA behind)
  kMWaitFull,         // MMA thread waits for operands
  kMWaitAccEmpty,     // MMA thread waits for the epilogue to drain
  kEWaitAccFull,      // epilogue waits for the MMAs
  kEWaitStage,        // epilogue waits for the store warp to drain out_stage
  kIWaitConsumed,     // ingest waits for a ring entry to be released
  kIWaitBox,          // ingest waits for its TMA box
  kIBusy,             // ingest converting and storing
  kIWaitSlabs,        // cluster ingest: waiting until the previous slabs have left staging
  kIPush,             // cluster ingest: issuing the slab copies to the peers
  kCtaCycles,         // whole kernel, per CTA
  kNumFusedCounters
};

template <bool PROF, bool PAIR>
__global__ void __launch_bounds__(FUSED_THREADS, 1) tc_fused_kernel(const __grid_constant__ FusedParams p) {
  constexpr int NST = PAIR ? P_STAGES : FSTAGES;
  constexpr int SBYTES = PAIR ? P_STAGE_BYTES : STAGE_BYTES;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t *rawbuf = smem + NST * SBYTES;
  uint32_t *out_stage = reinterpret_cast<uint32_t *>(rawbuf + F_RAW_BYTES);   // [32 m][64 n], swizzled
  uint64_t *full = reinterpret_cast<uint64_t *>(rawbuf + F_RAW_BYTES + F_OUT_BYTES);
  uint64_t *empty = full + NST;
  uint64_t *acc_full = empty + NST;
  uint64_t *acc_empty = acc_full + 2;
  uint64_t *raw_bar = acc_empty + 2;
  uint64_t *stage_unit = raw_bar + 1;                 // [NST]
  uint64_t *acc_unit = stage_unit + NST;              // [2]
  uint64_t *task_slot = acc_unit + 2;                 // claimed ingest task
  uint64_t *ostage_full = task_slot + 1;              // out_stage holds a unit's block
  uint64_t *ostage_empty = ostage_full + 1;           // the store warp has drained it
  uint64_t *ostage_unit = ostage_empty + 1;           // whose block (or kNoUnit)
  uint64_t *pfull = ostage_unit + 1;                  // pair: [NST] the odd CTA's operands have landed
  uint64_t *mail = pfull + (PAIR ? NST : 0);          // pair: [P_MAIL] claimed units, even -> odd CTA
  uint64_t *mail_full = mail + (PAIR ? P_MAIL : 0);
  uint64_t *mail_empty = mail_full + (PAIR ? P_MAIL : 0);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mail_empty + (PAIR ? P_MAIL : 0));
  volatile uint32_t *abort_flag = tmem_slot + 1;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = PAIR ? cluster_rank() : 0u;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      if (PAIR) mbar_init(&pfull[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 2);      // the MMA commit + the MMA thread's arrive after writing acc_unit
      // pair: the even CTA's MMAs wait for both CTAs' epilogues
      mbar_init(&acc_empty[b], (PAIR && rank == 0) ? 2 * F_EPI_WARPS : F_EPI_WARPS);
    }
    if (PAIR)
      for (int i = 0; i < P_MAIL; ++i) {
        mbar_init(&mail_full[i], 1);
        mbar_init(&mail_empty[i], 1);
      }
    mbar_init(raw_bar, 1);
    mbar_init(ostage_full, F_EPI_WARPS);
    mbar_init(ostage_empty, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    if constexpr (PAIR) {
      // one warp of each CTA of the pair allocates the same columns in both
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                   "r"(TMEM_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                   "r"(TMEM_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
  }
  tc_fence_before();
  if constexpr (PAIR)
    cluster_sync_all();   // both CTAs' barriers and tensor memory exist before either uses the other's
  else
    __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  auto try_wait = [&](uint64_t *bar, uint32_t parity) -> bool {
    if constexpr (PAIR)
      return mbar_try_wait_cluster(bar, parity);
    else
      return mbar_try_wait(bar, parity);
  };
  auto wait = [&](uint64_t *bar, uint32_t parity, unsigned int code) -> bool {
    if (try_wait(bar, parity)) return true;
    uint64_t t0 = globaltimer_ns();
    for (uint32_t n = 1;; ++n) {
      if (try_wait(bar, parity)) return true;
      if ((n & 63u) == 0) {
        if (*abort_flag) return false;
        if (globaltimer_ns() - t0 > kWaitLimitNs) {
          atomicCAS(p.err, 0u, code);
          *abort_flag = 1;
          return false;
        }
      }
    }
  };
  // Bounded wait for the unit claim counter to reach `target`.
  auto wait_claims = [&](uint64_t target) -> bool {
    auto seen = [&]() {
      unsigned long long v;
      asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(&p.ctr[0]) : "memory");
      return v >= target;
    };
    if (seen()) return true;
    uint64_t t0 = globaltimer_ns();
    for (uint32_t n = 1;; ++n) {
      __nanosleep(64);
      if (seen()) return true;
      if ((n & 15u) == 0) {
        if (*abort_flag) return false;
        if (globaltimer_ns() - t0 > kWaitLimitNs) {
          atomicCAS(p.err, 0u, (unsigned int)kErrQueueWait);
          *abort_flag = 1;
          return false;
        }
      }
    }
  };
  // Bounded wait for a global counter to reach `target`.
  auto wait_count = [&](const uint32_t *ctr, uint32_t target) -> bool {
    if (ld_acquire(ctr) >= target) return true;
    uint64_t t0 = globaltimer_ns();
    for (uint32_t n = 1;; ++n) {
      __nanosleep(64);
      if (ld_acquire(ctr) >= target) return true;
      if ((n & 15u) == 0) {
        if (*abort_flag) return false;
        if (globaltimer_ns() - t0 > kWaitLimitNs) {
          atomicCAS(p.err, 0u, (unsigned int)kErrQueueWait);
          *abort_flag = 1;
          return false;
        }
      }
    }
  };
  uint64_t pc[PROF ? kNumFusedCounters : 1];
#pragma unroll
  for (int i = 0; i < (PROF ? kNumFusedCounters : 1); ++i) pc[i] = 0;
  const uint64_t kstart = PROF ? clock64() : 0;
  // time a wait into counter `k` (traced instantiation only)
#define FUSED_TIMED(k, expr)                              \
  ([&]() {                                                 \
    const uint64_t _t0 = PROF ? clock64() : 0;             \
    const bool _r = (expr);                                \
    if (PROF) pc[PROF ? (k) : 0] += clock64() - _t0;       \
    return _r;                                             \
  }())

  if (warp == 0) {
    // ---------------- producer: claims units ----------------
    if (lane == 0) {
      uint32_t st = 0, ph = 0;
      bool ok = true;
      const uint64_t pol_first = l2_policy_evict_first();
      constexpr uint32_t B_BYTES = PAIR ? B_TILE_BYTES / 2 : B_TILE_BYTES;   // pair: this CTA's half of B
      uint32_t mi = 0;                                                      // pair: mailbox sequence number
      for (;;) {
        uint64_t u;
        if constexpr (PAIR) {
          const uint32_t ms = mi % P_MAIL, mph = (mi / P_MAIL) & 1u;
          ++mi;
          if (rank == 0) {
            u = atomicAdd(&p.ctr[0], 1ull);
            if (u >= p.n_units) u = kNoUnit;
            if (!(ok = wait(&mail_empty[ms], mph ^ 1u, kErrQueueWait))) break;
            st_cluster_u64(map_peer(smem_u32(&mail[ms]), 1), u);
            mbar_arrive_remote(map_peer(smem_u32(&mail_full[ms]), 1));
          } else {
            if (!(ok = wait(&mail_full[ms], mph, kErrQueueWait))) break;
            u = *reinterpret_cast<volatile uint64_t *>(&mail[ms]);
            mbar_arrive_remote(map_peer(smem_u32(&mail_empty[ms]), 0));
          }
          if (u == kNoUnit) break;
        } else {
          u = atomicAdd(&p.ctr[0], 1ull);
          if (u >= p.n_units) break;
        }
        const uint64_t E = PAIR ? (u / p.upe) * 2 + rank : u / p.upe;
        const uint32_t w = (uint32_t)(u % p.upe), sl = w / p.nblk, nb = w % p.nblk;
        const uint32_t g = (uint32_t)(E / p.mblk);
        const uint64_t slot = (uint64_t)(g / p.gpl) * p.N + (g % p.gpl) * 8 + sl;
        if (!(ok = FUSED_TIMED(kPWaitReady,
                               wait_count(&p.ready[E % p.R], (uint32_t)((E / p.R + 1) * p.kch))))) break;
        fence_proxy_async_global();
        const uint8_t *a_src = p.ring + (((E % p.R) * 8 + sl) * p.kch) * (uint64_t)A_TILE_BYTES;
        const uint8_t *b_src = (const uint8_t *)p.b_tiles + ((slot * p.nblk + nb) * p.kch) * (uint64_t)B_TILE_BYTES +
                               (PAIR ? rank * (uint64_t)B_BYTES : 0ull);
        for (uint32_t kc = 0; kc < p.kch; ++kc) {
          if (!(ok = FUSED_TIMED(kPWaitEmpty, wait(&empty[st], ph ^ 1u, kErrTmaWait)))) break;
          stage_unit[st] = u;   // read by the MMA thread on the unit's first stage
          uint8_t *sa = smem + st * SBYTES;
          mbar_arrive_expect_tx(&full[st], SBYTES);
          bulk_g2s(sa, a_src + (uint64_t)kc * A_TILE_BYTES, A_TILE_BYTES, &full[st]);
          if (p.hints & kHintDbEvictFirst)
            bulk_g2s_hint(sa + A_TILE_BYTES, b_src + (uint64_t)kc * B_TILE_BYTES, B_BYTES, &full[st], pol_first);
          else
            bulk_g2s(sa + A_TILE_BYTES, b_src + (uint64_t)kc * B_TILE_BYTES, B_BYTES, &full[st]);
          if (++st == NST) {
            st = 0;
            ph ^= 1u;
          }
        }
        if (!ok) break;
      }
      // end of work: one empty stage carrying the sentinel
      if (ok && wait(&empty[st], ph ^ 1u, kErrTmaWait)) {
        stage_unit[st] = kNoUnit;
        mbar_arrive(&full[st]);
        if constexpr (PAIR) {
          // the last multicast commits target this CTA's empty barriers too:
          // let them land before the CTA can leave
          for (int s2 = 1; s2 < NST; ++s2) {
            if (++st == NST) {
              st = 0;
              ph ^= 1u;
            }
            mbar_wait_bounded(&empty[st], ph ^ 1u, nullptr, 0);
          }
        }
      } else {
        for (int s2 = 0; s2 < NST; ++s2) mbar_wait_bounded(&empty[s2], ph ^ 1u, nullptr, 0);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      uint32_t st = 0, ph = 0, buf = 0;
      uint32_t aph[2] = {0, 0};
      bool ok = true;
      const uint32_t kgroups = (p.kch + F_KGROUP_CHUNKS - 1) / F_KGROUP_CHUNKS;
      for (;;) {
        // first stage of the next unit (or the sentinel)
        if (!(ok = FUSED_TIMED(kMWaitFull, wait(&full[st], ph, kErrTmaWait)))) break;
        const uint64_t u = stage_unit[st];
        if (u == kNoUnit) {
          if ((ok = wait(&acc_empty[buf], aph[buf] ^ 1u, kErrMmaWait))) {
            acc_unit[buf] = kNoUnit;
            mbar_arrive_cnt(&acc_full[buf], 2);
          }
          break;
        }
        bool first = true;
        for (uint32_t gi = 0; gi < kgroups && ok; ++gi) {
          if (!(ok = FUSED_TIMED(kMWaitAccEmpty, wait(&acc_empty[buf], aph[buf] ^ 1u, kErrMmaWait)))) break;
          tc_fence_after();
          const uint32_t tmem_d = tmem_base + buf * 256;
          const uint32_t c0 = gi * F_KGROUP_CHUNKS;
          const uint32_t c1 = min(p.kch, c0 + F_KGROUP_CHUNKS);
          for (uint32_t kc = c0; kc < c1; ++kc) {
            if (!first && !(ok = FUSED_TIMED(kMWaitFull, wait(&full[st], ph, kErrTmaWait)))) break;
            first = false;
            if constexpr (PAIR) {
              if (rank != 0) {
                // odd CTA: its operands of stage st have landed (the bulk copies
                // completed before full[st] did); tell the issuer
                mbar_arrive_remote_relaxed(map_peer(smem_u32(&pfull[st]), 0));
                if (++st == NST) {
                  st = 0;
                  ph ^= 1u;
                }
                continue;
              }
              if (!(ok = FUSED_TIMED(kMWaitFull, wait(&pfull[st], ph, kErrTmaWait)))) break;
            }
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + st * SBYTES);
            const uint32_t sb = sa + A_TILE_BYTES;
#pragma unroll
            for (int k16 = 0; k16 < KCHUNK / 16; ++k16) {
              if constexpr (PAIR)
                mma_f16_pair(tmem_d, sw128_desc(sa + k16 * 32), sw128_desc(sb + k16 * 32),
                             (kc > c0 || k16 > 0) ? 1u : 0u);
              else
                mma_f16(tmem_d, sw128_desc(sa + k16 * 32), sw128_desc(sb + k16 * 32),
                        (kc > c0 || k16 > 0) ? 1u : 0u);
            }
            if constexpr (PAIR)
              mma_commit_pair(&empty[st]);
            else
              mma_commit(&empty[st]);
            if (++st == NST) {
              st = 0;
              ph ^= 1u;
            }
          }
          if (!ok) break;
          acc_unit[buf] = u | ((gi + 1 == kgroups) ? (1ull << 63) : 0ull);   // unit id, top bit: last group
          if constexpr (PAIR) {
            if (rank == 0) mma_commit_pair(&acc_full[buf]);   // the odd CTA gets this commit too
          } else {
            mma_commit(&acc_full[buf]);
          }
          mbar_arrive(&acc_full[buf]);
          aph[buf] ^= 1u;
          buf ^= 1u;
        }
        if (!ok) break;
      }
      if (!ok)
        for (int b = 0; b < 2; ++b) mbar_wait_bounded(&acc_full[b], aph[b], nullptr, 0);
    }
  } else if (warp < 2 + F_EPI_WARPS) {
    // ---------------- epilogue (8 warps) ----------------
    constexpr int CHUNKS = 8 / (F_EPI_WARPS / 4);
    const uint32_t quarter = warp & 3;
    const int jbase = ((warp - 2) >> 2) * CHUNKS;
    const int u = lane >> 3, m_lo = lane & 7;
    const int m_local = quarter * 8 + m_lo;
    const bool odd = (u & 1) != 0, high = (u & 2) != 0;
    const bool signaller = (warp == 2 && lane == 0);
    const int et = (int)threadIdx.x - 64;   // 0..255 over the epilogue warps
    // Barrier 2 spans the 256 epilogue threads; every exit decision goes
    // through a barrier AND, so no thread leaves while others wait there.
    auto epi_sync = [&]() { asm volatile("bar.sync 2, %0;" ::"n"(32 * F_EPI_WARPS) : "memory"); };
    auto epi_all = [&](bool v) -> bool {
      uint32_t r = v ? 1u : 0u;
      asm volatile(
          "{\n .reg .pred pin, pout;\n setp.ne.u32 pin, %1, 0;\n bar.red.and.pred pout, 2, %2, pin;\n"
          " selp.u32 %0, 1, 0, pout;\n}"
          : "=r"(r)
          : "r"(r), "n"(32 * F_EPI_WARPS)
          : "memory");
      return r != 0;
    };
    uint32_t buf = 0, oph = 0, ngroups = 0;
    uint32_t aph[2] = {0, 0};
    uint32_t res[2 * CHUNKS];     // reduced partial results of the current unit
    int64_t acc64[2 * CHUNKS];    // unreduced group sums since the last reduction
#pragma unroll
    for (int i = 0; i < 2 * CHUNKS; ++i) {
      res[i] = 0;
      acc64[i] = 0;
    }
    for (;;) {
      bool okw;
      if (warp == 2 && lane == 0) okw = FUSED_TIMED(kEWaitAccFull, wait(&acc_full[buf], aph[buf], kErrMmaWait));
      else okw = wait(&acc_full[buf], aph[buf], kErrMmaWait);
      if (!epi_all(okw)) break;
      tc_fence_after();
      const uint64_t tag = acc_unit[buf];
      if (tag == kNoUnit) {
        // pass the end of work on to the store warp
        if (epi_all(wait(ostage_empty, oph ^ 1u, kErrMmaWait))) {
          if (et == 0) *ostage_unit = kNoUnit;
          __syncwarp();
          if (lane == 0) mbar_arrive(ostage_full);
        }
        break;
      }
      const uint64_t un = tag & ~(1ull << 63);
      const bool last = (tag >> 63) != 0;
      const uint64_t E = PAIR ? (un / p.upe) * 2 + rank : un / p.upe;   // this CTA's entry
      const uint32_t l = (uint32_t)(E / p.mblk) / p.gpl;
      const TcLimb &lm = p.limb[l];
      if (last && signaller) atomicAdd(&p.consumed[E % p.R], 1u);   // its ring tiles are no longer needed
      const int32_t c0 = lm.c[u], c1 = lm.c[u + 1], c2 = lm.c[u + 2], c3 = lm.c[u + 3];
      const uint32_t taddr = tmem_base + ((quarter * 32u) << 16) + buf * 256 + jbase * 32;
#pragma unroll
      for (int j = 0; j < CHUNKS; ++j) {
        uint32_t d[32];
        tmem_ld32(taddr + j * 32, d);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          int64_t P[4];
#pragma unroll
          for (int ww = 0; ww < 4; ++ww) {
            const int n8 = h * 4 + ww;
            const int32_t b0 = __float2int_rn(__uint_as_float(d[n8 * 4 + 0]));
            const int32_t b1 = __float2int_rn(__uint_as_float(d[n8 * 4 + 1]));
            const int32_t b2 = __float2int_rn(__uint_as_float(d[n8 * 4 + 2]));
            const int32_t b3 = __float2int_rn(__uint_as_float(d[n8 * 4 + 3]));
            P[ww] = (int64_t)b0 * c0 + (int64_t)b1 * c1 + (int64_t)b2 * c2 + (int64_t)b3 * c3;
          }
          int64_t k0 = odd ? P[1] : P[0], k1 = odd ? P[3] : P[2];
          const int64_t s0 = odd ? P[0] : P[1], s1 = odd ? P[2] : P[3];
          k0 += __shfl_xor_sync(0xffffffffu, s0, 8);
          k1 += __shfl_xor_sync(0xffffffffu, s1, 8);
          int64_t keep = high ? k1 : k0;
          const int64_t send = high ? k0 : k1;
          keep += __shfl_xor_sync(0xffffffffu, send, 16);
          acc64[j * 2 + h] += keep;
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&acc_empty[buf]);
        // the issuer's count; the tensor-memory loads above have completed
        if (PAIR && rank != 0) mbar_arrive_remote_relaxed(map_peer(smem_u32(&acc_empty[buf]), 0));
      }
      aph[buf] ^= 1u;
      buf ^= 1u;
      if (last || ++ngroups == F_FLUSH_GROUPS) {
        // one Barrett reduction for up to F_FLUSH_GROUPS groups
#pragma unroll
        for (int i = 0; i < 2 * CHUNKS; ++i) {
          const uint32_t rr = reduce64((uint64_t)(acc64[i] + (int64_t)lm.off58), lm.q, lm.mu);
          const uint32_t a = res[i] + rr;
          res[i] = a >= lm.q ? a - lm.q : a;
          acc64[i] = 0;
        }
        ngroups = 0;
      }
      if (last) {
        // Hand the unit's 32 x 64 block to the store warp through out_stage
        // (the scattered 4-byte output stores then stay off these warps).
        const bool oke = (et == 0) ? FUSED_TIMED(kEWaitStage, wait(ostage_empty, oph ^ 1u, kErrMmaWait))
                                   : wait(ostage_empty, oph ^ 1u, kErrMmaWait);
        if (!epi_all(oke)) break;
        const uint32_t swz = (uint32_t)m_lo << 2;   // 16-byte groups swizzled by row: conflict-free
#pragma unroll
        for (int j = 0; j < CHUNKS; ++j)
#pragma unroll
          for (int h = 0; h < 2; ++h)
            out_stage[m_local * NCOLS + ((uint32_t)((jbase + j) * 8 + h * 4 + u) ^ swz)] = res[j * 2 + h];
        if (et == 0) *ostage_unit = un;
        __syncwarp();
        if (lane == 0) mbar_arrive(ostage_full);
        oph ^= 1u;
#pragma unroll
        for (int i = 0; i < 2 * CHUNKS; ++i) res[i] = 0;
      }
    }
  } else if (warp == F_STORE_WARP) {
    // ---------------- output store warp ----------------
    // Drains out_stage into the p-major output. out[c][n][r][l][t] has the
    // slot innermost and a unit owns one slot, so these are 4-byte stores,
    // one sector each; issuing them here keeps them off the epilogue warps.
    uint32_t ph = 0;
    for (;;) {
      const bool okw = __all_sync(0xffffffffu, wait(ostage_full, ph, kErrMmaWait));
      if (!okw) break;
      const uint64_t un = *ostage_unit;
      if (un == kNoUnit) break;
      const uint64_t E = PAIR ? (un / p.upe) * 2 + rank : un / p.upe;
      const uint32_t w = (uint32_t)(un % p.upe), sl = w / p.nblk, nb = w % p.nblk;
      const uint32_t g = (uint32_t)(E / p.mblk), mb = (uint32_t)(E % p.mblk);
      const uint32_t l = g / p.gpl, t = (g % p.gpl) * 8 + sl;
      const uint32_t mrows = min((uint32_t)MROWS, p.M - mb * MROWS);
      const uint32_t ncols = min((uint32_t)NCOLS, p.d1 - nb * NCOLS);
      for (uint32_t m = 0; m < mrows; ++m) {
        const uint32_t mg = mb * MROWS + m, c = mg >> 1, rr = mg & 1;
        const uint32_t sw = (m & 7u) << 2;
        uint32_t *orow = p.out + (((uint64_t)c * p.d1 + nb * NCOLS) * 2 + rr) * p.L * p.N + (uint64_t)l * p.N + t;
        const uint64_t nstride = (uint64_t)2 * p.L * p.N;
#pragma unroll
        for (uint32_t h = 0; h < NCOLS / 32; ++h) {
          const uint32_t n = h * 32 + lane;
          if (n < ncols) orow[n * nstride] = out_stage[m * NCOLS + (n ^ sw)];
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(ostage_empty);
      ph ^= 1u;
    }
  } else {
    // ---------------- ingest (8 warps, 256 threads) ----------------
    // Task = (entry E, k-chunk kc): 64 k of 8 slots x 32 rows, one 64 KB TMA
    // box. Thread (m_local, j) handles k octet j of row m_local for all 8
    // slots; its 16-byte chunk goes to position cp = j ^ (m_local % 8) of tile
    // row m_hi*32 + u*8 + m_lo, so each warp store covers 8 contiguous 64-byte
    // half rows of one tile. Every exit decision is uniform over the 256
    // threads (a value thread 0 publishes before a named barrier, or a barrier
    // AND), so no thread can leave while the others wait at the next named
    // barrier.
    const int iw = warp - (2 + F_EPI_WARPS);
    const int it = iw * 32 + lane;
    const int m_hi = iw >> 1, m_lo = lane & 7;
    const int j = (iw & 1) * 4 + (lane >> 3);
    const int m_local = m_hi * 8 + m_lo;
    const int cc = m_local >> 1, rp = m_local & 1;
    const uint64_t pol_first = l2_policy_evict_first(), pol_last = l2_policy_evict_last();
    const bool ring_last = (p.hints & kHintRingEvictLast) != 0;
    uint32_t rph = 0;
    bool issued = false;
    for (;;) {
      if (it == 0) {
        const uint64_t c = atomicAdd(&p.ctr[1], 1ull);
        *task_slot = (c < p.n_tasks && !*abort_flag) ? c : kNoUnit;
      }
      asm volatile("bar.sync 1, %0;" ::"n"(32 * F_INGEST_WARPS) : "memory");
      const uint64_t c = *task_slot;
      if (c == kNoUnit) break;
      const uint64_t E = c / p.kch;
      const uint32_t kc = (uint32_t)(c % p.kch);
      const uint32_t g = (uint32_t)(E / p.mblk), mb = (uint32_t)(E % p.mblk);
      const uint32_t l = g / p.gpl, t0 = (g % p.gpl) * 8;
      asm volatile("bar.sync 1, %0;" ::"n"(32 * F_INGEST_WARPS) : "memory");   // everyone has read task_slot
      if (it == 0) {
        // the ring entry's previous occupant must be fully consumed, and the
        // ingest stays within `lookahead` entries of the GEMM units' claims
        // (so that ring lines are read back while still in L2)
        const bool near = p.lookahead == 0 || E < p.lookahead ||
                          FUSED_TIMED(kIWaitConsumed, wait_claims(((E - p.lookahead) >> (PAIR ? 1 : 0)) * p.upe));
        if (near && (E < p.R || FUSED_TIMED(kIWaitConsumed,
                                            wait_count(&p.consumed[E % p.R], (uint32_t)((E / p.R) * p.upe))))) {
          mbar_arrive_expect_tx(raw_bar, F_RAW_BYTES);
          if (p.hints & kHintCtEvictFirst)
            tma_load_5d_hint(rawbuf, &p.ct_map, raw_bar, (int)t0, (int)l, 0, (int)(kc * KCHUNK),
                             (int)(mb * (MROWS / 2)), pol_first);
          else
            tma_load_5d(rawbuf, &p.ct_map, raw_bar, (int)t0, (int)l, 0, (int)(kc * KCHUNK), (int)(mb * (MROWS / 2)));
          issued = true;
          *task_slot = c;
        } else {
          *task_slot = kNoUnit;
        }
      }
      asm volatile("bar.sync 1, %0;" ::"n"(32 * F_INGEST_WARPS) : "memory");
      if (*task_slot == kNoUnit) break;
      uint32_t got = (it == 0 ? FUSED_TIMED(kIWaitBox, wait(raw_bar, rph, kErrTmaWait))
                              : wait(raw_bar, rph, kErrTmaWait)) ? 1u : 0u;
      asm volatile(
          "{\n .reg .pred pin, pout;\n setp.ne.u32 pin, %1, 0;\n bar.red.and.pred pout, 1, %2, pin;\n"
          " selp.u32 %0, 1, 0, pout;\n}"
          : "=r"(got)
          : "r"(got), "n"(32 * F_INGEST_WARPS)
          : "memory");
      if (!got) break;
      rph ^= 1u;
      if (it == 0) issued = false;
      const uint64_t tbusy = PROF ? clock64() : 0;
      const int cp = (int)(j ^ m_lo);
      const uint4 *raw4 = reinterpret_cast<const uint4 *>(rawbuf);
      uint4 *ring4 = reinterpret_cast<uint4 *>(p.ring);
#pragma unroll
      for (int s4 = 0; s4 < 2; ++s4) {                  // which 4-slot half of the 32-byte row
        uint32_t v[8][4];   // [kk][slot in half]: residue + 0x808080
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          const uint4 q4 = raw4[((cc * KCHUNK + j * 8 + kk) * 2 + rp) * 2 + s4];
          v[kk][0] = q4.x + 0x808080u;
          v[kk][1] = q4.y + 0x808080u;
          v[kk][2] = q4.z + 0x808080u;
          v[kk][3] = q4.w + 0x808080u;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int sl = s4 * 4 + i;
          if (t0 + sl >= p.N) continue;
          uint4 *tile = ring4 + ((((E % p.R) * 8 + sl) * p.kch + kc) * (uint64_t)A_TILE_BYTES) / 16;
#pragma unroll
          for (int uu = 0; uu < 4; ++uu) {
            uint4 w4;
            w4.x = digits2_f16(v[0][i], v[1][i], uu);
            w4.y = digits2_f16(v[2][i], v[3][i], uu);
            w4.z = digits2_f16(v[4][i], v[5][i], uu);
            w4.w = digits2_f16(v[6][i], v[7][i], uu);
            if (ring_last)
              st_global_v4_hint(&tile[(m_hi * 32 + uu * 8 + m_lo) * 8 + cp], w4, pol_last);
            else
              tile[(m_hi * 32 + uu * 8 + m_lo) * 8 + cp] = w4;
          }
        }
      }
      fence_proxy_async_global();
      asm volatile("bar.sync 1, %0;" ::"n"(32 * F_INGEST_WARPS) : "memory");
      if (it == 0) {
        __threadfence();   // cumulative: orders the group's tile stores (seen through the barrier) before the count
        atomicAdd(&p.ready[E % p.R], 1u);
      }
      if (PROF) pc[PROF ? kIBusy : 0] += clock64() - tbusy;
    }
    if (it == 0 && issued) mbar_wait_bounded(raw_bar, rph, nullptr, 0);   // let a late box land
  }
#undef FUSED_TIMED
  if (PROF) {
    // one counting thread per role: producer, MMA, epilogue warp 2, ingest thread 0
    const bool counter = (lane == 0) && (warp <= 2 || warp == 2 + F_EPI_WARPS);
    if (counter)
      for (int i = 0; i < (PROF ? kNumFusedCounters : 1) - 1; ++i)
        if (pc[i]) atomicAdd(&p.prof[i], pc[i]);
    if (threadIdx.x == 0) atomicAdd(&p.prof[kCtaCycles], clock64() - kstart);
  }
  tc_fence_before();
  if constexpr (PAIR)
    cluster_sync_all();   // no peer still reads this CTA's memory or arrives on its barriers
  else
    __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    if constexpr (PAIR)
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                   : "memory");
    else
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                   : "memory");
  }
}

// ---- cluster kernel: the 8 CTAs of a cluster share the raw ciphertexts ----
//
// A thread-block cluster of 8 CTAs takes one entry E = (8-slot group g,
// m-block mb) at a time; CTA rank r computes slot r of the group (all n-blocks
// in turn). The raw residues of the entry arrive p-major, 8 slots per 32-byte
// row, so each CTA loads only its share of the rows (2 of the 16 clients)
// with one 8 KB TMA box per k-chunk, splits them into digits for all 8 slots,
// and stores each slot's digit rows straight into the owning CTA's A stage
// through distributed shared memory. No digit tile ever leaves the cluster,
// so the ciphertexts cross HBM once and the L2 sees only raw boxes and
// database tiles.
//
// Per stage st (one k-chunk of one unit (E, nb)) in every CTA:
//   full_a[st]  8 arrivals: each CTA of the cluster has written its rows
//   full_b[st]  the CTA's own database tile (bulk copy, 32 KB)
//   empty[st]   8 arrivals: every CTA's MMAs have read stage st (multicast
//               commits), so the stage may be refilled everywhere
// All CTAs walk the same static sequence of stages (entries E = cluster id
// + i x clusters), so the barrier phases stay aligned across the cluster.
// All waits are bounded; before exiting, each CTA drains the arrivals that
// target its own barriers and the cluster synchronizes once, so no CTA
// leaves while a peer may still write into its shared memory.

constexpr int CL = 8;                                           // CTAs per cluster = slots per group
constexpr int C_STAGES = 4;                                     // operand stages (48 KB each)
constexpr int C_SHARE_CLIENTS = 16 / CL;                        // clients of an m-block per CTA
constexpr int C_RAW_BYTES = C_SHARE_CLIENTS * 2 * KCHUNK * 8 * 4;   // 8 KB share of a raw box
constexpr int C_SLAB_BYTES = A_TILE_BYTES / CL;                 // one CTA's 16 rows of an A tile (2 KB)
constexpr int C_STAGING_STRIDE = C_SLAB_BYTES + 16;             // padded: conflict-free staging stores
constexpr int C_STAGING_BYTES = CL * C_STAGING_STRIDE;
constexpr size_t CLUSTER_SMEM =
    1024 + (size_t)C_STAGES * STAGE_BYTES + C_RAW_BYTES + C_STAGING_BYTES + F_OUT_BYTES + 512;
static_assert(CLUSTER_SMEM <= 232448, "cluster kernel shared memory exceeds 227 KB");
static_assert(CL == F_INGEST_WARPS, "one ingest warp per k octet and per destination slab");

struct ClusterParams {
  uint32_t L, N, M, d0, d1, mblk, nblk, kch;
  uint32_t gpl;
  uint64_t n_entries;                   // 8-slot groups x m-blocks
  const uint16_t *b_tiles;
  uint32_t *out;
  unsigned int *err;
  unsigned long long *prof;             // wait-cycle counters (traced instantiation only)
  CUtensorMap ct_map;                   // box (8 slots, 1, 2, 64 k, 2 clients)
  TcLimb limb[GPIR_MAX_LIMBS];
};

template <bool PROF>
__global__ void __launch_bounds__(FUSED_THREADS, 1) tc_cluster_kernel(const __grid_constant__ ClusterParams p) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t *rawbuf = smem + C_STAGES * STAGE_BYTES;                                // 8 KB share of a raw box
  uint8_t *staging = rawbuf + C_RAW_BYTES;                                          // [8 slabs] outgoing rows
  uint32_t *out_stage = reinterpret_cast<uint32_t *>(staging + C_STAGING_BYTES);    // [32 m][64 n], swizzled
  uint64_t *full_a = reinterpret_cast<uint64_t *>(staging + C_STAGING_BYTES + F_OUT_BYTES);
  uint64_t *full_b = full_a + C_STAGES;
  uint64_t *empty = full_b + C_STAGES;
  uint64_t *acc_full = empty + C_STAGES;
  uint64_t *acc_empty = acc_full + 2;
  uint64_t *raw_bar = acc_empty + 2;
  uint64_t *stage_unit = raw_bar + 1;                 // [C_STAGES]
  uint64_t *acc_unit = stage_unit + C_STAGES;         // [2]
  uint64_t *ostage_full = acc_unit + 2;
  uint64_t *ostage_empty = ostage_full + 1;
  uint64_t *ostage_unit = ostage_empty + 1;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(ostage_unit + 1);
  volatile uint32_t *abort_flag = tmem_slot + 1;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const uint64_t cid = cluster_id_x(), ncl = cluster_count_x();
  if (threadIdx.x == 0) {
    for (int s = 0; s < C_STAGES; ++s) {
      mbar_init(&full_a[s], 1);      // the owner's expect-tx arrival; the 8 slabs complete the bytes
      mbar_init(&full_b[s], 1);
      mbar_init(&empty[s], CL);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 2);
      mbar_init(&acc_empty[b], F_EPI_WARPS);
    }
    mbar_init(raw_bar, 1);
    mbar_init(ostage_full, F_EPI_WARPS);
    mbar_init(ostage_empty, 1);
    *abort_flag = 0;
    fence_mbar_init();
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  // every CTA's barriers are initialised before any peer may arrive on them
  asm volatile("barrier.cluster.arrive.release.aligned;\n barrier.cluster.wait.acquire.aligned;" ::: "memory");
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  // Bounded wait on one of this CTA's barriers.
  auto wait_bar = [&](uint64_t *bar, uint32_t parity, unsigned int code) -> bool {
    auto poll = [&]() { return mbar_try_wait(bar, parity); };
    if (poll()) return true;
    uint64_t t0 = globaltimer_ns();
    for (uint32_t n = 1;; ++n) {
      if (poll()) return true;
      if ((n & 63u) == 0) {
        if (*abort_flag) return false;
        if (globaltimer_ns() - t0 > kWaitLimitNs) {
          atomicCAS(p.err, 0u, code);
          *abort_flag = 1;
          return false;
        }
      }
    }
  };
  uint64_t pc[PROF ? kNumFusedCounters : 1];
#pragma unroll
  for (int i = 0; i < (PROF ? kNumFusedCounters : 1); ++i) pc[i] = 0;
  const uint64_t kstart = PROF ? clock64() : 0;
#define CL_TIMED(k, expr)                                  \
  ([&]() {                                                 \
    const uint64_t _t0 = PROF ? clock64() : 0;             \
    const bool _r = (expr);                                \
    if (PROF) pc[PROF ? (k) : 0] += clock64() - _t0;       \
    return _r;                                             \
  }())
  // entry E -> limb, first slot of its group, m-block
  auto entry_of = [&](uint64_t E, uint32_t &l, uint32_t &t0, uint32_t &mb) {
    const uint32_t g = (uint32_t)(E / p.mblk);
    mb = (uint32_t)(E % p.mblk);
    l = g / p.gpl;
    t0 = (g % p.gpl) * 8;
  };

  if (warp == 0) {
    // ---------------- producer: this CTA's database tiles ----------------
    if (lane == 0) {
      uint32_t st = 0, ph = 0;
      bool ok = true;
      for (uint64_t E = cid; E < p.n_entries && ok; E += ncl) {
        uint32_t l, t0, mb;
        entry_of(E, l, t0, mb);
        const uint64_t slot = (uint64_t)l * p.N + t0 + rank;
        for (uint32_t nb = 0; nb < p.nblk && ok; ++nb) {
          const uint8_t *b_src = (const uint8_t *)p.b_tiles + ((slot * p.nblk + nb) * p.kch) * (uint64_t)B_TILE_BYTES;
          for (uint32_t kc = 0; kc < p.kch; ++kc) {
            if (!(ok = CL_TIMED(kPWaitEmpty, wait_bar(&empty[st], ph ^ 1u, kErrTmaWait)))) break;
            stage_unit[st] = E * p.nblk + nb;
            mbar_arrive_expect_tx(&full_a[st], A_TILE_BYTES);   // the 8 CTAs' slabs of this stage
            uint8_t *sb = smem + st * STAGE_BYTES + A_TILE_BYTES;
            mbar_arrive_expect_tx(&full_b[st], B_TILE_BYTES);
            bulk_g2s(sb, b_src + (uint64_t)kc * B_TILE_BYTES, B_TILE_BYTES, &full_b[st]);
            if (++st == C_STAGES) {
              st = 0;
              ph ^= 1u;
            }
          }
        }
      }
      // end of work: one empty stage carrying the sentinel, then drain the
      // last multicast commits that target this CTA's empty barriers
      if (ok && wait_bar(&empty[st], ph ^ 1u, kErrTmaWait)) {
        stage_unit[st] = kNoUnit;
        mbar_arrive(&full_b[st]);
      }
      for (int s2 = 0; s2 < C_STAGES; ++s2) {
        mbar_wait_bounded(&empty[st], ph ^ 1u, nullptr, 0);
        if (++st == C_STAGES) {
          st = 0;
          ph ^= 1u;
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      uint32_t st = 0, ph = 0, buf = 0;
      uint32_t aph[2] = {0, 0};
      bool ok = true;
      const uint32_t kgroups = (p.kch + F_KGROUP_CHUNKS - 1) / F_KGROUP_CHUNKS;
      for (;;) {
        if (!(ok = CL_TIMED(kMWaitFull, wait_bar(&full_b[st], ph, kErrTmaWait)))) break;
        const uint64_t u = stage_unit[st];
        if (u == kNoUnit) {
          if ((ok = wait_bar(&acc_empty[buf], aph[buf] ^ 1u, kErrMmaWait))) {
            acc_unit[buf] = kNoUnit;
            mbar_arrive_cnt(&acc_full[buf], 2);
          }
          break;
        }
        bool first = true;
        for (uint32_t gi = 0; gi < kgroups && ok; ++gi) {
          if (!(ok = CL_TIMED(kMWaitAccEmpty, wait_bar(&acc_empty[buf], aph[buf] ^ 1u, kErrMmaWait)))) break;
          tc_fence_after();
          const uint32_t tmem_d = tmem_base + buf * 256;
          const uint32_t c0 = gi * F_KGROUP_CHUNKS;
          const uint32_t c1 = min(p.kch, c0 + F_KGROUP_CHUNKS);
          for (uint32_t kc = c0; kc < c1; ++kc) {
            if (!first && !(ok = CL_TIMED(kMWaitFull, wait_bar(&full_b[st], ph, kErrTmaWait)))) break;
            first = false;
            if (!(ok = CL_TIMED(kMWaitFull, wait_bar(&full_a[st], ph, kErrTmaWait)))) break;
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + st * STAGE_BYTES);
            const uint32_t sb = sa + A_TILE_BYTES;
#pragma unroll
            for (int k16 = 0; k16 < KCHUNK / 16; ++k16)
              mma_f16(tmem_d, sw128_desc(sa + k16 * 32), sw128_desc(sb + k16 * 32), (kc > c0 || k16 > 0) ? 1u : 0u);
            mma_commit_cluster(&empty[st], (uint16_t)((1u << CL) - 1u));
            if (++st == C_STAGES) {
              st = 0;
              ph ^= 1u;
            }
          }
          if (!ok) break;
          acc_unit[buf] = u | ((gi + 1 == kgroups) ? (1ull << 63) : 0ull);
          mma_commit(&acc_full[buf]);
          mbar_arrive(&acc_full[buf]);
          aph[buf] ^= 1u;
          buf ^= 1u;
        }
        if (!ok) break;
      }
      if (!ok)
        for (int b = 0; b < 2; ++b) mbar_wait_bounded(&acc_full[b], aph[b], nullptr, 0);
    }
  } else if (warp < 2 + F_EPI_WARPS) {
    // ---------------- epilogue (8 warps) ----------------
    constexpr int CHUNKS = 8 / (F_EPI_WARPS / 4);
    const uint32_t quarter = warp & 3;
    const int jbase = ((warp - 2) >> 2) * CHUNKS;
    // A rows are ordered m_hi*32 + (m_lo / 4)*16 + 4u + m_lo % 4, so that
    // each CTA's 16 rows are contiguous: lane = (m_lo / 4)*16 + 4u + m_lo % 4
    const int u = (lane >> 2) & 3, m_lo = ((lane >> 4) << 2) | (lane & 3);
    const int m_local = quarter * 8 + m_lo;
    const bool odd = (u & 1) != 0, high = (u & 2) != 0;
    const int et = (int)threadIdx.x - 64;
    auto epi_all = [&](bool v) -> bool {
      uint32_t r = v ? 1u : 0u;
      asm volatile(
          "{\n .reg .pred pin, pout;\n setp.ne.u32 pin, %1, 0;\n bar.red.and.pred pout, 2, %2, pin;\n"
          " selp.u32 %0, 1, 0, pout;\n}"
          : "=r"(r)
          : "r"(r), "n"(32 * F_EPI_WARPS)
          : "memory");
      return r != 0;
    };
    uint32_t buf = 0, oph = 0, ngroups = 0;
    uint32_t aph[2] = {0, 0};
    uint32_t res[2 * CHUNKS];
    int64_t acc64[2 * CHUNKS];
#pragma unroll
    for (int i = 0; i < 2 * CHUNKS; ++i) {
      res[i] = 0;
      acc64[i] = 0;
    }
    for (;;) {
      bool okw;
      if (warp == 2 && lane == 0) okw = CL_TIMED(kEWaitAccFull, wait_bar(&acc_full[buf], aph[buf], kErrMmaWait));
      else okw = wait_bar(&acc_full[buf], aph[buf], kErrMmaWait);
      if (!epi_all(okw)) break;
      tc_fence_after();
      const uint64_t tag = acc_unit[buf];
      if (tag == kNoUnit) {
        if (epi_all(wait_bar(ostage_empty, oph ^ 1u, kErrMmaWait))) {
          if (et == 0) *ostage_unit = kNoUnit;
          __syncwarp();
          if (lane == 0) mbar_arrive(ostage_full);
        }
        break;
      }
      const uint64_t un = tag & ~(1ull << 63);
      const bool last = (tag >> 63) != 0;
      const uint64_t E = un / p.nblk;
      const uint32_t l = (uint32_t)(E / p.mblk) / p.gpl;
      const TcLimb &lm = p.limb[l];
      const int32_t c0 = lm.c[u], c1 = lm.c[u + 1], c2 = lm.c[u + 2], c3 = lm.c[u + 3];
      const uint32_t taddr = tmem_base + ((quarter * 32u) << 16) + buf * 256 + jbase * 32;
#pragma unroll
      for (int j = 0; j < CHUNKS; ++j) {
        uint32_t d[32];
        tmem_ld32(taddr + j * 32, d);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          int64_t P[4];
#pragma unroll
          for (int ww = 0; ww < 4; ++ww) {
            const int n8 = h * 4 + ww;
            const int32_t b0 = __float2int_rn(__uint_as_float(d[n8 * 4 + 0]));
            const int32_t b1 = __float2int_rn(__uint_as_float(d[n8 * 4 + 1]));
            const int32_t b2 = __float2int_rn(__uint_as_float(d[n8 * 4 + 2]));
            const int32_t b3 = __float2int_rn(__uint_as_float(d[n8 * 4 + 3]));
            P[ww] = (int64_t)b0 * c0 + (int64_t)b1 * c1 + (int64_t)b2 * c2 + (int64_t)b3 * c3;
          }
          int64_t k0 = odd ? P[1] : P[0], k1 = odd ? P[3] : P[2];
          const int64_t s0 = odd ? P[0] : P[1], s1 = odd ? P[2] : P[3];
          k0 += __shfl_xor_sync(0xffffffffu, s0, 4);    // partner lane: u ^ 1
          k1 += __shfl_xor_sync(0xffffffffu, s1, 4);
          int64_t keep = high ? k1 : k0;
          const int64_t send = high ? k0 : k1;
          keep += __shfl_xor_sync(0xffffffffu, send, 8);  // partner lane: u ^ 2
          acc64[j * 2 + h] += keep;
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[buf]);
      aph[buf] ^= 1u;
      buf ^= 1u;
      if (last || ++ngroups == F_FLUSH_GROUPS) {
#pragma unroll
        for (int i = 0; i < 2 * CHUNKS; ++i) {
          const uint32_t rr = reduce64((uint64_t)(acc64[i] + (int64_t)lm.off58), lm.q, lm.mu);
          const uint32_t a = res[i] + rr;
          res[i] = a >= lm.q ? a - lm.q : a;
          acc64[i] = 0;
        }
        ngroups = 0;
      }
      if (last) {
        const bool oke = (et == 0) ? CL_TIMED(kEWaitStage, wait_bar(ostage_empty, oph ^ 1u, kErrMmaWait))
                                   : wait_bar(ostage_empty, oph ^ 1u, kErrMmaWait);
        if (!epi_all(oke)) break;
        const uint32_t swz = (uint32_t)m_lo << 2;
#pragma unroll
        for (int j = 0; j < CHUNKS; ++j)
#pragma unroll
          for (int h = 0; h < 2; ++h)
            out_stage[m_local * NCOLS + ((uint32_t)((jbase + j) * 8 + h * 4 + u) ^ swz)] = res[j * 2 + h];
        if (et == 0) *ostage_unit = un;
        __syncwarp();
        if (lane == 0) mbar_arrive(ostage_full);
        oph ^= 1u;
#pragma unroll
        for (int i = 0; i < 2 * CHUNKS; ++i) res[i] = 0;
      }
    }
  } else if (warp == F_STORE_WARP) {
    // ---------------- output store warp (slot `rank` of the group) ----------------
    uint32_t ph = 0;
    for (;;) {
      const bool okw = __all_sync(0xffffffffu, wait_bar(ostage_full, ph, kErrMmaWait));
      if (!okw) break;
      const uint64_t un = *ostage_unit;
      if (un == kNoUnit) break;
      const uint64_t E = un / p.nblk;
      const uint32_t nb = (uint32_t)(un % p.nblk);
      uint32_t l, t0, mb;
      entry_of(E, l, t0, mb);
      const uint32_t t = t0 + rank;
      const uint32_t mrows = min((uint32_t)MROWS, p.M - mb * MROWS);
      const uint32_t ncols = min((uint32_t)NCOLS, p.d1 - nb * NCOLS);
      for (uint32_t m = 0; m < mrows; ++m) {
        const uint32_t mg = mb * MROWS + m, c = mg >> 1, rr = mg & 1;
        const uint32_t sw = (m & 7u) << 2;
        uint32_t *orow = p.out + (((uint64_t)c * p.d1 + nb * NCOLS) * 2 + rr) * p.L * p.N + (uint64_t)l * p.N + t;
        const uint64_t nstride = (uint64_t)2 * p.L * p.N;
#pragma unroll
        for (uint32_t h = 0; h < NCOLS / 32; ++h) {
          const uint32_t n = h * 32 + lane;
          if (n < ncols) orow[n * nstride] = out_stage[m * NCOLS + (n ^ sw)];
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(ostage_empty);
      ph ^= 1u;
    }
  } else {
    // ---------------- ingest (8 warps, 256 threads) ----------------
    // This CTA's share of entry E is clients 2r, 2r+1 of the m-block: rows
    // m = 4r .. 4r+3 (m = 2 client + polynomial), which in every slot's A
    // tile are the 16 contiguous rows 16r .. 16r+15 (row = 16r + 4u + mm).
    // Warp j takes k octet j; lane (mm, s) takes row 4r + mm of slot s and
    // writes its four 16-byte digit chunks (u = 0..3) into the staging slab
    // of destination CTA s, already in the SW128 position (j ^ (row % 8)).
    // Thread 0 then pushes the 8 slabs (2 KB each) to their CTAs with bulk
    // copies that complete on the owners' full_a barriers. Exit decisions go
    // through a barrier AND.
    const int it = (warp - (2 + F_EPI_WARPS)) * 32 + lane;     // 0..255 (ingest warps 10..17)
    const int j = warp - (2 + F_EPI_WARPS);                     // k octet
    const uint32_t s = (uint32_t)(lane & 7);                    // destination slot = CTA rank
    const int mm = lane >> 3;                                   // row of the share
    const int c2 = mm >> 1, comp = mm & 1;
    auto iall = [&](bool v) -> bool {
      uint32_t r = v ? 1u : 0u;
      asm volatile(
          "{\n .reg .pred pin, pout;\n setp.ne.u32 pin, %1, 0;\n bar.red.and.pred pout, 1, %2, pin;\n"
          " selp.u32 %0, 1, 0, pout;\n}"
          : "=r"(r)
          : "r"(r), "n"(32 * F_INGEST_WARPS)
          : "memory");
      return r != 0;
    };
    auto isync = [&]() { asm volatile("bar.sync 1, %0;" ::"n"(32 * F_INGEST_WARPS) : "memory"); };
    const uint32_t smem_base = smem_u32(smem);
    const uint32_t my_full_a = smem_u32(full_a);
    const uint32_t staging_s = smem_u32(staging);
    // staging byte offsets of this thread's four chunks
    uint32_t soff[4];
#pragma unroll
    for (int uu = 0; uu < 4; ++uu)
      soff[uu] = s * C_STAGING_STRIDE + (uint32_t)((uu * 4 + mm) * 128 + ((j ^ ((uu & 1) * 4 + mm)) * 16));
    uint64_t E = cid;
    uint32_t nb = 0, kc = 0;
    auto issue_box = [&](uint64_t e, uint32_t k) {
      uint32_t l, t0, mb;
      entry_of(e, l, t0, mb);
      mbar_arrive_expect_tx(raw_bar, C_RAW_BYTES);
      tma_load_5d(rawbuf, &p.ct_map, raw_bar, (int)t0, (int)l, 0, (int)(k * KCHUNK),
                  (int)(mb * 16 + rank * C_SHARE_CLIENTS));
    };
    uint32_t st = 0, ph = 0, rph = 0;
    bool issued = false, copies = false;
    if (it == 0 && E < p.n_entries) {
      issue_box(E, 0);
      issued = true;
    }
    while (E < p.n_entries) {
      uint64_t En = E;
      uint32_t nbn = nb, kcn = kc + 1;
      if (kcn == p.kch) {
        kcn = 0;
        if (++nbn == p.nblk) {
          nbn = 0;
          En += ncl;
        }
      }
      bool ok = (it == 0) ? CL_TIMED(kIWaitBox, wait_bar(raw_bar, rph, kErrTmaWait))
                          : wait_bar(raw_bar, rph, kErrTmaWait);
      ok = ok && ((it == 0) ? CL_TIMED(kIWaitConsumed, wait_bar(&empty[st], ph ^ 1u, kErrTmaWait))
                            : wait_bar(&empty[st], ph ^ 1u, kErrTmaWait));
      if (!iall(ok)) break;
      rph ^= 1u;
      if (it == 0) issued = false;
      const uint64_t tbusy = PROF ? clock64() : 0;
      // raw box layout: [client c2][k][poly][slot], 4 bytes each
      const uint32_t *raw = reinterpret_cast<const uint32_t *>(rawbuf);
      uint32_t v[8];
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) v[kk] = raw[((c2 * KCHUNK + j * 8 + kk) * 2 + comp) * 8 + s] + 0x808080u;
      isync();   // the raw box is read: prefetch the next one; the previous slabs must have left staging
      if (it == 0 && En < p.n_entries) {
        issue_box(En, kcn);
        issued = true;
      }
      if (lane == 0 && copies) {
        const uint64_t tw = PROF ? clock64() : 0;
        asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");   // this warp's slab copy
        if (PROF && j == 0) pc[PROF ? kIWaitSlabs : 0] += clock64() - tw;
      }
      isync();
#pragma unroll
      for (int uu = 0; uu < 4; ++uu) {
        uint4 w4;
        w4.x = digits2_f16(v[0], v[1], uu);
        w4.y = digits2_f16(v[2], v[3], uu);
        w4.z = digits2_f16(v[4], v[5], uu);
        w4.w = digits2_f16(v[6], v[7], uu);
        *reinterpret_cast<uint4 *>(staging + soff[uu]) = w4;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // the bulk copies read staging
      isync();
      if (lane == 0) {
        // warp j pushes slab j (this CTA's rows of stage st) to CTA j
        const uint64_t tpush = PROF ? clock64() : 0;
        const uint32_t d = (uint32_t)j;
        const uint32_t dst_local = smem_base + st * STAGE_BYTES + rank * C_SLAB_BYTES;
        asm volatile(
            "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                map_peer(dst_local, d)),
            "r"(staging_s + d * C_STAGING_STRIDE), "n"(C_SLAB_BYTES), "r"(map_peer(my_full_a + st * 8, d))
            : "memory");
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        copies = true;
        if (PROF && j == 0) pc[PROF ? kIPush : 0] += clock64() - tpush;
      }
      if (PROF) pc[PROF ? kIBusy : 0] += clock64() - tbusy;
      if (++st == C_STAGES) {
        st = 0;
        ph ^= 1u;
      }
      E = En;
      nb = nbn;
      kc = kcn;
    }
    if (it == 0 && issued) mbar_wait_bounded(raw_bar, rph, nullptr, 0);   // let a late box land
    if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");   // this warp's slabs have landed
  }
#undef CL_TIMED
  if (PROF) {
    const bool counter = (lane == 0) && (warp <= 2 || warp == 2 + F_EPI_WARPS);
    if (counter)
      for (int i = 0; i < (PROF ? kNumFusedCounters : 1) - 1; ++i)
        if (pc[i]) atomicAdd(&p.prof[i], pc[i]);
    if (threadIdx.x == 0) atomicAdd(&p.prof[kCtaCycles], clock64() - kstart);
  }
  tc_fence_before();
  __syncthreads();
  // no peer may still be writing into this CTA's shared memory or arriving
  // on its barriers once every CTA has passed this point
  asm volatile("barrier.cluster.arrive.release.aligned;\n barrier.cluster.wait.acquire.aligned;" ::: "memory");
  tc_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS) : "memory");
}

static TcLimb make_limb(uint32_t q) {
  TcLimb t;
  t.q = q;
  t.pad = 0;
  t.mu = ~0ull / q;
  const uint64_t two55 = 1ull << 55;
  t.off = ((two55 + q - 1) / q) * (uint64_t)q;
  uint64_t pw = 1;
  for (int s = 0; s < 7; ++s) {
    t.c[s] = (int32_t)(pw % q);
    pw = (pw << 8) % q;
  }
  t.c[7] = 0;
  int64_t csum = 0;
  for (int u = 0; u < 4; ++u)
    for (int v = 0; v < 4; ++v) csum += t.c[u + v];
  t.kfix = (int64_t)0x4B400000 * csum;
  const uint64_t two58 = 1ull << 58;
  t.off58 = ((two58 + q - 1) / q) * (uint64_t)q;
  return t;
}

}  // namespace

// Untuned batches: the tensor-memory kernel, single CTA (variant 8), which
// the autotuner picks from batch 8 up on every database shape measured.
int rowsel_tc_default_variant(uint32_t, uint32_t, uint32_t) { return 8; }

int rowsel_tc_prepare(gpir_db *db, cudaStream_t stream) {
  const uint32_t L = db->params.num_limbs, N = db->params.n;
  const uint32_t nblk = (db->d1 + NCOLS - 1) / NCOLS, kch = (db->d0 + KCHUNK - 1) / KCHUNK;
  const uint64_t slots = (uint64_t)L * N;
  const size_t bytes = (size_t)slots * nblk * kch * B_TILE_BYTES;
  cudaError_t e = dev_malloc(reinterpret_cast<void **>(&db->db_digits), bytes);
  if (e != cudaSuccess) {
    db->db_digits = nullptr;
    return set_cuda_error(e);
  }
  db->db_digits_bytes = bytes;
  PackParams pp;
  pp.d0 = db->d0;
  pp.d1 = db->d1;
  pp.L = L;
  pp.N = N;
  pp.nblk = nblk;
  pp.kch = kch;
  pp.db = db->db_pmajor;
  pp.b_tiles = reinterpret_cast<uint4 *>(db->db_digits);
  const uint64_t total = slots * nblk * kch * 256 * 8;
  tc_pack_db_kernel<<<sm_count() * 16, 256, 0, stream>>>(pp, total);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_cuda_error(e);
  e = cudaStreamSynchronize(stream);
  return e == cudaSuccess ? GPIR_OK : set_cuda_error(e);
}

// ---- host side: shared launch helper ----------------------------------------

namespace {

struct TcShape {
  uint32_t M, mblk, nblk, kch;
  uint64_t slots;
  size_t a_bytes;       // digit-tile workspace of this job
};

TcShape tc_shape(const gpir_db *db, uint32_t batch) {
  TcShape sh;
  sh.M = 2 * batch;
  sh.mblk = (sh.M + MROWS - 1) / MROWS;
  sh.nblk = (db->d1 + NCOLS - 1) / NCOLS;
  sh.kch = (db->d0 + KCHUNK - 1) / KCHUNK;
  sh.slots = (uint64_t)db->params.num_limbs * db->params.n;
  sh.a_bytes = (size_t)sh.slots * sh.mblk * sh.kch * A_TILE_BYTES;
  return sh;
}

std::mutex g_attr_mu;
bool g_attr_done[64];

int tc_set_attributes() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_cuda_error(e);
  if (dev < 0 || dev >= 64) return GPIR_EINVAL;
  std::lock_guard<std::mutex> lk(g_attr_mu);
  if (g_attr_done[dev]) return GPIR_OK;
  e = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GEMM_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc_ingest_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)INGEST_SMEM);
  if (e != cudaSuccess) return set_cuda_error(e);
  g_attr_done[dev] = true;
  return GPIR_OK;
}

// Ingest + persistent GEMM for up to MAX_JOBS problems sharing (N, L, primes);
// job k's digit tiles go to ws + a_off[k]. Two launches on `stream`.
int tc_launch_jobs(const gpir_job_t *jobs, uint32_t njobs, uint8_t *ws, const size_t *a_off, cudaStream_t stream) {
  if (njobs == 0 || njobs > (uint32_t)MAX_JOBS) return GPIR_EINVAL;
  int rc = tc_set_attributes();
  if (rc != GPIR_OK) return rc;
  const gpir_params &prm = jobs[0].db->params;
  const uint32_t L = prm.num_limbs, N = prm.n;
  const uint64_t slots = (uint64_t)L * N;

  IngestParams ip;
  memset(&ip, 0, sizeof(ip));
  ip.L = L;
  ip.N = N;
  ip.gpl = (N + 7) / 8;
  ip.groups8 = ip.gpl * L;
  ip.njobs = njobs;
  ip.err = device_error_word();
  TcParams tp;
  memset(&tp, 0, sizeof(tp));
  tp.L = L;
  tp.N = N;
  tp.njobs = njobs;
  tp.err = device_error_word();
  uint64_t blocks = 0, units = 0;
  for (uint32_t k = 0; k < njobs; ++k) {
    const gpir_db *db = jobs[k].db;
    if (!db->db_digits) return GPIR_ENOTSUP;
    const TcShape sh = tc_shape(db, jobs[k].batch);
    IngestJob &ij = ip.job[k];
    {
      const uint64_t dims[5] = {N, L, 2, db->d0, jobs[k].batch};
      const uint64_t str[4] = {(uint64_t)N * 4, (uint64_t)L * N * 4, (uint64_t)2 * L * N * 4,
                               (uint64_t)db->d0 * 2 * L * N * 4};
      const uint32_t box[5] = {8, 1, 2, (uint32_t)KCHUNK, (uint32_t)(MROWS / 2)};
      int rc2 = encode_tiled_u32(&ip.ct_map[k], jobs[k].ct, 5, dims, str, box);
      if (rc2 != GPIR_OK) return rc2;
    }
    ij.a_tiles = reinterpret_cast<uint4 *>(ws + a_off[k]);
    ij.M = sh.M;
    ij.d0 = db->d0;
    ij.mblk = sh.mblk;
    ij.kch = sh.kch;
    ij.block_begin = (uint32_t)blocks;
    blocks += (uint64_t)ip.groups8 * sh.mblk * sh.kch;
    TcJob &tj = tp.job[k];
    tj.a_tiles = reinterpret_cast<const uint16_t *>(ws + a_off[k]);
    tj.b_tiles = db->db_digits;
    tj.out = jobs[k].out;
    tj.M = sh.M;
    tj.d0 = db->d0;
    tj.d1 = db->d1;
    tj.mblk = sh.mblk;
    tj.nblk = sh.nblk;
    tj.kch = sh.kch;
    tj.unit_begin = units;
    units += slots * sh.mblk * sh.nblk;
    if (blocks > 0x7fffffffull) return GPIR_EINVAL;
  }
  tp.units = units;
  for (uint32_t l = 0; l < L; ++l) tp.limb[l] = make_limb(prm.primes[l]);
  int tr = trace_begin("tc_ingest", stream);
  tc_ingest_kernel<<<(unsigned)blocks, INGEST_THREADS, INGEST_SMEM, stream>>>(ip);
  trace_end(tr, stream);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_cuda_error(e);
  const int grid = (int)std::min<uint64_t>((uint64_t)sm_count(), units);
  tr = trace_begin("tc_gemm", stream);
  tc_gemm_kernel<<<grid, GEMM_THREADS, GEMM_SMEM, stream>>>(tp);
  trace_end(tr, stream);
  e = cudaGetLastError();
  return e == cudaSuccess ? GPIR_OK : set_cuda_error(e);
}

// Digit-tile workspaces, one per (device, stream): work on one stream runs in
// order, so a stream's workspace is never used by two launches at once.
// Grown on demand (after draining that stream), never while the stream is
// being captured.
struct Workspace {
  void *ptr = nullptr;
  size_t bytes = 0;
};
std::mutex g_ws_mu;
std::map<std::pair<int, cudaStream_t>, Workspace> g_ws;

int stream_workspace(cudaStream_t stream, size_t need, uint8_t **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_cuda_error(e);
  std::lock_guard<std::mutex> lk(g_ws_mu);
  Workspace &w = g_ws[{dev, stream}];
  if (w.bytes < need) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(stream, &cs);
    if (cs != cudaStreamCaptureStatusNone) return GPIR_ENOMEM;   // no allocation inside a capture
    if (w.ptr) {
      cudaStreamSynchronize(stream);
      cudaFree(w.ptr);
    }
    w.ptr = nullptr;
    w.bytes = 0;
    e = dev_malloc(&w.ptr, need);
    if (e != cudaSuccess) {
      w.ptr = nullptr;
      return set_cuda_error(e);
    }
    w.bytes = need;
  }
  *out = reinterpret_cast<uint8_t *>(w.ptr);
  return GPIR_OK;
}

}  // namespace

int tc_stream_workspace(cudaStream_t stream, size_t need, uint8_t **out) {
  return stream_workspace(stream, need, out);
}

void rowsel_tc_release_stream(cudaStream_t stream) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  std::lock_guard<std::mutex> lk(g_ws_mu);
  auto it = g_ws.find({dev, stream});
  if (it == g_ws.end()) return;
  if (it->second.ptr) {
    cudaStreamSynchronize(stream);
    cudaFree(it->second.ptr);
  }
  g_ws.erase(it);
}

namespace {

// Fused-kernel tile variants: digit-ring size (against the 129 MB L2) and L2
// eviction hints; the autotuner picks one per shape.
enum TcKernelKind : uint32_t {
  kKindFused = 0,
  kKindTwoPass = 1,
  kKindCluster = 2,
  kKindPair = 3,
  kKindTmem = 4,       // rowsel_tmem.cu: A in tensor memory, 12 digit products
  kKindTmemPair = 5,   // its SM-pair form
};
struct FusedVariant {
  uint32_t kind;           // TcKernelKind
  uint32_t ring_mb;
  uint32_t hints;
  uint32_t lookahead_mb;   // ingest lead over the claim frontier, in ring MB (0: bounded by the ring only)
};
constexpr uint32_t kHintRing = kHintCtEvictFirst | kHintRingEvictLast;
constexpr FusedVariant kFusedVariants[] = {
    {kKindFused, 48, 0, 16},            // 0
    {kKindTwoPass, 0, 0, 0},            // 1: two-pass (ingest to HBM, then GEMM)
    {kKindFused, 48, kHintRing, 0},     // 2
    {kKindFused, 48, 0, 0},             // 3
    {kKindFused, 48, kHintRing, 16},    // 4
    {kKindFused, 40, kHintRing, 16},    // 5
    {kKindCluster, 0, 0, 0},            // 6: 8-CTA clusters sharing raw boxes over DSMEM
    {kKindPair, 48, 0, 16},             // 7: SM pairs (cta_group::2) sharing each database tile
    {kKindTmem, 24, 0, 8},              // 8: A operand in tensor memory, 12 digit products
    {kKindTmemPair, 48, 0, 16},         // 9: its SM-pair form
    {kKindTmem, 24, 1, 8},              // 10: 8 with raw boxes evict-first, ring stores evict-last
    {kKindTmemPair, 48, 1, 16},         // 11: 9 with those hints
};
constexpr int kNumTcVariants = (int)(sizeof(kFusedVariants) / sizeof(kFusedVariants[0]));

std::mutex g_fused_attr_mu;
bool g_fused_attr_done[64];
int g_pair_clusters[64];   // resident CTA pairs of the pair kernel per device (0: not queried yet, -1: none)

cudaLaunchConfig_t pair_config(unsigned grid, cudaStream_t stream, cudaLaunchAttribute *attr) {
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(FUSED_THREADS);
  cfg.dynamicSmemBytes = PAIR_SMEM;
  cfg.stream = stream;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

// One RowSel problem through the fused persistent kernel (ingest warps and
// GEMM warps in one launch; digit tiles only pass through an L2-sized ring).
// pair: the SM-pair form (cta_group::2); GPIR_ENOTSUP when the batch has an
// odd number of 32-row m-blocks or no CTA pair can be resident.
int tc_launch_fused(const gpir_db *db, uint32_t batch, const uint32_t *ct, uint32_t *out, size_t ring_target,
                    uint32_t hints, uint32_t lookahead_mb, bool pair, cudaStream_t stream) {
  if (!db->db_digits) return GPIR_ENOTSUP;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_cuda_error(e);
  if (dev < 0 || dev >= 64) return GPIR_EINVAL;
  const TcShape sh = tc_shape(db, batch);
  if (pair && (sh.mblk & 1u)) return GPIR_ENOTSUP;
  {
    std::lock_guard<std::mutex> lk(g_fused_attr_mu);
    if (!g_fused_attr_done[dev]) {
      e = cudaFuncSetAttribute(tc_fused_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)FUSED_SMEM);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_fused_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)FUSED_SMEM);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_fused_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)PAIR_SMEM);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_fused_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)PAIR_SMEM);
      if (e != cudaSuccess) return set_cuda_error(e);
      cudaLaunchAttribute attr[1];
      const cudaLaunchConfig_t cfg = pair_config((unsigned)(sm_count() / 2 * 2), nullptr, attr);
      int n = 0;
      e = cudaOccupancyMaxActiveClusters(&n, tc_fused_kernel<false, true>, &cfg);
      if (e != cudaSuccess) {
        cudaGetLastError();
        n = 0;
      }
      g_pair_clusters[dev] = n > 0 ? n : -1;
      g_fused_attr_done[dev] = true;
    }
  }
  if (pair && g_pair_clusters[dev] < 0) return GPIR_ENOTSUP;
  const gpir_params &prm = db->params;
  const uint32_t L = prm.num_limbs, N = prm.n;
  FusedParams fp;
  memset(&fp, 0, sizeof(fp));
  fp.L = L;
  fp.N = N;
  fp.M = sh.M;
  fp.d0 = db->d0;
  fp.d1 = db->d1;
  fp.mblk = sh.mblk;
  fp.nblk = sh.nblk;
  fp.kch = sh.kch;
  fp.gpl = (N + 7) / 8;
  fp.n_entries = (uint64_t)fp.gpl * L * sh.mblk;
  fp.spg = N < 8 ? N : 8u;                      // N is a power of two >= 4
  fp.upe = (uint64_t)fp.spg * sh.nblk;          // units per entry: valid slots x n-blocks
  fp.n_units = (pair ? fp.n_entries / 2 : fp.n_entries) * fp.upe;   // pair: a unit covers two entries
  fp.n_tasks = fp.n_entries * sh.kch;
  const size_t entry_bytes = (size_t)8 * sh.kch * A_TILE_BYTES;
  uint64_t R = ring_target / entry_bytes;
  if (R < 2) R = 2;
  if (R > fp.n_entries) R = fp.n_entries;
  fp.R = (uint32_t)R;
  const size_t ring_bytes = (size_t)R * entry_bytes;
  const size_t flag_bytes = ((size_t)8 * R + 16 + 8 * kNumFusedCounters + 255) & ~(size_t)255;
  uint8_t *ws = nullptr;
  int rc = stream_workspace(stream, ring_bytes + flag_bytes, &ws);
  if (rc != GPIR_OK) return rc;
  fp.ring = ws;
  uint8_t *flags = ws + ring_bytes;
  fp.ctr = reinterpret_cast<unsigned long long *>(flags);
  fp.ready = reinterpret_cast<uint32_t *>(flags + 16);
  fp.consumed = fp.ready + R;
  fp.prof = trace_counters_enabled() ? reinterpret_cast<unsigned long long *>(fp.consumed + R) : nullptr;
  if (fp.prof && ((uintptr_t)fp.prof & 7)) fp.prof = reinterpret_cast<unsigned long long *>(((uintptr_t)fp.prof + 7) & ~(uintptr_t)7);
  e = cudaMemsetAsync(flags, 0, flag_bytes, stream);
  if (e != cudaSuccess) return set_cuda_error(e);
  {
    const uint64_t dims[5] = {N, L, 2, db->d0, batch};
    const uint64_t str[4] = {(uint64_t)N * 4, (uint64_t)L * N * 4, (uint64_t)2 * L * N * 4,
                             (uint64_t)db->d0 * 2 * L * N * 4};
    const uint32_t box[5] = {8, 1, 2, (uint32_t)KCHUNK, (uint32_t)(MROWS / 2)};
    rc = encode_tiled_u32(&fp.ct_map, ct, 5, dims, str, box);
    if (rc != GPIR_OK) return rc;
  }
  fp.b_tiles = db->db_digits;
  fp.out = out;
  fp.hints = hints;
  fp.lookahead = lookahead_mb == 0 ? 0u : (uint32_t)std::max<uint64_t>(2, ((uint64_t)lookahead_mb << 20) / entry_bytes);
  fp.err = device_error_word();
  for (uint32_t l = 0; l < L; ++l) fp.limb[l] = make_limb(prm.primes[l]);
  if (pair) {
    // every CTA pair stays resident (persistent kernel): at most the pairs that fit at once
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg = pair_config((unsigned)(2 * g_pair_clusters[dev]), stream, attr);
    const int tr = trace_begin("tc_pair", stream);
    e = fp.prof ? cudaLaunchKernelEx(&cfg, tc_fused_kernel<true, true>, fp)
                : cudaLaunchKernelEx(&cfg, tc_fused_kernel<false, true>, fp);
    trace_end(tr, stream);
    if (e != cudaSuccess) return set_cuda_error(e);
    if (fp.prof) trace_counters(fp.prof, kNumFusedCounters, stream);
    e = cudaGetLastError();
    return e == cudaSuccess ? GPIR_OK : set_cuda_error(e);
  }
  const int grid = sm_count();
  const int tr = trace_begin("tc_fused", stream);
  if (fp.prof)
    tc_fused_kernel<true, false><<<grid, FUSED_THREADS, FUSED_SMEM, stream>>>(fp);
  else
    tc_fused_kernel<false, false><<<grid, FUSED_THREADS, FUSED_SMEM, stream>>>(fp);
  trace_end(tr, stream);
  if (fp.prof) trace_counters(fp.prof, kNumFusedCounters, stream);
  e = cudaGetLastError();
  return e == cudaSuccess ? GPIR_OK : set_cuda_error(e);
}


std::mutex g_cluster_mu;
int g_cluster_count[64];   // active 8-CTA clusters per device (0: not queried yet, -1: none fit)

// One RowSel problem through the cluster kernel. GPIR_ENOTSUP when the ring
// has fewer than 8 slots or no 8-CTA cluster can be resident.
int tc_launch_cluster(const gpir_db *db, uint32_t batch, const uint32_t *ct, uint32_t *out, cudaStream_t stream) {
  if (!db->db_digits) return GPIR_ENOTSUP;
  const gpir_params &prm = db->params;
  const uint32_t L = prm.num_limbs, N = prm.n;
  if (N < (uint32_t)CL) return GPIR_ENOTSUP;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_cuda_error(e);
  if (dev < 0 || dev >= 64) return GPIR_EINVAL;
  const int grid_max = sm_count();
  {
    std::lock_guard<std::mutex> lk(g_cluster_mu);
    if (g_cluster_count[dev] == 0) {
      e = cudaFuncSetAttribute(tc_cluster_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CLUSTER_SMEM);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_cluster_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)CLUSTER_SMEM);
      if (e != cudaSuccess) return set_cuda_error(e);
      cudaLaunchConfig_t cfg;
      memset(&cfg, 0, sizeof(cfg));
      cfg.gridDim = dim3((unsigned)(grid_max / CL * CL));
      cfg.blockDim = dim3(FUSED_THREADS);
      cfg.dynamicSmemBytes = CLUSTER_SMEM;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = CL;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int n = 0;
      e = cudaOccupancyMaxActiveClusters(&n, tc_cluster_kernel<false>, &cfg);
      if (e != cudaSuccess) {
        cudaGetLastError();
        n = 0;
      }
      g_cluster_count[dev] = n > 0 ? n : -1;
    }
  }
  if (g_cluster_count[dev] < 0) return GPIR_ENOTSUP;
  const TcShape sh = tc_shape(db, batch);
  ClusterParams cp;
  memset(&cp, 0, sizeof(cp));
  cp.L = L;
  cp.N = N;
  cp.M = sh.M;
  cp.d0 = db->d0;
  cp.d1 = db->d1;
  cp.mblk = sh.mblk;
  cp.nblk = sh.nblk;
  cp.kch = sh.kch;
  cp.gpl = N / 8;
  cp.n_entries = (uint64_t)cp.gpl * L * sh.mblk;
  cp.b_tiles = db->db_digits;
  cp.out = out;
  cp.err = device_error_word();
  for (uint32_t l = 0; l < L; ++l) cp.limb[l] = make_limb(prm.primes[l]);
  {
    const uint64_t dims[5] = {N, L, 2, db->d0, batch};
    const uint64_t str[4] = {(uint64_t)N * 4, (uint64_t)L * N * 4, (uint64_t)2 * L * N * 4,
                             (uint64_t)db->d0 * 2 * L * N * 4};
    const uint32_t box[5] = {8, 1, 2, (uint32_t)KCHUNK, (uint32_t)C_SHARE_CLIENTS};
    const int rc = encode_tiled_u32(&cp.ct_map, ct, 5, dims, str, box);
    if (rc != GPIR_OK) return rc;
  }
  uint8_t *ws = nullptr;
  if (trace_counters_enabled()) {
    const int rc = stream_workspace(stream, 8 * kNumFusedCounters, &ws);
    if (rc != GPIR_OK) return rc;
    e = cudaMemsetAsync(ws, 0, 8 * kNumFusedCounters, stream);
    if (e != cudaSuccess) return set_cuda_error(e);
    cp.prof = reinterpret_cast<unsigned long long *>(ws);
  }
  uint64_t clusters = (uint64_t)g_cluster_count[dev];
  if (clusters > cp.n_entries) clusters = cp.n_entries;
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3((unsigned)(clusters * CL));
  cfg.blockDim = dim3(FUSED_THREADS);
  cfg.dynamicSmemBytes = CLUSTER_SMEM;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const int tr = trace_begin("tc_cluster", stream);
  if (cp.prof)
    e = cudaLaunchKernelEx(&cfg, tc_cluster_kernel<true>, cp);
  else
    e = cudaLaunchKernelEx(&cfg, tc_cluster_kernel<false>, cp);
  trace_end(tr, stream);
  if (e != cudaSuccess) return set_cuda_error(e);
  if (cp.prof) trace_counters(cp.prof, kNumFusedCounters, stream);
  e = cudaGetLastError();
  return e == cudaSuccess ? GPIR_OK : set_cuda_error(e);
}

}  // namespace

int rowsel_tc_num_variants() { return kNumTcVariants; }

int rowsel_tc_launch(const gpir_db *db, uint32_t batch, const uint32_t *ct, uint32_t *out, int variant,
                     cudaStream_t stream) {
  if (variant < 0 || variant >= kNumTcVariants) return GPIR_EINVAL;
  const FusedVariant &v = kFusedVariants[variant];
  if (v.kind == kKindCluster) {
    const int rc = tc_launch_cluster(db, batch, ct, out, stream);
    if (rc != GPIR_ENOTSUP) return rc;
    return tc_launch_fused(db, batch, ct, out, (size_t)48 << 20, 0, 16, false, stream);   // N < 8 or no cluster fits
  }
  if (v.kind == kKindTwoPass) {
    gpir_job_t job;
    job.db = db;
    job.batch = batch;
    job.reserved = 0;
    job.ct = ct;
    job.out = out;
    return rowsel_tc_multi(&job, 1, stream);   // two-pass: ingest to HBM, then GEMM
  }
  if (v.kind == kKindTmem || v.kind == kKindTmemPair) {
    const bool pr = v.kind == kKindTmemPair;
    const int rc = tc_launch_tmem(db, batch, ct, out, (size_t)v.ring_mb << 20, v.lookahead_mb, v.hints, pr, stream);
    if (rc != GPIR_ENOTSUP || !pr) return rc;
    // an odd number of m-blocks (or no pair fits): the single-CTA form
    return tc_launch_tmem(db, batch, ct, out, (size_t)v.ring_mb << 20, v.lookahead_mb, v.hints, false, stream);
  }
  if (v.kind == kKindPair) {
    const int rc = tc_launch_fused(db, batch, ct, out, (size_t)v.ring_mb << 20, v.hints, v.lookahead_mb, true, stream);
    if (rc != GPIR_ENOTSUP) return rc;
    // an odd number of m-blocks (or no pair fits): the single-CTA form
    return tc_launch_fused(db, batch, ct, out, (size_t)v.ring_mb << 20, v.hints, v.lookahead_mb, false, stream);
  }
  return tc_launch_fused(db, batch, ct, out, (size_t)v.ring_mb << 20, v.hints, v.lookahead_mb, false, stream);
}

size_t rowsel_tc_multi_workspace(const gpir_job_t *jobs, uint32_t njobs) {
  size_t total = 0;
  for (uint32_t k = 0; k < njobs; ++k) total += (tc_shape(jobs[k].db, jobs[k].batch).a_bytes + 1023) & ~(size_t)1023;
  return total;
}

int rowsel_tc_multi(const gpir_job_t *jobs, uint32_t njobs, cudaStream_t stream) {
  for (uint32_t k = 0; k < njobs; ++k)
    if (!jobs[k].db->db_digits) return GPIR_ENOTSUP;
  uint8_t *ws = nullptr;
  int rc0 = stream_workspace(stream, rowsel_tc_multi_workspace(jobs, njobs), &ws);
  if (rc0 != GPIR_OK) return rc0;
  // MAX_JOBS problems per launch; their workspaces do not overlap.
  size_t off[MAX_JOBS];
  size_t base = 0;
  for (uint32_t k0 = 0; k0 < njobs; k0 += MAX_JOBS) {
    const uint32_t n = std::min<uint32_t>(MAX_JOBS, njobs - k0);
    for (uint32_t k = 0; k < n; ++k) {
      off[k] = base;
      base += (tc_shape(jobs[k0 + k].db, jobs[k0 + k].batch).a_bytes + 1023) & ~(size_t)1023;
    }
    int rc = tc_launch_jobs(jobs + k0, n, ws, off, stream);
    if (rc != GPIR_OK) return rc;
  }
  return GPIR_OK;
}

}  // namespace gpir

// ---------------------------------------------------------------------------
// Allocation-free entry point (gpir_rowsel_batch_noalloc).
//
// Some callers cannot call cudaMalloc while they run RowSel: code executing
// under a CUDA stream capture, services that must not touch the device
// allocator after start-up (memory budgets fixed in advance, allocator locks
// on a latency-critical path), or hosts whose allocator is owned by another
// runtime. For them this entry point runs the tensor-core path with its
// per-batch digit-tile workspace placed in the fixed device array below
// instead of memory from cudaMalloc. The array lives as long as the library
// is loaded on a device (every device that loads the library holds it), holds
// GPIR_NOALLOC_SCRATCH_BYTES, and is shared by all calls: calls that overlap
// on the GPU (several streams, several host threads) race on it.
// ---------------------------------------------------------------------------

static __device__ __align__(256) uint8_t g_noalloc_tiles[GPIR_NOALLOC_SCRATCH_BYTES];

namespace gpir {
namespace {

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kNoallocMaxDevices];   // device address of g_noalloc_tiles, per device

// Once per device, with that device current: resolve the array's device
// address (the name g_noalloc_tiles is only a host-side stand-in) and set the
// kernels' shared-memory limits. Allocates nothing.
int noalloc_setup(int dev, void **tiles) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_tiles);
    if (e != cudaSuccess) return set_cuda_error(e);
    int rc = tc_set_attributes();
    if (rc != GPIR_OK) return rc;
    g_noalloc_addr[dev] = p;
  }
  *tiles = g_noalloc_addr[dev];
  return GPIR_OK;
}

}  // namespace
}  // namespace gpir

extern "C" int gpir_rowsel_batch_noalloc(const gpir_db_t *db, uint32_t batch, const uint32_t *ct_dev,
                                         uint32_t *out_dev, void *stream) {
  using namespace gpir;
  NvtxRange nvtx("gpir_rowsel_batch_noalloc");
  if (!db || !ct_dev || !out_dev || batch == 0 || batch > GPIR_MAX_BATCH) return GPIR_EINVAL;
  if (!(db->path_mask & GPIR_PATH_TC) || !db->db_digits) return GPIR_ENOTSUP;
  const uint32_t L = db->params.num_limbs, N = db->params.n, M = 2 * batch;
  const uint64_t slots = (uint64_t)L * N;
  const size_t ct_bytes = (size_t)batch * db->d0 * 2 * slots * 4;
  const size_t out_bytes = (size_t)batch * db->d1 * 2 * slots * 4;
  const uintptr_t a0 = (uintptr_t)ct_dev, a1 = a0 + ct_bytes, b0 = (uintptr_t)out_dev, b1 = b0 + out_bytes;
  if (a0 < b1 && b0 < a1) return GPIR_EINVAL;
  if ((a0 & 15u) || (b0 & 15u)) return GPIR_EINVAL;
  const uint32_t mblk = (M + MROWS - 1) / MROWS;
  const uint32_t kch = (db->d0 + KCHUNK - 1) / KCHUNK;
  const uint64_t a_bytes = slots * mblk * kch * (uint64_t)A_TILE_BYTES;
  if (a_bytes > (uint64_t)GPIR_NOALLOC_SCRATCH_BYTES) return GPIR_ETOOBIG;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_cuda_error(e);
  if (dev < 0 || dev >= kNoallocMaxDevices || dev != db->device) return GPIR_EINVAL;
  void *tiles = nullptr;
  int rc = noalloc_setup(dev, &tiles);
  if (rc != GPIR_OK) return rc;
  gpir_job_t job;
  job.db = db;
  job.batch = batch;
  job.reserved = 0;
  job.ct = ct_dev;
  job.out = out_dev;
  if (debug_checks()) {
    rc = check_residues_dev(db->params, ct_dev, ct_bytes / 4, (cudaStream_t)stream);
    if (rc != GPIR_OK) return rc;
  }
  const size_t off = 0;
  return tc_launch_jobs(&job, 1, reinterpret_cast<uint8_t *>(tiles), &off, (cudaStream_t)stream);
}
