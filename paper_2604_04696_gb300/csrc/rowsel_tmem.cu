// RowSel on the tensor cores with the A operand in tensor memory and 12 digit
// products per modular MAC (the tensor-memory kernel: tile variants 8-11, and
// the multi-job form of several RowSel problems in one launch).
//
// What is computed: the per-point modular GEMM of Sec. 2.3 / Sec. 5.1 of the
// GPIR paper, out[p][m][n] = sum_k ct[p][m][k] * db[p][k][n] mod q, with
// p = (limb, slot), m = (client, polynomial), k = DB row, n = DB column.
//
// Exactness. Both operands are centred first (x -> x - q when x > (q-1)/2):
// congruent mod q, magnitude below 2^27.
//   - Ciphertext residues become four digits of 7 bits, d_u = field_u - 64 in
//     [-64, 64], fields of y = x~ + O_A with O_A = 64 (1 + 2^7 + 2^14 + 2^21)
//     (fields 0..2 are 7 bits, field 3 = y >> 21 <= 128).
//   - Database residues become three digits, e_0, e_1 in [-512, 511] and
//     e_2 in [-128, 128], of Y = v~ + O_B, O_B = 512 (1 + 2^10) (base 2^10,
//     the top one by arithmetic shift).
//   - A digit product has |d e| <= 2^15: a group of 512 rows sums to at most
//     2^24 and every partial sum is an integer fp32 holds exactly. The tensor
//     core computes the 12 group sums D_uv exactly, and
//         out = sum_groups sum_{u,v} D_uv * (2^(7u + 10v) mod q)   (mod q)
//     in 64-bit integers: < 2^55.6 per group, four groups (< 2^57.6) plus
//     off58 (a multiple of q, >= 2^58) before one Barrett reduction.
// Compared with the four-digit form of rowsel_tc.cu (16 products of base-256
// digits), the tensor work and the database digit bytes drop by a quarter.
//
// Data movement. The database is packed once, at upload, into per-slot digit
// tiles in the shared-memory image the MMA reads: [slot][n-block][k-chunk] x
// (192 rows x 64 k) fp16, K-major, 128-byte swizzle, rows v*64 + n (24 KB).
// Per batch, in one persistent launch (one CTA per SM, or per SM pair):
//   - ingest warps TMA-load raw p-major boxes (8 slots x 64 k x the rows of
//     one m-block), encode every residue once into its 4 digit fields (one
//     byte each), transpose them into digit planes and store slot-major 8 KB
//     tiles [32 rows][64 k] into a ring in global memory (4 bytes per
//     residue, half the digit bytes), counted in ready[E % R];
//   - the producer bulk-copies, per k-chunk of a unit, the ring tile (8 KB)
//     and the database tile (24 KB, or its 12 KB half in the SM-pair form) into
//     a shared-memory stage;
//   - converter warps read their digit's plane of the ring tile (a quarter
//     of the row), turn it into fp16 digits in registers (one PRMT and one
//     HADD2 per pair of digits) and store them straight into a tensor-memory
//     A buffer (tcgen05.st): no digit tile in shared memory, and the MMA reads
//     only B from shared memory;
//   - one thread issues tcgen05.mma .kind::f16 with A in tensor memory
//     (M = 128 or 256, N = 192, K = 16);
//   - epilogue warps drain the double-buffered accumulators and a store warp
//     writes the p-major output.
// Tensor memory (512 columns): accumulators at [0, 192) and [192, 384), and
// 128 columns of A buffers at 384: four buffers of one k-chunk (64 k of fp16
// pairs, 32 columns) or two of two consecutive k-chunks (64 columns, one
// k-chunk from each converter set), per form. The MMA thread waits for a
// buffer once and issues its MMAs back to back.
#include <cuda.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "tcgen05.cuh"

namespace gpir {
namespace {

constexpr int T_KCHUNK = 64;                         // k per stage
constexpr int T_MROWS = 32;                          // ciphertext rows per tile (x 4 digits = 128 lanes)
constexpr int T_NCOLS = 64;                          // DB columns per tile (x 3 digits = 192)
constexpr int T_NDIG = 3 * T_NCOLS;                  // MMA N
constexpr int T_KGROUP = 8;                          // k-chunks per exact group: 512 rows
constexpr int T_FLUSH = 4;                           // groups summed before one reduction
constexpr int T_RAW_TILE = T_MROWS * T_KCHUNK * 4;   // 8 KB ring tile
constexpr int T_B_TILE = T_NDIG * T_KCHUNK * 2;      // 24 KB
constexpr int T_ABUF_MAX = 4;                        // A buffer barriers reserved
constexpr uint32_t T_ACC_COLS = T_NDIG;
constexpr uint32_t T_A_COL0 = 2 * T_ACC_COLS;        // 384
constexpr uint32_t T_TMEM_COLS = 512;
constexpr uint32_t kOffA = 64u * (1u + (1u << 7) + (1u << 14) + (1u << 21));
constexpr int32_t kOffB = 512 * (1 + (1 << 10));

// Warp roles (896 threads). Tensor-memory lane quarter of a warp = warp % 4.
constexpr int W_PROD = 0, W_MMA = 1, W_STORE = 2;
constexpr int W_RELAY = 3;                           // SM pair: hands finished groups to the odd CTA
constexpr int W_CONV0 = 4, N_CONV = 8;               // two converter sets of 4 warps (quarters 0..3),
                                                     // set s converts stages s and s + 2
constexpr int W_EPI0 = 12, N_EPI = 8;                // 8 epilogue warps: quarter, column half
constexpr int W_ING0 = 20, N_ING = 8;                // 8 ingest warps
constexpr int T_THREADS = 32 * (W_ING0 + N_ING);     // 896
static_assert(W_CONV0 % 4 == 0 && W_EPI0 % 4 == 0, "tensor-memory roles start on a lane quarter 0 warp");
constexpr int T_TASK_CLIENTS = T_MROWS / 2;         // clients of one ingest task (one m-block)
constexpr int T_OUT_BYTES = T_MROWS * T_NCOLS * 4;   // 8 KB

// Shared memory holds NS B stages (this CTA's part of a database tile) and RS
// ring slots (a ring tile each), filled and released separately: k-chunk i of
// a CTA uses B stage i % NS (freed by the commit of its MMAs), ring slot i % RS
// (freed by its converters as soon as they have read it) and part i % KPB of
// tensor-memory A buffer (i / KPB) % NBUF. The ingest loads its task's 64 KB of
// raw residues as 16 / BOX_CLIENTS boxes into one box buffer, so a smaller box
// leaves room for more stages.
template <bool PAIR>
struct TmemCfg {
  static constexpr int B_BYTES = PAIR ? T_B_TILE / 2 : T_B_TILE;   // this CTA's part of B
  static constexpr int KPB = PAIR ? 2 : 1;                          // k-chunks per A buffer
  static constexpr int NBUF = 4 / KPB;                              // A buffers (128 columns)
  static constexpr int BOX_CLIENTS = 8;                             // clients per ingest box (two buffers)
  static constexpr int RAW_BOX = BOX_CLIENTS * T_KCHUNK * 2 * 8 * 4;   // x 64 k x 2 x 8 slots x 4 B
  static constexpr int NS = PAIR ? 8 : 5;                           // B stages
  static constexpr int RS = PAIR ? 6 : 4;                           // ring slots
  static constexpr size_t SMEM =
      1024 + (size_t)NS * B_BYTES + (size_t)RS * T_RAW_TILE + 2 * (size_t)RAW_BOX + T_OUT_BYTES + 1024;
  static_assert(KPB == 1 || KPB == 2, "an A buffer holds one k-chunk or one of each converter set");
  static_assert(T_TASK_CLIENTS % BOX_CLIENTS == 0 && BOX_CLIENTS % 4 == 0, "whole boxes per ingest task");
  // A converter set waits on the ring slots of k-chunks i, i + 2, ...: the
  // slot's previous k-chunk i - RS must be one the same set has already waited
  // for (RS even), else a parity wait could pass on the phase before it. For
  // the B stage of k-chunk i it first waits for its A buffer's previous use,
  // whose MMAs (k-chunk i - 4 and earlier) follow the landing of B stage use
  // i - NS when NS >= 4: any such count is safe.
  static_assert(RS % 2 == 0, "two converter sets need an even number of ring slots");
  static_assert(NS >= NBUF * KPB, "a B stage's previous use must precede the A buffer's");
};
static_assert(TmemCfg<false>::SMEM <= 232448, "tensor-memory kernel shared memory exceeds 227 KB");
static_assert(TmemCfg<true>::SMEM <= 232448, "tensor-memory kernel shared memory exceeds 227 KB");

struct TmLimb {
  uint32_t q, h;         // prime, (q - 1) / 2
  uint64_t mu;           // floor(2^64 / q)
  uint64_t off58;        // multiple of q, >= 2^58
  int32_t w[4][3];       // 2^(7u + 10v) mod q
};

// Division of a 32-bit index by a launch constant d >= 1 (Granlund and
// Montgomery, "Division by invariant integers using multiplication", 1994):
// with l = ceil(log2 d) and the 33-bit multiplier 2^32 + m,
// m = floor(2^32 (2^l - d) / d) + 1, n / d = (umulhi(n, m) + n) >> l for
// every n < 2^32. Written on the host by tm_div.
struct TmDiv {
  uint32_t d, m, l;
  __device__ __forceinline__ uint32_t div(uint32_t n) const {
    return (uint32_t)(((uint64_t)__umulhi(n, m) + n) >> l);
  }
  __device__ __forceinline__ uint32_t mod(uint32_t n) const { return n - div(n) * d; }
};

// One RowSel problem of a launch. Its entries, units and ingest tasks are
// numbered after those of the jobs before it, in one index space per launch.
constexpr int T_MAX_JOBS = 8;
struct TmJob {
  CUtensorMap ct_map;                   // box (8 slots, 1, 2, 64 k, BOX_CLIENTS clients)
  uint32_t M, d1, mblk, nblk, kch, upe;
  TmDiv mblk_d, nblk_d, kch_d, upe_d;   // the same four as divisors
  uint64_t entry0, unit0, task0;        // first entry / unit / ingest task of the job
  const uint16_t *b_tiles;              // [slot][nblk][kch] x 24 KB
  uint32_t *out;
};

struct TmemParams {
  TmJob job[T_MAX_JOBS];
  uint32_t L, N, njobs, kch_max;
  uint32_t R, gpl, spg, lookahead;
  TmDiv R_d, gpl_d;
  uint32_t hints;                       // 1: raw boxes evict-first, ring stores evict-last in L2
  uint64_t n_entries, n_units, n_tasks; // over all jobs
  uint8_t *ring;                        // [R][8 slots][kch_max] x 8 KB
  uint32_t *ready, *consumed;           // [n_entries] each: tasks ingested, units that read the entry
  unsigned long long *ctr;              // [0] next unit, [1] next ingest task
  unsigned int *err;
  unsigned long long *prof;             // wait-cycle counters (traced instantiation only)
  TmLimb limb[GPIR_MAX_LIMBS];
};

// Job of a global unit / entry / ingest task (jobs in index order, at most
// 8); job 0 at compile time in the single-job instantiations.
template <bool MULTI>
__device__ __forceinline__ uint32_t job_of_unit(const TmemParams &p, uint64_t u) {
  uint32_t j = 0;
  if constexpr (MULTI)
    while (j + 1 < p.njobs && u >= p.job[j + 1].unit0) ++j;
  return j;
}
template <bool MULTI>
__device__ __forceinline__ uint32_t job_of_entry(const TmemParams &p, uint64_t e) {
  uint32_t j = 0;
  if constexpr (MULTI)
    while (j + 1 < p.njobs && e >= p.job[j + 1].entry0) ++j;
  return j;
}
template <bool MULTI>
__device__ __forceinline__ uint32_t job_of_task(const TmemParams &p, uint64_t t) {
  uint32_t j = 0;
  if constexpr (MULTI)
    while (j + 1 < p.njobs && t >= p.job[j + 1].task0) ++j;
  return j;
}


// Wait / busy cycle counters of the traced instantiation (SM clock cycles
// summed over CTAs, one counting thread per role), read through
// gpir_trace_counters.
enum TmemCounter {
  kTPWaitReady = 0,   // producer: ring entry not yet ingested
  kTPWaitEmpty,       // producer: no free stage
  kTCWaitFull,        // converter: stage not landed
  kTCBusy,            // converter: shared-memory loads and digit conversion
  kTCStore,           // converter: tensor-memory store, its wait and the signal
  kTMWaitA,           // MMA: A buffer not converted
  kTMWaitAcc,         // MMA: accumulator not drained
  kTMIssue,           // MMA: issuing a k-chunk's MMAs and commits
  kTMHandoff,         // MMA: handing a finished group to the epilogues (tag, commit, arrives)
  kTEWaitAcc,         // epilogue: MMAs of the group not done
  kTEBusy,            // epilogue: draining and reducing
  kTIWaitSlot,        // ingest: ring entry not released, or lookahead
  kTIWaitBox,         // ingest: TMA box in flight
  kTIBusy,            // ingest: encoding and ring stores
  kTIFence,           // ingest: fence and ready count
  kTCta,              // kernel cycles per CTA
  kNumTmemCounters
};

constexpr uint64_t kNoUnit = ~0ull;

// kind::f16, D = f32, A = B = f16, K-major, N = 192, M = 128 (one CTA) or 256 (pair).
constexpr uint32_t kIdescT1 = (1u << 4) | ((uint32_t)(T_NDIG >> 3) << 17) | ((128u >> 4) << 24);
constexpr uint32_t kIdescT2 = (1u << 4) | ((uint32_t)(T_NDIG >> 3) << 17) | ((256u >> 4) << 24);

// D[tmem_d] (+)= A[tmem_a] * B[bdesc]: A read from tensor memory (lane = row,
// column j = k pair 2j, 2j+1), B from shared memory.
__device__ __forceinline__ void mma_tmem_a(uint32_t tmem_d, uint32_t tmem_a, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}" ::"r"(tmem_d),
      "r"(tmem_a), "l"(bdesc), "r"(kIdescT1), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_tmem_a_pair(uint32_t tmem_d, uint32_t tmem_a, uint64_t bdesc,
                                                uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::2.kind::f16 [%0], [%1], %2, %3, p;\n}" ::"r"(tmem_d),
      "r"(tmem_a), "l"(bdesc), "r"(kIdescT2), "r"(accumulate)
      : "memory");
}

// 32 consecutive tensor-memory columns of this warp's lane quarter <- r[0..31].
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,"
      "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
      "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]),
      "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]),
      "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}

// Three loads of 4 columns each (the three database digits of 4 columns).
__device__ __forceinline__ void tmem_ld4x3(uint32_t t0, uint32_t t1, uint32_t t2, uint32_t (&r)[12]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%12];\n"
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%4,%5,%6,%7}, [%13];\n"
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%8,%9,%10,%11}, [%14];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11])
      : "r"(t0), "r"(t1), "r"(t2));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Ring encoding of a ciphertext residue x < q: the four 7-bit fields of
// y = centred(x) + O_A, one per byte (bit 7 of bytes 0..2 clear, byte 3
// holds y >> 21 <= 128 whole).
__device__ __forceinline__ uint32_t ct_fields(uint32_t x, uint32_t q, uint32_t h) {
  const uint32_t y = x + kOffA - (x > h ? q : 0u);   // < 2^29
  // byte u = field u of y with bit 7 clear (u < 3), byte 3 = y >> 21, by two
  // spreads done as adds: bits 14.. of y up by 2 (a = y + 3 (y & ~0x3FFF)),
  // then bits 7..13 and 21.. of each 16-bit half up by 1
  const uint32_t a = y + 3u * (y & 0xFFFFC000u);
  return a + (a & 0x7F807F80u);
}

// Ring tile row (256 bytes, one ciphertext row of a k-chunk): 16-byte chunk
// c16 = 2 j + h holds, for k octet j, the bytes of digits 2h and 2h + 1 of its
// 8 residues in k order ([digit 2h: 8 bytes][digit 2h + 1: 8 bytes]), stored
// at position c16 ^ (row % 8). Byte u of a ring word z is field u of y
// (bit 7 clear for u < 3), so a digit plane holds the fields as they are.

// Four ring words (k0..k3 in the order the selectors give) -> their four digit
// planes p[u] = (byte u of k0, k1, k2, k3). sa / sb pick bytes 0, 1 / 2, 3 of
// a word pair: 0x5140 / 0x7362 in order, 0x1504 / 0x3726 with the pair
// swapped.
__device__ __forceinline__ void digit_planes(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3, uint32_t sa,
                                             uint32_t sb, uint32_t p[4]) {
  const uint32_t t0 = __byte_perm(w0, w1, sa), t1 = __byte_perm(w0, w1, sb);
  const uint32_t t2 = __byte_perm(w2, w3, sa), t3 = __byte_perm(w2, w3, sb);
  p[0] = __byte_perm(t0, t2, 0x5410);
  p[1] = __byte_perm(t0, t2, 0x7632);
  p[2] = __byte_perm(t1, t3, 0x5410);
  p[3] = __byte_perm(t1, t3, 0x7632);
}

// fp16 pair of the fields in bytes 2s and 2s + 1 of plane word w: each byte
// under 0x6400 (= 1024 + field exactly), then field - 64 by one HADD2.
__device__ __forceinline__ uint32_t plane_pair(uint32_t w, uint32_t sel) {
  const uint32_t t = __byte_perm(w, 0x64646464u, sel);   // 0x5140: bytes 0, 1; 0x5342: bytes 2, 3
  const __half2 h = __hadd2(*reinterpret_cast<const __half2 *>(&t),
                            __half2half2(__ushort_as_half((unsigned short)0xE440)));   // -1088
  return *reinterpret_cast<const uint32_t *>(&h);
}

// fp16 bit pattern of database digit v (0..2) of a residue below q.
__device__ __forceinline__ uint16_t db_digit_bits(uint32_t x, uint32_t q, int v) {
  const int32_t xt = (int32_t)x - (x > (q - 1) / 2 ? (int32_t)q : 0);
  const int32_t Y = xt + kOffB;
  const int32_t e = v == 0 ? (Y & 1023) - 512 : v == 1 ? ((Y >> 10) & 1023) - 512 : (Y >> 20);
  return __half_as_ushort(__int2half_rn(e));   // |e| <= 512: exact
}

// ---- database packing (once per upload) -------------------------------------

struct Pack12Params {
  uint32_t d0, d1, L, N, nblk, kch;
  const uint32_t *db;
  uint4 *b_tiles;
  uint32_t q[GPIR_MAX_LIMBS];
};

// One thread per (slot, n-block, k-chunk, digit row, k octet); slots fastest so
// the reads of the p-major database are coalesced. Row r = v * 64 + n of the
// 192-row tile, 16-byte chunk (k octet) j stored at j ^ (r % 8): the 128-byte
// swizzle of the MMA's shared-memory operand.
__global__ void tm_pack_db_kernel(const Pack12Params p, uint64_t total) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t x = i;
    const uint32_t slot = (uint32_t)(x % ((uint64_t)p.L * p.N));
    x /= (uint64_t)p.L * p.N;
    const uint32_t k_oct = (uint32_t)(x % 8);
    x /= 8;
    const uint32_t row = (uint32_t)(x % T_NDIG);
    x /= T_NDIG;
    const uint32_t kc = (uint32_t)(x % p.kch);
    const uint32_t nb = (uint32_t)(x / p.kch);
    const uint32_t v = row / T_NCOLS, n = nb * T_NCOLS + row % T_NCOLS;
    const uint32_t l = slot / p.N, t = slot % p.N;
    uint32_t bits[8];
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      const uint32_t k = kc * T_KCHUNK + k_oct * 8 + kk;
      bits[kk] = (n < p.d1 && k < p.d0)
                     ? db_digit_bits(p.db[(((uint64_t)k * p.d1 + n) * p.L + l) * p.N + t], p.q[l], (int)v)
                     : 0u;   // padding: digit 0
    }
    uint4 w;
    w.x = bits[0] | (bits[1] << 16);
    w.y = bits[2] | (bits[3] << 16);
    w.z = bits[4] | (bits[5] << 16);
    w.w = bits[6] | (bits[7] << 16);
    p.b_tiles[(((uint64_t)slot * p.nblk + nb) * p.kch + kc) * (T_B_TILE / 16) + row * 8 + (k_oct ^ (row & 7))] = w;
  }
}

// ---- the persistent kernel -------------------------------------------------
//
// Work: entries E = (8-slot group g, 32-row m-block), units (E, slot, n-block)
// of kch k-chunks, ingest tasks (E, k-chunk), numbered job after job (MULTI:
// several jobs, each with its own shape, database tiles, output and tensor
// map; one parameter set). Claiming, ring flow control and the deadlock
// argument are those of the fused kernel in rowsel_tc.cu (both sides claim in
// increasing order; an ingest task waits only for the entry R back in the
// ring and for claims already made), with one ready and one consumed counter
// per entry (entries of different jobs need different counts); ring entries
// are strided by the largest job's k-chunk count. The ring holds encoded raw
// residues and an entry is released as soon as its units' last k-chunks have
// landed in shared memory. SM-pair form (PAIR, one job): a pair unit covers
// entries 2 E2 (even CTA) and 2 E2 + 1 (odd CTA) against one database tile;
// each CTA copies its own ring tile and its half of B and converts its own A
// into its own tensor memory; the even CTA's MMA thread issues M = 256 MMAs
// once both CTAs' A buffers are ready; commits go to both CTAs.
template <bool PROF, bool PAIR, bool MULTI>
__global__ void __launch_bounds__(T_THREADS, 1) tc_tmem_kernel(const __grid_constant__ TmemParams p) {
  using Cfg = TmemCfg<PAIR>;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  // B stage st at smem + st * B_BYTES (1024-aligned), then the ring slots
  constexpr int NS = Cfg::NS, RS = Cfg::RS;
  uint8_t *rslots = smem + NS * Cfg::B_BYTES;
  uint8_t *rawbox = rslots + RS * T_RAW_TILE;
  uint32_t *out_stage = reinterpret_cast<uint32_t *>(rawbox + 2 * Cfg::RAW_BOX);
  uint64_t *full = reinterpret_cast<uint64_t *>(rawbox + 2 * Cfg::RAW_BOX + T_OUT_BYTES);   // [NS] B part landed
  uint64_t *empty = full + NS;                    // [NS] B part read by its MMAs
  uint64_t *rfull = empty + NS;                   // [RS] ring tile landed
  uint64_t *rempty = rfull + RS;                  // [RS] ring tile read by its converters
  uint64_t *afull = rempty + RS;                  // [NBUF] A buffer converted (pair: both CTAs')
  uint64_t *aempty = afull + T_ABUF_MAX;          // [NBUF] A buffer read by its MMAs
  uint64_t *acc_full = aempty + T_ABUF_MAX;
  uint64_t *acc_empty = acc_full + 2;
  uint64_t *box_bar = acc_empty + 2;             // [2] ingest box buffer landed
  uint64_t *ostage_full = box_bar + 2;
  uint64_t *ostage_empty = ostage_full + 1;
  uint64_t *stage_unit = ostage_empty + 1;        // [NS] unit of the B stage
  uint64_t *slot_unit = stage_unit + NS;          // [RS] unit of the ring slot
  uint64_t *slot_kc = slot_unit + RS;             // [RS] k-chunk of the unit in the ring slot
  uint64_t *acc_unit = slot_kc + RS;              // [2]
  uint64_t *task_slot = acc_unit + 2;
  uint64_t *ostage_unit = task_slot + 1;
  uint64_t *mail = ostage_unit + 1;               // pair: [4] claimed units, even -> odd CTA
  uint64_t *mail_full = mail + 4;
  uint64_t *mail_empty = mail_full + 4;
  uint64_t *hand_full = mail_empty + 4;           // pair (even CTA): [2] group handed to the relay
  uint64_t *task_ok = hand_full + 2;              // ingest: the current task may write its ring entry
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(task_ok + 1);
  volatile uint32_t *abort_flag = tmem_slot + 1;
  // barriers and tags above, in 8-byte words, within the 1 KB reserved for them
  static_assert(8 * (3 * NS + 4 * RS + 2 * T_ABUF_MAX + 4 + 4 + 2 + 2 + 12 + 2 + 1 + 1) <= 1024,
                "tensor-memory kernel barrier area exceeds its reservation");

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = PAIR ? cluster_rank() : 0u;
  if (threadIdx.x == 0) {
    for (int s2 = 0; s2 < NS; ++s2) {
      mbar_init(&full[s2], 1);
      mbar_init(&empty[s2], 1);
    }
    for (int r = 0; r < RS; ++r) {
      mbar_init(&rfull[r], 1);
      mbar_init(&rempty[r], 4);   // the 4 warps of the converter set that read it
    }
    for (int a = 0; a < Cfg::NBUF; ++a) {
      // the 4 warps of each converter set filling the buffer (KPB sets); in
      // the pair, the even CTA counts both CTAs' warps
      mbar_init(&afull[a], 4 * Cfg::KPB * ((PAIR && rank == 0) ? 2 : 1));
      mbar_init(&aempty[a], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 2);
      mbar_init(&acc_empty[b], (PAIR && rank == 0) ? 2 * N_EPI : N_EPI);
    }
    for (int i = 0; i < 4; ++i) {
      mbar_init(&mail_full[i], 1);
      mbar_init(&mail_empty[i], 1);
    }
    for (int b = 0; b < 2; ++b) mbar_init(&hand_full[b], 1);
    mbar_init(&box_bar[0], 1);
    mbar_init(&box_bar[1], 1);
    mbar_init(ostage_full, N_EPI);
    mbar_init(ostage_empty, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == W_MMA) {
    if constexpr (PAIR) {
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                   "r"(T_TMEM_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                   "r"(T_TMEM_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
  }
  tc_fence_before();
  if constexpr (PAIR)
    cluster_sync_all();
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
    const uint64_t t0 = globaltimer_ns();
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
  auto wait_claims = [&](uint64_t target) -> bool {
    auto seen = [&]() {
      unsigned long long v;
      asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(&p.ctr[0]) : "memory");
      return v >= target;
    };
    if (seen()) return true;
    const uint64_t t0 = globaltimer_ns();
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
  auto wait_count = [&](const uint32_t *ctr, uint32_t target) -> bool {
    if (ld_acquire(ctr) >= target) return true;
    const uint64_t t0 = globaltimer_ns();
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
  // entry of a unit for this CTA
  // global entry of a unit for this CTA
  auto entry_of = [&](uint64_t u) -> uint64_t {
    const TmJob &jb = p.job[job_of_unit<MULTI>(p, u)];
    const uint32_t ul = (uint32_t)(u - jb.unit0);
    return jb.entry0 + (PAIR ? (uint64_t)jb.upe_d.div(ul) * 2 + rank : (uint64_t)jb.upe_d.div(ul));
  };
  // index of the first unit that reads entry e
  auto first_unit_of = [&](uint64_t e) -> uint64_t {
    const TmJob &jb = p.job[job_of_entry<MULTI>(p, e)];
    return jb.unit0 + ((e - jb.entry0) >> (PAIR ? 1 : 0)) * jb.upe;
  };
  uint64_t pc[PROF ? kNumTmemCounters : 1];
#pragma unroll
  for (int i = 0; i < (PROF ? kNumTmemCounters : 1); ++i) pc[i] = 0;
  const uint64_t kstart = PROF ? clock64() : 0;
#define TM_TIMED(k, expr)                                 \
  ([&]() {                                                 \
    const uint64_t _t0 = PROF ? clock64() : 0;             \
    const bool _r = (expr);                                \
    if (PROF) pc[PROF ? (k) : 0] += clock64() - _t0;       \
    return _r;                                             \
  }())

  if (warp == W_PROD) {
    // ---------------- producer: claims units, copies ring + B tiles ----------------
    // Claims one unit ahead, so that a claim (a global atomic, and in the pair
    // the mailbox round trip) is off the copy path. Per k-chunk: the ring tile
    // into the next ring slot once its converters have read it, then the B
    // part into the next B stage once its MMAs have run.
    if (lane == 0) {
      uint32_t st = 0, ph = 0, r = 0, rph = 0, mi = 0;
      uint32_t b_issued = 0, b_ph = 0, r_issued = 0, r_ph = 0;   // copies issued, parity of the last one
      bool ok = true;
      auto claim = [&](uint64_t &u) -> bool {
        if constexpr (PAIR) {
          const uint32_t ms = mi & 3u, mph = (mi >> 2) & 1u;
          ++mi;
          if (rank == 0) {
            u = atomicAdd(&p.ctr[0], 1ull);
            if (u >= p.n_units) u = kNoUnit;
            if (!wait(&mail_empty[ms], mph ^ 1u, kErrQueueWait)) return false;
            st_cluster_u64(map_peer(smem_u32(&mail[ms]), 1), u);
            mbar_arrive_remote(map_peer(smem_u32(&mail_full[ms]), 1));
          } else {
            if (!wait(&mail_full[ms], mph, kErrQueueWait)) return false;
            u = *reinterpret_cast<volatile uint64_t *>(&mail[ms]);
            mbar_arrive_remote(map_peer(smem_u32(&mail_empty[ms]), 0));
          }
        } else {
          u = atomicAdd(&p.ctr[0], 1ull);
          if (u >= p.n_units) u = kNoUnit;
        }
        return true;
      };
      auto next_stage = [&]() {
        if (++st == NS) {
          st = 0;
          ph ^= 1u;
        }
      };
      auto next_slot = [&]() {
        if (++r == RS) {
          r = 0;
          rph ^= 1u;
        }
      };
      uint64_t u = kNoUnit, un = kNoUnit;
      ok = claim(u);
      if (ok && u != kNoUnit) ok = claim(un);
      while (ok && u != kNoUnit) {
        const TmJob &jb = p.job[job_of_unit<MULTI>(p, u)];
        const uint64_t E = entry_of(u);
        const uint32_t w = jb.upe_d.mod((uint32_t)(u - jb.unit0)), sl = jb.nblk_d.div(w), nb = w - sl * jb.nblk;
        const uint32_t g = jb.mblk_d.div((uint32_t)(E - jb.entry0));
        const uint32_t gl = p.gpl_d.div(g);
        const uint64_t slot = (uint64_t)gl * p.N + (g - gl * p.gpl) * 8 + sl;
        const uint8_t *src_a = p.ring + (((uint64_t)p.R_d.mod((uint32_t)E) * 8 + sl) * p.kch_max) * (uint64_t)T_RAW_TILE;
        const uint8_t *src_b = (const uint8_t *)jb.b_tiles + ((slot * jb.nblk + nb) * jb.kch) * (uint64_t)T_B_TILE +
                               (PAIR ? rank * (uint64_t)Cfg::B_BYTES : 0ull);
        const uint32_t kch = jb.kch;
        if (!(ok = TM_TIMED(kTPWaitReady, wait_count(&p.ready[E], kch)))) break;
        fence_proxy_async_global();
        for (uint32_t kc = 0; kc < kch; ++kc) {
          if (!(ok = TM_TIMED(kTPWaitEmpty, wait(&rempty[r], rph ^ 1u, kErrTmaWait)))) break;
          slot_unit[r] = u;
          slot_kc[r] = kc;
          mbar_arrive_expect_tx(&rfull[r], T_RAW_TILE);
          bulk_g2s(rslots + r * T_RAW_TILE, src_a + (uint64_t)kc * T_RAW_TILE, T_RAW_TILE, &rfull[r]);
          r_issued |= 1u << r;
          r_ph = (r_ph & ~(1u << r)) | (rph << r);
          next_slot();
          if (!(ok = TM_TIMED(kTPWaitEmpty, wait(&empty[st], ph ^ 1u, kErrTmaWait)))) break;
          stage_unit[st] = u;
          mbar_arrive_expect_tx(&full[st], Cfg::B_BYTES);
          bulk_g2s(smem + st * Cfg::B_BYTES, src_b + (uint64_t)kc * T_B_TILE, Cfg::B_BYTES, &full[st]);
          b_issued |= 1u << st;
          b_ph = (b_ph & ~(1u << st)) | (ph << st);
          next_stage();
        }
        if (!ok) break;
        u = un;
        un = kNoUnit;
        if (u != kNoUnit) ok = claim(un);
      }
      // end of work: a sentinel in the next two k-chunks, one for each
      // converter set; the B stage's tag is written first, so that the ring
      // slot's arrive (a release) publishes it to the MMA thread too
      for (int k = 0; k < 2 && ok; ++k) {
        if (!(ok = wait(&empty[st], ph ^ 1u, kErrTmaWait))) break;
        stage_unit[st] = kNoUnit;
        next_stage();
        if (!(ok = wait(&rempty[r], rph ^ 1u, kErrTmaWait))) break;
        slot_unit[r] = kNoUnit;
        mbar_arrive(&rfull[r]);
        next_slot();
      }
      if (ok) {
        if constexpr (PAIR) {
          // the last multicast commits target this CTA's empty barriers too:
          // let them land on the other stages before the CTA leaves
          for (int s2 = 2; s2 < NS; ++s2) {
            mbar_wait_bounded(&empty[st], ph ^ 1u, nullptr, 0);
            next_stage();
          }
        }
      } else {
        // let this CTA's copies in flight land before it leaves
        for (int s2 = 0; s2 < NS; ++s2)
          if ((b_issued >> s2) & 1u) mbar_wait_bounded(&full[s2], (b_ph >> s2) & 1u, nullptr, 0);
        for (int r2 = 0; r2 < RS; ++r2)
          if ((r_issued >> r2) & 1u) mbar_wait_bounded(&rfull[r2], (r_ph >> r2) & 1u, nullptr, 0);
      }
    }
  } else if (warp >= W_CONV0 && warp < W_CONV0 + N_CONV) {
    // ---------------- converters: ring tile (smem) -> fp16 digits -> tensor memory ----------------
    // Thread = tensor-memory lane (row m_hi*32 + u*8 + m_lo of the A operand):
    // ciphertext row m = m_hi*8 + m_lo of the m-block, digit u. Set cs
    // converts k-chunks i = cs, cs + 2, ... (two sets hide each other's
    // latency) into part i % KPB of A buffer (i / KPB) % NBUF.
    const uint32_t qw = (uint32_t)(warp & 3);
    const uint32_t cs = (uint32_t)(warp - W_CONV0) >> 2;
    const int u = lane >> 3, m_lo = lane & 7;
    const int m = (int)qw * 8 + m_lo;
    const uint32_t lane_base = tmem_base + ((qw * 32u) << 16);
    const bool conv_counter = PROF && warp == W_CONV0 && lane == 0;
    for (uint32_t it = 0;; ++it) {
      const uint32_t i = 2u * it + cs;                      // this CTA's k-chunk sequence number
      const uint32_t st = i % NS, ph = (i / NS) & 1u;
      const uint32_t r = i % RS, rph = (i / RS) & 1u;
      const uint32_t bi = i / Cfg::KPB, ab = bi % Cfg::NBUF, aph = (bi / Cfg::NBUF) & 1u;
      const uint32_t acol = T_A_COL0 + ab * (32u * Cfg::KPB) + (i % Cfg::KPB) * 32u;
      const bool okf = conv_counter ? TM_TIMED(kTCWaitFull, wait(&rfull[r], rph, kErrTmaWait))
                                    : wait(&rfull[r], rph, kErrTmaWait);
      if (!__all_sync(0xffffffffu, okf)) break;
      const uint64_t tconv = PROF ? clock64() : 0;
      const uint64_t un = slot_unit[r];
      if (un == kNoUnit) {
        // Wait for the A buffer's previous k-chunk to be read by its MMAs even
        // here: in the pair form an early sentinel arrival could complete the
        // even CTA's count-8 afull phase of that previous k-chunk without the
        // other CTA's arrivals.
        __all_sync(0xffffffffu, wait(&aempty[ab], aph ^ 1u, kErrMmaWait));
        __syncwarp();
        if (lane == 0) {
          if (PAIR && rank != 0)
            mbar_arrive_remote_relaxed(map_peer(smem_u32(&afull[ab]), 0));
          else
            mbar_arrive(&afull[ab]);
        }
        break;
      }
      // the unit's last ring tile is in shared memory: its ring entry may be reused
      if (qw == 0 && lane == 0 && slot_kc[r] + 1 == p.job[job_of_unit<MULTI>(p, un)].kch)
        atomicAdd(&p.consumed[entry_of(un)], 1u);
      // this thread's digit plane: 8 bytes per k octet (conflict-free: the
      // warp's 32 reads of a step cover every bank twice)
      const uint2 *row = reinterpret_cast<const uint2 *>(rslots + r * T_RAW_TILE) + m * 32;
      uint32_t wv[32];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const uint2 z = row[(((2 * j + (u >> 1)) ^ (m & 7)) << 1) | (u & 1)];
        wv[4 * j] = plane_pair(z.x, 0x5140u);
        wv[4 * j + 1] = plane_pair(z.x, 0x5342u);
        wv[4 * j + 2] = plane_pair(z.y, 0x5140u);
        wv[4 * j + 3] = plane_pair(z.y, 0x5342u);
      }
      // the digits are in registers (every loaded word went into them): the
      // ring slot may be refilled
      __syncwarp();
      if (lane == 0) mbar_arrive(&rempty[r]);
      const uint64_t tst = PROF ? clock64() : 0;
      if (conv_counter) pc[PROF ? kTCBusy : 0] += tst - tconv;
      // the A buffer's previous k-chunk must have been read by its MMAs before
      // the digits overwrite it, and the MMAs of this k-chunk also read the B
      // stage: signal the buffer only once that has landed
      if (!__all_sync(0xffffffffu, wait(&aempty[ab], aph ^ 1u, kErrMmaWait))) break;
      if (!__all_sync(0xffffffffu, wait(&full[st], ph, kErrTmaWait))) break;
      tc_fence_after();
      tmem_st32(lane_base + acol, wv);
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        if (PAIR && rank != 0)
          mbar_arrive_remote_relaxed(map_peer(smem_u32(&afull[ab]), 0));
        else
          mbar_arrive(&afull[ab]);
      }
      if (conv_counter) pc[PROF ? kTCStore : 0] += clock64() - tst;
    }
  } else if (warp == W_MMA) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      // k-chunk i of this CTA sits in part i % KPB of A buffer (i / KPB) %
      // NBUF; the MMA thread waits for a buffer at its first part (all parts
      // are converted by then: the count spans their sets) and commits it
      // after the last
      uint32_t st = 0, ph = 0, buf = 0, i = 0;
      uint32_t aph[2] = {0, 0};
      bool ok = true;
      auto wait_a = [&]() -> bool {
        if (i % Cfg::KPB) return true;
        const uint32_t bi = i / Cfg::KPB;
        return TM_TIMED(kTMWaitA, wait(&afull[bi % Cfg::NBUF], (bi / Cfg::NBUF) & 1u, kErrTmaWait));
      };
      for (;;) {
        if (PAIR && rank != 0) {
          // odd CTA: its converters signal the even CTA directly; nothing to issue
          break;
        }
        if (!(ok = wait_a())) break;
        const uint64_t u = stage_unit[st];
        if (u == kNoUnit) {
          if ((ok = wait(&acc_empty[buf], aph[buf] ^ 1u, kErrMmaWait))) {
            acc_unit[buf] = kNoUnit;
            // pair: the relay tells the odd CTA's epilogue (its own acc_unit)
            if constexpr (PAIR) mbar_arrive(&hand_full[buf]);
            mbar_arrive_cnt(&acc_full[buf], 2);
          }
          break;
        }
        bool first = true;
        const uint32_t kch = p.job[job_of_unit<MULTI>(p, u)].kch;
        const uint32_t kgroups = (kch + T_KGROUP - 1) / T_KGROUP;
        for (uint32_t gi = 0; gi < kgroups && ok; ++gi) {
          if (!(ok = TM_TIMED(kTMWaitAcc, wait(&acc_empty[buf], aph[buf] ^ 1u, kErrMmaWait)))) break;
          tc_fence_after();
          const uint32_t tmem_d = tmem_base + buf * T_ACC_COLS;
          const uint32_t c0 = gi * T_KGROUP;
          const uint32_t c1 = min(kch, c0 + T_KGROUP);
          for (uint32_t kc = c0; kc < c1; ++kc) {
            if (!first && !(ok = wait_a())) break;
            first = false;
            tc_fence_after();
            const uint64_t tiss = PROF ? clock64() : 0;
            const uint32_t sb = smem_u32(smem + st * Cfg::B_BYTES);
            const uint32_t ab = (i / Cfg::KPB) % Cfg::NBUF;
            const bool a_done = i % Cfg::KPB == Cfg::KPB - 1;
            const uint32_t ta = tmem_base + T_A_COL0 + ab * (32u * Cfg::KPB) + (i % Cfg::KPB) * 32u;
#pragma unroll
            for (int k16 = 0; k16 < T_KCHUNK / 16; ++k16) {
              const uint32_t acc = (kc > c0 || k16 > 0) ? 1u : 0u;
              if constexpr (PAIR)
                mma_tmem_a_pair(tmem_d, ta + k16 * 8, sw128_desc(sb + k16 * 32), acc);
              else
                mma_tmem_a(tmem_d, ta + k16 * 8, sw128_desc(sb + k16 * 32), acc);
            }
            if constexpr (PAIR) {
              mma_commit_pair(&empty[st]);
              if (a_done) mma_commit_pair(&aempty[ab]);
            } else {
              mma_commit(&empty[st]);
              if (a_done) mma_commit(&aempty[ab]);
            }
            if (PROF) pc[PROF ? kTMIssue : 0] += clock64() - tiss;
            if (++st == NS) {
              st = 0;
              ph ^= 1u;
            }
            ++i;
          }
          if (!ok) break;
          const uint64_t thand = PROF ? clock64() : 0;
          const uint64_t tag = u | ((gi + 1 == kgroups) ? (1ull << 63) : 0ull);
          acc_unit[buf] = tag;
          if constexpr (PAIR) {
            // the tag reaches the odd CTA through the relay warp: its
            // cluster-scope release arrive can wait for the SM's outstanding
            // ring stores, which must not hold up the next group's MMAs
            mma_commit_pair(&acc_full[buf]);
            mbar_arrive(&hand_full[buf]);
          } else {
            mma_commit(&acc_full[buf]);
          }
          mbar_arrive(&acc_full[buf]);
          if (PROF) pc[PROF ? kTMHandoff : 0] += clock64() - thand;
          aph[buf] ^= 1u;
          buf ^= 1u;
        }
        if (!ok) break;
      }
      if (!ok && !(PAIR && rank != 0))
        for (int b = 0; b < 2; ++b) mbar_wait_bounded(&acc_full[b], aph[b], nullptr, 0);
    }
  } else if (warp >= W_EPI0 && warp < W_EPI0 + N_EPI) {
    // ---------------- epilogue (8 warps) ----------------
    const uint32_t qw = (uint32_t)(warp & 3);
    const uint32_t half = (uint32_t)(warp - W_EPI0) >> 2;   // columns [32 half, 32 half + 32)
    const int u = lane >> 3, m_lo = lane & 7;
    const int m_local = (int)qw * 8 + m_lo;
    const int et = (int)threadIdx.x - 32 * W_EPI0;
    auto epi_all = [&](bool v) -> bool {
      uint32_t r = v ? 1u : 0u;
      asm volatile(
          "{\n .reg .pred pin, pout;\n setp.ne.u32 pin, %1, 0;\n bar.red.and.pred pout, 2, %2, pin;\n"
          " selp.u32 %0, 1, 0, pout;\n}"
          : "=r"(r)
          : "r"(r), "n"(32 * N_EPI)
          : "memory");
      return r != 0;
    };
    uint32_t buf = 0, oph = 0, ngroups = 0;
    uint32_t aph[2] = {0, 0};
    uint32_t res[8];
    int64_t acc64[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      res[i] = 0;
      acc64[i] = 0;
    }
    const bool epi_counter = PROF && et == 0;
    for (;;) {
      const bool oka = epi_counter ? TM_TIMED(kTEWaitAcc, wait(&acc_full[buf], aph[buf], kErrMmaWait))
                                   : wait(&acc_full[buf], aph[buf], kErrMmaWait);
      if (!epi_all(oka)) break;
      const uint64_t tepi = PROF ? clock64() : 0;
      tc_fence_after();
      const uint64_t tag = acc_unit[buf];
      if (tag == kNoUnit) {
        if (epi_all(wait(ostage_empty, oph ^ 1u, kErrMmaWait))) {
          if (et == 0) *ostage_unit = kNoUnit;
          __syncwarp();
          if (lane == 0) mbar_arrive(ostage_full);
        }
        break;
      }
      const uint64_t un = tag & ~(1ull << 63);
      const bool last = (tag >> 63) != 0;
      const TmJob &jb = p.job[job_of_unit<MULTI>(p, un)];
      const uint32_t l = p.gpl_d.div(jb.mblk_d.div((uint32_t)(entry_of(un) - jb.entry0)));
      const TmLimb &lm = p.limb[l];
      const int32_t w0 = lm.w[u][0], w1 = lm.w[u][1], w2 = lm.w[u][2];
      const uint32_t tbase = tmem_base + ((qw * 32u) << 16) + buf * T_ACC_COLS + half * 32u;
      // column groups c = 0..7 in a loop (not unrolled: a small hot loop for
      // the instruction caches); the sums rotate so that acc64[0] is c's
#pragma unroll 1
      for (int c = 0; c < 8; ++c) {
        uint32_t d[12];
        tmem_ld4x3(tbase + c * 4, tbase + 64 + c * 4, tbase + 128 + c * 4, d);
        int64_t P[4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
          P[i] = (int64_t)__float2int_rn(__uint_as_float(d[i])) * w0 +
                 (int64_t)__float2int_rn(__uint_as_float(d[4 + i])) * w1 +
                 (int64_t)__float2int_rn(__uint_as_float(d[8 + i])) * w2;
        // reduce-scatter over the 4 digits u (lanes u*8 + m_lo): thread u keeps
        // column c*4 + u of its half
        const int b0 = u & 1, b1 = (u >> 1) & 1;
        int64_t K1[2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          const int64_t keep = b0 ? P[2 * i + 1] : P[2 * i];
          const int64_t send = b0 ? P[2 * i] : P[2 * i + 1];
          K1[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
        }
        const int64_t keep = b1 ? K1[1] : K1[0];
        const int64_t send = b1 ? K1[0] : K1[1];
        const int64_t a0 = acc64[0] + keep + __shfl_xor_sync(0xffffffffu, send, 16);
#pragma unroll
        for (int k2 = 0; k2 < 7; ++k2) acc64[k2] = acc64[k2 + 1];
        acc64[7] = a0;   // after the 8 steps acc64[c] is column group c's again
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&acc_empty[buf]);
        if (PAIR && rank != 0) mbar_arrive_remote_relaxed(map_peer(smem_u32(&acc_empty[buf]), 0));
      }
      aph[buf] ^= 1u;
      buf ^= 1u;
      if (epi_counter) pc[PROF ? kTEBusy : 0] += clock64() - tepi;
      if (last || ++ngroups == T_FLUSH) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const uint32_t rr = reduce64((uint64_t)(acc64[i] + (int64_t)lm.off58), lm.q, lm.mu);
          const uint32_t a = res[i] + rr;
          res[i] = a >= lm.q ? a - lm.q : a;
          acc64[i] = 0;
        }
        ngroups = 0;
      }
      if (last) {
        if (!epi_all(wait(ostage_empty, oph ^ 1u, kErrMmaWait))) break;
        const uint32_t swz = (uint32_t)m_lo << 2;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const uint32_t n = half * 32u + c * 4u + (uint32_t)u;
          out_stage[m_local * T_NCOLS + (n ^ swz)] = res[c];
        }
        if (et == 0) *ostage_unit = un;
        __syncwarp();
        if (lane == 0) mbar_arrive(ostage_full);
        oph ^= 1u;
#pragma unroll
        for (int i = 0; i < 8; ++i) res[i] = 0;
      }
    }
  } else if (PAIR && warp == W_RELAY) {
    // ---------------- relay (pair, even CTA): group tags to the odd CTA ----------------
    // The odd CTA's acc_full completes on the MMA commit (multicast) and on
    // this remote arrive, whose release orders the tag store before it. The
    // MMA thread cannot reuse acc_unit[b] before the odd epilogue, which needs
    // this arrive, has drained the accumulator.
    if (rank == 0 && lane == 0) {
      uint32_t hb = 0, hph[2] = {0, 0};
      for (;;) {
        if (!wait(&hand_full[hb], hph[hb], kErrMmaWait)) break;
        const uint64_t tag = acc_unit[hb];
        st_cluster_u64(map_peer(smem_u32(&acc_unit[hb]), 1), tag);
        mbar_arrive_remote(map_peer(smem_u32(&acc_full[hb]), 1));
        if (tag == kNoUnit) {
          mbar_arrive_remote(map_peer(smem_u32(&acc_full[hb]), 1));   // no commit comes after the last group
          break;
        }
        hph[hb] ^= 1u;
        hb ^= 1u;
      }
    }
  } else if (warp == W_STORE) {
    // ---------------- output store warp ----------------
    uint32_t ph = 0;
    for (;;) {
      if (!__all_sync(0xffffffffu, wait(ostage_full, ph, kErrMmaWait))) break;
      const uint64_t un = *ostage_unit;
      if (un == kNoUnit) break;
      const TmJob &jb = p.job[job_of_unit<MULTI>(p, un)];
      const uint64_t El = entry_of(un) - jb.entry0;
      const uint32_t w = jb.upe_d.mod((uint32_t)(un - jb.unit0)), sl = jb.nblk_d.div(w), nb = w - sl * jb.nblk;
      const uint32_t g = jb.mblk_d.div((uint32_t)El), mb = (uint32_t)El - g * jb.mblk;
      const uint32_t l = p.gpl_d.div(g), t = (g - l * p.gpl) * 8 + sl;
      const uint32_t mrows = min((uint32_t)T_MROWS, jb.M - mb * T_MROWS);
      const uint32_t ncols = min((uint32_t)T_NCOLS, jb.d1 - nb * T_NCOLS);
      const uint64_t nstride = (uint64_t)2 * p.L * p.N;
      for (uint32_t mm = 0; mm < mrows; ++mm) {
        const uint32_t mg = mb * T_MROWS + mm, c = mg >> 1, rr = mg & 1;
        const uint32_t sw = (mm & 7u) << 2;
        uint32_t *orow = jb.out + (((uint64_t)c * jb.d1 + nb * T_NCOLS) * 2 + rr) * p.L * p.N + (uint64_t)l * p.N + t;
#pragma unroll
        for (uint32_t hh = 0; hh < T_NCOLS / 32; ++hh) {
          const uint32_t n = hh * 32 + lane;
          if (n < ncols) orow[n * nstride] = out_stage[mm * T_NCOLS + (n ^ sw)];
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(ostage_empty);
      ph ^= 1u;
    }
  } else if (warp >= W_ING0) {
    // ---------------- ingest (8 warps, 256 threads) ----------------
    // Task = (entry E, k-chunk kc): 64 KB of raw residues, 8 slots x 32 rows
    // x 64 k, loaded as 16 / BOX_CLIENTS TMA boxes of BOX_CLIENTS clients
    // into two box buffers in turn: box g + 1 (the task's next box, or the
    // next task's first) loads while box g is processed. A task's ring wait
    // (its entry's previous occupant consumed, the lookahead bound) stays at
    // its start, after the previous task is published: it may depend on that
    // task. A thread handles (row, k octet, slot half) items; for each slot it
    // stores the 8 encoded residues of its row and octet as their four digit
    // planes in two 16-byte chunks of the slot's ring tile, chunk c16 of row m
    // at position c16 ^ (m % 8).
    const int it = (warp - W_ING0) * 32 + lane;
    constexpr int NT = 32 * N_ING;
    constexpr int NPART = T_TASK_CLIENTS / Cfg::BOX_CLIENTS;
    const uint64_t pol_last = l2_policy_evict_last();
    uint32_t pend = 0, pend_ph = 0;   // thread 0: box buffers loading, parity of their phase
    auto issue = [&](uint32_t gb, uint64_t task, int part) {
      // box gb (global box index) of `task`, part `part`, into buffer gb % 2
      const TmJob &jb = p.job[job_of_task<MULTI>(p, task)];
      const uint32_t tl = (uint32_t)(task - jb.task0), El = jb.kch_d.div(tl);
      const uint32_t kc = tl - El * jb.kch;
      const uint32_t g = jb.mblk_d.div(El), mb = El - g * jb.mblk;
      const uint32_t l = p.gpl_d.div(g), t0 = (g - l * p.gpl) * 8;
      const uint32_t b = gb & 1u;
      const int c0 = (int)(mb * T_TASK_CLIENTS) + part * Cfg::BOX_CLIENTS;
      uint8_t *dst = rawbox + b * Cfg::RAW_BOX;
      mbar_arrive_expect_tx(&box_bar[b], Cfg::RAW_BOX);
      if (p.hints)
        tma_load_5d_hint(dst, &jb.ct_map, &box_bar[b], (int)t0, (int)l, 0, (int)(kc * T_KCHUNK), c0,
                         l2_policy_evict_first());
      else
        tma_load_5d(dst, &jb.ct_map, &box_bar[b], (int)t0, (int)l, 0, (int)(kc * T_KCHUNK), c0);
      pend |= 1u << b;
      pend_ph = (pend_ph & ~(1u << b)) | (((gb >> 1) & 1u) << b);
    };
    auto claim_task = [&]() -> uint64_t {
      const uint64_t c = atomicAdd(&p.ctr[1], 1ull);
      return (c < p.n_tasks && !*abort_flag) ? c : kNoUnit;
    };
    if (it == 0) {
      const uint64_t c = claim_task();
      if (c != kNoUnit) issue(0, c, 0);
      *task_slot = c;
    }
    asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
    uint64_t c = *task_slot;
    uint32_t gbox = 0;
    // Lane = (k octet j, row parity rp, slot half sh). A thread takes the 4
    // slots of its half one at a time, reading one 4-byte word per k offset:
    // a loop over the slots keeps the ingest's code small (fully unrolled over
    // slots, with 16-byte reads, the kernel's hot code outgrew the instruction
    // caches and ran 2-5% slower). With k offset kk ^ (j & 1) and slot half
    // sh = (lane & 1) ^ ((j >> 1) & 1) a read instruction touches 8 banks, 4
    // lanes each (4 wavefronts; 8 without the swaps); the byte selectors of
    // the plane transpose undo the swap of k offsets in odd octets.
    const int j = lane >> 2, rp = (lane >> 1) & 1;
    const int j0 = j & 1, sh = (lane & 1) ^ ((j >> 1) & 1);
    const uint32_t sel_a = j0 ? 0x1504u : 0x5140u, sel_b = j0 ? 0x3726u : 0x7362u;
    uint4 *ring4 = reinterpret_cast<uint4 *>(p.ring);
    while (c != kNoUnit) {
      const TmJob &jb = p.job[job_of_task<MULTI>(p, c)];
      const uint32_t tl = (uint32_t)(c - jb.task0), El = jb.kch_d.div(tl);
      const uint64_t E = jb.entry0 + El;   // global entry
      const uint32_t kc = tl - El * jb.kch;
      const uint32_t g = jb.mblk_d.div(El);
      const uint32_t l = p.gpl_d.div(g), t0 = (g - l * p.gpl) * 8;
      if (it == 0) {
        // ring slot E % R: its previous entry E - R read by all of its units;
        // and at most `lookahead` entries ahead of the units claimed
        const bool near = p.lookahead == 0 || E < p.lookahead ||
                          TM_TIMED(kTIWaitSlot, wait_claims(first_unit_of(E - p.lookahead)));
        const bool free =
            near && (E < p.R || TM_TIMED(kTIWaitSlot, wait_count(&p.consumed[E - p.R],
                                                                 p.job[job_of_entry<MULTI>(p, E - p.R)].upe)));
        *task_ok = free ? 1u : 0u;   // task_slot may still be read for this task
      }
      asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
      if (*task_ok == 0u) break;
      const uint64_t tbusy = PROF ? clock64() : 0;
      uint64_t twait = 0;
      const uint32_t q = p.limb[l].q, h = p.limb[l].h;
      uint64_t cn = kNoUnit;
      bool got_all = true;
#pragma unroll 1
      for (int part = 0; part < NPART; ++part, ++gbox) {
        if (it == 0) {
          // the other buffer was read out before the last barrier
          if (part + 1 < NPART) {
            issue(gbox + 1, c, part + 1);
          } else {
            cn = claim_task();
            if (cn != kNoUnit) issue(gbox + 1, cn, 0);
          }
        }
        const uint32_t b = gbox & 1u;
        const uint64_t tw0 = PROF ? clock64() : 0;
        uint32_t got = wait(&box_bar[b], (gbox >> 1) & 1u, kErrTmaWait) ? 1u : 0u;
        if (PROF && it == 0) twait += clock64() - tw0;
        asm volatile(
            "{\n .reg .pred pin, pout;\n setp.ne.u32 pin, %1, 0;\n bar.red.and.pred pout, 1, %2, pin;\n"
            " selp.u32 %0, 1, 0, pout;\n}"
            : "=r"(got)
            : "r"(got), "n"(NT)
            : "memory");
        if (!got) {
          got_all = false;
          break;
        }
        if (it == 0) pend &= ~(1u << b);
        const uint32_t *raw1 = reinterpret_cast<const uint32_t *>(rawbox + b * Cfg::RAW_BOX);
#pragma unroll 1
        for (int cb = it >> 5; cb < Cfg::BOX_CLIENTS; cb += NT / 32) {
          const int m_local = (part * Cfg::BOX_CLIENTS + cb) * 2 + rp;
#pragma unroll 1
          for (int i = 0; i < 4; ++i) {
            const int sl = sh * 4 + i;
            if (t0 + sl >= p.N) continue;
            // ring words of k offsets 8j + (kk ^ j0), position kk: box word
            // ((cb * 64 + k) * 2 + rp) * 8 + sh * 4 + i, from one base for the
            // even positions and one for the odd (k offset kk + j0 / kk - j0)
            uint32_t z[8];
            const uint32_t *be = raw1 + ((cb * T_KCHUNK + j * 8) * 2 + rp) * 8 + sh * 4 + i + j0 * 16;
            const uint32_t *bo = be - 2 * j0 * 16;
#pragma unroll
            for (int kk = 0; kk < 8; ++kk)
              z[kk] = ct_fields((kk & 1) ? bo[kk * 16] : be[kk * 16], q, h);
            uint4 *tile = ring4 + ((((uint64_t)p.R_d.mod((uint32_t)E) * 8 + sl) * p.kch_max + kc) * (uint64_t)T_RAW_TILE) / 16;
            uint32_t pl[4], ph[4];   // digit planes of k 8j .. 8j + 3 and 8j + 4 .. 8j + 7
            digit_planes(z[0], z[1], z[2], z[3], sel_a, sel_b, pl);
            digit_planes(z[4], z[5], z[6], z[7], sel_a, sel_b, ph);
            const uint4 lo = make_uint4(pl[0], ph[0], pl[1], ph[1]);   // chunk 2j: digits 0, 1
            const uint4 hi = make_uint4(pl[2], ph[2], pl[3], ph[3]);   // chunk 2j + 1: digits 2, 3
            if (p.hints) {
              st_global_v4_hint(&tile[m_local * 16 + ((2 * j) ^ (m_local & 7))], lo, pol_last);
              st_global_v4_hint(&tile[m_local * 16 + ((2 * j + 1) ^ (m_local & 7))], hi, pol_last);
            } else {
              tile[m_local * 16 + ((2 * j) ^ (m_local & 7))] = lo;
              tile[m_local * 16 + ((2 * j + 1) ^ (m_local & 7))] = hi;
            }
          }
        }
        asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");   // box buffer b read out
      }
      if (!got_all) break;
      if (PROF && it == 0) pc[PROF ? kTIWaitBox : 0] += twait;
      fence_proxy_async_global();
      const uint64_t tfence = PROF ? clock64() : 0;
      if (PROF && it == 0) pc[PROF ? kTIBusy : 0] += tfence - tbusy - twait;
      asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
      if (it == 0) {
        __threadfence();
        atomicAdd(&p.ready[E], 1u);
        if (PROF) pc[PROF ? kTIFence : 0] += clock64() - tfence;
        *task_slot = cn;
      }
      asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
      c = *task_slot;
    }
    // let box loads still in flight land before the CTA leaves
    if (it == 0)
      for (uint32_t b = 0; b < 2; ++b)
        if ((pend >> b) & 1u) mbar_wait_bounded(&box_bar[b], (pend_ph >> b) & 1u, nullptr, 0);
  }
#undef TM_TIMED
  if (PROF) {
    // one counting thread per role: producer, MMA, converter warp 0, epilogue thread 0, ingest thread 0
    const bool counter = lane == 0 && (warp == W_PROD || warp == W_MMA || warp == W_CONV0 || warp == W_EPI0 ||
                                       warp == W_ING0);
    if (counter)
      for (int i = 0; i < (PROF ? kNumTmemCounters : 1) - 1; ++i)
        if (pc[i]) atomicAdd(&p.prof[i], pc[i]);
    if (threadIdx.x == 0) atomicAdd(&p.prof[kTCta], clock64() - kstart);
  }
  tc_fence_before();
  if constexpr (PAIR)
    cluster_sync_all();
  else
    __syncthreads();
  tc_fence_after();
  if (warp == W_MMA) {
    if constexpr (PAIR)
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(T_TMEM_COLS)
                   : "memory");
    else
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(T_TMEM_COLS)
                   : "memory");
  }
}

TmLimb make_tm_limb(uint32_t q) {
  TmLimb t;
  t.q = q;
  t.h = (q - 1) / 2;
  t.mu = ~0ull / q;
  const uint64_t two58 = 1ull << 58;
  t.off58 = ((two58 + q - 1) / q) * (uint64_t)q;
  for (int u = 0; u < 4; ++u)
    for (int v = 0; v < 3; ++v) {
      uint64_t pw = 1;
      for (int e = 0; e < 7 * u + 10 * v; ++e) pw = (pw * 2) % q;
      t.w[u][v] = (int32_t)pw;
    }
  return t;
}

std::mutex g_tm_mu;
bool g_tm_attr_done[64];
int g_tm_pairs[64];   // resident CTA pairs of the pair form per device (-1: none)

cudaLaunchConfig_t tm_pair_config(unsigned grid, cudaStream_t stream, cudaLaunchAttribute *attr) {
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(T_THREADS);
  cfg.dynamicSmemBytes = TmemCfg<true>::SMEM;
  cfg.stream = stream;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

}  // namespace

int rowsel_tmem_prepare(gpir_db *db, cudaStream_t stream) {
  const uint32_t L = db->params.num_limbs, N = db->params.n;
  const uint32_t nblk = (db->d1 + T_NCOLS - 1) / T_NCOLS, kch = (db->d0 + T_KCHUNK - 1) / T_KCHUNK;
  const uint64_t slots = (uint64_t)L * N;
  const size_t bytes = (size_t)slots * nblk * kch * T_B_TILE;
  cudaError_t e = dev_malloc(reinterpret_cast<void **>(&db->db_digits12), bytes);
  if (e != cudaSuccess) {
    db->db_digits12 = nullptr;
    return set_cuda_error(e);
  }
  db->db_digits12_bytes = bytes;
  Pack12Params pp;
  memset(&pp, 0, sizeof(pp));
  pp.d0 = db->d0;
  pp.d1 = db->d1;
  pp.L = L;
  pp.N = N;
  pp.nblk = nblk;
  pp.kch = kch;
  pp.db = db->db_pmajor;
  pp.b_tiles = reinterpret_cast<uint4 *>(db->db_digits12);
  for (uint32_t l = 0; l < L; ++l) pp.q[l] = db->params.primes[l];
  const uint64_t total = slots * nblk * kch * T_NDIG * 8;
  tm_pack_db_kernel<<<sm_count() * 16, 256, 0, stream>>>(pp, total);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_cuda_error(e);
  e = cudaStreamSynchronize(stream);
  return e == cudaSuccess ? GPIR_OK : set_cuda_error(e);
}

// RowSel problems (at most T_MAX_JOBS, one parameter set) through one launch
// of the tensor-memory kernel. pair: the SM-pair form; GPIR_ENOTSUP when a
// job has an odd number of 32-row m-blocks or no CTA pair can be resident.
int tc_launch_tmem_jobs(const gpir_job_t *jobs, uint32_t njobs, size_t ring_target, uint32_t lookahead_mb,
                        uint32_t hints, bool pair, cudaStream_t stream) {
  if (njobs == 0 || njobs > (uint32_t)T_MAX_JOBS) return GPIR_EINVAL;
  if (pair && njobs > 1) return GPIR_ENOTSUP;   // the SM-pair form runs one job
  for (uint32_t k = 0; k < njobs; ++k) {
    if (!jobs[k].db->db_digits12) return GPIR_ENOTSUP;
    const uint32_t mblk = (2 * jobs[k].batch + T_MROWS - 1) / T_MROWS;
    if (pair && (mblk & 1u)) return GPIR_ENOTSUP;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_cuda_error(e);
  if (dev < 0 || dev >= 64) return GPIR_EINVAL;
  {
    std::lock_guard<std::mutex> lk(g_tm_mu);
    if (!g_tm_attr_done[dev]) {
      e = cudaFuncSetAttribute(tc_tmem_kernel<false, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)TmemCfg<false>::SMEM);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_tmem_kernel<true, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)TmemCfg<false>::SMEM);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_tmem_kernel<false, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)TmemCfg<false>::SMEM);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_tmem_kernel<true, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)TmemCfg<false>::SMEM);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_tmem_kernel<false, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)TmemCfg<true>::SMEM);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_tmem_kernel<true, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)TmemCfg<true>::SMEM);
      if (e != cudaSuccess) return set_cuda_error(e);
      cudaLaunchAttribute attr[1];
      const cudaLaunchConfig_t cfg = tm_pair_config((unsigned)(sm_count() / 2 * 2), nullptr, attr);
      int n = 0;
      e = cudaOccupancyMaxActiveClusters(&n, tc_tmem_kernel<false, true, false>, &cfg);
      if (e != cudaSuccess) {
        cudaGetLastError();
        n = 0;
      }
      g_tm_pairs[dev] = n > 0 ? n : -1;
      g_tm_attr_done[dev] = true;
    }
  }
  if (pair && g_tm_pairs[dev] < 0) return GPIR_ENOTSUP;
  const gpir_params &prm = jobs[0].db->params;
  const uint32_t L = prm.num_limbs, N = prm.n;
  auto tm_div = [](uint32_t d) {
    TmDiv v;
    if (d == 0) d = 1;   // not reached: every divisor counts at least one item
    v.d = d;
    v.l = 0;
    while ((1ull << v.l) < d) ++v.l;
    v.m = (uint32_t)((((uint64_t)1 << 32) * ((1ull << v.l) - d)) / d + 1);
    return v;
  };
  TmemParams tp;
  memset(&tp, 0, sizeof(tp));
  tp.L = L;
  tp.N = N;
  tp.njobs = njobs;
  tp.gpl = (N + 7) / 8;
  tp.spg = N < 8 ? N : 8u;
  uint64_t entries = 0, units = 0, tasks = 0;
  uint32_t kch_max = 1;
  for (uint32_t k = 0; k < njobs; ++k) {
    const gpir_db *db = jobs[k].db;
    TmJob &jb = tp.job[k];
    jb.M = 2 * jobs[k].batch;
    jb.d1 = db->d1;
    jb.mblk = (jb.M + T_MROWS - 1) / T_MROWS;
    jb.nblk = (db->d1 + T_NCOLS - 1) / T_NCOLS;
    jb.kch = (db->d0 + T_KCHUNK - 1) / T_KCHUNK;
    jb.upe = tp.spg * jb.nblk;
    jb.mblk_d = tm_div(jb.mblk);
    jb.nblk_d = tm_div(jb.nblk);
    jb.kch_d = tm_div(jb.kch);
    jb.upe_d = tm_div(jb.upe);
    jb.entry0 = entries;
    jb.unit0 = units;
    jb.task0 = tasks;
    jb.b_tiles = db->db_digits12;
    jb.out = jobs[k].out;
    const uint64_t ne = (uint64_t)tp.gpl * L * jb.mblk;
    entries += ne;
    units += (pair ? ne / 2 : ne) * jb.upe;
    tasks += ne * jb.kch;
    kch_max = std::max(kch_max, jb.kch);
    const uint64_t dims[5] = {N, L, 2, db->d0, jobs[k].batch};
    const uint64_t str[4] = {(uint64_t)N * 4, (uint64_t)L * N * 4, (uint64_t)2 * L * N * 4,
                             (uint64_t)db->d0 * 2 * L * N * 4};
    const uint32_t box[5] = {8, 1, 2, (uint32_t)T_KCHUNK,
                             (uint32_t)(pair ? TmemCfg<true>::BOX_CLIENTS : TmemCfg<false>::BOX_CLIENTS)};
    const int rc = encode_tiled_u32(&jb.ct_map, jobs[k].ct, 5, dims, str, box);
    if (rc != GPIR_OK) return rc;
  }
  // The kernel divides unit, entry and ingest-task indices in 32 bits. Any
  // launch whose ciphertexts fit in device memory has far fewer than 2^32 of
  // each (an entry alone covers 16 clients' 8 slots of every row).
  if (units > UINT32_MAX || entries > UINT32_MAX || tasks > UINT32_MAX) return GPIR_ETOOBIG;
  tp.n_entries = entries;
  tp.n_units = units;
  tp.n_tasks = tasks;
  tp.kch_max = kch_max;
  const size_t entry_bytes = (size_t)8 * kch_max * T_RAW_TILE;
  uint64_t R = ring_target / entry_bytes;
  if (R < 2) R = 2;
  if (pair && (R & 1)) ++R;   // both entries of a pair unit share R's parity classes
  if (R > tp.n_entries) R = tp.n_entries;
  tp.R = (uint32_t)R;
  tp.R_d = tm_div(tp.R);
  tp.gpl_d = tm_div(tp.gpl);
  const size_t ring_bytes = (size_t)R * entry_bytes;
  // counters: [2] claims, ready[n_entries], consumed[n_entries], role counters
  const size_t flag_bytes = ((size_t)16 + 8 * entries + 8 + 8 * kNumTmemCounters + 255) & ~(size_t)255;
  uint8_t *ws = nullptr;
  int rc = tc_stream_workspace(stream, ring_bytes + flag_bytes, &ws);
  if (rc != GPIR_OK) return rc;
  tp.ring = ws;
  uint8_t *flags = ws + ring_bytes;
  tp.ctr = reinterpret_cast<unsigned long long *>(flags);
  tp.ready = reinterpret_cast<uint32_t *>(flags + 16);
  tp.consumed = tp.ready + entries;
  tp.prof = trace_counters_enabled()
                ? reinterpret_cast<unsigned long long *>(((uintptr_t)(tp.consumed + entries) + 7) & ~(uintptr_t)7)
                : nullptr;
  e = cudaMemsetAsync(flags, 0, flag_bytes, stream);
  if (e != cudaSuccess) return set_cuda_error(e);
  tp.hints = hints;
  tp.lookahead =
      lookahead_mb == 0 ? 0u : (uint32_t)std::max<uint64_t>(2, ((uint64_t)lookahead_mb << 20) / entry_bytes);
  tp.err = device_error_word();
  for (uint32_t l = 0; l < L; ++l) tp.limb[l] = make_tm_limb(prm.primes[l]);
  if (pair) {
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg = tm_pair_config((unsigned)(2 * g_tm_pairs[dev]), stream, attr);
    const int tr = trace_begin("tc_tmem_pair", stream);
    e = tp.prof ? cudaLaunchKernelEx(&cfg, tc_tmem_kernel<true, true, false>, tp)
                : cudaLaunchKernelEx(&cfg, tc_tmem_kernel<false, true, false>, tp);
    trace_end(tr, stream);
    if (e != cudaSuccess) return set_cuda_error(e);
    if (tp.prof) trace_counters(tp.prof, kNumTmemCounters, stream);
    e = cudaGetLastError();
    return e == cudaSuccess ? GPIR_OK : set_cuda_error(e);
  }
  const int tr = trace_begin("tc_tmem", stream);
  if (tp.prof)
    (njobs > 1 ? tc_tmem_kernel<true, false, true> : tc_tmem_kernel<true, false, false>)
        <<<sm_count(), T_THREADS, TmemCfg<false>::SMEM, stream>>>(tp);
  else
    (njobs > 1 ? tc_tmem_kernel<false, false, true> : tc_tmem_kernel<false, false, false>)
        <<<sm_count(), T_THREADS, TmemCfg<false>::SMEM, stream>>>(tp);
  trace_end(tr, stream);
  if (tp.prof) trace_counters(tp.prof, kNumTmemCounters, stream);
  e = cudaGetLastError();
  return e == cudaSuccess ? GPIR_OK : set_cuda_error(e);
}


// Several jobs, T_MAX_JOBS per launch, in the single-CTA form with the ring
// and lookahead of tile variant 8.
int rowsel_tmem_multi(const gpir_job_t *jobs, uint32_t njobs, cudaStream_t stream) {
  for (uint32_t k0 = 0; k0 < njobs; k0 += T_MAX_JOBS) {
    const uint32_t n = std::min<uint32_t>(T_MAX_JOBS, njobs - k0);
    const int rc = tc_launch_tmem_jobs(jobs + k0, n, (size_t)24 << 20, 8, 0, false, stream);
    if (rc != GPIR_OK) return rc;
  }
  return GPIR_OK;
}

int tc_launch_tmem(const gpir_db *db, uint32_t batch, const uint32_t *ct, uint32_t *out, size_t ring_target,
                   uint32_t lookahead_mb, uint32_t hints, bool pair, cudaStream_t stream) {
  gpir_job_t job;
  memset(&job, 0, sizeof(job));
  job.db = db;
  job.batch = batch;
  job.ct = ct;
  job.out = out;
  return tc_launch_tmem_jobs(&job, 1, ring_target, lookahead_mb, hints, pair, stream);
}

}  // namespace gpir
