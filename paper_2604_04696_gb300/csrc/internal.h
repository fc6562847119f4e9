// Internal declarations shared by the translation units of libgpir.so.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <tuple>

#include "../../include/gpir.h"

#include <nvtx3/nvToolsExt.h>

namespace gpir {

// Per-limb modulus data passed by value to kernels.
struct Modulus {
  uint32_t q;
  uint32_t pad;
  uint64_t mu;   // floor(2^64 / q): Barrett constant for 64-bit reduction
};

struct LimbTable {
  Modulus m[GPIR_MAX_LIMBS];
};

// Shape of one RowSel problem (Sec. 2.3 extents): M = 2 * batch rows,
// K = D0 reduction, Nc = D1 columns, per (limb, slot) point.
struct Shape {
  uint32_t batch, d0, d1, L, N;
};

}  // namespace gpir

struct gpir_params {
  uint32_t n;
  uint32_t num_limbs;
  uint32_t primes[GPIR_MAX_LIMBS];
  gpir::LimbTable limbs;
};

struct gpir_db {
  gpir_params params;
  uint32_t d0, d1;
  uint32_t path_mask;
  int device;
  // CUDA-core and IMMA paths read the p-major database as uploaded.
  uint32_t *db_pmajor;          // [D0][D1][L][N]
  // tcgen05 path: balanced base-256 digits as fp16, slot-major (rowsel_tc.cu),
  // and the three base-2^10 digits of the centred residues (rowsel_tmem.cu).
  uint16_t *db_digits;
  size_t db_digits_bytes;
  uint16_t *db_digits12;
  size_t db_digits12_bytes;
  // Host-buffer entry point workspace.
  uint32_t *ws_ct, *ws_out;
  size_t ws_ct_bytes, ws_out_bytes;
  // Autotune cache: (path, batch) -> variant
  std::map<std::pair<int, uint32_t>, int> *variants;
  std::mutex *mu;
};

namespace gpir {

// Error helpers
int set_cuda_error(cudaError_t e);

// Every device allocation of the library goes through this wrapper: cudaMalloc,
// unless the allocation-failure injection (GPIR_FAIL_ALLOC /
// gpir_set_fail_alloc) makes it fail with cudaErrorMemoryAllocation.
cudaError_t dev_malloc(void **p, size_t bytes);

// TMA descriptor encoding (driver entry point resolved at first use).
int encode_tiled_u32(CUtensorMap *map, const void *base, int rank, const uint64_t *dims,
                     const uint64_t *strides_bytes /* rank-1 entries */, const uint32_t *box);
int encode_tiled(CUtensorMap *map, CUtensorMapDataType dt, const void *base, int rank,
                 const uint64_t *dims, const uint64_t *strides_bytes, const uint32_t *box,
                 CUtensorMapSwizzle swz);

// Device error word written by bounded waits in kernels (0 = ok).
unsigned int *device_error_word();
int sm_count();

// Debug checks (gpir_set_debug / GPIR_DEBUG): on or off.
bool debug_checks();
// Debug check of a device tensor whose two innermost dimensions are [L][N]:
// GPIR_ERANGE if a residue is not below its limb's prime. Synchronizes s;
// allocates nothing.
int check_residues_dev(const gpir_params &prm, const uint32_t *v, uint64_t count, cudaStream_t s);

// Scoped NVTX range around an ABI call (a no-op unless a profiler injects
// itself).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

// Path entry points (one per translation unit).
int rowsel_cc_launch(const gpir_db *db, uint32_t batch, const uint32_t *ct, uint32_t *out,
                     int variant, cudaStream_t stream);
int rowsel_cc_num_variants();
int rowsel_cc_default_variant(uint32_t batch, uint32_t d0, uint32_t d1);

int rowsel_imma_launch(const gpir_db *db, uint32_t batch, const uint32_t *ct, uint32_t *out,
                       int variant, cudaStream_t stream);
int rowsel_imma_num_variants();
int rowsel_imma_default_variant(uint32_t batch, uint32_t d0, uint32_t d1);

int rowsel_tc_prepare(gpir_db *db, cudaStream_t stream);
int rowsel_tc_launch(const gpir_db *db, uint32_t batch, const uint32_t *ct, uint32_t *out,
                     int variant, cudaStream_t stream);
int rowsel_tc_num_variants();
int rowsel_tc_default_variant(uint32_t batch, uint32_t d0, uint32_t d1);

// Tracing hooks: trace_begin returns -1 (and records nothing) when disabled.
int trace_begin(const char *name, cudaStream_t s);
void trace_end(int id, cudaStream_t s);
bool trace_enabled();
bool trace_counters_enabled();   // tracing at level 2: the role-counting kernel instantiations
void trace_counters(const unsigned long long *dev, int n, cudaStream_t s);

// Tensor-memory kernel (rowsel_tmem.cu): its database layout, built at upload,
// and one launch (pair: the SM-pair form; GPIR_ENOTSUP if it does not apply).
int rowsel_tmem_prepare(gpir_db *db, cudaStream_t stream);
// the path gpir_rowsel_batch runs for (db, batch) under `path` (GPIR_PATH_AUTO:
// the autotuned one, else tensor cores from batch 8, CUDA cores below); < 0: none
int resolve_path(const gpir_db *db, int path, uint32_t batch);
// several RowSel jobs (one parameter set) in tensor-memory kernel launches of up to 8 jobs each
int rowsel_tmem_multi(const gpir_job_t *jobs, uint32_t njobs, cudaStream_t stream);
int tc_launch_tmem(const gpir_db *db, uint32_t batch, const uint32_t *ct, uint32_t *out, size_t ring_target,
                   uint32_t lookahead_mb, uint32_t hints, bool pair, cudaStream_t stream);
// The tensor-core workspace kept for (current device, stream), grown on demand
// (never inside a stream capture: GPIR_ENOMEM then).
int tc_stream_workspace(cudaStream_t stream, size_t need, uint8_t **out);

int rowsel_tc_multi(const gpir_job_t *jobs, uint32_t njobs, cudaStream_t stream);
// Free the tensor-core workspace kept for (current device, stream), if any.
void rowsel_tc_release_stream(cudaStream_t stream);
size_t rowsel_tc_multi_workspace(const gpir_job_t *jobs, uint32_t njobs);

int rowsel_multi_launch(const gpir_job_t *jobs, uint32_t njobs, int path, cudaStream_t stream);
int dispatch(const gpir_db *db, uint32_t batch, const uint32_t *ct, uint32_t *out, int path, int variant,
             cudaStream_t s);
int pick_variant(const gpir_db *db, uint32_t batch, int path);

}  // namespace gpir
