// C ABI of libgpir.so: parameter checks, database residency, dispatch to the
// RowSel kernels, host-buffer entry point, bounded synchronization.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <mutex>
#include <new>
#include <thread>

#include <atomic>
#include <cstdlib>

#include "common.cuh"
#include "internal.h"

namespace gpir {

static __device__ unsigned int g_device_error = 0;
static __device__ unsigned int g_range_flag = 0;   // debug checks: a residue >= q was seen

static thread_local cudaError_t t_last_cuda_error = cudaSuccess;

int set_cuda_error(cudaError_t e) {
  t_last_cuda_error = e;
  if (e == cudaErrorMemoryAllocation) return GPIR_ENOMEM;
  return GPIR_ECUDA;
}

// Allocation-failure injection, for tests of the GPIR_ENOMEM paths that
// exhaust no GPU: armed with n > 0, the n-th device allocation the library
// makes from then on fails as if the device were out of memory, and the
// injection disarms itself. Armed from the environment variable
// GPIR_FAIL_ALLOC when the library first allocates, or by gpir_set_fail_alloc.
static std::atomic<long> g_fail_alloc{-1};   // -1: environment not read yet, 0: off

static void fail_alloc_init() {
  if (g_fail_alloc.load() >= 0) return;
  const char *v = std::getenv("GPIR_FAIL_ALLOC");
  long n = v ? std::strtol(v, nullptr, 10) : 0;
  long expect = -1;
  g_fail_alloc.compare_exchange_strong(expect, n > 0 ? n : 0);
}

cudaError_t dev_malloc(void **p, size_t bytes) {
  fail_alloc_init();
  for (;;) {
    long v = g_fail_alloc.load();
    if (v <= 0) break;
    if (g_fail_alloc.compare_exchange_weak(v, v - 1)) {
      if (v == 1) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
      }
      break;
    }
  }
  return cudaMalloc(p, bytes);
}

unsigned int *device_error_word() {
  int dev = 0;
  cudaGetDevice(&dev);
  static std::mutex mu;
  static std::map<int, unsigned int *> cache;
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_device_error) != cudaSuccess) return nullptr;
  cache[dev] = (unsigned int *)p;
  return (unsigned int *)p;
}

// Debug checks: -1 = not read yet, else 0 / 1.
static std::atomic<int> g_debug{-1};

bool debug_checks() {
  int d = g_debug.load(std::memory_order_relaxed);
  if (d < 0) {
    const char *v = std::getenv("GPIR_DEBUG");
    d = (v && std::strtol(v, nullptr, 10) != 0) ? 1 : 0;
    int expect = -1;
    g_debug.compare_exchange_strong(expect, d);
    d = g_debug.load(std::memory_order_relaxed);
  }
  return d == 1;
}

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n;
}

static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void *p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

int encode_tiled(CUtensorMap *map, CUtensorMapDataType dt, const void *base, int rank, const uint64_t *dims,
                 const uint64_t *strides_bytes, const uint32_t *box, CUtensorMapSwizzle swz) {
  auto fn = get_encode();
  if (!fn) return GPIR_ECUDA;
  if (((uintptr_t)base & 15u) != 0) return GPIR_EINVAL;
  for (int i = 0; i < rank - 1; ++i)
    if (strides_bytes[i] % 16 != 0) return GPIR_EINVAL;
  cuuint64_t gd[5];
  cuuint64_t gs[4];
  cuuint32_t bx[5], es[5];
  for (int i = 0; i < rank; ++i) {
    gd[i] = dims[i];
    bx[i] = box[i];
    es[i] = 1;
  }
  for (int i = 0; i < rank - 1; ++i) gs[i] = strides_bytes[i];
  CUresult r = fn(map, dt, (cuuint32_t)rank, const_cast<void *>(base), gd, gs, bx, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  swz, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? GPIR_OK : GPIR_EINVAL;
}

int encode_tiled_u32(CUtensorMap *map, const void *base, int rank, const uint64_t *dims,
                     const uint64_t *strides_bytes, const uint32_t *box) {
  return encode_tiled(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, base, rank, dims, strides_bytes, box,
                      CU_TENSOR_MAP_SWIZZLE_NONE);
}

// ---- device helpers for upload / synthetic fill ---------------------------

__global__ void range_check_kernel(const uint32_t *__restrict__ v, uint64_t count, uint32_t N, uint32_t L,
                                   LimbTable limbs, unsigned int *bad) {
  uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  unsigned int local = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
    uint32_t l = (uint32_t)((i / N) % L);
    local |= (v[i] >= limbs.m[l].q) ? 1u : 0u;
  }
  if (local) atomicOr(bad, 1u);
}

int check_residues_dev(const gpir_params &prm, const uint32_t *v, uint64_t count, cudaStream_t s) {
  static std::mutex mu;                       // one check at a time: they share the device flag
  static std::map<int, unsigned int *> flags;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_cuda_error(e);
  std::lock_guard<std::mutex> lk(mu);
  auto it = flags.find(dev);
  if (it == flags.end()) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_range_flag);
    if (e != cudaSuccess) return set_cuda_error(e);
    try {
      it = flags.emplace(dev, static_cast<unsigned int *>(p)).first;
    } catch (...) {   // no exception crosses the C ABI
      return GPIR_ENOMEM;
    }
  }
  if (count == 0) return GPIR_OK;
  unsigned int *flag = it->second;
  e = cudaMemsetAsync(flag, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return set_cuda_error(e);
  range_check_kernel<<<sm_count() * 4, 256, 0, s>>>(v, count, prm.n, prm.num_limbs, prm.limbs, flag);
  unsigned int h = 0;
  e = cudaMemcpyAsync(&h, flag, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return set_cuda_error(e);
  return h ? GPIR_ERANGE : GPIR_OK;
}

__device__ __forceinline__ uint64_t splitmix_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void fill_uniform_kernel(uint32_t *__restrict__ dst, uint64_t count, uint64_t start, uint64_t key,
                                    uint64_t inner, uint32_t L, LimbTable limbs) {
  uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
    uint64_t f = start + i;
    uint64_t v = splitmix_mix(key + (f + 1) * 0x9E3779B97F4A7C15ull);
    uint32_t l = (uint32_t)((f / inner) % L);
    dst[i] = reduce64(v, limbs.m[l].q, limbs.m[l].mu);
  }
}

static uint64_t host_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static bool is_prime_u32(uint32_t n) {
  if (n < 2) return false;
  if (n % 2 == 0) return n == 2;
  for (uint32_t d = 3; (uint64_t)d * d <= n; d += 2)
    if (n % d == 0) return false;
  return true;
}

int pick_variant(const gpir_db *db, uint32_t batch, int path) {
  {
    std::lock_guard<std::mutex> lk(*db->mu);
    auto it = db->variants->find({path, batch});
    if (it != db->variants->end()) return it->second;
  }
  switch (path) {
    case GPIR_PATH_CUDACORE: return rowsel_cc_default_variant(batch, db->d0, db->d1);
    case GPIR_PATH_IMMA: return rowsel_imma_default_variant(batch, db->d0, db->d1);
    case GPIR_PATH_TC: return rowsel_tc_default_variant(batch, db->d0, db->d1);
  }
  return -1;
}

// GPIR_PATH_AUTO: the path the autotuner measured fastest for this batch size,
// else a static choice: tensor cores once a batch fills a 32-row tile well
// (batch >= 8), CUDA cores below that (one client wastes 15/16 of an MMA tile).
int resolve_path(const gpir_db *db, int path, uint32_t batch) {
  if (path == GPIR_PATH_AUTO) {
    {
      std::lock_guard<std::mutex> lk(*db->mu);
      auto it = db->variants->find({GPIR_PATH_AUTO, batch});
      if (it != db->variants->end()) return it->second;
    }
    const bool tc = db->path_mask & GPIR_PATH_TC, cc = db->path_mask & GPIR_PATH_CUDACORE;
    if (tc && (batch >= 8 || !cc)) return GPIR_PATH_TC;
    if (cc) return GPIR_PATH_CUDACORE;
    if (db->path_mask & GPIR_PATH_IMMA) return GPIR_PATH_IMMA;
    return -1;
  }
  if (path != GPIR_PATH_CUDACORE && path != GPIR_PATH_IMMA && path != GPIR_PATH_TC) return -1;
  if (!(db->path_mask & path)) return -2;
  return path;
}

int dispatch(const gpir_db *db, uint32_t batch, const uint32_t *ct, uint32_t *out, int path, int variant,
             cudaStream_t s) {
  switch (path) {
    case GPIR_PATH_CUDACORE: return rowsel_cc_launch(db, batch, ct, out, variant, s);
    case GPIR_PATH_IMMA: return rowsel_imma_launch(db, batch, ct, out, variant, s);
    case GPIR_PATH_TC: return rowsel_tc_launch(db, batch, ct, out, variant, s);
  }
  return GPIR_EINVAL;
}

static int num_variants(int path) {
  switch (path) {
    case GPIR_PATH_CUDACORE: return rowsel_cc_num_variants();
    case GPIR_PATH_IMMA: return rowsel_imma_num_variants();
    case GPIR_PATH_TC: return rowsel_tc_num_variants();
  }
  return 0;
}

}  // namespace gpir

using namespace gpir;

// One thread waits on an mbarrier that nothing arrives on (phase 0 never
// completes), through the bounded wait of the RowSel kernels.
static __global__ void selftest_wait_kernel(unsigned int *err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    gpir::mbar_init(&bar, 1);
    gpir::fence_mbar_init();
    gpir::mbar_wait_bounded(&bar, 0, err, gpir::kErrQueueWait);
  }
}

extern "C" {

int gpir_version(void) { return 100; }

const char *gpir_last_cuda_error(void) { return cudaGetErrorString(t_last_cuda_error); }

const char *gpir_strerror(int code) {
  switch (code) {
    case GPIR_OK: return "ok";
    case GPIR_EINVAL: return "invalid argument";
    case GPIR_ERANGE: return "database residue not below its prime";
    case GPIR_ENOMEM: return "out of memory";
    case GPIR_ECUDA: return "CUDA runtime error";
    case GPIR_ETIMEOUT: return "bounded wait expired";
    case GPIR_ENOTSUP: return "path not prepared or not supported";
    case GPIR_ETOOBIG: return "problem exceeds a fixed-size workspace or the kernel index range";
  }
  return "unknown gpir error";
}

int gpir_params_create(uint32_t n, uint32_t num_limbs, const uint32_t *primes, gpir_params_t **out) {
  if (!out || !primes) return GPIR_EINVAL;
  *out = nullptr;
  if (n < GPIR_MIN_N || n > GPIR_MAX_N || (n & (n - 1)) != 0) return GPIR_EINVAL;
  if (num_limbs < 1 || num_limbs > GPIR_MAX_LIMBS) return GPIR_EINVAL;
  for (uint32_t l = 0; l < num_limbs; ++l) {
    uint32_t q = primes[l];
    if (q < 3 || q >= (1u << GPIR_MAX_PRIME_BITS)) return GPIR_EINVAL;
    if ((q - 1) % (2 * n) != 0) return GPIR_EINVAL;
    if (!is_prime_u32(q)) return GPIR_EINVAL;
  }
  gpir_params *p = new (std::nothrow) gpir_params;
  if (!p) return GPIR_ENOMEM;
  memset(p, 0, sizeof(*p));
  p->n = n;
  p->num_limbs = num_limbs;
  for (uint32_t l = 0; l < num_limbs; ++l) {
    p->primes[l] = primes[l];
    p->limbs.m[l].q = primes[l];
    p->limbs.m[l].mu = ~0ull / primes[l];  // floor((2^64 - 1) / q) = floor(2^64 / q) for q not a power of 2
  }
  *out = p;
  return GPIR_OK;
}

int gpir_params_destroy(gpir_params_t *params) {
  delete params;
  return GPIR_OK;
}

int gpir_db_upload(const gpir_params_t *params, uint32_t d0, uint32_t d1, const uint32_t *db_ntt, int db_on_device,
                   uint32_t path_mask, void *stream, gpir_db_t **out) {
  if (!params || !db_ntt || !out || d0 == 0 || d1 == 0) return GPIR_EINVAL;
  *out = nullptr;
  if (path_mask == 0) path_mask = GPIR_PATH_ALL;
  if (path_mask & ~(uint32_t)GPIR_PATH_ALL) return GPIR_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const uint64_t count = (uint64_t)d0 * d1 * params->num_limbs * params->n;
  const size_t bytes = count * 4;
  gpir_db *db = new (std::nothrow) gpir_db;
  if (!db) return GPIR_ENOMEM;
  memset((void *)db, 0, sizeof(*db));
  db->params = *params;
  db->d0 = d0;
  db->d1 = d1;
  db->path_mask = path_mask;
  cudaGetDevice(&db->device);
  db->variants = new (std::nothrow) std::map<std::pair<int, uint32_t>, int>();
  db->mu = new (std::nothrow) std::mutex();
  int rc = GPIR_OK;
  cudaError_t e = cudaSuccess;
  if (!db->variants || !db->mu) {
    rc = GPIR_ENOMEM;
    goto fail;
  }
  e = dev_malloc(reinterpret_cast<void **>(&db->db_pmajor), bytes);
  if (e != cudaSuccess) {
    db->db_pmajor = nullptr;
    rc = set_cuda_error(e);
    goto fail;
  }
  e = cudaMemcpyAsync(db->db_pmajor, db_ntt, bytes, db_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                      s);
  if (e != cudaSuccess) {
    rc = set_cuda_error(e);
    goto fail;
  }
  // every residue below its limb's prime ([D0][D1] polynomials of [L][N]);
  // synchronizes s, allocates nothing
  rc = check_residues_dev(params[0], db->db_pmajor, count, s);
  if (rc != GPIR_OK) goto fail;
  if (path_mask & GPIR_PATH_TC) {
    rc = rowsel_tc_prepare(db, s);
    if (rc == GPIR_OK) rc = rowsel_tmem_prepare(db, s);
    if (rc != GPIR_OK) goto fail;
  }
  *out = db;
  return GPIR_OK;
fail:
  gpir_db_free(db);
  return rc;
}

int gpir_db_free(gpir_db_t *db) {
  if (!db) return GPIR_OK;
  if (db->db_pmajor) cudaFree(db->db_pmajor);
  if (db->db_digits) cudaFree(db->db_digits);
  if (db->db_digits12) cudaFree(db->db_digits12);
  if (db->ws_ct) cudaFree(db->ws_ct);
  if (db->ws_out) cudaFree(db->ws_out);
  delete db->variants;
  delete db->mu;
  delete db;
  return GPIR_OK;
}

size_t gpir_db_device_bytes(const gpir_db_t *db) {
  if (!db) return 0;
  size_t b = (size_t)db->d0 * db->d1 * db->params.num_limbs * db->params.n * 4;
  return b + db->db_digits_bytes + db->db_digits12_bytes;
}

int gpir_rowsel_batch(const gpir_db_t *db, uint32_t batch, const uint32_t *ct_dev, uint32_t *out_dev, int path,
                      void *stream) {
  NvtxRange nvtx("gpir_rowsel_batch");
  if (!db || !ct_dev || !out_dev || batch == 0 || batch > GPIR_MAX_BATCH) return GPIR_EINVAL;
  int p = resolve_path(db, path, batch);
  if (p == -1) return GPIR_EINVAL;
  if (p == -2) return GPIR_ENOTSUP;
  const size_t ct_bytes = (size_t)batch * db->d0 * 2 * db->params.num_limbs * db->params.n * 4;
  const size_t out_bytes = (size_t)batch * db->d1 * 2 * db->params.num_limbs * db->params.n * 4;
  const uintptr_t a0 = (uintptr_t)ct_dev, a1 = a0 + ct_bytes, b0 = (uintptr_t)out_dev, b1 = b0 + out_bytes;
  if (a0 < b1 && b0 < a1) return GPIR_EINVAL;  // overlapping input / output
  if ((a0 & 15u) || (b0 & 15u)) return GPIR_EINVAL;
  if (debug_checks()) {
    const int rc = check_residues_dev(db->params, ct_dev, ct_bytes / 4, (cudaStream_t)stream);
    if (rc != GPIR_OK) return rc;
  }
  return dispatch(db, batch, ct_dev, out_dev, p, pick_variant(db, batch, p), (cudaStream_t)stream);
}

int gpir_pir_batch(const gpir_db_t *db, uint32_t batch, uint32_t stages, const uint32_t *query_dev,
                   const uint32_t *evk_dev, const uint32_t *rgsw_dev, uint32_t *sel_dev, uint32_t *rows_dev,
                   uint32_t *out_dev, int path, void *stream) {
  NvtxRange nvtx("gpir_pir_batch");
  if (!db || batch == 0 || batch > GPIR_MAX_BATCH || !query_dev || !rgsw_dev || !sel_dev || !rows_dev || !out_dev) return GPIR_EINVAL;
  if (db->d1 < 2 || (db->d1 & (db->d1 - 1)) != 0) return GPIR_EINVAL;
  if (stages >= 32 || db->d0 > (1u << stages)) return GPIR_EINVAL;
  const size_t ctw = (size_t)2 * db->params.num_limbs * db->params.n * 4;
  const uintptr_t q0 = (uintptr_t)query_dev, q1 = q0 + batch * ctw;
  const uintptr_t s0 = (uintptr_t)sel_dev, s1 = s0 + (size_t)batch * db->d0 * ctw;
  const uintptr_t r0 = (uintptr_t)rows_dev, r1 = r0 + (size_t)batch * db->d1 * ctw;
  const uintptr_t o0 = (uintptr_t)out_dev, o1 = o0 + batch * ctw;
  if ((q0 < s1 && s0 < q1) || (s0 < r1 && r0 < s1) || (r0 < o1 && o0 < r1) || (s0 < o1 && o0 < s1))
    return GPIR_EINVAL;
  int rc = gpir_expand_query(&db->params, batch, stages, db->d0, query_dev, evk_dev, sel_dev, stream);
  if (rc != GPIR_OK) return rc;
  rc = gpir_rowsel_batch(db, batch, sel_dev, rows_dev, path, stream);
  if (rc != GPIR_OK) return rc;
  return gpir_coltor(&db->params, batch, db->d1, rows_dev, rgsw_dev, out_dev, stream);
}

namespace {
// Internal copy streams and events of the host-buffer entry point, per device.
struct HostPipe {
  cudaStream_t in = nullptr, out = nullptr;
  static constexpr int kMaxChunks = 8;
  cudaEvent_t start = nullptr, copied[kMaxChunks] = {}, computed[kMaxChunks] = {}, done = nullptr;
};
std::mutex g_pipe_mu;
std::map<int, HostPipe> g_pipes;

int host_pipe(int dev, HostPipe **out) {
  auto it = g_pipes.find(dev);
  if (it != g_pipes.end()) {
    *out = &it->second;
    return GPIR_OK;
  }
  HostPipe hp;
  cudaError_t e = cudaStreamCreateWithFlags(&hp.in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&hp.out, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&hp.start, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&hp.done, cudaEventDisableTiming);
  for (int k = 0; k < HostPipe::kMaxChunks && e == cudaSuccess; ++k) {
    e = cudaEventCreateWithFlags(&hp.copied[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&hp.computed[k], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) {
    try {
      *out = &g_pipes.emplace(dev, hp).first->second;
      return GPIR_OK;
    } catch (...) {   // no exception crosses the C ABI
      e = cudaErrorMemoryAllocation;
    }
  }
  if (hp.in) cudaStreamDestroy(hp.in);
  if (hp.out) cudaStreamDestroy(hp.out);
  if (hp.start) cudaEventDestroy(hp.start);
  if (hp.done) cudaEventDestroy(hp.done);
  for (int k = 0; k < HostPipe::kMaxChunks; ++k) {
    if (hp.copied[k]) cudaEventDestroy(hp.copied[k]);
    if (hp.computed[k]) cudaEventDestroy(hp.computed[k]);
  }
  return set_cuda_error(e);
}
}  // namespace

int gpir_rowsel_batch_host(const gpir_db_t *db_c, uint32_t batch, const uint32_t *ct_host, uint32_t *out_host,
                           int path, void *stream) {
  NvtxRange nvtx("gpir_rowsel_batch_host");
  if (!db_c || !ct_host || !out_host || batch == 0 || batch > GPIR_MAX_BATCH) return GPIR_EINVAL;
  gpir_db *db = const_cast<gpir_db *>(db_c);
  if (debug_checks()) {
    // the host buffer, on the CPU: residue i belongs to limb (i / N) % L
    const uint32_t L = db->params.num_limbs, N = db->params.n;
    const uint64_t count = (uint64_t)batch * db->d0 * 2 * L * N;
    for (uint64_t i = 0; i < count; ++i)
      if (ct_host[i] >= db->params.limbs.m[(i / N) % L].q) return GPIR_ERANGE;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const size_t ct_client = (size_t)db->d0 * 2 * db->params.num_limbs * db->params.n * 4;
  const size_t out_client = (size_t)db->d1 * 2 * db->params.num_limbs * db->params.n * 4;
  const size_t ct_bytes = (size_t)batch * ct_client, out_bytes = (size_t)batch * out_client;
  cudaError_t e;
  if (db->ws_ct_bytes < ct_bytes) {
    if (db->ws_ct) {
      cudaStreamSynchronize(s);
      cudaFree(db->ws_ct);
    }
    db->ws_ct = nullptr;
    db->ws_ct_bytes = 0;
    e = dev_malloc(reinterpret_cast<void **>(&db->ws_ct), ct_bytes);
    if (e != cudaSuccess) {
      db->ws_ct = nullptr;
      return set_cuda_error(e);
    }
    db->ws_ct_bytes = ct_bytes;
  }
  if (db->ws_out_bytes < out_bytes) {
    if (db->ws_out) {
      cudaStreamSynchronize(s);
      cudaFree(db->ws_out);
    }
    db->ws_out = nullptr;
    db->ws_out_bytes = 0;
    e = dev_malloc(reinterpret_cast<void **>(&db->ws_out), out_bytes);
    if (e != cudaSuccess) {
      db->ws_out = nullptr;
      return set_cuda_error(e);
    }
    db->ws_out_bytes = out_bytes;
  }
  // Small batches: one copy in, RowSel, one copy out, all on `stream`.
  if (batch < 16) {
    e = cudaMemcpyAsync(db->ws_ct, ct_host, ct_bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return set_cuda_error(e);
    int rc = gpir_rowsel_batch(db, batch, db->ws_ct, db->ws_out, path, stream);
    if (rc != GPIR_OK) return rc;
    e = cudaMemcpyAsync(out_host, db->ws_out, out_bytes, cudaMemcpyDeviceToHost, s);
    return e == cudaSuccess ? GPIR_OK : set_cuda_error(e);
  }
  // Larger batches: the host link (about 210 GB/s each way on GB300) is the
  // bound, so the batch goes in client chunks through three ordered streams:
  // chunk k's upload (internal copy-in stream), chunk k-1's RowSel (`stream`),
  // chunk k-2's download (internal copy-out stream). Everything waits on the
  // work already in `stream` first, and `stream` waits on the last download,
  // so the call stays asynchronous on `stream` like the others. Eight equal
  // chunks measured best at 32 clients (half-size first and last chunks, to
  // shorten the pipeline's fill and drain, measured 2% slower).
  const uint32_t chunks = std::min<uint32_t>(8, batch / 4);
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_cuda_error(e);
  std::lock_guard<std::mutex> lk(g_pipe_mu);
  HostPipe *hp = nullptr;
  int rc = host_pipe(dev, &hp);
  if (rc != GPIR_OK) return rc;
  if ((e = cudaEventRecord(hp->start, s)) != cudaSuccess) return set_cuda_error(e);
  if ((e = cudaStreamWaitEvent(hp->in, hp->start, 0)) != cudaSuccess) return set_cuda_error(e);
  if ((e = cudaStreamWaitEvent(hp->out, hp->start, 0)) != cudaSuccess) return set_cuda_error(e);
  uint32_t c0 = 0;
  for (uint32_t k = 0; k < chunks; ++k) {
    const uint32_t bc = batch / chunks + (k < batch % chunks ? 1u : 0u);
    const uint8_t *src = reinterpret_cast<const uint8_t *>(ct_host) + (size_t)c0 * ct_client;
    uint32_t *ct_dev = reinterpret_cast<uint32_t *>(reinterpret_cast<uint8_t *>(db->ws_ct) + (size_t)c0 * ct_client);
    uint32_t *o_dev = reinterpret_cast<uint32_t *>(reinterpret_cast<uint8_t *>(db->ws_out) + (size_t)c0 * out_client);
    uint8_t *dst = reinterpret_cast<uint8_t *>(out_host) + (size_t)c0 * out_client;
    if ((e = cudaMemcpyAsync(ct_dev, src, (size_t)bc * ct_client, cudaMemcpyHostToDevice, hp->in)) != cudaSuccess ||
        (e = cudaEventRecord(hp->copied[k], hp->in)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(s, hp->copied[k], 0)) != cudaSuccess)
      return set_cuda_error(e);
    rc = gpir_rowsel_batch(db, bc, ct_dev, o_dev, path, stream);
    if (rc != GPIR_OK) return rc;
    if ((e = cudaEventRecord(hp->computed[k], s)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(hp->out, hp->computed[k], 0)) != cudaSuccess ||
        (e = cudaMemcpyAsync(dst, o_dev, (size_t)bc * out_client, cudaMemcpyDeviceToHost, hp->out)) != cudaSuccess)
      return set_cuda_error(e);
    c0 += bc;
  }
  if ((e = cudaEventRecord(hp->done, hp->out)) != cudaSuccess || (e = cudaStreamWaitEvent(s, hp->done, 0)) != cudaSuccess)
    return set_cuda_error(e);
  return GPIR_OK;
}

int gpir_rowsel_multi(const gpir_job_t *jobs, uint32_t njobs, int path, void *stream) {
  NvtxRange nvtx("gpir_rowsel_multi");
  if (!jobs || njobs == 0) return GPIR_EINVAL;
  for (uint32_t k = 0; k < njobs; ++k) {
    if (!jobs[k].db || !jobs[k].ct || !jobs[k].out || jobs[k].batch == 0 || jobs[k].batch > GPIR_MAX_BATCH)
      return GPIR_EINVAL;
    const gpir_params &a = jobs[0].db->params, &b = jobs[k].db->params;
    if (a.n != b.n || a.num_limbs != b.num_limbs || memcmp(a.primes, b.primes, sizeof(a.primes)) != 0)
      return GPIR_EINVAL;
    if (((uintptr_t)jobs[k].ct & 15u) || ((uintptr_t)jobs[k].out & 15u)) return GPIR_EINVAL;
  }
  // no output may overlap any ciphertext or output buffer of the call
  for (uint32_t k = 0; k < njobs; ++k) {
    const gpir_params &prm = jobs[k].db->params;
    const size_t poly = (size_t)2 * prm.num_limbs * prm.n * 4;
    const uintptr_t o0 = (uintptr_t)jobs[k].out, o1 = o0 + (size_t)jobs[k].batch * jobs[k].db->d1 * poly;
    for (uint32_t k2 = 0; k2 < njobs; ++k2) {
      const uintptr_t c0 = (uintptr_t)jobs[k2].ct, c1 = c0 + (size_t)jobs[k2].batch * jobs[k2].db->d0 * poly;
      if (c0 < o1 && o0 < c1) return GPIR_EINVAL;
      if (k2 == k) continue;
      const uintptr_t p0 = (uintptr_t)jobs[k2].out, p1 = p0 + (size_t)jobs[k2].batch * jobs[k2].db->d1 * poly;
      if (p0 < o1 && o0 < p1) return GPIR_EINVAL;
    }
  }
  if (debug_checks())
    for (uint32_t k = 0; k < njobs; ++k) {
      const gpir_params &prm = jobs[k].db->params;
      const uint64_t count = (uint64_t)jobs[k].batch * jobs[k].db->d0 * 2 * prm.num_limbs * prm.n;
      const int rc = check_residues_dev(prm, jobs[k].ct, count, (cudaStream_t)stream);
      if (rc != GPIR_OK) return rc;
    }
  return rowsel_multi_launch(jobs, njobs, path, (cudaStream_t)stream);
}

int gpir_sync(void *stream, uint32_t timeout_ms) {
  cudaStream_t s = (cudaStream_t)stream;
  auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t e = cudaStreamQuery(s);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) return set_cuda_error(e);
    if (timeout_ms && std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(timeout_ms))
      return GPIR_ETIMEOUT;
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  unsigned int *w = device_error_word();
  if (!w) return GPIR_ECUDA;
  unsigned int h = 0;
  cudaError_t e = cudaMemcpy(&h, w, sizeof(h), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return set_cuda_error(e);
  if (h != 0) {
    unsigned int zero = 0;
    cudaMemcpy(w, &zero, sizeof(zero), cudaMemcpyHostToDevice);
    return GPIR_ETIMEOUT;
  }
  return GPIR_OK;
}

int gpir_selftest_bounded_wait(void *stream) {
  unsigned int *w = device_error_word();
  if (!w) return GPIR_ECUDA;
  selftest_wait_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(w);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GPIR_OK : set_cuda_error(e);
}

int gpir_set_debug(int on) {
  const int prev = debug_checks() ? 1 : 0;
  g_debug.store(on ? 1 : 0);
  return prev;
}

long gpir_set_fail_alloc(long n) {
  fail_alloc_init();
  return g_fail_alloc.exchange(n > 0 ? n : 0);
}

int gpir_num_variants(int path) { return num_variants(path); }

int gpir_selected_variant(const gpir_db_t *db, uint32_t batch, int path) {
  if (!db) return -1;
  std::lock_guard<std::mutex> lk(*db->mu);
  auto it = db->variants->find({path, batch});
  return it == db->variants->end() ? -1 : it->second;
}

int gpir_set_variant(const gpir_db_t *db, uint32_t batch, int path, int variant) {
  if (!db || variant < 0 || variant >= num_variants(path)) return GPIR_EINVAL;
  std::lock_guard<std::mutex> lk(*db->mu);
  try {
    (*db->variants)[{path, batch}] = variant;
  } catch (...) {   // no exception crosses the C ABI
    return GPIR_ENOMEM;
  }
  return GPIR_OK;
}

int gpir_autotune(const gpir_db_t *db, uint32_t batch, const uint32_t *ct_dev, uint32_t *out_dev, int path,
                  void *stream, int *variant_out) {
  if (!db || !ct_dev || !out_dev || batch == 0 || batch > GPIR_MAX_BATCH) return GPIR_EINVAL;
  int paths[3], np = 0;
  if (path == GPIR_PATH_AUTO) {
    for (int p : {GPIR_PATH_CUDACORE, GPIR_PATH_IMMA, GPIR_PATH_TC})
      if (db->path_mask & p) paths[np++] = p;
  } else {
    int p = resolve_path(db, path, batch);
    if (p == -1) return GPIR_EINVAL;
    if (p == -2) return GPIR_ENOTSUP;
    paths[np++] = p;
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return GPIR_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return GPIR_ECUDA;
  }
  int best_path = -1, best_v = -1;
  float best_ms = 1e30f;
  for (int pi = 0; pi < np; ++pi) {
    const int p = paths[pi];
    int pv = -1;
    float pv_ms = 1e30f;
    const int nv = num_variants(p);
    for (int v = 0; v < nv; ++v) {
      int rc = dispatch(db, batch, ct_dev, out_dev, p, v, s);  // warm-up (and support check)
      if (rc != GPIR_OK) continue;
      float tot = 0.f;
      bool okv = true;
      for (int rep = 0; rep < 3 && okv; ++rep) {
        cudaEventRecord(e0, s);
        rc = dispatch(db, batch, ct_dev, out_dev, p, v, s);
        cudaEventRecord(e1, s);
        if (rc != GPIR_OK || cudaEventSynchronize(e1) != cudaSuccess) {
          okv = false;
          break;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        tot += ms;
      }
      if (okv && tot < pv_ms) {
        pv_ms = tot;
        pv = v;
      }
    }
    if (pv >= 0) {
      std::lock_guard<std::mutex> lk(*db->mu);
      try {
        (*db->variants)[{p, batch}] = pv;
      } catch (...) {
        return GPIR_ENOMEM;
      }
    }
    if (pv >= 0 && pv_ms < best_ms) {
      best_ms = pv_ms;
      best_path = p;
      best_v = pv;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best_path < 0) return GPIR_ENOTSUP;
  if (path == GPIR_PATH_AUTO) {
    std::lock_guard<std::mutex> lk(*db->mu);
    try {
      (*db->variants)[{GPIR_PATH_AUTO, batch}] = best_path;
    } catch (...) {
      return GPIR_ENOMEM;
    }
  }
  if (variant_out) *variant_out = best_v;
  return GPIR_OK;
}

int gpir_selected_path(const gpir_db_t *db, uint32_t batch) {
  if (!db) return -1;
  return resolve_path(db, GPIR_PATH_AUTO, batch);
}

int gpir_fill_uniform(uint32_t *dst_dev, uint64_t count, uint64_t start, uint64_t seed, uint64_t tag,
                      const gpir_params_t *params, uint64_t inner, void *stream) {
  if (!dst_dev || !params || inner == 0) return GPIR_EINVAL;
  if (count == 0) return GPIR_OK;
  const uint64_t key = host_mix((seed * 0x9E3779B97F4A7C15ull) ^ ((tag + 1) * 0xD1B54A32D192ED03ull));
  fill_uniform_kernel<<<sm_count() * 8, 256, 0, (cudaStream_t)stream>>>(dst_dev, count, start, key, inner,
                                                                         params->num_limbs, params->limbs);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GPIR_OK : set_cuda_error(e);
}

}  // extern "C"
