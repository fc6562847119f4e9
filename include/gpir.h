/*
 * gpir.h -- C ABI of the GB300 RowSel library (libgpir.so).
 *
 * RowSel is the encrypted row-selection step of batched lattice PIR as the
 * GPIR paper (arXiv 2604.04696) defines it: each client's D0 NTT-domain RLWE
 * selection ciphertexts are multiplied point-wise with the D0 x D1 NTT-form
 * plaintext database and summed over the rows (Sec. 2.2, "RowSel"). Written
 * per NTT point p this is the GEMM of Sec. 2.3,
 *     M_out[p, m, n] = sum_k M_in0[p, m, k] * M_in1[p, k, n]   (mod q_l),
 * with m = (client, polynomial) of extent 2*batch (Sec. 5.1.1), k the D0 rows,
 * n the D1 columns, and p = (limb l, slot t) over L RNS limbs of N slots
 * (Sec. 2.4.1: "4N points" for four limbs).
 *
 * Conventions for every call:
 *  - Residues are canonical uint32 values in [0, q_l).
 *  - Device pointers are CUDA device addresses of the current device; host
 *    pointers are ordinary (preferably pinned) host memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Calls that take a stream are asynchronous on it unless stated otherwise.
 *  - The caller owns ciphertext and output buffers; the library owns the
 *    params object, its device copy of each database and any workspace.
 *  - Every call returns GPIR_OK (0) or a negative gpir error code; nothing
 *    aborts the process. gpir_strerror() names the code.
 *
 * Array layouts (row-major, last index fastest; the paper's p-major layout of
 * Sec. 2.3 / Sec. 5.1.2, every polynomial's N points contiguous):
 *    db  [D0][D1][L][N]          DB[i][j], NTT form           (Sec. 2.2)
 *    ct  [B][D0][2][L][N]        client c, selection ct i, polynomial r
 *    out [B][D1][2][L][N]        client c, output ct j, polynomial r
 */
#ifndef GPIR_H
#define GPIR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------- */
#define GPIR_OK          0
#define GPIR_EINVAL     -1  /* bad argument: shape, pointer, params, path   */
#define GPIR_ERANGE     -2  /* a database residue >= its limb's prime       */
#define GPIR_ENOMEM     -3  /* device or host allocation failed             */
#define GPIR_ECUDA      -4  /* a CUDA runtime call failed                   */
#define GPIR_ETIMEOUT   -5  /* a bounded wait (host or device) expired      */
#define GPIR_ENOTSUP    -6  /* path not prepared for this database / device */
#define GPIR_ETOOBIG    -7  /* problem exceeds a fixed buffer or index size */

/* ---- compute paths (also usable as a bit mask at upload) ---------------- */
#define GPIR_PATH_AUTO      0  /* fastest prepared path for the shape        */
#define GPIR_PATH_CUDACORE  1  /* 32x32->64-bit IMAD products, CUDA cores     */
#define GPIR_PATH_IMMA      2  /* INT8 tensor cores (mma.sync u8), byte limbs */
#define GPIR_PATH_TC        4  /* tcgen05 fp16 tensor cores, signed 8-bit
                                  digits, exact fp32 partial sums            */
#define GPIR_PATH_ALL       7

/* Limits enforced by gpir_params_create. */
#define GPIR_MAX_LIMBS      8
#define GPIR_MIN_N          4
#define GPIR_MAX_N      65536
#define GPIR_MAX_PRIME_BITS 28   /* q < 2^28: every accumulator bound below
                                    is proven for this width               */
#define GPIR_MAX_BATCH (1u << 30) /* clients per RowSel call (2*batch rows must
                                    fit 32-bit row indices): GPIR_EINVAL above */

typedef struct gpir_params gpir_params_t;
typedef struct gpir_db gpir_db_t;

/* One RowSel problem of a multi-job launch: `batch` clients against `db`. */
typedef struct gpir_job {
  const gpir_db_t *db;
  uint32_t batch;          /* B >= 1                                         */
  uint32_t reserved;
  const uint32_t *ct;      /* device, [B][D0][2][L][N]                       */
  uint32_t *out;           /* device, [B][D1][2][L][N]                       */
} gpir_job_t;

/* Ring and RNS parameters (Sec. 2.4.1): ring degree n (power of two in
 * [GPIR_MIN_N, GPIR_MAX_N]) and num_limbs primes, each prime, below
 * 2^GPIR_MAX_PRIME_BITS and equal to 1 mod 2n (NTT-friendly). The primes are
 * copied. Returns GPIR_EINVAL if any check fails. Host-only, synchronous. */
int gpir_params_create(uint32_t n, uint32_t num_limbs, const uint32_t *primes,
                       gpir_params_t **out);
int gpir_params_destroy(gpir_params_t *params);

/* Make an NTT-form database resident on the current device (Sec. 2.2: DB is
 * D0 x D1 plaintext polynomials, stored after the NTT). `db_ntt` is
 * [D0][D1][L][N] uint32, on the device if db_on_device != 0, else on the
 * host. `path_mask` (GPIR_PATH_* bits, 0 = all) selects which packed layouts
 * are built; each path reads only its own layout. Every residue is checked
 * against its limb's prime: GPIR_ERANGE if any is >= q_l. The database is
 * prepared once, before queries (the paper transposes its DB offline, Sec.
 * 5.2.1), so this call synchronizes `stream`. The caller keeps ownership of
 * `db_ntt`; the handle owns the device copies until gpir_db_free. */
int gpir_db_upload(const gpir_params_t *params, uint32_t d0, uint32_t d1,
                   const uint32_t *db_ntt, int db_on_device, uint32_t path_mask,
                   void *stream, gpir_db_t **out);
int gpir_db_free(gpir_db_t *db);

/* Device bytes held by the database handle (all packed layouts). */
size_t gpir_db_device_bytes(const gpir_db_t *db);

/* Batched RowSel (Sec. 2.2 and Sec. 5.1.1) on `stream`:
 *   out[c][j][r][l][t] = sum_{i<D0} ct[c][i][r][l][t] * db[i][j][l][t] mod q_l
 * for every client c < batch, output ct j < D1, polynomial r < 2, limb l and
 * slot t. `ct_dev` and `out_dev` are device buffers in the layouts above and
 * must not overlap. Inputs must be canonical residues (< q_l): this is a
 * precondition, checked only with the debug checks on (gpir_set_debug),
 * because a check adds a pass over the ciphertext stream. Results are
 * canonical and identical for every path.
 * GPIR_ENOTSUP if `path` was not prepared at upload; GPIR_ETOOBIG if a
 * tensor-core launch would number 2^32 or more work units (never for inputs
 * that fit in device memory). The tensor-core path
 * keeps its per-batch digit tiles (2x the ciphertext bytes) in a workspace
 * owned by the library per (device, stream), grown on demand; calls on
 * different streams may overlap. Asynchronous. */
int gpir_rowsel_batch(const gpir_db_t *db, uint32_t batch, const uint32_t *ct_dev,
                      uint32_t *out_dev, int path, void *stream);

/* Same computation with HOST buffers: copies ct host->device, runs RowSel and
 * copies out device->host, through a device workspace the handle owns (grown
 * on demand; GPIR_ENOMEM if that fails). Batches of 16 or more go in client
 * chunks so that uploads, RowSel and downloads overlap (two internal copy
 * streams per device, ordered after the work already in `stream`; `stream`
 * waits on the last download). Returns after enqueueing; the host output is
 * valid after gpir_sync(stream). For full copy speed the host buffers should
 * be pinned. Not safe to call concurrently on the same handle from several
 * streams. */
int gpir_rowsel_batch_host(const gpir_db_t *db, uint32_t batch, const uint32_t *ct_host,
                           uint32_t *out_host, int path, void *stream);

/* Several RowSel problems at once (Sec. 5.1.1's batched GEMMs over a list of
 * jobs): different databases, uneven D0 / D1 and batch sizes. On the
 * tensor-core path one job runs the kernel tuned for its batch; the entries,
 * work units and ingest tasks of up to 8 jobs are numbered into one index
 * space and processed by ONE persistent launch of the tensor-memory kernel
 * (one CTA per SM, work claimed in index order); larger lists use one launch
 * per 8 jobs (databases uploaded without that kernel's digit tiles: the
 * two-pass kernels). CUDA-core and IMMA paths use one launch per job.
 * GPIR_PATH_AUTO runs each job on the path gpir_rowsel_batch would choose for
 * its batch (the autotuned one, else tensor cores from batch 8), the
 * tensor-core jobs together. All jobs must share the same params (N, L,
 * primes) and every job's
 * ct / out must not overlap any other buffer of the call. The tensor-core
 * workspace for the call is grown on demand (not while the stream is being
 * captured: GPIR_ENOMEM then); it is per (device, stream), so calls on
 * different streams may run concurrently. Asynchronous. */
int gpir_rowsel_multi(const gpir_job_t *jobs, uint32_t njobs, int path, void *stream);

/* CUDA-graph plan of one gpir_rowsel_multi call (the paper replays its
 * fine-grained launches from CUDA graphs, Sec. 5.2.2). Create runs the call
 * once eagerly on `stream` (sizing workspaces; synchronizes), then captures
 * it; launch replays it on any stream. The job list (buffers, batch sizes)
 * is fixed at creation: refill the same ct buffers and replay. `stream` must
 * not be the legacy default stream; create waits for the work already on it.
 * Each graph owns its tensor-core workspace (allocated at create, outside the
 * capture, freed by destroy), so later calls on any stream cannot disturb it;
 * two replays of the SAME graph must not overlap (they share that workspace
 * and the job's buffers). GPIR_ENOMEM if the workspace cannot be allocated. */
typedef struct gpir_graph gpir_graph_t;
int gpir_graph_create(const gpir_job_t *jobs, uint32_t njobs, int path, void *stream,
                      gpir_graph_t **out);
int gpir_graph_launch(gpir_graph_t *graph, void *stream);
int gpir_graph_destroy(gpir_graph_t *graph);

/* Bounded synchronization (no counterpart in the paper; the library's own
 * failure reporting): wait for `stream` for at most timeout_ms milliseconds
 * (0 = no limit), then read and clear the device error word. GPIR_ETIMEOUT if
 * the stream is still busy, or if a kernel of this library reported that one
 * of its bounded device-side waits expired; GPIR_ECUDA if the stream reported
 * an error. The error word is one per DEVICE, not per stream: an expiry
 * raised by a kernel on another stream of the device is reported (and
 * cleared) by whichever gpir_sync reads it first, and one still running on
 * another stream is not seen yet. Callers that run several streams should
 * sync after all of them have drained when they need the status of each. */
int gpir_sync(void *stream, uint32_t timeout_ms);

/* Debug checks (off by default; on when the environment variable GPIR_DEBUG
 * is a nonzero number when the library first needs the setting, or after
 * gpir_set_debug(1)). While on, gpir_rowsel_batch, gpir_rowsel_batch_noalloc,
 * gpir_rowsel_multi and gpir_rowsel_batch_host first check that every
 * ciphertext residue is below its limb's prime and return GPIR_ERANGE,
 * computing nothing, if one is not. The device-side check synchronizes
 * `stream` (so these calls are not asynchronous and cannot be captured into a
 * CUDA graph while it is on); the host entry checks its host buffer on the
 * CPU. Returns the previous setting (0 or 1). */
int gpir_set_debug(int on);

/* Self-test of the device-side failure path. Enqueues on `stream` one kernel
 * whose single thread waits, through the same bounded mbarrier wait the RowSel
 * kernels use, on a barrier that nothing ever arrives on. The wait gives up
 * after its limit (2 s), records the expiry in the device error word and the
 * kernel returns normally: no trap, no hang, the context stays usable. A
 * following gpir_sync(stream, t) with t > 2000 then returns GPIR_ETIMEOUT and
 * clears the word, so the sync after it returns GPIR_OK. Asynchronous;
 * GPIR_ECUDA if the launch fails. */
int gpir_selftest_bounded_wait(void *stream);

/* Autotuner: time every compiled tile variant of `path` (three runs each,
 * after a warm-up) for `batch` clients against this database, using the
 * caller's device buffers ct_dev / out_dev (layouts as in gpir_rowsel_batch;
 * out_dev is overwritten), and remember the fastest for (path, batch); later
 * calls with that batch use it. With path == GPIR_PATH_AUTO every prepared
 * path is tuned and the fastest path is also remembered, so later
 * GPIR_PATH_AUTO calls with that batch use it. Synchronizes `stream`.
 * `*variant_out` (may be NULL) receives the chosen variant id. */
int gpir_autotune(const gpir_db_t *db, uint32_t batch, const uint32_t *ct_dev,
                  uint32_t *out_dev, int path, void *stream, int *variant_out);

/* Allocation-failure injection, for tests of the out-of-memory paths (no
 * counterpart in the paper). With n > 0 the n-th device allocation the library
 * makes from now on (1 = the next one) fails as if the device were out of
 * memory -- the call that made it returns GPIR_ENOMEM and leaves its handle as
 * it was -- and the injection then disarms itself; n <= 0 disarms it. The
 * environment variable GPIR_FAIL_ALLOC=n arms it when the library first
 * allocates. Returns the previous countdown (0 = off). Host-only. */
long gpir_set_fail_alloc(long n);

/* Number of kernel variants compiled for `path` and the id in use for a
 * shape (-1 if none chosen yet). Host-only. */
int gpir_num_variants(int path);
/* The path GPIR_PATH_AUTO resolves to for `batch` clients (tuned, else the
 * static rule: tensor cores from 8 clients up when prepared). Host-only. */
int gpir_selected_path(const gpir_db_t *db, uint32_t batch);
int gpir_selected_variant(const gpir_db_t *db, uint32_t batch, int path);
/* Force a variant for (path, batch, D0, D1) of this database (testing). */
int gpir_set_variant(const gpir_db_t *db, uint32_t batch, int path, int variant);

/* Fill `count` uint32 residues on the device: element f gets
 * SplitMix64-stream value (f + start) of (seed, tag) mod q_l, with
 * l = ((f + start) / inner) % num_limbs -- the synthetic-input generator,
 * identical to the host one. Asynchronous. */
int gpir_fill_uniform(uint32_t *dst_dev, uint64_t count, uint64_t start, uint64_t seed,
                      uint64_t tag, const gpir_params_t *params, uint64_t inner,
                      void *stream);

/* Allocation-free RowSel (no counterpart in the paper: an interface for
 * callers that cannot allocate device memory while they run, such as code
 * running under a CUDA stream capture, or services whose device-memory budget
 * is fixed at start-up and that must not call the allocator on their request
 * path). Same result as gpir_rowsel_batch(db, batch, ct_dev, out_dev,
 * GPIR_PATH_TC, stream), but the tensor-core path's per-batch digit-tile
 * workspace lives in a fixed device array of GPIR_NOALLOC_SCRATCH_BYTES
 * compiled into the library instead of memory from cudaMalloc; the call
 * allocates nothing. The caller passes the input and output buffers as usual.
 *  - The workspace needed is L*N * ceil(2*batch/32) * ceil(D0/64) * 16 KiB;
 *    larger problems are rejected with GPIR_ETOOBIG before anything is
 *    enqueued.
 *  - The database must have been uploaded with the GPIR_PATH_TC bit
 *    (GPIR_ENOTSUP otherwise) on the current device.
 *  - The first call on each device looks up the array's device address and
 *    sets kernel attributes (no allocation); make that first call before any
 *    stream capture that will contain later calls.
 *  - All calls share the one array, which keeps the last call's contents:
 *    calls whose work overlaps on the GPU (different streams, or different
 *    host threads) race on it and must be serialized by the caller.
 *  - Every device that loads the library holds the array until the process
 *    exits. Asynchronous on `stream`. */
#define GPIR_NOALLOC_SCRATCH_BYTES (64u << 20)
int gpir_rowsel_batch_noalloc(const gpir_db_t *db, uint32_t batch, const uint32_t *ct_dev,
                              uint32_t *out_dev, void *stream);

/* Tracing (the paper reports per-kernel device times, Sec. 5.1.2): with
 * on = 1, each kernel the library launches is bracketed by CUDA events on its
 * launch stream; on = 2 also runs the tensor-core kernels' role-counting
 * instantiations (slower: for gpir_trace_counters); on = 0 turns tracing off
 * (the default; a disabled trace costs nothing); other values are
 * GPIR_EINVAL. gpir_trace_read waits for the recorded launches, copies up to
 * max_records (name, milliseconds) pairs in launch order, sets *count, and
 * clears the log. */
typedef struct gpir_trace_record {
  char name[32];
  float ms;
} gpir_trace_record_t;
int gpir_trace_enable(int on);
int gpir_trace_read(gpir_trace_record_t *out, uint32_t max_records, uint32_t *count);
/* Wait-cycle counters of the last fused or cluster tensor-core launch made
 * while tracing was at level 2 (SM clock cycles summed over CTAs, one counting thread
 * per role): [0] producer waiting for ingested tiles, [1] producer waiting for
 * a free stage, [2] MMA waiting for operands, [3] MMA waiting for the
 * epilogue, [4] epilogue waiting for MMAs, [5] epilogue waiting for the store
 * warp, [6] ingest waiting for a ring entry (cluster kernel: for a free stage),
 * [7] ingest waiting for its TMA box, [8] ingest converting, [9] cluster
 * ingest waiting for its slab copies to leave staging, [10] cluster ingest
 * issuing slab copies, [11] kernel cycles per CTA; the tensor-memory
 * kernel's counters are listed with its binding. Tracing at level 2 makes that
 * launch synchronous. */
int gpir_trace_counters(unsigned long long *out, uint32_t max_counters, uint32_t *count);

/* ColTor, the column tournament after RowSel (Sec. 2.2, "ColTor"), with the
 * external product of Sec. 2.5.1. For every client c < batch, log2(d1) stages
 * halve its d1 ciphertexts (d1 a power of two, at least 2): stage s pairs the
 * stage's inputs (2k, 2k+1) and keeps
 *     ct_{2k} + RGSW_s [x] (ct_{2k+1} - ct_{2k}),
 * so the result selects, bit by bit from the least significant, the column
 * the RGSW ciphertexts encrypt. The external product takes the inverse NTT of
 * both polynomials, rebuilds each coefficient from its limbs (CRT) centred to
 * (-Q/2, Q/2], splits it into ell balanced base-2^22 digits (ell =
 * gpir_coltor_gadget_digits), takes the forward NTT of the 2 ell digit
 * polynomials and multiplies-accumulates them with the RGSW rows
 * (row p ell + i multiplies digit i of polynomial p).
 *   ct_dev    device, [B][d1][2][L][N]  (gpir_rowsel_batch's output layout)
 *   rgsw_dev  device, [B][log2 d1][2 ell][2][L][N]
 *   out_dev   device, [B][2][L][N]
 * Everything is in NTT form A_s = sum_j a_j psi^((2s+1) j) mod q_l, natural
 * slot order, psi = g^((q_l - 1) / 2N) with g the smallest generator of the
 * multiplicative group mod q_l. Limits: L <= 2 and 16 <= N <= 4096, else
 * GPIR_ENOTSUP. Twiddle tables are built once per (device, N, primes); the
 * library keeps a workspace per (device, stream) for the intermediate stages
 * (d1/2 + d1/4 ciphertexts per client). ct_dev is not modified; out_dev must
 * not overlap it (GPIR_EINVAL). Argument errors are returned before any CUDA
 * call. Asynchronous. */
int gpir_coltor(const gpir_params_t *params, uint32_t batch, uint32_t d1, const uint32_t *ct_dev,
                const uint32_t *rgsw_dev, uint32_t *out_dev, void *stream);
/* ell, the number of base-2^22 digits of the external product: the smallest
 * count with 2^(22 ell) >= Q (3 for two 28-bit limbs). GPIR_EINVAL for NULL. */
int gpir_coltor_gadget_digits(const gpir_params_t *params);

/* ExpandQuery, the query-expansion tree before RowSel (Sec. 2.2,
 * "ExpandQuery"), with the homomorphic substitution Subs of Sec. 2.5.1. For
 * every client c < batch, `stages` = J stages turn its query ciphertext into
 * 2^J ciphertexts, of which the first n_out (1 <= n_out <= 2^J) are written.
 * Stage j maps the list [c_0 .. c_{2^j - 1}] to a list twice as long: node k
 * computes t = Subs(c_k, N/2^j + 1, evk_j) and writes c_k + t at index k and
 * X^(-2^j) (c_k - t) at index k + 2^j. Subs(ct = (a, b), k) applies X -> X^k
 * to a and b and switches keys with Dcp on the substituted a (inverse NTT,
 * CRT centred to (-Q/2, Q/2], ell balanced base-2^22 digits as in
 * gpir_coltor, forward NTT): t = (sum_i d_i (.) evk[i][0],
 * tau(b) + sum_i d_i (.) evk[i][1]). If the query encrypts m(X), output r
 * encrypts 2^J sum_i m_{2^J i + r} X^(2^J i).
 *   query_dev device, [B][2][L][N]
 *   evk_dev   device, [B][J][ell][2][L][N] (may be NULL when J = 0)
 *   out_dev   device, [B][n_out][2][L][N]; must not overlap query_dev. The
 *             tree runs in place in it: no other workspace.
 * NTT form and limits as gpir_coltor; J <= log2 N (else GPIR_EINVAL: X^k with
 * k = N/2^j + 1 is an automorphism only for j < log2 N). J = 0 copies the
 * query. query_dev and evk_dev are not modified. Argument errors are returned
 * before any CUDA call. Asynchronous. */
int gpir_expand_query(const gpir_params_t *params, uint32_t batch, uint32_t stages, uint32_t n_out,
                      const uint32_t *query_dev, const uint32_t *evk_dev, uint32_t *out_dev, void *stream);

/* One server step of the PIR protocol (Sec. 2.2, the three phases) for
 * `batch` clients against `db`, on `stream`:
 *   1. gpir_expand_query: each query ciphertext expands, in `stages` = J
 *      stages (D0 <= 2^J), into the D0 selection ciphertexts, written to sel_dev;
 *   2. gpir_rowsel_batch(db, batch, sel_dev, rows_dev, path): D1 ciphertexts;
 *   3. gpir_coltor over those D1 (a power of two, at least 2): out_dev.
 *   query_dev device, [B][2][L][N]
 *   evk_dev   device, [B][J][ell][2][L][N]
 *   rgsw_dev  device, [B][log2 D1][2 ell][2][L][N]
 *   sel_dev   device, [B][D0][2][L][N]: caller-owned buffer for the expanded ciphertexts
 *   rows_dev  device, [B][D1][2][L][N]: caller-owned buffer for RowSel's output
 *   out_dev   device, [B][2][L][N]
 * No buffer may overlap another. Each phase's limits and workspaces are those
 * of its own call; the first error is returned and later phases are not
 * enqueued. After one call with the same shapes on the same stream (tables,
 * workspaces and kernel attributes then exist), the call allocates nothing and
 * can be captured into a CUDA graph. Asynchronous. */
int gpir_pir_batch(const gpir_db_t *db, uint32_t batch, uint32_t stages, const uint32_t *query_dev,
                   const uint32_t *evk_dev, const uint32_t *rgsw_dev, uint32_t *sel_dev, uint32_t *rows_dev,
                   uint32_t *out_dev, int path, void *stream);

const char *gpir_strerror(int code);
/* Text of the last CUDA runtime error that made a call of this thread return
 * GPIR_ECUDA or GPIR_ENOMEM ("no error" if none). */
const char *gpir_last_cuda_error(void);
/* Library version: major*10000 + minor*100 + patch. */
int gpir_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GPIR_H */
