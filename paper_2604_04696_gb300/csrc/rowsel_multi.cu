// Several RowSel problems in one call (batching across clients and resident
// databases of uneven D0 / D1, Sec. 5.1.1's batched GEMMs generalised to a
// job list), and CUDA-graph plans of such calls.
//
// Tensor-core path: one job runs the kernel tuned for its batch; several jobs
// have their entries, work units and ingest tasks numbered into one index
// space and run in ONE persistent launch of the tensor-memory kernel, up to 8
// jobs per launch. CUDA-core and IMMA paths: one launch per job.
// GPIR_PATH_AUTO: each job on the path gpir_rowsel_batch would choose for it.
#include <cuda_runtime.h>
#include <string.h>

#include <new>
#include <vector>

#include "internal.h"

namespace gpir {

// Tensor-core jobs of one call: one job runs the kernel tuned for its batch;
// several run in one persistent tensor-memory launch per 8 jobs (databases
// uploaded without its digit tiles: the two-pass kernels).
static int tc_jobs(const gpir_job_t *jobs, uint32_t njobs, cudaStream_t stream) {
  if (njobs == 1)
    return dispatch(jobs[0].db, jobs[0].batch, jobs[0].ct, jobs[0].out, GPIR_PATH_TC,
                    pick_variant(jobs[0].db, jobs[0].batch, GPIR_PATH_TC), stream);
  bool tmem = true;
  for (uint32_t k = 0; k < njobs; ++k) tmem = tmem && jobs[k].db->db_digits12 != nullptr;
  return tmem ? rowsel_tmem_multi(jobs, njobs, stream) : rowsel_tc_multi(jobs, njobs, stream);
}

int rowsel_multi_launch(const gpir_job_t *jobs, uint32_t njobs, int path, cudaStream_t stream) {
  if (path == GPIR_PATH_AUTO) {
    // each job on the path gpir_rowsel_batch would take for it (small batches
    // on the CUDA cores); the tensor-core jobs together
    std::vector<gpir_job_t> tc;
    try {
      tc.reserve(njobs);   // push_back below then never allocates (no exception crosses the C ABI)
    } catch (...) {
      return GPIR_ENOMEM;
    }
    for (uint32_t k = 0; k < njobs; ++k) {
      const int p = resolve_path(jobs[k].db, GPIR_PATH_AUTO, jobs[k].batch);
      if (p < 0) return GPIR_ENOTSUP;
      if (p == GPIR_PATH_TC) {
        tc.push_back(jobs[k]);
        continue;
      }
      const int rc = dispatch(jobs[k].db, jobs[k].batch, jobs[k].ct, jobs[k].out, p,
                              pick_variant(jobs[k].db, jobs[k].batch, p), stream);
      if (rc) return rc;
    }
    return tc.empty() ? GPIR_OK : tc_jobs(tc.data(), (uint32_t)tc.size(), stream);
  }
  for (uint32_t k = 0; k < njobs; ++k)
    if (!(jobs[k].db->path_mask & path)) return GPIR_ENOTSUP;
  if (path == GPIR_PATH_TC) return tc_jobs(jobs, njobs, stream);
  for (uint32_t k = 0; k < njobs; ++k) {
    int rc = dispatch(jobs[k].db, jobs[k].batch, jobs[k].ct, jobs[k].out, path,
                      pick_variant(jobs[k].db, jobs[k].batch, path), stream);
    if (rc) return rc;
  }
  return GPIR_OK;
}

}  // namespace gpir

// A graph owns a private stream: the eager run and the capture both issue on
// it, so the tensor-core workspace the captured kernels address is the one
// kept for that stream, which no other call uses and which lives until
// gpir_graph_destroy. Later calls on the caller's streams (say a larger batch
// that grows their workspaces) cannot free memory the graph replays into.
struct gpir_graph {
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  cudaStream_t own;
};

using namespace gpir;

namespace {
void graph_free(gpir_graph *g) {
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->own) {
    rowsel_tc_release_stream(g->own);
    cudaStreamDestroy(g->own);
  }
  delete g;
}
}  // namespace

extern "C" {

int gpir_graph_create(const gpir_job_t *jobs, uint32_t njobs, int path, void *stream, gpir_graph_t **out) {
  if (!jobs || njobs == 0 || !out || !stream) return GPIR_EINVAL;
  *out = nullptr;
  gpir_graph *g = new (std::nothrow) gpir_graph;
  if (!g) return GPIR_ENOMEM;
  g->graph = nullptr;
  g->exec = nullptr;
  g->own = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&g->own, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    g->own = nullptr;
    graph_free(g);
    return set_cuda_error(e);
  }
  // The eager run sees everything already enqueued on the caller's stream
  // (say the fill of its ciphertext buffers), sizes the graph's own workspace
  // outside the capture and checks the arguments; replays overwrite its results.
  cudaEvent_t ready = nullptr;
  e = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(ready, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(g->own, ready, 0);
  if (ready) cudaEventDestroy(ready);
  if (e != cudaSuccess) {
    graph_free(g);
    return set_cuda_error(e);
  }
  int rc = gpir_rowsel_multi(jobs, njobs, path, g->own);
  if (rc == GPIR_OK) {
    e = cudaStreamSynchronize(g->own);
    if (e != cudaSuccess) rc = set_cuda_error(e);
  }
  if (rc != GPIR_OK) {
    graph_free(g);
    return rc;
  }
  e = cudaStreamBeginCapture(g->own, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    graph_free(g);
    return set_cuda_error(e);
  }
  rc = gpir_rowsel_multi(jobs, njobs, path, g->own);
  e = cudaStreamEndCapture(g->own, &g->graph);
  if (rc != GPIR_OK || e != cudaSuccess) {
    graph_free(g);
    return rc != GPIR_OK ? rc : set_cuda_error(e);
  }
  e = cudaGraphInstantiate(&g->exec, g->graph, 0);
  if (e != cudaSuccess) {
    g->exec = nullptr;
    graph_free(g);
    return set_cuda_error(e);
  }
  *out = g;
  return GPIR_OK;
}

int gpir_graph_launch(gpir_graph_t *g, void *stream) {
  if (!g) return GPIR_EINVAL;
  cudaError_t e = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
  return e == cudaSuccess ? GPIR_OK : set_cuda_error(e);
}

int gpir_graph_destroy(gpir_graph_t *g) {
  if (!g) return GPIR_OK;
  graph_free(g);
  return GPIR_OK;
}

}  // extern "C"
