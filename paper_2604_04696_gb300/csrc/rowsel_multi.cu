// Multi-job RowSel (placeholder: one launch per job).
#include "internal.h"
namespace gpir {
int dispatch(const gpir_db *db, uint32_t batch, const uint32_t *ct, uint32_t *out, int path, int variant,
             cudaStream_t s);
int rowsel_multi_launch(const gpir_job_t *jobs, uint32_t njobs, int path, cudaStream_t stream) {
  for (uint32_t k = 0; k < njobs; ++k) {
    int p = path == GPIR_PATH_AUTO ? GPIR_PATH_CUDACORE : path;
    int rc = dispatch(jobs[k].db, jobs[k].batch, jobs[k].ct, jobs[k].out, p,
                      rowsel_cc_default_variant(jobs[k].batch, jobs[k].db->d0, jobs[k].db->d1), stream);
    if (rc) return rc;
  }
  return GPIR_OK;
}
}  // namespace gpir
