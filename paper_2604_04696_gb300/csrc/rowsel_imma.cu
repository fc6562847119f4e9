// RowSel on INT8 tensor cores (placeholder until the IMMA kernel lands).
#include "internal.h"
namespace gpir {
int rowsel_imma_num_variants() { return 0; }
int rowsel_imma_default_variant(uint32_t, uint32_t, uint32_t) { return 0; }
int rowsel_imma_launch(const gpir_db *, uint32_t, const uint32_t *, uint32_t *, int, cudaStream_t) {
  return GPIR_ENOTSUP;
}
}  // namespace gpir
