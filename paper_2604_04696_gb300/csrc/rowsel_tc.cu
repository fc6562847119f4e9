// RowSel on tcgen05 tensor cores (placeholder until the kernel lands).
#include "internal.h"
namespace gpir {
int rowsel_tc_prepare(gpir_db *, cudaStream_t) { return GPIR_ENOTSUP; }
int rowsel_tc_num_variants() { return 0; }
int rowsel_tc_default_variant(uint32_t, uint32_t, uint32_t) { return 0; }
int rowsel_tc_launch(const gpir_db *, uint32_t, const uint32_t *, uint32_t *, int, cudaStream_t) {
  return GPIR_ENOTSUP;
}
}  // namespace gpir
