// ntt_matrix.cu -- matrix-form (tensor-core) column-DFT path.
#include "ntt_plan.h"

namespace gb300ntt {

bool matrix_path_available(ntt_plan) { return false; }
ntt_status enqueue_matrix_transform(ntt_plan, int, const void *, void *, cudaStream_t) { return NTT_ERR_UNSUPPORTED; }
uint32_t matrix_launches(ntt_plan) { return 0; }
void release_matrix_resources(ntt_plan) {}

}  // namespace gb300ntt
