// The BF16 deviation storage form of the step kernels (lbm_step.cuh).
#include "lbm_step.cuh"

namespace lbm {
const StorageOps *storage_ops_bf16() { return Launch<LBM_STORAGE_BF16>::ops(); }
}  // namespace lbm
