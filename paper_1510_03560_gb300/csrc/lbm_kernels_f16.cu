// The FP16 deviation storage form of the step kernels (lbm_step.cuh).
#include "lbm_step.cuh"

namespace lbm {
const StorageOps *storage_ops_fp16() { return Launch<LBM_STORAGE_FP16>::ops(); }
}  // namespace lbm
