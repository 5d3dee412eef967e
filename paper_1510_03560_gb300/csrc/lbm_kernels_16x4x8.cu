// The FP32 step kernels (lbm_step.cuh) for blocks of 16 x 4 x 8 cells.
#define LBM_BLOCK_X 16
#define LBM_BLOCK_Y 4
#define LBM_BLOCK_Z 8
#include "lbm_step.cuh"

namespace lbm {
const StorageOps *storage_ops_fp32_16x4x8() { return Launch<LBM_STORAGE_FP32>::ops(); }
}  // namespace lbm
