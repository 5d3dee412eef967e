// The FP32 step kernels (lbm_step.cuh) for blocks of 16 x 8 x 4 cells.
#define LBM_BLOCK_X 16
#define LBM_BLOCK_Y 8
#define LBM_BLOCK_Z 4
#include "lbm_step.cuh"

namespace lbm {
const StorageOps *storage_ops_fp32_16x8x4() { return Launch<LBM_STORAGE_FP32>::ops(); }
}  // namespace lbm
