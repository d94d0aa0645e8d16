// batch_bricks.cu -- the batched form's brick-sparse-grid kernels with shared-memory records
// (batch_kernels.cuh), dispatched from batch.cu.
#include "batch_kernels.cuh"

namespace cow {

COW_FOR_STORAGE(COW_INST_BATCH_SMEM, kBrickBit)

}  // namespace cow
