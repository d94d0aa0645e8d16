// batch_param_bricks.cu -- the batched form's brick-sparse-grid kernels with records in the parameter buffer
// (batch_kernels.cuh), dispatched from batch.cu.
#include "batch_kernels.cuh"

namespace cow {

COW_FOR_STORAGE(COW_INST_BATCH_PARAM, kBrickBit)

}  // namespace cow
