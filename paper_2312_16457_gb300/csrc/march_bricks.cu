// march_bricks.cu -- the brick-sparse-grid variants of the view and ray
// marchers (march_kernels.cuh), dispatched from march.cu.
#include "march_kernels.cuh"

namespace cow {

COW_FOR_STORAGE(COW_INST_MARCH, kBrickBit)

}  // namespace cow
