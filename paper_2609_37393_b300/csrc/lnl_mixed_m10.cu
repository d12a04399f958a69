// FP32-mixed kernels instantiated for points with up to 10 modes.
#include "lnl_mixed_impl.cuh"

namespace rift {
RIFT_INSTANTIATE_MIXED(10)
}  // namespace rift
