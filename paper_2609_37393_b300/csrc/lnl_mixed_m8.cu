// FP32-mixed kernels instantiated for points with up to 8 modes.
#include "lnl_mixed_impl.cuh"

namespace rift {
RIFT_INSTANTIATE_MIXED(8)
}  // namespace rift
