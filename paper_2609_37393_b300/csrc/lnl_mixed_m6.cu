// FP32-mixed kernels instantiated for points with up to 6 modes.
#include "lnl_mixed_impl.cuh"

namespace rift {
RIFT_INSTANTIATE_MIXED(6)
}  // namespace rift
