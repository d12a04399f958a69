// FP32-mixed kernels instantiated for points with up to 10 modes (and the
// composite response's mixed kernel for its mode bucket).
#include "lnl_mixed_impl.cuh"
#include "comp_mixed_impl.cuh"

namespace rift {
RIFT_INSTANTIATE_MIXED(10)
RIFT_INSTANTIATE_COMP_MIXED(10)
}  // namespace rift
