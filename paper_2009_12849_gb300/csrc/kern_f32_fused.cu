// FP32 fused persistent kernels (opt-in).
#include "fused.cuh"
#include "pickers.h"

namespace mp {
template <> KernelFn pick_fwd_fused<float>(int n) { MP_PICK_F32(k_fwd_fused, nullptr) }
template <> KernelFn pick_inv_fused<float>(int n) { MP_PICK_F32(k_inv_fused, nullptr) }
}  // namespace mp
