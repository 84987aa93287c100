// FP32 row-transform kernels (forward divergence + x-transform, inverse
// x-transform + correction).
#include "pickers.h"

namespace mp {
template <> KernelFn pick_k_fwd_rows<float>(int n) {
    if (KernelFn f = pick_f32_ext(kFwdRows, n)) return f;
    MP_PICK_F32(k_fwd_rows, (k_fwd_rows<float, 0>))
}
template <> KernelFn pick_k_inv_rows<float>(int n) {
    if (KernelFn f = pick_f32_ext(kInvRows, n)) return f;
    MP_PICK_F32(k_inv_rows, (k_inv_rows<float, 0>))
}
}  // namespace mp
