// FP32 column-transform kernels and the vertical solve.
#include "persist.cuh"
#include "pickers.h"
#include "tma.cuh"

namespace mp {
template <> KernelFn pick_k_fwd_cols<float>(int n) {
    if (KernelFn f = pick_f32_ext(kFwdCols, n)) return f;
    MP_PICK_F32(k_fwd_cols, (k_fwd_cols<float, 0>))
}
template <> KernelFn pick_k_inv_cols<float>(int n) {
    if (KernelFn f = pick_f32_ext(kInvCols, n)) return f;
    MP_PICK_F32(k_inv_cols, (k_inv_cols<float, 0>))
}
template <> KernelFn pick_fwd_cols_persist<float>(int n) { MP_PICK_F32(k_cols_persist, nullptr, , false) }
template <> KernelFn pick_inv_cols_persist<float>(int n) { MP_PICK_F32(k_cols_persist, nullptr, , true) }
template <> KernelFn pick_tridiag<float>() { return k_tridiag<float>; }
template <> ColsTmaFn pick_cols_tma<float>(int n, bool inv) {
    if (inv) { MP_PICK_F32(k_cols_tma, nullptr, , true) }
    MP_PICK_F32(k_cols_tma, nullptr, , false)
}
}  // namespace mp
