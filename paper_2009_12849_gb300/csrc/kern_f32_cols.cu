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
KernelFn pick_cols_square_f32(int ny, int nxp, int tw, int bs, bool inv) {
#define MP_SQ(N, NXP, TW)                                                                    \
    if (ny == N && nxp == NXP && tw == TW && bs == ColPitch<N>::value)                      \
        return inv ? (KernelFn)k_inv_cols<float, N, false, NXP, TW> : (KernelFn)k_fwd_cols<float, N, NXP, TW>;
    MP_SQ(1024, 516, 8)
    MP_SQ(512, 260, 16)
    MP_SQ(256, 132, 32)
#undef MP_SQ
    return nullptr;
}
template <> ColsTmaFn pick_cols_tma<float>(int n, bool inv) {
    if (inv) { MP_PICK_F32(k_cols_tma, nullptr, , true) }
    MP_PICK_F32(k_cols_tma, nullptr, , false)
}
}  // namespace mp
