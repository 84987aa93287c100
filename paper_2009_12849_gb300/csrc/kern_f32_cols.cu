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
KernelFn pick_cols_square_f32(int ny, int nxp, int tw, int bs, bool inv, int e) {
#define MP_SQ(N, NXP, TW, E)                                                                           \
    if (ny == N && nxp == NXP && tw == TW && e == E && bs == ColPitch<N>::value)                      \
        return inv ? (KernelFn)k_inv_cols<float, N, false, NXP, TW, E> : (KernelFn)k_fwd_cols<float, N, NXP, TW, E>;
    // the default schedule (E = 32) with the default tiles (256 threads)
    MP_SQ(1024, 516, 8, 32)
    MP_SQ(512, 260, 16, 32)
    MP_SQ(256, 132, 32, 32)
    MP_SQ(192, 100, 32, 32)
    MP_SQ(128, 68, 32, 32)
    MP_SQ(96, 52, 32, 32)
    MP_SQ(64, 36, 32, 32)
    // the E = 16 schedule with 256-thread tiles
    MP_SQ(1024, 516, 4, 16)
    MP_SQ(512, 260, 8, 16)
    MP_SQ(256, 132, 16, 16)
#undef MP_SQ
    return nullptr;
}
template <> ColsTmaFn pick_cols_tma<float>(int n, bool inv) {
    if (inv) { MP_PICK_F32(k_cols_tma, nullptr, , true) }
    MP_PICK_F32(k_cols_tma, nullptr, , false)
}
}  // namespace mp
