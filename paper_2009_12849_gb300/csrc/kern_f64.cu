// FP64 kernels (every step in double precision).
#include "fused.cuh"
#include "pickers.h"

namespace mp {
template <> KernelFn pick_k_fwd_rows<double>(int n) { MP_PICK_F64(k_fwd_rows, (k_fwd_rows<double, 0>)) }
template <> KernelFn pick_k_inv_rows<double>(int n) { MP_PICK_F64(k_inv_rows, (k_inv_rows<double, 0>)) }
template <> KernelFn pick_k_fwd_cols<double>(int n) { MP_PICK_F64(k_fwd_cols, (k_fwd_cols<double, 0>)) }
template <> KernelFn pick_k_inv_cols<double>(int n) { MP_PICK_F64(k_inv_cols, (k_inv_cols<double, 0>)) }
template <> KernelFn pick_fwd_cols_persist<double>(int n) { MP_PICK_F64(k_cols_persist, nullptr, , false) }
template <> KernelFn pick_inv_cols_persist<double>(int n) { MP_PICK_F64(k_cols_persist, nullptr, , true) }
template <> KernelFn pick_fwd_fused<double>(int n) { MP_PICK_F64(k_fwd_fused, nullptr) }
template <> KernelFn pick_inv_fused<double>(int n) { MP_PICK_F64(k_inv_fused, nullptr) }
template <> KernelFn pick_tridiag<double>() { return k_tridiag<double>; }
template <> ColsTmaFn pick_cols_tma<double>(int, bool) { return nullptr; }
}  // namespace mp
