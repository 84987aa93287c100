// Kernel selection across translation units.  The host code picks kernels
// through these functions; each precision's kernels are instantiated (and
// compiled in parallel) in their own translation unit (kern_*.cu).
//
// Lengths with a compile-time FFT plan (FP32: 64, 96, 128, 192, 256, 512,
// 1024; FP64: 64, 128, 256, 1024) get their own instantiation; every other
// 2^a 3^b 5^c length runs the run-time plan (template argument 0).
#pragma once
#include "tma.cuh"

namespace mp {

using KernelFn = void (*)(ProjParams);
using ColsTmaFn = void (*)(ProjParams, ColMaps);

template <typename R> KernelFn pick_k_fwd_rows(int n);
template <typename R> KernelFn pick_k_inv_rows(int n);
template <typename R> KernelFn pick_k_fwd_cols(int n);
template <typename R> KernelFn pick_k_inv_cols(int n);
template <typename R> KernelFn pick_fwd_cols_persist(int n);   // nullptr if no compile-time plan
template <typename R> KernelFn pick_inv_cols_persist(int n);
template <typename R> KernelFn pick_fwd_fused(int n);
template <typename R> KernelFn pick_inv_fused(int n);
template <typename R> KernelFn pick_tridiag();
template <typename R> ColsTmaFn pick_cols_tma(int n, bool inv);  // nullptr if none

}  // namespace mp

// Body of a picker: the compile-time lengths of the precision, else DEFAULT.
#define MP_PICK_F32(KERNEL, DEFAULT, ...)                              \
    switch (n) {                                                       \
        case 64: return KERNEL<float, 64 __VA_ARGS__>;                 \
        case 96: return KERNEL<float, 96 __VA_ARGS__>;                 \
        case 128: return KERNEL<float, 128 __VA_ARGS__>;               \
        case 192: return KERNEL<float, 192 __VA_ARGS__>;               \
        case 256: return KERNEL<float, 256 __VA_ARGS__>;               \
        case 512: return KERNEL<float, 512 __VA_ARGS__>;               \
        case 1024: return KERNEL<float, 1024 __VA_ARGS__>;             \
        default: return DEFAULT;                                       \
    }
#define MP_PICK_F64(KERNEL, DEFAULT, ...)                              \
    switch (n) {                                                       \
        case 64: return KERNEL<double, 64 __VA_ARGS__>;                \
        case 128: return KERNEL<double, 128 __VA_ARGS__>;              \
        case 256: return KERNEL<double, 256 __VA_ARGS__>;              \
        case 1024: return KERNEL<double, 1024 __VA_ARGS__>;            \
        default: return DEFAULT;                                       \
    }
