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
// FP32 column kernels with the spectral pitch, tile width and radix schedule
// (e: elements per thread, 32 or 16) fixed at compile time (nx = ny = 64, 96,
// 128, 192, 256, 512, 1024 with the default tiles; E = 16 for 256, 512, 1024
// with 256-thread tiles); nullptr otherwise
KernelFn pick_cols_square_f32(int ny, int nxp, int tw, int bs, bool inv, int e);
// grouped-launch kernels of batched FP32 projections (group.cuh): phase 0..4
// = forward rows, forward columns, vertical solve, inverse columns, inverse
// rows, for length n (the rows' nx or the columns' ny; any n for phase 2);
// nullptr when n has no compile-time plan
struct GroupArgs;
using GroupFn = void (*)(const GroupArgs);
// (square: nx = ny; with nxp and tw the group's spectral pitch and tile width,
// which select the column kernels that have them compiled in when they match)
GroupFn pick_group_f32(int phase, int n, bool square = false, int nxp = 0, int tw = 0);
// FP32 persistent pipelines of the forward and inverse transforms (pipe.cuh);
// nullptr for grids without them
// (ef: the variants streaming u, v, w with evict-first L2 priority)
KernelFn pick_fwd_pipe(int nx, int ny, bool ef = false);
KernelFn pick_inv_pipe(int nx, int ny, bool ef = false);
// tensor-core split-precision forward column transforms (tcdft.cuh), format
// 1 (TF32 x 3) or 2 (BF16 x 6): nullptr unless ny = 1024; and their dynamic
// shared memory
KernelFn pick_fwd_cols_tc(int ny, int fmt);
unsigned fwd_cols_tc_smem(int fmt);
// refinement passes: FP32 transforms on FP64 fields (row kernels with F = double)
KernelFn pick_refined_fwd_rows(int n);
KernelFn pick_refined_inv_rows(int n);
KernelFn pick_refined_inv_cols(int n);   // the potential alone
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
// Extended FP32 compile-time lengths: every other 2^a 3^b 5^c length from
// 128 to 512 (the sizes a serving workload of such grids meets).  They get the
// default kernels only, compiled in groups of up to 8 lengths, rows and
// columns apart, so that the translation units build in parallel
// (kern_f32_ext.cu, compiled once per group and part).
#define MP_F32_CT_EXT1(F) F(135) F(144) F(150) F(160) F(162) F(180) F(200) F(216)
#define MP_F32_CT_EXT2(F) F(225) F(240) F(243) F(250) F(270) F(288) F(300) F(320)
#define MP_F32_CT_EXT3(F) F(324) F(360) F(375) F(384) F(400) F(405) F(432) F(450)
#define MP_F32_CT_EXT4(F) F(480) F(486) F(500)
// FP32 lengths that also have the opt-in variants (persistent, TMA, fused)
#define MP_F32_CT_CORE(F) F(64) F(96) F(128) F(192) F(256) F(512) F(1024)

namespace mp {
enum KernelKind { kFwdRows = 0, kInvRows = 1, kFwdCols = 2, kInvCols = 3 };
// group g (1..4), part 0 (rows: kFwdRows, kInvRows) or 1 (columns); nullptr
// when n is not in the group or kind not in the part
#define MP_EXT_DECL(G, P) KernelFn pick_f32_ext_##G##_##P(KernelKind kind, int n);
MP_EXT_DECL(1, 0) MP_EXT_DECL(1, 1) MP_EXT_DECL(2, 0) MP_EXT_DECL(2, 1)
MP_EXT_DECL(3, 0) MP_EXT_DECL(3, 1) MP_EXT_DECL(4, 0) MP_EXT_DECL(4, 1)
#undef MP_EXT_DECL
inline KernelFn pick_f32_ext(KernelKind kind, int n) {
    KernelFn (*const fns[])(KernelKind, int) = {pick_f32_ext_1_0, pick_f32_ext_1_1, pick_f32_ext_2_0,
                                                pick_f32_ext_2_1, pick_f32_ext_3_0, pick_f32_ext_3_1,
                                                pick_f32_ext_4_0, pick_f32_ext_4_1};
    for (auto f : fns)
        if (KernelFn k = f(kind, n)) return k;
    return nullptr;
}
// FP32 lengths with a compile-time plan (core or extended)
inline bool ct_length_f32(int n) {
#define MP_CT_CASE(N) case N:
    switch (n) {
        MP_F32_CT_CORE(MP_CT_CASE)
        MP_F32_CT_EXT1(MP_CT_CASE) MP_F32_CT_EXT2(MP_CT_CASE) MP_F32_CT_EXT3(MP_CT_CASE) MP_F32_CT_EXT4(MP_CT_CASE)
            return true;
        default:
            return false;
    }
#undef MP_CT_CASE
}
inline bool ct_core_f32(int n) {
#define MP_CT_CASE(N) case N:
    switch (n) {
        MP_F32_CT_CORE(MP_CT_CASE)
            return true;
        default:
            return false;
    }
#undef MP_CT_CASE
}
}  // namespace mp

#define MP_PICK_F64(KERNEL, DEFAULT, ...)                              \
    switch (n) {                                                       \
        case 64: return KERNEL<double, 64 __VA_ARGS__>;                \
        case 128: return KERNEL<double, 128 __VA_ARGS__>;              \
        case 256: return KERNEL<double, 256 __VA_ARGS__>;              \
        case 1024: return KERNEL<double, 1024 __VA_ARGS__>;            \
        default: return DEFAULT;                                       \
    }
