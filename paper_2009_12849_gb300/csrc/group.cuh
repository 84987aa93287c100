// Grouped launches of a batch of projections.
//
// A batch of independent projections (paper, Section 4: each solve is a
// forward FFT, a vertical solve per wavenumber and a backward FFT) of uneven
// sizes runs, per phase, one launch for all the instances of a group: the
// instances that share the horizontal size, the precision and the task
// shapes.  Blocks are numbered instance after instance (start[i] is the
// first block of instance i), so the launch is as wide as the group's work
// and small instances fill the GPU together instead of one after another.
// Each instance's parameters travel in the launch's parameter space
// (__grid_constant__, no upload, so a batch can be captured into a graph);
// kGroupMax instances fit in the 32 KB of kernel parameters.
#pragma once
#include "kernels.cuh"

namespace mp {

constexpr int kGroupMax = 20;

struct GroupArgs {
    int n;                          // instances in this launch
    int start[kGroupMax + 1];       // first block of each instance; start[n] = grid size
    ProjParams p[kGroupMax];
};

__device__ __forceinline__ int group_instance(const GroupArgs& g, int b) {
    int i = 0;
    while (i + 1 < g.n && g.start[i + 1] <= b) ++i;
    return i;
}

// a1 + a2 (x): block b of an instance = (level, row block)
template <int NX>
__global__ void __launch_bounds__(512) k_fwd_rows_grp(const __grid_constant__ GroupArgs g) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int i = group_instance(g, blockIdx.x);
    const ProjParams& p = g.p[i];
    const int b = blockIdx.x - g.start[i];
    const int k = b / p.nrb_fwd;
    fwd_rows_task<float, NX, float, false, BlockScope>(p, smem_raw, k, (b - k * p.nrb_fwd) * p.rows_fwd,
                                                       p.rows_fwd);
}

// Spectral pitch and tile width of an n x n FP32 plan with the default
// 256-thread column tiles (the plan's set_task_shapes), for the column kernels
// that take them at compile time.
template <int N> struct GroupCols {
    static constexpr int NXP = ((N / 2 + 1) + 3) & ~3;
    static constexpr int TW0 = 256 * 32 / N < 32 ? 256 * 32 / N : 32;
    static constexpr int TW = TW0 < N / 2 + 1 ? TW0 : N / 2 + 1;
};

// a2 (y): block = (level, tile); SQ: square grid with GroupCols' pitch and tile
template <int NY, bool SQ = false>
__global__ void __launch_bounds__(512) k_fwd_cols_grp(const __grid_constant__ GroupArgs g) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int i = group_instance(g, blockIdx.x);
    const ProjParams& p = g.p[i];
    const int b = blockIdx.x - g.start[i];
    const int k = b / p.ntiles;
    if constexpr (SQ) fwd_cols_task<float, NY, GroupCols<NY>::NXP, GroupCols<NY>::TW>(p, smem_raw, k, b - k * p.ntiles);
    else fwd_cols_task<float, NY>(p, smem_raw, k, b - k * p.ntiles);
}

// a3: kTriThreads columns per block (any horizontal size)
template <typename R>
__global__ void __launch_bounds__(kTriThreads, 1024 / kTriThreads) k_tridiag_grp(const __grid_constant__ GroupArgs g) {
    const int i = group_instance(g, blockIdx.x);
    tridiag_task<R>(g.p[i], (long long)(blockIdx.x - g.start[i]) * blockDim.x + threadIdx.x);
}

// a4 (y): block = (level, tile, kind)
template <int NY, bool SQ = false>
__global__ void __launch_bounds__(512) k_inv_cols_grp(const __grid_constant__ GroupArgs g) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int i = group_instance(g, blockIdx.x);
    const ProjParams& p = g.p[i];
    const int b = blockIdx.x - g.start[i];
    const int task = b >> 1;
    const int k = task / p.ntiles;
    using GC = GroupCols<NY>;
    if constexpr (SQ)
        inv_cols_tile<float, NY, false, GC::NXP, GC::TW>(p, smem_raw, k, (task - k * p.ntiles) * GC::TW, b & 1);
    else
        inv_cols_tile<float, NY, false>(p, smem_raw, k, (task - k * p.ntiles) * p.tw_cols, b & 1);
}

// a4 (x) + a5: block = (level, row block, channel)
template <int NX>
__global__ void __launch_bounds__(512) k_inv_rows_grp(const __grid_constant__ GroupArgs g) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int i = group_instance(g, blockIdx.x);
    const ProjParams& p = g.p[i];
    const int b = blockIdx.x - g.start[i];
    const int ch = b % p.nch;
    const int t2 = b / p.nch;
    const int k = t2 / p.nrb_inv;
    inv_rows_ct<float, NX, float, false, BlockScope>(p, smem_raw, k, (t2 - k * p.nrb_inv) * p.rows_inv, ch,
                                                     p.rows_inv);
}

using GroupFn = void (*)(const GroupArgs);

}  // namespace mp
