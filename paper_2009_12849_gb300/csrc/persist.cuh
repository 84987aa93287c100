// Persistent, cp.async-staged variants of the transform kernels for the
// compile-time lengths.
//
// One block per SM loops over tasks.  While the block transforms task t, the
// global->shared copies of task t + gridDim.x are in flight (cp.async, 16-byte
// chunks, no register staging), so DRAM stays busy through the FFT arithmetic.
// Shared memory holds two input stages and the FFT buffer.
#pragma once
#include "kernels.cuh"

namespace mp {

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ---------------------------------------------------------------------------
// Column transforms (a2 y-part forward, a4 y-part inverse), length NY.
// Forward task: (level k, tile of tw columns): T -> S.
// Inverse task: (level k, tile, field f): f = 0: S -> Tp, f = 1: S*ey -> Tgy,
// f = 2: G -> Tgz (nothing at k = 0).
// Shared memory: stage[2][NY * tw] (rows of the tile, as in global memory),
// then the FFT buffer [tw][bs_col].
// ---------------------------------------------------------------------------
template <typename R, int NY, bool INV>
__global__ void __launch_bounds__(256, 1) k_cols_persist(ProjParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using C = cplx<R>;
    constexpr int S = INV ? 1 : -1;
    constexpr int CPC = 16 / (int)sizeof(C);     // complex values per 16-byte chunk
    const int tw = p.tw_cols, nz = p.nz, ny = p.ny, nxh = p.nxh, nxp = p.nxp;
    const int ntiles = p.ntiles;
    // inverse: task kind 0 transforms the staged S tile into every field that
    // derives from p^ (Tp with ex, Tgy, and Tphi if requested); kind 1 the G tile
    const int nkind = INV ? 2 : 1;
    const int ntask = nz * ntiles * nkind;
    C* stage[2] = {(C*)smem_raw, (C*)smem_raw + (size_t)NY * tw};
    C* fbuf = (C*)smem_raw + (size_t)2 * NY * tw;
    const int cpr = tw / CPC;                    // chunks per tile row

    auto decode = [&](int task, int& k, int& kx0, int& kind) {
        kind = task % nkind;
        const int t2 = task / nkind;
        k = t2 / ntiles;
        kx0 = (t2 - k * ntiles) * tw;
    };
    auto source = [&](int kind) -> const C* {
        if (!INV) return (const C*)p.T;
        return (kind == 1) ? (const C*)p.G : (const C*)p.S;
    };
    const C* ex = ctab<R>(p.ex);
    auto issue = [&](int task, C* st) {
        int k, kx0, kind;
        decode(task, k, kx0, kind);
        if (INV && kind == 1 && k == 0) return;
        const C* src = source(kind);
        const int nchunk = NY * cpr;
        for (int c = threadIdx.x; c < nchunk; c += blockDim.x) {
            const int j = c / cpr;
            const int part = c - j * cpr;
            const int kx = kx0 + part * CPC;
            C* dst = st + j * tw + part * CPC;
            if (kx < nxp) {
                cp_async16(dst, src + ((size_t)k * ny + j) * nxp + kx);
            } else {
#pragma unroll
                for (int e = 0; e < CPC; ++e) dst[e] = cmk<R>((R)0, (R)0);
            }
        }
    };
    // one transform of the staged tile into dst (f: 0 x-gradient, 1 y-gradient, else plain)
    auto transform = [&](const C* st, int k, int kx0, int f, C* dst) {
        const C* ey = (INV && f == 1) ? ctab<R>(p.ey) : nullptr;
        auto load = [&](int c, int j) -> C {
            const C v = st[j * tw + c];
            return ey ? cmul(v, ey[j]) : v;
        };
        ct_first<R, NY, S, true>(fbuf, tw, p.bs_col, load);
        CtMid<R, NY, StageInfo<R, NY, 1>::NEXT, S>::run(fbuf, tw, p.bs_col, ctab<R>(p.twy));
        const bool mul_ex = INV && f == 0;
        auto store = [&](int c, int q, const C* x, int ns) {
            const int kx = kx0 + c;
            if (kx >= nxh) return;
            constexpr int RAD = StageInfo<R, NY, LastNs<R, NY>::value>::RAD;
            const C e = mul_ex ? ex[kx] : cmk<R>((R)1, (R)0);
#pragma unroll
            for (int r = 0; r < RAD; ++r)
                dst[((size_t)k * ny + q + r * ns) * nxp + kx] = mul_ex ? cmul(x[r], e) : x[r];
        };
        ct_last<R, NY, S, true>(fbuf, tw, p.bs_col, ctab<R>(p.twy), store);
        __syncthreads();
    };

    // tasks are handed out by a ticket counter (zeroed before the launch);
    // a block takes its next ticket before transforming the current task so
    // that the next tile's copies are in flight meanwhile
    __shared__ int s_next;
    unsigned* ticket = p.sync;
    auto take = [&]() {
        if (threadIdx.x == 0) s_next = (int)atomicAdd(ticket, 1u);
        __syncthreads();
        const int t = s_next;
        __syncthreads();
        return t;
    };
    int task = take();
    int s = 0;
    if (task < ntask) issue(task, stage[0]);
    cp_async_commit();
    while (task < ntask) {
        const int next = take();
        if (next < ntask) issue(next, stage[s ^ 1]);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        int k, kx0, kind;
        decode(task, k, kx0, kind);
        const C* st = stage[s];
        if (!INV) {
            transform(st, k, kx0, -1, (C*)p.S);
        } else if (kind == 0) {
            transform(st, k, kx0, 0, (C*)p.Tp);
            transform(st, k, kx0, 1, (C*)p.Tgy);
            if (p.nch == 4) transform(st, k, kx0, 3, (C*)p.Tphi);
        } else if (k > 0) {
            transform(st, k, kx0, 2, (C*)p.Tgz);
        }
        __syncthreads();
        s ^= 1;
        task = next;
    }
    cp_async_wait<0>();
}

}  // namespace mp
