// Column transforms with TMA-staged tiles (a2 y-part forward, a4 y-part
// inverse) for the FP32 compile-time lengths.
//
// One block per SM loops over work items in a fixed round-robin order:
//   forward: item = (level k, tile of tw columns), T -> S
//   inverse: item = (level k, tile, field f), f = 0: S -> Tp (x-gradient, ex
//            applied after the transform), 1: S*ey -> Tgy, 2: G -> Tgz
//            (no item at k = 0), 3: S -> Tphi (only when phi is requested)
// Two shared buffers alternate.  The TMA engine loads an item's tile
// (tw columns x NY rows of the [nz*ny][nxp] array, rows as in global memory)
// into a buffer and signals an mbarrier; the block transforms the tile in
// place, writes the result back into the same buffer in the global row
// layout and hands it to a TMA store; once the store has read the buffer the
// block's first thread refills it with the item two steps ahead.  So while the
// block transforms one tile, the next tile is in flight and the previous
// result drains, with no register staging of either.
//
// Opt-in (MONC_PROJ_TMA=1): at 1024^2 x 256 the register-staged column
// kernels measured faster (forward 0.46 vs 0.52 ms, inverse 1.28 vs 1.69 ms).
// With one block of 8 warps per SM the transform arithmetic, not the copies,
// limits these kernels; the register-staged kernels run 16 warps per SM.
//
// Every mbarrier wait is bounded: after kMbarSpinLimit polls the block
// latches bit 0 of the plan's error word (reported as a timeout), stops
// issuing copies, waits for the stores it issued and returns.
#pragma once
#include <cuda.h>
#include "kernels.cuh"

namespace mp {

// Tensor maps of one launch (2D views [nz*ny rows][nxh valid columns] of
// complex arrays with row pitch nxp).
struct ColMaps {
    CUtensorMap src[2];     // forward: T;  inverse: S (p^), G (gz^)
    CUtensorMap dst[4];     // forward: S;  inverse: Tp, Tgy, Tgz, Tphi
};

constexpr long long kMbarSpinLimit = 1ll << 22;

__device__ __forceinline__ unsigned smem_u32(const void* ptr) {
    return (unsigned)__cvta_generic_to_shared(ptr);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// true once the phase of the given parity has completed
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, const void* src) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];"
                 ::"l"(map), "r"(x), "r"(y), "r"(smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

template <typename R, int NY, bool INV>
__global__ void __launch_bounds__(256, 1) k_cols_tma(ProjParams p, const __grid_constant__ ColMaps maps) {
    constexpr int NBUF = 2;
    // dynamic shared memory: [up to 127 bytes to a 128-byte boundary]
    // [NBUF buffers][NBUF mbarriers][abort flag]
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using C = cplx<R>;
    constexpr int S = INV ? 1 : -1;
    constexpr int BOXR = NY <= 256 ? NY : 256;        // rows per TMA box
    static_assert(NY % BOXR == 0, "box rows");
    const int tw = p.tw_cols, nz = p.nz, nxh = p.nxh, ntiles = p.ntiles;
    const int nf = INV ? p.nch : 1;
    const int nitems = nz * ntiles * nf;
    unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    const size_t buf_bytes = (size_t)tw * p.bs_col * sizeof(C);
    C* buf[2] = {(C*)base, (C*)(base + (NBUF - 1) * buf_bytes)};
    unsigned long long* bar = (unsigned long long*)(base + NBUF * buf_bytes);
    int& s_abort = *(int*)(bar + NBUF);
    const unsigned tile_bytes = (unsigned)((size_t)tw * NY * sizeof(C));

    auto decode = [&](int item, int& k, int& tile, int& f) {
        f = item % nf;
        const int t2 = item / nf;
        k = t2 / ntiles;
        tile = t2 - k * ntiles;
    };
    auto valid = [&](int item) -> bool {
        if (item >= nitems) return false;
        int k, t, f;
        decode(item, k, t, f);
        return !(INV && f == 2 && k == 0);
    };
    auto issue = [&](int item, int s) {                 // first thread only
        int k, t, f;
        decode(item, k, t, f);
        const CUtensorMap* m = &maps.src[(INV && f == 2) ? 1 : 0];
        mbar_expect_tx(&bar[s], tile_bytes);
#pragma unroll
        for (int b = 0; b < NY / BOXR; ++b)
            tma_load_2d(buf[s] + (size_t)b * BOXR * tw, m, t * tw, k * NY + b * BOXR, &bar[s]);
    };

    if (threadIdx.x == 0) {
        for (int sb = 0; sb < NBUF; ++sb) mbar_init(&bar[sb], 1);
        s_abort = 0;
        fence_async_smem();
    }
    __syncthreads();
    const int first = blockIdx.x, stride = gridDim.x;
    unsigned pending = 0u;                              // first thread: bit s = a load on buffer s in flight
    if (threadIdx.x == 0) {
        if (valid(first)) { issue(first, 0); pending |= 1u; }
        if (NBUF > 1 && valid(first + stride)) { issue(first + stride, 1); pending |= 2u; }
    }
    unsigned phase = 0u;                                // bit s: parity of buffer s's next completion
    const C* ex = ctab<R>(p.ex);
    const C* ey = ctab<R>(p.ey);
    int n = 0;
    for (int item = first; item < nitems; item += stride, ++n) {
        const int s = n % NBUF;
        if (valid(item)) {
            long long spins = 0;
            bool ok = true;
            while (!mbar_try_wait(&bar[s], (phase >> s) & 1u)) {
                if (++spins > kMbarSpinLimit) { ok = false; break; }
            }
            if (ok) {
                phase ^= 1u << s;
                pending &= ~(1u << s);
            } else {
                s_abort = 1;
            }
            __syncthreads();
            if (s_abort) break;
            int k, t, f;
            decode(item, k, t, f);
            C* b = buf[s];
            const int kx0 = t * tw;
            // stage 1 reads the tile in its global row layout and writes the
            // transform layout into the same buffer
            const bool mul_ey = INV && f == 1;
            auto load = [&](int c, int j) -> C {
                const C v = b[j * tw + c];
                return mul_ey ? cmul(v, ey[j]) : v;
            };
            ct_first<R, NY, S, true, true>(b, tw, p.bs_col, load);
            CtMid<R, NY, StageInfo<R, NY, 1>::NEXT, S>::run(b, tw, p.bs_col, ctab<R>(p.twy));
            const bool mul_ex = INV && f == 0;
            auto store = [&](int c, int q, const C* x, int ns) {
                constexpr int RAD = StageInfo<R, NY, LastNs<R, NY>::value>::RAD;
                const int kx = kx0 + c;
                const C e = (mul_ex && kx < nxh) ? ex[kx] : cmk<R>((R)1, (R)0);
#pragma unroll
                for (int r = 0; r < RAD; ++r) b[(q + r * ns) * tw + c] = mul_ex ? cmul(x[r], e) : x[r];
            };
            ct_last_sync<R, NY, S, true>(b, tw, p.bs_col, ctab<R>(p.twy), store);
            fence_async_smem();
            __syncthreads();
            if (threadIdx.x == 0) {
                const CUtensorMap* m = &maps.dst[INV ? f : 0];
#pragma unroll
                for (int bb = 0; bb < NY / BOXR; ++bb)
                    tma_store_2d(m, kx0, k * NY + bb * BOXR, b + (size_t)bb * BOXR * tw);
                bulk_commit();
            }
        }
        // refill this buffer with the item two steps ahead once the store
        // has read it
        if (threadIdx.x == 0) {
            bulk_wait_read_all();
            const int next = item + NBUF * stride;
            if (valid(next)) { issue(next, s); pending |= 1u << s; }
        }
    }
    if (threadIdx.x == 0) {
        bulk_wait_all();
        if (s_abort) {
            atomicOr(p.err, 1);
            // give the loads still in flight a bounded time to land before the
            // block's shared memory goes away
            for (int sb = 0; sb < NBUF; ++sb) {
                long long spins = 0;
                while ((pending >> sb & 1u) && !mbar_try_wait(&bar[sb], (phase >> sb) & 1u) &&
                       ++spins <= kMbarSpinLimit) {
                }
            }
        }
    }
}

}  // namespace mp
