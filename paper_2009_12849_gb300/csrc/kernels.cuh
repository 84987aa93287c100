// Kernels of one anelastic projection (paper, Section 4: forward FFT, a
// vertical ODE per horizontal wavenumber in Fourier space, backward FFT),
// with the divergence (step a1) fused into the forward transform and the
// pressure-gradient correction (step a5) fused into the inverse transform.
//
// Layouts (element = one complex value of the storage precision R):
//   spectral arrays  S, G, T, Tp, Tgy, Tgz, Tphi : [nz][ny][nxp], kx < nxh valid
//   u, v, phi        : [nz][ny][nx] real;   w : [nz+1][ny][nx] real
#pragma once
#include "handoff.cuh"
#include "fft.cuh"

namespace mp {

struct ProjParams {
    int nx, ny, nz, nxh, nxp;
    FftFactors fx, fy;
    const void* twx;            // per-stage twiddle tables of the x plan (storage precision)
    const void* twy;            // per-stage twiddle tables of the y plan
    const void* twy16;          // the same for the E = 16 radix schedule (FP32 square grids; else null)
    const double* svol;         // [nz]   rho_c[k] dz[k]
    const double* rflo;         // [nz]   rho_f[k]   (0 at k = 0)
    const double* rfhi;         // [nz]   rho_f[k+1] (0 at k = nz-1)
    const double* acoef;        // [nz+1] A[k] = rho_f[k]/dzn[k], A[0] = A[nz] = 0
    const double* idzn;         // [nz+1] 1/dzn[k] (0 at k = 0, nz)
    const double* csum;         // [nz]   A[k] + A[k+1]
    const float* svol32;        // FP32 copies of svol, acoef, csum, idzn
    const float* acoef32;
    const float* csum32;
    const float* idzn32;
    const float* rflo32;        // FP32 copies of rflo, rfhi (the forward rows of FP32 fields)
    const float* rfhi32;
    double lam_fp64;            // mixed plans: |lambda| below which a column runs in FP64
    const double* lamx;         // [nxh]  2(cos(2 pi kx/nx) - 1)/dx^2
    const double* lamy;         // [ny]
    const void* ex;             // [nxh]  (exp(2 pi i kx/nx) - 1)/dx, storage precision
    const void* ey;             // [ny]
    double idx, idy;            // 1/dx, 1/dy
    float idx32, idy32;
    double scale;               // 1/(nx ny)
    // fields
    const void* u; const void* v; const void* w;
    void* uo; void* vo; void* wo; void* phi;
    // workspace
    void* S; void* G; void* T; void* Tp; void* Tgy; void* Tgz; void* Tphi;
    double2* Y; double* Gp;
    int* err;
    unsigned* sync;             // fused kernels: tickets and per-level counters (zeroed per solve)
    int ring;                   // levels in the intermediate rings (fused) or nz
    int lag;                    // fused kernels: levels between producer and consumer tasks
    // task shapes
    int rows_fwd;               // real rows per forward row task (even)
    int nrb_fwd;                // row tasks per level (forward)
    int rows_inv;               // real rows per inverse row task (even)
    int nrb_inv;
    int nch;                    // real channels per row in the inverse (3, or 4 with phi)
    int phi_only;               // 1: the inverse produces phi alone (refinement passes)
    void* phi_pass;             // refinement passes: this pass's potential (FP64, [nz][ny][nx])
    double* phi_mean;           // refinement passes: level-0 horizontal mean of the summed potential
    int tw_cols;                // kx columns per column task
    int ntiles;                 // column tasks per level
    int bs_row;                 // smem stride of a row transform (complex elements)
    int bs_col;                 // smem stride of a column transform
    HandoffArgs ho;             // hand-off of intermediates in L2 (pipelines); zero: none
    long long spin_limit;       // polls before a bounded dependency wait gives up (timeout bit)
    // sub-domains of a distributed solve (the pencil decomposition): arrays
    // hold levels kbase .. kbase + nz - 1 of a column of nz_glob levels (the
    // plan's tables and the top and bottom boundaries are global), and the
    // vertical solve's spectral rows are ky_base .. ky_base + ny - 1.  A whole
    // solve has kbase = ky_base = 0 and nz_glob = nz.
    int kbase, nz_glob, ky_base;
    // mixed plans: the pivots of the FP64 warps' columns as FP32 pairs,
    // [nz][nslots] each: pvm = a_k / e_{k-1}, pvgb = (1/e_k, a_{k+1} / e_k);
    // and the first slot of each warp ([ny][nwr], -1 for FP32 warps); null otherwise
    const float2* pvm;
    const float4* pvgb;
    const int* wslot;
    int nslots, nwr;
};

template <typename R> __device__ __forceinline__ const cplx<R>* ctab(const void* p) { return (const cplx<R>*)p; }

// Elements whose global loads one thread issues before using any of them.
constexpr int kLoadBatch = 8;

// Threads of a compile-time-length task (a thread holds E elements of a
// stage): row tasks of one warp (one complex transform at nx = 1024) measured
// fastest, 1.47 ms for the inverse rows of 1024^2 x 256 against 1.63 ms with
// 256 threads; column tiles of 256 threads (8 columns of 1024, 64-byte row
// segments) beat both narrower and wider tiles.
constexpr int kRowTaskThreads = 32;
constexpr int kColTaskThreads = 256;

// Transform nb sequences held in shared memory at buf[b*bs + spad(e)].
// N > 0: compile-time in-place plan (one buffer); N == 0: run-time plan,
// ping-pong with a second buffer right after the first.  Returns the buffer
// holding the result.
template <typename R, int N, int S, class Sc = BlockScope>
__device__ __forceinline__ cplx<R>* run_fft(cplx<R>* buf, int nb, int bs, const FftFactors& f,
                                            const cplx<R>* __restrict__ tw) {
    if constexpr (N == 0) {
        return fft_batch<R, S>(buf, buf + nb * bs, nb, bs, f, tw);
    } else {
        CtFFT<R, N, 1, S, Sc>::run(buf, nb, bs, tw);
        return buf;
    }
}

// ---------------------------------------------------------------------------
// a1 + a2 (x part): divergence of a block of rows, real FFT along x.
// Two real rows share one complex transform: z = d_j + i d_{j+1}; after the
// transform X_j[k] = (Z[k] + conj Z[n-k])/2, X_{j+1}[k] = (Z[k] - conj Z[n-k])/(2i).
// Output is the level's x-spectrum in T, scaled by rho_c dz (the symmetric
// form of the vertical operator).
// F is the field type: R, or double with R = float for the refinement passes
// (the divergence is formed in F, then rounded to the transform precision).
// ---------------------------------------------------------------------------
// EF: u, v, w stream through L2 with evict-first priority (the pipelines,
// whose x-spectra must stay resident until the column tasks read them).
// One task: `rows` rows from j0 of level k, by the threads of scope Sc (the
// block, or one warp with its own shared-memory slice at smem_raw).
template <typename R, int NX, typename F, bool EF, class Sc>
__device__ __forceinline__ void fwd_rows_task(const ProjParams& p, unsigned char* smem_raw, int k, int j0,
                                              int rows) {
    using C = cplx<R>;
    const int nx = p.nx, ny = p.ny;
    const int npair = rows / 2;
    const int bs = p.bs_row;
    C* bufA = (C*)smem_raw;

    const F* u = (const F*)p.u;
    const F* v = (const F*)p.v;
    const F* w = (const F*)p.w;
    const size_t plane = (size_t)ny * nx;
    // per-level coefficients in the field precision (FP32 fields read the
    // FP32 tables: no FP64 conversions in the kernel)
    constexpr bool f32 = sizeof(F) == 4;
    const int kg = p.kbase + k;                 // global level: tables and boundaries
    const bool below = kg > 0, above = kg < p.nz_glob - 1;
    const F sv = f32 ? (F)p.svol32[kg] : (F)p.svol[kg];
    const F rlo = f32 ? (F)p.rflo32[kg] : (F)p.rflo[kg];
    const F rhi = f32 ? (F)p.rfhi32[kg] : (F)p.rfhi[kg];
    const F idx = f32 ? (F)p.idx32 : (F)p.idx, idy = f32 ? (F)p.idy32 : (F)p.idy;

    const C* res;
    if constexpr (NX > 0 && NX % 4 == 0 && sizeof(R) == 4 && sizeof(F) == 4) {
        // FP32, compile-time length: every thread takes groups of 4 adjacent
        // cells of a row and loads them as float4 (u, v, v of the row below,
        // w below and above), 4 groups in flight per thread.
        constexpr int G = 4, NG = NX / 4;
        const int tot = rows * NG;
        const int step = G * Sc::size();
        // EF: u, v, w stream through L2 with evict-first priority, so that the
        // x-spectra handed to the column tasks stay resident
        const unsigned long long pol = EF ? l2_evict_first() : 0ull;
        auto ld4 = [&](size_t o, const float* a) -> float4 {
            if constexpr (EF) return ld_ef((const float4*)&a[o], pol);
            else return *(const float4*)&a[o];
        };
        auto ld1 = [&](size_t o, const float* a) -> float {
            if constexpr (EF) return ld_ef(&a[o], pol);
            else return a[o];
        };
        for (int base = Sc::tid(); base < tot; base += step) {
            float4 u4[G], v4[G], vm4[G], wl4[G], wh4[G];
            float um1[G];
#pragma unroll
            for (int c = 0; c < G; ++c) {
                const int t = base + c * Sc::size();
                const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
                u4[c] = v4[c] = vm4[c] = wl4[c] = wh4[c] = z;
                um1[c] = 0.f;
                if (t < tot) {
                    const int r = t / NG;
                    const int i0 = 4 * (t - r * NG);
                    const int j = j0 + r;
                    if (j < ny) {
                        const size_t row = (size_t)k * plane + (size_t)j * NX;
                        const size_t rowm = (size_t)k * plane + (size_t)(j == 0 ? ny - 1 : j - 1) * NX;
                        u4[c] = ld4(row + i0, u);
                        um1[c] = i0 == 0 ? ld1(row + NX - 1, u) : u[row + i0 - 1];
                        v4[c] = ld4(row + i0, v);
                        vm4[c] = ld4(rowm + i0, v);
                        if (below) wl4[c] = ld4(row + i0, w);
                        if (above) wh4[c] = ld4(row + plane + i0, w);
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < G; ++c) {
                const int t = base + c * Sc::size();
                if (t < tot) {
                    const int r = t / NG;
                    const int i0 = 4 * (t - r * NG);
                    const float uu[5] = {um1[c], u4[c].x, u4[c].y, u4[c].z, u4[c].w};
                    const float vv[4] = {v4[c].x, v4[c].y, v4[c].z, v4[c].w};
                    const float vm[4] = {vm4[c].x, vm4[c].y, vm4[c].z, vm4[c].w};
                    const float wl[4] = {wl4[c].x, wl4[c].y, wl4[c].z, wl4[c].w};
                    const float wh[4] = {wh4[c].x, wh4[c].y, wh4[c].z, wh4[c].w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float hdiv = (uu[e + 1] - uu[e]) * (float)idx + (vv[e] - vm[e]) * (float)idy;
                        const float d = (float)sv * hdiv + ((float)rhi * wh[e] - (float)rlo * wl[e]);
                        float* slot = (float*)&bufA[(r >> 1) * bs + spad(i0 + e)];
                        slot[r & 1] = d;
                    }
                }
            }
        }
        Sc::sync();
        res = run_fft<R, NX, -1, Sc>(bufA, npair, bs, p.fx, ctab<R>(p.twx));
    } else {
        // Loads are batched (kLoadBatch elements per thread issued before any is
        // used) so that enough bytes are in flight to cover DRAM latency.
        const int tot = rows * nx;
        const int step = kLoadBatch * Sc::size();
        for (int base = Sc::tid(); base < tot; base += step) {
            F uc[kLoadBatch], um[kLoadBatch], vc[kLoadBatch], vm[kLoadBatch], wl[kLoadBatch], wh[kLoadBatch];
#pragma unroll
            for (int c = 0; c < kLoadBatch; ++c) {
                const int t = base + c * Sc::size();
                uc[c] = um[c] = vc[c] = vm[c] = wl[c] = wh[c] = (F)0;
                if (t < tot) {
                    const int r = (NX > 0) ? t / NX : t / nx;
                    const int i = t - r * nx;
                    const int j = j0 + r;
                    if (j < ny) {
                        const size_t row = (size_t)k * plane + (size_t)j * nx;
                        const size_t rowm = (size_t)k * plane + (size_t)(j == 0 ? ny - 1 : j - 1) * nx;
                        const int im = (i == 0) ? nx - 1 : i - 1;
                        uc[c] = u[row + i];
                        um[c] = u[row + im];
                        vc[c] = v[row + i];
                        vm[c] = v[rowm + i];
                        if (below) wl[c] = w[row + i];
                        if (above) wh[c] = w[row + plane + i];
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < kLoadBatch; ++c) {
                const int t = base + c * Sc::size();
                if (t < tot) {
                    const int r = (NX > 0) ? t / NX : t / nx;
                    const int i = t - r * nx;
                    F d;
                    if constexpr (sizeof(F) == 8 && sizeof(R) == 4) {
                        // FP64 fields of the refinement passes: the same sum in
                        // fused multiply-adds (FP64 arithmetic is this GPU's
                        // scarce resource)
                        d = fma(sv * idx, uc[c] - um[c], fma(sv * idy, vc[c] - vm[c], fma(rhi, wh[c], -rlo * wl[c])));
                    } else {
                        const F hdiv = (uc[c] - um[c]) * idx + (vc[c] - vm[c]) * idy;
                        d = sv * hdiv + (rhi * wh[c] - rlo * wl[c]);
                    }
                    R* slot = (R*)&bufA[(r >> 1) * bs + spad(i)];
                    slot[r & 1] = (R)d;
                }
            }
        }
        Sc::sync();
        res = run_fft<R, NX, -1, Sc>(bufA, npair, bs, p.fx, ctab<R>(p.twx));
    }

    C* T = (C*)p.T;
    const int nxh = p.nxh;
    for (int q = 0; q < npair; ++q) {
        const int j = j0 + 2 * q;
        if (j >= ny) break;
        const C* rq = res + q * bs;
        C* to = T + ((size_t)k * ny + j) * p.nxp;
        const bool second = j + 1 < ny;
        for (int kx = Sc::tid(); kx < nxh; kx += Sc::size()) {
            const C z = rq[spad(kx)];
            const C zc = cconj(rq[spad(kx == 0 ? 0 : nx - kx)]);
            const C a = cscale(cadd(z, zc), (R)0.5);
            const C dd = csub(z, zc);
            to[kx] = a;
            if (second) to[kx + p.nxp] = cmk<R>((R)0.5 * dd.y, (R)-0.5 * dd.x);
        }
    }
}

template <typename R, int NX, typename F = R, bool EF = false>
__global__ void __launch_bounds__(512) k_fwd_rows(ProjParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nrb = p.nrb_fwd;
    const int kl = blockIdx.x / nrb;
    fwd_rows_task<R, NX, F, EF, BlockScope>(p, smem_raw, kl, (blockIdx.x - kl * nrb) * p.rows_fwd,
                                            p.rows_fwd);
}

// Shared-memory pitch of a column tile's transforms (the plan's bs_col): the
// padded length rounded to 4 (mod 16) complex values, which spreads the
// columns of a tile over distinct banks.
template <int NY> struct ColPitch {
    static constexpr int value = [] {
        int b = NY + (NY >> 5) + 1;
        while (b % 16 != 4) ++b;
        return b;
    }();
};

// ---------------------------------------------------------------------------
// Column transforms along y for a tile of kx columns of one level.
// DIR = -1: forward (T -> S).  The inverse uses k_inv_cols.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void load_cols(cplx<R>* buf, const cplx<R>* src, int k, int kx0, const ProjParams& p,
                                          const cplx<R>* mul_y) {
    const int tw = p.tw_cols, ny = p.ny, bs = p.bs_col;
    const int tot = ny * tw;
    const int step = 2 * kLoadBatch * blockDim.x;
    for (int base = threadIdx.x; base < tot; base += step) {
        cplx<R> val[2 * kLoadBatch];
#pragma unroll
        for (int c = 0; c < 2 * kLoadBatch; ++c) {
            const int t = base + c * blockDim.x;
            val[c] = cmk<R>((R)0, (R)0);
            if (t < tot) {
                const int j = t / tw;
                const int kx = kx0 + (t - j * tw);
                if (kx < p.nxh) val[c] = src[((size_t)k * ny + j) * p.nxp + kx];
            }
        }
#pragma unroll
        for (int c = 0; c < 2 * kLoadBatch; ++c) {
            const int t = base + c * blockDim.x;
            if (t < tot) {
                const int j = t / tw;
                const int cc = t - j * tw;
                cplx<R> v = val[c];
                if (mul_y) v = cmul(v, mul_y[j]);
                buf[cc * bs + spad(j)] = v;
            }
        }
    }
}

template <typename R>
__device__ __forceinline__ void store_cols(cplx<R>* dst, const cplx<R>* buf, int k, int kx0, const ProjParams& p) {
    const int tw = p.tw_cols, ny = p.ny, bs = p.bs_col;
    const int tot = ny * tw;
    for (int t = threadIdx.x; t < tot; t += blockDim.x) {
        const int j = t / tw;
        const int c = t - j * tw;
        const int kx = kx0 + c;
        if (kx < p.nxh) dst[((size_t)k * ny + j) * p.nxp + kx] = buf[c * bs + spad(j)];
    }
}

// Chained forward columns: the tiles whose columns share 128-byte lines of T
// (16 complex FP32 values) count their reads in p.ho.groups; the last tile of
// a group to finish reading discards the group's lines of the level.  Tiles
// of 16 or more columns own their lines and discard them at once.
template <typename R>
__device__ __forceinline__ void discard_fwd_tile(const ProjParams& p, int k, int tile) {
    constexpr int LINE = 128 / (int)sizeof(cplx<R>);       // complex values per line
    const int tw = p.tw_cols;
    int c0, nc;                                             // first column, columns to discard
    if (tw >= LINE) {
        // the last tile may reach past the padded row: its lines stop at nxp
        c0 = tile * tw;
        nc = min(tw, p.nxp - c0);
        if (nc <= 0) return;
    } else {
        __shared__ unsigned s_last;
        const int g = LINE / tw;                            // tiles per line group
        const int grp = tile / g;
        const int members = min(g, p.ntiles - grp * g);
        if (threadIdx.x == 0) {
            unsigned last = 1;
            if (members > 1) {
                __threadfence();
                const int ngrp = (p.ntiles + g - 1) / g;
                last = (atomicAdd(&p.ho.groups[(size_t)k * ngrp + grp], 1u) + 1u) % (unsigned)members == 0;
            }
            s_last = last;
        }
        __syncthreads();
        if (!s_last) return;
        c0 = grp * LINE;
        nc = LINE;
    }
    const cplx<R>* T = (const cplx<R>*)p.T + (size_t)k * p.ny * p.nxp;
    const int lpr = nc / LINE;                              // lines per row
    for (int t = threadIdx.x; t < p.ny * lpr; t += blockDim.x) {
        const int j = t / lpr;
        l2_discard(T + (size_t)j * p.nxp + c0 + (t - j * lpr) * LINE);
    }
}

// One column task of a compile-time length: tile `tile` of level k, T -> S.
// NXP and TW as in inv_cols_ct_task.
template <typename R, int NY, int NXP = 0, int TW = 0, int E = ept<R>()>
__device__ __forceinline__ void fwd_cols_task(const ProjParams& p, unsigned char* smem_raw, int k, int tile) {
    using C = cplx<R>;
    const int nxh = p.nxh;
    const int nxp = NXP ? NXP : p.nxp;
    const int tw = TW ? TW : p.tw_cols;
    const int bs = TW ? ColPitch<NY>::value : p.bs_col;
    const int kx0 = tile * tw;
    C* buf = (C*)smem_raw;
    const C* T = (const C*)p.T + (size_t)k * NY * nxp + kx0;
    C* S = (C*)p.S + (size_t)k * NY * nxp + kx0;
    auto load = [&](int c, int j) -> C {
        return (kx0 + c < nxh) ? T[j * nxp + c] : cmk<R>((R)0, (R)0);
    };
    const C* twy = ctab<R>(E == ept<R>() ? p.twy : p.twy16);
    ct_first<R, NY, -1, true, false, BlockScope, E>(buf, tw, bs, load);
    if (p.ho.discard) discard_fwd_tile<R>(p, k, tile);
    CtMid<R, NY, StageInfo<R, NY, 1, E>::NEXT, -1, BlockScope, E>::run(buf, tw, bs, twy);
    auto store = [&](int c, int q, const C* x, int ns) {
        if (kx0 + c >= nxh) return;
        constexpr int RAD = StageInfo<R, NY, LastNs<R, NY, E>::value, E>::RAD;
        C* d = S + q * nxp + c;
#pragma unroll
        for (int r = 0; r < RAD; ++r) d[r * ns * nxp] = x[r];
    };
    ct_last<R, NY, -1, true, BlockScope, E>(buf, tw, bs, twy, store);
}

template <typename R, int NY, int NXP = 0, int TW = 0, int E = ept<R>()>
__global__ void __launch_bounds__(512) k_fwd_cols(ProjParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using C = cplx<R>;
    const int kl = blockIdx.x / p.ntiles;
    const int k = kl;
    const int tile = blockIdx.x - kl * p.ntiles;
    if constexpr (NY > 0) {
        fwd_cols_task<R, NY, NXP, TW, E>(p, smem_raw, k, tile);
    } else {
        C* buf = (C*)smem_raw;
        load_cols<R>(buf, (const C*)p.T, k, tile * p.tw_cols, p, nullptr);
        __syncthreads();
        const C* res = run_fft<R, NY, -1>(buf, p.tw_cols, p.bs_col, p.fy, ctab<R>(p.twy));
        store_cols<R>((C*)p.S, res, k, tile * p.tw_cols, p);
    }
}

// ---------------------------------------------------------------------------
// a3: vertical tridiagonal problem per (kx, ky), one thread per column.
// Symmetric form (rows multiplied by rho_c dz):
//   A[k] p[k-1] + b[k] p[k] + A[k+1] p[k+1] = D'[k],  b[k] = lambda s[k] - (A[k] + A[k+1])
// Forward: e = b - A^2/e_prev, y = D' - (A/e_prev) y_prev.  Back:
// p[k] = (y[k] - A[k+1] p[k+1]) / e[k].  The (0,0) column pins p[0] = 0 by
// starting its elimination with y[0] = 0 and 1/e[0] = 0, which also decouples
// level 0 from level 1.  Outputs p^ and the spectral w-gradient
// (p[k]-p[k-1])/dzn[k], both scaled by 1/(nx ny) for the inverse transform.
//
// A warp takes 32 consecutive kx of one ky row.  Mixed plans run a warp in
// FP32 unless its smallest |lambda| (at its first kx) is below lam_fp64, the
// near-zero wavenumbers whose conditioning needs FP64; FP64 plans run every
// column in FP64.  The forward sweep keeps y in S and 1/e in G (or, for FP64
// columns of a mixed plan, y split over S and G and 1/e in Gp); the back
// sweep reads them back and overwrites them with p^ and gz^.
// ---------------------------------------------------------------------------
constexpr int kTriPrefetch = 8;

template <typename T> struct VCoef;
template <> struct VCoef<double> {
    const double *a, *s, *c, *iz;
    __device__ VCoef(const ProjParams& p) : a(p.acoef), s(p.svol), c(p.csum), iz(p.idzn) {}
};
template <> struct VCoef<float> {
    const float *a, *s, *c, *iz;
    __device__ VCoef(const ProjParams& p) : a(p.acoef32), s(p.svol32), c(p.csum32), iz(p.idzn32) {}
};

// Arithmetic and storage in the same precision T: y in S[k], 1/e in G[k].x.
template <typename T>
__device__ __forceinline__ void tridiag_column_inplace(const ProjParams& p, size_t base, T lam, bool mean) {
    using C = cplx<T>;
    const int nz = p.nz;
    const size_t LS = (size_t)p.ny * p.nxp;
    C* S = (C*)p.S;
    C* G = (C*)p.G;
    const VCoef<T> vc(p);
    const T scale = (T)p.scale;
    T g = (T)0;
    C y = cmk<T>((T)0, (T)0);
    C cur[kTriPrefetch], nxt[kTriPrefetch];
#pragma unroll
    for (int i = 0; i < kTriPrefetch; ++i) cur[i] = (i < nz) ? S[i * LS + base] : cmk<T>((T)0, (T)0);
    for (int kb = 0; kb < nz; kb += kTriPrefetch) {
#pragma unroll
        for (int i = 0; i < kTriPrefetch; ++i) {
            const int k = kb + kTriPrefetch + i;
            nxt[i] = (k < nz) ? S[k * LS + base] : cmk<T>((T)0, (T)0);
        }
#pragma unroll
        for (int i = 0; i < kTriPrefetch; ++i) {
            const int k = kb + i;
            if (k < nz) {
                const T ak = vc.a[k];
                const T m = ak * g;
                const T e = lam * vc.s[k] - vc.c[k] - ak * m;
                T gk = (T)1 / e;
                C yk = cmk<T>(cur[i].x - m * y.x, cur[i].y - m * y.y);
                if (mean && k == 0) { gk = (T)0; yk = cmk<T>((T)0, (T)0); }
                g = gk;
                y = yk;
                S[k * LS + base] = yk;
                ((T*)&G[k * LS + base])[0] = gk;
            }
        }
#pragma unroll
        for (int i = 0; i < kTriPrefetch; ++i) cur[i] = nxt[i];
    }
    // back substitution, top to bottom
    C ph = cmk<T>(y.x * g, y.y * g);
    S[(nz - 1) * LS + base] = cmk<T>(ph.x * scale, ph.y * scale);
    C cy[kTriPrefetch], ny_[kTriPrefetch];
    T cg[kTriPrefetch], ng[kTriPrefetch];
#pragma unroll
    for (int i = 0; i < kTriPrefetch; ++i) {
        const int k = nz - 2 - i;
        cy[i] = (k >= 0) ? S[k * LS + base] : cmk<T>((T)0, (T)0);
        cg[i] = (k >= 0) ? ((const T*)&G[k * LS + base])[0] : (T)0;
    }
    for (int kb = nz - 2; kb >= 0; kb -= kTriPrefetch) {
#pragma unroll
        for (int i = 0; i < kTriPrefetch; ++i) {
            const int k = kb - kTriPrefetch - i;
            ny_[i] = (k >= 0) ? S[k * LS + base] : cmk<T>((T)0, (T)0);
            ng[i] = (k >= 0) ? ((const T*)&G[k * LS + base])[0] : (T)0;
        }
#pragma unroll
        for (int i = 0; i < kTriPrefetch; ++i) {
            const int k = kb - i;
            if (k >= 0) {
                const T a1 = vc.a[k + 1];
                const C pn = cmk<T>((cy[i].x - a1 * ph.x) * cg[i], (cy[i].y - a1 * ph.y) * cg[i]);
                const T iz = vc.iz[k + 1] * scale;
                G[(k + 1) * LS + base] = cmk<T>((ph.x - pn.x) * iz, (ph.y - pn.y) * iz);
                S[k * LS + base] = cmk<T>(pn.x * scale, pn.y * scale);
                ph = pn;
            }
        }
#pragma unroll
        for (int i = 0; i < kTriPrefetch; ++i) { cy[i] = ny_[i]; cg[i] = ng[i]; }
    }
}

// FP64 arithmetic on FP32 storage (near-zero wavenumbers of a mixed plan):
// y.x in S[k] and y.y in G[k] (each slot reinterpreted as one double), 1/e in
// Gp.  Loads go out kTriBatch64 levels at a time before the levels' stores,
// so a column waits on DRAM once per batch rather than once per level.
constexpr int kTriBatch64 = 8;

__device__ __forceinline__ void tridiag_column_mixed64(const ProjParams& p, size_t base, double lam, bool mean) {
    constexpr int B = kTriBatch64;
    const int nz = p.nz;
    const size_t LS = (size_t)p.ny * p.nxp;
    float2* S = (float2*)p.S;
    float2* G = (float2*)p.G;
    double* Sd = (double*)p.S;
    double* Gd = (double*)p.G;
    double* Gp = p.Gp;
    const double scale = p.scale;
    double g = 0.0;
    double2 y = make_double2(0.0, 0.0);
    for (int kb = 0; kb < nz; kb += B) {
        float2 dv[B];
#pragma unroll
        for (int i = 0; i < B; ++i) dv[i] = (kb + i < nz) ? S[(kb + i) * LS + base] : make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < B; ++i) {
            const int k = kb + i;
            if (k >= nz) break;
            const size_t o = k * LS + base;
            const double ak = p.acoef[k];
            const double m = ak * g;
            const double e = lam * p.svol[k] - p.csum[k] - ak * m;
            double gk = 1.0 / e;
            double2 yk = make_double2((double)dv[i].x - m * y.x, (double)dv[i].y - m * y.y);
            if (mean && k == 0) { gk = 0.0; yk = make_double2(0.0, 0.0); }
            g = gk;
            y = yk;
            Sd[o] = yk.x;
            Gd[o] = yk.y;
            Gp[o] = gk;
        }
    }
    double2 ph = make_double2(y.x * g, y.y * g);
    S[(nz - 1) * LS + base] = make_float2((float)(ph.x * scale), (float)(ph.y * scale));
    for (int kb = nz - 2; kb >= 0; kb -= B) {
        double yx[B], yy[B], gv[B];
#pragma unroll
        for (int i = 0; i < B; ++i) {
            const int k = kb - i;
            const size_t o = (k >= 0 ? k : 0) * LS + base;
            yx[i] = (k >= 0) ? Sd[o] : 0.0;
            yy[i] = (k >= 0) ? Gd[o] : 0.0;
            gv[i] = (k >= 0) ? Gp[o] : 0.0;
        }
#pragma unroll
        for (int i = 0; i < B; ++i) {
            const int k = kb - i;
            if (k < 0) break;
            const size_t o = k * LS + base;
            const double a1 = p.acoef[k + 1];
            const double2 pn = make_double2((yx[i] - a1 * ph.x) * gv[i], (yy[i] - a1 * ph.y) * gv[i]);
            const double iz = p.idzn[k + 1] * scale;
            G[o + LS] = make_float2((float)((ph.x - pn.x) * iz), (float)((ph.y - pn.y) * iz));
            S[o] = make_float2((float)(pn.x * scale), (float)(pn.y * scale));
            ph = pn;
        }
    }
}

// Arithmetic on FP32 pairs (hi + lo, |lo| <= ulp(hi)/2; Dekker's and Knuth's
// error-free transformations, the product through a fused multiply-add): about
// 48 bits of precision on the FP32 pipes, which GB300 runs 64 times faster than
// its FP64 pipe.
struct F2P {
    float hi, lo;
};
__device__ __forceinline__ F2P fp_fast_two_sum(float a, float b) {     // |a| >= |b|
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ F2P fp_two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ F2P fp_mul(F2P a, F2P b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    return fp_fast_two_sum(p, e);
}
__device__ __forceinline__ F2P fp_sub(F2P a, F2P b) {
    const F2P s = fp_two_sum(a.hi, -b.hi);
    return fp_fast_two_sum(s.hi, s.lo + (a.lo - b.lo));
}

// Pivots of the FP64 warps' columns (one thread per column, plan time): the
// forward sweep's 1/e_k = 1 / (lambda s_k - c_k - a_k^2 / e_{k-1}) depend
// only on lambda and the vertical coefficients (1/e_{-1} = 0; the pinned mean
// column has 1/e_0 = 0).  Computed in FP64 and stored as FP32 pairs: pvm[k] =
// a_k / e_{k-1}, pvgb[k] = (1/e_k, a_{k+1} / e_k).  wlist holds (ky, kx0) per warp.
__device__ __forceinline__ float2 split_pair(double x) {
    const float h = (float)x;
    return make_float2(h, (float)(x - (double)h));
}
template <int D = 0>
__global__ void __launch_bounds__(128) k_fp64_pivots(const int* __restrict__ wlist, const double* __restrict__ lamx,
                                                     const double* __restrict__ lamy, const double* __restrict__ a,
                                                     const double* __restrict__ sv, const double* __restrict__ cs,
                                                     int nxh, int nz, int nslots, float2* __restrict__ pvm,
                                                     float4* __restrict__ pvgb) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nslots) return;
    const int ky = wlist[2 * (t >> 5)], kx = wlist[2 * (t >> 5) + 1] + (t & 31);
    const double lam = kx < nxh ? lamx[kx] + lamy[ky] : -1.0;
    const bool mean = kx == 0 && ky == 0;
    double g = 0.0;
    for (int k = 0; k < nz; ++k) {
        const double m = a[k] * g;
        const double e = fma(-a[k], m, fma(lam, sv[k], -cs[k]));
        g = (mean && k == 0) ? 0.0 : 1.0 / e;
        const double b = (k + 1 < nz ? a[k + 1] : 0.0) * g;
        const size_t o = (size_t)k * nslots + t;
        pvm[o] = split_pair(m);
        const float2 gh = split_pair(g), bh = split_pair(b);
        pvgb[o] = make_float4(gh.x, gh.y, bh.x, bh.y);
    }
}

// FP64-class column of a mixed plan on FP32 pairs with the plan's pivots:
// forward y_k = D'_k - (a_k/e_{k-1}) y_{k-1}, back p_k = y_k/e_k - (a_{k+1}/e_k)
// p_{k+1}, everything in FP32-pair arithmetic; y is kept between the sweeps
// as pairs (real part in S[k], imaginary part in G[k]).
__device__ __forceinline__ void tridiag_column_pair(const ProjParams& p, size_t base, int slot, bool mean) {
    constexpr int B = 4;                    // levels per batch of loads (registers)
    const int nz = p.nz;
    const size_t LS = (size_t)p.ny * p.nxp;
    float2* S = (float2*)p.S;
    float2* G = (float2*)p.G;
    const float2* pm = p.pvm + slot;
    const float4* pg = p.pvgb + slot;
    const size_t GS = (size_t)p.nslots;
    const float scale = (float)p.scale;
    F2P yr{0.f, 0.f}, yi{0.f, 0.f};
    for (int kb = 0; kb < nz; kb += B) {
        float2 dv[B], mv[B];
#pragma unroll
        for (int i = 0; i < B; ++i) {
            const bool in = kb + i < nz;
            dv[i] = in ? S[(kb + i) * LS + base] : make_float2(0.f, 0.f);
            mv[i] = in ? pm[(kb + i) * GS] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int i = 0; i < B; ++i) {
            const int k = kb + i;
            if (k >= nz) break;
            const F2P m{mv[i].x, mv[i].y};
            yr = fp_sub(F2P{dv[i].x, 0.f}, fp_mul(m, yr));
            yi = fp_sub(F2P{dv[i].y, 0.f}, fp_mul(m, yi));
            if (mean && k == 0) yr = yi = F2P{0.f, 0.f};
            const size_t o = k * LS + base;
            S[o] = make_float2(yr.hi, yr.lo);
            G[o] = make_float2(yi.hi, yi.lo);
        }
    }
    // top level: p = y / e
    const float4 gt = pg[(size_t)(nz - 1) * GS];
    F2P pr = fp_mul(yr, F2P{gt.x, gt.y}), pi = fp_mul(yi, F2P{gt.x, gt.y});
    S[(nz - 1) * LS + base] = make_float2(pr.hi * scale, pi.hi * scale);
    for (int kb = nz - 2; kb >= 0; kb -= B) {
        float2 ys[B], yg[B];
        float4 gv[B];
#pragma unroll
        for (int i = 0; i < B; ++i) {
            const int k = kb - i;
            const size_t o = (k >= 0 ? k : 0) * LS + base;
            ys[i] = (k >= 0) ? S[o] : make_float2(0.f, 0.f);
            yg[i] = (k >= 0) ? G[o] : make_float2(0.f, 0.f);
            gv[i] = (k >= 0) ? pg[(size_t)k * GS] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int i = 0; i < B; ++i) {
            const int k = kb - i;
            if (k < 0) break;
            const size_t o = k * LS + base;
            const F2P g{gv[i].x, gv[i].y}, b{gv[i].z, gv[i].w};
            const F2P nr = fp_sub(fp_mul(F2P{ys[i].x, ys[i].y}, g), fp_mul(b, pr));
            const F2P ni = fp_sub(fp_mul(F2P{yg[i].x, yg[i].y}, g), fp_mul(b, pi));
            const float iz = (float)p.idzn[k + 1] * scale;
            const F2P dr = fp_sub(pr, nr), di = fp_sub(pi, ni);
            G[o + LS] = make_float2((dr.hi + dr.lo) * iz, (di.hi + di.lo) * iz);
            S[o] = make_float2(nr.hi * scale, ni.hi * scale);
            pr = nr;
            pi = ni;
        }
    }
}

// FP32 column without a stored forward sweep: the forward sweep keeps only a
// checkpoint (y, 1/e) at the start of every kTriSeg levels (thread-local
// memory); the back substitution recomputes each segment's forward values in
// registers from its checkpoint, re-reading D'.  D' is read twice, but y and
// 1/e never travel to DRAM and back.
constexpr int kTriSeg = 8;
constexpr int kTriMaxSeg = 128;              // nz <= kTriSeg * kTriMaxSeg

__device__ __forceinline__ void tridiag_column_ckpt32(const ProjParams& p, size_t base, float lam) {
    using C = float2;
    const int nz = p.nz;
    const size_t LS = (size_t)p.ny * p.nxp;
    C* S = (C*)p.S;
    C* G = (C*)p.G;
    const VCoef<float> vc(p);
    const float scale = (float)p.scale;
    float ck_g[kTriMaxSeg];
    C ck_y[kTriMaxSeg];
    float g = 0.f;
    C y = make_float2(0.f, 0.f);
    const int nseg = (nz + kTriSeg - 1) / kTriSeg;
    // forward sweep, checkpoints at segment starts
    for (int sg = 0; sg < nseg; ++sg) {
        ck_g[sg] = g;
        ck_y[sg] = y;
        const int k0 = sg * kTriSeg;
        C d[kTriSeg];
#pragma unroll
        for (int i = 0; i < kTriSeg; ++i) d[i] = (k0 + i < nz) ? S[(k0 + i) * LS + base] : make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < kTriSeg; ++i) {
            const int k = k0 + i;
            if (k < nz) {
                const float ak = vc.a[k];
                const float m = ak * g;
                const float e = lam * vc.s[k] - vc.c[k] - ak * m;
                g = __frcp_rn(e);
                y = make_float2(d[i].x - m * y.x, d[i].y - m * y.y);
            }
        }
    }
    // back substitution segment by segment, top to bottom
    C ph = make_float2(y.x * g, y.y * g);
    bool top = true;
    for (int sg = nseg - 1; sg >= 0; --sg) {
        const int k0 = sg * kTriSeg;
        C d[kTriSeg], ys[kTriSeg];
        float gs[kTriSeg];
#pragma unroll
        for (int i = 0; i < kTriSeg; ++i) d[i] = (k0 + i < nz) ? S[(k0 + i) * LS + base] : make_float2(0.f, 0.f);
        float gg = ck_g[sg];
        C yy = ck_y[sg];
#pragma unroll
        for (int i = 0; i < kTriSeg; ++i) {
            const int k = k0 + i;
            if (k < nz) {
                const float ak = vc.a[k];
                const float m = ak * gg;
                const float e = lam * vc.s[k] - vc.c[k] - ak * m;
                gg = __frcp_rn(e);
                yy = make_float2(d[i].x - m * yy.x, d[i].y - m * yy.y);
            }
            ys[i] = yy;
            gs[i] = gg;
        }
#pragma unroll
        for (int i = kTriSeg - 1; i >= 0; --i) {
            const int k = k0 + i;
            if (k >= nz) continue;
            if (top) {                       // the top level: p = y g
                top = false;
                __stcs(&S[k * LS + base], make_float2(ph.x * scale, ph.y * scale));
                continue;
            }
            const float a1 = vc.a[k + 1];
            const C pn = make_float2((ys[i].x - a1 * ph.x) * gs[i], (ys[i].y - a1 * ph.y) * gs[i]);
            const float iz = vc.iz[k + 1] * scale;
            __stcs(&G[(k + 1) * LS + base], make_float2((ph.x - pn.x) * iz, (ph.y - pn.y) * iz));
            __stcs(&S[k * LS + base], make_float2(pn.x * scale, pn.y * scale));
            ph = pn;
        }
    }
}

// Rows are taken in the order ky = 0, ny-1, 1, ny-2, ...: the columns of
// small |lambda| (the FP64 ones of a mixed plan, limited by the FP64 rate) sit at
// both ends of the ky range and so start in the first wave of blocks, where
// they overlap the FP32 columns instead of forming a tail.
// Threads per block of the vertical solve (one column each).  One-warp
// blocks, which spread the FP64 warps over more SMs, measured no faster and
// spill more registers.
constexpr int kTriThreads = 128;

// Column `col` of the launch (rows of nxw = nxh rounded up to 32 columns).
template <typename R>
__device__ __forceinline__ void tridiag_task(const ProjParams& p, long long col) {
    const int nxw = (p.nxh + 31) & ~31;
    const int r = (int)(col / nxw);
    const int kx = (int)(col - (long long)r * nxw);
    if (r >= p.ny || kx >= p.nxh) return;
    const int ky = (r & 1) ? p.ny - 1 - (r >> 1) : (r >> 1);      // local spectral row
    const int kyg = p.ky_base + ky;                                 // global wavenumber row
    const size_t base = (size_t)ky * p.nxp + kx;
    const double lam = p.lamx[kx] + p.lamy[kyg];
    const bool mean = (kx == 0 && kyg == 0);
    if (sizeof(R) == 8) {
        tridiag_column_inplace<double>(p, base, lam, mean);
    } else {
        const double lam_warp = p.lamx[kx & ~31] + p.lamy[kyg];  // smallest |lambda| of the warp
        // the warp holding the mean column always runs FP64 (it carries the pin)
        if (-lam_warp < p.lam_fp64 || (kyg == 0 && kx < 32)) {
            const int ws = p.pvm ? p.wslot[kyg * p.nwr + (kx >> 5)] : -1;
            if (ws >= 0) tridiag_column_pair(p, base, ws + (kx & 31), mean);
            else tridiag_column_mixed64(p, base, lam, mean);
        }
        else if (p.nz <= kTriSeg * kTriMaxSeg) tridiag_column_ckpt32(p, base, (float)lam);
        else tridiag_column_inplace<float>(p, base, (float)lam, mean);
    }
}

template <typename R>
__global__ void __launch_bounds__(kTriThreads, 1024 / kTriThreads) k_tridiag(ProjParams p) {
    tridiag_task<R>(p, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

// ---------------------------------------------------------------------------
// a4 (y part): inverse y-transforms of one level's tile, one field per task:
//   f = 0: Tp   = IFFT_y(p^) * ex   (x-gradient; ex depends on the column only)
//   f = 1: Tgy  = IFFT_y(p^ * ey)   (y-gradient)
//   f = 2: Tgz  = IFFT_y(gz^)       (z-gradient; nothing at k = 0)
//   f = 3: Tphi = IFFT_y(p^)        (only when phi is requested)
// ---------------------------------------------------------------------------
template <typename R>
struct InvColField {
    const cplx<R>* src;
    cplx<R>* dst;
    const cplx<R>* ey;      // non-null: multiply the input by ey[j]
    bool ex;                // multiply the output by ex[kx]
    bool skip;
};
template <typename R>
__device__ __forceinline__ InvColField<R> inv_col_field(const ProjParams& p, int f, int k) {
    using C = cplx<R>;
    InvColField<R> r;
    r.src = (f == 2) ? (const C*)p.G : (const C*)p.S;
    r.dst = (f == 0) ? (C*)p.Tp : (f == 1) ? (C*)p.Tgy : (f == 2) ? (C*)p.Tgz : (C*)p.Tphi;
    r.ey = (f == 1) ? ctab<R>(p.ey) : nullptr;
    r.ex = (f == 0);
    r.skip = (f == 2 && p.kbase + k == 0);
    return r;
}

// Compile-time lengths: task = (level, tile, kind); kind 0 reads the p^ tile
// and writes every field derived from it (x-gradient with ex, y-gradient,
// phi if requested; the re-reads of the tile hit L2), kind 1 transforms gz^.
// F (the field, as inv_col_field) is a template argument so that the loads
// and stores carry no run-time branch; NXP and TW, when non-zero, are the
// spectral row pitch and the tile width known at compile time (square grids
// with the default tiles), which turns the element addresses into constant
// offsets from one per-thread pointer.
template <typename R, int NY, int F, int NXP = 0, int TW = 0, int E = ept<R>()>
__device__ __forceinline__ void inv_cols_ct_task(const ProjParams& p, int k, int kx0, cplx<R>* buf) {
    using C = cplx<R>;
    const int nxh = p.nxh;
    const int nxp = NXP ? NXP : p.nxp;
    const int tw = TW ? TW : p.tw_cols;
    const int bs = TW ? ColPitch<NY>::value : p.bs_col;
    const C* src = (F == 2 ? (const C*)p.G : (const C*)p.S) + (size_t)k * NY * nxp + kx0;
    const C* ey = ctab<R>(p.ey);
    auto load = [&](int c, int j) -> C {
        if (kx0 + c >= nxh) return cmk<R>((R)0, (R)0);
        const C v = src[j * nxp + c];
        if constexpr (F == 1) return cmul(v, ey[j]);
        else return v;
    };
    const C* twy = ctab<R>(E == ept<R>() ? p.twy : p.twy16);
    ct_first<R, NY, 1, true, false, BlockScope, E>(buf, tw, bs, load);
    CtMid<R, NY, StageInfo<R, NY, 1, E>::NEXT, 1, BlockScope, E>::run(buf, tw, bs, twy);
    const C* ex = ctab<R>(p.ex);
    C* dst = (F == 0 ? (C*)p.Tp : F == 1 ? (C*)p.Tgy : F == 2 ? (C*)p.Tgz : (C*)p.Tphi) + (size_t)k * NY * nxp + kx0;
    auto store = [&](int c, int q, const C* x, int ns) {
        if (kx0 + c >= nxh) return;
        constexpr int RAD = StageInfo<R, NY, LastNs<R, NY, E>::value, E>::RAD;
        C* d = dst + q * nxp + c;
        if constexpr (F == 0) {
            const C e = ex[kx0 + c];
#pragma unroll
            for (int r = 0; r < RAD; ++r) d[r * ns * nxp] = cmul(x[r], e);
        } else {
#pragma unroll
            for (int r = 0; r < RAD; ++r) d[r * ns * nxp] = x[r];
        }
    };
    ct_last<R, NY, 1, true, BlockScope, E>(buf, tw, bs, twy, store);
}

// One column task of a compile-time length: tile from kx0 of level k; kind
// 0 transforms the p^ tile (x- and y-gradient, and phi if requested; with
// PHI the potential alone), kind 1 the gz^ tile.
template <typename R, int NY, bool PHI, int NXP = 0, int TW = 0, int E = ept<R>()>
__device__ __forceinline__ void inv_cols_tile(const ProjParams& p, unsigned char* smem_raw, int k, int kx0,
                                              int kind) {
    cplx<R>* buf = (cplx<R>*)smem_raw;
    if constexpr (PHI) {
        if (kind == 0) inv_cols_ct_task<R, NY, 3, NXP, TW, E>(p, k, kx0, buf);
    } else if (kind == 0) {
        inv_cols_ct_task<R, NY, 0, NXP, TW, E>(p, k, kx0, buf);
        __syncthreads();
        inv_cols_ct_task<R, NY, 1, NXP, TW, E>(p, k, kx0, buf);
        if (p.nch == 4) {
            __syncthreads();
            inv_cols_ct_task<R, NY, 3, NXP, TW, E>(p, k, kx0, buf);
        }
    } else if (p.kbase + k > 0) {
        inv_cols_ct_task<R, NY, 2, NXP, TW, E>(p, k, kx0, buf);
    }
}

// PHI: the potential alone (refinement passes): kind 0 transforms the p^ tile
// into Tphi, kind 1 does nothing.
template <typename R, int NY, bool PHI = false, int NXP = 0, int TW = 0, int E = ept<R>()>
__global__ void __launch_bounds__(512) k_inv_cols(ProjParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using C = cplx<R>;
    if constexpr (NY > 0) {
        const int task = blockIdx.x >> 1;
        const int kl = task / p.ntiles;
        const int tw = TW ? TW : p.tw_cols;
        inv_cols_tile<R, NY, PHI, NXP, TW, E>(p, smem_raw, kl, (task - kl * p.ntiles) * tw, blockIdx.x & 1);
        return;
    }
    const int nf = p.nch;
    const int f = PHI ? 3 : blockIdx.x % nf;
    const int task = blockIdx.x / nf;
    const int k = task / p.ntiles;
    const int kx0 = (task - k * p.ntiles) * p.tw_cols;
    const InvColField<R> fd = inv_col_field<R>(p, f, k);
    if (fd.skip) return;
    C* buf = (C*)smem_raw;
    load_cols<R>(buf, fd.src, k, kx0, p, fd.ey);
    __syncthreads();
    C* res = run_fft<R, NY, 1>(buf, p.tw_cols, p.bs_col, p.fy, ctab<R>(p.twy));
    if (fd.ex) {
        const C* ex = ctab<R>(p.ex);
        const int tot = p.ny * p.tw_cols;
        for (int t = threadIdx.x; t < tot; t += blockDim.x) {
            const int j = t / p.tw_cols;
            const int c = t - j * p.tw_cols;
            const int kx = min(kx0 + c, p.nxh - 1);
            C* e = &res[c * p.bs_col + spad(j)];
            *e = cmul(*e, ex[kx]);
        }
        __syncthreads();
    }
    store_cols<R>(fd.dst, res, k, kx0, p);
}

// ---------------------------------------------------------------------------
// a4 (x part) + a5: inverse real transforms along x, then u -= gx, v -= gy,
// w -= gz (w = 0 on the bottom and top faces) and optionally phi.  Channels:
//   0: Tp (x-gradient)   1: Tgy (y-gradient)   2: Tgz (z-gradient)   3: Tphi (phi)
// One complex transform carries one channel of two adjacent rows,
// Z = A_j + i A_{j+1} with Hermitian-extended A; the real part of the inverse
// is row j, the imaginary part row j+1.  Channels are never mixed in one
// transform: phi is dominated by its largest scales and would otherwise put
// its rounding error into a gradient channel.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ const cplx<R>* inv_channel_spectrum(const ProjParams& p, int ch) {
    using C = cplx<R>;
    return (ch == 0) ? (const C*)p.Tp : (ch == 1) ? (const C*)p.Tgy : (ch == 2) ? (const C*)p.Tgz : (const C*)p.Tphi;
}

// Hermitian-extended spectrum of one row at kx in [0, nx).
template <typename R>
__device__ __forceinline__ cplx<R> hermitian_at(const cplx<R>* row, int nx, int nxh, int kx) {
    const bool neg = kx >= nxh;
    const int kk = neg ? nx - kx : kx;
    cplx<R> val = row[kk];
    if (kk == 0 || 2 * kk == nx) val.y = (R)0;      // real-only DC / Nyquist
    if (neg) val.y = -val.y;
    return val;
}

template <typename R>
__device__ __forceinline__ cplx<R> inv_spectrum(const ProjParams& p, int k, int j, int ch, int kx) {
    if (j >= p.ny || (ch == 2 && p.kbase + k == 0)) return cmk<R>((R)0, (R)0);
    const cplx<R>* row = inv_channel_spectrum<R>(p, ch) + ((size_t)k * p.ny + j) * p.nxp;
    return hermitian_at<R>(row, p.nx, p.nxh, kx);
}

// Compile-time lengths: one channel per task, task = (level, row block, channel).
// Generic lengths: all channels of a row block in one task.  F is the field
// type (R, or double with R = float for the refinement passes: the gradient
// is subtracted from the FP64 field in FP64).
// Compile-time length along x: one channel of one row pair per task (the
// body of k_inv_rows; returns early for the bottom face of w).
template <typename R, int NX, typename F, bool EF, class Sc>
__device__ __forceinline__ void inv_rows_ct(const ProjParams& p, unsigned char* smem_raw, int k, int j0, int ch,
                                            int rows) {
    using C = cplx<R>;
    const int ny = p.ny;
    const int bs = p.bs_row;
    C* bufA = (C*)smem_raw;
    const size_t plane = (size_t)ny * NX;
    constexpr int NXH = NX / 2 + 1;
    const int npr = rows / 2;                    // transforms (row pairs) per task
    F* out = (ch == 0) ? (F*)p.uo : (ch == 1) ? (F*)p.vo : (ch == 2) ? (F*)p.wo : (F*)p.phi;
    const int kg = p.kbase + k;                   // global level (boundaries)
    const bool top = kg == p.nz_glob - 1;
    if (ch == 2 && kg == 0) {
        // bottom face: w = 0
        for (int t = Sc::tid(); t < rows * NX; t += Sc::size()) {
            const int j = j0 + t / NX;
            if (j < ny) {
                out[(size_t)j * NX + (t % NX)] = (F)0;
                if (top) out[plane + (size_t)j * NX + (t % NX)] = (F)0;   // top face too
            }
        }
        return;
    }
    const F* in = (ch == 0) ? (const F*)p.u : (ch == 1) ? (const F*)p.v : (const F*)p.w;
    const bool upd = ch < 3;
    const C* spec = inv_channel_spectrum<R>(p, ch) + (size_t)k * ny * p.nxp;
    const int nxp = p.nxp;
    auto load = [&](int b, int kx) -> C {
        const int j = j0 + 2 * b;
        C a = cmk<R>((R)0, (R)0), c = cmk<R>((R)0, (R)0);
        if (j < ny) a = hermitian_at<R>(spec + (size_t)j * nxp, NX, NXH, kx);
        if (j + 1 < ny) c = hermitian_at<R>(spec + (size_t)(j + 1) * nxp, NX, NXH, kx);
        return cmk<R>(a.x - c.y, a.y + c.x);
    };
    ct_first<R, NX, 1, false, false, Sc>(bufA, npr, bs, load);
    if (p.ho.discard) {
        // pipelines: this task is the only reader of its rows of the channel
        // spectrum; the lines are dead once the first stage has read them
        constexpr int LINE = 128 / (int)sizeof(C);
        const int lpr = nxp / LINE;
        for (int t = Sc::tid(); t < rows * lpr; t += Sc::size()) {
            const int r = t / lpr;
            if (j0 + r < ny) l2_discard(spec + (size_t)(j0 + r) * nxp + (t - r * lpr) * LINE);
        }
    }
    CtMid<R, NX, StageInfo<R, NX, 1>::NEXT, 1, Sc>::run(bufA, npr, bs, ctab<R>(p.twx));
    // the correction reads u, v or w where it writes them (outputs may
    // alias inputs)
    constexpr int LRAD = StageInfo<R, NX, LastNs<R, NX>::value>::RAD;
    if constexpr (sizeof(F) == sizeof(R)) {
        // every value this thread will update is loaded before the last
        // stage writes any
        constexpr int LNB = (ElemsPerThread<R>::value + LRAD - 1) / LRAD;
        F prev[LNB][2][LRAD];
        // EF: u, v, w stream through L2 with evict-first priority
        constexpr bool ef = EF && sizeof(F) == 4;
        const unsigned long long pol = ef ? l2_evict_first() : 0ull;
        auto pre = [&](int b, int q, int ns, int i) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = j0 + 2 * b + h;
                const size_t row = (size_t)k * plane + (size_t)j * NX + q;
#pragma unroll
                for (int r = 0; r < LRAD; ++r) {
                    F val = (F)0;
                    if (upd && j < ny) {
                        if constexpr (ef) val = ld_ef((const float*)&in[row + r * ns], pol);
                        else val = in[row + r * ns];
                    }
                    prev[i][h][r] = val;
                }
            }
        };
        auto store = [&](int b, int q, const C* x, int ns, int i) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = j0 + 2 * b + h;
                if (j >= ny) continue;
                const size_t row = (size_t)k * plane + (size_t)j * NX + q;
#pragma unroll
                for (int r = 0; r < LRAD; ++r) {
                    const F val = (F)(h ? x[r].y : x[r].x);
                    const F res = (ch < 3) ? prev[i][h][r] - val : (upd ? prev[i][h][r] + val : val);
                    if constexpr (ef) st_ef((float*)&out[row + r * ns], res, pol);
                    else out[row + r * ns] = res;
                    if (ch == 2 && top) out[row + r * ns + plane] = (F)0;
                }
            }
        };
        ct_last_pre<R, NX, 1, false, Sc>(bufA, npr, bs, ctab<R>(p.twx), pre, store);
    } else {
        // wider fields (refinement passes): one butterfly's operands at a
        // time, which keeps the FP64 values in registers
        auto store = [&](int b, int q, const C* x, int ns) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = j0 + 2 * b + h;
                if (j >= ny) continue;
                const size_t row = (size_t)k * plane + (size_t)j * NX + q;
                F prev[LRAD];
#pragma unroll
                for (int r = 0; r < LRAD; ++r) prev[r] = upd ? in[row + r * ns] : (F)0;
#pragma unroll
                for (int r = 0; r < LRAD; ++r) {
                    const F val = (F)(h ? x[r].y : x[r].x);
                    out[row + r * ns] = (ch < 3) ? prev[r] - val : (upd ? prev[r] + val : val);
                    if (ch == 2 && top) out[row + r * ns + plane] = (F)0;
                }
            }
        };
        ct_last<R, NX, 1, false, Sc>(bufA, npr, bs, ctab<R>(p.twx), store);
    }
}

// EF: u, v, w stream through L2 with evict-first priority (pipelines).
template <typename R, int NX, typename F = R, bool EF = false>
__global__ void __launch_bounds__(512) k_inv_rows(ProjParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using C = cplx<R>;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int nrb = p.nrb_inv;
    const int nch = p.nch;
    const int bs = p.bs_row;
    C* bufA = (C*)smem_raw;
    const size_t plane = (size_t)ny * nx;
    if constexpr (NX > 0) {
        const int nrb = p.nrb_inv;
        const int ch = p.phi_only ? 3 : blockIdx.x % nch;
        const int t2 = blockIdx.x / nch;
        const int kl = t2 / nrb;
        inv_rows_ct<R, NX, F, EF, BlockScope>(p, smem_raw, kl, (t2 - kl * nrb) * p.rows_inv, ch,
                                              p.rows_inv);
    } else {
        const int k = blockIdx.x / nrb;
        const int j0 = (blockIdx.x - k * nrb) * p.rows_inv;
        const int npr = p.rows_inv / 2;
        const int np = nch * npr;
        const F* u = (const F*)p.u;
        const F* v = (const F*)p.v;
        const F* w = (const F*)p.w;
        F* uo = (F*)p.uo;
        F* vo = (F*)p.vo;
        F* wo = (F*)p.wo;
        F* ph = (F*)p.phi;
        const int tot = np * nx;
        const int step = kLoadBatch * blockDim.x;
        for (int base = threadIdx.x; base < tot; base += step) {
            C av[kLoadBatch], bv[kLoadBatch];
#pragma unroll
            for (int c = 0; c < kLoadBatch; ++c) {
                const int t = base + c * blockDim.x;
                av[c] = bv[c] = cmk<R>((R)0, (R)0);
                if (t < tot) {
                    const int q = t / nx;
                    const int kx = t - q * nx;
                    const int ch = q / npr;
                    const int m = q - ch * npr;
                    const int j = j0 + 2 * m;
                    const int chs = p.phi_only ? 3 : ch;
                    av[c] = inv_spectrum<R>(p, k, j, chs, kx);
                    bv[c] = inv_spectrum<R>(p, k, j + 1, chs, kx);
                }
            }
#pragma unroll
            for (int c = 0; c < kLoadBatch; ++c) {
                const int t = base + c * blockDim.x;
                if (t < tot) {
                    const int q = t / nx;
                    const int kx = t - q * nx;
                    bufA[q * bs + spad(kx)] = cmk<R>(av[c].x - bv[c].y, av[c].y + bv[c].x);
                }
            }
        }
        __syncthreads();
        const C* res = run_fft<R, NX, 1>(bufA, np, bs, p.fx, ctab<R>(p.twx));
        const int tot2 = p.rows_inv * nx;
        const int step2 = kLoadBatch * blockDim.x;
        for (int base = threadIdx.x; base < tot2; base += step2) {
            F uu[kLoadBatch], vv[kLoadBatch], ww[kLoadBatch];
#pragma unroll
            for (int c = 0; c < kLoadBatch; ++c) {
                const int t = base + c * blockDim.x;
                uu[c] = vv[c] = ww[c] = (F)0;
                if (t < tot2) {
                    const int r = t / nx;
                    const int i = t - r * nx;
                    const int j = j0 + r;
                    if (j < ny && !p.phi_only) {
                        const size_t o = (size_t)k * plane + (size_t)j * nx + i;
                        uu[c] = u[o];
                        vv[c] = v[o];
                        if (p.kbase + k > 0) ww[c] = w[o];
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < kLoadBatch; ++c) {
                const int t = base + c * blockDim.x;
                if (t >= tot2) continue;
                const int r = t / nx;
                const int i = t - r * nx;
                const int j = j0 + r;
                if (j >= ny) continue;
                const int m = r >> 1;
                F val[4] = {(F)0, (F)0, (F)0, (F)0};
#pragma unroll
                for (int ch = 0; ch < 4; ++ch) {
                    if (ch < nch) {
                        const C z = res[(ch * npr + m) * bs + spad(i)];
                        val[ch] = (F)((r & 1) ? z.y : z.x);
                    }
                }
                const size_t o = (size_t)k * plane + (size_t)j * nx + i;
                if (p.phi_only) {
                    ph[o] = val[0];
                    continue;
                }
                uo[o] = uu[c] - val[0];
                vo[o] = vv[c] - val[1];
                wo[o] = (p.kbase + k == 0) ? (F)0 : (F)(ww[c] - val[2]);
                if (p.kbase + k == p.nz_glob - 1) wo[o + plane] = (F)0;
                if (nch == 4) ph[o] = val[3];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Refinement passes, a5 in physical space: u -= (phi[i+1]-phi[i])/dx,
// v -= (phi[j+1]-phi[j])/dy, w[k] -= (phi[k]-phi[k-1])/dzn[k] (w = 0 on the
// bottom and top faces), all in F, with phi this pass's potential (periodic
// in x and y).  The correction is then the exact discrete gradient of a
// stored potential, so the next pass's divergence is exactly this pass's
// remaining error.  phi_sum (optional) accumulates the passes' potentials;
// on the last pass it also subtracts *mean_sub, the level-0 horizontal mean of
// the sum (the pin of the potential: the FP32 transforms leave each pass's
// potential a rounding-size constant off, which no later pass can see).
// One block row per (level, row).
// ---------------------------------------------------------------------------
template <typename F>
__global__ void __launch_bounds__(256) k_fd_correct(ProjParams p, const F* __restrict__ phi, F* phi_sum,
                                                    int accumulate, const double* mean_sub) {
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int k = blockIdx.x / ny;
    const int j = blockIdx.x - k * ny;
    const size_t plane = (size_t)ny * nx;
    const size_t row = (size_t)k * plane + (size_t)j * nx;
    const size_t rowp = (size_t)k * plane + (size_t)(j + 1 == ny ? 0 : j + 1) * nx;
    const F* u = (const F*)p.u;
    const F* v = (const F*)p.v;
    const F* w = (const F*)p.w;
    F* uo = (F*)p.uo;
    F* vo = (F*)p.vo;
    F* wo = (F*)p.wo;
    const F idx = (F)p.idx, idy = (F)p.idy;
    const F iz = (F)p.idzn[k];
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        const F ph = phi[row + i];
        const F pe = phi[row + (i + 1 == nx ? 0 : i + 1)];
        const F pn = phi[rowp + i];
        const F uu = u[row + i], vv = v[row + i];
        const F ww = (k > 0) ? w[row + i] : (F)0;
        const F pb = (k > 0) ? phi[row - plane + i] : (F)0;
        uo[row + i] = fma(-idx, pe - ph, uu);
        vo[row + i] = fma(-idy, pn - ph, vv);
        wo[row + i] = (k > 0) ? fma(-iz, ph - pb, ww) : (F)0;
        if (k == nz - 1) wo[row + plane + i] = (F)0;
        if (phi_sum) {
            const F sum = accumulate ? phi_sum[row + i] + ph : ph;
            phi_sum[row + i] = mean_sub ? sum - (F)*mean_sub : sum;
        }
    }
}

// *acc += mean of phi[0..n) (one block; FP64 sums).
template <typename F>
__global__ void __launch_bounds__(1024) k_mean_add(const F* __restrict__ phi, int n, double* acc) {
    __shared__ double part[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += (double)phi[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = (threadIdx.x < (blockDim.x + 31) / 32) ? part[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) *acc += s / (double)n;
    }
}

}  // namespace mp
