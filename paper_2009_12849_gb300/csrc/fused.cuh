// Fused persistent kernels for square grids of a compile-time length N.
//
// Forward (a1 + a2): row tasks (divergence + r2c along x of a block of rows of
// level k) and column tasks (c2c along y of a tile of kx columns of level k)
// share one kernel.  Blocks take tasks from a ticket counter in the order
//   rows(0..L-1), rows(L), cols(0), rows(L+1), cols(1), ..., cols(nz-1)   (lag L)
// and a task only ever waits for tasks with smaller tickets, which are held by
// blocks that are already running, so the schedule cannot deadlock.  The
// x-spectra pass through a ring of `ring` levels that stays in L2: a column
// task of level k waits until every row task of level k is done; a row task of
// level k waits until the column tasks of level k - ring have read its slot.
//
// Inverse (a4 + a5): column tasks (c2c along y of one field of a tile) and
// row tasks (c2r along x of one channel of a block of rows, plus the
// correction) in the order cols(0..L-1), cols(L), rows(0), cols(L+1), rows(1), ...
// with the channel spectra in rings of `ring` levels.
//
// Every wait is bounded: after p.spin_limit polls the block latches bit 0 of the
// plan's error word (reported as a timeout) and carries on without waiting.
#pragma once
#include "persist.cuh"

namespace mp {

// Thread 0 waits until *ctr >= target (acquire), for at most `limit` polls
// after the first; the block then synchronises.
__device__ __forceinline__ void block_wait(const unsigned* ctr, unsigned target, int* err, long long limit) {
    if (threadIdx.x == 0) {
        long long spins = 0;
        while (true) {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
            if (v >= target) break;
            if (++spins > limit) {
                atomicOr(err, 1);
                break;
            }
            __nanosleep(64);
        }
    }
    __syncthreads();
}

// All threads' writes of this task are done; publish them (release).
__device__ __forceinline__ void block_signal(unsigned* ctr) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(ctr, 1u);
    }
}

// Ticket order of two task kinds with a lag of L levels: the first L levels of
// kind P, then for every level g the P tasks of level g + L (while they
// exist) followed by the Q tasks of level g.  P tasks per level: a, Q: b.
// Returns true for a P task; *k gets its level and *idx its index.
__device__ __forceinline__ bool decode_lagged(int t, int nz, int L, int a, int b, int* k, int* idx) {
    if (t < L * a) { *k = t / a; *idx = t - *k * a; return true; }
    const int t1 = t - L * a;
    const int g1 = nz - L;                     // groups holding both kinds
    if (t1 < g1 * (a + b)) {
        const int g = t1 / (a + b);
        const int r = t1 - g * (a + b);
        if (r < a) { *k = g + L; *idx = r; return true; }
        *k = g; *idx = r - a; return false;
    }
    const int t2 = t1 - g1 * (a + b);
    *k = g1 + t2 / b;
    *idx = t2 - (t2 / b) * b;
    return false;
}

__device__ __forceinline__ int block_ticket(unsigned* ticket) {
    __shared__ int s_ticket;
    if (threadIdx.x == 0) s_ticket = (int)atomicAdd(ticket, 1u);
    __syncthreads();
    const int t = s_ticket;
    __syncthreads();
    return t;
}

// ---------------------------------------------------------------------------
// Forward task bodies
// ---------------------------------------------------------------------------
template <typename R, int N>
__device__ __forceinline__ void fwd_row_task(const ProjParams& p, int k, int j0, cplx<R>* Tl, cplx<R>* buf) {
    using C = cplx<R>;
    const int ny = p.ny, nz = p.nz;
    const int npair = p.rows_fwd / 2;
    const int bs = p.bs_row;
    const R* u = (const R*)p.u;
    const R* v = (const R*)p.v;
    const R* w = (const R*)p.w;
    const size_t plane = (size_t)ny * N;
    const R sv = (R)p.svol[k];
    const R rlo = (R)p.rflo[k];
    const R rhi = (R)p.rfhi[k];
    const R idx = (R)p.idx, idy = (R)p.idy;
    constexpr int LB = 4;
    const int tot = p.rows_fwd * N;
    const int step = LB * blockDim.x;
    for (int base = threadIdx.x; base < tot; base += step) {
        R uc[LB], um[LB], vc[LB], vm[LB], wl[LB], wh[LB];
#pragma unroll
        for (int c = 0; c < LB; ++c) {
            const int t = base + c * blockDim.x;
            uc[c] = um[c] = vc[c] = vm[c] = wl[c] = wh[c] = (R)0;
            if (t < tot) {
                const int r = t / N;
                const int i = t - r * N;
                const int j = j0 + r;
                if (j < ny) {
                    const size_t row = (size_t)k * plane + (size_t)j * N;
                    const size_t rowm = (size_t)k * plane + (size_t)(j == 0 ? ny - 1 : j - 1) * N;
                    const int im = (i == 0) ? N - 1 : i - 1;
                    uc[c] = u[row + i];
                    um[c] = u[row + im];
                    vc[c] = v[row + i];
                    vm[c] = v[rowm + i];
                    if (k > 0) wl[c] = w[row + i];
                    if (k < nz - 1) wh[c] = w[row + plane + i];
                }
            }
        }
#pragma unroll
        for (int c = 0; c < LB; ++c) {
            const int t = base + c * blockDim.x;
            if (t < tot) {
                const int r = t / N;
                const int i = t - r * N;
                const R hdiv = (uc[c] - um[c]) * idx + (vc[c] - vm[c]) * idy;
                const R d = sv * hdiv + (rhi * wh[c] - rlo * wl[c]);
                R* slot = (R*)&buf[(r >> 1) * bs + spad(i)];
                slot[r & 1] = d;
            }
        }
    }
    __syncthreads();
    CtFFT<R, N, 1, -1>::run(buf, npair, bs, ctab<R>(p.twx));
    const int nxh = p.nxh, nxp = p.nxp;
    const int tot2 = npair * nxh;
    for (int t = threadIdx.x; t < tot2; t += blockDim.x) {
        const int q = t / nxh;
        const int kx = t - q * nxh;
        const int j = j0 + 2 * q;
        const C z = buf[q * bs + spad(kx)];
        const C zc = cconj(buf[q * bs + spad(kx == 0 ? 0 : N - kx)]);
        const C a = cscale(cadd(z, zc), (R)0.5);
        const C dd = csub(z, zc);
        const C b = cmk<R>((R)0.5 * dd.y, (R)-0.5 * dd.x);
        if (j < ny) Tl[(size_t)j * nxp + kx] = a;
        if (j + 1 < ny) Tl[(size_t)(j + 1) * nxp + kx] = b;
    }
}

template <typename R, int N>
__device__ __forceinline__ void fwd_col_task(const ProjParams& p, int k, int kx0, const cplx<R>* Tl, cplx<R>* buf) {
    using C = cplx<R>;
    const int nxh = p.nxh, nxp = p.nxp, ny = p.ny;
    C* S = (C*)p.S;
    auto load = [&](int c, int j) -> C {
        const int kx = kx0 + c;
        return (kx < nxh) ? __ldcg(&Tl[(size_t)j * nxp + kx]) : cmk<R>((R)0, (R)0);
    };
    ct_first<R, N, -1, true>(buf, p.tw_cols, p.bs_col, load);
    CtMid<R, N, StageInfo<R, N, 1>::NEXT, -1>::run(buf, p.tw_cols, p.bs_col, ctab<R>(p.twy));
    auto store = [&](int c, int q, const C* x, int ns) {
        const int kx = kx0 + c;
        if (kx >= nxh) return;
        constexpr int RAD = StageInfo<R, N, LastNs<R, N>::value>::RAD;
#pragma unroll
        for (int r = 0; r < RAD; ++r) S[((size_t)k * ny + q + r * ns) * nxp + kx] = x[r];
    };
    ct_last<R, N, -1, true>(buf, p.tw_cols, p.bs_col, ctab<R>(p.twy), store);
}

template <typename R, int N>
__global__ void __launch_bounds__(256, 2) k_fwd_fused(ProjParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using C = cplx<R>;
    const int nz = p.nz, ny = p.ny, nxp = p.nxp;
    const int A = p.nrb_fwd, B = p.ntiles, ring = p.ring;
    unsigned* ticket = p.sync;
    unsigned* rows_done = p.sync + 2;
    unsigned* cols_done = rows_done + nz;
    const int ntotal = nz * (A + B);
    C* buf = (C*)smem_raw;
    C* T = (C*)p.T;
    while (true) {
        const int t = block_ticket(ticket);
        if (t >= ntotal) break;
        int k, idx;
        const bool is_row = decode_lagged(t, nz, p.lag, A, B, &k, &idx);
        C* Tl = T + (size_t)(k % ring) * ny * nxp;
        if (is_row) {
            if (k >= ring) block_wait(&cols_done[k - ring], (unsigned)B, p.err, p.spin_limit);
            fwd_row_task<R, N>(p, k, idx * p.rows_fwd, Tl, buf);
            block_signal(&rows_done[k]);
        } else {
            block_wait(&rows_done[k], (unsigned)A, p.err, p.spin_limit);
            fwd_col_task<R, N>(p, k, idx * p.tw_cols, Tl, buf);
            block_signal(&cols_done[k]);
        }
    }
}

// ---------------------------------------------------------------------------
// Inverse task bodies
// ---------------------------------------------------------------------------
// Column task: field f of a tile at level k into ring slot Tfl (see
// inv_col_field).  The tile is staged with cp.async in its global layout in
// the front of the FFT buffer, which the first stage then overwrites.
template <typename R, int N>
__device__ __forceinline__ void inv_col_task(const ProjParams& p, int k, int kx0, int f, cplx<R>* Tfl, cplx<R>* buf) {
    using C = cplx<R>;
    constexpr int CPC = 16 / (int)sizeof(C);
    const int tw = p.tw_cols, ny = p.ny, nxh = p.nxh, nxp = p.nxp;
    const InvColField<R> fd = inv_col_field<R>(p, f, k);
    const int cpr = tw / CPC;
    for (int c = threadIdx.x; c < N * cpr; c += blockDim.x) {
        const int j = c / cpr;
        const int part = c - j * cpr;
        const int kx = kx0 + part * CPC;
        C* dst = buf + j * tw + part * CPC;
        if (kx < nxp) cp_async16(dst, fd.src + ((size_t)k * ny + j) * nxp + kx);
        else {
#pragma unroll
            for (int e = 0; e < CPC; ++e) dst[e] = cmk<R>((R)0, (R)0);
        }
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    const C* ey = fd.ey;
    auto load = [&](int c, int j) -> C {
        const C v = buf[j * tw + c];
        return ey ? cmul(v, ey[j]) : v;
    };
    ct_first<R, N, 1, true, true>(buf, tw, p.bs_col, load);
    CtMid<R, N, StageInfo<R, N, 1>::NEXT, 1>::run(buf, tw, p.bs_col, ctab<R>(p.twy));
    const C* ex = ctab<R>(p.ex);
    const bool mul_ex = fd.ex;
    auto store = [&](int c, int q, const C* x, int ns) {
        const int kx = kx0 + c;
        if (kx >= nxh) return;
        constexpr int RAD = StageInfo<R, N, LastNs<R, N>::value>::RAD;
        const C e = mul_ex ? ex[kx] : cmk<R>((R)1, (R)0);
#pragma unroll
        for (int r = 0; r < RAD; ++r) Tfl[(size_t)(q + r * ns) * nxp + kx] = mul_ex ? cmul(x[r], e) : x[r];
    };
    ct_last<R, N, 1, true>(buf, tw, p.bs_col, ctab<R>(p.twy), store);
}

// Row task: channel ch of a block of rows at level k from ring slot Tcl.
template <typename R, int N>
__device__ __forceinline__ void inv_row_task(const ProjParams& p, int k, int j0, int ch, const cplx<R>* Tcl, cplx<R>* buf) {
    using C = cplx<R>;
    constexpr int NXH = N / 2 + 1;
    const int ny = p.ny, nz = p.nz, nxp = p.nxp;
    const size_t plane = (size_t)ny * N;
    const int npr = p.rows_inv / 2;
    R* out = (ch == 0) ? (R*)p.uo : (ch == 1) ? (R*)p.vo : (ch == 2) ? (R*)p.wo : (R*)p.phi;
    if (ch == 2 && k == 0) {
        for (int t = threadIdx.x; t < p.rows_inv * N; t += blockDim.x) {
            const int j = j0 + t / N;
            if (j < ny) {
                out[(size_t)j * N + (t % N)] = (R)0;
                if (nz == 1) out[plane + (size_t)j * N + (t % N)] = (R)0;
            }
        }
        return;
    }
    const R* in = (ch == 0) ? (const R*)p.u : (ch == 1) ? (const R*)p.v : (const R*)p.w;
    auto at = [&](int j, int kx) -> C {
        const bool neg = kx >= NXH;
        const int kk = neg ? N - kx : kx;
        C val = __ldcg(&Tcl[(size_t)j * nxp + kk]);
        if (kk == 0 || 2 * kk == N) val.y = (R)0;
        if (neg) val.y = -val.y;
        return val;
    };
    auto load = [&](int b, int kx) -> C {
        const int j = j0 + 2 * b;
        C a = cmk<R>((R)0, (R)0), c = cmk<R>((R)0, (R)0);
        if (j < ny) a = at(j, kx);
        if (j + 1 < ny) c = at(j + 1, kx);
        return cmk<R>(a.x - c.y, a.y + c.x);
    };
    ct_first<R, N, 1, false>(buf, npr, p.bs_row, load);
    CtMid<R, N, StageInfo<R, N, 1>::NEXT, 1>::run(buf, npr, p.bs_row, ctab<R>(p.twx));
    auto store = [&](int b, int q, const C* x, int ns) {
        constexpr int RAD = StageInfo<R, N, LastNs<R, N>::value>::RAD;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = j0 + 2 * b + h;
            if (j >= ny) continue;
            const size_t row = (size_t)k * plane + (size_t)j * N + q;
            R prev[RAD];
#pragma unroll
            for (int r = 0; r < RAD; ++r) prev[r] = (ch < 3) ? in[row + r * ns] : (R)0;
#pragma unroll
            for (int r = 0; r < RAD; ++r) {
                const R val = h ? x[r].y : x[r].x;
                out[row + r * ns] = (ch < 3) ? prev[r] - val : val;
                if (ch == 2 && k == nz - 1) out[row + r * ns + plane] = (R)0;
            }
        }
    };
    ct_last<R, N, 1, false>(buf, npr, p.bs_row, ctab<R>(p.twx), store);
}

template <typename R, int N>
__global__ void __launch_bounds__(256, 2) k_inv_fused(ProjParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using C = cplx<R>;
    const int nz = p.nz, ny = p.ny, nxp = p.nxp, nch = p.nch;
    const int A = p.ntiles * nch;             // column tasks per level (tile x field)
    const int B = p.nrb_inv * nch;            // row tasks per level (row block x channel)
    const int ring = p.ring;
    unsigned* ticket = p.sync + 1;
    unsigned* cols_done = p.sync + 2 + 2 * nz;          // [nz][4]
    unsigned* rows_done = cols_done + 4 * nz;           // [nz][4]
    const int ntotal = nz * (A + B);
    C* buf = (C*)smem_raw;
    C* arr[4] = {(C*)p.Tp, (C*)p.Tgy, (C*)p.Tgz, (C*)p.Tphi};
    while (true) {
        const int t = block_ticket(ticket);
        if (t >= ntotal) break;
        int k, idx;
        const bool is_col = decode_lagged(t, nz, p.lag, A, B, &k, &idx);
        const size_t slot = (size_t)(k % ring) * ny * nxp;
        if (is_col) {
            const int f = idx % nch;
            const int tile = idx / nch;
            if (k >= ring) block_wait(&rows_done[(k - ring) * 4 + f], (unsigned)p.nrb_inv, p.err, p.spin_limit);
            if (!(f == 2 && k == 0)) {
                C* dst = (f == 0) ? (C*)p.Tp : (f == 1) ? (C*)p.Tgy : (f == 2) ? (C*)p.Tgz : (C*)p.Tphi;
                inv_col_task<R, N>(p, k, tile * p.tw_cols, f, dst + slot, buf);
            }
            block_signal(&cols_done[k * 4 + f]);
        } else {
            const int ch = idx % nch;
            const int rb = idx / nch;
            block_wait(&cols_done[k * 4 + ch], (unsigned)p.ntiles, p.err, p.spin_limit);
            const C* src = (ch == 0) ? (const C*)p.Tp : (ch == 1) ? (const C*)p.Tgy
                         : (ch == 2) ? (const C*)p.Tgz : (const C*)p.Tphi;
            inv_row_task<R, N>(p, k, rb * p.rows_inv, ch, src + slot, buf);
            block_signal(&rows_done[k * 4 + ch]);
        }
        (void)arr;
    }
}

}  // namespace mp
