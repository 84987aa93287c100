// Kernels of one anelastic projection (paper, Section 4: forward FFT, a
// vertical ODE per horizontal wavenumber in Fourier space, backward FFT),
// with the divergence (step a1) fused into the forward transform and the
// pressure-gradient correction (step a5) fused into the inverse transform.
//
// Layouts (element = one complex value of the storage precision R):
//   spectral arrays  S, G, T, Tp, Tgy, Tgz : [nz][ny][nxp], kx < nxh valid
//   u, v, phi        : [nz][ny][nx] real;   w : [nz+1][ny][nx] real
#pragma once
#include "fft.cuh"

namespace mp {

struct ProjParams {
    int nx, ny, nz, nxh, nxp;
    FftFactors fx, fy;
    const void* twx;            // [nx] exp(-2 pi i m/nx), storage precision
    const void* twy;            // [ny]
    const double* svol;         // [nz]   rho_c[k] dz[k]
    const double* rflo;         // [nz]   rho_f[k]   (0 at k = 0)
    const double* rfhi;         // [nz]   rho_f[k+1] (0 at k = nz-1)
    const double* acoef;        // [nz+1] A[k] = rho_f[k]/dzn[k], A[0] = A[nz] = 0
    const double* idzn;         // [nz+1] 1/dzn[k] (0 at k = 0, nz)
    const double* lamx;         // [nxh]  2(cos(2 pi kx/nx) - 1)/dx^2
    const double* lamy;         // [ny]
    const void* ex;             // [nxh]  (exp(2 pi i kx/nx) - 1)/dx, storage precision
    const void* ey;             // [ny]
    double idx, idy;            // 1/dx, 1/dy
    double scale;               // 1/(nx ny)
    // fields
    const void* u; const void* v; const void* w;
    void* uo; void* vo; void* wo; void* phi;
    // workspace
    void* S; void* G; void* T; void* Tp; void* Tgy; void* Tgz;
    double2* Y; double* Gp;
    int* err;
    // task shapes
    int rows_fwd;               // real rows per forward row task (even)
    int nrb_fwd;                // row tasks per level (forward)
    int rows_inv;               // real rows per inverse row task
    int nrb_inv;
    int nch;                    // real channels per row in the inverse (3, or 4 with phi)
    int tw_cols;                // kx columns per column task
    int ntiles;                 // column tasks per level
    int bs_row;                 // smem stride of a row transform (complex elements)
    int bs_col;                 // smem stride of a column transform
};

template <typename R> __device__ __forceinline__ const cplx<R>* ctab(const void* p) { return (const cplx<R>*)p; }

// ---------------------------------------------------------------------------
// a1 + a2 (x part): divergence of a block of rows, real FFT along x.
// Two real rows share one complex transform: z = d_j + i d_{j+1}; after the
// transform X_j[k] = (Z[k] + conj Z[n-k])/2, X_{j+1}[k] = (Z[k] - conj Z[n-k])/(2i).
// Output is the level's x-spectrum in T, scaled by rho_c dz (the symmetric
// form of the vertical operator).
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256) k_fwd_rows(ProjParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using C = cplx<R>;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int nrb = p.nrb_fwd;
    const int k = blockIdx.x / nrb;
    const int j0 = (blockIdx.x - k * nrb) * p.rows_fwd;
    const int npair = p.rows_fwd / 2;
    const int bs = p.bs_row;
    C* bufA = (C*)smem_raw;
    C* bufB = bufA + npair * bs;

    const R* u = (const R*)p.u;
    const R* v = (const R*)p.v;
    const R* w = (const R*)p.w;
    const size_t plane = (size_t)ny * nx;
    const R sv = (R)p.svol[k];
    const R rlo = (R)p.rflo[k];
    const R rhi = (R)p.rfhi[k];
    const R idx = (R)p.idx, idy = (R)p.idy;

    const int tot = p.rows_fwd * nx;
    for (int t = threadIdx.x; t < tot; t += blockDim.x) {
        const int r = t / nx;
        const int i = t - r * nx;
        const int j = j0 + r;
        R d = (R)0;
        if (j < ny) {
            const size_t row = (size_t)k * plane + (size_t)j * nx;
            const size_t rowm = (size_t)k * plane + (size_t)(j == 0 ? ny - 1 : j - 1) * nx;
            const int im = (i == 0) ? nx - 1 : i - 1;
            R hdiv = (u[row + i] - u[row + im]) * idx + (v[row + i] - v[rowm + i]) * idy;
            R wl = (k > 0) ? w[row + i] : (R)0;
            R wh = (k < nz - 1) ? w[row + plane + i] : (R)0;
            d = sv * hdiv + (rhi * wh - rlo * wl);
        }
        R* slot = (R*)&bufA[(r >> 1) * bs + i];
        slot[r & 1] = d;
    }
    __syncthreads();
    C* res = fft_batch<R, -1>(bufA, bufB, npair, bs, p.fx, ctab<R>(p.twx));

    C* T = (C*)p.T;
    const int nxh = p.nxh;
    const int tot2 = npair * nxh;
    for (int t = threadIdx.x; t < tot2; t += blockDim.x) {
        const int q = t / nxh;
        const int kx = t - q * nxh;
        const int j = j0 + 2 * q;
        C z = res[q * bs + kx];
        C zc = cconj(res[q * bs + (kx == 0 ? 0 : nx - kx)]);
        C a = cscale(cadd(z, zc), (R)0.5);
        C dd = csub(z, zc);
        C b = cmk<R>((R)0.5 * dd.y, (R)-0.5 * dd.x);
        const size_t o = ((size_t)k * ny + j) * p.nxp + kx;
        if (j < ny) T[o] = a;
        if (j + 1 < ny) T[o + p.nxp] = b;
    }
}

// ---------------------------------------------------------------------------
// Column transforms along y for a tile of kx columns of one level.
// DIR = -1: forward (T -> S).  The inverse uses k_inv_cols.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void load_cols(cplx<R>* buf, const cplx<R>* src, int k, int kx0, const ProjParams& p,
                                          const cplx<R>* mul_y) {
    const int tw = p.tw_cols, ny = p.ny, bs = p.bs_col;
    const int tot = ny * tw;
    for (int t = threadIdx.x; t < tot; t += blockDim.x) {
        const int j = t / tw;
        const int c = t - j * tw;
        const int kx = kx0 + c;
        cplx<R> val = cmk<R>((R)0, (R)0);
        if (kx < p.nxh) {
            val = src[((size_t)k * ny + j) * p.nxp + kx];
            if (mul_y) val = cmul(val, mul_y[j]);
        }
        buf[c * bs + j] = val;
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
        if (kx < p.nxh) dst[((size_t)k * ny + j) * p.nxp + kx] = buf[c * bs + j];
    }
}

template <typename R>
__global__ void __launch_bounds__(256) k_fwd_cols(ProjParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using C = cplx<R>;
    const int k = blockIdx.x / p.ntiles;
    const int kx0 = (blockIdx.x - k * p.ntiles) * p.tw_cols;
    C* bufA = (C*)smem_raw;
    C* bufB = bufA + p.tw_cols * p.bs_col;
    load_cols<R>(bufA, (const C*)p.T, k, kx0, p, nullptr);
    __syncthreads();
    C* res = fft_batch<R, -1>(bufA, bufB, p.tw_cols, p.bs_col, p.fy, ctab<R>(p.twy));
    store_cols<R>((C*)p.S, res, k, kx0, p);
}

// ---------------------------------------------------------------------------
// a3: vertical tridiagonal problem per (kx, ky), one thread per column, FP64.
// Symmetric form (rows multiplied by rho_c dz):
//   A[k] p[k-1] + b[k] p[k] + A[k+1] p[k+1] = D'[k],  b[k] = lambda s[k] - A[k] - A[k+1]
// Forward: e = b - A^2/e_prev, y = D' - (A/e_prev) y_prev.  Back:
// p[k] = (y[k] - A[k+1] p[k+1]) / e[k].  The (0,0) column pins p[0] = 0.
// Writes p^ and the spectral w-gradient (p[k]-p[k-1])/dzn[k], both scaled
// by 1/(nx ny) for the inverse transform.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(128) k_tridiag(ProjParams p) {
    using C = cplx<R>;
    const int ncol = p.ny * p.nxh;
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= ncol) return;
    const int ky = col / p.nxh;
    const int kx = col - ky * p.nxh;
    const size_t LS = (size_t)p.ny * p.nxp;
    const size_t base = (size_t)ky * p.nxp + kx;
    const int nz = p.nz;
    C* S = (C*)p.S;
    C* G = (C*)p.G;
    const double lam = p.lamx[kx] + p.lamy[ky];
    const bool mean = (kx == 0 && ky == 0);
    const int k0 = mean ? 1 : 0;
    const double scale = p.scale;

    if (k0 < nz) {
        double g = 0.0;
        double2 y = make_double2(0.0, 0.0);
        for (int k = k0; k < nz; ++k) {
            const double ak = (k > k0) ? p.acoef[k] : 0.0;
            const double b = lam * p.svol[k] - p.acoef[k] - p.acoef[k + 1];
            const double m = ak * g;
            const double e = b - ak * m;
            g = 1.0 / e;
            C dv = S[k * LS + base];
            y.x = (double)dv.x - m * y.x;
            y.y = (double)dv.y - m * y.y;
            p.Y[k * LS + base] = y;
            p.Gp[k * LS + base] = g;
        }
        double2 ph = make_double2(y.x * g, y.y * g);
        S[(nz - 1) * LS + base] = cmk<R>((R)(ph.x * scale), (R)(ph.y * scale));
        for (int k = nz - 2; k >= k0; --k) {
            const double a1 = p.acoef[k + 1];
            const double2 yk = p.Y[k * LS + base];
            const double gk = p.Gp[k * LS + base];
            double2 pn = make_double2((yk.x - a1 * ph.x) * gk, (yk.y - a1 * ph.y) * gk);
            const double iz = p.idzn[k + 1] * scale;
            G[(k + 1) * LS + base] = cmk<R>((R)((ph.x - pn.x) * iz), (R)((ph.y - pn.y) * iz));
            S[k * LS + base] = cmk<R>((R)(pn.x * scale), (R)(pn.y * scale));
            ph = pn;
        }
        if (mean) {
            // p[0] = 0 (the pin); face 1 gradient from p[1] - 0.
            const double iz = p.idzn[1] * scale;
            G[LS + base] = cmk<R>((R)(ph.x * iz), (R)(ph.y * iz));
        }
    }
    if (mean) S[base] = cmk<R>((R)0, (R)0);
}

// ---------------------------------------------------------------------------
// a4 (y part): inverse y-transforms of one level's tile:
//   Tp  = IFFT_y(p^),  Tgy = IFFT_y(p^ * ey),  Tgz = IFFT_y(gz^)  (gz^ not at k = 0)
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256) k_inv_cols(ProjParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using C = cplx<R>;
    const int k = blockIdx.x / p.ntiles;
    const int kx0 = (blockIdx.x - k * p.ntiles) * p.tw_cols;
    C* bufA = (C*)smem_raw;
    C* bufB = bufA + p.tw_cols * p.bs_col;
    const C* ey = ctab<R>(p.ey);
    for (int f = 0; f < 3; ++f) {
        if (f == 2 && k == 0) break;
        const C* src = (f == 2) ? (const C*)p.G : (const C*)p.S;
        C* dst = (f == 0) ? (C*)p.Tp : (f == 1) ? (C*)p.Tgy : (C*)p.Tgz;
        load_cols<R>(bufA, src, k, kx0, p, f == 1 ? ey : nullptr);
        __syncthreads();
        C* res = fft_batch<R, 1>(bufA, bufB, p.tw_cols, p.bs_col, p.fy, ctab<R>(p.twy));
        store_cols<R>(dst, res, k, kx0, p);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// a4 (x part) + a5: inverse real transforms along x of the gradient
// channels of a block of rows, then u -= gx, v -= gy, w -= gz (w = 0 on the
// bottom and top faces) and optionally phi.  Channels of a row:
//   0: Tp * ex (x-gradient)   1: Tgy (y-gradient)   2: Tgz (z-gradient)   3: Tp (phi)
// One complex transform carries one channel of two adjacent rows,
// Z = A_j + i A_{j+1} with Hermitian-extended A; the real part of the inverse
// is row j, the imaginary part row j+1.  Channels are never mixed in one
// transform: phi is dominated by its largest scales and would otherwise put
// its rounding error into a gradient channel.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ cplx<R> inv_spectrum(const ProjParams& p, int k, int j, int ch, int kx) {
    using C = cplx<R>;
    if (j >= p.ny || (ch == 2 && k == 0)) return cmk<R>((R)0, (R)0);
    const int nx = p.nx;
    const bool neg = kx >= p.nxh;
    const int kk = neg ? nx - kx : kx;
    const C* src = (ch == 1) ? (const C*)p.Tgy : (ch == 2) ? (const C*)p.Tgz : (const C*)p.Tp;
    C val = src[((size_t)k * p.ny + j) * p.nxp + kk];
    if (ch == 0) val = cmul(val, ctab<R>(p.ex)[kk]);
    if (kk == 0 || 2 * kk == nx) val.y = (R)0;      // real-only DC / Nyquist
    if (neg) val.y = -val.y;
    return val;
}

template <typename R>
__global__ void __launch_bounds__(256) k_inv_rows(ProjParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using C = cplx<R>;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int nrb = p.nrb_inv;
    const int k = blockIdx.x / nrb;
    const int j0 = (blockIdx.x - k * nrb) * p.rows_inv;
    const int nch = p.nch;
    const int npr = p.rows_inv / 2;          // row pairs per task
    const int np = nch * npr;                // complex transforms per task
    const int bs = p.bs_row;
    C* bufA = (C*)smem_raw;
    C* bufB = bufA + np * bs;

    const int tot = np * nx;
    for (int t = threadIdx.x; t < tot; t += blockDim.x) {
        const int q = t / nx;
        const int kx = t - q * nx;
        const int ch = q / npr;
        const int m = q - ch * npr;
        const int j = j0 + 2 * m;
        C a = inv_spectrum<R>(p, k, j, ch, kx);
        C b = inv_spectrum<R>(p, k, j + 1, ch, kx);
        bufA[q * bs + kx] = cmk<R>(a.x - b.y, a.y + b.x);
    }
    __syncthreads();
    C* res = fft_batch<R, 1>(bufA, bufB, np, bs, p.fx, ctab<R>(p.twx));

    const R* u = (const R*)p.u;
    const R* v = (const R*)p.v;
    const R* w = (const R*)p.w;
    R* uo = (R*)p.uo;
    R* vo = (R*)p.vo;
    R* wo = (R*)p.wo;
    R* ph = (R*)p.phi;
    const size_t plane = (size_t)ny * nx;
    const int tot2 = p.rows_inv * nx;
    for (int t = threadIdx.x; t < tot2; t += blockDim.x) {
        const int r = t / nx;
        const int i = t - r * nx;
        const int j = j0 + r;
        if (j >= ny) continue;
        const int m = r >> 1;
        R val[4];
#pragma unroll
        for (int ch = 0; ch < 4; ++ch) {
            if (ch < nch) {
                const C z = res[(ch * npr + m) * bs + i];
                val[ch] = (r & 1) ? z.y : z.x;
            }
        }
        const size_t o = (size_t)k * plane + (size_t)j * nx + i;
        uo[o] = u[o] - val[0];
        vo[o] = v[o] - val[1];
        wo[o] = (k == 0) ? (R)0 : (R)(w[o] - val[2]);
        if (k == nz - 1) wo[o + plane] = (R)0;
        if (nch == 4) ph[o] = val[3];
    }
}

}  // namespace mp
