// Batched mixed-radix (2,3,4,5,8) complex FFT in shared memory.
//
// Steps a2 and a4 of the projection (paper, Section 4: a forward FFT on every
// level and a backward FFT) need length-nx transforms along x and length-ny
// transforms along y, n = 2^a 3^b 5^c.  Each transform lives in shared memory;
// the Stockham auto-sort formulation ping-pongs between two buffers so that
// every stage reads with unit stride across threads and no bit-reversal pass
// is needed.  One stage of radix R with Ns = product of the radices already
// applied processes n/R butterflies: butterfly q reads elements q + r n/R,
// multiplies element r by W_{Ns R}^{r (q mod Ns)}, takes a length-R DFT and
// writes element r to (q div Ns) Ns R + (q mod Ns) + r Ns.
#pragma once
#include <cuda_runtime.h>

namespace mp {

template <typename R> struct CT;
template <> struct CT<double> { using T = double2; };
template <> struct CT<float> { using T = float2; };
template <typename R> using cplx = typename CT<R>::T;

template <typename R> __device__ __forceinline__ cplx<R> cmk(R x, R y) { cplx<R> c; c.x = x; c.y = y; return c; }
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    C c; c.x = a.x * b.x - a.y * b.y; c.y = a.x * b.y + a.y * b.x; return c;
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
    C c; c.x = a.x * b.x + a.y * b.y; c.y = a.y * b.x - a.x * b.y; return c;
}
template <typename C, typename R> __device__ __forceinline__ C cscale(C a, R s) { a.x *= s; a.y *= s; return a; }
template <typename C> __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
// multiply by s*i, s = +1 or -1
template <typename C> __device__ __forceinline__ C cmul_si(C a, int s) {
    C c; if (s > 0) { c.x = -a.y; c.y = a.x; } else { c.x = a.y; c.y = -a.x; } return c;
}

// Radix plan of one transform length.
struct FftFactors {
    int n;
    int nstages;
    int radix[24];
};

// Length-R DFTs on registers, exponent sign S (-1 forward, +1 inverse).
template <typename R, int S> struct Dft2 {
    static __device__ __forceinline__ void run(cplx<R>* x) {
        cplx<R> a = x[0], b = x[1];
        x[0] = cadd(a, b); x[1] = csub(a, b);
    }
};
template <typename R, int S> struct Dft4 {
    static __device__ __forceinline__ void run(cplx<R>* x) {
        cplx<R> s02 = cadd(x[0], x[2]), d02 = csub(x[0], x[2]);
        cplx<R> s13 = cadd(x[1], x[3]), d13 = cmul_si(csub(x[1], x[3]), S);
        x[0] = cadd(s02, s13); x[2] = csub(s02, s13);
        x[1] = cadd(d02, d13); x[3] = csub(d02, d13);
    }
};
template <typename R, int S> struct Dft8 {
    static __device__ __forceinline__ void run(cplx<R>* x) {
        const R h = (R)0.70710678118654752440;   // 1/sqrt(2)
        cplx<R> e[4] = {x[0], x[2], x[4], x[6]};
        cplx<R> o[4] = {x[1], x[3], x[5], x[7]};
        Dft4<R, S>::run(e);
        Dft4<R, S>::run(o);
        // twiddles w8^k, w8 = (1 + S i)/sqrt(2)
        cplx<R> o1 = cmk<R>(h * (o[1].x - S * o[1].y), h * (o[1].y + S * o[1].x));
        cplx<R> o2 = cmul_si(o[2], S);
        cplx<R> o3 = cmk<R>(h * (-o[3].x - S * o[3].y), h * (-o[3].y + S * o[3].x));
        x[0] = cadd(e[0], o[0]); x[4] = csub(e[0], o[0]);
        x[1] = cadd(e[1], o1);   x[5] = csub(e[1], o1);
        x[2] = cadd(e[2], o2);   x[6] = csub(e[2], o2);
        x[3] = cadd(e[3], o3);   x[7] = csub(e[3], o3);
    }
};
template <typename R, int S> struct Dft3 {
    static __device__ __forceinline__ void run(cplx<R>* x) {
        const R c = (R)0.86602540378443864676;   // sqrt(3)/2
        cplx<R> t = cadd(x[1], x[2]);
        cplx<R> d = csub(x[1], x[2]);
        cplx<R> m = cmk<R>(x[0].x - (R)0.5 * t.x, x[0].y - (R)0.5 * t.y);
        cplx<R> r = cscale(cmul_si(d, S), c);
        x[0] = cadd(x[0], t);
        x[1] = cadd(m, r);
        x[2] = csub(m, r);
    }
};
template <typename R, int S> struct Dft5 {
    static __device__ __forceinline__ void run(cplx<R>* x) {
        const R c1 = (R)0.30901699437494742410;    // cos(2 pi/5) = (sqrt5-1)/4
        const R c2 = (R)-0.80901699437494742410;   // cos(4 pi/5) = -(sqrt5+1)/4
        const R s1 = (R)0.95105651629515357212;    // sin(2 pi/5)
        const R s2 = (R)0.58778525229247312917;    // sin(4 pi/5)
        cplx<R> t1 = cadd(x[1], x[4]), t2 = cadd(x[2], x[3]);
        cplx<R> d1 = csub(x[1], x[4]), d2 = csub(x[2], x[3]);
        cplx<R> a1 = cmk<R>(x[0].x + c1 * t1.x + c2 * t2.x, x[0].y + c1 * t1.y + c2 * t2.y);
        cplx<R> a2 = cmk<R>(x[0].x + c2 * t1.x + c1 * t2.x, x[0].y + c2 * t1.y + c1 * t2.y);
        cplx<R> b1 = cmul_si(cmk<R>(s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y), S);
        cplx<R> b2 = cmul_si(cmk<R>(s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y), S);
        x[0] = cadd(x[0], cadd(t1, t2));
        x[1] = cadd(a1, b1); x[4] = csub(a1, b1);
        x[2] = cadd(a2, b2); x[3] = csub(a2, b2);
    }
};

template <typename R, int RAD, int S> struct DftSel;
template <typename R, int S> struct DftSel<R, 2, S> { using T = Dft2<R, S>; };
template <typename R, int S> struct DftSel<R, 3, S> { using T = Dft3<R, S>; };
template <typename R, int S> struct DftSel<R, 4, S> { using T = Dft4<R, S>; };
template <typename R, int S> struct DftSel<R, 5, S> { using T = Dft5<R, S>; };
template <typename R, int S> struct DftSel<R, 8, S> { using T = Dft8<R, S>; };

// One Stockham stage over `nb` transforms: element e of transform b sits at
// base[b*bstride + e].  tw[m] = exp(-2 pi i m / n).
template <typename R, int RAD, int S>
__device__ __forceinline__ void fft_stage(const cplx<R>* __restrict__ in, cplx<R>* __restrict__ out,
                                          int n, int Ns, int nb, int bstride,
                                          const cplx<R>* __restrict__ tw) {
    const int nq = n / RAD;
    const int total = nq * nb;
    const int tstep = n / (Ns * RAD);
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int b = t / nq;
        const int q = t - b * nq;
        const int k = q % Ns;
        const cplx<R>* src = in + b * bstride + q;
        cplx<R> x[RAD];
#pragma unroll
        for (int r = 0; r < RAD; ++r) x[r] = src[r * nq];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < RAD; ++r) {
                cplx<R> wv = tw[r * k * tstep];
                x[r] = (S < 0) ? cmul(x[r], wv) : cmulc(x[r], wv);
            }
        }
        DftSel<R, RAD, S>::T::run(x);
        cplx<R>* dst = out + b * bstride + (q / Ns) * Ns * RAD + k;
#pragma unroll
        for (int r = 0; r < RAD; ++r) dst[r * Ns] = x[r];
    }
}

// Full transform of nb sequences.  `a` holds the input; `b` is scratch of the
// same size.  Returns the buffer that holds the result.  Every thread of the
// block must call this (it synchronises between stages).
template <typename R, int S>
__device__ cplx<R>* fft_batch(cplx<R>* a, cplx<R>* b, int nb, int bstride,
                              const FftFactors& f, const cplx<R>* __restrict__ tw) {
    int Ns = 1;
    for (int s = 0; s < f.nstages; ++s) {
        const int rad = f.radix[s];
        switch (rad) {
            case 8: fft_stage<R, 8, S>(a, b, f.n, Ns, nb, bstride, tw); break;
            case 4: fft_stage<R, 4, S>(a, b, f.n, Ns, nb, bstride, tw); break;
            case 2: fft_stage<R, 2, S>(a, b, f.n, Ns, nb, bstride, tw); break;
            case 5: fft_stage<R, 5, S>(a, b, f.n, Ns, nb, bstride, tw); break;
            default: fft_stage<R, 3, S>(a, b, f.n, Ns, nb, bstride, tw); break;
        }
        __syncthreads();
        cplx<R>* t = a; a = b; b = t;
        Ns *= rad;
    }
    return a;
}

}  // namespace mp
