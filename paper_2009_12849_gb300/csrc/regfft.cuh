// Compile-time-sized DFTs held in registers, and compile-time twiddles.
//
// RegFFT<R, N, S> transforms x[0..N) (natural order in and out) with exponent
// sign S (-1 forward, +1 inverse).  N = 2, 3, 4, 5, 8 use the hand-written
// kernels of fft.cuh's base set; composite N = P*Q recurse by decimation in
// time: Q-point transforms of the P decimated sub-sequences, multiplication by
// W_N^{p q}, then P-point transforms across the sub-sequences.  Every index
// and every twiddle is a compile-time constant, so the arrays stay in
// registers and the twiddles become immediates.
#pragma once

namespace mp {

// ---------------------------------------------------------------------------
// constexpr cos / sin of 2 pi m / n.  The angle is reduced exactly (integer
// arithmetic) to [0, pi/4] and the Taylor series is summed there (terms up
// to x^25, truncation below 1e-25).
// ---------------------------------------------------------------------------
constexpr double ct_pi = 3.14159265358979323846264338327950288;

constexpr double ct_sin_small(double x) {
    double x2 = x * x, term = x, sum = x;
    for (int i = 1; i < 14; ++i) {
        term *= -x2 / (double)((2 * i) * (2 * i + 1));
        sum += term;
    }
    return sum;
}
constexpr double ct_cos_small(double x) {
    double x2 = x * x, term = 1.0, sum = 1.0;
    for (int i = 1; i < 14; ++i) {
        term *= -x2 / (double)((2 * i - 1) * (2 * i));
        sum += term;
    }
    return sum;
}
// cos(2 pi m/n) and sin(2 pi m/n)
constexpr double ct_cos2pi(long long m, long long n) {
    const long long mm = ((m % n) + n) % n;
    const long long q = (4 * mm) / n;           // quadrant
    const long long r = 4 * mm - q * n;         // (pi/2) r / n inside the quadrant
    const double c0 = (2 * r <= n) ? ct_cos_small(ct_pi / 2 * (double)r / (double)n)
                                   : ct_sin_small(ct_pi / 2 * (double)(n - r) / (double)n);
    const double s0 = (2 * r <= n) ? ct_sin_small(ct_pi / 2 * (double)r / (double)n)
                                   : ct_cos_small(ct_pi / 2 * (double)(n - r) / (double)n);
    return q == 0 ? c0 : q == 1 ? -s0 : q == 2 ? -c0 : s0;
}
constexpr double ct_sin2pi(long long m, long long n) {
    const long long mm = ((m % n) + n) % n;
    const long long q = (4 * mm) / n;
    const long long r = 4 * mm - q * n;
    const double c0 = (2 * r <= n) ? ct_cos_small(ct_pi / 2 * (double)r / (double)n)
                                   : ct_sin_small(ct_pi / 2 * (double)(n - r) / (double)n);
    const double s0 = (2 * r <= n) ? ct_sin_small(ct_pi / 2 * (double)r / (double)n)
                                   : ct_cos_small(ct_pi / 2 * (double)(n - r) / (double)n);
    return q == 0 ? s0 : q == 1 ? c0 : q == 2 ? -s0 : -c0;
}

// W_N^E with exponent sign S: exp(S 2 pi i E / N)
template <int N, int E, int S> struct CtTw {
    static constexpr double re = ct_cos2pi(E, N);
    static constexpr double im = S * ct_sin2pi(E, N);
};

// ---------------------------------------------------------------------------
// compile-time loops
// ---------------------------------------------------------------------------
template <int I> struct Ic {
    static constexpr int value = I;
    __host__ __device__ constexpr operator int() const { return I; }
};

template <int I, int E> struct SFor {
    template <class F> static MP_HD void run(F&& f) {
        f(Ic<I>{});
        SFor<I + 1, E>::run(f);
    }
};
template <int E> struct SFor<E, E> {
    template <class F> static MP_HD void run(F&&) {}
};

template <int N> struct FirstFactor {
    static constexpr int value = (N % 4 == 0 && N != 8) ? 4 : (N % 2 == 0) ? 2 : (N % 3 == 0) ? 3 : 5;
};

template <typename R, int N, int S> struct RegFFT {
    static_assert(N % FirstFactor<N>::value == 0, "unsupported length");
    static constexpr int P = FirstFactor<N>::value;
    static constexpr int Q = N / P;
    static MP_HD void run(cplx<R>* x) {
        cplx<R> sub[P][Q];
        SFor<0, P>::run([&](auto p) {
            SFor<0, Q>::run([&](auto m) { sub[p][m] = x[p + P * m]; });
            RegFFT<R, Q, S>::run(sub[p]);
        });
        SFor<0, Q>::run([&](auto q) {
            cplx<R> t[P];
            SFor<0, P>::run([&](auto p) {
                constexpr int e = (decltype(p)::value * decltype(q)::value) % N;
                if (e == 0) {
                    t[p] = sub[p][q];
                } else {
                    const R wr = (R)CtTw<N, e, S>::re;
                    const R wi = (R)CtTw<N, e, S>::im;
                    const cplx<R> v = sub[p][q];
                    t[p] = cmk<R>(v.x * wr - v.y * wi, v.x * wi + v.y * wr);
                }
            });
            RegFFT<R, P, S>::run(t);
            SFor<0, P>::run([&](auto s) { x[q + Q * s] = t[s]; });
        });
    }
};
template <typename R, int S> struct RegFFT<R, 1, S> { static MP_HD void run(cplx<R>*) {} };
template <typename R, int S> struct RegFFT<R, 2, S> { static MP_HD void run(cplx<R>* x) { Dft2<R, S>::run(x); } };
template <typename R, int S> struct RegFFT<R, 3, S> { static MP_HD void run(cplx<R>* x) { Dft3<R, S>::run(x); } };
template <typename R, int S> struct RegFFT<R, 4, S> { static MP_HD void run(cplx<R>* x) { Dft4<R, S>::run(x); } };
template <typename R, int S> struct RegFFT<R, 5, S> { static MP_HD void run(cplx<R>* x) { Dft5<R, S>::run(x); } };
template <typename R, int S> struct RegFFT<R, 8, S> { static MP_HD void run(cplx<R>* x) { Dft8<R, S>::run(x); } };

}  // namespace mp
