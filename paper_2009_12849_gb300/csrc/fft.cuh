// Batched mixed-radix (2,3,4,5,8,16,32) complex FFT in shared memory.
//
// Steps a2 and a4 of the projection (paper, Section 4: a forward FFT on every
// level and a backward FFT) need length-nx transforms along x and length-ny
// transforms along y, n = 2^a 3^b 5^c.  Each transform lives in shared memory;
// the Stockham auto-sort formulation ping-pongs between two buffers so that
// every stage reads with unit stride across threads and no bit-reversal pass
// is needed.  One stage of radix R with Ns = product of the radices already
// applied processes n/R butterflies: butterfly q reads elements q + r n/R,
// multiplies element r by W_{Ns R}^{r (q mod Ns)}, takes a length-R DFT and
// writes element r to (q div Ns) Ns R + (q mod Ns) + r Ns.  Radices 16 and 32
// run as compile-time register DFTs (regfft.cuh), so a length-1024 transform
// takes two passes through shared memory.
#pragma once
#include <cuda_runtime.h>

#define MP_HD __host__ __device__ __forceinline__

namespace mp {

template <typename R> struct CT;
template <> struct CT<double> { using T = double2; };
template <> struct CT<float> { using T = float2; };
template <typename R> using cplx = typename CT<R>::T;

template <typename R> MP_HD cplx<R> cmk(R x, R y) { cplx<R> c; c.x = x; c.y = y; return c; }
template <typename C> MP_HD C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> MP_HD C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C> MP_HD C cmul(C a, C b) {
    C c; c.x = a.x * b.x - a.y * b.y; c.y = a.x * b.y + a.y * b.x; return c;
}
// a * conj(b)
template <typename C> MP_HD C cmulc(C a, C b) {
    C c; c.x = a.x * b.x + a.y * b.y; c.y = a.y * b.x - a.x * b.y; return c;
}
template <typename C, typename R> MP_HD C cscale(C a, R s) { a.x *= s; a.y *= s; return a; }
template <typename C> MP_HD C cconj(C a) { a.y = -a.y; return a; }
// multiply by s*i, s = +1 or -1
template <typename C> MP_HD C cmul_si(C a, int s) {
    C c; if (s > 0) { c.x = -a.y; c.y = a.x; } else { c.x = a.y; c.y = -a.x; } return c;
}

// FP32 complex values on sm_100 and later: the two parts of an add, subtract
// or real scale go through one paired-FP32 instruction (add/sub/mul .f32x2 on
// the register pair holding the value), halving the instructions of the
// butterflies' additions.  Each lane rounds as the scalar operation would.
#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 1000) && !defined(MP_SCALAR_F32)
#define MP_PAIRED_F32 1
__device__ __forceinline__ unsigned long long f2bits(float2 a) {
    return ((unsigned long long)__float_as_uint(a.y) << 32) | __float_as_uint(a.x);
}
__device__ __forceinline__ float2 bits2f(unsigned long long b) {
    return make_float2(__uint_as_float((unsigned)b), __uint_as_float((unsigned)(b >> 32)));
}
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2bits(a)), "l"(f2bits(b)));
    return bits2f(d);
}
#endif
MP_HD float2 cadd(float2 a, float2 b) {
#ifdef MP_PAIRED_F32
    return __fadd2_rn(a, b);
#else
    a.x += b.x; a.y += b.y; return a;
#endif
}
MP_HD float2 csub(float2 a, float2 b) {
#ifdef MP_PAIRED_F32
    return f2sub(a, b);
#else
    a.x -= b.x; a.y -= b.y; return a;
#endif
}
MP_HD float2 cscale(float2 a, float s) {
#ifdef MP_PAIRED_F32
    return __fmul2_rn(a, make_float2(s, s));
#else
    a.x *= s; a.y *= s; return a;
#endif
}

// Length-R DFTs on registers, exponent sign S (-1 forward, +1 inverse).
template <typename R, int S> struct Dft2 {
    static MP_HD void run(cplx<R>* x) {
        cplx<R> a = x[0], b = x[1];
        x[0] = cadd(a, b); x[1] = csub(a, b);
    }
};
template <typename R, int S> struct Dft4 {
    static MP_HD void run(cplx<R>* x) {
        cplx<R> s02 = cadd(x[0], x[2]), d02 = csub(x[0], x[2]);
        cplx<R> s13 = cadd(x[1], x[3]), d13 = cmul_si(csub(x[1], x[3]), S);
        x[0] = cadd(s02, s13); x[2] = csub(s02, s13);
        x[1] = cadd(d02, d13); x[3] = csub(d02, d13);
    }
};
template <typename R, int S> struct Dft8 {
    static MP_HD void run(cplx<R>* x) {
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
    static MP_HD void run(cplx<R>* x) {
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
    static MP_HD void run(cplx<R>* x) {
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

}  // namespace mp

#include "regfft.cuh"

namespace mp {

// Division by a run-time constant d as a multiply-high and shift (the
// round-up method of Granlund and Montgomery, "Division by invariant integers
// using multiplication", 1994): q = (umulhi(t, m) + t) >> s with
// s = ceil(log2 d), m = floor(2^32 (2^s - d) / d) + 1, exact for t < 2^31.
struct FastDiv {
    unsigned m, s;
};
__device__ __forceinline__ unsigned fdiv(unsigned t, FastDiv f) { return (__umulhi(t, f.m) + t) >> f.s; }

// One Stockham stage: radix R applied with Ns = product of the earlier radices.
struct FftStage {
    int radix, ns, nq;           // nq = n / R
    FastDiv fq, fns;             // division by nq and by Ns
};

// Radix plan of one transform length (largest radices first).
struct FftFactors {
    int n;
    int nstages;
    FftStage st[16];
};

// Shared-memory index of element i of a transform: one pad element every 32
// keeps the stride-R accesses of the first stages free of bank conflicts.
__device__ __forceinline__ int spad(int i) { return i + (i >> 5); }
__host__ __device__ inline int spad_len(int n) { return n + (n >> 5) + 1; }
// spad(i0 + r * STRIDE) for i0 >= 0: with STRIDE a multiple of 32 it is
// spad(i0) + r * (STRIDE + STRIDE / 32), so a butterfly's RAD accesses are one
// index computation plus compile-time offsets.
template <int STRIDE>
__device__ __forceinline__ int spad_at(int sp0, int i0, int r) {
    if constexpr (STRIDE % 32 == 0) return sp0 + r * (STRIDE + STRIDE / 32);
    else return spad(i0 + r * STRIDE);
}

// Twiddle tables: stage s of a length-n plan owns entries [s*n, s*n + R*Ns)
// of the plan's table, laid out [r][k]: entry r*Ns + k = W_{Ns R}^{r k}, so
// that threads with consecutive k read consecutive entries.
//
// One Stockham stage over `nb` transforms: element e of transform b sits at
// base[b*bstride + spad(e)]; tw points at this stage's table.
template <typename R, int RAD, int S>
__device__ __forceinline__ void fft_stage(const cplx<R>* __restrict__ in, cplx<R>* __restrict__ out,
                                          const FftStage& st, int nb, int bstride,
                                          const cplx<R>* __restrict__ tw) {
    const int nq = st.nq, Ns = st.ns;
    const int total = nq * nb;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int b = (int)fdiv((unsigned)t, st.fq);
        const int q = t - b * nq;
        const int qd = (int)fdiv((unsigned)q, st.fns);
        const int k = q - qd * Ns;
        const cplx<R>* src = in + b * bstride;
        cplx<R> x[RAD];
#pragma unroll
        for (int r = 0; r < RAD; ++r) x[r] = src[spad(q + r * nq)];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < RAD; ++r) {
                const cplx<R> wv = __ldg(&tw[r * Ns + k]);
                x[r] = (S < 0) ? cmul(x[r], wv) : cmulc(x[r], wv);
            }
        }
        RegFFT<R, RAD, S>::run(x);
        cplx<R>* dst = out + b * bstride;
        const int base = qd * Ns * RAD + k;
#pragma unroll
        for (int r = 0; r < RAD; ++r) dst[spad(base + r * Ns)] = x[r];
    }
}

// Full transform of nb sequences.  `a` holds the input; `b` is scratch of the
// same size.  Returns the buffer that holds the result.  Every thread of the
// block must call this (it synchronises between stages).
template <typename R, int S>
__device__ cplx<R>* fft_batch(cplx<R>* a, cplx<R>* b, int nb, int bstride,
                              const FftFactors& f, const cplx<R>* __restrict__ tw) {
    for (int s = 0; s < f.nstages; ++s) {
        const FftStage& st = f.st[s];
        switch (st.radix) {
            case 32:
                if constexpr (sizeof(R) == 4) fft_stage<R, 32, S>(a, b, st, nb, bstride, tw + s * f.n);
                break;
            case 16: fft_stage<R, 16, S>(a, b, st, nb, bstride, tw + s * f.n); break;
            case 8: fft_stage<R, 8, S>(a, b, st, nb, bstride, tw + s * f.n); break;
            case 4: fft_stage<R, 4, S>(a, b, st, nb, bstride, tw + s * f.n); break;
            case 2: fft_stage<R, 2, S>(a, b, st, nb, bstride, tw + s * f.n); break;
            case 5: fft_stage<R, 5, S>(a, b, st, nb, bstride, tw + s * f.n); break;
            default: fft_stage<R, 3, S>(a, b, st, nb, bstride, tw + s * f.n); break;
        }
        __syncthreads();
        cplx<R>* t = a; a = b; b = t;
    }
    return a;
}

// Thread scope of a compile-time transform: the whole block (threads of the
// block cooperate on its transforms and synchronise with __syncthreads), or
// one warp (a warp transforms its own sequences in its own shared-memory
// slice and synchronises with __syncwarp; the persistent pipeline kernels run
// row transforms this way, eight independent warps to a block).
struct BlockScope {
    static __device__ __forceinline__ int tid() { return threadIdx.x; }
    static __device__ __forceinline__ int size() { return blockDim.x; }
    static __device__ __forceinline__ void sync() { __syncthreads(); }
};
struct WarpScope {
    static __device__ __forceinline__ int tid() { return threadIdx.x & 31; }
    static __device__ __forceinline__ int size() { return 32; }
    static __device__ __forceinline__ void sync() { __syncwarp(); }
};

// ---------------------------------------------------------------------------
// Compile-time plans for the common lengths.  Every stage's radix, Ns, n/R
// and twiddle stride are constants; every thread holds at most E elements of
// a stage (its ceil(E/R) butterflies) in registers, the block synchronises,
// and the outputs overwrite the inputs in the single shared buffer.  The
// caller sizes the block so that blockDim.x * E >= nb * N.
// ---------------------------------------------------------------------------
// Largest radix of the compile-time plans, which is also the number of
// elements a thread holds in a stage (FP32, FP64).
constexpr int kMaxRadixF32 = 32;
constexpr int kMaxRadixF64 = 16;
template <typename R> struct ElemsPerThread { static constexpr int value = sizeof(R) == 4 ? kMaxRadixF32 : kMaxRadixF64; };

// Radix of the next compile-time stage for the remaining length M with E
// elements per thread: the largest power of two from 8 to E that divides M;
// else the largest divisor d <= E whose ceil(E/d) butterflies per thread
// hold at most E + E/2 elements (so lengths with factors 3 and 5 take few,
// composite-radix stages: 384 = 32*12, 500 = 20*5*5, 450 = 18*5*5).
// The stage order is ct_stage_radix below.
MP_HD constexpr int ct_radix(int M, int E) {
    for (int r = E; r >= 8; r /= 2)
        if (M % r == 0) return r;
    for (int d = E; d >= 2; --d)
        if (M % d == 0 && ((E + d - 1) / d) * d <= E + E / 2) return d;
    return M;
}

// Stage order of a compile-time plan: the greedy factors of ct_radix, in
// reverse (largest power-of-two radix last) when the greedy order starts
// with a power of two followed by a factor that is not one.  Measured on
// GB300 at nz = 128: the inverse rows of 384 (32*12) and 480 (32*15) ran
// 3x faster with the big radix last, while lengths whose greedy order starts
// with a composite radix (405 = 9*9*5, 243, 135) ran faster as they are.
MP_HD constexpr bool ct_reverse_order(int N, int E) {
    const int r0 = ct_radix(N, E);
    if (r0 == N || (r0 & (r0 - 1)) != 0) return false;
    for (int m = N / r0; m > 1;) {
        const int r = ct_radix(m, E);
        if (r & (r - 1)) return true;
        m /= r;
    }
    return false;
}

// Radix of the stage of the length-N plan whose input stride is NS (the
// product of the earlier stages' radices); the host builds its twiddle
// tables from the same function.
MP_HD constexpr int ct_stage_radix(int N, int NS, int E) {
    int f[32] = {};
    int s = 0;
    for (int m = N; m > 1 && s < 32; ++s) {
        f[s] = ct_radix(m, E);
        m /= f[s];
    }
    const bool rev = ct_reverse_order(N, E);
    int ns = 1;
    for (int i = 0; i < s; ++i) {
        const int r = rev ? f[s - 1 - i] : f[i];
        if (ns == NS) return r;
        ns *= r;
    }
    return 1;
}

// E (the elements a thread holds in a stage, which bounds the radix) is the
// plan's radix schedule: the default is ElemsPerThread; a schedule with a
// smaller E takes more, smaller stages (1024 = 32*32 with E = 32, 16*16*4
// with E = 16) with fewer registers per thread.
template <typename R> MP_HD constexpr int ept() { return ElemsPerThread<R>::value; }

template <typename R, int N, int NS, int E = ept<R>()> struct StageRadix {
    static constexpr int value = ct_stage_radix(N, NS, E);
};

// Position of the stage with the given Ns in the compile-time plan.
template <int N, int E> constexpr int stage_index_impl(int target) {
    int ns = 1, s = 0;
    while (ns < target) {
        ns *= ct_stage_radix(N, ns, E);
        ++s;
    }
    return s;
}
template <typename R, int N, int NS, int E = ept<R>()> struct StageIndex {
    static constexpr int value = stage_index_impl<N, E>(NS);
};

template <typename R, int N, int NS, int S, class Sc = BlockScope, int E = ept<R>()>
__device__ __forceinline__ void ct_stage(cplx<R>* buf, int nb, int bstride, const cplx<R>* __restrict__ tws) {
    const cplx<R>* __restrict__ tw = tws + StageIndex<R, N, NS, E>::value * N;
    constexpr int RAD = StageRadix<R, N, NS, E>::value;
    constexpr int NB = (E + RAD - 1) / RAD;
    constexpr int NQ = N / RAD;
    const int total = NQ * nb;
    cplx<R> x[NB][RAD];
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const int t = Sc::tid() + i * Sc::size();
        if (t < total) {
            const int b = t / NQ;
            const int q = t - b * NQ;
            const cplx<R>* src = buf + b * bstride;
            const int sq = spad(q);
#pragma unroll
            for (int r = 0; r < RAD; ++r) x[i][r] = src[spad_at<NQ>(sq, q, r)];
        }
    }
    Sc::sync();
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const int t = Sc::tid() + i * Sc::size();
        if (t < total) {
            const int b = t / NQ;
            const int q = t - b * NQ;
            const int qd = q / NS;
            const int k = q - qd * NS;
            if (NS > 1) {
#pragma unroll
                for (int r = 1; r < RAD; ++r) {
                    const cplx<R> wv = __ldg(&tw[r * NS + k]);
                    x[i][r] = (S < 0) ? cmul(x[i][r], wv) : cmulc(x[i][r], wv);
                }
            }
            RegFFT<R, RAD, S>::run(x[i]);
            cplx<R>* dst = buf + b * bstride;
            const int base = qd * NS * RAD + k;
            const int sb = spad(base);
#pragma unroll
            for (int r = 0; r < RAD; ++r) dst[spad_at<NS>(sb, base, r)] = x[i][r];
        }
    }
    Sc::sync();
}

template <typename R, int N, int NS, int S, class Sc = BlockScope, int E = ept<R>()> struct CtFFT {
    static __device__ __forceinline__ void run(cplx<R>* buf, int nb, int bstride, const cplx<R>* tw) {
        ct_stage<R, N, NS, S, Sc, E>(buf, nb, bstride, tw);
        CtFFT<R, N, NS * StageRadix<R, N, NS, E>::value, S, Sc, E>::run(buf, nb, bstride, tw);
    }
};
template <typename R, int N, int S, class Sc, int E> struct CtFFT<R, N, N, S, Sc, E> {
    static __device__ __forceinline__ void run(cplx<R>*, int, int, const cplx<R>*) {}
};

// ---------------------------------------------------------------------------
// First and last stages fused with the caller's global loads and stores.
// The first stage (Ns = 1) takes its inputs from load(b, e) straight into
// registers and writes its outputs to shared memory; the last stage reads
// shared memory and hands each butterfly's outputs to store(b, q, x, NS):
// x[r] is element q + r*NS of transform b.  The middle
// stages run as above.  BFAST selects the butterfly-to-thread map:
// consecutive threads take consecutive transforms (columns of a tile, whose
// global elements are adjacent) or consecutive butterflies of one transform
// (rows, whose elements are adjacent).
// ---------------------------------------------------------------------------
template <typename R, int N, int NS, int E = ept<R>()> struct StageInfo {
    static constexpr int RAD = StageRadix<R, N, NS, E>::value;
    static constexpr int NQ = N / RAD;
    static constexpr int NEXT = NS * RAD;
    static constexpr bool LAST = (NEXT == N);
};

template <int N, int E> constexpr int last_stage_ns_impl() {
    int ns = 1;
    while (ns < N) {
        const int rad = ct_stage_radix(N, ns, E);
        if (ns * rad == N) return ns;
        ns *= rad;
    }
    return ns;
}

// Ns of the last stage of the compile-time plan for length N.
template <typename R, int N, int E = ept<R>()> struct LastNs {
    static constexpr int value = last_stage_ns_impl<N, E>();
};

template <bool BFAST, int NQ>
__device__ __forceinline__ void bfly_map(int t, int nb, int& b, int& q) {
    if (BFAST) { q = t / nb; b = t - q * nb; }
    else { b = t / NQ; q = t - b * NQ; }
}

// SYNC_IN: the inputs are read from the same shared buffer the stage writes,
// so the block synchronises between the reads and the writes.
template <typename R, int N, int S, bool BFAST, bool SYNC_IN = false, class Sc = BlockScope, int E = ept<R>(),
          class Load>
__device__ __forceinline__ void ct_first(cplx<R>* buf, int nb, int bstride, Load&& load) {
    using SI = StageInfo<R, N, 1, E>;
    constexpr int RAD = SI::RAD, NQ = SI::NQ;
    constexpr int NB = (E + RAD - 1) / RAD;
    const int total = NQ * nb;
    cplx<R> x[NB][RAD];
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const int t = Sc::tid() + i * Sc::size();
        if (t < total) {
            int b, q;
            bfly_map<BFAST, NQ>(t, nb, b, q);
#pragma unroll
            for (int r = 0; r < RAD; ++r) x[i][r] = load(b, q + r * NQ);
        }
    }
    if (SYNC_IN) Sc::sync();
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const int t = Sc::tid() + i * Sc::size();
        if (t < total) {
            int b, q;
            bfly_map<BFAST, NQ>(t, nb, b, q);
            RegFFT<R, RAD, S>::run(x[i]);
            cplx<R>* dst = buf + b * bstride;
            if constexpr (RAD % 32 == 0) {
                // spad(q RAD + r) = q (RAD + RAD/32) + r + r/32
                cplx<R>* d0 = dst + q * (RAD + RAD / 32);
#pragma unroll
                for (int r = 0; r < RAD; ++r) d0[r + (r >> 5)] = x[i][r];
            } else {
#pragma unroll
                for (int r = 0; r < RAD; ++r) dst[spad(q * RAD + r)] = x[i][r];
            }
        }
    }
    Sc::sync();
}

template <typename R, int N, int NS, int S, class Sc = BlockScope, int E = ept<R>(),
          bool STOP = StageInfo<R, N, NS, E>::LAST>
struct CtMid {
    static __device__ __forceinline__ void run(cplx<R>* buf, int nb, int bstride, const cplx<R>* tw) {
        ct_stage<R, N, NS, S, Sc, E>(buf, nb, bstride, tw);
        CtMid<R, N, StageInfo<R, N, NS, E>::NEXT, S, Sc, E>::run(buf, nb, bstride, tw);
    }
};
template <typename R, int N, int NS, int S, class Sc, int E> struct CtMid<R, N, NS, S, Sc, E, true> {
    static __device__ __forceinline__ void run(cplx<R>*, int, int, const cplx<R>*) {}
};

template <typename R, int N, int S, bool BFAST, class Sc = BlockScope, int E = ept<R>(), class Store>
__device__ __forceinline__ void ct_last(const cplx<R>* buf, int nb, int bstride, const cplx<R>* __restrict__ tws,
                                        Store&& store) {
    constexpr int NS = LastNs<R, N, E>::value;
    const cplx<R>* __restrict__ tw = tws + StageIndex<R, N, NS, E>::value * N;
    using SI = StageInfo<R, N, NS, E>;
    static_assert(SI::LAST, "last stage");
    constexpr int RAD = SI::RAD, NQ = SI::NQ;
    constexpr int NB = (E + RAD - 1) / RAD;
    const int total = NQ * nb;
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const int t = Sc::tid() + i * Sc::size();
        if (t < total) {
            int b, q;
            bfly_map<BFAST, NQ>(t, nb, b, q);
            const cplx<R>* src = buf + b * bstride;
            cplx<R> x[RAD];
            const int sq = spad(q);
#pragma unroll
            for (int r = 0; r < RAD; ++r) x[r] = src[spad_at<NQ>(sq, q, r)];
            // last stage: Ns * RAD = N, so q < Ns and q is the twiddle index k
            if (NS > 1) {
#pragma unroll
                for (int r = 1; r < RAD; ++r) {
                    const cplx<R> wv = __ldg(&tw[r * NS + q]);
                    x[r] = (S < 0) ? cmul(x[r], wv) : cmulc(x[r], wv);
                }
            }
            RegFFT<R, RAD, S>::run(x);
            store(b, q, x, NS);
        }
    }
}

// Last stage with a prefetch: pre(b, q, NS, i) runs for every butterfly i
// of the thread before any butterfly is transformed, so loads it issues (the
// operands of the store's read-modify-write) are all in flight at once
// instead of one butterfly at a time; then store(b, q, x, NS, i) as ct_last.
template <typename R, int N, int S, bool BFAST, class Sc = BlockScope, int E = ept<R>(), class Pre, class Store>
__device__ __forceinline__ void ct_last_pre(const cplx<R>* buf, int nb, int bstride, const cplx<R>* __restrict__ tws,
                                            Pre&& pre, Store&& store) {
    constexpr int NS = LastNs<R, N, E>::value;
    const cplx<R>* __restrict__ tw = tws + StageIndex<R, N, NS, E>::value * N;
    using SI = StageInfo<R, N, NS, E>;
    static_assert(SI::LAST, "last stage");
    constexpr int RAD = SI::RAD, NQ = SI::NQ;
    constexpr int NB = (E + RAD - 1) / RAD;
    const int total = NQ * nb;
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const int t = Sc::tid() + i * Sc::size();
        if (t < total) {
            int b, q;
            bfly_map<BFAST, NQ>(t, nb, b, q);
            pre(b, q, NS, i);
        }
    }
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const int t = Sc::tid() + i * Sc::size();
        if (t < total) {
            int b, q;
            bfly_map<BFAST, NQ>(t, nb, b, q);
            const cplx<R>* src = buf + b * bstride;
            cplx<R> x[RAD];
            const int sq = spad(q);
#pragma unroll
            for (int r = 0; r < RAD; ++r) x[r] = src[spad_at<NQ>(sq, q, r)];
            if (NS > 1) {
#pragma unroll
                for (int r = 1; r < RAD; ++r) {
                    const cplx<R> wv = __ldg(&tw[r * NS + q]);
                    x[r] = (S < 0) ? cmul(x[r], wv) : cmulc(x[r], wv);
                }
            }
            RegFFT<R, RAD, S>::run(x);
            store(b, q, x, NS, i);
        }
    }
}

// Last stage for an output buffer that aliases the input: every thread
// computes its butterflies into registers, the block synchronises, then the
// results go to store(b, q, x, NS).
template <typename R, int N, int S, bool BFAST, class Sc = BlockScope, int E = ept<R>(), class Store>
__device__ __forceinline__ void ct_last_sync(const cplx<R>* buf, int nb, int bstride, const cplx<R>* __restrict__ tws,
                                             Store&& store) {
    constexpr int NS = LastNs<R, N, E>::value;
    const cplx<R>* __restrict__ tw = tws + StageIndex<R, N, NS, E>::value * N;
    using SI = StageInfo<R, N, NS, E>;
    static_assert(SI::LAST, "last stage");
    constexpr int RAD = SI::RAD, NQ = SI::NQ;
    constexpr int NB = (E + RAD - 1) / RAD;
    const int total = NQ * nb;
    cplx<R> x[NB][RAD];
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const int t = Sc::tid() + i * Sc::size();
        if (t < total) {
            int b, q;
            bfly_map<BFAST, NQ>(t, nb, b, q);
            const cplx<R>* src = buf + b * bstride;
            const int sq = spad(q);
#pragma unroll
            for (int r = 0; r < RAD; ++r) x[i][r] = src[spad_at<NQ>(sq, q, r)];
            if (NS > 1) {
#pragma unroll
                for (int r = 1; r < RAD; ++r) {
                    const cplx<R> wv = __ldg(&tw[r * NS + q]);
                    x[i][r] = (S < 0) ? cmul(x[i][r], wv) : cmulc(x[i][r], wv);
                }
            }
            RegFFT<R, RAD, S>::run(x[i]);
        }
    }
    Sc::sync();
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const int t = Sc::tid() + i * Sc::size();
        if (t < total) {
            int b, q;
            bfly_map<BFAST, NQ>(t, nb, b, q);
            store(b, q, x[i], NS);
        }
    }
}

}  // namespace mp
