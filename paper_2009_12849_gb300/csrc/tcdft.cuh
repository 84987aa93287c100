// Split-precision tensor-core DFT for the forward column transforms (step a2,
// y part; opt-in for mixed plans with ny = 1024: MONC_PROJ_TC=1 split TF32
// with three products, MONC_PROJ_TC=2 split BF16 with six).
//
// The length-1024 transform along y is two radix-32 stages (1024 = 32 x 32,
// decimation in time): with j = q + 32 r and the output index k1 + 32 k2,
//   Y1[q][k1] = sum_r x[q + 32 r] W_32^{r k1}            (stage 1)
//   Z[q][k1]  = Y1[q][k1] W_1024^{q k1}                   (twiddles)
//   X[k1 + 32 k2] = sum_q Z[q][k1] W_32^{q k2}            (stage 2)
// For a tile of 8 columns c each stage is one real matrix product
//   D (256 x 64) = A (256 x 64) B (64 x 64)
// with A's rows the 256 (q, c) sequences (stage 2: (k1, c)), A's columns the
// 32 real then 32 imaginary parts of the inputs, and B the 32-point DFT in real
// block form [[Re F, Im F], [-Im F, Re F]] (columns: real then imaginary parts
// of the outputs).  The products run on the tensor cores (tcgen05.mma,
// M = 128, N = 64, accumulators in tensor memory) in split precision, the
// parts and their products accumulated in FP32:
//  - TF32 x 3 (kind::tf32, K = 8): A = A_hi + A_lo and B = B_hi + B_lo, each
//    part rounded to TF32 (11 significant bits); D = A_hi B_hi + A_hi B_lo +
//    A_lo B_hi.  The parts carry about 22 bits of each operand, which leaves
//    about 2^-21 relative error per product;
//  - BF16 x 6 (kind::f16, K = 16): three BF16 parts (8 significant bits each)
//    carry 24 bits; D = hi hi + hi mid + mid hi + mid mid + hi lo + lo hi,
//    the dropped products of order 2^-24, so FP32-level accuracy.
// The twiddles run on the CUDA cores between the stages.
//
// Operands sit in shared memory in the tensor core's K-major layout without
// swizzling: 8-row x 16-byte core matrices of 128 contiguous bytes, core (row
// group g, K group h) at byte (g * KG + h) * 128 with KG = 64 elements x the
// element size / 16 bytes; descriptors give the K step between core matrices
// (128 B) and the row-group step (KG * 128 B).  One thread
// issues the products; a tcgen05.commit arrives on an mbarrier that every
// thread waits on (bounded: past kTcSpinLimit polls the block latches bit 0
// of the plan's error word, waits once more, frees its tensor memory and
// returns).  Thread t of the block owns row t of A and of D, which is the
// tensor-memory lane the warp may read (warp w: lanes 32 (w % 4) ..., the
// accumulator of rows 128 (w / 4) ...).
#pragma once
#include <cuda_bf16.h>

#include "tma.cuh"
#include "regfft.cuh"

namespace mp {

constexpr int kTcThreads = 256;
constexpr int kTcCols = 8;                  // columns per tile
constexpr int kTcRows = kTcThreads;         // rows of A = 32 sequences x 8 columns
constexpr int kTcK = 64;                    // 32 complex inputs as 64 reals
constexpr int kTcN = 64;                    // 32 complex outputs as 64 reals
constexpr long long kTcSpinLimit = 1ll << 22;

// exp(-2 pi i m / 32): the 32-point DFT's entries, exactly reduced at compile
// time (regfft.cuh)
struct W32 {
    double c[32], s[32];
    constexpr W32() : c(), s() {
        for (int m = 0; m < 32; ++m) {
            c[m] = ct_cos2pi(m, 32);
            s[m] = -ct_sin2pi(m, 32);
        }
    }
};
static __constant__ W32 kW32 = W32();

__device__ __forceinline__ float tf32_round(float x) {
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// The two split formats.  ELEM: bytes per part element; PARTS: parts per
// operand; KMMA: K of one product instruction; pa(i)/pb(i): the A part and B
// part of product i.
template <int FMT> struct TcFmt;
template <> struct TcFmt<1> {                  // TF32 x 3
    static constexpr int ELEM = 4, PARTS = 2, KMMA = 8, PRODUCTS = 3;
    static __host__ __device__ constexpr int pa(int i) { return i == 2 ? 1 : 0; }
    static __host__ __device__ constexpr int pb(int i) { return i == 1 ? 1 : 0; }
    // D FP32, A and B TF32, both K-major, N = 64, M = 128
    static constexpr unsigned IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(kTcN >> 3) << 17) |
                                      ((unsigned)(128 >> 4) << 24);
    static __device__ __forceinline__ void split(float x, float* part) {
        part[0] = tf32_round(x);
        part[1] = tf32_round(x - part[0]);
    }
    static __device__ __forceinline__ void put(unsigned char* at, float v) { *(float*)at = v; }
    static __device__ __forceinline__ void mma(unsigned d, unsigned long long a, unsigned long long b, int acc) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
            ::"r"(d), "l"(a), "l"(b), "r"(IDESC), "r"(acc)
            : "memory");
    }
};
template <> struct TcFmt<2> {                  // BF16 x 6
    static constexpr int ELEM = 2, PARTS = 3, KMMA = 16, PRODUCTS = 6;
    // (hi, hi) (hi, mid) (mid, hi) (mid, mid) (hi, lo) (lo, hi)
    static __host__ __device__ constexpr int pa(int i) { return i == 2 || i == 3 ? 1 : i == 5 ? 2 : 0; }
    static __host__ __device__ constexpr int pb(int i) { return i == 1 || i == 3 ? 1 : i == 4 ? 2 : 0; }
    // D FP32, A and B BF16, both K-major, N = 64, M = 128
    static constexpr unsigned IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(kTcN >> 3) << 17) |
                                      ((unsigned)(128 >> 4) << 24);
    static __device__ __forceinline__ void split(float x, float* part) {
        // x - hi and the next residual are exact in FP32
        part[0] = __bfloat162float(__float2bfloat16_rn(x));
        const float r1 = x - part[0];
        part[1] = __bfloat162float(__float2bfloat16_rn(r1));
        part[2] = __bfloat162float(__float2bfloat16_rn(r1 - part[1]));
    }
    static __device__ __forceinline__ void put(unsigned char* at, float v) {
        *(__nv_bfloat16*)at = __float2bfloat16_rn(v);
    }
    static __device__ __forceinline__ void mma(unsigned d, unsigned long long a, unsigned long long b, int acc) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
            ::"r"(d), "l"(a), "l"(b), "r"(IDESC), "r"(acc)
            : "memory");
    }
};

template <int FMT> struct TcLayout {
    using F = TcFmt<FMT>;
    static constexpr int KG = kTcK * F::ELEM / 16;                    // K groups of 16 bytes per row group
    static constexpr unsigned SBO = KG * 128;                        // row-group step
    static constexpr unsigned A_BYTES = kTcRows * kTcK * F::ELEM;    // one A part
    static constexpr unsigned B_BYTES = kTcN * kTcK * F::ELEM;       // one B part
    static constexpr unsigned SMEM = F::PARTS * (A_BYTES + B_BYTES) + 128;   // + alignment slack
    // byte offset of element (row, kk) in a K-major operand with 64 columns
    static __device__ __forceinline__ unsigned off(int row, int kk) {
        constexpr int EPG = 16 / F::ELEM;                            // elements per 16 bytes
        return (unsigned)(((row >> 3) * KG + kk / EPG) * 128 + (row & 7) * 16 + (kk % EPG) * F::ELEM);
    }
};

// Shared-memory matrix descriptor: no swizzling, K step `lbo` bytes between
// core matrices, `sbo` bytes between row groups.
__device__ __forceinline__ unsigned long long tc_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
    return (unsigned long long)((saddr & 0x3FFFFu) >> 4) | ((unsigned long long)(lbo >> 4) << 16) |
           ((unsigned long long)(sbo >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ void tc_commit(unsigned long long* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive 32-bit columns of this thread's lane, starting at taddr.
__device__ __forceinline__ void tc_ld16(unsigned taddr, float* v) {
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Bounded wait on the mbarrier's phase `parity` by every thread; false if it
// gave up (the timeout bit is latched).
__device__ __forceinline__ bool tc_wait(unsigned long long* bar, unsigned parity, int* err) {
    long long spins = 0;
    while (!mbar_try_wait(bar, parity)) {
        if (++spins > kTcSpinLimit) {
            atomicOr(err, 1);
            return false;
        }
        __nanosleep(20);
    }
    return true;
}

// Store row `row` of a split operand: v[0..31] real parts, v[32..63]
// imaginary parts, one part per buffer.
template <int FMT>
__device__ __forceinline__ void tc_put_row(unsigned char* const* parts, int row, const float* v) {
    using F = TcFmt<FMT>;
    using L = TcLayout<FMT>;
#pragma unroll
    for (int kk = 0; kk < kTcK; ++kk) {
        float pv[F::PARTS];
        F::split(v[kk], pv);
#pragma unroll
        for (int i = 0; i < F::PARTS; ++i) F::put(parts[i] + L::off(row, kk), pv[i]);
    }
}

// The products of one stage into the two accumulators (rows 0-127 at
// tensor-memory column 0, rows 128-255 at column 64).
template <int FMT>
__device__ __forceinline__ void tc_stage_mmas(unsigned tmem, const unsigned* a, const unsigned* b) {
    using F = TcFmt<FMT>;
    using L = TcLayout<FMT>;
    constexpr unsigned LBO = 128;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const unsigned a_off = (unsigned)h * 16 * L::SBO;
        const unsigned d = tmem + (unsigned)h * kTcN;
#pragma unroll
        for (int s = 0; s < kTcK / F::KMMA; ++s) {
            const unsigned ko = (unsigned)s * 2 * 128;       // KMMA elements = two core matrices
#pragma unroll
            for (int pr = 0; pr < F::PRODUCTS; ++pr)
                F::mma(d, tc_desc(a[F::pa(pr)] + a_off + ko, LBO, L::SBO), tc_desc(b[F::pb(pr)] + ko, LBO, L::SBO),
                       (s > 0 || pr > 0) ? 1 : 0);
        }
    }
}

// This thread's row of D: 32 complex values (real parts in columns 0-31,
// imaginary parts in 32-63 of its accumulator).
__device__ __forceinline__ void tc_get_row(unsigned tmem, float2* out) {
    const int w = threadIdx.x >> 5;
    const unsigned taddr = tmem + ((unsigned)(32 * (w & 3)) << 16) + (unsigned)(w >> 2) * kTcN;
    float re[32], im[32];
    tc_ld16(taddr, re);
    tc_ld16(taddr + 16, re + 16);
    tc_ld16(taddr + 32, im);
    tc_ld16(taddr + 48, im + 16);
    tc_wait_ld();
#pragma unroll
    for (int i = 0; i < 32; ++i) out[i] = make_float2(re[i], im[i]);
}

// Forward y transform of one tile (8 columns from kx0 of level k), T -> S.
template <int FMT>
__global__ void __launch_bounds__(kTcThreads, 1) k_fwd_cols_tc(ProjParams p) {
    using F = TcFmt<FMT>;
    using L = TcLayout<FMT>;
    extern __shared__ __align__(128) unsigned char tc_smem[];
    unsigned char* base = (unsigned char*)(((uintptr_t)tc_smem + 127) & ~(uintptr_t)127);
    unsigned char* ap[F::PARTS];
    unsigned char* bp[F::PARTS];
    unsigned sa[F::PARTS], sb[F::PARTS];
#pragma unroll
    for (int i = 0; i < F::PARTS; ++i) {
        ap[i] = base + i * L::A_BYTES;
        bp[i] = base + F::PARTS * L::A_BYTES + i * L::B_BYTES;
        sa[i] = smem_u32(ap[i]);
        sb[i] = smem_u32(bp[i]);
    }
    __shared__ unsigned long long bar;
    __shared__ unsigned tmem_slot;
    const int tid = threadIdx.x;
    const int k = blockIdx.x / p.ntiles;
    const int kx0 = (blockIdx.x - k * p.ntiles) * kTcCols;
    const int ny = 1024, nxh = p.nxh, nxp = p.nxp;

    if (tid < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(smem_u32(&tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // B: the 32-point DFT W_32^{r k} = c + i s in real block form, row n
    // (output: k real, 32 + k imaginary), column kk (input: r real, 32 + r
    // imaginary): out_re = sum in_re c - in_im s, out_im = sum in_re s + in_im c.
    // Its parts are split from the FP64 value.
    for (int e = tid; e < kTcN * kTcK; e += kTcThreads) {
        const int n = e / kTcK, kk = e - n * kTcK;
        const int m = ((n & 31) * (kk & 31)) & 31;
        const double c = kW32.c[m], s = kW32.s[m];
        double val = (n < 32) ? ((kk < 32) ? c : -s) : ((kk < 32) ? s : c);
#pragma unroll
        for (int i = 0; i < F::PARTS; ++i) {
            float part[F::PARTS];
            F::split((float)val, part);
            F::put(bp[i] + L::off(n, kk), part[0]);
            val -= (double)part[0];
        }
    }
    // A (stage 1): row tid = (q, c), entries x[q + 32 r]
    const int q = tid >> 3, c = tid & 7, kx = kx0 + c;
    {
        const float2* T = (const float2*)p.T + (size_t)k * ny * nxp + kx;
        float v[kTcK];
#pragma unroll
        for (int r = 0; r < 32; ++r) {
            const float2 x = (kx < nxh) ? T[(size_t)(q + 32 * r) * nxp] : make_float2(0.f, 0.f);
            v[r] = x.x;
            v[32 + r] = x.y;
        }
        tc_put_row<FMT>(ap, tid, v);
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = tmem_slot;
    if (tid == 0) {
        tc_stage_mmas<FMT>(tmem, sa, sb);
        tc_commit(&bar);
    }
    unsigned phase = 0;                      // the phase that the products in flight complete
    bool ok = tc_wait(&bar, phase, p.err);
    tc_fence_after();
    float2 y[32];
    if (ok) tc_get_row(tmem, y);
    // twiddles W_1024^{q k1} (stage table of the y plan), then A (stage 2):
    // row (k1, c), entries Z[q][k1] at K index q
    if (ok) {
        const float2* tw = (const float2*)p.twy + 1024;
#pragma unroll
        for (int k1 = 0; k1 < 32; ++k1) {
            const float2 z = cmul(y[k1], __ldg(&tw[k1 * 32 + q]));
            const int row = k1 * 8 + c;
            const float zr[2] = {z.x, z.y};
#pragma unroll
            for (int part = 0; part < 2; ++part) {
                float pv[F::PARTS];
                F::split(zr[part], pv);
#pragma unroll
                for (int i = 0; i < F::PARTS; ++i) F::put(ap[i] + L::off(row, 32 * part + q), pv[i]);
            }
        }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (ok && tid == 0) {
        tc_stage_mmas<FMT>(tmem, sa, sb);
        tc_commit(&bar);
    }
    if (ok) {
        phase = 1;
        ok = tc_wait(&bar, phase, p.err);
    }
    tc_fence_after();
    if (ok) {
        tc_get_row(tmem, y);
        // row (k1, c) holds X[k1 + 32 k2] for k2 = 0..31
        const int k1 = tid >> 3;
        if (kx < nxh) {
            float2* S = (float2*)p.S + (size_t)k * ny * nxp + kx;
#pragma unroll
            for (int k2 = 0; k2 < 32; ++k2) S[(size_t)(k1 + 32 * k2) * nxp] = y[k2];
        }
    } else {
        // a product may still be in flight: give it one more bounded wait
        // before the tensor memory it writes is freed
        if (tid == 0) {
            long long spins = 0;
            while (!mbar_try_wait(&bar, phase) && ++spins < kTcSpinLimit) __nanosleep(20);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (tid < 32) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem) : "memory");
    }
}

}  // namespace mp
