// Krylov pressure solver (paper, Section 4: BiCGStab on the Poisson problem
// L phi = D(u*) of the FFT solver; the paper preconditions it with ILU, runs
// it in single precision to a 1e-4 stopping criterion as well as in double,
// and names a bespoke, structure-aware preconditioner as further work).
//
// L = D o G as a 7-point stencil: periodic second differences in x and y and
// the rows of the vertical operator,
//   (L x)[k] = (x_e - 2x + x_w)/dx^2 + (x_n - 2x + x_s)/dy^2
//            + sub[k] x[k-1] + diag0[k] x[k] + sup[k] x[k+1],
//   sub[k] = A[k]/V[k], sup[k] = A[k+1]/V[k], diag0[k] = -(A[k] + A[k+1])/V[k],
// with A[k] = rho_f[k]/dzn[k] (A[0] = A[nz] = 0) and V[k] = rho_c[k] dz[k].
//
// Preconditioner (precond = 1): the vertical lines of L, i.e. the vertical
// rows plus the diagonal of the horizontal part (-2/dx^2 - 2/dy^2).  Every
// column (i, j) has the same matrix, so its Thomas factors (cp[k] and the
// inverse pivots) are formed once per solve by a one-thread kernel and each
// application is one forward and one backward sweep per column, a thread per
// column, coalesced across i.  It takes the place of ILU, whose triangular
// sweeps run through the whole grid one cell after another.
//
// BiCGStab (van der Vorst 1992) with the preconditioner applied to the search
// directions, in the order of the preconditioned algorithm of Barrett et al.,
// Templates (1994): x0 = 0, shadow residual r~ = r0 = b, stop when
// ||r|| <= tol ||b|| on the recurrence residual, also after the half step on s.
// Vectors are in the field precision T (FP64 plans: double; mixed plans:
// float, whose arithmetic GB300 runs 64 times faster than FP64).  The iterate
// x = (x + alpha p^) + omega s^ is updated once per iteration: in FP64 for
// FP64 plans, and for FP32 as an unevaluated sum x_hi + x_lo of two floats
// (Knuth's TwoSum adds each FP32 increment to x_hi and carries the rounding
// error into x_lo), so the final gradient G phi is formed from a potential
// accurate to about 2^-48 without FP64 arithmetic in the loop.
// Inner products: per-thread sums in T, block and global sums in FP64; the
// scalars (rho, alpha, omega, beta) live in device memory as FP64.  Each block
// of a reducing kernel writes its partial sums; the last block to finish (a
// ticket counter) adds all partials in a fixed order and forms the next
// scalar, so results are deterministic run to run and no separate reduction
// launch is needed.  The host enqueues kKryCheckEvery iterations at a time
// and then reads the scalar block to test convergence; the kernels of the
// iterations after the one that stopped return at once, so the iteration
// count and the result are those of a test after every iteration.  A denominator that is zero or not finite (rounding past the
// attainable accuracy) ends the method as a breakdown.
//
// After the solve phi is pinned as in the FFT solver (level-0 horizontal mean
// zero) and the outputs are u - G phi (w zero on the bottom and top faces).
#include <algorithm>
#include <cstddef>
#include <cstdint>

#include "krylov.h"

namespace mp {
namespace {

constexpr int kKryThreads = 256;
constexpr int kKryBlocksPerSm = 8;       // streaming kernels: 2048 threads per SM
constexpr int kKryIlp = 4;               // elements in flight per thread (streaming kernels)
constexpr int kKrySums = 2;              // partial sums per block
constexpr int kKryCheckEvery = 8;        // iterations enqueued between host convergence tests
constexpr int kTileX = 32, kTileY = 8;   // stencil kernels: a 32 x 8 tile of columns
constexpr int kTileZ = 32;               //   marching over 32 levels (one reduction per block)
constexpr int kApplyBatch = 8;           // FP32 stencil: levels whose operands load together
// line sweeps: levels loaded before use (32 FP32 or 16 FP64 values: about
// 128 bytes per thread in flight, enough to cover DRAM latency with the few
// threads one per column gives)
template <typename T> constexpr int kLineBatch = 128 / sizeof(T);

// Scalars of the iteration, in device memory.
struct KrySc {
    double bnorm;                        // ||b||
    double rho, alpha, omega, beta;
    double relres;                       // ||r|| / ||b|| of the last completed step
    double srel;                         // ||s|| / ||b|| of the current half step
    double mean;                         // level-0 horizontal mean of phi (pin)
    int done;                            // 1: stopped
    int half;                            // 1: stop after x += alpha p^ (half-step end)
    int status;                          // 0 converged, 2 breakdown
    int iters;                           // completed iterations
};

enum Stage { kStRhs = 0, kStAlpha = 1, kStS = 2, kStOmega = 3, kStR = 4, kStMean = 5 };

template <typename T>
struct Tabs {
    T* vsub; T* vdiag; T* vsup;          // vertical rows of L
    T* lcp; T* livd;                     // line preconditioner: cp[k], 1/pivot[k]
    T* flo; T* fhi;                      // divergence: rho_f[k]/V[k], rho_f[k+1]/V[k] (0 at the ends)
};

template <typename T>
struct Ws {
    T* xh;                               // the iterate: x_hi (FP64 plans: x itself)
    T* xl;                               // FP32: x_lo of x = x_hi + x_lo
    T *r, *rt, *p, *v, *ph, *sh, *t;
    double* part;                        // [nparts][kKrySums]
    KrySc* sc;
    unsigned* ticket;                    // blocks of the running reduction that have finished
    Tabs<T> tab;
};

size_t al256(size_t n) { return (n + 255) & ~size_t(255); }

struct Shape {
    int nblk;                            // streaming kernels
    dim3 tiles;                          // stencil kernels
    int ntile;
    int nparts;                          // partial-sum slots: max of the two
};

Shape shape(int nx, int ny, int nz, int nsm) {
    Shape sh;
    sh.nblk = std::max(1, nsm) * kKryBlocksPerSm;
    sh.tiles = dim3((nx + kTileX - 1) / kTileX, (ny + kTileY - 1) / kTileY, (nz + kTileZ - 1) / kTileZ);
    sh.ntile = (int)(sh.tiles.x * sh.tiles.y * sh.tiles.z);
    sh.nparts = std::max(sh.nblk, sh.ntile);
    return sh;
}

// Workspace layout: the iterate (one T field, two for FP32), seven T fields,
// the partial sums, the scalars and ticket, the tables.  With base == nullptr
// only the size is computed.
template <typename T>
Ws<T> carve(void* base, int nx, int ny, int nz, int nparts, size_t* bytes) {
    const size_t N = (size_t)nx * ny * nz;
    size_t off = 0;
    Ws<T> w{};
    auto take = [&](size_t n) -> unsigned char* {
        unsigned char* q = base ? (unsigned char*)base + off : nullptr;
        off = al256(off + n);
        return q;
    };
    w.xh = (T*)take(N * sizeof(T));
    w.xl = (sizeof(T) == 4) ? (T*)take(N * sizeof(T)) : nullptr;
    T** vecs[7] = {&w.r, &w.rt, &w.p, &w.v, &w.ph, &w.sh, &w.t};
    for (T** q : vecs) *q = (T*)take(N * sizeof(T));
    w.part = (double*)take((size_t)nparts * kKrySums * sizeof(double));
    w.sc = (KrySc*)take(sizeof(KrySc));
    w.ticket = (unsigned*)take(sizeof(unsigned));
    T** tabs[7] = {&w.tab.vsub, &w.tab.vdiag, &w.tab.vsup, &w.tab.lcp, &w.tab.livd, &w.tab.flo, &w.tab.fhi};
    for (T** q : tabs) *q = (T*)take((size_t)nz * sizeof(T));
    if (bytes) *bytes = off;
    return w;
}

template <typename T>
struct Grid {
    int nx, ny, nz;
    size_t plane, n;
    T idx, idy, idx2, idy2;
    double idx64, idy64;
};

// The scalars a finished reduction forms (a and b: the two global sums).
__device__ void finish_stage(KrySc* sc, int stage, double a, double b, double tol, int iter, int max_iter,
                             double plane) {
    if (stage == kStMean) { sc->mean = a / plane; return; }
    if (stage == kStRhs) {
        sc->bnorm = sqrt(a);
        sc->rho = a;                        // (r~, r0) = ||b||^2
        sc->alpha = sc->omega = 1.0;
        sc->beta = 0.0;
        sc->relres = sc->srel = (a > 0.0) ? 1.0 : 0.0;
        sc->done = (a > 0.0) ? 0 : 1;
        sc->half = 0;
        sc->status = 0;
        sc->iters = 0;
        return;
    }
    if (sc->done) return;
    if (stage == kStAlpha) {                // a = (r~, v)
        if (a == 0.0 || !isfinite(a)) { sc->done = 1; sc->status = 2; return; }
        sc->alpha = sc->rho / a;
    } else if (stage == kStS) {             // a = ||s||^2
        const double sn = sqrt(a);
        sc->srel = sn / sc->bnorm;
        if (sn <= tol * sc->bnorm) { sc->half = 1; sc->status = 0; }
    } else if (stage == kStOmega) {         // a = (t, s), b = (t, t)
        if (sc->half) return;
        if (b == 0.0 || !isfinite(b)) { sc->half = 1; sc->status = 2; return; }
        sc->omega = a / b;
    } else if (stage == kStR) {             // a = ||r||^2, b = (r~, r)
        sc->iters = iter;
        if (sc->half) { sc->relres = sc->srel; sc->done = 1; return; }
        sc->relres = sqrt(a) / sc->bnorm;
        if (sc->relres <= tol) { sc->done = 1; sc->status = 0; return; }
        // omega = 0 ends the method now; rho = (r~, r) = 0 would end the next
        // iteration before its first step
        const bool bad_omega = sc->omega == 0.0 || !isfinite(sc->omega);
        const bool bad_rho = (b == 0.0 || !isfinite(b)) && iter < max_iter;
        if (bad_omega || bad_rho) { sc->done = 1; sc->status = 2; return; }
        sc->beta = (b / sc->rho) * (sc->alpha / sc->omega);
        sc->rho = b;
    }
}

// What a reducing kernel does with its two block sums.
struct Reduce {
    double* part;                       // [nparts][kKrySums]
    unsigned* ticket;
    KrySc* sc;
    int nparts;                         // blocks of the launch
    int stage, iter, max_iter;
    double tol, plane;
};

// Block sum of up to two values into part[slot]; the last block of the launch
// to get here adds all partials in slot order and forms the stage's scalars.
__device__ __forceinline__ void block_reduce(double a, double b, const Reduce& rd, int slot) {
    __shared__ double sa[kKryThreads / 32], sb[kKryThreads / 32];
    __shared__ double fa[kKryThreads], fb[kKryThreads];
    __shared__ bool last;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    const int wid = t >> 5, lane = t & 31;
    if (lane == 0) { sa[wid] = a; sb[wid] = b; }
    __syncthreads();
    if (t == 0) {
        double ta = 0.0, tb = 0.0;
        for (int i = 0; i < kKryThreads / 32; ++i) { ta += sa[i]; tb += sb[i]; }
        rd.part[slot * kKrySums + 0] = ta;
        rd.part[slot * kKrySums + 1] = tb;
        __threadfence();
        last = atomicAdd(rd.ticket, 1u) == (unsigned)(rd.nparts - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // four independent sums per thread keep four loads in flight; the order
    // of the additions is fixed by the slot index
    double ga[4] = {0.0, 0.0, 0.0, 0.0}, gb[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i0 = t; i0 < rd.nparts; i0 += 4 * kKryThreads) {
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int i = i0 + m * kKryThreads;
            if (i < rd.nparts) {
                ga[m] += __ldcg(&rd.part[i * kKrySums]);
                gb[m] += __ldcg(&rd.part[i * kKrySums + 1]);
            }
        }
    }
    fa[t] = (ga[0] + ga[1]) + (ga[2] + ga[3]);
    fb[t] = (gb[0] + gb[1]) + (gb[2] + gb[3]);
    __syncthreads();
    for (int s = kKryThreads / 2; s > 0; s >>= 1) {
        if (t < s) { fa[t] += fa[t + s]; fb[t] += fb[t + s]; }
        __syncthreads();
    }
    if (t == 0) {
        finish_stage(rd.sc, rd.stage, fa[0], fb[0], rd.tol, rd.iter, rd.max_iter, rd.plane);
        *rd.ticket = 0;
    }
}

__device__ __forceinline__ int tile_slot() { return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z); }

// Column (i, j) of a stencil tile and the offsets of its periodic neighbours
// within a level.  Returns false for threads past the grid's edge.
struct Col {
    size_t c, ce, cw, cn, cs;
    int k0, k1;
};
template <typename T>
__device__ __forceinline__ bool tile_column(const Grid<T>& g, Col& cl) {
    const int i = blockIdx.x * kTileX + threadIdx.x;
    const int j = blockIdx.y * kTileY + threadIdx.y;
    cl.k0 = blockIdx.z * kTileZ;
    cl.k1 = min(g.nz, cl.k0 + kTileZ);
    if (i >= g.nx || j >= g.ny) return false;
    const size_t row = (size_t)j * g.nx;
    cl.c = row + i;
    cl.ce = row + (i == g.nx - 1 ? 0 : i + 1);
    cl.cw = row + (i == 0 ? g.nx - 1 : i - 1);
    cl.cn = (size_t)(j == g.ny - 1 ? 0 : j + 1) * g.nx + i;
    cl.cs = (size_t)(j == 0 ? g.ny - 1 : j - 1) * g.nx + i;
    return true;
}

// Vertical rows of L, the divergence's vertical weights and the Thomas
// factors of the line matrix (one thread, FP64, stored in T).
template <typename T>
__global__ void k_kry_tables(Tabs<T> tb, const double* acoef, const double* svol, const double* rflo,
                             const double* rfhi, int nz, double hdiag) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double cp_prev = 0.0;
    for (int k = 0; k < nz; ++k) {
        const double iv = 1.0 / svol[k];
        const double sub = acoef[k] * iv, sup = acoef[k + 1] * iv;
        const double d0 = -(acoef[k] + acoef[k + 1]) * iv;
        tb.vsub[k] = (T)sub;
        tb.vdiag[k] = (T)d0;
        tb.vsup[k] = (T)sup;
        tb.flo[k] = (T)(rflo[k] * iv);
        tb.fhi[k] = (T)(rfhi[k] * iv);
        const double den = (d0 + hdiag) - (k > 0 ? sub * cp_prev : 0.0);
        const double ivd = 1.0 / den;
        const double cp = (k < nz - 1) ? sup * ivd : 0.0;
        tb.livd[k] = (T)ivd;
        tb.lcp[k] = (T)cp;
        cp_prev = cp;
    }
}

// b = D(u, v, w) into r and r~; partials: ||b||^2.  (Stencil tiles.)
template <typename T>
__global__ void __launch_bounds__(kKryThreads) k_kry_rhs(Grid<T> g, Tabs<T> tb, const T* u, const T* v, const T* w,
                                                         T* r, T* rt, Reduce rd) {
    T acc = 0;
    Col cl;
    if (tile_column(g, cl)) {
        T wb = (cl.k0 > 0) ? w[(size_t)cl.k0 * g.plane + cl.c] : (T)0;
        for (int k = cl.k0; k < cl.k1; ++k) {
            const size_t o = (size_t)k * g.plane;
            const T wa = (k < g.nz - 1) ? w[o + g.plane + cl.c] : (T)0;
            const T d = (u[o + cl.c] - u[o + cl.cw]) * g.idx + (v[o + cl.c] - v[o + cl.cs]) * g.idy +
                        (tb.fhi[k] * wa - tb.flo[k] * wb);
            r[o + cl.c] = d;
            rt[o + cl.c] = d;
            acc += d * d;
            wb = wa;
        }
    }
    block_reduce((double)acc, 0.0, rd, tile_slot());
}

// y = L x; partials: (a, y) and, if yy, (y, y).  (Stencil tiles.)  FP32:
// the operands of kApplyBatch levels are loaded before the first is used;
// FP64 marches up the levels keeping the vertical neighbours in registers
// (the batched form needs 118 registers and measured slower).
template <typename T>
__global__ void __launch_bounds__(kKryThreads) k_kry_apply(Grid<T> g, Tabs<T> tb, const T* x, T* y, const T* a,
                                                           bool yy, Reduce rd) {
    if (rd.sc->done || rd.sc->half) return;
    T s1 = 0, s2 = 0;
    Col cl;
    if constexpr (sizeof(T) == 8) {
        if (tile_column(g, cl)) {
            T xd = (cl.k0 > 0) ? x[(size_t)(cl.k0 - 1) * g.plane + cl.c] : (T)0;
            T xc = x[(size_t)cl.k0 * g.plane + cl.c];
            for (int k = cl.k0; k < cl.k1; ++k) {
                const size_t o = (size_t)k * g.plane;
                const T xu = (k < g.nz - 1) ? x[o + g.plane + cl.c] : (T)0;
                const T o1 = (x[o + cl.ce] - (T)2 * xc + x[o + cl.cw]) * g.idx2 +
                             (x[o + cl.cn] - (T)2 * xc + x[o + cl.cs]) * g.idy2 + tb.vdiag[k] * xc +
                             tb.vsub[k] * xd + tb.vsup[k] * xu;
                y[o + cl.c] = o1;
                s1 += a[o + cl.c] * o1;
                if (yy) s2 += o1 * o1;
                xd = xc;
                xc = xu;
            }
        }
    } else if (tile_column(g, cl)) {
        constexpr int Zb = kApplyBatch;
        for (int kb = cl.k0; kb < cl.k1; kb += Zb) {
            T xc[Zb + 2], xe[Zb], xw[Zb], xn[Zb], xs[Zb], av[Zb];
            xc[0] = (kb > 0) ? x[(size_t)(kb - 1) * g.plane + cl.c] : (T)0;
#pragma unroll
            for (int i = 0; i <= Zb; ++i) {
                const int k = kb + i;
                xc[i + 1] = (k < g.nz) ? x[(size_t)k * g.plane + cl.c] : (T)0;
            }
#pragma unroll
            for (int i = 0; i < Zb; ++i) {
                const int k = kb + i;
                const size_t o = (size_t)(k < cl.k1 ? k : kb) * g.plane;
                xe[i] = x[o + cl.ce];
                xw[i] = x[o + cl.cw];
                xn[i] = x[o + cl.cn];
                xs[i] = x[o + cl.cs];
                av[i] = a[o + cl.c];
            }
#pragma unroll
            for (int i = 0; i < Zb; ++i) {
                const int k = kb + i;
                if (k < cl.k1) {
                    const T c = xc[i + 1];
                    const T o1 = (xe[i] - (T)2 * c + xw[i]) * g.idx2 + (xn[i] - (T)2 * c + xs[i]) * g.idy2 +
                                 tb.vdiag[k] * c + tb.vsub[k] * xc[i] + tb.vsup[k] * xc[i + 2];   // vsub[0] = vsup[nz-1] = 0
                    y[(size_t)k * g.plane + cl.c] = o1;
                    s1 += av[i] * o1;
                    if (yy) s2 += o1 * o1;
                }
            }
        }
    }
    block_reduce((double)s1, (double)s2, rd, tile_slot());
}

// out = M^-1 in: Thomas down every column of the line matrix, one thread per
// column, kLineBatch levels loaded before use; the forward sweep leaves its
// values in out.
template <typename T>
__global__ void __launch_bounds__(kKryThreads, 2) k_kry_line(Grid<T> g, Tabs<T> tb, const T* __restrict__ in,
                                                          T* __restrict__ out, const KrySc* sc) {
    if (sc->done || sc->half) return;
    constexpr int B = kLineBatch<T>;
    const T* __restrict__ vsub = tb.vsub;
    const T* __restrict__ livd = tb.livd;
    const T* __restrict__ lcp = tb.lcp;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < g.plane; c += (size_t)gridDim.x * blockDim.x) {
        T dp = 0;
        for (int kb = 0; kb < g.nz; kb += B) {
            T b[B];
#pragma unroll
            for (int i = 0; i < B; ++i) b[i] = (kb + i < g.nz) ? in[(size_t)(kb + i) * g.plane + c] : (T)0;
#pragma unroll
            for (int i = 0; i < B; ++i) {
                const int k = kb + i;
                if (k < g.nz) {
                    dp = (b[i] - __ldg(&vsub[k]) * dp) * __ldg(&livd[k]);      // vsub[0] = 0
                    out[(size_t)k * g.plane + c] = dp;
                }
            }
        }
        T xk = dp;
        for (int kb = g.nz - 2; kb >= 0; kb -= B) {
            T b[B];
#pragma unroll
            for (int i = 0; i < B; ++i) b[i] = (kb - i >= 0) ? out[(size_t)(kb - i) * g.plane + c] : (T)0;
#pragma unroll
            for (int i = 0; i < B; ++i) {
                const int k = kb - i;
                if (k >= 0) {
                    xk = b[i] - __ldg(&lcp[k]) * xk;
                    out[(size_t)k * g.plane + c] = xk;
                }
            }
        }
    }
}

// Streaming kernels: thread t takes elements t + m * stride for m < kKryIlp,
// then the next kKryIlp * stride.
#define KRY_STREAM_LOOP(body)                                                              \
    {                                                                                      \
        const size_t stride = (size_t)gridDim.x * blockDim.x;                              \
        for (size_t q0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q0 < g.n;          \
             q0 += stride * kKryIlp) {                                                     \
            _Pragma("unroll") for (int m = 0; m < kKryIlp; ++m) {                          \
                const size_t q = q0 + m * stride;                                          \
                if (q < g.n) { body }                                                      \
            }                                                                              \
        }                                                                                  \
    }

// p = r (first iteration) or p = r + beta (p - omega v).
template <typename T>
__global__ void __launch_bounds__(kKryThreads) k_kry_p(Grid<T> g, T* p, const T* r, const T* v, bool first,
                                                       const KrySc* sc) {
    if (sc->done) return;
    const T beta = (T)sc->beta, omega = (T)sc->omega;
    KRY_STREAM_LOOP(p[q] = first ? r[q] : r[q] + beta * (p[q] - omega * v[q]);)
}

// s = r - alpha v (into r); partials: ||s||^2.
template <typename T>
__global__ void __launch_bounds__(kKryThreads) k_kry_s(Grid<T> g, T* r, const T* v, Reduce rd) {
    if (rd.sc->done) return;
    const T alpha = (T)rd.sc->alpha;
    T acc = 0;
    KRY_STREAM_LOOP(const T s = r[q] - alpha * v[q]; r[q] = s; acc += s * s;)
    block_reduce((double)acc, 0.0, rd, blockIdx.x);
}

// x += y: FP64 in place, FP32 as x_hi + x_lo with Knuth's TwoSum.
__device__ __forceinline__ void acc_x(double* xh, double*, size_t q, double y) { xh[q] = xh[q] + y; }
__device__ __forceinline__ void acc_x(float* xh, float* xl, size_t q, float y) {
    const float a = xh[q];
    const float s = a + y;
    const float bb = s - a;
    const float err = (a - (s - bb)) + (y - bb);
    xh[q] = s;
    xl[q] = xl[q] + err;
}

// x += alpha p^ + omega s^, r = s - omega t (r holds s); partials: ||r||^2,
// (r~, r).  After a half-step end only x += alpha p^.  (FP64 plans add the
// two terms one after the other, as (x + alpha p^) + omega s^.)
template <typename T>
__global__ void __launch_bounds__(kKryThreads) k_kry_update(Grid<T> g, T* xh, T* xl, const T* ph, const T* sh, T* r,
                                                            const T* t, const T* rt, Reduce rd) {
    const KrySc* sc = rd.sc;
    if (sc->done) return;
    const T alpha = (T)sc->alpha;
    if (sc->half) {
        KRY_STREAM_LOOP(acc_x(xh, xl, q, alpha * ph[q]);)
        block_reduce(0.0, 0.0, rd, blockIdx.x);
        return;
    }
    const T om = (T)sc->omega;
    T rr = 0, rtr = 0;
    if constexpr (sizeof(T) == 8) {
        KRY_STREAM_LOOP(xh[q] = (xh[q] + alpha * ph[q]) + om * sh[q]; const T rn = r[q] - om * t[q]; r[q] = rn;
                        rr += rn * rn; rtr += rt[q] * rn;)
    } else {
        KRY_STREAM_LOOP(acc_x(xh, xl, q, alpha * ph[q] + om * sh[q]); const T rn = r[q] - om * t[q]; r[q] = rn;
                        rr += rn * rn; rtr += rt[q] * rn;)
    }
    block_reduce((double)rr, (double)rtr, rd, blockIdx.x);
}

__device__ __forceinline__ double x_at(const double* xh, const double*, size_t q) { return xh[q]; }
__device__ __forceinline__ double x_at(const float* xh, const float* xl, size_t q) {
    return (double)xh[q] + (double)xl[q];
}

// Level-0 sum of x (the pin).
template <typename T>
__global__ void __launch_bounds__(kKryThreads) k_kry_level0(size_t plane, const T* xh, const T* xl, Reduce rd) {
    double acc = 0.0;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < plane; q += (size_t)gridDim.x * blockDim.x)
        acc += x_at(xh, xl, q);
    block_reduce(acc, 0.0, rd, blockIdx.x);
}

// u_out = u - G phi with phi the iterate shifted by the pin; w zero on the
// bottom and top faces.  (Stencil tiles.)  FP64 plans: in FP64.  FP32: the
// differences of x = x_hi + x_lo are taken part by part, (x_hi' - x_hi) +
// (x_lo' - x_lo); each part's difference of two floats is rounded once,
// relative to the difference itself, so the gradient keeps FP32 accuracy
// relative to G phi (not to phi) without FP64 arithmetic.
template <typename T>
__global__ void __launch_bounds__(kKryThreads) k_kry_correct(Grid<T> g, const T* xh, const T* xl, const T* u,
                                                             const T* v, const T* w, const double* idzn, T* uo, T* vo,
                                                             T* wo, T* phi, const KrySc* sc) {
    Col cl;
    if (!tile_column(g, cl)) return;
    const double m = sc->mean;
    if constexpr (sizeof(T) == 8) {
        double xd = (cl.k0 > 0) ? xh[(size_t)(cl.k0 - 1) * g.plane + cl.c] - m : 0.0;
        for (int k = cl.k0; k < cl.k1; ++k) {
            const size_t o = (size_t)k * g.plane;
            const size_t q = o + cl.c;
            const double c = xh[q] - m;
            uo[q] = u[q] - ((xh[o + cl.ce] - m) - c) * g.idx64;
            vo[q] = v[q] - ((xh[o + cl.cn] - m) - c) * g.idy64;
            wo[q] = (k > 0) ? w[q] - (c - xd) * idzn[k] : 0.0;
            if (phi) phi[q] = c;
            xd = c;
        }
    } else {
        const size_t qd = (size_t)(cl.k0 > 0 ? cl.k0 - 1 : 0) * g.plane + cl.c;
        float hd = xh[qd], ld = xl[qd];
        for (int k = cl.k0; k < cl.k1; ++k) {
            const size_t o = (size_t)k * g.plane;
            const size_t q = o + cl.c;
            const float hc = xh[q], lc = xl[q];
            const float gx = (xh[o + cl.ce] - hc) + (xl[o + cl.ce] - lc);
            const float gy = (xh[o + cl.cn] - hc) + (xl[o + cl.cn] - lc);
            uo[q] = u[q] - gx * g.idx;
            vo[q] = v[q] - gy * g.idy;
            wo[q] = (k > 0) ? w[q] - ((hc - hd) + (lc - ld)) * (float)idzn[k] : 0.f;
            if (phi) phi[q] = (float)(((double)hc + (double)lc) - m);
            hd = hc;
            ld = lc;
        }
    }
    if (cl.k1 == g.nz) wo[g.n + cl.c] = (T)0;
}

template <typename T>
cudaError_t run(const KrylovProblem& kp, cudaStream_t st, KrylovResult* res) {
    const Shape sh = shape(kp.nx, kp.ny, kp.nz, kp.nsm);
    Ws<T> ws = carve<T>(kp.workspace, kp.nx, kp.ny, kp.nz, sh.nparts, nullptr);
    Grid<T> g;
    g.nx = kp.nx; g.ny = kp.ny; g.nz = kp.nz;
    g.plane = (size_t)kp.nx * kp.ny;
    g.n = g.plane * kp.nz;
    g.idx64 = 1.0 / kp.dx; g.idy64 = 1.0 / kp.dy;
    g.idx = (T)g.idx64; g.idy = (T)g.idy64;
    g.idx2 = (T)(g.idx64 * g.idx64); g.idy2 = (T)(g.idy64 * g.idy64);
    const double hdiag = -2.0 * g.idx64 * g.idx64 - 2.0 * g.idy64 * g.idy64;
    const int nblk = sh.nblk;
    const dim3 tb(kTileX, kTileY);
    const int cblk = (int)std::min<size_t>((size_t)nblk, (g.plane + kKryThreads - 1) / kKryThreads);
    const bool pc = kp.precond == 1;
    T* const ph = pc ? ws.ph : ws.p;          // M = I: p^ is p, s^ is s
    T* const shv = pc ? ws.sh : ws.r;
    const T* u = (const T*)kp.u; const T* v = (const T*)kp.v; const T* w = (const T*)kp.w;
    const int mi = kp.max_iter;
    cudaError_t e;
#define KRY_CHECK()                                      \
    if ((e = cudaGetLastError()) != cudaSuccess) return e
    if ((e = cudaMemsetAsync(ws.xh, 0, g.n * sizeof(T), st)) != cudaSuccess) return e;
    if (ws.xl && (e = cudaMemsetAsync(ws.xl, 0, g.n * sizeof(T), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(ws.ticket, 0, sizeof(unsigned), st)) != cudaSuccess) return e;
    auto rd = [&](int nparts, int stage, int it) {
        Reduce r;
        r.part = ws.part; r.ticket = ws.ticket; r.sc = ws.sc; r.nparts = nparts;
        r.stage = stage; r.iter = it; r.max_iter = mi; r.tol = kp.tol; r.plane = (double)g.plane;
        return r;
    };
    k_kry_tables<T><<<1, 32, 0, st>>>(ws.tab, kp.acoef, kp.svol, kp.rflo, kp.rfhi, kp.nz, hdiag);
    k_kry_rhs<T><<<sh.tiles, tb, 0, st>>>(g, ws.tab, u, v, w, ws.r, ws.rt, rd(sh.ntile, kStRhs, 0));
    KRY_CHECK();
    KrySc h{};
    if ((e = cudaMemcpyAsync(&h, ws.sc, sizeof(KrySc), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    for (int it = 1; it <= mi && !h.done; ++it) {
        const bool check = (it % kKryCheckEvery == 0) || it == mi;
        k_kry_p<T><<<nblk, kKryThreads, 0, st>>>(g, ws.p, ws.r, ws.v, it == 1, ws.sc);
        if (pc) k_kry_line<T><<<cblk, kKryThreads, 0, st>>>(g, ws.tab, ws.p, ws.ph, ws.sc);
        k_kry_apply<T><<<sh.tiles, tb, 0, st>>>(g, ws.tab, ph, ws.v, ws.rt, false, rd(sh.ntile, kStAlpha, it));
        k_kry_s<T><<<nblk, kKryThreads, 0, st>>>(g, ws.r, ws.v, rd(nblk, kStS, it));
        if (pc) k_kry_line<T><<<cblk, kKryThreads, 0, st>>>(g, ws.tab, ws.r, ws.sh, ws.sc);
        k_kry_apply<T><<<sh.tiles, tb, 0, st>>>(g, ws.tab, shv, ws.t, ws.r, true, rd(sh.ntile, kStOmega, it));
        k_kry_update<T><<<nblk, kKryThreads, 0, st>>>(g, ws.xh, ws.xl, ph, shv, ws.r, ws.t, ws.rt,
                                                      rd(nblk, kStR, it));
        KRY_CHECK();
        if (!check) continue;
        if ((e = cudaMemcpyAsync(&h, ws.sc, sizeof(KrySc), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    }
    k_kry_level0<T><<<cblk, kKryThreads, 0, st>>>(g.plane, ws.xh, ws.xl, rd(cblk, kStMean, 0));
    k_kry_correct<T><<<sh.tiles, tb, 0, st>>>(g, ws.xh, ws.xl, u, v, w, kp.idzn, (T*)kp.u_out, (T*)kp.v_out,
                                              (T*)kp.w_out, (T*)kp.phi_out, ws.sc);
    KRY_CHECK();
#undef KRY_CHECK
    res->iterations = h.done ? h.iters : mi;
    res->rel_residual = h.relres;
    res->status = h.done ? h.status : 1;
    return cudaSuccess;
}

}  // namespace

size_t krylov_workspace_bytes(int nx, int ny, int nz, int nsm, bool fp32) {
    size_t bytes = 0;
    const int np = shape(nx, ny, nz, nsm).nparts;
    if (fp32) carve<float>(nullptr, nx, ny, nz, np, &bytes);
    else carve<double>(nullptr, nx, ny, nz, np, &bytes);
    return bytes;
}

cudaError_t krylov_run(const KrylovProblem& kp, cudaStream_t st, KrylovResult* res) {
    return kp.fp32 ? run<float>(kp, st, res) : run<double>(kp, st, res);
}

}  // namespace mp
