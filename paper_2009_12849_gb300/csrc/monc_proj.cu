// C ABI of the anelastic pressure projection (paper, Section 4): plan
// construction, workspace layout, launch sequence and status handling.
#include "monc_proj.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <vector>

#include <cudaTypedefs.h>

#include "krylov.h"
#include "pickers.h"
#include "group.cuh"
#include "pipe.cuh"

using namespace mp;

struct monc_proj_plan_s {
    int nx, ny, nz, nxh, nxp, precision;
    int precision_api;                    // as requested (MONC_PROJ_MIXED_Z64 runs as MONC_PROJ_MIXED)
    double dx, dy;
    FftFactors fx, fy;
    int device;
    // device tables (one allocation)
    void* dev_tables;
    const void* twx; const void* twy;
    const void* twy16;                    // y twiddles of the E = 16 schedule (FP32, ny = 256/512/1024), or null
    const double* svol; const double* rflo; const double* rfhi;
    const double* acoef; const double* idzn; const double* csum;
    const float* svol32; const float* acoef32; const float* csum32; const float* idzn32;
    const float* rflo32; const float* rfhi32;
    double lam_fp64;
    long long fp64_cols;
    int nslots;                           // columns of the FP64 warps with a 1/e table (mixed plans)
    int nwr;                              // warps per spectral row of the vertical solve
    size_t gtab_bytes;                    // bytes of that table
    const int* wlist;                     // device: (ky, kx0) of each FP64 warp
    const int* wslot;                     // device: [ny][nwr] first slot of a warp, or -1
    float2* pvm;                          // device: [nz][nslots] a_k / e_{k-1} (FP32 pair)
    float4* pvgb;                         // device: [nz][nslots] (1/e_k, a_{k+1} / e_k) (FP32 pairs)
    const double* lamx; const double* lamy;
    const void* ex; const void* ey;
    int* err;
    // task shapes
    int rows_fwd, nrb_fwd, tw_cols, ntiles;
    int thr_fwd_rows, thr_cols;
    int rows_inv[2], thr_inv_rows[2];
    int nsm;                              // SMs of the plan's device (persistent grids)
    bool persist_cols;                    // compile-time lengths: persistent cp.async column kernels
    bool ct_rows;                         // compile-time length along x
    bool ct_cols;                         // compile-time length along y
    bool fused;                           // square compile-time grid: fused persistent kernels
    int row_threads, col_threads;         // threads of a compile-time row task / column tile
    int col_e;                            // radix schedule of the compile-time column plans (elements per thread)
    int refine_passes;                    // MONC_PROJ_REFINED: passes per solve
    bool tma_cols;                        // FP32 compile-time column lengths: TMA-staged column kernels
    size_t smem_tma;                      // their dynamic shared memory (two tile buffers)
    int ring;                             // levels in the L2 rings of the fused kernels
    int lag;                              // producer/consumer lag of the fused kernels
    int grid_fwd_fused, grid_inv_fused;
    int thr_fwd_fused, thr_inv_fused[2];
    size_t smem_fwd_fused, smem_inv_fused[2];
    size_t off_sync, sync_bytes;
    int bs_row, bs_col;
    size_t smem_fwd_rows, smem_cols, smem_fcols, smem_inv_rows[2];
    bool pipe;                            // persistent pipelines of the transforms (pipe.cuh), opt-in
    int tc_cols;                          // tensor-core split-precision forward columns (tcdft.cuh), opt-in:
                                          // 0 off, 1 TF32 x 3, 2 BF16 x 6
    long long spin_limit;                 // polls before a bounded dependency wait gives up
    monc_proj_free_fn tables_free;        // how dev_tables is released (NULL: cudaFree)
    void* tables_user;
    bool pipe_ef;                         // their evict-first variants
    int pipe_lag_fwd, pipe_lag_inv;       // their producer/consumer lags in levels
    int grid_fwd_pipe, grid_inv_pipe;     // their grids (resident blocks)
    size_t smem_pipe;
    size_t off_groups, groups_bytes;      // pipelines: per (level, line group) counters of the hand-off
    // workspace layout
    size_t ws_bytes;
    size_t off_S, off_G, off_T, off_Tp, off_Tgy, off_Tgz, off_Tphi, off_Y, off_Gp, off_phipass, off_phimean;
    // per-phase timing
    bool profiling;
    int nprof;
    std::vector<cudaEvent_t> prof_events;
    std::vector<unsigned> prof_mask;
};

namespace {

constexpr int kPhases = 10;
const char* const kPhaseNames[kPhases] = {"fwd_rows", "fwd_cols", "tridiag", "inv_cols", "inv_rows",
                                          "fwd_fused", "inv_fused", "fwd_pipe", "inv_pipe", "fwd_cols_tc"};

// Start/end events of every phase of one recorded solve (null when not recording).
struct PhaseMarks {
    cudaEvent_t* ev = nullptr;       // [kPhases][2]
    unsigned* mask = nullptr;        // phases recorded in this solve
    void start(int ph, cudaStream_t st) const {
        if (ev) { cudaEventRecord(ev[2 * ph], st); *mask |= 1u << ph; }
    }
    void end(int ph, cudaStream_t st) const { if (ev) cudaEventRecord(ev[2 * ph + 1], st); }
};

PhaseMarks begin_marks(monc_proj_plan_s* p) {
    PhaseMarks m;
    if (!p->profiling || p->nprof >= MONC_PROJ_PROFILE_MAX) return m;
    const size_t need = (size_t)(p->nprof + 1) * (2 * kPhases);
    while (p->prof_events.size() < need) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return m;
        p->prof_events.push_back(e);
    }
    if (p->prof_mask.size() < (size_t)p->nprof + 1) p->prof_mask.resize(p->nprof + 1);
    m.ev = &p->prof_events[(size_t)p->nprof * (2 * kPhases)];
    m.mask = &p->prof_mask[p->nprof];
    *m.mask = 0;
    p->nprof++;
    return m;
}

constexpr size_t kSmemMax = 200 * 1024;
constexpr size_t kSmemPersist = 220 * 1024;
// Mixed plans: a3 runs in FP64 for columns with |lambda| < kFp64Fraction * v_max.
// The FP32 sweep's contribution to the divergence residual was measured (in an
// FP32 emulation of the sweep) at about 7e-8 above this bound and grows to
// 2e-7..5e-7 when the lowest wavenumbers are included.
constexpr double kFp64Fraction = 0.02;

bool is_smooth(int n) {
    if (n < 1) return false;
    for (int f : {2, 3, 5})
        while (n % f == 0) n /= f;
    return n == 1;
}

FastDiv make_fastdiv(unsigned d) {
    unsigned sh = 0;
    while ((1u << sh) < d) ++sh;
    const unsigned long long m = ((1ull << 32) * ((1ull << sh) - d)) / d + 1;
    return FastDiv{(unsigned)m, sh};
}

// Stockham radix plan, largest radices first (32 at most in FP32, 16 in FP64
// where a 32-point register DFT would not fit the register file).
// ct: the stages of a compile-time plan (ct_radix, the rule the kernels
// unroll); otherwise the run-time plan's radices 32/16/8/4/2 (up to maxrad),
// then 5, then 3.
FftFactors factorize(int n, int maxrad, bool ct) {
    FftFactors f{};
    f.n = n;
    int m = n, s = 0, ns = 1;
    auto push = [&](int r) {
        FftStage& st = f.st[s++];
        st.radix = r;
        st.ns = ns;
        st.nq = n / r;
        st.fq = make_fastdiv((unsigned)st.nq);
        st.fns = make_fastdiv((unsigned)ns);
        ns *= r;
        m /= r;
    };
    if (ct) {
        while (m > 1) push(ct_stage_radix(n, ns, maxrad));
    } else {
        for (int r : {32, 16, 8, 4, 2})
            while (r <= maxrad && m % r == 0) push(r);
        while (m % 5 == 0) push(5);
        while (m % 3 == 0) push(3);
    }
    f.nstages = s;
    return f;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// The persistent cp.async inverse-column kernel is opt-in (MONC_PROJ_PERSIST_COLS=1).
bool persist_cols_enabled() {
    const char* e = std::getenv("MONC_PROJ_PERSIST_COLS");
    return e && e[0] == '1';
}

int env_int(const char* name, int dflt) {
    const char* e = std::getenv(name);
    return (e && *e) ? std::max(1, std::atoi(e)) : dflt;
}

// As env_int, but 0 is allowed.
long long env_ll0(const char* name, long long dflt) {
    const char* e = std::getenv(name);
    return (e && *e) ? std::max(0ll, std::atoll(e)) : dflt;
}

// Polls of a bounded dependency wait (pipelines, fused kernels) before it
// gives up and latches the timeout bit, about a second at the 64 ns poll
// interval; MONC_PROJ_SPIN_LIMIT, read when the plan is made, overrides it
// (0 gives up at the first poll that finds the dependency unmet, which lets
// a test drive the timeout path without hanging anything).
constexpr long long kSpinLimit = 1ll << 24;

// Process-wide allocator of plan tables (monc_proj_set_allocator).
std::mutex g_alloc_mu;
monc_proj_alloc_fn g_alloc = nullptr;
monc_proj_free_fn g_free = nullptr;
void* g_alloc_user = nullptr;

// The fused persistent kernels are opt-in (MONC_PROJ_FUSED=1 in the
// environment; MONC_PROJ_FUSED_LAG and MONC_PROJ_FUSED_RING set the
// producer/consumer lag and the ring depth in levels): on GB300 they measured
// slower than the split kernels at every lag and ring depth tried.
bool fused_disabled() {
    const char* e = std::getenv("MONC_PROJ_FUSED");
    return !(e && e[0] == '1');
}

// Block size for a batch of `elems` transform elements at E per thread.
int threads_for(int elems, int E) {
    int t = (elems + E - 1) / E;
    t = (t + 31) & ~31;
    return std::max(32, std::min(512, t));
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

// Persistent pipelines (pipe.cuh) replace the four transform launches of
// mixed plans on square grids of 256, 512 or 1024 when MONC_PROJ_PIPE=1 (read
// when the plan is made): they hand the intermediate spectra over in L2 and
// cut the DRAM traffic of the transforms to the fields and D^, but measured
// slower than the one-launch-per-pass kernels, whose time is set by
// instruction issue rather than DRAM.  Lags in levels: the forward pass has
// about 130 tasks per level of 1024^2, the inverse 320.
constexpr int kPipeLagFwd = 4;
constexpr int kPipeLagInv = 2;
bool pipe_enabled() {
    const char* e = std::getenv("MONC_PROJ_PIPE");
    return e && e[0] == '1';
}

// exp(-2 pi i m / n): *c = cos(2 pi m/n), *s = -sin(2 pi m/n).  The angle is
// reduced exactly (integer arithmetic) to [0, pi/4] before libm is called.
void twiddle(int m, int n, double* c, double* s) {
    const double half_pi = 1.57079632679489661923;
    const long long mm = ((long long)m % n + n) % n;
    const long long q = (4 * mm) / n;            // quadrant 0..3
    const long long r = 4 * mm - q * n;          // angle in quadrant = (pi/2) r / n
    double c0, s0;
    if (2 * r <= n) {
        const double ph = half_pi * (double)r / (double)n;
        c0 = std::cos(ph); s0 = std::sin(ph);
    } else {
        const double ps = half_pi * (double)(n - r) / (double)n;
        c0 = std::sin(ps); s0 = std::cos(ps);
    }
    double cs, sn;
    switch (q) {
        case 0: cs = c0; sn = s0; break;
        case 1: cs = -s0; sn = c0; break;
        case 2: cs = -c0; sn = -s0; break;
        default: cs = s0; sn = -c0; break;
    }
    *c = cs;
    *s = -sn;
}

// sin(pi m / n)^2 -> used for 2(cos(2 pi m/n) - 1) = -4 sin^2(pi m/n) without cancellation
double sin_half_sq(int m, int n) {
    double c, s;
    twiddle(m, 2 * n, &c, &s);   // exp(-i pi m / n): s = -sin(pi m/n)
    return s * s;
}

template <typename R>
void push_complex(std::vector<unsigned char>& blob, const std::vector<double>& re,
                  const std::vector<double>& im) {
    for (size_t i = 0; i < re.size(); ++i) {
        R v[2] = {(R)re[i], (R)im[i]};
        const unsigned char* b = (const unsigned char*)v;
        blob.insert(blob.end(), b, b + sizeof(v));
    }
}

void push_doubles(std::vector<unsigned char>& blob, const std::vector<double>& x) {
    const unsigned char* b = (const unsigned char*)x.data();
    blob.insert(blob.end(), b, b + x.size() * sizeof(double));
}

void push_floats(std::vector<unsigned char>& blob, const std::vector<double>& x) {
    for (double v : x) {
        const float f = (float)v;
        const unsigned char* b = (const unsigned char*)&f;
        blob.insert(blob.end(), b, b + sizeof(float));
    }
}

void pad_blob(std::vector<unsigned char>& blob) {
    while (blob.size() % 256) blob.push_back(0);
}

int nz_all_levels(const monc_proj_plan_s* p) { return p->nz; }

ProjParams make_params(const monc_proj_plan_s* p, const void* u, const void* v, const void* w,
                       void* uo, void* vo, void* wo, void* phi, void* ws) {
    ProjParams q{};
    q.nx = p->nx; q.ny = p->ny; q.nz = p->nz; q.nxh = p->nxh; q.nxp = p->nxp;
    q.fx = p->fx; q.fy = p->fy;
    q.twx = p->twx; q.twy = p->twy; q.twy16 = p->twy16;
    q.svol = p->svol; q.rflo = p->rflo; q.rfhi = p->rfhi; q.acoef = p->acoef; q.idzn = p->idzn;
    q.csum = p->csum; q.svol32 = p->svol32; q.acoef32 = p->acoef32; q.csum32 = p->csum32;
    q.rflo32 = p->rflo32; q.rfhi32 = p->rfhi32;
    q.idzn32 = p->idzn32; q.lam_fp64 = p->lam_fp64;
    q.lamx = p->lamx; q.lamy = p->lamy; q.ex = p->ex; q.ey = p->ey;
    q.idx = 1.0 / p->dx; q.idy = 1.0 / p->dy;
    q.idx32 = (float)q.idx; q.idy32 = (float)q.idy;
    q.scale = 1.0 / ((double)p->nx * (double)p->ny);
    q.u = u; q.v = v; q.w = w; q.uo = uo; q.vo = vo; q.wo = wo; q.phi = phi;
    unsigned char* b = (unsigned char*)ws;
    q.S = b + p->off_S; q.G = b + p->off_G; q.T = b + p->off_T;
    q.Tp = b + p->off_Tp; q.Tgy = b + p->off_Tgy; q.Tgz = b + p->off_Tgz; q.Tphi = b + p->off_Tphi;
    q.Y = (double2*)(b + p->off_Y); q.Gp = (double*)(b + p->off_Gp);
    q.sync = (unsigned*)(b + p->off_sync);
    q.phi_pass = b + p->off_phipass;
    q.phi_mean = (double*)(b + p->off_phimean);
    q.ring = p->fused ? p->ring : nz_all_levels(p);
    q.lag = p->lag;
    q.err = p->err;
    q.rows_fwd = p->rows_fwd; q.nrb_fwd = p->nrb_fwd;
    q.tw_cols = p->tw_cols; q.ntiles = p->ntiles;
    q.bs_row = p->bs_row; q.bs_col = p->bs_col;
    q.nch = phi ? 4 : 3;
    q.spin_limit = p->spin_limit;
    q.kbase = 0;
    q.nz_glob = p->nz;
    q.ky_base = 0;
    q.pvm = p->pvm; q.pvgb = p->pvgb; q.wslot = p->wslot; q.nslots = p->nslots; q.nwr = p->nwr;
    q.rows_inv = p->rows_inv[q.nch == 4 ? 1 : 0];
    q.nrb_inv = (p->ny + q.rows_inv - 1) / q.rows_inv;
    return q;
}

// ---------------------------------------------------------------------------
// Kernel selection: lengths with a compile-time FFT plan get their own
// instantiation; every other 2^a 3^b 5^c length runs the run-time plan.
// ---------------------------------------------------------------------------
bool ct_length(int n, bool fp64) {
    if (fp64) return n == 64 || n == 128 || n == 256 || n == 1024;
    return ct_length_f32(n);
}

// Lengths that also have the opt-in kernel variants (persistent, TMA, fused).
bool ct_core_length(int n, bool fp64) { return fp64 ? ct_length(n, true) : ct_core_f32(n); }


struct SolveKernels {
    KernelFn fwd_rows, fwd_cols, inv_cols, inv_rows;
};

template <typename R> SolveKernels pick_kernels(const monc_proj_plan_s* p) {
    const int nx = p->nx, ny = p->ny;
    const bool ref = p->precision == MONC_PROJ_REFINED;
    SolveKernels ks{ref ? pick_refined_fwd_rows(nx) : pick_k_fwd_rows<R>(nx),
                    pick_k_fwd_cols<R>(ny),
                    ref ? pick_refined_inv_cols(ny)
                        : p->persist_cols ? pick_inv_cols_persist<R>(ny) : pick_k_inv_cols<R>(ny),
                    ref ? pick_refined_inv_rows(nx) : pick_k_inv_rows<R>(nx)};
    if (sizeof(R) == 4) {
        if (KernelFn f = pick_cols_square_f32(ny, p->nxp, p->tw_cols, p->bs_col, false, p->col_e)) ks.fwd_cols = f;
        if (!ref && !p->persist_cols)
            if (KernelFn f = pick_cols_square_f32(ny, p->nxp, p->tw_cols, p->bs_col, true, p->col_e)) ks.inv_cols = f;
    }
    return ks;
}

// ---------------------------------------------------------------------------
// Tensor maps of the TMA column kernels.  cuTensorMapEncodeTiled comes from
// the driver through the runtime's entry-point query, so the library needs no
// link-time dependency on the driver API.
// ---------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            f = nullptr;
        }
        return (PFN_cuTensorMapEncodeTiled_v12000)f;
    }();
    return fn;
}

// The TMA column kernels are opt-in (MONC_PROJ_TMA=1): they measured slower
// than the register-staged column kernels on GB300.
bool tma_enabled() {
    const char* e = std::getenv("MONC_PROJ_TMA");
    return e && e[0] == '1';
}

// 2D view of a spectral array [nz*ny rows][nxh valid columns], row pitch nxp
// complex values, boxes of tw columns x min(ny, 256) rows; columns at and past
// nxh read as zero and are not written.
bool encode_cols_map(const monc_proj_plan_s* p, CUtensorMap* m, const void* base) {
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
    if (!enc || !base) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)p->nxh, (cuuint64_t)p->nz * (cuuint64_t)p->ny};
    const cuuint64_t strides[1] = {(cuuint64_t)p->nxp * 8};
    const cuuint32_t box[2] = {(cuuint32_t)p->tw_cols, (cuuint32_t)std::min(p->ny, 256)};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<void*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_64B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Forward (T -> S) or inverse (S, G -> Tp, Tgy, Tgz[, Tphi]) column phase on
// the TMA kernels; false (nothing launched) if a map cannot be encoded.
template <typename R>
bool launch_cols_tma(const monc_proj_plan_s* p, const ProjParams& q, bool inv, cudaStream_t st) {
    const ColsTmaFn fn = pick_cols_tma<R>(p->ny, inv);
    if (!fn) return false;
    ColMaps m;
    std::memset(&m, 0, sizeof(m));
    bool ok;
    if (!inv) {
        ok = encode_cols_map(p, &m.src[0], q.T) && encode_cols_map(p, &m.dst[0], q.S);
    } else {
        ok = encode_cols_map(p, &m.src[0], q.S) && encode_cols_map(p, &m.src[1], q.G) &&
             encode_cols_map(p, &m.dst[0], q.Tp) && encode_cols_map(p, &m.dst[1], q.Tgy) &&
             encode_cols_map(p, &m.dst[2], q.Tgz) && (q.nch < 4 || encode_cols_map(p, &m.dst[3], q.Tphi));
    }
    if (!ok) return false;
    const long long items = (long long)p->nz * p->ntiles * (inv ? q.nch : 1);
    const int grid = (int)std::min<long long>(items, p->nsm);
    fn<<<grid, p->thr_cols, p->smem_tma, st>>>(q, m);
    return true;
}

// Forward pipeline, vertical solve, inverse pipeline (pipe.cuh).
int launch_piped(monc_proj_plan_s* p, const ProjParams& q, cudaStream_t st, const PhaseMarks& pm) {
    const int nz = p->nz;
    unsigned* groups = (unsigned*)((unsigned char*)q.S - p->off_S + p->off_groups);
    if (cudaMemsetAsync(q.sync, 0, (size_t)(2 + 2 * nz) * sizeof(unsigned), st) != cudaSuccess ||
        cudaMemsetAsync(groups, 0, p->groups_bytes, st) != cudaSuccess) {
        cudaGetLastError();
        return MONC_PROJ_ECUDA;
    }
    ProjParams qp = q;
    qp.ho.discard = 1;
    qp.ho.groups = groups;
    const long long per_fwd = (long long)nz * ((p->ny + 1) / 2 + p->ntiles);
    const long long per_inv = (long long)nz * (2 * p->ntiles + p->ny);
    pm.start(7, st);
    qp.lag = p->pipe_lag_fwd;
    pick_fwd_pipe(p->nx, p->ny, p->pipe_ef)<<<(unsigned)std::min<long long>(p->grid_fwd_pipe, per_fwd), kPipeThreads, p->smem_pipe,
                                  st>>>(qp);
    pm.end(7, st);
    const long long ncol = (long long)p->ny * ((p->nxh + 31) & ~31);
    pm.start(2, st);
    pick_tridiag<float>()<<<(unsigned)((ncol + kTriThreads - 1) / kTriThreads), kTriThreads, 0, st>>>(q);
    pm.end(2, st);
    pm.start(8, st);
    qp.lag = p->pipe_lag_inv;
    pick_inv_pipe(p->nx, p->ny, p->pipe_ef)<<<(unsigned)std::min<long long>(p->grid_inv_pipe, per_inv), kPipeThreads, p->smem_pipe,
                                  st>>>(qp);
    pm.end(8, st);
    return cudaGetLastError() == cudaSuccess ? MONC_PROJ_OK : MONC_PROJ_ECUDA;
}

template <typename R>
int launch_solve(monc_proj_plan_s* p, const ProjParams& q, cudaStream_t st) {
    const int nz = p->nz;
    const int inv_idx = (q.nch == 4) ? 1 : 0;
    const PhaseMarks pm = begin_marks(p);
    const long long ncol = (long long)p->ny * ((p->nxh + 31) & ~31);
    if (p->pipe && sizeof(R) == 4) return launch_piped(p, q, st, pm);
    if (p->fused) {
        if (cudaMemsetAsync(q.sync, 0, p->sync_bytes, st) != cudaSuccess) { cudaGetLastError(); return MONC_PROJ_ECUDA; }
        pm.start(5, st);
        pick_fwd_fused<R>(p->nx)<<<p->grid_fwd_fused, p->thr_fwd_fused, p->smem_fwd_fused, st>>>(q);
        pm.end(5, st);
        pm.start(2, st);
        pick_tridiag<R>()<<<(unsigned)((ncol + kTriThreads - 1) / kTriThreads), kTriThreads, 0, st>>>(q);
        pm.end(2, st);
        pm.start(6, st);
        pick_inv_fused<R>(p->nx)<<<p->grid_inv_fused, p->thr_inv_fused[inv_idx], p->smem_inv_fused[inv_idx], st>>>(q);
        pm.end(6, st);
    } else {
        const SolveKernels ks = pick_kernels<R>(p);
        const int n_fcols = nz * p->ntiles;
        const int n_icols = nz * p->ntiles * ((p->persist_cols || p->ct_cols) ? 2 : q.nch);
        const int n_irows = nz * q.nrb_inv * (p->ct_rows ? q.nch : 1);
        pm.start(0, st);
        ks.fwd_rows<<<nz * p->nrb_fwd, p->thr_fwd_rows, p->smem_fwd_rows, st>>>(q);
        pm.end(0, st);
        const int fc_phase = (p->tc_cols && sizeof(R) == 4) ? 9 : 1;
        pm.start(fc_phase, st);
        if (fc_phase == 9) {
            // the tensor-core kernel's own tiles of 8 columns
            ProjParams qt = q;
            qt.ntiles = (p->nxh + 7) / 8;
            pick_fwd_cols_tc(p->ny, p->tc_cols)<<<nz * qt.ntiles, 256, fwd_cols_tc_smem(p->tc_cols), st>>>(qt);
        } else if (!(p->tma_cols && launch_cols_tma<R>(p, q, false, st))) {
            ks.fwd_cols<<<n_fcols, p->thr_cols, p->smem_fcols, st>>>(q);
        }
        pm.end(fc_phase, st);
        pm.start(2, st);
        pick_tridiag<R>()<<<(unsigned)((ncol + kTriThreads - 1) / kTriThreads), kTriThreads, 0, st>>>(q);
        pm.end(2, st);
        pm.start(3, st);
        if (p->persist_cols && cudaMemsetAsync(q.sync, 0, sizeof(unsigned), st) != cudaSuccess) {
            cudaGetLastError();
            return MONC_PROJ_ECUDA;
        }
        if (!(p->tma_cols && launch_cols_tma<R>(p, q, true, st)))
            ks.inv_cols<<<p->persist_cols ? std::min(n_icols, p->nsm) : n_icols, p->thr_cols, p->smem_cols, st>>>(q);
        pm.end(3, st);
        pm.start(4, st);
        ks.inv_rows<<<n_irows, p->thr_inv_rows[inv_idx], p->smem_inv_rows[inv_idx], st>>>(q);
        pm.end(4, st);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MONC_PROJ_OK : MONC_PROJ_ECUDA;
}

// One projection on a plan.  Refinement plans run kRefinePasses passes on the
// FP64 fields: each pass solves for a potential with the mixed pipeline (the
// divergence of the pass's input formed in FP64) and subtracts that
// potential's discrete gradient in FP64.  The correction is an exact gradient,
// so the next pass's divergence is exactly the remaining error, and each pass
// shrinks it by the mixed solver's relative accuracy; phi is the sum of the
// passes' potentials.
constexpr int kRefinePasses = 3;                  // default; MONC_PROJ_REFINE_PASSES overrides (1..4)

int run_solve(monc_proj_plan_s* p, const ProjParams& q, cudaStream_t st) {
    if (p->precision == MONC_PROJ_FP64) return launch_solve<double>(p, q, st);
    if (p->precision != MONC_PROJ_REFINED) return launch_solve<float>(p, q, st);
    const int npass = p->refine_passes;
    for (int pass = 0; pass < npass; ++pass) {
        // the mixed pipeline produces this pass's potential alone ...
        ProjParams qp = q;
        if (pass > 0) {
            qp.u = q.uo;
            qp.v = q.vo;
            qp.w = q.wo;
        }
        qp.phi = q.phi_pass;
        qp.phi_only = 1;
        qp.nch = 1;
        qp.rows_inv = p->rows_inv[0];
        qp.nrb_inv = (p->ny + qp.rows_inv - 1) / qp.rows_inv;
        const int rc = launch_solve<float>(p, qp, st);
        if (rc != MONC_PROJ_OK) return rc;
        // ... and the correction subtracts its exact discrete gradient in FP64
        const bool last = pass + 1 == npass;
        if (q.phi) {
            if (pass == 0 && cudaMemsetAsync(q.phi_mean, 0, sizeof(double), st) != cudaSuccess) {
                cudaGetLastError();
                return MONC_PROJ_ECUDA;
            }
            k_mean_add<double><<<1, 1024, 0, st>>>((const double*)q.phi_pass, p->nx * p->ny, q.phi_mean);
        }
        k_fd_correct<double><<<p->nz * p->ny, 256, 0, st>>>(qp, (const double*)q.phi_pass, (double*)q.phi,
                                                            pass > 0 ? 1 : 0, last ? q.phi_mean : nullptr);
        if (cudaGetLastError() != cudaSuccess) return MONC_PROJ_ECUDA;
    }
    return MONC_PROJ_OK;
}

// Raise the dynamic shared-memory limit of the kernels a plan uses; fails if
// the plan's blocks need more than the device allows.  The L1/shared carveout
// is left to the driver: forcing the largest shared carveout (least L1)
// measured 30% slower, since the transforms re-read twiddles, Hermitian
// partners and neighbouring rows through L1.
template <typename R>
int set_kernel_attrs(const monc_proj_plan_s* p) {
    const size_t lim_cols = p->persist_cols ? kSmemPersist : kSmemMax;
    const size_t lim_rows = kSmemMax;
    if (p->smem_fwd_rows > kSmemMax || p->smem_cols > lim_cols || p->smem_fcols > kSmemMax ||
        std::max(p->smem_inv_rows[0], p->smem_inv_rows[1]) > lim_rows)
        return MONC_PROJ_EUNSUPPORTED;
    const SolveKernels ks = pick_kernels<R>(p);
    if (p->tma_cols) {
        for (int inv = 0; inv < 2; ++inv) {
            const ColsTmaFn f = pick_cols_tma<R>(p->ny, inv != 0);
            if (f && cudaFuncSetAttribute((const void*)f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)p->smem_tma) != cudaSuccess) {
                cudaGetLastError();
                return MONC_PROJ_ECUDA;
            }
        }
    }
    const KernelFn fns[] = {ks.fwd_rows, ks.fwd_cols, ks.inv_cols, ks.inv_rows};
    const size_t lims[] = {kSmemMax, kSmemMax, lim_cols, lim_rows};
    for (int i = 0; i < 4; ++i) {
        if (cudaFuncSetAttribute((const void*)fns[i], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lims[i]) !=
            cudaSuccess) {
            cudaGetLastError();
            return MONC_PROJ_ECUDA;
        }
    }
    return MONC_PROJ_OK;
}

// Fused path: raise the shared-memory limits and size the persistent grids
// from the occupancy of each kernel.
template <typename R>
int setup_fused(monc_proj_plan_s* p) {
    const KernelFn ff = pick_fwd_fused<R>(p->nx), fi = pick_inv_fused<R>(p->nx);
    if (!ff || !fi) { p->fused = false; return MONC_PROJ_OK; }
    const size_t smi = std::max(p->smem_inv_fused[0], p->smem_inv_fused[1]);
    if (p->smem_fwd_fused > kSmemMax || smi > kSmemMax) { p->fused = false; return MONC_PROJ_OK; }
    if (cudaFuncSetAttribute((const void*)ff, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax) != cudaSuccess ||
        cudaFuncSetAttribute((const void*)fi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax) != cudaSuccess) {
        cudaGetLastError();
        return MONC_PROJ_ECUDA;
    }
    int bf = 0, bi = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bf, (const void*)ff, p->thr_fwd_fused, p->smem_fwd_fused) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bi, (const void*)fi, std::max(p->thr_inv_fused[0], p->thr_inv_fused[1]),
                                                      smi) != cudaSuccess) {
        cudaGetLastError();
        return MONC_PROJ_ECUDA;
    }
    if (bf < 1 || bi < 1) { p->fused = false; return MONC_PROJ_OK; }
    p->grid_fwd_fused = bf * p->nsm;
    p->grid_inv_fused = bi * p->nsm;
    return MONC_PROJ_OK;
}

// Pipelines: raise their shared-memory limits and size their grids to the
// blocks that fit the device at once (the schedule needs no residency, but
// more blocks than fit would only wait for a slot).
int setup_pipe(monc_proj_plan_s* p) {
    const KernelFn ff = pick_fwd_pipe(p->nx, p->ny, p->pipe_ef), fi = pick_inv_pipe(p->nx, p->ny, p->pipe_ef);
    // the pipelines' column tasks have the padded pitch and the 256-thread tile
    // width compiled in (PipeCols)
    if (!ff || !fi || p->smem_pipe > kSmemMax || p->thr_cols != kPipeThreads ||
        p->tw_cols * p->ny != kPipeThreads * kMaxRadixF32 || p->nxp != ((p->nxh + 15) & ~15)) {
        p->pipe = false;
        return MONC_PROJ_OK;
    }
    int bf = 0, bi = 0;
    if (cudaFuncSetAttribute((const void*)ff, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->smem_pipe) != cudaSuccess ||
        cudaFuncSetAttribute((const void*)fi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->smem_pipe) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bf, (const void*)ff, kPipeThreads, p->smem_pipe) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bi, (const void*)fi, kPipeThreads, p->smem_pipe) != cudaSuccess) {
        cudaGetLastError();
        return MONC_PROJ_ECUDA;
    }
    if (bf < 1 || bi < 1) { p->pipe = false; return MONC_PROJ_OK; }
    p->grid_fwd_pipe = bf * p->nsm;
    p->grid_inv_pipe = bi * p->nsm;
    return MONC_PROJ_OK;
}

int plan_kernel_attrs(monc_proj_plan_s* p) {
    const int r = p->precision == MONC_PROJ_FP64 ? set_kernel_attrs<double>(p) : set_kernel_attrs<float>(p);
    if (r != MONC_PROJ_OK) return r;
    if (p->tc_cols && cudaFuncSetAttribute((const void*)pick_fwd_cols_tc(p->ny, p->tc_cols),
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)fwd_cols_tc_smem(p->tc_cols)) != cudaSuccess) {
        cudaGetLastError();
        p->tc_cols = 0;
    }
    if (p->pipe) {
        const int rp = setup_pipe(p);
        if (rp != MONC_PROJ_OK) return rp;
    }
    if (!p->fused) return MONC_PROJ_OK;
    return p->precision == MONC_PROJ_FP64 ? setup_fused<double>(p) : setup_fused<float>(p);
}

// Argument checks shared by every entry point that takes grid arguments.
int validate_grid(int nx, int ny, int nz, double dx, double dy, const double* dz,
                  const double* rho_c, const double* rho_f, int precision) {
    if (nx < 1 || ny < 1 || nz < 1 || !dz || !rho_c || !rho_f) return MONC_PROJ_EINVAL;
    if (precision != MONC_PROJ_FP64 && precision != MONC_PROJ_MIXED && precision != MONC_PROJ_REFINED &&
        precision != MONC_PROJ_MIXED_Z64)
        return MONC_PROJ_EINVAL;
    if (!finite_pos(dx) || !finite_pos(dy)) return MONC_PROJ_EINVAL;
    for (int k = 0; k < nz; ++k)
        if (!finite_pos(dz[k]) || !finite_pos(rho_c[k])) return MONC_PROJ_EINVAL;
    for (int k = 0; k <= nz; ++k)
        if (!finite_pos(rho_f[k])) return MONC_PROJ_EINVAL;
    if (nx > MONC_PROJ_MAX_N || ny > MONC_PROJ_MAX_N || !is_smooth(nx) || !is_smooth(ny))
        return MONC_PROJ_EUNSUPPORTED;

    return MONC_PROJ_OK;
}

// Offsets of the plan's device tables inside one contiguous blob.
struct TableOffsets {
    size_t twx, twy, twy16, sv, rl, rh, a, iz, cs, sv32, a32, cs32, iz32, rl32, rh32, lx, ly, ex, ey, err;
    size_t wlist, wslot;   // FP64 warps of a mixed plan: (ky, kx0) list and per-warp slot map
    size_t gtab;           // 1/e table of their columns, filled on the device (past the uploaded blob)
};

// Fill the host-side part of a plan (sizes, radix plans, task shapes,
// workspace layout) and build its device tables in `blob` (host memory).
// Task shapes of the row and column kernels.  Compile-time lengths: one
// shared buffer, blocks of p->row_threads (rows) or p->col_threads (column
// tiles) threads x E elements (E = the largest radix: 32 FP32, 16 FP64);
// monc_proj_autotune searches these two counts.  Run-time lengths: two
// buffers (ping-pong) within ~96 KB, 256 threads.  The shapes decide how work
// is split into blocks, never the arithmetic of a transform, so every choice
// gives bitwise the same result.
void set_task_shapes(monc_proj_plan_s* p) {
    const int nx = p->nx, ny = p->ny;
    const bool fp64 = p->precision == MONC_PROJ_FP64;
    const size_t csz = fp64 ? 16 : 8;
    const bool ctx = p->ct_rows, cty = p->ct_cols;
    const int E = fp64 ? kMaxRadixF64 : kMaxRadixF32;
    const int Ec = fp64 ? kMaxRadixF64 : p->col_e;      // the column plans' schedule
    p->bs_row = spad_len(nx);
    // column tiles: a pitch of 4 (mod 16) complex elements spreads the
    // columns of a tile over distinct shared-memory banks
    p->bs_col = spad_len(ny);
    while (p->bs_col % 16 != 4) ++p->bs_col;
    const size_t budget = 96 * 1024;
    int npair = ctx ? std::max(1, std::min(16, p->row_threads * E / nx))
                    : (int)std::max<size_t>(1, std::min<size_t>(8, budget / (2 * (size_t)p->bs_row * csz)));
    npair = std::min(npair, (ny + 1) / 2);
    p->rows_fwd = 2 * npair;
    p->nrb_fwd = (ny + p->rows_fwd - 1) / p->rows_fwd;
    p->thr_fwd_rows = ctx ? threads_for(npair * nx, E) : 256;
    p->smem_fwd_rows = (size_t)(ctx ? 1 : 2) * npair * p->bs_row * csz;
    int tw = cty ? std::max(1, std::min(32, p->col_threads * Ec / ny))
                 : (int)std::max<size_t>(1, std::min<size_t>(8, budget / (2 * (size_t)p->bs_col * csz)));
    tw = std::min(tw, p->nxh);
    p->tw_cols = tw;
    p->ntiles = (p->nxh + tw - 1) / tw;
    p->thr_cols = cty ? threads_for(tw * ny, Ec) : 256;
    p->smem_cols = (size_t)(cty ? 1 : 2) * tw * p->bs_col * csz;
    p->smem_fcols = p->smem_cols;
    // inverse row tasks: pairs of rows, one complex transform per channel and
    // row pair; index 0 without phi output (3 channels), 1 with (4 channels)
    for (int idx = 0; idx < 2; ++idx) {
        const int nch = 3 + idx;
        int pairs = std::max(1, npair / nch);
        pairs = std::min(pairs, (ny + 1) / 2);
        const int np = nch * pairs;
        p->rows_inv[idx] = 2 * pairs;
        p->thr_inv_rows[idx] = ctx ? threads_for(np * nx, E) : 256;
        p->smem_inv_rows[idx] = (size_t)(ctx ? 1 : 2) * np * p->bs_row * csz;
        if (ctx) {
            // one channel per task: rows_inv rows = rows_inv/2 transforms
            int npr = std::max(1, std::min({16, p->row_threads * E / nx, (ny + 1) / 2}));
            p->rows_inv[idx] = 2 * npr;
            p->thr_inv_rows[idx] = threads_for(npr * nx, E);
            p->smem_inv_rows[idx] = (size_t)npr * p->bs_row * csz;
        }
    }

}

void plan_prepare(monc_proj_plan_s* p, int nx, int ny, int nz, double dx, double dy,
                  const double* dz, const double* rho_c, const double* rho_f, int precision_api,
                  std::vector<unsigned char>& blob, TableOffsets& to) {
    // MONC_PROJ_MIXED_Z64 is a mixed plan whose every column runs a3 in FP64
    const bool z64 = precision_api == MONC_PROJ_MIXED_Z64;
    const int precision = z64 ? MONC_PROJ_MIXED : precision_api;
    p->precision_api = precision_api;
    p->nx = nx; p->ny = ny; p->nz = nz; p->dx = dx; p->dy = dy; p->precision = precision;
    p->nxh = nx / 2 + 1;
    p->nxp = (p->nxh + 3) & ~3;
    const bool fp64 = precision == MONC_PROJ_FP64;
    const int maxrad = fp64 ? kMaxRadixF64 : kMaxRadixF32;
    // compile-time plans along x and y (refinement passes: the x kernels on
    // FP64 fields exist for the core lengths only)
    const bool ctx = ct_length(nx, fp64) && (precision != MONC_PROJ_REFINED || ct_core_length(nx, false));
    const bool cty = ct_length(ny, fp64) && (precision != MONC_PROJ_REFINED || ct_core_length(ny, false));
    p->fx = factorize(nx, maxrad, ctx);
    p->fy = factorize(ny, maxrad, cty);

    const size_t csz = fp64 ? 16 : 8;
    {
        int dev = 0, nsm = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) {
            cudaGetLastError();
            nsm = 1;
        }
        p->nsm = nsm;
    }

    // ---- host tables
    std::vector<double> cx(nx), sx(nx), cy(ny), sy(ny);
    for (int m = 0; m < nx; ++m) twiddle(m, nx, &cx[m], &sx[m]);
    for (int m = 0; m < ny; ++m) twiddle(m, ny, &cy[m], &sy[m]);
    std::vector<double> zf(nz + 1, 0.0), zc(nz), dzn(nz + 1, 0.0);
    for (int k = 0; k < nz; ++k) zf[k + 1] = zf[k] + dz[k];
    for (int k = 0; k < nz; ++k) zc[k] = 0.5 * (zf[k] + zf[k + 1]);
    for (int k = 1; k < nz; ++k) dzn[k] = zc[k] - zc[k - 1];
    std::vector<double> svol(nz), rflo(nz), rfhi(nz), acoef(nz + 1, 0.0), idzn(nz + 1, 0.0);
    for (int k = 0; k < nz; ++k) {
        svol[k] = rho_c[k] * dz[k];
        rflo[k] = (k > 0) ? rho_f[k] : 0.0;
        rfhi[k] = (k < nz - 1) ? rho_f[k + 1] : 0.0;
    }
    for (int k = 1; k < nz; ++k) { acoef[k] = rho_f[k] / dzn[k]; idzn[k] = 1.0 / dzn[k]; }
    std::vector<double> csum(nz);
    for (int k = 0; k < nz; ++k) csum[k] = acoef[k] + acoef[k + 1];
    std::vector<double> lamx(p->nxh), lamy(ny);
    for (int m = 0; m < p->nxh; ++m) lamx[m] = -4.0 * sin_half_sq(m, nx) / (dx * dx);
    for (int m = 0; m < ny; ++m) lamy[m] = -4.0 * sin_half_sq(m, ny) / (dy * dy);
    // a3 precision split (mixed plans): columns whose |lambda| is below
    // kFp64Fraction of the largest vertical eigenvalue bound
    // v_max = max_k 2 (A[k] + A[k+1]) / (rho_c dz)[k] run in FP64.
    double vmax = 0.0;
    for (int k = 0; k < nz; ++k) vmax = std::max(vmax, 2.0 * (acoef[k] + acoef[k + 1]) / svol[k]);
    p->lam_fp64 = (precision == MONC_PROJ_FP64 || z64) ? INFINITY : kFp64Fraction * vmax;
    {
        const int nxw = (p->nxh + 31) & ~31;
        long long n64 = 0;
        for (int ky = 0; ky < ny; ++ky)
            for (int kx0 = 0; kx0 < p->nxh; kx0 += 32)
                if (-(lamx[kx0] + lamy[ky]) < p->lam_fp64) n64 += std::min(32, p->nxh - kx0);
        (void)nxw;
        p->fp64_cols = n64;
    }
    // (exp(+2 pi i m/n) - 1)/d = (-2 sin^2(pi m/n) + i sin(2 pi m/n)) / d
    std::vector<double> exr(p->nxh), exi(p->nxh), eyr(ny), eyi(ny);
    for (int m = 0; m < p->nxh; ++m) { exr[m] = -2.0 * sin_half_sq(m, nx) / dx; exi[m] = -sx[m] / dx; }
    for (int m = 0; m < ny; ++m) { eyr[m] = -2.0 * sin_half_sq(m, ny) / dy; eyi[m] = -sy[m] / dy; }

    // per-stage twiddle tables of the x and y plans: stage s owns entries
    // [s*n, s*n + R*Ns), entry r*Ns + k = exp(-2 pi i r k / (Ns R))
    auto stage_tables = [](const FftFactors& f, std::vector<double>& re, std::vector<double>& im) {
        const int n = f.n;
        re.assign((size_t)std::max(1, f.nstages) * n, 0.0);
        im.assign(re.size(), 0.0);
        for (int s = 0; s < f.nstages; ++s) {
            const int R = f.st[s].radix, ns = f.st[s].ns;
            for (int r = 0; r < R; ++r)
                for (int k = 0; k < ns; ++k)
                    twiddle(r * k, ns * R, &re[(size_t)s * n + r * ns + k], &im[(size_t)s * n + r * ns + k]);
        }
    };
    std::vector<double> tsxr, tsxi, tsyr, tsyi;
    stage_tables(p->fx, tsxr, tsxi);
    stage_tables(p->fy, tsyr, tsyi);
    to.twx = blob.size();
    if (fp64) push_complex<double>(blob, tsxr, tsxi); else push_complex<float>(blob, tsxr, tsxi);
    pad_blob(blob);
    to.twy = blob.size();
    if (fp64) push_complex<double>(blob, tsyr, tsyi); else push_complex<float>(blob, tsyr, tsyi);
    pad_blob(blob);
    // the E = 16 schedule of the y plan (FP32 square-grid column kernels)
    to.twy16 = 0;
    if (!fp64 && cty && (ny == 256 || ny == 512 || ny == 1024)) {
        std::vector<double> t16r, t16i;
        stage_tables(factorize(ny, 16, true), t16r, t16i);
        to.twy16 = blob.size();
        push_complex<float>(blob, t16r, t16i);
        pad_blob(blob);
    }
    to.sv = blob.size(); push_doubles(blob, svol); pad_blob(blob);
    to.rl = blob.size(); push_doubles(blob, rflo); pad_blob(blob);
    to.rh = blob.size(); push_doubles(blob, rfhi); pad_blob(blob);
    to.a = blob.size(); push_doubles(blob, acoef); pad_blob(blob);
    to.iz = blob.size(); push_doubles(blob, idzn); pad_blob(blob);
    to.cs = blob.size(); push_doubles(blob, csum); pad_blob(blob);
    to.sv32 = blob.size(); push_floats(blob, svol); pad_blob(blob);
    to.rl32 = blob.size(); push_floats(blob, rflo); pad_blob(blob);
    to.rh32 = blob.size(); push_floats(blob, rfhi); pad_blob(blob);
    to.a32 = blob.size(); push_floats(blob, acoef); pad_blob(blob);
    to.cs32 = blob.size(); push_floats(blob, csum); pad_blob(blob);
    to.iz32 = blob.size(); push_floats(blob, idzn); pad_blob(blob);
    to.lx = blob.size(); push_doubles(blob, lamx); pad_blob(blob);
    to.ly = blob.size(); push_doubles(blob, lamy); pad_blob(blob);
    to.ex = blob.size();
    if (fp64) push_complex<double>(blob, exr, exi); else push_complex<float>(blob, exr, exi);
    pad_blob(blob);
    to.ey = blob.size();
    if (fp64) push_complex<double>(blob, eyr, eyi); else push_complex<float>(blob, eyr, eyi);
    pad_blob(blob);
    to.err = blob.size();
    blob.resize(blob.size() + 256, 0);
    // FP64 warps of a mixed plan (the near-zero wavenumbers and the warp of
    // the pinned mean, the same rule as the vertical solve's): their 1/e
    // depend on the column's lambda and the vertical coefficients only, so a
    // table of them is built once per plan and the solve's FP64 chain per level
    // shrinks to the y update
    p->nslots = 0;
    p->nwr = ((p->nxh + 31) & ~31) / 32;
    p->gtab_bytes = 0;
    to.wlist = to.wslot = to.gtab = 0;
    if (precision == MONC_PROJ_MIXED && !z64) {
        std::vector<int> wl, ws((size_t)ny * p->nwr, -1);
        for (int ky = 0; ky < ny; ++ky)
            for (int w = 0; w < p->nwr; ++w) {
                const int kx0 = 32 * w;
                if (-(lamx[kx0] + lamy[ky]) < p->lam_fp64 || (ky == 0 && w == 0)) {
                    ws[(size_t)ky * p->nwr + w] = p->nslots;
                    wl.push_back(ky);
                    wl.push_back(kx0);
                    p->nslots += 32;
                }
            }
        auto push_ints = [&](const std::vector<int>& v) {
            const size_t o = blob.size();
            blob.resize(o + v.size() * sizeof(int));
            std::memcpy(blob.data() + o, v.data(), v.size() * sizeof(int));
            pad_blob(blob);
            return o;
        };
        to.wlist = push_ints(wl);
        to.wslot = push_ints(ws);
        p->gtab_bytes = (size_t)p->nslots * nz * (sizeof(float2) + sizeof(float4));
        to.gtab = align256(blob.size());
    }

    p->ct_rows = ctx;
    p->ct_cols = cty;
    p->row_threads = kRowTaskThreads;
    p->col_e = kMaxRadixF32;
    p->col_threads = kColTaskThreads;
    set_task_shapes(p);
    const int npair = p->rows_fwd / 2;
    const int tw = p->tw_cols;
    // the persistent inverse column kernel (opt-in) holds two input stages
    // of ny x tw values plus the FFT buffer
    p->persist_cols = cty && ct_core_length(ny, fp64) && precision != MONC_PROJ_REFINED && persist_cols_enabled();
    // TMA column kernels (opt-in): FP32 compile-time lengths (rows of tw >= 2
    // complex values, a multiple of 16 bytes)
    p->smem_tma = (size_t)2 * tw * p->bs_col * csz + 128 + 32;    // + alignment slack, mbarriers
    p->tma_cols = !fp64 && cty && ct_core_length(ny, fp64) && precision != MONC_PROJ_REFINED && !p->persist_cols && (tw * csz) % 16 == 0 && p->smem_tma <= kSmemMax &&
                  tma_enabled() && tmap_encoder() != nullptr;
    if (p->persist_cols) p->smem_cols = ((size_t)2 * ny * tw + (size_t)tw * p->bs_col) * csz;
    // fused persistent kernels for square compile-time grids: one block size
    // and shared-memory size for both task kinds of each kernel
    p->fused = ctx && cty && nx == ny && ct_core_length(nx, fp64) && precision != MONC_PROJ_REFINED &&
               !fused_disabled();
    p->ring = std::min(nz, fp64 ? 4 : 8);
    p->thr_fwd_fused = std::max(p->thr_fwd_rows, p->thr_cols);
    p->smem_fwd_fused = std::max((size_t)npair * p->bs_row * csz, (size_t)tw * p->bs_col * csz);
    for (int idx = 0; idx < 2; ++idx) {
        p->thr_inv_fused[idx] = std::max(p->thr_inv_rows[idx], p->thr_cols);
        p->smem_inv_fused[idx] = std::max({p->smem_inv_rows[idx], (size_t)tw * p->bs_col * csz,
                                           (size_t)ny * tw * csz});
    }
    // consumers trail producers by `lag` levels; a ring of lag + 3 levels
    // lets producers run ahead without waiting for slots
    p->lag = std::min(nz, env_int("MONC_PROJ_FUSED_LAG", 3));
    if (p->fused) p->ring = std::min(nz, std::max(p->lag + 1, env_int("MONC_PROJ_FUSED_RING", p->lag + 3)));

    // the pipelines' consumers discard whole 128-byte lines of the
    // intermediate spectra, so rows are padded to whole lines
    p->pipe = precision == MONC_PROJ_MIXED && ctx && cty && !p->persist_cols && !p->tma_cols && !p->fused &&
              pick_fwd_pipe(nx, ny) && pick_inv_pipe(nx, ny) && pipe_enabled();
    p->pipe_lag_fwd = (int)std::min<long long>(nz, env_ll0("MONC_PROJ_PIPE_LAG_FWD", kPipeLagFwd));
    p->pipe_lag_inv = (int)std::min<long long>(nz, env_ll0("MONC_PROJ_PIPE_LAG_INV", kPipeLagInv));
    p->spin_limit = env_ll0("MONC_PROJ_SPIN_LIMIT", kSpinLimit);
    {
        const char* e = std::getenv("MONC_PROJ_PIPE_EF");
        p->pipe_ef = e && e[0] == '1';
    }
    if (p->pipe) p->nxp = (p->nxh + 15) & ~15;
    // tensor-core split-precision forward columns: MONC_PROJ_TC=1 (TF32 x 3) or
    // 2 (BF16 x 6), mixed plans with ny = 1024 (read when the plan is made)
    {
        const char* e = std::getenv("MONC_PROJ_TC");
        const int fmt = (e && (e[0] == '1' || e[0] == '2')) ? e[0] - '0' : 0;
        p->tc_cols = (fmt && precision == MONC_PROJ_MIXED && cty && pick_fwd_cols_tc(ny, fmt) && !p->pipe &&
                      !p->fused && !p->tma_cols) ? fmt : 0;
    }
    p->smem_pipe = std::max((size_t)8 * std::max(1, 1024 / nx) * p->bs_row * csz, (size_t)p->tw_cols * p->bs_col * csz);

    // ---- workspace layout
    const size_t L = (size_t)nz * ny * p->nxp;
    size_t off = 0;
    p->off_S = off; off = align256(off + L * csz);
    p->off_G = off; off = align256(off + L * csz);
    p->off_T = off; off = align256(off + L * csz);
    p->off_Tp = off; off = align256(off + L * csz);
    p->off_Tgy = off; off = align256(off + L * csz);
    p->off_Tgz = off; off = align256(off + L * csz);
    p->off_Tphi = off; off = align256(off + L * csz);
    p->off_Y = off;                                   // (unused)
    p->off_Gp = off; if (!fp64) off = align256(off + L * 8);   // 1/e of FP64 columns (mixed)
    p->off_sync = off;                                // tickets and per-level counters of the fused kernels
    p->sync_bytes = (size_t)(2 + 10 * nz) * sizeof(unsigned);
    off = align256(off + p->sync_bytes);
    p->off_groups = off;                              // pipelines: per (level, line group) counters
    p->groups_bytes = p->pipe ? (size_t)nz * (p->nxp / 16 + 1) * sizeof(unsigned) : 0;
    off = align256(off + p->groups_bytes);
    p->refine_passes = std::min(4, env_int("MONC_PROJ_REFINE_PASSES", kRefinePasses));
    p->off_phipass = off;                             // refinement passes: one pass's potential (FP64)
    if (precision == MONC_PROJ_REFINED) off = align256(off + (size_t)nx * ny * nz * sizeof(double));
    p->off_phimean = off;                             // refinement passes: level-0 mean of the potential
    if (precision == MONC_PROJ_REFINED) off = align256(off + sizeof(double));
    p->ws_bytes = off;
}

// Point the plan's table pointers into device memory `db` holding the blob.
void plan_bind(monc_proj_plan_s* p, unsigned char* db, const TableOffsets& to) {
    p->twx = db + to.twx; p->twy = db + to.twy;
    p->twy16 = to.twy16 ? db + to.twy16 : nullptr;
    p->svol = (const double*)(db + to.sv); p->rflo = (const double*)(db + to.rl);
    p->rfhi = (const double*)(db + to.rh); p->acoef = (const double*)(db + to.a);
    p->idzn = (const double*)(db + to.iz); p->lamx = (const double*)(db + to.lx);
    p->csum = (const double*)(db + to.cs);
    p->svol32 = (const float*)(db + to.sv32); p->acoef32 = (const float*)(db + to.a32);
    p->csum32 = (const float*)(db + to.cs32); p->idzn32 = (const float*)(db + to.iz32);
    p->rflo32 = (const float*)(db + to.rl32); p->rfhi32 = (const float*)(db + to.rh32);
    p->lamy = (const double*)(db + to.ly); p->ex = db + to.ex; p->ey = db + to.ey;
    p->err = (int*)(db + to.err);
    p->wlist = p->nslots ? (const int*)(db + to.wlist) : nullptr;
    p->wslot = p->nslots ? (const int*)(db + to.wslot) : nullptr;
    p->pvm = p->nslots ? (float2*)(db + to.gtab) : nullptr;
    p->pvgb = p->nslots ? (float4*)(db + to.gtab + (size_t)p->nslots * p->nz * sizeof(float2)) : nullptr;
}

// Device bytes of a plan's tables: the uploaded blob, then the 1/e table.
size_t plan_table_bytes(const monc_proj_plan_s* p, size_t blob_bytes, const TableOffsets& to) {
    return p->nslots ? to.gtab + p->gtab_bytes : blob_bytes;
}

// Fill the tables computed on the device (after the upload, on `st`).
int plan_fill_tables(monc_proj_plan_s* p, cudaStream_t st) {
    if (!p->nslots) return MONC_PROJ_OK;
    k_fp64_pivots<<<(p->nslots + 127) / 128, 128, 0, st>>>(p->wlist, p->lamx, p->lamy, p->acoef, p->svol,
                                                            p->csum, p->nxh, p->nz, p->nslots, p->pvm, p->pvgb);
    return cudaGetLastError() == cudaSuccess ? MONC_PROJ_OK : MONC_PROJ_ECUDA;
}

// Streams on which a batch's instances run concurrently (per device), with
// the fork/join events that order them after and before the caller's stream.
constexpr int kBatchStreams = 16;
struct StreamPool {
    std::mutex mu;
    bool ready = false;
    cudaStream_t s[kBatchStreams];
    cudaEvent_t fork;
    cudaEvent_t join[kBatchStreams];
};
constexpr int kPoolMaxDevices = 64;
std::mutex g_pool_mu;
StreamPool g_pools[kPoolMaxDevices];

int stream_pool(StreamPool** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return MONC_PROJ_ECUDA; }
    if (dev < 0 || dev >= kPoolMaxDevices) return MONC_PROJ_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    StreamPool& p = g_pools[dev];
    if (!p.ready) {
        bool ok = cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming) == cudaSuccess;
        for (int j = 0; ok && j < kBatchStreams; ++j)
            ok = cudaStreamCreateWithFlags(&p.s[j], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&p.join[j], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) { cudaGetLastError(); return MONC_PROJ_ECUDA; }
        p.ready = true;
    }
    *out = &p;
    return MONC_PROJ_OK;
}

}  // namespace

extern "C" {

const char* monc_proj_status_string(int status) {
    switch (status) {
        case MONC_PROJ_OK: return "ok";
        case MONC_PROJ_EINVAL: return "invalid argument";
        case MONC_PROJ_EUNSUPPORTED: return "unsupported size (nx, ny must be 2^a 3^b 5^c, <= 4096)";
        case MONC_PROJ_ENOMEM: return "device allocation failed";
        case MONC_PROJ_ECUDA: return "CUDA runtime error";
        case MONC_PROJ_ETIMEOUT: return "bounded device wait timed out";
        case MONC_PROJ_EDEVICE: return "device-detected error";
        case MONC_PROJ_ESCRATCH: return "problem too large for the no-alloc static scratch";
        case MONC_PROJ_ENOCONV: return "Krylov solve reached its iteration limit";
        case MONC_PROJ_EBREAKDOWN: return "Krylov solve broke down (zero denominator)";
        default: return "unknown status";
    }
}

int monc_proj_plan(monc_proj_plan_t* out, int nx, int ny, int nz, double dx, double dy,
                   const double* dz, const double* rho_c, const double* rho_f,
                   int precision, void* stream) {
    if (!out) return MONC_PROJ_EINVAL;
    *out = nullptr;
    const int vr = validate_grid(nx, ny, nz, dx, dy, dz, rho_c, rho_f, precision);
    if (vr != MONC_PROJ_OK) return vr;

    monc_proj_plan_s* p = new (std::nothrow) monc_proj_plan_s();
    if (!p) return MONC_PROJ_ENOMEM;
    std::vector<unsigned char> blob;
    TableOffsets to{};
    plan_prepare(p, nx, ny, nz, dx, dy, dz, rho_c, rho_f, precision, blob, to);
    cudaGetDevice(&p->device);

    // the tables' device memory, from the caller's allocator if one is set
    void* d = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_alloc_mu);
        const size_t tb = plan_table_bytes(p, blob.size(), to);
        if (g_alloc) {
            d = g_alloc(tb, g_alloc_user);
            p->tables_free = g_free;
            p->tables_user = g_alloc_user;
        } else if (cudaMalloc(&d, tb) != cudaSuccess) {
            cudaGetLastError();
            d = nullptr;
        }
    }
    if (!d) { delete p; return MONC_PROJ_ENOMEM; }
    p->dev_tables = d;
    auto fail = [&](int rc) {
        if (p->tables_free) p->tables_free(d, p->tables_user);
        else cudaFree(d);
        delete p;
        return rc;
    };
    if ((uintptr_t)d & 255) return fail(MONC_PROJ_EINVAL);
    const int ar = plan_kernel_attrs(p);
    if (ar != MONC_PROJ_OK) return fail(ar);
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(d, blob.data(), blob.size(), cudaMemcpyHostToDevice, st) != cudaSuccess) {
        cudaGetLastError();
        return fail(MONC_PROJ_ECUDA);
    }
    plan_bind(p, (unsigned char*)d, to);
    if (plan_fill_tables(p, st) != MONC_PROJ_OK || cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return fail(MONC_PROJ_ECUDA);
    }
    *out = p;
    return MONC_PROJ_OK;
}

int monc_proj_set_allocator(monc_proj_alloc_fn alloc, monc_proj_free_fn release, void* user) {
    if ((alloc == nullptr) != (release == nullptr)) return MONC_PROJ_EINVAL;
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    g_alloc = alloc;
    g_free = release;
    g_alloc_user = alloc ? user : nullptr;
    return MONC_PROJ_OK;
}

int monc_proj_workspace_size(monc_proj_plan_t plan, size_t* bytes) {
    if (!plan || !bytes) return MONC_PROJ_EINVAL;
    *bytes = plan->ws_bytes;
    return MONC_PROJ_OK;
}

int monc_proj_solve(monc_proj_plan_t plan, const void* u, const void* v, const void* w,
                    void* u_out, void* v_out, void* w_out, void* phi_out,
                    void* workspace, void* stream) {
    if (!plan || !u || !v || !w || !u_out || !v_out || !w_out || !workspace) return MONC_PROJ_EINVAL;
    const void* ptrs[] = {u, v, w, u_out, v_out, w_out, phi_out};
    for (const void* x : ptrs)
        if (((uintptr_t)x) & 15) return MONC_PROJ_EINVAL;
    if (((uintptr_t)workspace) & 255) return MONC_PROJ_EINVAL;
    ProjParams q = make_params(plan, u, v, w, u_out, v_out, w_out, phi_out, workspace);
    cudaStream_t st = (cudaStream_t)stream;
    return run_solve(plan, q, st);
}

// ---------------------------------------------------------------------------
// Phases of a distributed solve (the pencil decomposition): the forward
// transform of a slab of levels, the vertical solve of a pencil of spectral
// rows, the inverse transform of a slab.  They run the kernels of the whole
// solve on sub-domains (ProjParams.kbase / nz_glob / ky_base).
// ---------------------------------------------------------------------------
}  // extern "C"

namespace mp {
// Reordering of spectral rows between a z-slab and the blocks sent to the
// pencils of a distributed solve.  slab: [nzl][ny][row]; packed: the blocks
// of parts s = 0 .. parts-1 one after the other, block s [nzl][rows of s][row],
// where part s holds the rows [s*q + min(s, r), ...) of ny = q*parts + r (the
// first r parts one row more).  A row is `units` 16-byte words.  One block
// per slab row; dir 0 copies slab -> packed, dir 1 packed -> slab.
__global__ void __launch_bounds__(128) k_pencil_pack(const float4* __restrict__ src, float4* __restrict__ dst,
                                                     int ny, int nzl, int parts, int units, int dir) {
    const int row = blockIdx.x;                 // k * ny + j
    const int k = row / ny, j = row - k * ny;
    const int q = ny / parts, r = ny - q * parts;
    int j0, nys;
    if (j < r * (q + 1)) {
        j0 = (j / (q + 1)) * (q + 1);
        nys = q + 1;
    } else {
        j0 = r * (q + 1) + ((j - r * (q + 1)) / q) * q;
        nys = q;
    }
    const size_t poff = ((size_t)nzl * j0 + (size_t)k * nys + (j - j0)) * units;
    const size_t soff = (size_t)row * units;
    const float4* a = src + (dir ? poff : soff);
    float4* b = dst + (dir ? soff : poff);
    for (int i = threadIdx.x; i < units; i += blockDim.x) b[i] = a[i];
}
}  // namespace mp

namespace {
size_t spec_elem(const monc_proj_plan_s* p) { return p->precision == MONC_PROJ_FP64 ? 16 : 8; }

template <typename R>
int launch_forward_slab(monc_proj_plan_s* p, const ProjParams& q, cudaStream_t st) {
    const SolveKernels ks = pick_kernels<R>(p);
    const int nzl = q.nz;
    ks.fwd_rows<<<nzl * p->nrb_fwd, p->thr_fwd_rows, p->smem_fwd_rows, st>>>(q);
    ks.fwd_cols<<<nzl * p->ntiles, p->thr_cols, p->smem_fcols, st>>>(q);
    return cudaGetLastError() == cudaSuccess ? MONC_PROJ_OK : MONC_PROJ_ECUDA;
}

template <typename R>
int launch_inverse_slab(monc_proj_plan_s* p, const ProjParams& q, cudaStream_t st) {
    const SolveKernels ks = pick_kernels<R>(p);
    const int nzl = q.nz;
    const int n_icols = nzl * p->ntiles * (p->ct_cols ? 2 : q.nch);
    const int n_irows = nzl * q.nrb_inv * (p->ct_rows ? q.nch : 1);
    ks.inv_cols<<<n_icols, p->thr_cols, p->smem_cols, st>>>(q);
    ks.inv_rows<<<n_irows, p->thr_inv_rows[0], p->smem_inv_rows[0], st>>>(q);
    return cudaGetLastError() == cudaSuccess ? MONC_PROJ_OK : MONC_PROJ_ECUDA;
}

// The kernels of the opt-in variants (fused, persistent, pipelined) and the
// refinement passes are not sub-domain aware; slab phases run the default
// kernels of FP64 and mixed plans.
bool slab_plan_ok(const monc_proj_plan_s* p) {
    return (p->precision == MONC_PROJ_FP64 || p->precision == MONC_PROJ_MIXED) && !p->fused && !p->persist_cols &&
           !p->pipe;
}
}  // namespace

extern "C" {

int monc_proj_spectral_pitch(monc_proj_plan_t plan, int* nxp) {
    if (!plan || !nxp) return MONC_PROJ_EINVAL;
    *nxp = plan->nxp;
    return MONC_PROJ_OK;
}

int monc_proj_forward_slab(monc_proj_plan_t plan, int k0, int k1, const void* u, const void* v, const void* w,
                           void* dhat, void* workspace, void* stream) {
    if (!plan || !u || !v || !w || !dhat || !workspace) return MONC_PROJ_EINVAL;
    if (k0 < 0 || k1 <= k0 || k1 > plan->nz) return MONC_PROJ_EINVAL;
    if (!slab_plan_ok(plan)) return MONC_PROJ_EUNSUPPORTED;
    const void* ptrs[] = {u, v, w, dhat};
    for (const void* x : ptrs)
        if (((uintptr_t)x) & 15) return MONC_PROJ_EINVAL;
    if (((uintptr_t)workspace) & 255) return MONC_PROJ_EINVAL;
    ProjParams q = make_params(plan, u, v, w, nullptr, nullptr, nullptr, nullptr, workspace);
    q.nz = k1 - k0;
    q.kbase = k0;
    q.S = dhat;
    cudaStream_t st = (cudaStream_t)stream;
    return plan->precision == MONC_PROJ_FP64 ? launch_forward_slab<double>(plan, q, st)
                                             : launch_forward_slab<float>(plan, q, st);
}

int monc_proj_vertical_pencil(monc_proj_plan_t plan, int j0, int j1, void* spec, void* gz, void* workspace,
                              void* stream) {
    if (!plan || !spec || !gz || !workspace) return MONC_PROJ_EINVAL;
    if (j0 < 0 || j1 <= j0 || j1 > plan->ny) return MONC_PROJ_EINVAL;
    if (!slab_plan_ok(plan)) return MONC_PROJ_EUNSUPPORTED;
    if ((((uintptr_t)spec) & 15) || (((uintptr_t)gz) & 15) || (((uintptr_t)workspace) & 255)) return MONC_PROJ_EINVAL;
    ProjParams q = make_params(plan, spec, spec, spec, nullptr, nullptr, nullptr, nullptr, workspace);
    q.ny = j1 - j0;
    q.ky_base = j0;
    q.S = spec;
    q.G = gz;
    const long long ncol = (long long)q.ny * ((plan->nxh + 31) & ~31);
    cudaStream_t st = (cudaStream_t)stream;
    const KernelFn tri = plan->precision == MONC_PROJ_FP64 ? pick_tridiag<double>() : pick_tridiag<float>();
    tri<<<(unsigned)((ncol + kTriThreads - 1) / kTriThreads), kTriThreads, 0, st>>>(q);
    return cudaGetLastError() == cudaSuccess ? MONC_PROJ_OK : MONC_PROJ_ECUDA;
}

int monc_proj_inverse_slab(monc_proj_plan_t plan, int k0, int k1, const void* phat, const void* gz, const void* u,
                           const void* v, const void* w, void* u_out, void* v_out, void* w_out, void* workspace,
                           void* stream) {
    if (!plan || !phat || !gz || !u || !v || !w || !u_out || !v_out || !w_out || !workspace) return MONC_PROJ_EINVAL;
    if (k0 < 0 || k1 <= k0 || k1 > plan->nz) return MONC_PROJ_EINVAL;
    if (!slab_plan_ok(plan)) return MONC_PROJ_EUNSUPPORTED;
    const void* ptrs[] = {phat, gz, u, v, w, u_out, v_out, w_out};
    for (const void* x : ptrs)
        if (((uintptr_t)x) & 15) return MONC_PROJ_EINVAL;
    if (((uintptr_t)workspace) & 255) return MONC_PROJ_EINVAL;
    ProjParams q = make_params(plan, u, v, w, u_out, v_out, w_out, nullptr, workspace);
    q.nz = k1 - k0;
    q.kbase = k0;
    q.S = const_cast<void*>(phat);
    q.G = const_cast<void*>(gz);
    cudaStream_t st = (cudaStream_t)stream;
    return plan->precision == MONC_PROJ_FP64 ? launch_inverse_slab<double>(plan, q, st)
                                             : launch_inverse_slab<float>(plan, q, st);
}

static int pencil_reorder(monc_proj_plan_t plan, int nzl, int parts, const void* src, void* dst, int dir,
                          void* stream) {
    if (!plan || !src || !dst || nzl < 1 || nzl > plan->nz || parts < 1) return MONC_PROJ_EINVAL;
    if ((((uintptr_t)src) & 15) || (((uintptr_t)dst) & 15)) return MONC_PROJ_EINVAL;
    if (!slab_plan_ok(plan)) return MONC_PROJ_EUNSUPPORTED;
    const int units = (int)((size_t)plan->nxp * spec_elem(plan) / 16);
    k_pencil_pack<<<(unsigned)(nzl * plan->ny), 128, 0, (cudaStream_t)stream>>>((const float4*)src, (float4*)dst,
                                                                               plan->ny, nzl, parts, units, dir);
    return cudaGetLastError() == cudaSuccess ? MONC_PROJ_OK : MONC_PROJ_ECUDA;
}

int monc_proj_pack_pencils(monc_proj_plan_t plan, int nzl, int parts, const void* slab, void* packed, void* stream) {
    return pencil_reorder(plan, nzl, parts, slab, packed, 0, stream);
}

int monc_proj_unpack_pencils(monc_proj_plan_t plan, int nzl, int parts, const void* packed, void* slab,
                             void* stream) {
    return pencil_reorder(plan, nzl, parts, packed, slab, 1, stream);
}

int monc_proj_krylov_workspace_size(monc_proj_plan_t plan, size_t* bytes) {
    if (!plan || !bytes) return MONC_PROJ_EINVAL;
    *bytes = krylov_workspace_bytes(plan->nx, plan->ny, plan->nz, plan->nsm, plan->precision == MONC_PROJ_MIXED);
    return MONC_PROJ_OK;
}

int monc_proj_solve_krylov(monc_proj_plan_t plan, const void* u, const void* v, const void* w,
                           void* u_out, void* v_out, void* w_out, void* phi_out, void* workspace,
                           double tol, int max_iter, int precond, int* iterations, double* rel_residual,
                           void* stream) {
    if (!plan || !u || !v || !w || !u_out || !v_out || !w_out || !workspace) return MONC_PROJ_EINVAL;
    if (!(tol >= 0.0) || !std::isfinite(tol) || max_iter < 0) return MONC_PROJ_EINVAL;
    if (precond != MONC_PROJ_PC_NONE && precond != MONC_PROJ_PC_LINE) return MONC_PROJ_EINVAL;
    const bool fp32 = plan->precision == MONC_PROJ_MIXED;
    const void* ptrs[] = {u, v, w, u_out, v_out, w_out, phi_out};
    for (const void* x : ptrs)
        if (((uintptr_t)x) & (fp32 ? 3 : 7)) return MONC_PROJ_EINVAL;
    if (((uintptr_t)workspace) & 255) return MONC_PROJ_EINVAL;
    KrylovProblem kp{};
    kp.fp32 = fp32;
    kp.nx = plan->nx; kp.ny = plan->ny; kp.nz = plan->nz; kp.nsm = plan->nsm;
    kp.dx = plan->dx; kp.dy = plan->dy;
    kp.acoef = plan->acoef; kp.svol = plan->svol; kp.rflo = plan->rflo; kp.rfhi = plan->rfhi;
    kp.idzn = plan->idzn;
    kp.u = u; kp.v = v; kp.w = w;
    kp.u_out = u_out; kp.v_out = v_out; kp.w_out = w_out; kp.phi_out = phi_out;
    kp.workspace = workspace;
    kp.tol = tol; kp.max_iter = max_iter; kp.precond = precond;
    KrylovResult res{};
    if (krylov_run(kp, (cudaStream_t)stream, &res) != cudaSuccess) {
        cudaGetLastError();
        return MONC_PROJ_ECUDA;
    }
    if (iterations) *iterations = res.iterations;
    if (rel_residual) *rel_residual = res.rel_residual;
    return res.status == 0 ? MONC_PROJ_OK : res.status == 1 ? MONC_PROJ_ENOCONV : MONC_PROJ_EBREAKDOWN;
}

namespace {
// element size of a plan's fields and the byte sizes of its arrays
void field_layout(const monc_proj_plan_s* p, size_t* elem, size_t* cbytes, size_t* fbytes) {
    *elem = p->precision == MONC_PROJ_MIXED ? sizeof(float) : sizeof(double);
    *cbytes = (size_t)p->nz * p->ny * p->nx * *elem;          // u, v, phi
    *fbytes = (size_t)(p->nz + 1) * p->ny * p->nx * *elem;    // w
}
}  // namespace

int monc_proj_host_staging_size(monc_proj_plan_t plan, int with_phi, size_t* bytes) {
    if (!plan || !bytes) return MONC_PROJ_EINVAL;
    size_t e, c, f;
    field_layout(plan, &e, &c, &f);
    *bytes = align256(c) * 2 + align256(f) + (with_phi ? align256(c) : 0);
    return MONC_PROJ_OK;
}

int monc_proj_solve_host(monc_proj_plan_t plan, const void* u, const void* v, const void* w,
                         void* u_out, void* v_out, void* w_out, void* phi_out,
                         void* staging, size_t staging_bytes, void* workspace, void* stream) {
    if (!plan || !u || !v || !w || !u_out || !v_out || !w_out || !staging || !workspace) return MONC_PROJ_EINVAL;
    size_t need = 0;
    monc_proj_host_staging_size(plan, phi_out != nullptr, &need);
    if (staging_bytes < need || (((uintptr_t)staging) & 255)) return MONC_PROJ_EINVAL;
    size_t e, c, f;
    field_layout(plan, &e, &c, &f);
    unsigned char* d = (unsigned char*)staging;
    unsigned char* du = d;
    unsigned char* dv = du + align256(c);
    unsigned char* dw = dv + align256(c);
    unsigned char* dp = phi_out ? dw + align256(f) : nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(du, u, c, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(dv, v, c, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(dw, w, f, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        cudaGetLastError();
        return MONC_PROJ_ECUDA;
    }
    const int rc = monc_proj_solve(plan, du, dv, dw, du, dv, dw, dp, workspace, stream);
    if (rc != MONC_PROJ_OK) return rc;
    if (cudaMemcpyAsync(u_out, du, c, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(v_out, dv, c, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(w_out, dw, f, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        (phi_out && cudaMemcpyAsync(phi_out, dp, c, cudaMemcpyDeviceToHost, st) != cudaSuccess)) {
        cudaGetLastError();
        return MONC_PROJ_ECUDA;
    }
    return MONC_PROJ_OK;
}

int monc_proj_batch_workspace_size(const monc_proj_plan_t* plans, int count, size_t* bytes) {
    if (!plans || !bytes || count < 0) return MONC_PROJ_EINVAL;
    size_t total = 0;
    for (int i = 0; i < count; ++i) {
        if (!plans[i]) return MONC_PROJ_EINVAL;
        total += align256(plans[i]->ws_bytes);
    }
    *bytes = total;
    return MONC_PROJ_OK;
}

int monc_proj_solve_batch(const monc_proj_plan_t* plans, const monc_proj_fields* fields,
                          int count, void* workspace, size_t workspace_bytes, void* stream) {
    if (!plans || !fields || count < 0 || (count > 0 && !workspace)) return MONC_PROJ_EINVAL;
    size_t need = 0;
    int rc = monc_proj_batch_workspace_size(plans, count, &need);
    if (rc) return rc;
    if (workspace_bytes < need) return MONC_PROJ_EINVAL;
    if (count == 0) return MONC_PROJ_OK;
    for (int i = 0; i < count; ++i) {
        const monc_proj_fields& f = fields[i];
        if (!f.u || !f.v || !f.w || !f.u_out || !f.v_out || !f.w_out) return MONC_PROJ_EINVAL;
    }
    StreamPool* pool = nullptr;
    rc = stream_pool(&pool);
    if (rc) return rc;
    // workspace offsets in argument order; launch order largest first so the
    // round-robin over the pool's streams balances the work
    std::vector<size_t> off(count);
    std::vector<int> order(count);
    size_t o = 0;
    for (int i = 0; i < count; ++i) {
        off[i] = o;
        o += align256(plans[i]->ws_bytes);
        order[i] = i;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const double na = (double)plans[a]->nx * plans[a]->ny * plans[a]->nz;
        const double nb = (double)plans[b]->nx * plans[b]->ny * plans[b]->nz;
        return na > nb;
    });
    std::lock_guard<std::mutex> lock(pool->mu);
    cudaStream_t st = (cudaStream_t)stream;
    const int nstreams = std::min(count, kBatchStreams);
    if (cudaEventRecord(pool->fork, st) != cudaSuccess) { cudaGetLastError(); return MONC_PROJ_ECUDA; }
    for (int j = 0; j < nstreams; ++j)
        if (cudaStreamWaitEvent(pool->s[j], pool->fork, 0) != cudaSuccess) { cudaGetLastError(); return MONC_PROJ_ECUDA; }
    unsigned char* ws = (unsigned char*)workspace;
    int first_error = MONC_PROJ_OK;
    for (int n = 0; n < count; ++n) {
        const int i = order[n];
        const monc_proj_fields& f = fields[i];
        const int r = monc_proj_solve(plans[i], f.u, f.v, f.w, f.u_out, f.v_out, f.w_out, f.phi_out, ws + off[i],
                                      pool->s[n % nstreams]);
        if (r && !first_error) first_error = r;
    }
    // join: the caller's stream waits for every pool stream used
    for (int j = 0; j < nstreams; ++j) {
        if (cudaEventRecord(pool->join[j], pool->s[j]) != cudaSuccess ||
            cudaStreamWaitEvent(st, pool->join[j], 0) != cudaSuccess) {
            cudaGetLastError();
            return MONC_PROJ_ECUDA;
        }
    }
    return first_error;
}

// ---------------------------------------------------------------------------
// Grouped batch: one launch per phase and group of instances (group.cuh).
// ---------------------------------------------------------------------------
}  // extern "C"

namespace {
// Plans whose solve is the default FP32 split kernels of compile-time lengths
bool group_eligible(const monc_proj_plan_s* p) {
    return p->precision == MONC_PROJ_MIXED && p->ct_rows && p->ct_cols && p->col_e == kMaxRadixF32 && !p->fused && !p->pipe &&
           !p->persist_cols && !p->tma_cols && !p->tc_cols && pick_group_f32(0, p->nx) && pick_group_f32(1, p->ny);
}

// The five phase launches of one chunk of a group (instances idx, all with
// the task shapes of plans[idx[0]]) on stream st.
int launch_group_chunk(const monc_proj_plan_t* plans, const monc_proj_fields* fields, const std::vector<int>& idx,
                       const std::vector<size_t>& off, unsigned char* ws, cudaStream_t st) {
    const monc_proj_plan_s* p0 = plans[idx[0]];
    const int m = (int)idx.size();
    std::unique_ptr<GroupArgs> a(new (std::nothrow) GroupArgs());
    if (!a) return MONC_PROJ_ENOMEM;
    a->n = m;
    for (int j = 0; j < m; ++j) {
        const int i = idx[j];
        const monc_proj_fields& f = fields[i];
        a->p[j] = make_params(plans[i], f.u, f.v, f.w, f.u_out, f.v_out, f.w_out, f.phi_out, ws + off[i]);
    }
    const int inv_idx = a->p[0].nch == 4 ? 1 : 0;
    const long long ncol = (long long)p0->ny * ((p0->nxh + 31) & ~31);
    for (int phase = 0; phase < 5; ++phase) {
        int thr = 0;
        size_t smem = 0;
        a->start[0] = 0;
        for (int j = 0; j < m; ++j) {
            const ProjParams& q = a->p[j];
            long long nb = 0;
            switch (phase) {
                case 0: nb = (long long)q.nz * p0->nrb_fwd; break;
                case 1: nb = (long long)q.nz * p0->ntiles; break;
                case 2: nb = (ncol + kTriThreads - 1) / kTriThreads; break;
                case 3: nb = (long long)q.nz * p0->ntiles * 2; break;
                default: nb = (long long)q.nz * q.nrb_inv * q.nch; break;
            }
            if (a->start[j] + nb > 0x7fffffffLL) return MONC_PROJ_EUNSUPPORTED;
            a->start[j + 1] = a->start[j] + (int)nb;
        }
        switch (phase) {
            case 0: thr = p0->thr_fwd_rows; smem = p0->smem_fwd_rows; break;
            case 1: thr = p0->thr_cols; smem = p0->smem_fcols; break;
            case 2: thr = kTriThreads; smem = 0; break;
            case 3: thr = p0->thr_cols; smem = p0->smem_cols; break;
            default: thr = p0->thr_inv_rows[inv_idx]; smem = p0->smem_inv_rows[inv_idx]; break;
        }
        const GroupFn fn = pick_group_f32(phase, (phase == 0 || phase == 4) ? p0->nx : p0->ny, p0->nx == p0->ny,
                                          p0->nxp, p0->tw_cols);
        if (!fn) return MONC_PROJ_EUNSUPPORTED;
        if (smem > 48 * 1024 &&
            cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                cudaSuccess) {
            cudaGetLastError();
            return MONC_PROJ_ECUDA;
        }
        if (a->start[m] > 0) fn<<<a->start[m], thr, smem, st>>>(*a);
        if (cudaGetLastError() != cudaSuccess) return MONC_PROJ_ECUDA;
    }
    return MONC_PROJ_OK;
}
}  // namespace

extern "C" {

int monc_proj_solve_batch_grouped(const monc_proj_plan_t* plans, const monc_proj_fields* fields, int count,
                                  void* workspace, size_t workspace_bytes, void* stream) {
    if (!plans || !fields || count < 0 || (count > 0 && !workspace)) return MONC_PROJ_EINVAL;
    size_t need = 0;
    int rc = monc_proj_batch_workspace_size(plans, count, &need);
    if (rc) return rc;
    if (workspace_bytes < need || (((uintptr_t)workspace) & 255)) return MONC_PROJ_EINVAL;
    if (count == 0) return MONC_PROJ_OK;
    for (int i = 0; i < count; ++i) {
        const monc_proj_fields& f = fields[i];
        if (!f.u || !f.v || !f.w || !f.u_out || !f.v_out || !f.w_out) return MONC_PROJ_EINVAL;
        const void* ptrs[] = {f.u, f.v, f.w, f.u_out, f.v_out, f.w_out, f.phi_out};
        for (const void* x : ptrs)
            if (((uintptr_t)x) & 15) return MONC_PROJ_EINVAL;
    }
    StreamPool* pool = nullptr;
    rc = stream_pool(&pool);
    if (rc) return rc;
    std::vector<size_t> off(count);
    size_t o = 0;
    for (int i = 0; i < count; ++i) {
        off[i] = o;
        o += align256(plans[i]->ws_bytes);
    }
    // groups: same horizontal size, task shapes and channel count; chunks of
    // at most kGroupMax instances, largest first within a group
    std::map<std::vector<int>, std::vector<int>> groups;
    std::vector<int> singles;
    for (int i = 0; i < count; ++i) {
        const monc_proj_plan_s* p = plans[i];
        if (!group_eligible(p)) {
            singles.push_back(i);
            continue;
        }
        groups[{p->nx, p->ny, p->row_threads, p->col_threads, fields[i].phi_out ? 4 : 3}].push_back(i);
    }
    std::vector<std::vector<int>> chunks;
    for (auto& g : groups) {
        std::vector<int>& v = g.second;
        std::stable_sort(v.begin(), v.end(), [&](int a, int b) { return plans[a]->nz > plans[b]->nz; });
        for (size_t c = 0; c < v.size(); c += kGroupMax)
            chunks.emplace_back(v.begin() + c, v.begin() + std::min(v.size(), c + (size_t)kGroupMax));
    }
    std::lock_guard<std::mutex> lock(pool->mu);
    cudaStream_t st = (cudaStream_t)stream;
    const int nstreams = std::min<int>((int)(chunks.size() + singles.size()), kBatchStreams);
    if (cudaEventRecord(pool->fork, st) != cudaSuccess) { cudaGetLastError(); return MONC_PROJ_ECUDA; }
    for (int j = 0; j < nstreams; ++j)
        if (cudaStreamWaitEvent(pool->s[j], pool->fork, 0) != cudaSuccess) { cudaGetLastError(); return MONC_PROJ_ECUDA; }
    unsigned char* ws = (unsigned char*)workspace;
    int first_error = MONC_PROJ_OK;
    int n = 0;
    for (const auto& c : chunks) {
        const int r = launch_group_chunk(plans, fields, c, off, ws, pool->s[n++ % nstreams]);
        if (r && !first_error) first_error = r;
    }
    for (int i : singles) {
        const monc_proj_fields& f = fields[i];
        const int r = monc_proj_solve(plans[i], f.u, f.v, f.w, f.u_out, f.v_out, f.w_out, f.phi_out, ws + off[i],
                                      pool->s[n++ % nstreams]);
        if (r && !first_error) first_error = r;
    }
    for (int j = 0; j < nstreams; ++j) {
        if (cudaEventRecord(pool->join[j], pool->s[j]) != cudaSuccess ||
            cudaStreamWaitEvent(st, pool->join[j], 0) != cudaSuccess) {
            cudaGetLastError();
            return MONC_PROJ_ECUDA;
        }
    }
    return first_error;
}

int monc_proj_sync_status(monc_proj_plan_t plan, void* stream) {
    if (!plan) return MONC_PROJ_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int h = 0;
    if (cudaMemcpyAsync(&h, plan->err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return MONC_PROJ_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return MONC_PROJ_ECUDA;
    if (h) {
        cudaMemsetAsync(plan->err, 0, sizeof(int), st);
        cudaStreamSynchronize(st);
        return (h & 1) ? MONC_PROJ_ETIMEOUT : MONC_PROJ_EDEVICE;
    }
    return MONC_PROJ_OK;
}

int monc_proj_profile(monc_proj_plan_t plan, int enable) {
    if (!plan) return MONC_PROJ_EINVAL;
    plan->profiling = enable != 0;
    if (enable) plan->nprof = 0;
    return MONC_PROJ_OK;
}

int monc_proj_profile_read(monc_proj_plan_t plan, int max_phases, double* total_ms,
                           int* nphases, int* nsolves) {
    if (!plan || !total_ms || max_phases < 1) return MONC_PROJ_EINVAL;
    for (int i = 0; i < max_phases; ++i) total_ms[i] = 0.0;
    if (nphases) *nphases = kPhases;
    if (nsolves) *nsolves = plan->nprof;
    if (plan->nprof == 0) return MONC_PROJ_OK;
    if (cudaDeviceSynchronize() != cudaSuccess) return MONC_PROJ_ECUDA;
    for (int s = 0; s < plan->nprof; ++s) {
        const cudaEvent_t* ev = &plan->prof_events[(size_t)s * (2 * kPhases)];
        for (int ph = 0; ph < kPhases && ph < max_phases; ++ph) {
            if (!(plan->prof_mask[s] & (1u << ph))) continue;
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev[2 * ph], ev[2 * ph + 1]) != cudaSuccess) return MONC_PROJ_ECUDA;
            total_ms[ph] += ms;
        }
    }
    return MONC_PROJ_OK;
}

const char* monc_proj_phase_name(int phase) {
    return (phase >= 0 && phase < kPhases) ? kPhaseNames[phase] : nullptr;
}

int monc_proj_destroy(monc_proj_plan_t plan) {
    if (!plan) return MONC_PROJ_OK;
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != plan->device) cudaSetDevice(plan->device);
    for (cudaEvent_t e : plan->prof_events) cudaEventDestroy(e);
    if (plan->tables_free) plan->tables_free(plan->dev_tables, plan->tables_user);
    else cudaFree(plan->dev_tables);
    if (dev != plan->device && dev >= 0) cudaSetDevice(dev);
    delete plan;
    return MONC_PROJ_OK;
}

// ---------------------------------------------------------------------------
// Autotuning of the task shapes (no counterpart in the paper).
// ---------------------------------------------------------------------------
namespace {
bool shapes_fit(const monc_proj_plan_s* p) {
    const size_t lim = kSmemMax;
    return p->thr_fwd_rows <= 512 && p->thr_cols <= 512 && p->thr_inv_rows[0] <= 512 && p->thr_inv_rows[1] <= 512 &&
           p->smem_fwd_rows <= lim && p->smem_cols <= lim && p->smem_inv_rows[0] <= lim && p->smem_inv_rows[1] <= lim;
}
// Task shapes and column radix schedule e (32, or 16 where the square-grid
// kernels of that schedule exist).
int apply_shapes(monc_proj_plan_s* p, int rt, int ct, int e) {
    p->row_threads = rt;
    p->col_threads = ct;
    p->col_e = e;
    set_task_shapes(p);
    p->smem_fcols = p->smem_cols;
    if (!shapes_fit(p)) return MONC_PROJ_EUNSUPPORTED;
    if (e != kMaxRadixF32 && (p->precision != MONC_PROJ_MIXED || !p->twy16 ||
                              !pick_cols_square_f32(p->ny, p->nxp, p->tw_cols, p->bs_col, false, e)))
        return MONC_PROJ_EUNSUPPORTED;
    return p->precision == MONC_PROJ_FP64 ? set_kernel_attrs<double>(p) : set_kernel_attrs<float>(p);
}
}  // namespace

int monc_proj_autotune(monc_proj_plan_t plan, const void* u, const void* v, const void* w, void* u_out,
                       void* v_out, void* w_out, void* workspace, int reps, void* stream, int* row_threads,
                       int* col_threads) {
    if (!plan || !u || !v || !w || !u_out || !v_out || !w_out || !workspace) return MONC_PROJ_EINVAL;
    const int r0 = plan->row_threads, c0 = plan->col_threads, e0s = plan->col_e;
    auto report = [&](int rc) {
        if (row_threads) *row_threads = plan->row_threads;
        if (col_threads) *col_threads = plan->col_threads;
        return rc;
    };
    if (plan->fused || plan->persist_cols || plan->tma_cols || plan->pipe || (!plan->ct_rows && !plan->ct_cols))
        return report(MONC_PROJ_OK);
    if (reps <= 0) reps = 3;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        return report(MONC_PROJ_ECUDA);
    }
    const int rts[] = {32, 64, 128};
    // column candidates: (threads per tile, radix schedule)
    const std::pair<int, int> cts[] = {{128, 32}, {256, 32}, {512, 32}, {256, 16}};
    float best = INFINITY;
    int br = r0, bc = c0, be = e0s;
    int rc = MONC_PROJ_OK;
    std::vector<std::vector<int>> seen;      // (rows per forward task, columns per tile, schedule) tried
    for (int rt : rts) {
        if (!plan->ct_rows && rt != r0) continue;
        for (const auto& cte : cts) {
            const int ct = cte.first, ce = cte.second;
            if (!plan->ct_cols && (ct != c0 || ce != e0s)) continue;
            if (apply_shapes(plan, rt, ct, ce) != MONC_PROJ_OK) continue;
            const std::vector<int> key{plan->rows_fwd, plan->tw_cols, plan->col_e};
            if (std::find(seen.begin(), seen.end(), key) != seen.end()) continue;
            seen.push_back(key);
            rc = monc_proj_solve(plan, u, v, w, u_out, v_out, w_out, nullptr, workspace, stream);
            if (rc != MONC_PROJ_OK) break;
            cudaEventRecord(e0, st);
            for (int i = 0; i < reps && rc == MONC_PROJ_OK; ++i)
                rc = monc_proj_solve(plan, u, v, w, u_out, v_out, w_out, nullptr, workspace, stream);
            cudaEventRecord(e1, st);
            if (rc != MONC_PROJ_OK || cudaEventSynchronize(e1) != cudaSuccess) {
                if (rc == MONC_PROJ_OK) rc = MONC_PROJ_ECUDA;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                br = rt;
                bc = ct;
                be = ce;
            }
        }
        if (rc != MONC_PROJ_OK) break;
    }
    cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const bool ok = rc == MONC_PROJ_OK;
    const int ra = apply_shapes(plan, ok ? br : r0, ok ? bc : c0, ok ? be : e0s);
    return report(rc != MONC_PROJ_OK ? rc : ra);
}

int monc_proj_set_schedule(monc_proj_plan_t plan, int row_threads, int col_threads, int col_elems) {
    if (!plan) return MONC_PROJ_EINVAL;
    if (plan->fused || plan->persist_cols || plan->tma_cols || plan->pipe || plan->tc_cols ||
        plan->precision == MONC_PROJ_FP64 || plan->precision == MONC_PROJ_REFINED)
        return MONC_PROJ_EUNSUPPORTED;
    const bool shape_ok = (row_threads == 32 || row_threads == 64 || row_threads == 128) &&
                          (col_threads == 128 || col_threads == 256 || col_threads == 512) &&
                          (col_elems == 32 || col_elems == 16);
    if (!shape_ok) return MONC_PROJ_EINVAL;
    if ((!plan->ct_rows && row_threads != plan->row_threads) ||
        (!plan->ct_cols && (col_threads != plan->col_threads || col_elems != plan->col_e)))
        return MONC_PROJ_EUNSUPPORTED;
    const int r0 = plan->row_threads, c0 = plan->col_threads, e0 = plan->col_e;
    const int rc = apply_shapes(plan, row_threads, col_threads, col_elems);
    if (rc != MONC_PROJ_OK) {
        apply_shapes(plan, r0, c0, e0);
        return rc;
    }
    return MONC_PROJ_OK;
}

int monc_proj_plan_schedule(monc_proj_plan_t plan, int* row_elems, int* col_elems, int* row_threads,
                            int* col_threads) {
    if (!plan) return MONC_PROJ_EINVAL;
    const bool fp64 = plan->precision == MONC_PROJ_FP64;
    if (row_elems) *row_elems = fp64 ? kMaxRadixF64 : kMaxRadixF32;
    if (col_elems) *col_elems = fp64 ? kMaxRadixF64 : plan->col_e;
    if (row_threads) *row_threads = plan->row_threads;
    if (col_threads) *col_threads = plan->col_threads;
    return MONC_PROJ_OK;
}

int monc_proj_plan_info(monc_proj_plan_t plan, int* nx, int* ny, int* nz, int* precision,
                        long long* fp64_columns, long long* total_columns) {
    if (!plan) return MONC_PROJ_EINVAL;
    if (nx) *nx = plan->nx;
    if (ny) *ny = plan->ny;
    if (nz) *nz = plan->nz;
    if (precision) *precision = plan->precision_api;
    const long long tot = (long long)plan->ny * plan->nxh;
    if (total_columns) *total_columns = tot;
    if (fp64_columns) *fp64_columns = plan->fp64_cols;
    return MONC_PROJ_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// No-alloc entry point: tables and workspace in a static device array.
// ---------------------------------------------------------------------------

static __device__ __align__(256) unsigned char g_noalloc_scratch[MONC_PROJ_NOALLOC_SCRATCH_BYTES];

namespace {

// Device address of the static array on the current device, looked up at
// every call (cheap; nothing cached that a context reset could leave stale).
int noalloc_base(void** out, int* device) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return MONC_PROJ_ECUDA; }
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) { cudaGetLastError(); return MONC_PROJ_ECUDA; }
    *out = ptr;
    *device = dev;
    return MONC_PROJ_OK;
}

}  // namespace

extern "C" int monc_proj_solve_noalloc(int nx, int ny, int nz, double dx, double dy,
                                       const double* dz, const double* rho_c, const double* rho_f,
                                       int precision, const void* u, const void* v, const void* w,
                                       void* u_out, void* v_out, void* w_out, void* phi_out,
                                       void* stream) {
    const int vr = validate_grid(nx, ny, nz, dx, dy, dz, rho_c, rho_f, precision);
    if (vr != MONC_PROJ_OK) return vr;
    if (!u || !v || !w || !u_out || !v_out || !w_out) return MONC_PROJ_EINVAL;
    const void* ptrs[] = {u, v, w, u_out, v_out, w_out, phi_out};
    for (const void* x : ptrs)
        if (((uintptr_t)x) & 15) return MONC_PROJ_EINVAL;

    monc_proj_plan_s plan{};
    std::vector<unsigned char> blob;
    TableOffsets to{};
    plan_prepare(&plan, nx, ny, nz, dx, dy, dz, rho_c, rho_f, precision, blob, to);
    const size_t tables = align256(plan_table_bytes(&plan, blob.size(), to));
    if (tables + plan.ws_bytes > (size_t)MONC_PROJ_NOALLOC_SCRATCH_BYTES) return MONC_PROJ_ESCRATCH;
    // the table upload reads `blob`, which dies with this call: a graph
    // captured here would replay a copy from freed host memory
    cudaStream_t st = (cudaStream_t)stream;
    {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) { cudaGetLastError(); return MONC_PROJ_ECUDA; }
        if (cs != cudaStreamCaptureStatusNone) return MONC_PROJ_EUNSUPPORTED;
    }

    void* base = nullptr;
    const int br = noalloc_base(&base, &plan.device);
    if (br != MONC_PROJ_OK) return br;
    const int ar = plan_kernel_attrs(&plan);
    if (ar != MONC_PROJ_OK) return ar;
    // The blob carries a zeroed device error word, so every call starts clean.
    if (cudaMemcpyAsync(base, blob.data(), blob.size(), cudaMemcpyHostToDevice, st) != cudaSuccess) {
        cudaGetLastError();
        return MONC_PROJ_ECUDA;
    }
    unsigned char* b = (unsigned char*)base;
    plan_bind(&plan, b, to);
    if (plan_fill_tables(&plan, st) != MONC_PROJ_OK) return MONC_PROJ_ECUDA;
    const ProjParams q = make_params(&plan, u, v, w, u_out, v_out, w_out, phi_out, b + tables);
    return run_solve(&plan, q, st);
}
