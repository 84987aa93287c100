/*
 * monc_proj.h -- C ABI of the GB300 anelastic pressure projection.
 *
 * The operation (paper, Section 4): the pressure terms of the anelastic
 * equations are handled by a forward FFT over the horizontally periodic
 * domain, a vertical ODE solved in Fourier space for each horizontal
 * wavenumber, and a backward FFT.  Concretely one solve computes, for a
 * provisional Arakawa-C velocity (u*, v*, w*):
 *
 *   a1  D   = (u_i - u_{i-1})/dx + (v_j - v_{j-1})/dy
 *             + (rho_f[k+1] w[k+1] - rho_f[k] w[k]) / (rho_c[k] dz[k])
 *   a2  D^  = forward real 2D FFT of D on every level
 *   a3  for every (kx,ky): the tridiagonal vertical problem
 *         (A[k] p[k-1] - (A[k]+A[k+1]) p[k] + A[k+1] p[k+1]) / (rho_c[k] dz[k])
 *           + lambda p[k] = D^[k],   A[k] = rho_f[k]/dzn[k], A[0]=A[nz]=0,
 *         lambda = 2(cos(2 pi kx/nx)-1)/dx^2 + 2(cos(2 pi ky/ny)-1)/dy^2,
 *         the (0,0) column pinned by p^[k=0] = 0
 *   a4  inverse FFT (of the spectral gradients of p)
 *   a5  u = u* - (p_{i+1}-p_i)/dx,  v = v* - (p_{j+1}-p_j)/dy,
 *       w = w* - (p_k - p_{k-1})/dzn[k] on interior faces, w = 0 at the
 *       bottom and top faces.
 *
 * Grid and layout.  Cells i < nx (x, fastest), j < ny, k < nz, C row-major:
 * u and v are [nz][ny][nx] (u on east faces, v on north faces); w is
 * [nz+1][ny][nx] on horizontal faces, face k at height sum(dz[0..k-1]).
 * dzn[k] = (dz[k-1]+dz[k])/2 is the centre-to-centre spacing at face k.
 * x and y are periodic.  The potential p is at cell centres, [nz][ny][nx].
 *
 * Precision.  MONC_PROJ_FP64: every field is double and every step runs in
 * FP64.  MONC_PROJ_MIXED: every field is float; divergence, horizontal
 * transforms and the correction run in FP32, the vertical solve (a3) runs in
 * FP64 for the columns whose conditioning needs it (near-zero horizontal
 * wavenumbers) and in FP32 for the rest.  MONC_PROJ_REFINED: every field is
 * double; the solve runs three passes, each a mixed-precision solve for a
 * potential (the divergence of the pass's input formed in FP64, FP32
 * transforms) followed by the subtraction of that potential's exact discrete
 * gradient in FP64.  Each pass's divergence is the previous passes' error, so
 * each pass shrinks it by the mixed solver's relative accuracy: one pass
 * leaves ~1e-7, two ~1e-11, three FP64-level relative error (the environment
 * variable MONC_PROJ_REFINE_PASSES, 1..4, read when a plan is made, sets the
 * count).  The workspace also holds one FP64 field.  This is the
 * single-precision solve with a double-precision restart that the paper
 * proposes as further work (§5).  MONC_PROJ_MIXED_Z64: as MONC_PROJ_MIXED,
 * but the vertical elimination runs in FP64 arithmetic for every column (the
 * FP32 storage of the spectra is unchanged); slower on this GPU, whose FP64
 * rate is a small fraction of its FP32 rate.  Plans of it report it as
 * their precision; everything else about them is that of MONC_PROJ_MIXED.
 *
 * Errors.  Every call returns a monc_proj_status.  Nothing aborts, traps or
 * throws across this boundary.  Problems found on the device (a bounded
 * wait that gave up, an index outside its buffer) are latched in a device
 * word of the plan and reported by monc_proj_sync_status().
 *
 * Threading.  A plan is immutable after creation.  Several solves with one
 * plan may run concurrently on different streams only with separate
 * workspaces.
 */
#ifndef MONC_PROJ_H
#define MONC_PROJ_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct monc_proj_plan_s* monc_proj_plan_t;

typedef enum {
    MONC_PROJ_OK = 0,
    MONC_PROJ_EINVAL = 1,        /* bad argument (NULL, size, non-finite or non-positive spacing) */
    MONC_PROJ_EUNSUPPORTED = 2,  /* nx or ny not of the form 2^a 3^b 5^c, or above the size limit */
    MONC_PROJ_ENOMEM = 3,        /* device allocation failed while building a plan */
    MONC_PROJ_ECUDA = 4,         /* a CUDA runtime call failed (launch, copy) */
    MONC_PROJ_ETIMEOUT = 5,      /* a bounded device wait gave up (latched device error) */
    MONC_PROJ_EDEVICE = 6,       /* another device-detected error (latched device error) */
    MONC_PROJ_ESCRATCH = 7,      /* monc_proj_solve_noalloc: problem too large for its static scratch */
    MONC_PROJ_ENOCONV = 8,       /* monc_proj_solve_krylov: iteration limit reached before the tolerance */
    MONC_PROJ_EBREAKDOWN = 9     /* monc_proj_solve_krylov: a BiCGStab denominator was exactly zero */
} monc_proj_status;

typedef enum {
    MONC_PROJ_FP64 = 0,
    MONC_PROJ_MIXED = 1,
    MONC_PROJ_REFINED = 2,
    MONC_PROJ_MIXED_Z64 = 3
} monc_proj_precision;

/* Largest nx or ny a plan accepts. */
#define MONC_PROJ_MAX_N 4096

/*
 * Allocator of plan tables (the paper has no counterpart).
 *
 * By default monc_proj_plan takes its device tables (a few tens of KB to a
 * few MB per plan) from cudaMalloc and monc_proj_destroy returns them with
 * cudaFree.  A host application that manages device memory through its own
 * pool installs its allocator here instead:
 *
 *   alloc(bytes, user)    returns device memory of at least `bytes` on the
 *                         current device, 256-byte aligned, or NULL on failure
 *   release(ptr, user)    returns memory obtained from alloc
 *   user                  passed back unchanged to both
 *
 * Both NULL restore cudaMalloc / cudaFree; exactly one NULL is EINVAL.  The
 * setting is process-wide and applies to plans created afterwards; a plan
 * keeps the release function it was created with.  When alloc returns NULL,
 * monc_proj_plan returns MONC_PROJ_ENOMEM before it touches the device.
 * Set it before plans are created concurrently from other threads.
 * Workspaces and fields are always the caller's.
 */
typedef void* (*monc_proj_alloc_fn)(size_t bytes, void* user);
typedef void (*monc_proj_free_fn)(void* ptr, void* user);
int monc_proj_set_allocator(monc_proj_alloc_fn alloc, monc_proj_free_fn release, void* user);

/*
 * Build a plan for one grid (the set-up of steps a2-a4: twiddle tables,
 * modified wavenumbers lambda(kx,ky) of the 5-point horizontal Laplacian, the
 * rho0-weighted vertical coefficients and the spectral gradient symbols).
 *
 *   out        receives the plan handle (owned by the caller until destroy)
 *   nx, ny     horizontal cell counts, 1..MONC_PROJ_MAX_N, each 2^a 3^b 5^c
 *   nz         number of levels, >= 1
 *   dx, dy     horizontal spacing [m], > 0 and finite
 *   dz         host array [nz], layer thicknesses [m], > 0
 *   rho_c      host array [nz], reference density at cell centres, > 0
 *   rho_f      host array [nz+1], reference density at w faces, > 0
 *   precision  MONC_PROJ_FP64, MONC_PROJ_MIXED, MONC_PROJ_REFINED or
 *              MONC_PROJ_MIXED_Z64
 *   stream     cudaStream_t (may be NULL) used for the plan's uploads and, in
 *              mixed plans, the kernel that fills the table of the FP64
 *              columns' pivots (1/e of the vertical elimination, which depend
 *              on lambda and the vertical coefficients only: 8 bytes per level
 *              and column of the near-zero-wavenumber warps); the call returns
 *              after they have completed
 *
 * The host arrays are copied; the caller may free them when this returns.
 * The plan's device tables live on the device that is current at the call.
 *
 * Returns MONC_PROJ_ENOMEM when the tables cannot be allocated (see
 * monc_proj_set_allocator).  The bounded dependency waits of the opt-in
 * persistent kernels give up after a fixed number of polls (about a second)
 * and latch a timeout that monc_proj_sync_status reports as
 * MONC_PROJ_ETIMEOUT; MONC_PROJ_SPIN_LIMIT in the environment, read here,
 * sets that number (0: give up at the first unmet poll, for tests).
 */
int monc_proj_plan(monc_proj_plan_t* out, int nx, int ny, int nz, double dx, double dy,
                   const double* dz, const double* rho_c, const double* rho_f,
                   int precision, void* stream);

/* Bytes of caller-owned device workspace one solve with this plan needs. */
int monc_proj_workspace_size(monc_proj_plan_t plan, size_t* bytes);

/*
 * One projection, enqueued on `stream` (cudaStream_t, NULL = legacy default);
 * the call returns without waiting for the device.
 *
 *   u, v       device [nz][ny][nx]     provisional velocities (double or float per precision)
 *   w          device [nz+1][ny][nx]   provisional vertical velocity; faces 0 and nz ignored
 *   u_out, v_out, w_out   device, same shapes; may alias u, v, w (in place)
 *   phi_out    device [nz][ny][nx] or NULL: the potential p (with its pin)
 *   workspace  device, >= monc_proj_workspace_size() bytes, 256-byte aligned;
 *              it must not be used by another solve in flight at the same time
 *
 * Pointers must be 16-byte aligned.  Outputs are complete when the stream
 * reaches the end of the enqueued work.
 */
int monc_proj_solve(monc_proj_plan_t plan, const void* u, const void* v, const void* w,
                    void* u_out, void* v_out, void* w_out, void* phi_out,
                    void* workspace, void* stream);

/*
 * One projection of host arrays: the fields are copied to a caller-owned
 * device staging area, projected there in place, and copied back, all
 * enqueued on `stream` (one cudaMemcpyAsync per array); the call returns
 * without waiting.  Host buffers should be page-locked for the copies to run
 * asynchronously (pageable ones make the copies wait on the host).  Two
 * solves on different streams with different staging areas and workspaces
 * overlap one's copies in with the other's copies out.
 *
 *   u, v, w            host, shapes and element type as in monc_proj_solve
 *   u_out, v_out, w_out host, same shapes (may be the input buffers)
 *   phi_out            host [nz][ny][nx] or NULL
 *   staging            device, >= monc_proj_host_staging_size(plan, phi_out != NULL)
 *                      bytes, 256-byte aligned
 *   workspace          as in monc_proj_solve
 * Errors: EINVAL for NULL plan, field, staging or workspace pointers or a
 * short staging area; ECUDA if a copy cannot be enqueued.
 */
int monc_proj_host_staging_size(monc_proj_plan_t plan, int with_phi, size_t* bytes);
int monc_proj_solve_host(monc_proj_plan_t plan, const void* u, const void* v, const void* w,
                         void* u_out, void* v_out, void* w_out, void* phi_out,
                         void* staging, size_t staging_bytes, void* workspace, void* stream);

/* One field set of a batched solve (device pointers, as in monc_proj_solve). */
typedef struct {
    const void* u;
    const void* v;
    const void* w;
    void* u_out;
    void* v_out;
    void* w_out;
    void* phi_out;      /* may be NULL */
} monc_proj_fields;

/*
 * Bytes of workspace for a batched solve over `count` plans: the sum of
 * their workspaces plus the batch's task tables.
 */
int monc_proj_batch_workspace_size(const monc_proj_plan_t* plans, int count, size_t* bytes);

/*
 * `count` independent projections (plans may differ in size and precision),
 * ordered after the work already on `stream` and before work enqueued on it
 * afterwards.  Inside, the instances run concurrently on an internal pool of
 * streams (largest first), so uneven small problems share the GPU; each
 * result equals that of monc_proj_solve on the same inputs.  Instance i uses
 * the workspace slice that starts at the sum of align256(workspace_size) of
 * instances 0..i-1.  The call only enqueues work; its fork and join are
 * events, so a caller may capture it into a CUDA graph on `stream`.  Errors:
 * EINVAL for a NULL plan or field pointer or a short workspace; the first
 * failing instance's status otherwise.
 */
int monc_proj_solve_batch(const monc_proj_plan_t* plans, const monc_proj_fields* fields,
                          int count, void* workspace, size_t workspace_bytes, void* stream);

/*
 * The same batch in grouped launches: the instances that share the
 * horizontal size, the task shapes and whether phi is requested form a
 * group, and each phase of the projection runs as one launch per group
 * (chunks of up to 20 instances) whose blocks cover every instance's tasks,
 * instance after instance; the groups run concurrently on the internal
 * stream pool.  Instances of FP32 mixed plans with compile-time transform
 * lengths (64, 96, 128, 192, 256, 512, 1024) and the default kernels are
 * grouped; any other instance runs as in monc_proj_solve_batch.  Each
 * instance's parameters travel in the launches' parameters (nothing is
 * uploaded), so the call may be captured into a CUDA graph on `stream`.
 * Results equal monc_proj_solve's bit for bit.  Arguments, workspace layout
 * and errors as monc_proj_solve_batch; the workspace must be 256-byte aligned.
 */
int monc_proj_solve_batch_grouped(const monc_proj_plan_t* plans, const monc_proj_fields* fields,
                                  int count, void* workspace, size_t workspace_bytes, void* stream);

/*
 * Synchronise `stream` and report (then clear) the plan's latched device
 * error: MONC_PROJ_OK, MONC_PROJ_ETIMEOUT or MONC_PROJ_EDEVICE.
 */
int monc_proj_sync_status(monc_proj_plan_t plan, void* stream);

/* Release the plan's device tables.  NULL is accepted. */
int monc_proj_destroy(monc_proj_plan_t plan);

/* Static, human-readable name of a status code. */
const char* monc_proj_status_string(int status);

/*
 * Per-phase device timing, for diagnostics and the benchmark's roofline.
 * enable != 0 clears what was recorded and starts recording CUDA events on
 * the solve's stream before and after every kernel of each following solve
 * with this plan (at most MONC_PROJ_PROFILE_MAX solves); enable == 0 stops.
 */
#define MONC_PROJ_PROFILE_MAX 4096
int monc_proj_profile(monc_proj_plan_t plan, int enable);

/*
 * Wait for the recorded solves and report, per kernel phase, the summed
 * device time in milliseconds (total_ms[max_phases]).  *nphases receives
 * the number of phases, *nsolves the number of solves recorded.
 */
int monc_proj_profile_read(monc_proj_plan_t plan, int max_phases, double* total_ms,
                           int* nphases, int* nsolves);

/* Static name of a kernel phase ("fwd_rows", "tridiag", ...), NULL if out of range. */
const char* monc_proj_phase_name(int phase);

/* ---------------------------------------------------------------------------
 * Phases of a distributed projection (paper, Section 4: the model's FFT
 * solver decomposes the domain into pencils and moves data between them with
 * a global all-to-all for every transform).  One large projection sharded
 * over P processes runs, per process:
 *   1. monc_proj_forward_slab   on its z-slab of levels [k0, k1): the
 *      divergence and the forward horizontal transform (steps a1-a2);
 *   2. an all-to-all (the caller's collective) that turns the slabs of the
 *      spectrum into pencils of spectral rows [j0, j1) over all levels;
 *   3. monc_proj_vertical_pencil on its pencil: the vertical solve (a3),
 *      giving p^ and the vertical gradient gz^;
 *   4. the reverse all-to-all of p^ and gz^ back to z-slabs;
 *   5. monc_proj_inverse_slab   on its slab: the inverse transforms and the
 *      correction of u, v, w (a4-a5).
 * Each call runs the kernels of monc_proj_solve on its sub-domain, so the
 * slab and pencil results are those of the whole solve (bitwise, for the
 * same plan).  The plan is made for the whole grid (nx, ny, nz and the whole
 * column's profiles); only FP64 and mixed plans with the default kernels are
 * accepted (EUNSUPPORTED otherwise).  All arrays are device arrays of the
 * plan's element type; spectra are complex (two reals per value).
 * Pointers must be 16-byte aligned, the workspace 256-byte aligned and at
 * least monc_proj_workspace_size() bytes; the calls enqueue on `stream` and
 * return without waiting.  Errors: EINVAL for a NULL pointer, a misaligned
 * pointer or an empty or out-of-range slab or pencil.
 * ------------------------------------------------------------------------- */

/* Row pitch (complex values) of the spectral arrays: rows hold the kx =
 * 0 .. nx/2 half spectrum and are padded to `*nxp` values. */
int monc_proj_spectral_pitch(monc_proj_plan_t plan, int* nxp);

/*
 * a1-a2 on the cell levels k0 .. k1-1 (0 <= k0 < k1 <= nz).
 *   u, v   [k1-k0][ny][nx]     the slab's levels of u and v
 *   w      [k1-k0+1][ny][nx]   the slab's faces k0 .. k1 (face k1 is read
 *                              only when k1 < nz; face 0 is never read)
 *   dhat   [k1-k0][ny][nxp]    out: the horizontal spectrum (unnormalised
 *                              forward transform) of rho_c[k] dz[k] D[k], D
 *                              the divergence of step a1 at level k
 */
int monc_proj_forward_slab(monc_proj_plan_t plan, int k0, int k1, const void* u, const void* v, const void* w,
                           void* dhat, void* workspace, void* stream);

/*
 * a3 on the spectral rows j0 .. j1-1 (0 <= j0 < j1 <= ny; row j holds
 * wavenumber ky = j for j <= ny/2 and j - ny above) of every level.
 *   spec   [nz][j1-j0][nxp]    in: D^ of the pencil's rows; out: p^
 *   gz     [nz][j1-j0][nxp]    out: the vertical gradient gz^ at faces
 *                              1 .. nz-1 (level 0 holds scratch)
 * p^ and gz^ carry the inverse transform's 1/(nx ny), so step a4 is an
 * unnormalised inverse transform.
 * The mean mode (kx = ky = 0) carries the potential's pin (level 0 zero);
 * in a mixed plan the rows of small |lambda| run FP64 as in the whole solve.
 */
int monc_proj_vertical_pencil(monc_proj_plan_t plan, int j0, int j1, void* spec, void* gz, void* workspace,
                              void* stream);

/*
 * a4-a5 on the cell levels k0 .. k1-1.
 *   phat, gz   [k1-k0][ny][nxp]    p^ and gz^ of the slab's levels (gz^ of
 *                                  level 0 is not read)
 *   u, v       [k1-k0][ny][nx]     the provisional velocities of the slab
 *   w          [k1-k0+1][ny][nx]   faces k0 .. k1 (face k1 is not read)
 *   u_out, v_out [k1-k0][ny][nx], w_out [k1-k0+1][ny][nx]: the projected
 *              fields; faces k0 .. k1-1 of w_out are written, and face k1
 *              (zero) only when k1 == nz; the outputs may alias the inputs
 */
int monc_proj_inverse_slab(monc_proj_plan_t plan, int k0, int k1, const void* phat, const void* gz, const void* u,
                           const void* v, const void* w, void* u_out, void* v_out, void* w_out, void* workspace,
                           void* stream);

/*
 * Reordering for the all-to-alls.  Items (levels or spectral rows) are split
 * over `parts` processes in contiguous blocks: with n = q*parts + r, part s
 * holds [s*q + min(s, r), (s+1)*q + min(s+1, r)) (the first r parts one item
 * more).  Pack turns a slab [nzl][ny][nxp] (complex) into the blocks for
 * parts 0 .. parts-1, one after the other, block s [nzl][rows of s][nxp]:
 * the send buffer of the slab -> pencil all-to-all, whose receive buffer,
 * the blocks of slabs 0 .. parts-1 one after the other, is the pencil
 * [nz][rows][nxp] itself.  Unpack is the inverse map, for the pencil -> slab
 * all-to-all (whose send buffer is the pencil itself: the levels of slab s
 * are one block).  1 <= nzl <= nz; src and dst must not overlap.
 */
int monc_proj_pack_pencils(monc_proj_plan_t plan, int nzl, int parts, const void* slab, void* packed, void* stream);
int monc_proj_unpack_pencils(monc_proj_plan_t plan, int nzl, int parts, const void* packed, void* slab,
                             void* stream);

/*
 * monc_proj_solve_noalloc -- one projection that allocates no device memory.
 *
 * The paper has no counterpart; this entry point exists for callers that
 * cannot allocate: host applications that own every byte of device memory
 * through their own pool and forbid libraries from calling cudaMalloc, model
 * components that are handed finished device arrays by their host model and
 * keep no allocator of their own, and latency-critical loops that cannot
 * afford cudaMalloc's implicit device-wide synchronisation.  Such a caller
 * passes only the grid, the host profiles and its device inputs and outputs.
 *
 * Everything else the solve needs -- the grid tables (twiddles, modified
 * wavenumbers, vertical coefficients) and the solve's workspace -- lives in
 * one static device array of MONC_PROJ_NOALLOC_SCRATCH_BYTES bytes compiled
 * into this library.  Every process that loads the library holds that array
 * on every GPU where the library's kernels are loaded, until it exits.
 *
 * Arguments are those of monc_proj_plan followed by those of monc_proj_solve
 * (same layouts, types, alignment and in-place rules); there is no plan and
 * no workspace argument.  The work is enqueued on `stream`.
 *
 * Limits and behaviour:
 *  - a grid whose tables plus workspace exceed MONC_PROJ_NOALLOC_SCRATCH_BYTES
 *    is rejected with MONC_PROJ_ESCRATCH before anything is enqueued (about
 *    64 x 64 x 64 in FP64 or 80 x 80 x 64 in mixed precision fit);
 *  - every call looks up the array's device address on the current device
 *    (cudaGetSymbolAddress), so nothing is cached across calls or contexts;
 *  - the tables are uploaded (and a mixed plan's FP64 pivot table filled by a
 *    kernel) at every call; the upload is a cudaMemcpyAsync from pageable
 *    host memory that the call owns only while it runs, so the call may wait
 *    for the work already on `stream` before it returns, and a call on a
 *    stream that is being captured into a CUDA graph is refused with
 *    MONC_PROJ_EUNSUPPORTED before anything is enqueued (a replay would read
 *    host memory that no longer exists);
 *  - every call on a device shares the one array and overwrites the previous
 *    call's tables and workspace: calls whose GPU work overlaps (different
 *    streams, or different host threads without ordering) race and give wrong
 *    results.  Calls on one stream are ordered and safe;
 *  - device-detected errors of the call are not reported (there is no plan
 *    to latch them in).
 */
#define MONC_PROJ_NOALLOC_SCRATCH_BYTES (32u << 20)
int monc_proj_solve_noalloc(int nx, int ny, int nz, double dx, double dy,
                            const double* dz, const double* rho_c, const double* rho_f,
                            int precision, const void* u, const void* v, const void* w,
                            void* u_out, void* v_out, void* w_out, void* phi_out, void* stream);

/*
 * monc_proj_autotune -- pick the plan's task shapes and column radix schedule
 * by timing them (a tuning step with no counterpart in the paper).
 *
 * For compile-time transform lengths the row kernels take tasks of 32, 64 or
 * 128 threads and the column kernels tiles of 128, 256 or 512 threads (the
 * candidates whose shared memory fits).  FP32 plans of square 256, 512 and
 * 1024 grids also try a second radix schedule for the column transforms:
 * 16 elements per thread (1024 = 16*16*4, three shared-memory passes, fewer
 * registers and more resident warps) against the default 32 (1024 = 32*32,
 * two passes), with 256-thread tiles.  Each distinct candidate runs one
 * warm-up solve and `reps` timed solves (3 if reps <= 0) of the caller's
 * fields on `stream`, timed with CUDA events; the fastest is kept in the plan.
 * The call waits for the stream.  The solves write u_out, v_out, w_out (they
 * may alias the inputs only if the inputs may be overwritten).  Task shapes
 * decide how the work is split into blocks, never the arithmetic: with one
 * schedule the results are bitwise the same for every shape.  The two
 * schedules add the same terms in a different order, so their results differ
 * by rounding (both within the mixed path's tolerance).  The call changes the
 * plan: make it before the plan is shared between threads or solves are
 * captured into a graph.  Plans running an opt-in kernel variant, or with
 * run-time lengths both ways, keep their shapes.
 *   row_threads, col_threads  host, nullable: the shapes kept
 *   (monc_proj_plan_schedule reports the schedule kept)
 * Errors: EINVAL for NULL plan, field or workspace pointers; the first failing
 * solve's status (the plan then keeps the shapes it had).
 */
int monc_proj_autotune(monc_proj_plan_t plan, const void* u, const void* v, const void* w, void* u_out,
                       void* v_out, void* w_out, void* workspace, int reps, void* stream, int* row_threads,
                       int* col_threads);

/* ---------------------------------------------------------------------------
 * Krylov pressure solve (paper, Section 4: the model's second pressure solver
 * runs a Krylov subspace method, BiCGStab preconditioned by ILU, on the same
 * Poisson problem; the closing section names a preconditioner built on the
 * problem's structure as further work).
 *
 * Solves L phi = D(u*) with L = D o G (the operator of monc_proj_solve,
 * written as its 7-point stencil) by BiCGStab from phi = 0, the
 * preconditioner applied to the search directions:
 *   MONC_PROJ_PC_NONE  none;
 *   MONC_PROJ_PC_LINE  the vertical lines of L (its vertical rows plus the
 *                      diagonal of its horizontal part): one Thomas solve per
 *                      column (i, j), all columns in parallel.
 * Stops when ||r||_2 <= tol ||b||_2 (b = D(u*), r the recurrence residual),
 * tested after each half step and each full step.  Precision follows the
 * plan: FP64 and REFINED plans run the vectors in FP64, MIXED plans in FP32
 * (the paper's single-precision solver; GB300 runs FP32 arithmetic 64 times
 * faster than FP64, and FP32 attains relative residuals down to about 1e-6).
 * The iterate is accumulated in FP64 in both and the gradient G phi of the
 * outputs formed in FP64.  The outputs are those of
 * monc_proj_solve: u - G phi, phi pinned to a zero level-0 horizontal mean,
 * w zero on the bottom and top faces.
 *
 *   plan        any plan; its precision sets the field type (FP32 for
 *               MIXED, FP64 otherwise)
 *   u .. phi_out  device arrays of that type laid out as for
 *               monc_proj_solve, aligned to the element size; outputs may
 *               alias the inputs; phi_out may be NULL
 *   workspace   device, caller-owned, 256-byte aligned, at least
 *               monc_proj_krylov_workspace_size bytes (one FP64 and seven
 *               field-type arrays of nx*ny*nz values, and a few KB)
 *   tol         >= 0 and finite (0: run max_iter iterations)
 *   max_iter    >= 0
 *   precond     MONC_PROJ_PC_NONE or MONC_PROJ_PC_LINE
 *   iterations, rel_residual  host, nullable: iterations completed and the
 *               final ||r||/||b|| (0 for a divergence-free input)
 * Returns OK when converged; MONC_PROJ_ENOCONV at the iteration limit and
 * MONC_PROJ_EBREAKDOWN when a BiCGStab denominator is exactly zero (in both
 * cases the outputs hold the projection with the last iterate); EINVAL for a
 * bad argument; ECUDA for a failed launch or copy.
 * The calling thread waits on `stream` every 8 iterations (the convergence
 * test reads the residual back; iterations enqueued past the one that stops
 * do nothing), so the call cannot be captured into a graph.
 */
typedef enum { MONC_PROJ_PC_NONE = 0, MONC_PROJ_PC_LINE = 1 } monc_proj_precond_t;
int monc_proj_krylov_workspace_size(monc_proj_plan_t plan, size_t* bytes);
int monc_proj_solve_krylov(monc_proj_plan_t plan, const void* u, const void* v, const void* w,
                           void* u_out, void* v_out, void* w_out, void* phi_out, void* workspace,
                           double tol, int max_iter, int precond, int* iterations, double* rel_residual,
                           void* stream);

/*
 * The plan's transform schedules: elements per thread of the compile-time
 * row and column plans (the largest radix of a stage: 32 or 16 in FP32, 16
 * in FP64) and the threads of a row task and of a column tile.  All outputs
 * host, nullable.
 */
int monc_proj_plan_schedule(monc_proj_plan_t plan, int* row_elems, int* col_elems, int* row_threads,
                            int* col_threads);

/*
 * Set the task shapes and column radix schedule of an FP32 mixed plan
 * directly (for example one that monc_proj_autotune chose in an earlier run):
 * row_threads 32, 64 or 128; col_threads 128, 256 or 512; col_elems 32, or
 * 16 for square 256, 512 and 1024 grids with col_threads 256.  EINVAL for
 * values outside those sets; EUNSUPPORTED for FP64 and refined plans, plans
 * running an opt-in kernel variant, a run-time length whose shape would
 * change, or a combination without kernels or shared memory (the plan then
 * keeps what it had).  Same threading rule as monc_proj_autotune.
 */
int monc_proj_set_schedule(monc_proj_plan_t plan, int row_threads, int col_threads, int col_elems);

/* Plan introspection: grid sizes, precision and the FP64-column count of a3. */
int monc_proj_plan_info(monc_proj_plan_t plan, int* nx, int* ny, int* nz, int* precision,
                        long long* fp64_columns, long long* total_columns);

#ifdef __cplusplus
}
#endif

#endif /* MONC_PROJ_H */
