// Krylov pressure solver (paper, Section 4: the model's second pressure
// solver, BiCGStab on the same Poisson problem as the FFT solver).  Host-side
// interface between the C ABI (monc_proj.cu) and the kernels (kern_krylov.cu).
#pragma once
#include <cstddef>
#include <cuda_runtime.h>

namespace mp {

struct KrylovProblem {
    int nx, ny, nz;
    int nsm;                      // SMs of the device (grid of the streaming kernels)
    double dx, dy;
    // FP64 device tables of the plan
    const double* acoef;          // [nz+1] A[k] = rho_f[k]/dzn[k], A[0] = A[nz] = 0
    const double* svol;           // [nz]   rho_c[k] dz[k]
    const double* rflo;           // [nz]   rho_f[k]   (0 at k = 0)
    const double* rfhi;           // [nz]   rho_f[k+1] (0 at k = nz-1)
    const double* idzn;           // [nz+1] 1/dzn[k]
    // fields (FP32 when fp32, else FP64): u, v, phi [nz][ny][nx], w [nz+1][ny][nx]
    int fp32;
    const void* u; const void* v; const void* w;
    void* u_out; void* v_out; void* w_out; void* phi_out;           // phi_out may be null
    void* workspace;
    double tol;
    int max_iter;
    int precond;                  // 0: none, 1: vertical lines
};

struct KrylovResult {
    int iterations;
    double rel_residual;
    int status;                   // 0 converged, 1 iteration limit, 2 breakdown
};

size_t krylov_workspace_bytes(int nx, int ny, int nz, int nsm, bool fp32);

// Runs the whole solve on `st`, reading the residual back every few
// iterations (the calling thread waits on the stream).  Returns a cudaError_t.
cudaError_t krylov_run(const KrylovProblem& kp, cudaStream_t st, KrylovResult* res);

}  // namespace mp
