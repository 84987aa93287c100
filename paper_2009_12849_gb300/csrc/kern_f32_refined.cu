// Kernels of the refinement passes: rows with FP32 transforms on FP64 fields
// (the divergence formed in FP64, the potential written in FP64) and the
// potential-only inverse column transform.  Compile-time plans for the core
// FP32 lengths, the run-time plan otherwise.
#include "pickers.h"

namespace mp {
KernelFn pick_refined_fwd_rows(int n) {
#define MP_REF_FWD(N) case N: return k_fwd_rows<float, N, double>;
    switch (n) {
        MP_F32_CT_CORE(MP_REF_FWD)
        default: return k_fwd_rows<float, 0, double>;
    }
#undef MP_REF_FWD
}
KernelFn pick_refined_inv_rows(int n) {
#define MP_REF_INV(N) case N: return k_inv_rows<float, N, double>;
    switch (n) {
        MP_F32_CT_CORE(MP_REF_INV)
        default: return k_inv_rows<float, 0, double>;
    }
#undef MP_REF_INV
}
KernelFn pick_refined_inv_cols(int n) {
#define MP_REF_COL(N) case N: return k_inv_cols<float, N, true>;
    switch (n) {
        MP_F32_CT_CORE(MP_REF_COL)
        default: return k_inv_cols<float, 0, true>;
    }
#undef MP_REF_COL
}
}  // namespace mp
