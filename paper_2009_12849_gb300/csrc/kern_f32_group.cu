// FP32 grouped-launch kernels of batched projections (group.cuh).
#include "group.cuh"
#include "pickers.h"

namespace mp {
#define MP_GROUP_CASE(N)                                                                  \
    case N: {                                                                              \
        const bool sq = square && nxp == GroupCols<N>::NXP && tw == GroupCols<N>::TW;      \
        switch (phase) {                                                                  \
            case 0: return k_fwd_rows_grp<N>;                                             \
            case 1: return sq ? k_fwd_cols_grp<N, true> : k_fwd_cols_grp<N>;              \
            case 3: return sq ? k_inv_cols_grp<N, true> : k_inv_cols_grp<N>;              \
            case 4: return k_inv_rows_grp<N>;                                             \
            default: return nullptr;                                                      \
        }                                                                                 \
    }
GroupFn pick_group_f32(int phase, int n, bool square, int nxp, int tw) {
    if (phase == 2) return k_tridiag_grp<float>;
    switch (n) {
        MP_F32_CT_CORE(MP_GROUP_CASE)
        default: return nullptr;
    }
}
#undef MP_GROUP_CASE
}  // namespace mp
