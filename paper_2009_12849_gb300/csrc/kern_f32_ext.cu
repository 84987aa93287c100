// FP32 row or column kernels of one group of the extended compile-time
// lengths.  Compiled once per group and part:
//   -DMP_EXT_GROUP=1..4 -DMP_EXT_PART=0 (rows) or 1 (columns)
#include "pickers.h"

#if !defined(MP_EXT_GROUP) || !defined(MP_EXT_PART)
#error "compile with -DMP_EXT_GROUP=<1..4> -DMP_EXT_PART=<0|1>"
#endif

#if MP_EXT_GROUP == 1
#define MP_EXT_LIST MP_F32_CT_EXT1
#elif MP_EXT_GROUP == 2
#define MP_EXT_LIST MP_F32_CT_EXT2
#elif MP_EXT_GROUP == 3
#define MP_EXT_LIST MP_F32_CT_EXT3
#else
#define MP_EXT_LIST MP_F32_CT_EXT4
#endif

#define MP_EXT_NAME2(G, P) pick_f32_ext_##G##_##P
#define MP_EXT_NAME(G, P) MP_EXT_NAME2(G, P)

namespace mp {
KernelFn MP_EXT_NAME(MP_EXT_GROUP, MP_EXT_PART)(KernelKind kind, int n) {
#if MP_EXT_PART == 0
#define MP_CASE_A(N) case N: return k_fwd_rows<float, N>;
#define MP_CASE_B(N) case N: return k_inv_rows<float, N>;
    const KernelKind ka = kFwdRows, kb = kInvRows;
#else
#define MP_CASE_A(N) case N: return k_fwd_cols<float, N>;
#define MP_CASE_B(N) case N: return k_inv_cols<float, N>;
    const KernelKind ka = kFwdCols, kb = kInvCols;
#endif
    if (kind == ka) {
        switch (n) { MP_EXT_LIST(MP_CASE_A) default: return nullptr; }
    }
    if (kind == kb) {
        switch (n) { MP_EXT_LIST(MP_CASE_B) default: return nullptr; }
    }
    return nullptr;
}
}  // namespace mp
