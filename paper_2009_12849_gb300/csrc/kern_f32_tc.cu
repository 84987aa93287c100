// Tensor-core split-precision forward column transforms (tcdft.cuh).
#include "pickers.h"
#include "tcdft.cuh"

namespace mp {
KernelFn pick_fwd_cols_tc(int ny, int fmt) {
    if (ny != 1024) return nullptr;
    return fmt == 1 ? k_fwd_cols_tc<1> : fmt == 2 ? k_fwd_cols_tc<2> : nullptr;
}
unsigned fwd_cols_tc_smem(int fmt) { return fmt == 1 ? TcLayout<1>::SMEM : TcLayout<2>::SMEM; }
}  // namespace mp
