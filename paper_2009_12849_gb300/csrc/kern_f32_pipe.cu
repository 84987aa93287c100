// FP32 persistent pipeline kernels of the transforms (pipe.cuh), for square
// grids of the compile-time lengths where the spectra outgrow L2.
#include "pickers.h"
#include "pipe.cuh"

namespace mp {
#define MP_PIPE_PICK(K)                                    \
    if (nx != ny) return nullptr;                          \
    switch (nx) {                                          \
        case 256: return ef ? K<256, 256, true> : K<256, 256, false>;     \
        case 512: return ef ? K<512, 512, true> : K<512, 512, false>;     \
        case 1024: return ef ? K<1024, 1024, true> : K<1024, 1024, false>; \
        default: return nullptr;                           \
    }
KernelFn pick_fwd_pipe(int nx, int ny, bool ef) { MP_PIPE_PICK(k_fwd_pipe) }
KernelFn pick_inv_pipe(int nx, int ny, bool ef) { MP_PIPE_PICK(k_inv_pipe) }
#undef MP_PIPE_PICK
}  // namespace mp
