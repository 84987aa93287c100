// Hand-off of intermediate spectra through L2 (the persistent pipelines of
// pipe.cuh): a consumer discards (discard.global.L2) every 128-byte line of an
// intermediate it has finished reading, so lines still in L2 are never
// written back to DRAM; streaming fields can be loaded and stored with an
// evict-first L2 policy so that they do not push the intermediates out.
#pragma once
#include <cuda_runtime.h>

namespace mp {

// Invalidate one 128-byte L2 line without writing it back (its contents
// become undefined).  `a` must be 128-byte aligned.
__device__ __forceinline__ void l2_discard(const void* a) {
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(a) : "memory");
}

// L2 policy with evict-first priority, for data that streams through once.
__device__ __forceinline__ unsigned long long l2_evict_first() {
    unsigned long long pol;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ float ld_ef(const float* a, unsigned long long pol) {
    float v;
    asm volatile("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ float4 ld_ef(const float4* a, unsigned long long pol) {
    float4 v;
    asm volatile("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ void st_ef(float* a, float v, unsigned long long pol) {
    asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(a), "f"(v), "l"(pol) : "memory");
}

// Hand-off parameters of a launch (zero-initialised: no discards).
struct HandoffArgs {
    int discard;              // 1: consumers discard the intermediate lines they have read
    unsigned* groups;         // per (level, line group) counts of forward column tiles done reading
};

}  // namespace mp
