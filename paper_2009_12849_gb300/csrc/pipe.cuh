// Persistent pipelines of the two transforms (steps a1-a2 and a4-a5 of the
// projection; paper, Section 4: a forward FFT on every level, a backward FFT).
//
// Each transform is two passes over a level: forward, the divergence and the
// real transforms of the rows (P) and the column transforms of the x-spectra
// (C); inverse, the column transforms of p^ and gz^ into the three gradient
// channels (P) and the row transforms with the correction of u, v, w (C).  A
// pipeline kernel runs both passes: its blocks take tasks by ticket in the
// order
//   P(0) .. P(L-1), P(L), C(0), P(L+1), C(1), ..., C(nz-1)      (lag L levels)
// where P(k) and C(k) are all the tasks of one pass over level k.  A C(k)
// task waits until every P(k) task is done (a per-level counter).  Tickets
// are taken only by running blocks and a task only waits for tasks with
// smaller tickets, so the schedule cannot deadlock whatever the residency.
//
// Why: the row passes are bound by DRAM, the column passes by arithmetic and
// shared memory, and one kernel per pass runs them one after the other.
// Here the blocks of an SM are at different points of the ticket order, so a
// row task's loads overlap a column task's arithmetic.  And the intermediate
// spectra of a level are read back a few levels after they were written,
// while still in L2; the reader discards each line once it is done with it
// (discard.global.L2), so the hand-off between the passes costs no DRAM bytes.
//
// EF: u, v, w stream through L2 with evict-first priority.
//
// Blocks are 256 threads.  A column task is one tile of 256*32/N columns,
// transformed by the whole block; a P task of the forward pipeline and a C
// task of the inverse are eight independent warps, each transforming its own
// row pair (two real rows in one complex transform) in its own slice of
// shared memory.  Every wait is bounded: past p.spin_limit polls the block
// latches bit 0 of the plan's error word (reported as a timeout) and goes on.
#pragma once
#include "kernels.cuh"

namespace mp {

constexpr int kPipeThreads = 256;
constexpr int kPipeWarps = kPipeThreads / 32;

// Sequences (complex transforms) per warp task and real rows per warp task
// for rows of length NX (a warp holds 32 * E elements of a stage).
template <int NX> struct PipeRows {
    static constexpr int E = ElemsPerThread<float>::value;
    static constexpr int kPairs = (32 * E / NX) < 1 ? 1 : (32 * E / NX);
    static constexpr int kRows = 2 * kPairs;
};

// Column tiles of the pipelines: the plan pads spectral rows to whole 128-byte
// lines and the 256-thread tiles hold 256 * 32 / NY columns, so the pitch and
// tile width are compile-time constants of (NX, NY).
template <int NX, int NY> struct PipeCols {
    static constexpr int NXP = ((NX / 2 + 1) + 15) & ~15;
    static constexpr int TW = kPipeThreads * ElemsPerThread<float>::value / NY;
};

// The block waits until *ctr >= target (acquire by thread 0, then a barrier),
// for at most `limit` polls after the first.
__device__ __forceinline__ void pipe_wait(const unsigned* ctr, unsigned target, int* err, long long limit) {
    if (threadIdx.x == 0) {
        long long spins = 0;
        while (true) {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
            if (v >= target) break;
            if (++spins > limit) {
                atomicOr(err, 1);
                break;
            }
            __nanosleep(32);
        }
    }
    __syncthreads();
}

// Every thread's writes of this task are made visible, then the task counts
// itself done.
__device__ __forceinline__ void pipe_signal(unsigned* ctr) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(ctr, 1u);
}

// Ticket t of the lagged order: true for a P task; *k its level, *idx its
// index within the level (a P tasks and b C tasks per level, lag L levels).
__device__ __forceinline__ bool pipe_decode(int t, int nz, int L, int a, int b, int* k, int* idx) {
    if (t < L * a) {
        *k = t / a;
        *idx = t - *k * a;
        return true;
    }
    const int t1 = t - L * a;
    const int g1 = nz - L;                    // levels whose group holds P(g + L) and C(g)
    if (t1 < g1 * (a + b)) {
        const int g = t1 / (a + b);
        const int r = t1 - g * (a + b);
        if (r < a) { *k = g + L; *idx = r; return true; }
        *k = g;
        *idx = r - a;
        return false;
    }
    const int t2 = t1 - g1 * (a + b);
    *k = g1 + t2 / b;
    *idx = t2 - (t2 / b) * b;
    return false;
}

// The next ticket, taken by thread 0 at the start of a task and handed to the
// block at its end (the atomic's latency hides behind the task).
struct PipeTicket {
    unsigned* ctr;
    unsigned next;
    __device__ __forceinline__ void take() {
        if (threadIdx.x == 0) next = atomicAdd(ctr, 1u);
    }
    __device__ __forceinline__ int hand(int* s_slot) {
        if (threadIdx.x == 0) *s_slot = (int)next;
        __syncthreads();
        const int t = *s_slot;
        __syncthreads();
        return t;
    }
};

// Forward pipeline: P = divergence + x transforms of row pairs (warps), C =
// y transforms of column tiles (the block).  p.sync: [0] ticket, [2 + k] the
// row tasks of level k done.
template <int NX, int NY, bool EF>
__global__ void __launch_bounds__(kPipeThreads, 2) k_fwd_pipe(ProjParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_ticket;
    using RW = PipeRows<NX>;
    const int nz = p.nz;
    const int nwt = (p.ny + RW::kRows - 1) / RW::kRows;            // warp tasks per level
    const int a = (nwt + kPipeWarps - 1) / kPipeWarps;             // P block tasks per level
    const int b = p.ntiles;                                         // C tasks per level
    const int L = min(p.lag, nz);
    const int total = nz * (a + b);
    unsigned* done = p.sync + 2;
    const int warp = threadIdx.x >> 5;
    unsigned char* wslice = smem_raw + (size_t)warp * RW::kPairs * p.bs_row * sizeof(float2);
    PipeTicket tk{p.sync, 0u};
    tk.take();
    int t = tk.hand(&s_ticket);
    while (t < total) {
        tk.take();
        int k, idx;
        if (pipe_decode(t, nz, L, a, b, &k, &idx)) {
            const int wt = idx * kPipeWarps + warp;
            if (wt < nwt) fwd_rows_task<float, NX, float, EF, WarpScope>(p, wslice, k, wt * RW::kRows, RW::kRows);
            pipe_signal(&done[k]);
        } else {
            pipe_wait(&done[k], (unsigned)a, p.err, p.spin_limit);
            fwd_cols_task<float, NY, PipeCols<NX, NY>::NXP, PipeCols<NX, NY>::TW>(p, smem_raw, k, idx);
        }
        t = tk.hand(&s_ticket);
    }
}

// Inverse pipeline: P = y transforms of p^ / gz^ column tiles (the block), C =
// x transforms of (row pair, channel) warp tasks with the correction.
// p.sync: [1] ticket, [2 + nz + k] the column tasks of level k done.
template <int NX, int NY, bool EF>
__global__ void __launch_bounds__(kPipeThreads, 2) k_inv_pipe(ProjParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_ticket;
    using RW = PipeRows<NX>;
    const int nz = p.nz;
    const int nch = p.nch;
    constexpr int BROWS = RW::kRows * kPipeWarps;                   // rows of a C task (the block's transforms)
    const int nrb = (p.ny + BROWS - 1) / BROWS;
    const int a = 2 * p.ntiles;                                     // P tasks per level
    const int b = nrb * nch;                                        // C block tasks per level
    const int L = min(p.lag, nz);
    const int total = nz * (a + b);
    unsigned* done = p.sync + 2 + nz;
    const int warp = threadIdx.x >> 5;
    unsigned char* wslice = smem_raw + (size_t)warp * RW::kPairs * p.bs_row * sizeof(float2);
    PipeTicket tk{p.sync + 1, 0u};
    tk.take();
    int t = tk.hand(&s_ticket);
    while (t < total) {
        tk.take();
        int k, idx;
        if (pipe_decode(t, nz, L, a, b, &k, &idx)) {
            using PC = PipeCols<NX, NY>;
            inv_cols_tile<float, NY, false, PC::NXP, PC::TW>(p, smem_raw, k, (idx >> 1) * PC::TW, idx & 1);
            pipe_signal(&done[k]);
        } else {
            pipe_wait(&done[k], (unsigned)a, p.err, p.spin_limit);
            inv_rows_ct<float, NX, float, EF, BlockScope>(p, smem_raw, k, (idx / nch) * BROWS, idx % nch, BROWS);
        }
        t = tk.hand(&s_ticket);
    }
}

}  // namespace mp
