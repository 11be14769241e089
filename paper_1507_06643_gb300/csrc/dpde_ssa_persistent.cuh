// dpde_ssa_persistent.cuh -- the colour-class SSA sequence (Sec. III.A.2,
// III.B.2) as one persistent, cooperative launch: every block of a grid
// sized to full co-residency takes its share of the cells of a class (a
// thread per cell chain, as the per-class launches do), then all blocks meet
// at a grid barrier before the next class. The barrier's wait is bounded:
// after `budget` clock cycles a waiting block raises ST_TIMEOUT and leaves,
// and every block then leaves at its next barrier, so a launch whose blocks
// cannot meet (a budget too small, a block that never arrives) ends with a
// status the host reads instead of hanging.
#pragma once

#include "dpde_kernels.cuh"

namespace dpde {

// Grid barrier state: arrivals of the current round, then the round counter.
// Cleared before every launch.
struct GridBarrier {
    unsigned int count;
    unsigned int round;
};

// All blocks of the launch meet here. Returns false, with ST_TIMEOUT raised,
// when this block gave up waiting after `budget` clock cycles (or the
// equivalent number of polls).
__device__ __forceinline__ bool grid_barrier(GridBarrier* bar, unsigned int nblocks, long long budget,
                                             unsigned int* status) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned int* vround = &bar->round;
        const unsigned int round = *vround;
        __threadfence();
        if (atomicAdd(&bar->count, 1u) + 1u == nblocks) {
            bar->count = 0u;
            __threadfence();
            atomicAdd(&bar->round, 1u);
        } else {
            const long long t0 = clock64();
            const long long max_polls = budget / 64 + 1024;
            for (long long it = 0; *vround == round; ++it) {
                if (clock64() - t0 >= budget || it >= max_polls) {
                    ok = 0;
                    flag(status, ST_TIMEOUT);
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// The classes of the colour order in sequence: class k holds the cells
// cells[off[k] .. off[k + 1]). A block stops at the first barrier it gave up
// on; the others then give up at their next one.
template <class T>
__global__ void __launch_bounds__(SSA_THREADS_MAX) k_ssa_persistent(Ctx<T> C, const int* __restrict__ cells,
                                                                    const int* __restrict__ off, T dt, T sqrt_dt,
                                                                    GridBarrier* bar, long long budget) {
    extern __shared__ int ssa_rows[];
    const int bdim = blockDim.x;
    const int tid = threadIdx.x;
    const int stride = gridDim.x * bdim;
    bool first = true;
    for (int k = 0; k < NCOLOURS; ++k) {
        const int k0 = __ldg(off + k), n = __ldg(off + k + 1) - k0;
        if (n == 0) continue;   // uniform over the grid
        if (!first && !grid_barrier(bar, gridDim.x, budget, C.status)) return;
        first = false;
        for (int u = blockIdx.x * bdim + tid; u < n; u += stride)
            ssa_cell_chain(C, __ldg(cells + k0 + u), dt, sqrt_dt, ssa_rows, ssa_rows + SSA_ROWS * bdim, bdim, tid);
    }
}

}  // namespace dpde
