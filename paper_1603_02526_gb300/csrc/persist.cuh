// persist.cuh -- pieces shared by the persistent packing and SVM kernels:
// the grid-wide barrier with a time limit and the fire-and-forget integer
// addition used by the fixed-point accumulators.
#pragma once

#include <cuda_runtime.h>

#include "sweep.cuh"
#include "tile_internal.h"

namespace fga {

// What one pass over a unit does:
//  T_FIRST: the first iteration of a call (n from the stored u);
//  T_MID:   one iteration;
//  T_CHK:   one iteration, preceded by the residual and the stored state of
//           the previous iteration;
//  T_FINAL: only the residual and the stored state of the last iteration.
enum TileMode : int { T_FIRST = 0, T_MID = 1, T_CHK = 2, T_FINAL = 3 };

// One pass: its mode; RELOAD: the previous pass was the call's first (a
// check reads the stored u again); SAVE: the next pass checks (keep the
// displacements this pass replaces).  The pass functions are compiled
// twice: GEN = false for the plain pass (T_MID, neither flag, all folded at
// compile time, the code of every iteration) and GEN = true for the others,
// which test the fields at run time -- one copy of the rarely run code
// rather than one per combination keeps the kernel's instructions few.
struct PassMode {
    int mode;
    bool reload, save;
    long long it;   // the pass number within the call
};

// ---------------------------------------------------------------------------
// grid barrier: one counter that only grows; CTA b waits until it reaches
// G x (iterations so far).  Bounded by timeout_ns and a spin count; on
// expiry the CTA sets the error word and every CTA leaves.
// ---------------------------------------------------------------------------
// (the 64-bit release addition, relaxed addition and relaxed / acquire
// loads are in sweep.cuh)

// Count of contributions in the difference of two count-and-sum words
// (kTileCountUnit per contribution, the sum in the low bits).
static __device__ __forceinline__ unsigned tile_count(unsigned long long diff) {
    return (unsigned)(((diff + (1ull << 55)) >> 56) & 0xffull);
}

// The CTA's writes before the barrier are ordered by bar.sync and the
// cumulative release of the arrival; the waiting thread polls with relaxed
// loads and takes one acquire load once the count is reached, which orders
// the CTA's later reads (through bar.sync) after every CTA's writes.
static __device__ __forceinline__ bool tile_barrier(TileSync *s, unsigned long long target, long long timeout_ns,
                                                    bool skip) {
    __shared__ int s_err;
    __syncthreads();
    if (threadIdx.x == 0) {
        int err = 0;
        if (!skip) red_release_add_u64(&s->count, 1ull);
        if (ld_relaxed_u64(&s->count) < target) {
            const unsigned long long t0 = global_ns();
            unsigned int spins = 0;
            while (ld_relaxed_u64(&s->count) < target) {
                ++spins;
                if ((spins & 63u) == 0u) {
                    if (*(volatile int *)&s->error) { err = 1; break; }
                    if (global_ns() - t0 > (unsigned long long)timeout_ns || spins > (1u << 30)) {
                        atomicExch(&s->error, kETimeout);
                        err = 1;
                        break;
                    }
                }
            }
        }
        (void)ld_acquire_u64(&s->count);
        if (!err && *(volatile int *)&s->error) err = 1;
        s_err = err;
    }
    __syncthreads();
    return s_err == 0;
}

}  // namespace fga
