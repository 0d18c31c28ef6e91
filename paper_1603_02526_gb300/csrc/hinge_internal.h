// hinge_internal.h -- the hinge-bank sweep: descriptors shared by the host
// planner (fga_hinge.cpp) and the kernel (sweep_hinge.cu).  Not part of
// the public C-ABI.
//
// A graph qualifies when it is a linear soft-margin SVM written as a factor
// graph (Sec. V-C): hinge factors c max(0, 1 - y (w.x + b)) that all share
// one (w, b), plus L2 factors (lambda/2)|w|^2 on that w, in FP32 with one
// rho, alpha = 1 and m not kept, with dim(w) <= 64 and few enough points
// that each CTA's slice of the data fits in shared memory.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "fga_internal.h"
#include "tile_internal.h"

namespace fga {

constexpr int kHingeD = 64;          // data row length in the kernel (rows padded with zeros)
constexpr int kHingeWarps = 16;      // warps per CTA
constexpr int kHingeGroups = 4 * kHingeWarps;   // groups of 8 lanes, one hinge factor at a time each
constexpr int kHingeK = 16;          // hinge factors per group, at most
constexpr int kHingeMaxL2 = 4;       // L2 factors, at most
constexpr int kHingeAccStride = 16;  // one accumulator per 128-byte line

// Per CTA: its hinge factors [f0, f0 + nf).
struct HingeCta {
    int f0, nf;
};

struct HingeArgs {
    int G, N, D;                     // CTAs, hinge factors, dim(w)
    int nl2;                         // L2 factors
    const HingeCta *cta;
    const float *X;                  // [N][64] data rows, zero-padded
    const float4 *meta;              // per hinge factor: y, c, |x|^2 + 1, rho / (|x|^2 + 1)
    float lam[kHingeMaxL2];          // per L2 factor: lambda
    float rho, inv_rho;
    int deg_w, deg_b;                // number of edges of a w component, of b
    int rows_max;                    // hinge factors of the largest CTA (shared-memory layout)
    float *u;                        // per edge (storage order)
    float *xout;                     // x buffer written at checks and at the end
    const float *zin;                // z at the start of the call (w then b, scalar ids v0..v0+D)
    float *zout;                     // z written at checks and at the end
    const float *zpin;               // z before the stored state (resume)
    float *zpout;                    // written at checks with the state
    int vw, vb;                      // scalar ids of w_0 and of b
    int hb_e0;                       // storage of hinge factor f, edge j: hb_e0 + f (D + 1) + j
    int l2_e0, l2_nf;                // storage of L2 factor f, edge j: l2_e0 + j l2_nf + f
    unsigned long long *acc;         // [2][(D + 1) * kHingeAccStride] count-and-sum words by pass
                                     // parity (see kTileCountUnit), zeroed before a launch
    float *gsave;                    // [2][N] g kept for the next check (by pass parity)
    float *gres;                     // [N] g of the stored state
    float *l2save, *l2res;           // [nl2][64] the same for the L2 factors
    int resume;
    double *res;                     // [2][2][G]
    long long E;
    Ctl *ctl;
    TileSync *sync;
    long long k0, K;
    int check_every;
    double tol_pri, tol_dual;
    long long timeout_ns;
    int skip_block;
    int xw, zw;
};

struct HingeInput {
    int64_t N = 0;
    int D = 0;
    int vw = -1, vb = -1;            // scalar ids
    std::vector<float> X;            // N x D
    std::vector<float> yl, cl;       // per factor
    std::vector<float> lam;          // per L2 factor
    double rho = 1.0;
    int sms = 0;
    int smem_optin = 0;
};

struct HingePlan {
    int G = 0;
    int rows_max = 0;                // hinge factors of the largest CTA
    std::vector<HingeCta> cta;
    std::vector<float> X;            // N x 64
    std::vector<float4> meta;
};

// 0: planned; 1: the graph does not qualify (reason in `why`).
int hinge_plan(const HingeInput &in, HingePlan &P, std::string &why);
int hinge_smem_bytes(int rows_max);

cudaError_t hinge_sweep_launch(const HingeArgs &a, int smem, cudaStream_t s);
// The latency floor of a pass on the same grid (mode 0: barrier; 1: the
// count-and-sum exchange), `iters` passes.
cudaError_t hinge_floor_launch(const HingeArgs &a, long long iters, int mode, cudaStream_t s);

}  // namespace fga
