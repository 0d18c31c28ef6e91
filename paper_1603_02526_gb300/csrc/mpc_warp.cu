// mpc_warp.cu -- batched ragged MPC with one lane per time step (FP32, 12
// states and 4 inputs: the workload's sizes).
//
// The same solver as k_mpc_batch (Algorithm 2 on the factor graph
// FIX(x_0) | DYN_t | QUAD_t | QUAD_T | BOX_t of Appendix B, the same
// operations in the same order on every value), laid out differently: lane
// t of an instance owns time step t -- the x and u of its dynamics factor's
// 28 edges, the u of its stage cost's 16 edges and of its box's 4 edges, in
// registers for the whole solve -- and z of x_t and u_t.  An iteration is
// then, per lane, one 28 x 28 product with the projector (read from shared
// memory, the same address in every lane: a broadcast), the elementwise
// operators, the z-update of its 16 variables and the u-update of its
// edges; neighbouring steps exchange 12 values three times per iteration
// (the x_{t+1} z values and the dynamics factor's x_{t+1} messages).
// Instances of up to 32 steps take one warp (two instances per 64-thread
// CTA, independent of each other); instances of 33 to 64 steps take both
// warps, which exchange their boundary values through shared memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "mpc_internal.h"
#include "residual.cuh"

namespace fga {

namespace {

constexpr int WX = 12, WU = 4, WS = 16, WA = 28;
constexpr int kWarpCta = kMpcWarpThreads;
constexpr unsigned FULL = 0xffffffffu;

// Per instance slot in shared memory (one per warp): projector, the
// rho / (w + rho) factors of the 16 cost components, x_0, and the values of
// the edges only the first or the last step has (FIX: u; QUAD_T: u; z of
// x_T), exchange slots for a two-warp instance, residual sums.
struct WarpInst {
    float P[WA * WA];
    float cw[WS];
    float x0[WX];
    float uf[WX];      // FIX edges' u (step 0)
    float uqT[WX];     // terminal cost edges' u (step T - 1)
    float zT[WX];      // z of x_T (step T - 1)
    float xq[2][WX];   // boundary exchange of a two-warp instance
    float red[8];
    int flag[4];
};

// Value of lane + 1 / lane - 1 of a step-owned array, across the two warps
// of a long instance through shared memory (xch: this instance's exchange
// slots; `two`: the instance spans both warps).
template <int N>
__device__ __forceinline__ void from_next(const float (&v)[N], float (&o)[N], bool two, int w, float *xch) {
    const int lane = threadIdx.x & 31;
    #pragma unroll
    for (int c = 0; c < N; ++c) o[c] = __shfl_down_sync(FULL, v[c], 1);
    if (two) {
        // lane 0 of warp 1 hands its values to lane 31 of warp 0
        if (w == 1 && lane == 0) {
            #pragma unroll
            for (int c = 0; c < N; ++c) xch[c] = v[c];
        }
        __syncthreads();
        if (w == 0 && lane == 31) {
            #pragma unroll
            for (int c = 0; c < N; ++c) o[c] = xch[c];
        }
        __syncthreads();
    }
}

template <int N>
__device__ __forceinline__ void from_prev(const float (&v)[N], float (&o)[N], bool two, int w, float *xch) {
    const int lane = threadIdx.x & 31;
    #pragma unroll
    for (int c = 0; c < N; ++c) o[c] = __shfl_up_sync(FULL, v[c], 1);
    if (two) {
        if (w == 0 && lane == 31) {
            #pragma unroll
            for (int c = 0; c < N; ++c) xch[c] = v[c];
        }
        __syncthreads();
        if (w == 1 && lane == 0) {
            #pragma unroll
            for (int c = 0; c < N; ++c) o[c] = xch[c];
        }
        __syncthreads();
    }
}

}  // namespace

// Work items: inst[0], inst[1] two instances of at most 32 steps (inst[1] =
// -1: none), or inst[1] = -2: inst[0] is one instance of 33..64 steps.
__global__ void __launch_bounds__(kWarpCta) k_mpc_warp(const MpcArgs<float> a, const int2 *items, int n_items) {
    __shared__ WarpInst sh[2];
    __shared__ int s_item[2];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned k = atomicAdd(a.queue, 1u);
            const int2 it = k < (unsigned)n_items ? items[k] : make_int2(-1, -1);
            s_item[0] = it.x;
            s_item[1] = it.y;
        }
        __syncthreads();
        const int i0 = s_item[0], i1 = s_item[1];
        if (i0 < 0) return;
        const bool two = i1 == -2;
        const int inst = two ? i0 : (w == 0 ? i0 : i1);
        WarpInst &S = sh[two ? 0 : w];
        const int T = inst >= 0 ? a.T[inst] : 0;
        const int t = two ? (w * 32 + lane) : lane;   // this lane's step
        const bool act = t < T;
        const bool first = t == 0, last = t == T - 1;
        const long long eo = inst >= 0 ? a.eoff[inst] : 0, zof = inst >= 0 ? a.zoff[inst] : 0;
        // shared tables (both warps of a two-warp instance fill one slot)
        if (inst >= 0) {
            const int sy = a.sys[inst];
            const int base = two ? (int)threadIdx.x : lane, stride = two ? kWarpCta : 32;
            for (int j = base; j < WA * WA; j += stride) S.P[j] = a.P[(long long)sy * WA * WA + j];
            for (int j = base; j < WS; j += stride) {
                const float wt = j < WX ? a.q[sy * WX + j] : a.r[sy * WU + j - WX];
                S.cw[j] = a.rho / (wt + a.rho);
            }
            for (int j = base; j < WX; j += stride) {
                S.x0[j] = a.x0[(long long)inst * WX + j];
                S.uf[j] = a.u[eo + j];
                S.uqT[j] = a.u[eo + WX + (long long)WA * T + (long long)WS * T + j];
                S.zT[j] = a.z[zof + (long long)WS * T + j];
            }
        }
        // this step's registers
        float xd[WA], ud[WA], uq[WS], ub[WU], zx[WX], zu[WU];
        const long long ed = eo + WX + (long long)WA * t, eq = eo + WX + (long long)WA * T + (long long)WS * t;
        const long long eb = eo + 2 * WX + (long long)(WA + WS) * T + (long long)WU * t;
        #pragma unroll
        for (int k = 0; k < WA; ++k) {
            xd[k] = act ? a.x[ed + k] : 0.f;
            ud[k] = act ? a.u[ed + k] : 0.f;
        }
        #pragma unroll
        for (int k = 0; k < WS; ++k) uq[k] = act ? a.u[eq + k] : 0.f;
        #pragma unroll
        for (int k = 0; k < WU; ++k) ub[k] = act ? a.u[eb + k] : 0.f;
        #pragma unroll
        for (int c = 0; c < WX; ++c) zx[c] = act ? a.z[zof + (long long)WS * t + c] : 0.f;
        #pragma unroll
        for (int j = 0; j < WU; ++j) zu[j] = act ? a.z[zof + (long long)WS * t + WX + j] : 0.f;
        __syncthreads();

        const float rho = a.rho, alpha = a.alpha, lo = a.lo, hi = a.hi;
        ResidualTest rtp, rtd;
        const double Einst = (double)(2 * WX + 3 * WS * T);
        rtp.init(Einst, a.tol_pri);
        rtd.init(Einst, a.tol_dual);
        long long done = 0;
        int status = 0;
        double rp = nan(""), rd = nan("");
        const long long K = a.max_iters;
        const int ce = a.check_every;
        int rm = 1 % ce;
        float zxn[WX];   // z of x_{t+1}
        for (long long it = 1; it <= K && inst >= 0; ++it) {
            // ---- X: the dynamics factor, x = P n (n = z - u of the previous iteration)
            from_next<WX>(zx, zxn, two, w, S.xq[0]);
            if (last) {
                #pragma unroll
                for (int c = 0; c < WX; ++c) zxn[c] = S.zT[c];
            }
            // n in pairs (the packed FP32 multiply-add takes two lanes of
            // values per instruction; each lane rounds as a single fma)
            float2 nd[WA / 2];
            #pragma unroll
            for (int c = 0; c < WX; c += 2) nd[c / 2] = make_float2(zx[c] - ud[c], zx[c + 1] - ud[c + 1]);
            #pragma unroll
            for (int j = 0; j < WU; j += 2)
                nd[(WX + j) / 2] = make_float2(zu[j] - ud[WX + j], zu[j + 1] - ud[WX + j + 1]);
            #pragma unroll
            for (int c = 0; c < WX; c += 2)
                nd[(WS + c) / 2] = make_float2(zxn[c] - ud[WS + c], zxn[c + 1] - ud[WS + c + 1]);
            #pragma unroll
            for (int i = 0; i < WA; ++i) {
                const float4 *Pr = reinterpret_cast<const float4 *>(S.P + i * WA);
                float2 s01 = make_float2(0.f, 0.f), s23 = make_float2(0.f, 0.f);
                #pragma unroll
                for (int j = 0; j < WA / 4; ++j) {
                    const float4 p = Pr[j];
                    s01 = __ffma2_rn(make_float2(p.x, p.y), nd[2 * j], s01);
                    s23 = __ffma2_rn(make_float2(p.z, p.w), nd[2 * j + 1], s23);
                }
                xd[i] = (s01.x + s01.y) + (s23.x + s23.y);
            }
            // ---- elementwise operators and the z-update of x_t, u_t (and x_T)
            float mp[WX], mx[WX];
            #pragma unroll
            for (int c = 0; c < WX; ++c) mx[c] = xd[WS + c] + ud[WS + c];   // DYN_t's x_{t+1} messages
            from_prev<WX>(mx, mp, two, w, S.xq[1]);
            const bool chk = rm == 0 || it == K;
            float pri = 0.f, dual = 0.f, pl = 0.f, dl = 0.f;
            float xq[WS], xb[WU], zxo[WX], zuo[WU];
            #pragma unroll
            for (int c = 0; c < WX; ++c) {
                xq[c] = S.cw[c] * (zx[c] - uq[c]);
                const float m0 = first ? S.x0[c] + S.uf[c] : mp[c];
                const float S3 = (m0 + (xd[c] + ud[c])) + (xq[c] + uq[c]);
                zxo[c] = zx[c];
                zx[c] = S3 * (1.f / 3.f);
            }
            #pragma unroll
            for (int j = 0; j < WU; ++j) {
                xq[WX + j] = S.cw[WX + j] * (zu[j] - uq[WX + j]);
                float v = zu[j] - ub[j];
                if (v < lo) v = lo;
                if (v > hi) v = hi;
                xb[j] = v;
                const float S3 = ((xd[WX + j] + ud[WX + j]) + (xq[WX + j] + uq[WX + j])) + (xb[j] + ub[j]);
                zuo[j] = zu[j];
                zu[j] = S3 * (1.f / 3.f);
            }
            float xqT[WX], zTo[WX];
            if (last) {
                #pragma unroll
                for (int c = 0; c < WX; ++c) {
                    xqT[c] = S.cw[c] * (S.zT[c] - S.uqT[c]);
                    zTo[c] = S.zT[c];
                    S.zT[c] = (mx[c] + (xqT[c] + S.uqT[c])) * 0.5f;
                }
            }
            // z of x_{t+1} after the update, for the dynamics factor's last 12 edges
            from_next<WX>(zx, zxn, two, w, S.xq[0]);
            if (last) {
                #pragma unroll
                for (int c = 0; c < WX; ++c) zxn[c] = S.zT[c];
            }
            // ---- u-update on every edge of the step (and FIX / QUAD_T)
            if (act) {
                #pragma unroll
                for (int c = 0; c < WX; ++c) {
                    const float d0 = xd[c] - zx[c], d1 = xq[c] - zx[c], d2 = xd[WS + c] - zxn[c];
                    ud[c] = __fmaf_rn(alpha, d0, ud[c]);
                    uq[c] = __fmaf_rn(alpha, d1, uq[c]);
                    ud[WS + c] = __fmaf_rn(alpha, d2, ud[WS + c]);
                    if (chk) {
                        pri += d0 * d0 + d1 * d1 + d2 * d2;
                        const float dz = zx[c] - zxo[c];
                        dual += 3.f * rho * rho * dz * dz;
                    }
                }
                #pragma unroll
                for (int j = 0; j < WU; ++j) {
                    const float d0 = xd[WX + j] - zu[j], d1 = xq[WX + j] - zu[j], d2 = xb[j] - zu[j];
                    ud[WX + j] = __fmaf_rn(alpha, d0, ud[WX + j]);
                    uq[WX + j] = __fmaf_rn(alpha, d1, uq[WX + j]);
                    ub[j] = __fmaf_rn(alpha, d2, ub[j]);
                    if (chk) {
                        pri += d0 * d0 + d1 * d1 + d2 * d2;
                        const float dz = zu[j] - zuo[j];
                        dual += 3.f * rho * rho * dz * dz;
                    }
                }
                if (first) {
                    #pragma unroll
                    for (int c = 0; c < WX; ++c) {
                        const float d = S.x0[c] - zx[c];
                        S.uf[c] = __fmaf_rn(alpha, d, S.uf[c]);
                        if (chk) pri += d * d;
                    }
                }
                if (last) {
                    #pragma unroll
                    for (int c = 0; c < WX; ++c) {
                        const float d = xqT[c] - S.zT[c];
                        S.uqT[c] = __fmaf_rn(alpha, d, S.uqT[c]);
                        if (chk) {
                            pri += d * d;
                            const float dz = S.zT[c] - zTo[c];
                            dual += 2.f * rho * rho * dz * dz;
                        }
                    }
                }
            }
            rm = rm + 1 == ce ? 0 : rm + 1;
            if (chk) {
                // the elementwise edges' x of this iteration (the stored state
                // if the check stops)
                if (act) {
                    #pragma unroll
                    for (int k = 0; k < WS; ++k) a.x[eq + k] = xq[k];
                    #pragma unroll
                    for (int k = 0; k < WU; ++k) a.x[eb + k] = xb[k];
                    if (first) {
                        #pragma unroll
                        for (int c = 0; c < WX; ++c) a.x[eo + c] = S.x0[c];
                    }
                    if (last) {
                        #pragma unroll
                        for (int c = 0; c < WX; ++c) a.x[eo + WX + (long long)WA * T + (long long)WS * T + c] = xqT[c];
                    }
                }
                // residual sums of the instance: float pairs over the lanes
                // (and the two warps in order), the decision by lane 0
                warp_sum2_ff(pri, pl, dual, dl);
                if (two) {
                    if (lane == 0) {
                        S.red[4 * w] = pri;
                        S.red[4 * w + 1] = pl;
                        S.red[4 * w + 2] = dual;
                        S.red[4 * w + 3] = dl;
                    }
                    __syncthreads();
                    pri = S.red[0];
                    pl = S.red[1];
                    dual = S.red[2];
                    dl = S.red[3];
                    ff_add(pri, pl, S.red[4], S.red[5]);
                    ff_add(dual, dl, S.red[6], S.red[7]);
                    __syncthreads();
                }
                const bool finite = isfinite(pri) && isfinite(dual);
                const bool conv = finite && rtp.pass(pri, pl) && rtd.pass(dual, dl);
                if (!finite || conv || it == K) {
                    done = it;
                    status = !finite ? -6 : (conv || (a.tol_pri <= 0.0 && a.tol_dual <= 0.0)) ? 0 : -7;
                    rp = sqrt(((double)pri + (double)pl) / Einst);
                    rd = sqrt(((double)dual + (double)dl) / Einst);
                    break;
                }
            }
        }
        // store the state of the instance
        if (inst >= 0) {
            if (act) {
                #pragma unroll
                for (int k = 0; k < WA; ++k) {
                    a.x[ed + k] = xd[k];
                    a.u[ed + k] = ud[k];
                }
                #pragma unroll
                for (int k = 0; k < WS; ++k) a.u[eq + k] = uq[k];
                #pragma unroll
                for (int k = 0; k < WU; ++k) a.u[eb + k] = ub[k];
                #pragma unroll
                for (int c = 0; c < WX; ++c) a.z[zof + (long long)WS * t + c] = zx[c];
                #pragma unroll
                for (int j = 0; j < WU; ++j) a.z[zof + (long long)WS * t + WX + j] = zu[j];
                if (first) {
                    #pragma unroll
                    for (int c = 0; c < WX; ++c) a.u[eo + c] = S.uf[c];
                }
                if (last) {
                    #pragma unroll
                    for (int c = 0; c < WX; ++c) {
                        a.u[eo + WX + (long long)WA * T + (long long)WS * T + c] = S.uqT[c];
                        a.z[zof + (long long)WS * T + c] = S.zT[c];
                    }
                }
            }
            if (t == 0) {
                a.iters[inst] = done;
                a.status[inst] = status;
                a.rpri[inst] = rp;
                a.rdual[inst] = rd;
            }
        }
    }
}

// Work items for k_mpc_warp: instances of 33..64 steps alone (longest
// first), then those of at most 32 steps in pairs of similar horizons
// (longest first).  Returns false when some instance has more than 64 steps.
bool mpc_warp_items(const int *T, int n, std::vector<int2> &items) {
    std::vector<int> longi, shorti;
    for (int i = 0; i < n; ++i) {
        if (T[i] > 64) return false;
        (T[i] > 32 ? longi : shorti).push_back(i);
    }
    auto byT = [&](int x, int y) { return T[x] != T[y] ? T[x] > T[y] : x < y; };
    std::sort(longi.begin(), longi.end(), byT);
    std::sort(shorti.begin(), shorti.end(), byT);
    items.clear();
    for (int i : longi) items.push_back(make_int2(i, -2));
    for (size_t k = 0; k < shorti.size(); k += 2)
        items.push_back(make_int2(shorti[k], k + 1 < shorti.size() ? shorti[k + 1] : -1));
    return true;
}

cudaError_t mpc_warp_launch(const MpcArgs<float> &a, const int2 *items, int n_items, int grid, cudaStream_t s) {
    k_mpc_warp<<<grid, kWarpCta, 0, s>>>(a, items, n_items);
    return cudaGetLastError();
}

int mpc_warp_max_blocks_per_sm() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, (const void *)k_mpc_warp, kWarpCta, 0) != cudaSuccess)
        return 0;
    return n;
}

}  // namespace fga
