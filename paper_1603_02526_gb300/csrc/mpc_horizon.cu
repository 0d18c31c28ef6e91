// mpc_horizon.cu -- one long-horizon MPC (Sec. V-B: the sampled inverted
// pendulum, A 4 x 4, B 4 x 1, horizon K up to 10^5) solved by Algorithm 2
// with the horizon laid along the grid.
//
// The graph is the chain FIX(x_0) | DYN(x_t, u_t, x_{t+1}) t < K |
// QUAD(x_t, u_t) t < K | QUAD(x_K) (creation order).  Thread t of the grid
// owns step t: the 14 edges of DYN_t and QUAD_t (plus FIX on step 0 and the
// terminal cost on step K-1), and the variables x_t, u_t (and x_K).  Its
// messages live in registers for the whole call.  Every variable but x_t has
// all its edges in one thread; x_t also takes the x' edge of DYN_{t-1}, so
// each iteration a thread hands that contribution to its right neighbour
// (shared memory inside a CTA, a global slot across CTAs), and across a CTA
// boundary the left CTA also receives the right CTA's first contributions,
// so that both compute the boundary z with the same operations in the same
// order.  One grid-wide barrier per iteration, one more on check iterations.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <new>
#include <vector>

#include "../../include/fgadmm.h"
#include "fga_host.h"
#include "fga_internal.h"
#include "persist.cuh"

int fga_set_last_error(int code, const char *msg);   // fga_graph.cpp

namespace fga {
namespace {

constexpr int kHzNX = 4, kHzNU = 1;
constexpr int kHzD = 2 * kHzNX + kHzNU;   // edges of a dynamics factor
constexpr int kHzQ = kHzNX + kHzNU;       // edges of a stage cost
constexpr int kHzT = 224;                 // steps (threads) per CTA: 3 CTAs of 7 warps per SM

struct HzArgs {
    int K, G;
    long long E;              // scalar edges: 14 K + 8
    float rho, alpha;
    float srho3, srho2;       // rho x degree (3 for x_t, t < K; 2 for u_t and x_K)
    const float *P;           // dynamics projector, kHzD x kHzD, row-major
    const float *w;           // q[4], r[1]
    const float *x0;          // fixed initial state
    float *u, *x;             // edge state, creation order
    float *zx, *zu;           // z: x_0..x_K, then u_0..u_{K-1}
    float *fwd;               // [2][G][4]: DYN x' contributions of a CTA's last step
    float *bwd;               // [2][G][8]: DYN x and QUAD x contributions of a CTA's first step
    double *res;              // [G][2]: the CTAs' primal and dual partial sums
    TileSync *sync;
    Ctl *ctl;
    long long k0, iters;      // iterations before this call, iterations in it
    int check_every;
    double tol_pri, tol_dual;
    long long timeout_ns;
    int skip_block;
};

__device__ __forceinline__ double block_sum_hz(double v, double *s_w) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += s_w[i];
    return s;
}

__global__ void __launch_bounds__(kHzT, 3) k_horizon(const HzArgs a) {
    constexpr int NX = kHzNX, NU = kHzNU, D = kHzD, Q = kHzQ;
    __shared__ float sP[D * D];
    __shared__ float s_c[kHzT][NX];   // DYN_t x' contributions rho m, by step
    __shared__ float s_z[kHzT][NX];   // new z of x_t, by step
    __shared__ double s_w[2][kHzT / 32];
    __shared__ int s_stop;
    __shared__ double s_r[2];
    __shared__ float sW[Q];
    // the fixed x_0 and the terminal cost belong to one step each: their
    // edges' u and x wait in shared memory, not in every thread's registers
    __shared__ float s_uf[NX], s_xf[NX], s_ut[NX], s_xt[NX];
    for (int i = threadIdx.x; i < D * D; i += blockDim.x) sP[i] = a.P[i];
    if (threadIdx.x < Q) sW[threadIdx.x] = a.w[threadIdx.x];
    const int K = a.K;
    const int t = blockIdx.x * kHzT + threadIdx.x;
    const bool valid = t < K;
    const bool first = t == 0, last = t == K - 1;
    // the step at the right end of a full CTA that is not the grid's last
    const bool cta_last = valid && !last && threadIdx.x == kHzT - 1;
    const long long eD = NX + (long long)t * D;                 // DYN_t's first edge
    const long long eQ = NX + (long long)K * D + (long long)t * Q;   // QUAD_t's first edge
    const long long eT = NX + (long long)K * D + (long long)K * Q;   // terminal cost's first edge
    float ud[D], uq[Q], xd[D], xq[Q];
    float zx[NX], zu[NU], zx1[NX];
    #pragma unroll
    for (int i = 0; i < D; ++i) ud[i] = valid ? a.u[eD + i] : 0.f;
    #pragma unroll
    for (int i = 0; i < Q; ++i) uq[i] = valid ? a.u[eQ + i] : 0.f;
    #pragma unroll
    for (int i = 0; i < NX; ++i) {
        if (first) {
            s_uf[i] = a.u[i];
            s_xf[i] = 0.f;
        }
        if (last) {
            s_ut[i] = a.u[eT + i];
            s_xt[i] = 0.f;
        }
        zx[i] = valid ? a.zx[(long long)t * NX + i] : 0.f;
        zx1[i] = valid ? a.zx[(long long)(t + 1) * NX + i] : 0.f;
    }
    #pragma unroll
    for (int i = 0; i < NU; ++i) zu[i] = valid ? a.zu[(long long)t * NU + i] : 0.f;
    #pragma unroll
    for (int i = 0; i < D; ++i) xd[i] = 0.f;
    #pragma unroll
    for (int i = 0; i < Q; ++i) xq[i] = 0.f;
    __syncthreads();

    const float rho = a.rho, alpha = a.alpha;
    const unsigned long long G = (unsigned long long)a.G;
    unsigned long long nb = 0;   // grid barriers passed
    bool skip = a.skip_block == (int)blockIdx.x;
    long long it = 0, done = a.iters;
    double rp = 0.0, rd = 0.0;
    for (it = 1; it <= a.iters; ++it) {
        const int par = (int)(it & 1);
        const bool chk = ((a.k0 + it) % a.check_every == 0) || it == a.iters;
        float cdx[NX], cdu[NU], cdx1[NX], cqx[NX], cqu[NU];
        if (valid) {
            // x-update: dynamics (v = P n), stage cost, fixed x_0, terminal cost
            float n[D];
            #pragma unroll
            for (int i = 0; i < NX; ++i) {
                n[i] = zx[i] - ud[i];
                n[NX + NU + i] = zx1[i] - ud[NX + NU + i];
            }
            #pragma unroll
            for (int i = 0; i < NU; ++i) n[NX + i] = zu[i] - ud[NX + i];
            #pragma unroll
            for (int r = 0; r < D; ++r) {
                float s = 0.f;
                #pragma unroll
                for (int c = 0; c < D; ++c) s += sP[r * D + c] * n[c];
                xd[r] = s;
            }
            #pragma unroll
            for (int i = 0; i < NX; ++i) xq[i] = (rho * (zx[i] - uq[i])) / (sW[i] + rho);
            #pragma unroll
            for (int i = 0; i < NU; ++i) xq[NX + i] = (rho * (zu[i] - uq[NX + i])) / (sW[NX + i] + rho);
            if (first) {
                #pragma unroll
                for (int i = 0; i < NX; ++i) s_xf[i] = a.x0[i];
            }
            if (last) {
                #pragma unroll
                for (int i = 0; i < NX; ++i) s_xt[i] = (rho * (zx1[i] - s_ut[i])) / (sW[i] + rho);
            }
            // m = x + u, weighted by rho: the z-update's terms
            #pragma unroll
            for (int i = 0; i < NX; ++i) {
                cdx[i] = rho * (xd[i] + ud[i]);
                cdx1[i] = rho * (xd[NX + NU + i] + ud[NX + NU + i]);
                cqx[i] = rho * (xq[i] + uq[i]);
                s_c[threadIdx.x][i] = cdx1[i];
            }
            #pragma unroll
            for (int i = 0; i < NU; ++i) {
                cdu[i] = rho * (xd[NX + i] + ud[NX + i]);
                cqu[i] = rho * (xq[NX + i] + uq[NX + i]);
            }
            if (cta_last) {
                #pragma unroll
                for (int i = 0; i < NX; ++i) a.fwd[((long long)par * a.G + blockIdx.x) * NX + i] = cdx1[i];
            }
            if (threadIdx.x == 0 && blockIdx.x > 0) {
                #pragma unroll
                for (int i = 0; i < NX; ++i) {
                    a.bwd[((long long)par * a.G + blockIdx.x) * 2 * NX + i] = cdx[i];
                    a.bwd[((long long)par * a.G + blockIdx.x) * 2 * NX + NX + i] = cqx[i];
                }
            }
        }
        ++nb;
        if (!tile_barrier(a.sync, G * nb, a.timeout_ns, skip)) return;
        skip = false;
        // z-update: each sum in creation order of the variable's edges
        float zxn[NX], zun[NU], zx1n[NX];
        if (valid) {
            #pragma unroll
            for (int i = 0; i < NX; ++i) {
                float cprev;
                if (first) cprev = rho * (s_xf[i] + s_uf[i]);
                else if (threadIdx.x > 0) cprev = s_c[threadIdx.x - 1][i];
                else cprev = __ldcg(a.fwd + ((long long)par * a.G + blockIdx.x - 1) * NX + i);
                zxn[i] = ((cprev + cdx[i]) + cqx[i]) / a.srho3;
                s_z[threadIdx.x][i] = zxn[i];
            }
            #pragma unroll
            for (int i = 0; i < NU; ++i) zun[i] = (cdu[i] + cqu[i]) / a.srho2;
            if (last) {
                #pragma unroll
                for (int i = 0; i < NX; ++i) zx1n[i] = (cdx1[i] + rho * (s_xt[i] + s_ut[i])) / a.srho2;
            } else if (cta_last) {
                const float *nb2 = a.bwd + ((long long)par * a.G + blockIdx.x + 1) * 2 * NX;
                #pragma unroll
                for (int i = 0; i < NX; ++i) zx1n[i] = ((cdx1[i] + __ldcg(nb2 + i)) + __ldcg(nb2 + NX + i)) / a.srho3;
            }
        }
        __syncthreads();
        double pri = 0.0, dual = 0.0;
        if (valid) {
            if (!last && !cta_last) {
                #pragma unroll
                for (int i = 0; i < NX; ++i) zx1n[i] = s_z[threadIdx.x + 1][i];
            }
            if (chk) {
                // residuals: (x_e - z_b)^2 per edge; rho^2 deg_b (dz_b)^2 per owned variable
                #pragma unroll
                for (int i = 0; i < NX; ++i) {
                    const double e1 = (double)xd[i] - zxn[i], e2 = (double)xd[NX + NU + i] - zx1n[i];
                    const double e3 = (double)xq[i] - zxn[i];
                    pri += e1 * e1 + e2 * e2 + e3 * e3;
                    if (first) {
                        const double e4 = (double)s_xf[i] - zxn[i];
                        pri += e4 * e4;
                    }
                    if (last) {
                        const double e5 = (double)s_xt[i] - zx1n[i];
                        pri += e5 * e5;
                        const double d5 = (double)zx1n[i] - zx1[i];
                        dual += 2.0 * (double)rho * rho * d5 * d5;
                    }
                    const double dx = (double)zxn[i] - zx[i];
                    dual += 3.0 * (double)rho * rho * dx * dx;
                }
                #pragma unroll
                for (int i = 0; i < NU; ++i) {
                    const double e1 = (double)xd[NX + i] - zun[i], e3 = (double)xq[NX + i] - zun[i];
                    pri += e1 * e1 + e3 * e3;
                    const double du = (double)zun[i] - zu[i];
                    dual += 2.0 * (double)rho * rho * du * du;
                }
            }
            // u-update, u += alpha (x - z)
            #pragma unroll
            for (int i = 0; i < NX; ++i) {
                ud[i] += alpha * (xd[i] - zxn[i]);
                ud[NX + NU + i] += alpha * (xd[NX + NU + i] - zx1n[i]);
                uq[i] += alpha * (xq[i] - zxn[i]);
                if (first) s_uf[i] += alpha * (s_xf[i] - zxn[i]);
                if (last) s_ut[i] += alpha * (s_xt[i] - zx1n[i]);
                zx[i] = zxn[i];
                zx1[i] = zx1n[i];
            }
            #pragma unroll
            for (int i = 0; i < NU; ++i) {
                ud[NX + i] += alpha * (xd[NX + i] - zun[i]);
                uq[NX + i] += alpha * (xq[NX + i] - zun[i]);
                zu[i] = zun[i];
            }
        }
        if (chk) {
            const double sp = block_sum_hz(pri, s_w[0]);
            const double sd = block_sum_hz(dual, s_w[1]);
            if (threadIdx.x == 0) {
                a.res[2 * blockIdx.x] = sp;
                a.res[2 * blockIdx.x + 1] = sd;
            }
            ++nb;
            if (!tile_barrier(a.sync, G * nb, a.timeout_ns, false)) return;
            if (threadIdx.x < 32) {
                double p = 0.0, d = 0.0;
                for (int b = threadIdx.x; b < a.G; b += 32) {
                    p += __ldcg(a.res + 2 * b);
                    d += __ldcg(a.res + 2 * b + 1);
                }
                #pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    p += __shfl_xor_sync(0xffffffffu, p, o);
                    d += __shfl_xor_sync(0xffffffffu, d, o);
                }
                if (threadIdx.x == 0) {
                    const double E = (double)a.E;
                    s_r[0] = sqrt(p / E);
                    s_r[1] = sqrt(d / E);
                    const bool finite = isfinite(s_r[0]) && isfinite(s_r[1]);
                    s_stop = (!finite || (s_r[0] <= a.tol_pri && s_r[1] <= a.tol_dual)) ? 1 : 0;
                }
            }
            __syncthreads();
            rp = s_r[0];
            rd = s_r[1];
            if (s_stop) {
                done = it;
                break;
            }
        }
    }
    // the state after iteration `done`: edges in creation order, z
    if (valid) {
        #pragma unroll
        for (int i = 0; i < D; ++i) {
            a.u[eD + i] = ud[i];
            a.x[eD + i] = xd[i];
        }
        #pragma unroll
        for (int i = 0; i < Q; ++i) {
            a.u[eQ + i] = uq[i];
            a.x[eQ + i] = xq[i];
        }
        #pragma unroll
        for (int i = 0; i < NX; ++i) {
            if (first) {
                a.u[i] = s_uf[i];
                a.x[i] = s_xf[i];
            }
            if (last) {
                a.u[eT + i] = s_ut[i];
                a.x[eT + i] = s_xt[i];
                a.zx[(long long)K * NX + i] = zx1[i];
            }
            a.zx[(long long)t * NX + i] = zx[i];
        }
        #pragma unroll
        for (int i = 0; i < NU; ++i) a.zu[(long long)t * NU + i] = zu[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const bool finite = isfinite(rp) && isfinite(rd);
        int st = finite ? 0 : kENonFinite;
        if (st == 0 && !(rp <= a.tol_pri && rd <= a.tol_dual) && (a.tol_pri > 0.0 || a.tol_dual > 0.0))
            st = kEBudget;
        a.ctl->iters = done;
        a.ctl->r_pri = rp;
        a.ctl->r_dual = rd;
        a.ctl->status = st;
        a.ctl->checked = 1;
    }
}

int hfail(int code, const char *fmt, ...) {
    char buf[384];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return fga_set_last_error(code, buf);
}

struct HBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaError_t alloc(size_t b) {
        bytes = b;
        return cudaMalloc(&p, b ? b : 1);
    }
    ~HBuf() {
        if (p) cudaFree(p);
    }
    template <typename T>
    T *as() const {
        return static_cast<T *>(p);
    }
};

}  // namespace
}  // namespace fga

struct fga_horizon {
    int device = 0;
    int K = 0, G = 0;
    long long E = 0, nz = 0;
    double rho = 1.0, alpha = 1.0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    bool initialized = false;
    long long k0 = 0;
    fga::HBuf P, w, x0, u, x, zx, zu, fwd, bwd, res, sync, ctl;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

#define HZ_CUDA(call)                                                                                  \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) return fga::hfail(FGA_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

extern "C" int fga_horizon_create(fga_horizon **out, int32_t K, int32_t nx, int32_t nu, const double *A,
                                  const double *B, const double *q, const double *r, const double *x0, double rho,
                                  double alpha, int32_t device, void *cuda_stream) {
    using namespace fga;
    if (!out) return hfail(FGA_EINVAL, "fga_horizon_create: out is NULL");
    *out = nullptr;
    if (nx != kHzNX || nu != kHzNU)
        return hfail(FGA_EINVAL, "fga_horizon_create: built for nx = %d, nu = %d (got %d, %d)", kHzNX, kHzNU, nx, nu);
    if (K < 1) return hfail(FGA_EINVAL, "fga_horizon_create: K must be >= 1");
    if (!A || !B || !q || !r || !x0) return hfail(FGA_EINVAL, "fga_horizon_create: NULL system data");
    if (!(rho > 0.0) || !(alpha > 0.0) || !std::isfinite(rho) || !std::isfinite(alpha))
        return hfail(FGA_EINVAL, "fga_horizon_create: rho and alpha must be finite and > 0");
    for (int i = 0; i < nx * nx; ++i)
        if (!std::isfinite(A[i])) return hfail(FGA_EINVAL, "fga_horizon_create: non-finite A");
    for (int i = 0; i < nx * nu; ++i)
        if (!std::isfinite(B[i])) return hfail(FGA_EINVAL, "fga_horizon_create: non-finite B");
    for (int i = 0; i < nx; ++i)
        if (!(q[i] >= 0.0) || !std::isfinite(q[i]) || !std::isfinite(x0[i]))
            return hfail(FGA_EINVAL, "fga_horizon_create: q must be >= 0 and x0 finite");
    for (int i = 0; i < nu; ++i)
        if (!(r[i] >= 0.0) || !std::isfinite(r[i])) return hfail(FGA_EINVAL, "fga_horizon_create: r must be >= 0");
    HZ_CUDA(cudaSetDevice(device));
    int sms = 0, bps = 0;
    HZ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    HZ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_horizon, kHzT, 0));
    const int G = (K + kHzT - 1) / kHzT;
    if (bps < 1 || (long long)G > (long long)bps * sms)
        return hfail(FGA_EINVAL, "fga_horizon_create: K = %d needs %d CTAs of %d steps; at most %d are co-resident",
                     K, G, kHzT, bps * sms);
    std::vector<double> rv(kHzD, rho), Pd;
    if (!dyn_projector(nx, nu, A, B, rv.data(), Pd))
        return hfail(FGA_EINVAL, "fga_horizon_create: singular dynamics constraint");
    auto *h = new (std::nothrow) fga_horizon();
    if (!h) return hfail(FGA_ENOMEM, "fga_horizon_create: out of host memory");
    h->device = device;
    h->K = K;
    h->G = G;
    h->E = (long long)(kHzD + kHzQ) * K + 2 * kHzNX;
    h->nz = (long long)(K + 1) * kHzNX + (long long)K * kHzNU;
    h->rho = rho;
    h->alpha = alpha;
    auto bad = [&](int rc) {
        fga_horizon_destroy(h);
        return rc;
    };
    if (cuda_stream) {
        h->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess)
            return bad(hfail(FGA_ECUDA, "fga_horizon_create: stream"));
        h->own_stream = true;
    }
    std::vector<float> Pf(Pd.begin(), Pd.end()), wf(kHzQ), x0f(kHzNX);
    for (int i = 0; i < kHzNX; ++i) {
        wf[i] = (float)q[i];
        x0f[i] = (float)x0[i];
    }
    for (int i = 0; i < kHzNU; ++i) wf[kHzNX + i] = (float)r[i];
    struct {
        HBuf *b;
        size_t bytes;
    } al[] = {{&h->P, Pf.size() * 4},
              {&h->w, wf.size() * 4},
              {&h->x0, x0f.size() * 4},
              {&h->u, (size_t)h->E * 4},
              {&h->x, (size_t)h->E * 4},
              {&h->zx, (size_t)(K + 1) * kHzNX * 4},
              {&h->zu, (size_t)K * kHzNU * 4},
              {&h->fwd, (size_t)2 * G * kHzNX * 4},
              {&h->bwd, (size_t)2 * G * 2 * kHzNX * 4},
              {&h->res, (size_t)2 * G * 8},
              {&h->sync, sizeof(TileSync)},
              {&h->ctl, sizeof(Ctl)}};
    for (auto &e : al)
        if (e.b->alloc(e.bytes) != cudaSuccess) return bad(hfail(FGA_ENOMEM, "fga_horizon_create: device memory"));
    if (cudaMemcpy(h->P.p, Pf.data(), Pf.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->w.p, wf.data(), wf.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->x0.p, x0f.data(), x0f.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess)
        return bad(hfail(FGA_ECUDA, "fga_horizon_create: upload"));
    // the uploads ran on the legacy stream, which the solver's non-blocking
    // stream does not wait for
    if (cudaDeviceSynchronize() != cudaSuccess) return bad(hfail(FGA_ECUDA, "fga_horizon_create: upload"));
    *out = h;
    return FGA_OK;
}

extern "C" int fga_horizon_init(fga_horizon *h) {
    if (!h) return fga::hfail(FGA_EINVAL, "fga_horizon_init: NULL");
    HZ_CUDA(cudaSetDevice(h->device));
    HZ_CUDA(cudaMemsetAsync(h->u.p, 0, h->u.bytes, h->stream));
    HZ_CUDA(cudaMemsetAsync(h->x.p, 0, h->x.bytes, h->stream));
    HZ_CUDA(cudaMemsetAsync(h->zx.p, 0, h->zx.bytes, h->stream));
    HZ_CUDA(cudaMemsetAsync(h->zu.p, 0, h->zu.bytes, h->stream));
    HZ_CUDA(cudaStreamSynchronize(h->stream));
    h->k0 = 0;
    h->initialized = true;
    return FGA_OK;
}

extern "C" int fga_horizon_solve(fga_horizon *h, const fga_iter_opts *o, fga_iter_result *res) {
    using namespace fga;
    if (!h || !o || !res) return hfail(FGA_EINVAL, "fga_horizon_solve: NULL argument");
    if (!h->initialized) return hfail(FGA_ESTATE, "fga_horizon_solve: call fga_horizon_init first");
    if (o->max_iters < 0 || o->check_every < 1 || !(o->tol_pri >= 0.0) || !(o->tol_dual >= 0.0))
        return hfail(FGA_EINVAL, "fga_horizon_solve: bad options");
    if (!o->fused) return hfail(FGA_EINVAL, "fga_horizon_solve: fused launches only");
    std::memset(res, 0, sizeof *res);
    if (o->max_iters == 0) return FGA_OK;
    HZ_CUDA(cudaSetDevice(h->device));
    HzArgs a;
    std::memset(&a, 0, sizeof a);
    a.K = h->K;
    a.G = h->G;
    a.E = h->E;
    a.rho = (float)h->rho;
    a.alpha = (float)h->alpha;
    a.srho3 = (float)(3.0 * h->rho);
    a.srho2 = (float)(2.0 * h->rho);
    a.P = h->P.as<float>();
    a.w = h->w.as<float>();
    a.x0 = h->x0.as<float>();
    a.u = h->u.as<float>();
    a.x = h->x.as<float>();
    a.zx = h->zx.as<float>();
    a.zu = h->zu.as<float>();
    a.fwd = h->fwd.as<float>();
    a.bwd = h->bwd.as<float>();
    a.res = h->res.as<double>();
    a.sync = h->sync.as<TileSync>();
    a.ctl = h->ctl.as<Ctl>();
    a.k0 = h->k0;
    a.iters = o->max_iters;
    a.check_every = o->check_every;
    a.tol_pri = o->tol_pri;
    a.tol_dual = o->tol_dual;
    a.timeout_ns = o->barrier_timeout_ns > 0 ? o->barrier_timeout_ns : 2000000000LL;
    a.skip_block = o->fault_skip_block;
    cudaStream_t s = h->stream;
    HZ_CUDA(cudaMemsetAsync(h->sync.p, 0, sizeof(TileSync), s));
    HZ_CUDA(cudaMemsetAsync(h->ctl.p, 0, sizeof(Ctl), s));
    HZ_CUDA(cudaEventRecord(h->ev0, s));
    void *args[] = {(void *)&a};
    HZ_CUDA(cudaLaunchCooperativeKernel((const void *)k_horizon, dim3(h->G), dim3(kHzT), args, 0, s));
    HZ_CUDA(cudaEventRecord(h->ev1, s));
    HZ_CUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    HZ_CUDA(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    Ctl c;
    TileSync b;
    HZ_CUDA(cudaMemcpy(&c, h->ctl.p, sizeof c, cudaMemcpyDeviceToHost));
    HZ_CUDA(cudaMemcpy(&b, h->sync.p, sizeof b, cudaMemcpyDeviceToHost));
    res->ms = ms;
    if (b.error) {
        h->initialized = false;   // some CTAs stopped mid-iteration: the state is not one iterate
        res->iters = 0;
        res->r_pri = res->r_dual = std::numeric_limits<double>::quiet_NaN();
        res->status = FGA_ETIMEOUT;
        return hfail(FGA_ETIMEOUT, "fga_horizon_solve: a grid-wide wait ran out (the state needs fga_horizon_init)");
    }
    res->iters = c.iters;
    res->r_pri = c.r_pri;
    res->r_dual = c.r_dual;
    res->status = c.status;
    h->k0 += c.iters;
    if (c.status == FGA_ENONFINITE) return hfail(FGA_ENONFINITE, "fga_horizon_solve: residual became non-finite");
    return FGA_OK;
}

extern "C" int fga_horizon_read(fga_horizon *h, double *z, double *x_edges, double *u_edges) {
    using namespace fga;
    if (!h) return hfail(FGA_EINVAL, "fga_horizon_read: NULL");
    if (!h->initialized) return hfail(FGA_ESTATE, "fga_horizon_read: no state (call fga_horizon_init)");
    HZ_CUDA(cudaSetDevice(h->device));
    HZ_CUDA(cudaStreamSynchronize(h->stream));
    std::vector<float> buf;
    auto pull = [&](const HBuf &src, size_t n, double *dst) -> int {
        buf.resize(n);
        if (cudaMemcpy(buf.data(), src.p, n * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
            return hfail(FGA_ECUDA, "fga_horizon_read: copy");
        for (size_t i = 0; i < n; ++i) dst[i] = buf[i];
        return FGA_OK;
    };
    int rc;
    if (z) {
        const size_t nxz = (size_t)(h->K + 1) * kHzNX;
        if ((rc = pull(h->zx, nxz, z))) return rc;
        if ((rc = pull(h->zu, (size_t)h->K * kHzNU, z + nxz))) return rc;
    }
    if (x_edges && (rc = pull(h->x, (size_t)h->E, x_edges))) return rc;
    if (u_edges && (rc = pull(h->u, (size_t)h->E, u_edges))) return rc;
    return FGA_OK;
}

extern "C" int fga_horizon_info(const fga_horizon *h, int64_t *info, int32_t n) {
    if (!h || !info || n < 4) return fga::hfail(FGA_EINVAL, "fga_horizon_info: bad arguments");
    info[0] = h->G;
    info[1] = fga::kHzT;
    info[2] = h->E;
    info[3] = h->nz;
    return FGA_OK;
}

extern "C" int fga_horizon_destroy(fga_horizon *h) {
    if (!h) return FGA_OK;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
    return FGA_OK;
}
