// fga_batch.cpp -- host side of the batched MPC solver: instance layout,
// upload, CUDA-graph launch, readout, warm start, autotuner (C-ABI).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <limits>
#include <map>
#include <memory>
#include <numeric>
#include <sstream>
#include <string>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/fgadmm.h"
#include "fga_host.h"
#include "mpc_internal.h"

using namespace fga;

int fga_set_last_error(int code, const char *msg);   // fga_graph.cpp

static int bfail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return fga_set_last_error(code, buf);
}

#define BCUDA(call)                                                                                  \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess)                                                                       \
            return bfail(e_ == cudaErrorMemoryAllocation ? FGA_ENOMEM : FGA_ECUDA, "%s: %s (%s:%d)", \
                         #call, cudaGetErrorString(e_), __FILE__, __LINE__);                         \
    } while (0)

namespace {
struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
    ~Buf() {
        if (p) cudaFree(p);
    }
    cudaError_t alloc(size_t n) {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = n;
        return n ? cudaMalloc(&p, n) : cudaSuccess;
    }
    template <typename T>
    T *as() const { return static_cast<T *>(p); }
};

template <typename T>
int put(Buf &b, const std::vector<T> &v) {
    BCUDA(b.alloc(std::max<size_t>(v.size(), 1) * sizeof(T)));
    if (!v.empty()) BCUDA(cudaMemcpy(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return FGA_OK;
}
}  // namespace

struct GraphKey {
    int threads, ce;
    long long K;
    double tp, td;
    bool operator<(const GraphKey &o) const {
        return std::tie(threads, ce, K, tp, td) < std::tie(o.threads, o.ce, o.K, o.tp, o.td);
    }
};

struct fga_mpc_batch {
    int precision = FGA_F32, device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int n = 0, nx = 0, nu = 0, nsys = 0, tmax = 0;
    double lo = -1, hi = 1, rho = 1, alpha = 1;
    std::vector<int> T, sys;
    std::vector<long long> zoff, eoff;
    long long Z = 0, E = 0;
    Buf dT, dzoff, deoff, dsys, dorder, dP, dA, dB, dK, dq, dr, dx0, dz, du, dx, diters, dstatus, drp, drd, dqueue;
    // one lane per time step (threads = 32): FP32, 12 states, 4 inputs,
    // horizons up to 64; its work items
    bool warp_ok = false;
    int n_items = 0;
    Buf ditems;
    bool x0_set = false;
    int tuned_threads = 128, tuned_ce = 1;
    std::map<GraphKey, cudaGraphExec_t> graphs;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    size_t rsize() const { return precision == FGA_F32 ? 4 : 8; }
};

template <typename R>
static MpcArgs<R> make_args(const fga_mpc_batch *b) {
    MpcArgs<R> a;
    std::memset(&a, 0, sizeof a);
    a.n_inst = b->n;
    a.nx = b->nx;
    a.nu = b->nu;
    a.T = b->dT.as<int>();
    a.zoff = b->dzoff.as<long long>();
    a.eoff = b->deoff.as<long long>();
    a.sys = b->dsys.as<int>();
    a.order = b->dorder.as<int>();
    a.P = b->dP.as<R>();
    a.q = b->dq.as<R>();
    a.r = b->dr.as<R>();
    a.x0 = b->dx0.as<R>();
    a.lo = (R)b->lo;
    a.hi = (R)b->hi;
    a.rho = (R)b->rho;
    a.alpha = (R)b->alpha;
    a.z = b->dz.as<R>();
    a.u = b->du.as<R>();
    a.x = b->dx.as<R>();
    a.iters = b->diters.as<long long>();
    a.status = b->dstatus.as<int>();
    a.rpri = b->drp.as<double>();
    a.rdual = b->drd.as<double>();
    a.queue = b->dqueue.as<unsigned>();
    a.first_pending = 0;
    return a;
}

template <typename R>
static int upload_systems(fga_mpc_batch *b, const double *A, const double *B, const double *q, const double *r) {
    const int nx = b->nx, nu = b->nu, Ad = 2 * nx + nu;
    std::vector<R> P((size_t)b->nsys * Ad * Ad), Am((size_t)b->nsys * nx * nx), Bm((size_t)b->nsys * nx * nu),
        K((size_t)b->nsys * nx * Ad), qq((size_t)b->nsys * nx), rr((size_t)b->nsys * nu);
    std::vector<double> Pd, rho((size_t)Ad, b->rho);
    for (int s = 0; s < b->nsys; ++s) {
        const double *As = A + (size_t)s * nx * nx, *Bs = B + (size_t)s * nx * nu;
        if (!dyn_projector(nx, nu, As, Bs, rho.data(), Pd))
            return bfail(FGA_EINVAL, "fga_mpc_batch_create: singular dynamics of system %d", s);
        for (size_t j = 0; j < Pd.size(); ++j) P[(size_t)s * Ad * Ad + j] = (R)Pd[j];
        for (int j = 0; j < nx * nx; ++j) Am[(size_t)s * nx * nx + j] = (R)As[j];
        for (int j = 0; j < nx * nu; ++j) Bm[(size_t)s * nx * nu + j] = (R)Bs[j];
        for (int j = 0; j < nx; ++j) qq[(size_t)s * nx + j] = (R)q[(size_t)s * nx + j];
        for (int j = 0; j < nu; ++j) rr[(size_t)s * nu + j] = (R)r[(size_t)s * nu + j];
        // K = (M M^T)^{-1} M with M = [A B -I] (Gauss-Jordan on M M^T): maps a
        // dynamics edge's u back to its multiplier, lambda = -rho K u.
        std::vector<double> M((size_t)nx * Ad, 0.0), G((size_t)nx * 2 * nx, 0.0);
        for (int i = 0; i < nx; ++i) {
            for (int j = 0; j < nx; ++j) M[(size_t)i * Ad + j] = As[i * nx + j];
            for (int j = 0; j < nu; ++j) M[(size_t)i * Ad + nx + j] = Bs[i * nu + j];
            M[(size_t)i * Ad + nx + nu + i] = -1.0;
        }
        for (int i = 0; i < nx; ++i) {
            for (int k = 0; k < nx; ++k) {
                double t = 0.0;
                for (int j = 0; j < Ad; ++j) t += M[(size_t)i * Ad + j] * M[(size_t)k * Ad + j];
                G[(size_t)i * 2 * nx + k] = t;
            }
            G[(size_t)i * 2 * nx + nx + i] = 1.0;
        }
        for (int c = 0; c < nx; ++c) {   // Gauss-Jordan with partial pivoting
            int piv = c;
            for (int rr2 = c + 1; rr2 < nx; ++rr2)
                if (std::fabs(G[(size_t)rr2 * 2 * nx + c]) > std::fabs(G[(size_t)piv * 2 * nx + c])) piv = rr2;
            if (piv != c)
                for (int j = 0; j < 2 * nx; ++j) std::swap(G[(size_t)c * 2 * nx + j], G[(size_t)piv * 2 * nx + j]);
            const double d = G[(size_t)c * 2 * nx + c];
            for (int j = 0; j < 2 * nx; ++j) G[(size_t)c * 2 * nx + j] /= d;
            for (int rr2 = 0; rr2 < nx; ++rr2) {
                if (rr2 == c) continue;
                const double f = G[(size_t)rr2 * 2 * nx + c];
                for (int j = 0; j < 2 * nx; ++j) G[(size_t)rr2 * 2 * nx + j] -= f * G[(size_t)c * 2 * nx + j];
            }
        }
        for (int i = 0; i < nx; ++i)
            for (int j = 0; j < Ad; ++j) {
                double t = 0.0;
                for (int k = 0; k < nx; ++k) t += G[(size_t)i * 2 * nx + nx + k] * M[(size_t)k * Ad + j];
                K[((size_t)s * nx + i) * Ad + j] = (R)t;
            }
    }
    int rc;
    if ((rc = put(b->dP, P)) || (rc = put(b->dA, Am)) || (rc = put(b->dB, Bm)) || (rc = put(b->dK, K)) ||
        (rc = put(b->dq, qq)) || (rc = put(b->dr, rr)))
        return rc;
    return FGA_OK;
}

extern "C" int fga_mpc_batch_create(fga_mpc_batch **out, int32_t precision, int32_t device, void *stream,
                                    int32_t n_inst, const int32_t *T, int32_t nx, int32_t nu, int32_t n_sys,
                                    const int32_t *sys_of_inst, const double *A, const double *B, const double *q,
                                    const double *r, double umax, double rho, double alpha) {
    if (!out || !T || !A || !B || !q || !r) return bfail(FGA_EINVAL, "fga_mpc_batch_create: NULL argument");
    if (precision != FGA_F32 && precision != FGA_F64) return bfail(FGA_EINVAL, "fga_mpc_batch_create: precision");
    if (n_inst < 1 || nx < 1 || nu < 1 || 2 * nx + nu > 64 || n_sys < 1)
        return bfail(FGA_EINVAL, "fga_mpc_batch_create: sizes (need n_inst, nx, nu >= 1, 2 nx + nu <= 64)");
    if (!(umax > 0) || !(rho > 0) || !(alpha > 0)) return bfail(FGA_EINVAL, "fga_mpc_batch_create: umax, rho, alpha > 0");
    if (!sys_of_inst && n_sys != 1 && n_sys != n_inst)
        return bfail(FGA_EINVAL, "fga_mpc_batch_create: sys_of_inst needed unless n_sys is 1 or n_inst");
    for (int s = 0; s < n_sys * nx; ++s)
        if (!(q[s] >= 0)) return bfail(FGA_EINVAL, "fga_mpc_batch_create: negative state weight");
    for (int s = 0; s < n_sys * nu; ++s)
        if (!(r[s] >= 0)) return bfail(FGA_EINVAL, "fga_mpc_batch_create: negative input weight");
    fga_mpc_batch *b = new (std::nothrow) fga_mpc_batch();
    if (!b) return bfail(FGA_ENOMEM, "fga_mpc_batch_create: out of memory");
    std::unique_ptr<fga_mpc_batch> guard(b);
    b->precision = precision;
    b->device = device;
    b->n = n_inst;
    b->nx = nx;
    b->nu = nu;
    b->nsys = n_sys;
    b->lo = -umax;
    b->hi = umax;
    b->rho = rho;
    b->alpha = alpha;
    BCUDA(cudaSetDevice(device));
    if (stream) {
        b->stream = (cudaStream_t)stream;
    } else {
        BCUDA(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));   // graph capture needs a real stream
        b->own_stream = true;
    }
    b->T.assign(T, T + n_inst);
    b->sys.resize(n_inst);
    const int S = nx + nu;
    for (int i = 0; i < n_inst; ++i) {
        if (T[i] < 1 || T[i] > 100000) return bfail(FGA_EINVAL, "fga_mpc_batch_create: horizon %d out of [1, 1e5]", T[i]);
        const int s = sys_of_inst ? sys_of_inst[i] : (n_sys == 1 ? 0 : i);
        if (s < 0 || s >= n_sys) return bfail(FGA_EINVAL, "fga_mpc_batch_create: system index out of range");
        b->sys[i] = s;
        b->zoff.push_back(b->Z);
        b->eoff.push_back(b->E);
        b->Z += (long long)S * T[i] + nx;
        b->E += 2LL * nx + (3LL * nx + 3LL * nu) * T[i];
        b->tmax = std::max(b->tmax, T[i]);
    }
    std::vector<int> order(n_inst);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a2, int b2) { return T[a2] > T[b2]; });
    int rc;
    if ((rc = put(b->dT, b->T)) || (rc = put(b->dzoff, b->zoff)) || (rc = put(b->deoff, b->eoff)) ||
        (rc = put(b->dsys, b->sys)) || (rc = put(b->dorder, order)))
        return rc;
    if (precision == FGA_F32 && nx == 12 && nu == 4) {
        std::vector<int2> items;
        if (mpc_warp_items(b->T.data(), n_inst, items)) {
            if ((rc = put(b->ditems, items))) return rc;
            b->n_items = (int)items.size();
            b->warp_ok = true;
        }
    }
    rc = precision == FGA_F32 ? upload_systems<float>(b, A, B, q, r) : upload_systems<double>(b, A, B, q, r);
    if (rc) return rc;
    const size_t rs = b->rsize();
    BCUDA(b->dx0.alloc((size_t)n_inst * nx * rs));
    BCUDA(cudaMemset(b->dx0.p, 0, b->dx0.bytes));
    BCUDA(b->dz.alloc((size_t)b->Z * rs));
    BCUDA(b->du.alloc((size_t)b->E * rs));
    BCUDA(b->dx.alloc((size_t)b->E * rs));
    BCUDA(b->diters.alloc((size_t)n_inst * sizeof(long long)));
    BCUDA(b->dstatus.alloc((size_t)n_inst * sizeof(int)));
    BCUDA(b->drp.alloc((size_t)n_inst * sizeof(double)));
    BCUDA(b->drd.alloc((size_t)n_inst * sizeof(double)));
    BCUDA(b->dqueue.alloc(sizeof(unsigned)));
    BCUDA(cudaMemset(b->dz.p, 0, b->dz.bytes));
    BCUDA(cudaMemset(b->du.p, 0, b->du.bytes));
    BCUDA(cudaMemset(b->dx.p, 0, b->dx.bytes));
    BCUDA(cudaEventCreate(&b->ev0));
    BCUDA(cudaEventCreate(&b->ev1));
    BCUDA(cudaDeviceSynchronize());
    *out = guard.release();
    return FGA_OK;
}

template <typename R>
static int to_device_r(Buf &dst, const double *src, size_t n, cudaStream_t s) {
    std::vector<R> v(n);
    cudaPointerAttributes at;
    std::vector<double> h;
    const double *p = src;
    if (cudaPointerGetAttributes(&at, src) == cudaSuccess && at.type == cudaMemoryTypeDevice) {
        h.resize(n);
        BCUDA(cudaMemcpy(h.data(), src, n * sizeof(double), cudaMemcpyDeviceToHost));
        p = h.data();
    }
    cudaGetLastError();
    for (size_t i = 0; i < n; ++i) {
        if (!std::isfinite(p[i])) return bfail(FGA_EINVAL, "non-finite input value");
        v[i] = (R)p[i];
    }
    BCUDA(cudaMemcpyAsync(dst.p, v.data(), n * sizeof(R), cudaMemcpyHostToDevice, s));
    BCUDA(cudaStreamSynchronize(s));
    return FGA_OK;
}

extern "C" int fga_mpc_batch_set_x0(fga_mpc_batch *b, const double *x0) {
    if (!b || !x0) return bfail(FGA_EINVAL, "fga_mpc_batch_set_x0: NULL argument");
    BCUDA(cudaSetDevice(b->device));
    const size_t n = (size_t)b->n * b->nx;
    int rc = b->precision == FGA_F32 ? to_device_r<float>(b->dx0, x0, n, b->stream)
                                     : to_device_r<double>(b->dx0, x0, n, b->stream);
    if (rc) return rc;
    b->x0_set = true;
    return FGA_OK;
}

extern "C" int fga_mpc_batch_init(fga_mpc_batch *b, const double *z0, const double *u0) {
    if (!b) return bfail(FGA_EINVAL, "fga_mpc_batch_init: NULL batch");
    BCUDA(cudaSetDevice(b->device));
    const size_t rs = b->rsize();
    int rc = 0;
    if (z0) rc = b->precision == FGA_F32 ? to_device_r<float>(b->dz, z0, (size_t)b->Z, b->stream)
                                         : to_device_r<double>(b->dz, z0, (size_t)b->Z, b->stream);
    else BCUDA(cudaMemsetAsync(b->dz.p, 0, (size_t)b->Z * rs, b->stream));
    if (rc) return rc;
    if (u0) rc = b->precision == FGA_F32 ? to_device_r<float>(b->du, u0, (size_t)b->E, b->stream)
                                         : to_device_r<double>(b->du, u0, (size_t)b->E, b->stream);
    else BCUDA(cudaMemsetAsync(b->du.p, 0, (size_t)b->E * rs, b->stream));
    if (rc) return rc;
    BCUDA(cudaMemsetAsync(b->dx.p, 0, (size_t)b->E * rs, b->stream));
    BCUDA(cudaStreamSynchronize(b->stream));
    return FGA_OK;
}

extern "C" int fga_mpc_batch_warm_start(fga_mpc_batch *b, const float *pred, int64_t ld) {
    if (!b || !pred) return bfail(FGA_EINVAL, "fga_mpc_batch_warm_start: NULL argument");
    if (ld < 2LL * (b->nx + b->nu) * b->tmax) return bfail(FGA_EINVAL, "fga_mpc_batch_warm_start: ld too small");
    BCUDA(cudaSetDevice(b->device));
    if (b->precision == FGA_F32) {
        BCUDA(mpc_warm_start_impl<float>(make_args<float>(b), b->dA.as<float>(), b->dB.as<float>(), pred, ld,
                                         b->stream));
    } else {
        BCUDA(mpc_warm_start_impl<double>(make_args<double>(b), b->dA.as<double>(), b->dB.as<double>(), pred, ld,
                                          b->stream));
    }
    BCUDA(cudaStreamSynchronize(b->stream));
    return FGA_OK;
}

extern "C" int fga_mpc_batch_targets(fga_mpc_batch *b, float *out, int64_t ld) {
    if (!b || !out) return bfail(FGA_EINVAL, "fga_mpc_batch_targets: NULL argument");
    if (ld < 2LL * (b->nx + b->nu) * b->tmax) return bfail(FGA_EINVAL, "fga_mpc_batch_targets: ld too small");
    BCUDA(cudaSetDevice(b->device));
    if (b->precision == FGA_F32) {
        BCUDA(mpc_targets_impl<float>(make_args<float>(b), b->dK.as<float>(), out, ld, b->stream));
    } else {
        BCUDA(mpc_targets_impl<double>(make_args<double>(b), b->dK.as<double>(), out, ld, b->stream));
    }
    BCUDA(cudaStreamSynchronize(b->stream));
    return FGA_OK;
}

template <typename R>
static int launch_once(fga_mpc_batch *b, const MpcArgs<R> &a, int threads, cudaStream_t s) {
    const int smem = mpc_smem_bytes((int)sizeof(R), b->nx, b->nu, b->tmax, threads);
    const int bps = mpc_max_blocks_per_sm<R>(threads, smem);
    if (bps < 1) return bfail(FGA_EINVAL, "fga_mpc_batch_solve: horizon %d does not fit in shared memory", b->tmax);
    int sms = 0;
    BCUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
    const int grid = std::min(b->n, bps * sms);
    BCUDA(cudaMemsetAsync(a.queue, 0, sizeof(unsigned), s));
    BCUDA(mpc_launch<R>(a, threads, grid, smem, s));
    return FGA_OK;
}

static int launch_warp(fga_mpc_batch *b, const MpcArgs<float> &a, cudaStream_t s) {
    const int bps = mpc_warp_max_blocks_per_sm();
    if (bps < 1) return bfail(FGA_ECUDA, "fga_mpc_batch_solve: the per-step kernel cannot be resident");
    int sms = 0;
    BCUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
    const int grid = std::min(b->n_items, bps * sms);
    BCUDA(cudaMemsetAsync(a.queue, 0, sizeof(unsigned), s));
    BCUDA(mpc_warp_launch(a, b->ditems.as<int2>(), b->n_items, grid, s));
    return FGA_OK;
}

template <typename R>
static int launch_any(fga_mpc_batch *b, const MpcArgs<R> &a, int threads, cudaStream_t s) {
    if constexpr (sizeof(R) == 4) {
        if (threads == 32) return launch_warp(b, a, s);
    }
    return launch_once<R>(b, a, threads, s);
}

template <typename R>
static int solve_typed(fga_mpc_batch *b, const fga_mpc_opts &o, fga_mpc_result &res) {
    MpcArgs<R> a = make_args<R>(b);
    a.max_iters = o.max_iters;
    a.tol_pri = o.tol_pri;
    a.tol_dual = o.tol_dual;
    const int threads = o.threads > 0 ? o.threads : b->tuned_threads;
    a.check_every = o.check_every > 0 ? o.check_every : b->tuned_ce;
    if (threads == 32 && (sizeof(R) != 4 || !b->warp_ok))
        return bfail(FGA_EINVAL, "fga_mpc_batch_solve: threads 32 (one lane per step) needs FP32, 12 states, 4 "
                                 "inputs and horizons up to 64");
    if (threads != 32 && threads != 64 && threads != 128 && threads != 224 && threads != 256 && threads != 448 &&
        threads != 512)
        return bfail(FGA_EINVAL, "fga_mpc_batch_solve: threads must be 32, 64, 128, 224, 256, 448 or 512");
    int rc;
    BCUDA(cudaEventRecord(b->ev0, b->stream));
    if (o.use_graph) {
        const GraphKey key{threads, a.check_every, a.max_iters, a.tol_pri, a.tol_dual};
        auto it = b->graphs.find(key);
        if (it == b->graphs.end()) {
            cudaGraph_t graph;
            BCUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
            rc = launch_any<R>(b, a, threads, b->stream);
            cudaGraph_t captured = nullptr;
            cudaError_t ec = cudaStreamEndCapture(b->stream, &captured);
            if (rc) return rc;
            BCUDA(ec);
            graph = captured;
            cudaGraphExec_t exec;
            BCUDA(cudaGraphInstantiate(&exec, graph, 0));
            cudaGraphDestroy(graph);
            it = b->graphs.emplace(key, exec).first;
        }
        BCUDA(cudaGraphLaunch(it->second, b->stream));
    } else {
        if ((rc = launch_any<R>(b, a, threads, b->stream))) return rc;
    }
    BCUDA(cudaEventRecord(b->ev1, b->stream));
    BCUDA(cudaStreamSynchronize(b->stream));
    float ms = 0.f;
    BCUDA(cudaEventElapsedTime(&ms, b->ev0, b->ev1));
    std::vector<long long> iters((size_t)b->n);
    std::vector<int> st((size_t)b->n);
    BCUDA(cudaMemcpy(iters.data(), b->diters.p, iters.size() * sizeof(long long), cudaMemcpyDeviceToHost));
    BCUDA(cudaMemcpy(st.data(), b->dstatus.p, st.size() * sizeof(int), cudaMemcpyDeviceToHost));
    std::memset(&res, 0, sizeof res);
    for (int i = 0; i < b->n; ++i) {
        res.total_iters += iters[i];
        res.max_inst_iters = std::max<int64_t>(res.max_inst_iters, iters[i]);
        if (st[i] == 0) res.n_converged++;
        else if (st[i] == FGA_EBUDGET) res.n_budget++;
        else res.n_nonfinite++;
    }
    res.ms = ms;
    res.threads = threads;
    res.check_every = a.check_every;
    return FGA_OK;
}

extern "C" int fga_mpc_batch_solve(fga_mpc_batch *b, const fga_mpc_opts *opts, fga_mpc_result *res) {
    if (!b || !opts || !res) return bfail(FGA_EINVAL, "fga_mpc_batch_solve: NULL argument");
    if (!b->x0_set) return bfail(FGA_ESTATE, "fga_mpc_batch_solve: call fga_mpc_batch_set_x0 first");
    if (opts->max_iters < 0 || opts->tol_pri < 0 || opts->tol_dual < 0)
        return bfail(FGA_EINVAL, "fga_mpc_batch_solve: bad options");
    BCUDA(cudaSetDevice(b->device));
    fga_mpc_result r;
    int rc = b->precision == FGA_F32 ? solve_typed<float>(b, *opts, r) : solve_typed<double>(b, *opts, r);
    if (rc) return rc;
    *res = r;
    return FGA_OK;
}

template <typename R>
static int read_typed(fga_mpc_batch *b, double *z, double *u) {
    auto grab = [&](const Buf &src, long long n, double *dst) -> int {
        if (!dst) return FGA_OK;
        std::vector<R> h((size_t)n);
        BCUDA(cudaMemcpy(h.data(), src.p, (size_t)n * sizeof(R), cudaMemcpyDeviceToHost));
        for (long long i = 0; i < n; ++i) dst[i] = (double)h[i];
        return FGA_OK;
    };
    int rc;
    if ((rc = grab(b->dz, b->Z, z))) return rc;
    return grab(b->du, b->E, u);
}

extern "C" int fga_mpc_batch_read(fga_mpc_batch *b, double *z, double *u, int64_t *iters, int32_t *status,
                                  double *r_pri, double *r_dual) {
    if (!b) return bfail(FGA_EINVAL, "fga_mpc_batch_read: NULL batch");
    BCUDA(cudaSetDevice(b->device));
    BCUDA(cudaStreamSynchronize(b->stream));
    int rc = b->precision == FGA_F32 ? read_typed<float>(b, z, u) : read_typed<double>(b, z, u);
    if (rc) return rc;
    if (iters) BCUDA(cudaMemcpy(iters, b->diters.p, (size_t)b->n * sizeof(int64_t), cudaMemcpyDeviceToHost));
    if (status) BCUDA(cudaMemcpy(status, b->dstatus.p, (size_t)b->n * sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (r_pri) BCUDA(cudaMemcpy(r_pri, b->drp.p, (size_t)b->n * sizeof(double), cudaMemcpyDeviceToHost));
    if (r_dual) BCUDA(cudaMemcpy(r_dual, b->drd.p, (size_t)b->n * sizeof(double), cudaMemcpyDeviceToHost));
    return FGA_OK;
}

extern "C" int fga_mpc_batch_info(const fga_mpc_batch *b, int64_t *info, int32_t n) {
    if (!b || !info || n < 6) return bfail(FGA_EINVAL, "fga_mpc_batch_info: need an array of 6");
    info[0] = b->n;
    info[1] = b->E;
    info[2] = b->Z;
    info[3] = b->tmax;
    info[4] = b->tuned_threads;
    info[5] = b->tuned_ce;
    return FGA_OK;
}

// ---------------------------------------------------------------------------
// autotuner: times every (threads, check interval) candidate on the batch
// from its current start point and keeps the fastest; results are cached in
// a small text file keyed by problem shape, precision and GPU.
// ---------------------------------------------------------------------------
static std::string tune_key(const fga_mpc_batch *b, long long K, double tol) {
    cudaDeviceProp p;
    cudaGetDeviceProperties(&p, b->device);
    std::ostringstream k;
    k << "v3|" << p.name << "|sm" << p.major << p.minor << "|p" << b->precision << "|nx" << b->nx << "|nu" << b->nu << "|n"
      << b->n << "|tmax" << b->tmax << "|sys" << b->nsys << "|K" << K << "|tol" << tol;
    std::string s = k.str();
    for (char &c : s)
        if (c == ' ') c = '_';
    return s;
}

extern "C" int fga_mpc_batch_autotune(fga_mpc_batch *b, const char *cache_path, int64_t max_iters, double tol,
                                      int32_t *threads_out, int32_t *check_every_out) {
    if (!b) return bfail(FGA_EINVAL, "fga_mpc_batch_autotune: NULL batch");
    if (!b->x0_set) return bfail(FGA_ESTATE, "fga_mpc_batch_autotune: call fga_mpc_batch_set_x0 first");
    const std::string key = tune_key(b, max_iters, tol);
    if (cache_path) {
        std::ifstream in(cache_path);
        std::string k;
        int th, ce;
        double ms;
        while (in >> k >> th >> ce >> ms) {
            if (k == key) {
                b->tuned_threads = th;
                b->tuned_ce = ce;
                if (threads_out) *threads_out = th;
                if (check_every_out) *check_every_out = ce;
                return FGA_OK;
            }
        }
    }
    BCUDA(cudaSetDevice(b->device));
    // keep the start point: every candidate starts from it.  The copies go
    // on the batch's own stream (created non-blocking, so copies on the
    // legacy stream would not be ordered before the candidate's kernel and
    // a candidate could start from its predecessor's converged state).
    Buf z0, u0, x0;
    BCUDA(z0.alloc(b->dz.bytes));
    BCUDA(u0.alloc(b->du.bytes));
    BCUDA(x0.alloc(b->dx.bytes));
    auto copy_state = [&](bool save) -> int {
        const Buf *src[3] = {&b->dz, &b->du, &b->dx}, *dst[3] = {&z0, &u0, &x0};
        for (int i = 0; i < 3; ++i) {
            if (save) BCUDA(cudaMemcpyAsync(dst[i]->p, src[i]->p, src[i]->bytes, cudaMemcpyDeviceToDevice, b->stream));
            else BCUDA(cudaMemcpyAsync(src[i]->p, dst[i]->p, src[i]->bytes, cudaMemcpyDeviceToDevice, b->stream));
        }
        BCUDA(cudaStreamSynchronize(b->stream));
        return FGA_OK;
    };
    int rc;
    if ((rc = copy_state(true))) return rc;
    const int th_c[7] = {32, 64, 128, 224, 256, 448, 512};
    const int ce_c[4] = {1, 2, 5, 10};
    double best = std::numeric_limits<double>::infinity();
    int bt = 128, bc = 1;
    for (int th : th_c) {
        if (th == 32 && (b->precision != FGA_F32 || !b->warp_ok)) continue;
        for (int ce : ce_c) {
            fga_mpc_opts o;
            std::memset(&o, 0, sizeof o);
            o.max_iters = max_iters;
            o.tol_pri = o.tol_dual = tol;
            o.threads = th;
            o.check_every = ce;
            o.use_graph = 0;
            double tbest = std::numeric_limits<double>::infinity();
            bool finite = true;
            for (int rep = 0; rep < 2; ++rep) {
                if ((rc = copy_state(false))) return rc;
                fga_mpc_result r;
                rc = b->precision == FGA_F32 ? solve_typed<float>(b, o, r) : solve_typed<double>(b, o, r);
                if (rc) return rc;
                tbest = std::min(tbest, (double)r.ms);
                finite = finite && r.n_nonfinite == 0;
            }
            // a candidate whose solve produced a non-finite instance is not
            // a faster way to the same answer
            if (finite && tbest < best) {
                best = tbest;
                bt = th;
                bc = ce;
            }
        }
    }
    if ((rc = copy_state(false))) return rc;
    b->tuned_threads = bt;
    b->tuned_ce = bc;
    if (cache_path) {
        std::ofstream outf(cache_path, std::ios::app);
        outf << key << " " << bt << " " << bc << " " << best << "\n";
    }
    if (threads_out) *threads_out = bt;
    if (check_every_out) *check_every_out = bc;
    return FGA_OK;
}

extern "C" int fga_mpc_batch_destroy(fga_mpc_batch *b) {
    if (!b) return FGA_OK;
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return FGA_OK;
}
