// mpc_noalloc.cu -- a batched MPC solve that allocates no memory.
//
// Some callers cannot call cudaMalloc at solve time: code running inside a
// memory pool or arena they do not own, real-time control loops that must
// not touch the allocator after start-up, and plugins whose host process
// forbids device allocations.  fga_mpc_solve_noalloc serves them: it runs
// the same batched solver kernel as fga_mpc_batch_solve for instances of
// one shared system, but every byte of scratch it needs (the per-edge x and
// u, instance offsets, the dynamics projector, residuals, the work counter)
// lives in one file-scope device array of kNoAllocBytes.  The caller passes
// only inputs and outputs.  The array exists on every GPU that loads the
// library, for the life of the process.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "../../include/fgadmm.h"
#include "mpc_internal.h"

int fga_set_last_error(int code, const char *msg);   // fga_graph.cpp

namespace fga {

constexpr size_t kNoAllocBytes = (size_t)16 << 20;   // 16 MiB of scratch per device
constexpr int kNoAllocMaxInst = 4096;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {

// host-side device address of g_noalloc_scratch, per device, looked up by
// the first call on that device.  Threads that race on the first call store
// the same value.  The address belongs to the device's current context: the
// library must not be used across a cudaDeviceReset (the module may load
// again at another address).
std::atomic<unsigned char *> g_scratch_ptr[kNoAllocMaxDevices] = {};

int nfail(int code, const char *fmt, ...) {
    char buf[384];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return fga_set_last_error(code, buf);
}

size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

// Projector onto {v : M v = 0}, M = [A B -I], uniform rho:
// P = I - M^T (M M^T)^{-1} M, in FP64 by one CTA (Gauss-Jordan on M M^T in
// shared memory), written as FP32.
// A non-finite A or B, or a zero pivot, sets *bad (the solve then reports
// FGA_EINVAL for every instance, as the allocating path refuses the system).
__global__ void k_projector(const float *A, const float *B, int nx, int nu, float *P, int *bad) {
    extern __shared__ double sh[];
    const int n = 2 * nx + nu;
    double *M = sh;                       // nx x n
    double *G = M + nx * n;               // nx x 2nx  [M M^T | I]
    double *T = G + nx * 2 * nx;          // nx x n    (M M^T)^{-1} M
    for (int i = threadIdx.x; i < nx * n; i += blockDim.x) {
        const int r = i / n, c = i % n;
        double v;
        if (c < nx) v = A[r * nx + c];
        else if (c < nx + nu) v = B[r * nu + (c - nx)];
        else v = (c - nx - nu == r) ? -1.0 : 0.0;
        M[i] = v;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nx * nx; i += blockDim.x) {
        const int r = i / nx, k = i % nx;
        double t = 0.0;
        for (int j = 0; j < n; ++j) t += M[r * n + j] * M[k * n + j];
        G[r * 2 * nx + k] = t;
        G[r * 2 * nx + nx + k] = (r == k) ? 1.0 : 0.0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        *bad = 0;
        for (int c = 0; c < nx; ++c) {
            int piv = c;
            for (int r = c + 1; r < nx; ++r)
                if (fabs(G[r * 2 * nx + c]) > fabs(G[piv * 2 * nx + c])) piv = r;
            if (piv != c)
                for (int j = 0; j < 2 * nx; ++j) {
                    const double t = G[c * 2 * nx + j];
                    G[c * 2 * nx + j] = G[piv * 2 * nx + j];
                    G[piv * 2 * nx + j] = t;
                }
            const double d = G[c * 2 * nx + c];
            if (!(fabs(d) > 0.0) || !isfinite(d)) {
                *bad = 1;
                break;
            }
            for (int j = 0; j < 2 * nx; ++j) G[c * 2 * nx + j] /= d;
            for (int r = 0; r < nx; ++r) {
                if (r == c) continue;
                const double f = G[r * 2 * nx + c];
                for (int j = 0; j < 2 * nx; ++j) G[r * 2 * nx + j] -= f * G[c * 2 * nx + j];
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nx * n; i += blockDim.x) {
        const int r = i / n, j = i % n;
        double t = 0.0;
        for (int k = 0; k < nx; ++k) t += G[r * 2 * nx + nx + k] * M[k * n + j];
        T[i] = t;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
        const int r = i / n, c = i % n;
        double t = 0.0;
        for (int k = 0; k < nx; ++k) t += M[k * n + r] * T[k * n + c];
        P[i] = (float)((r == c ? 1.0 : 0.0) - t);
    }
}

// The horizons travel as a kernel parameter (16 KB, within the 32 KB
// parameter limit): the launch copies them from the caller's array while the
// call runs, so a later change to that array, or a replay of a captured
// launch, cannot make the device tables disagree with the sizes the host
// checked against the scratch array.
struct HorizonTable {
    int T[kNoAllocMaxInst];
};
static_assert(sizeof(HorizonTable) <= 32000, "kernel parameter limit");

// horizons into scratch, instance offsets (prefix sums of the per-instance
// sizes), identity hand-out order, every instance on system 0
__global__ void k_offsets(const HorizonTable tbl, int n, int nx, int nu, int *T, long long *zoff,
                          long long *eoff, int *order, int *sys) {
    if (threadIdx.x == 0) {
        long long z = 0, e = 0;
        for (int i = 0; i < n; ++i) {
            zoff[i] = z;
            eoff[i] = e;
            z += (long long)(nx + nu) * tbl.T[i] + nx;
            e += 2LL * nx + 3LL * (nx + nu) * tbl.T[i];
        }
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        T[i] = tbl.T[i];
        order[i] = i;
        sys[i] = 0;
    }
}

// after the solve: a refused system overrides every instance's status
__global__ void k_system_status(const int *bad, int n, int *status) {
    if (*bad == 0) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) status[i] = FGA_EINVAL;
}

}  // namespace
}  // namespace fga

using namespace fga;

extern "C" int fga_mpc_solve_noalloc(int32_t n_inst, const int32_t *T, int32_t nx, int32_t nu, const float *A,
                                     const float *B, const float *q, const float *r, const float *x0, float umax,
                                     float rho, float alpha, int64_t max_iters, double tol, int32_t check_every,
                                     float *z_out, int64_t *iters_out, int32_t *status_out, void *stream) {
    if (!T || !A || !B || !q || !r || !x0 || !z_out || !iters_out || !status_out)
        return nfail(FGA_EINVAL, "fga_mpc_solve_noalloc: NULL argument");
    if (n_inst < 1 || n_inst > kNoAllocMaxInst)
        return nfail(FGA_EINVAL, "fga_mpc_solve_noalloc: n_inst %d outside [1, %d]", n_inst, kNoAllocMaxInst);
    if (nx < 1 || nu < 1 || 2 * nx + nu > 64 || nx > 32)
        return nfail(FGA_EINVAL, "fga_mpc_solve_noalloc: need 1 <= nx <= 32, nu >= 1, 2 nx + nu <= 64");
    if (!(umax > 0.f) || !(rho > 0.f) || !(alpha > 0.f) || max_iters < 0 || !(tol >= 0.0) || check_every < 1)
        return nfail(FGA_EINVAL, "fga_mpc_solve_noalloc: bad scalar argument");
    // one read of the caller's horizons: the checks below and the launch
    // parameter use this copy
    HorizonTable tbl;
    std::memcpy(tbl.T, T, (size_t)n_inst * sizeof(int));
    long long E = 0, Z = 0;
    int tmax = 0;
    for (int i = 0; i < n_inst; ++i) {
        const int t = tbl.T[i];
        if (t < 1 || t > 100000) return nfail(FGA_EINVAL, "fga_mpc_solve_noalloc: horizon %d", t);
        E += 2LL * nx + 3LL * (nx + nu) * t;
        Z += (long long)(nx + nu) * t + nx;
        tmax = t > tmax ? t : tmax;
    }
    (void)Z;
    const int Ad = 2 * nx + nu;
    // scratch layout (256-byte aligned pieces)
    size_t off = 0;
    const size_t o_queue = off;
    off = up256(off + sizeof(unsigned));
    const size_t o_bad = off;
    off = up256(off + sizeof(int));
    const size_t o_P = off;
    off = up256(off + (size_t)Ad * Ad * sizeof(float));
    const size_t o_T = off;
    off = up256(off + (size_t)n_inst * sizeof(int));
    const size_t o_zoff = off;
    off = up256(off + (size_t)n_inst * sizeof(long long));
    const size_t o_eoff = off;
    off = up256(off + (size_t)n_inst * sizeof(long long));
    const size_t o_order = off;
    off = up256(off + (size_t)n_inst * sizeof(int));
    const size_t o_sys = off;
    off = up256(off + (size_t)n_inst * sizeof(int));
    const size_t o_rp = off;
    off = up256(off + (size_t)n_inst * sizeof(double));
    const size_t o_rd = off;
    off = up256(off + (size_t)n_inst * sizeof(double));
    const size_t o_x = off;
    off = up256(off + (size_t)E * sizeof(float));
    const size_t o_u = off;
    off = up256(off + (size_t)E * sizeof(float));
    if (off > kNoAllocBytes)
        return nfail(FGA_EINVAL,
                     "fga_mpc_solve_noalloc: the batch needs %zu bytes of scratch, the static array holds %zu "
                     "(%lld scalar edges; at most about %zu)",
                     off, kNoAllocBytes, E, kNoAllocBytes / 8);
    // set-up, once per device: the device address of the scratch array
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return nfail(FGA_ECUDA, "fga_mpc_solve_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return nfail(FGA_EINVAL, "fga_mpc_solve_noalloc: device %d", dev);
    unsigned char *s = g_scratch_ptr[dev].load(std::memory_order_acquire);
    if (!s) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr)
            return nfail(FGA_ECUDA, "fga_mpc_solve_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        s = static_cast<unsigned char *>(ptr);
        g_scratch_ptr[dev].store(s, std::memory_order_release);
    }
    cudaStream_t st = (cudaStream_t)stream;
    // inputs into scratch, derived tables, and the cold start (z, u, x = 0);
    // the array keeps the previous call's contents, so all of it is rewritten
#define NA_TRY(call)                                                                                        \
    do {                                                                                                    \
        cudaError_t e_ = (call);                                                                            \
        if (e_ != cudaSuccess) return nfail(FGA_ECUDA, "fga_mpc_solve_noalloc: %s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)
    const int psm = (nx * Ad + 2 * nx * nx + nx * Ad) * (int)sizeof(double);
    k_projector<<<1, 128, psm, st>>>(A, B, nx, nu, reinterpret_cast<float *>(s + o_P),
                                     reinterpret_cast<int *>(s + o_bad));
    NA_TRY(cudaGetLastError());
    k_offsets<<<1, 256, 0, st>>>(tbl, n_inst, nx, nu, reinterpret_cast<int *>(s + o_T),
                                 reinterpret_cast<long long *>(s + o_zoff), reinterpret_cast<long long *>(s + o_eoff),
                                 reinterpret_cast<int *>(s + o_order), reinterpret_cast<int *>(s + o_sys));
    NA_TRY(cudaGetLastError());
    NA_TRY(cudaMemsetAsync(z_out, 0, (size_t)Z * sizeof(float), st));
    NA_TRY(cudaMemsetAsync(s + o_x, 0, (size_t)E * sizeof(float), st));
    NA_TRY(cudaMemsetAsync(s + o_u, 0, (size_t)E * sizeof(float), st));
    NA_TRY(cudaMemsetAsync(s + o_queue, 0, sizeof(unsigned), st));
    MpcArgs<float> a;
    std::memset(&a, 0, sizeof a);
    a.n_inst = n_inst;
    a.nx = nx;
    a.nu = nu;
    a.T = reinterpret_cast<const int *>(s + o_T);
    a.zoff = reinterpret_cast<const long long *>(s + o_zoff);
    a.eoff = reinterpret_cast<const long long *>(s + o_eoff);
    a.sys = reinterpret_cast<const int *>(s + o_sys);
    a.order = reinterpret_cast<const int *>(s + o_order);
    a.P = reinterpret_cast<const float *>(s + o_P);
    a.q = q;
    a.r = r;
    a.x0 = x0;
    a.lo = -umax;
    a.hi = umax;
    a.rho = rho;
    a.alpha = alpha;
    a.z = z_out;
    a.u = reinterpret_cast<float *>(s + o_u);
    a.x = reinterpret_cast<float *>(s + o_x);
    a.iters = reinterpret_cast<long long *>(iters_out);
    a.status = status_out;
    a.rpri = reinterpret_cast<double *>(s + o_rp);
    a.rdual = reinterpret_cast<double *>(s + o_rd);
    a.queue = reinterpret_cast<unsigned *>(s + o_queue);
    a.max_iters = max_iters;
    a.tol_pri = tol;
    a.tol_dual = tol;
    a.check_every = check_every;
    a.first_pending = 0;
    const int threads = 128;
    const int smem = mpc_smem_bytes((int)sizeof(float), nx, nu, tmax, threads);
    const int bps = mpc_max_blocks_per_sm<float>(threads, smem);
    if (bps < 1) return nfail(FGA_EINVAL, "fga_mpc_solve_noalloc: horizon %d does not fit in shared memory", tmax);
    int sms = 0;
    NA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = n_inst < bps * sms ? n_inst : bps * sms;
    NA_TRY(mpc_launch<float>(a, threads, grid, smem, st));
    k_system_status<<<(n_inst + 255) / 256, 256, 0, st>>>(reinterpret_cast<const int *>(s + o_bad), n_inst,
                                                          status_out);
    NA_TRY(cudaGetLastError());
#undef NA_TRY
    return FGA_OK;
}
