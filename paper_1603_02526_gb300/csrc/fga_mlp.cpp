// fga_mlp.cpp -- host side of the warm-start MLP (C-ABI): parameters,
// buffers, forward, backward, Adam.  All arithmetic runs in mlp.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/fgadmm.h"
#include "mlp_internal.h"

using namespace fga;

int fga_set_last_error(int code, const char *msg);   // fga_graph.cpp

static int mfail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return fga_set_last_error(code, buf);
}

#define MCUDA(call)                                                                                  \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess)                                                                       \
            return mfail(e_ == cudaErrorMemoryAllocation ? FGA_ENOMEM : FGA_ECUDA, "%s: %s (%s:%d)", \
                         #call, cudaGetErrorString(e_), __FILE__, __LINE__);                         \
    } while (0)

namespace {
struct DBuf {
    void *p = nullptr;
    ~DBuf() {
        if (p) cudaFree(p);
    }
    cudaError_t alloc(size_t n) {
        if (p) cudaFree(p);
        p = nullptr;
        if (!n) return cudaSuccess;
        cudaError_t e = cudaMalloc(&p, n);
        if (e == cudaSuccess) e = cudaMemset(p, 0, n);
        return e;
    }
    template <typename T>
    T *as() const { return static_cast<T *>(p); }
};

// A host-to-device copy on the MLP's stream, finished before the host buffer
// can go away (a copy on the legacy stream would not be ordered before the
// kernels of a non-blocking stream).
static cudaError_t h2d(void *dst, const void *src, size_t bytes, cudaStream_t s) {
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
    return e == cudaSuccess ? cudaStreamSynchronize(s) : e;
}

// splitmix64 -> uniform (0, 1) -> standard normal (Box-Muller)
struct Rng {
    uint64_t s;
    uint64_t next() {
        uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        return z ^ (z >> 31);
    }
    double uni() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
    double normal() { return std::sqrt(-2.0 * std::log(uni())) * std::cos(6.283185307179586 * uni()); }
};

struct Layer {
    int rows = 0, cols = 0;       // W is rows x cols (out x in), row-major
    DBuf w, b, gw, gb, mw, vw, mb, vb, wb, wt;
};
}  // namespace

struct fga_mlp {
    int device = 0;
    cudaStream_t stream = nullptr;
    int in = 0, in_pad = 0, h1 = 0, h2 = 0, out = 0, max_batch = 0;
    Layer L[3];
    DBuf xb, a1, a2, y, dyf, dyb, d2, d1, loss_part, mean, stdv;
    DBuf err;                 // int: a tensor-core wait of a GEMM timed out
    DBuf ws;                  // split-K partials of the products of small batches
    long long ws_floats = 0;
    bool normalized = false;
    long long step = 0;
    int nparts = 256;
};

static int layer_alloc(Layer &l, int rows, int cols) {
    l.rows = rows;
    l.cols = cols;
    const size_t n = (size_t)rows * cols;
    MCUDA(l.w.alloc(n * 4));
    MCUDA(l.b.alloc((size_t)rows * 4));
    MCUDA(l.gw.alloc(n * 4));
    MCUDA(l.gb.alloc((size_t)rows * 4));
    MCUDA(l.mw.alloc(n * 4));
    MCUDA(l.vw.alloc(n * 4));
    MCUDA(l.mb.alloc((size_t)rows * 4));
    MCUDA(l.vb.alloc((size_t)rows * 4));
    MCUDA(l.wb.alloc(n * 2));
    MCUDA(l.wt.alloc(n * 2));
    return FGA_OK;
}

static int refresh_bf16(fga_mlp *m) {
    for (Layer &l : m->L) MCUDA(mlp_copy_bf16(l.w.as<float>(), l.rows, l.cols, l.wb.as<__nv_bfloat16>(),
                                              l.wt.as<__nv_bfloat16>(), m->stream));
    return FGA_OK;
}

extern "C" int fga_mlp_create(fga_mlp **outp, int32_t in, int32_t h1, int32_t h2, int32_t out, int32_t max_batch,
                              uint64_t seed, int32_t device, void *stream) {
    if (!outp) return mfail(FGA_EINVAL, "fga_mlp_create: out is NULL");
    if (in < 1 || h1 < 8 || h2 < 8 || out < 8 || max_batch < 8 || h1 % 8 || h2 % 8 || out % 8 || max_batch % 8)
        return mfail(FGA_EINVAL, "fga_mlp_create: sizes must be positive multiples of 8 (input any >= 1)");
    std::unique_ptr<fga_mlp> m(new (std::nothrow) fga_mlp());
    if (!m) return mfail(FGA_ENOMEM, "fga_mlp_create: out of memory");
    MCUDA(cudaSetDevice(device));
    m->device = device;
    m->stream = (cudaStream_t)stream;
    m->in = in;
    m->in_pad = (in + 15) / 16 * 16;
    m->h1 = h1;
    m->h2 = h2;
    m->out = out;
    m->max_batch = max_batch;
    int rc;
    if ((rc = layer_alloc(m->L[0], h1, m->in_pad)) || (rc = layer_alloc(m->L[1], h2, h1)) ||
        (rc = layer_alloc(m->L[2], out, h2)))
        return rc;
    const size_t B = (size_t)max_batch;
    MCUDA(m->xb.alloc(B * m->in_pad * 2));
    MCUDA(m->a1.alloc(B * h1 * 2));
    MCUDA(m->a2.alloc(B * h2 * 2));
    MCUDA(m->y.alloc(B * out * 4));
    MCUDA(m->dyf.alloc(B * out * 4));
    MCUDA(m->dyb.alloc(B * out * 2));
    MCUDA(m->d2.alloc(B * h2 * 2));
    MCUDA(m->d1.alloc(B * h1 * 2));
    MCUDA(m->loss_part.alloc((size_t)m->nparts * 8));
    MCUDA(m->mean.alloc((size_t)out * 4));
    MCUDA(m->stdv.alloc((size_t)out * 4));
    MCUDA(m->err.alloc(sizeof(int)));
    {
        const long long mn = std::max<long long>(std::max<long long>((long long)out * h2, (long long)h2 * h1),
                                                 (long long)h1 * m->in_pad);
        m->ws_floats = 16 * mn;
        MCUDA(m->ws.alloc((size_t)m->ws_floats * sizeof(float)));
    }
    // He initialisation (seeded), zero biases, zero padding columns
    Rng rng{seed};
    int dims[3][2] = {{h1, in}, {h2, h1}, {out, h2}};
    for (int li = 0; li < 3; ++li) {
        Layer &l = m->L[li];
        std::vector<float> w((size_t)l.rows * l.cols, 0.f);
        const double sd = std::sqrt(2.0 / dims[li][1]);
        for (int r = 0; r < l.rows; ++r)
            for (int c = 0; c < dims[li][1]; ++c) w[(size_t)r * l.cols + c] = (float)(sd * rng.normal());
        MCUDA(h2d(l.w.p, w.data(), w.size() * 4, m->stream));
    }
    std::vector<float> ones((size_t)out, 1.f);
    MCUDA(h2d(m->stdv.p, ones.data(), ones.size() * 4, m->stream));
    if ((rc = refresh_bf16(m.get()))) return rc;
    MCUDA(cudaDeviceSynchronize());
    *outp = m.release();
    return FGA_OK;
}

extern "C" int fga_mlp_num_params(const fga_mlp *m, int64_t *n) {
    if (!m || !n) return mfail(FGA_EINVAL, "fga_mlp_num_params: NULL argument");
    *n = (int64_t)m->h1 * m->in + m->h1 + (int64_t)m->h2 * m->h1 + m->h2 + (int64_t)m->out * m->h2 + m->out;
    return FGA_OK;
}

// packed order: W1 (h1 x in), b1, W2 (h2 x h1), b2, W3 (out x h2), b3
static int copy_params(fga_mlp *m, float *host, bool to_device, bool grads) {
    const int in_cols[3] = {m->in, m->h1, m->h2};
    size_t off = 0;
    for (int li = 0; li < 3; ++li) {
        Layer &l = m->L[li];
        float *dw = grads ? l.gw.as<float>() : l.w.as<float>();
        float *db = grads ? l.gb.as<float>() : l.b.as<float>();
        std::vector<float> w((size_t)l.rows * l.cols, 0.f);
        if (!to_device) MCUDA(cudaMemcpy(w.data(), dw, w.size() * 4, cudaMemcpyDeviceToHost));
        for (int r = 0; r < l.rows; ++r)
            for (int c = 0; c < in_cols[li]; ++c) {
                if (to_device) w[(size_t)r * l.cols + c] = host[off + (size_t)r * in_cols[li] + c];
                else host[off + (size_t)r * in_cols[li] + c] = w[(size_t)r * l.cols + c];
            }
        if (to_device) MCUDA(h2d(dw, w.data(), w.size() * 4, m->stream));
        off += (size_t)l.rows * in_cols[li];
        if (to_device) MCUDA(h2d(db, host + off, (size_t)l.rows * 4, m->stream));
        else MCUDA(cudaMemcpy(host + off, db, (size_t)l.rows * 4, cudaMemcpyDeviceToHost));
        off += l.rows;
    }
    return FGA_OK;
}

extern "C" int fga_mlp_set_params(fga_mlp *m, const float *params, int64_t n) {
    int64_t want;
    if (!m || !params) return mfail(FGA_EINVAL, "fga_mlp_set_params: NULL argument");
    fga_mlp_num_params(m, &want);
    if (n != want) return mfail(FGA_EINVAL, "fga_mlp_set_params: %lld values, want %lld", (long long)n, (long long)want);
    MCUDA(cudaSetDevice(m->device));
    int rc = copy_params(m, const_cast<float *>(params), true, false);
    if (rc) return rc;
    if ((rc = refresh_bf16(m))) return rc;
    MCUDA(cudaStreamSynchronize(m->stream));
    return FGA_OK;
}

extern "C" int fga_mlp_get_params(fga_mlp *m, float *params, int64_t n) {
    int64_t want;
    if (!m || !params) return mfail(FGA_EINVAL, "fga_mlp_get_params: NULL argument");
    fga_mlp_num_params(m, &want);
    if (n != want) return mfail(FGA_EINVAL, "fga_mlp_get_params: %lld values, want %lld", (long long)n, (long long)want);
    MCUDA(cudaSetDevice(m->device));
    MCUDA(cudaStreamSynchronize(m->stream));
    return copy_params(m, params, false, false);
}

extern "C" int fga_mlp_fit_normalization(fga_mlp *m, float *Y, int64_t rows) {
    if (!m || !Y || rows < 2) return mfail(FGA_EINVAL, "fga_mlp_fit_normalization: bad argument");
    MCUDA(cudaSetDevice(m->device));
    MCUDA(mlp_col_stats(Y, rows, m->out, m->mean.as<float>(), m->stdv.as<float>(), m->stream));
    MCUDA(cudaStreamSynchronize(m->stream));
    m->normalized = true;
    return FGA_OK;
}

extern "C" int fga_mlp_get_normalization(fga_mlp *m, float *mean, float *stdv) {
    if (!m) return mfail(FGA_EINVAL, "fga_mlp_get_normalization: NULL");
    MCUDA(cudaSetDevice(m->device));
    MCUDA(cudaStreamSynchronize(m->stream));
    if (mean) MCUDA(cudaMemcpy(mean, m->mean.p, (size_t)m->out * 4, cudaMemcpyDeviceToHost));
    if (stdv) MCUDA(cudaMemcpy(stdv, m->stdv.p, (size_t)m->out * 4, cudaMemcpyDeviceToHost));
    return FGA_OK;
}

static GemmEpi epi0(fga_mlp *m) {
    GemmEpi e;
    std::memset(&e, 0, sizeof e);
    e.err = m->err.as<int>();
    e.ws = m->ws.as<float>();        // split-K partials (products of small batches)
    e.ws_floats = m->ws_floats;
    return e;
}

// After a stream synchronisation: FGA_ETIMEOUT (and the word cleared) if a
// GEMM since the last check gave up waiting for its tensor-core work.
static int check_gemm_err(fga_mlp *m) {
    int h = 0;
    MCUDA(cudaMemcpy(&h, m->err.p, sizeof h, cudaMemcpyDeviceToHost));
    if (h) {
        MCUDA(cudaMemsetAsync(m->err.p, 0, sizeof(int), m->stream));
        MCUDA(cudaStreamSynchronize(m->stream));
        return mfail(FGA_ETIMEOUT, "MLP GEMM: a tensor-core wait timed out; outputs are not valid");
    }
    return FGA_OK;
}

// forward through the three layers; last = output epilogue
static int forward(fga_mlp *m, const float *X, int B, int last_epi, float *yout) {
    cudaStream_t s = m->stream;
    const __nv_bfloat16 *xb = m->xb.as<__nv_bfloat16>();
    MCUDA(mlp_to_bf16_pad(X, B, m->in, m->in_pad, m->xb.as<__nv_bfloat16>(), s));
    GemmEpi e = epi0(m);
    e.bias = m->L[0].b.as<float>();
    e.outb = m->a1.as<__nv_bfloat16>();
    e.ldc = m->h1;
    MCUDA(mlp_gemm(3, EPI_BIAS_RELU, B, m->h1, m->in_pad, xb, m->in_pad, m->L[0].wb.as<__nv_bfloat16>(), m->in_pad,
                   e, s));
    e = epi0(m);
    e.bias = m->L[1].b.as<float>();
    e.outb = m->a2.as<__nv_bfloat16>();
    e.ldc = m->h2;
    MCUDA(mlp_gemm(3, EPI_BIAS_RELU, B, m->h2, m->h1, m->a1.as<__nv_bfloat16>(), m->h1,
                   m->L[1].wb.as<__nv_bfloat16>(), m->h1, e, s));
    e = epi0(m);
    e.bias = m->L[2].b.as<float>();
    e.scale = m->stdv.as<float>();
    e.shift = m->mean.as<float>();
    e.outf = yout;
    e.ldc = m->out;
    MCUDA(mlp_gemm(3, last_epi, B, m->out, m->h2, m->a2.as<__nv_bfloat16>(), m->h2, m->L[2].wb.as<__nv_bfloat16>(),
                   m->h2, e, s));
    return FGA_OK;
}

// loss + gradients of every parameter into the layers' g* buffers
static int backward(fga_mlp *m, const float *X, const float *T, int B, double *loss) {
    cudaStream_t s = m->stream;
    int rc = forward(m, X, B, EPI_BIAS, m->y.as<float>());
    if (rc) return rc;
    const long long n = (long long)B * m->out;
    MCUDA(mlp_mse(m->y.as<float>(), T, n, 1.0f / (float)n, m->dyf.as<float>(), m->dyb.as<__nv_bfloat16>(),
                  m->loss_part.as<double>(), m->nparts, s));
    const __nv_bfloat16 *dyb = m->dyb.as<__nv_bfloat16>();
    // layer 3
    GemmEpi e = epi0(m);
    e.outf = m->L[2].gw.as<float>();
    e.ldc = m->h2;
    MCUDA(mlp_gemm(0, EPI_STORE, m->out, m->h2, B, dyb, m->out, m->a2.as<__nv_bfloat16>(), m->h2, e, s));
    MCUDA(mlp_colsum_f32(m->dyf.as<float>(), B, m->out, m->L[2].gb.as<float>(), s));
    e = epi0(m);
    e.mask = m->a2.as<__nv_bfloat16>();
    e.ldm = m->h2;
    e.outb = m->d2.as<__nv_bfloat16>();
    e.ldc = m->h2;
    MCUDA(mlp_gemm(3, EPI_RELU_MASK, B, m->h2, m->out, dyb, m->out, m->L[2].wt.as<__nv_bfloat16>(), m->out, e, s));
    // layer 2
    e = epi0(m);
    e.outf = m->L[1].gw.as<float>();
    e.ldc = m->h1;
    MCUDA(mlp_gemm(0, EPI_STORE, m->h2, m->h1, B, m->d2.as<__nv_bfloat16>(), m->h2, m->a1.as<__nv_bfloat16>(), m->h1,
                   e, s));
    MCUDA(mlp_colsum_bf16(m->d2.as<__nv_bfloat16>(), B, m->h2, m->L[1].gb.as<float>(), s));
    e = epi0(m);
    e.mask = m->a1.as<__nv_bfloat16>();
    e.ldm = m->h1;
    e.outb = m->d1.as<__nv_bfloat16>();
    e.ldc = m->h1;
    MCUDA(mlp_gemm(3, EPI_RELU_MASK, B, m->h1, m->h2, m->d2.as<__nv_bfloat16>(), m->h2, m->L[1].wt.as<__nv_bfloat16>(),
                   m->h2, e, s));
    // layer 1
    e = epi0(m);
    e.outf = m->L[0].gw.as<float>();
    e.ldc = m->in_pad;
    MCUDA(mlp_gemm(0, EPI_STORE, m->h1, m->in_pad, B, m->d1.as<__nv_bfloat16>(), m->h1, m->xb.as<__nv_bfloat16>(),
                   m->in_pad, e, s));
    MCUDA(mlp_colsum_bf16(m->d1.as<__nv_bfloat16>(), B, m->h1, m->L[0].gb.as<float>(), s));
    if (loss) {
        std::vector<double> lp((size_t)m->nparts);
        MCUDA(cudaMemcpyAsync(lp.data(), m->loss_part.p, lp.size() * 8, cudaMemcpyDeviceToHost, s));
        MCUDA(cudaStreamSynchronize(s));
        double t = 0.0;
        for (double v : lp) t += v;
        *loss = t / (double)n;
    }
    return FGA_OK;
}

static int check_batch(const fga_mlp *m, int B) {
    if (B < 8 || B > m->max_batch || B % 8) return mfail(FGA_EINVAL, "batch %d: need a multiple of 8 <= %d", B, m->max_batch);
    return FGA_OK;
}

extern "C" int fga_mlp_gradients(fga_mlp *m, const float *X, const float *Y, int32_t batch, float *grads,
                                 double *loss) {
    if (!m || !X || !Y || !grads) return mfail(FGA_EINVAL, "fga_mlp_gradients: NULL argument");
    int rc = check_batch(m, batch);
    if (rc) return rc;
    MCUDA(cudaSetDevice(m->device));
    if ((rc = backward(m, X, Y, batch, loss))) return rc;
    MCUDA(cudaStreamSynchronize(m->stream));
    if ((rc = check_gemm_err(m))) return rc;
    return copy_params(m, grads, false, true);
}

extern "C" int fga_mlp_train_step(fga_mlp *m, const float *X, const float *Y, int32_t batch, float lr, double *loss) {
    if (!m || !X || !Y) return mfail(FGA_EINVAL, "fga_mlp_train_step: NULL argument");
    int rc = check_batch(m, batch);
    if (rc) return rc;
    MCUDA(cudaSetDevice(m->device));
    if ((rc = backward(m, X, Y, batch, loss))) return rc;
    if (loss && (rc = check_gemm_err(m))) return rc;   // the loss read synchronised the stream
    m->step += 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - std::pow(b1, (float)m->step), c2 = 1.f - std::pow(b2, (float)m->step);
    for (Layer &l : m->L) {
        MCUDA(mlp_adam(l.w.as<float>(), l.mw.as<float>(), l.vw.as<float>(), l.gw.as<float>(), l.rows, l.cols, lr, b1,
                       b2, eps, c1, c2, l.wb.as<__nv_bfloat16>(), l.wt.as<__nv_bfloat16>(), m->stream));
        MCUDA(mlp_adam(l.b.as<float>(), l.mb.as<float>(), l.vb.as<float>(), l.gb.as<float>(), l.rows, 1, lr, b1, b2,
                       eps, c1, c2, nullptr, nullptr, m->stream));
    }
    return FGA_OK;
}

extern "C" int fga_mlp_forward(fga_mlp *m, const float *X, float *Y, int32_t batch) {
    if (!m || !X || !Y) return mfail(FGA_EINVAL, "fga_mlp_forward: NULL argument");
    int rc = check_batch(m, batch);
    if (rc) return rc;
    MCUDA(cudaSetDevice(m->device));
    if ((rc = forward(m, X, batch, EPI_BIAS_DENORM, Y))) return rc;
    MCUDA(cudaStreamSynchronize(m->stream));
    return check_gemm_err(m);
}

extern "C" int fga_mlp_destroy(fga_mlp *m) {
    if (!m) return FGA_OK;
    cudaSetDevice(m->device);
    cudaStreamSynchronize(m->stream);
    delete m;
    return FGA_OK;
}
