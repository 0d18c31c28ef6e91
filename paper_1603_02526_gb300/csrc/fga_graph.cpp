// fga_graph.cpp -- host side of libfgadmm: graph building (the paper's
// addNode, by type), layout for the GPU and upload (the paper's
// CopyGraphFromCPUtoGPU), iteration driver, readout, and the C-ABI.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <limits>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/fgadmm.h"
#include "fga_internal.h"
#include "fga_host.h"
#include "tile_internal.h"
#include "hinge_internal.h"
#include "user_internal.h"

using namespace fga;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string t_last_error;

static int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_last_error = buf;
    return code;
}

#define CUDA_TRY(call)                                                                       \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail(e_ == cudaErrorMemoryAllocation ? FGA_ENOMEM : FGA_ECUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                  \
    } while (0)

extern "C" const char *fga_last_error(void) { return t_last_error.c_str(); }

// shared with the batch layer (fga_batch.cpp)
int fga_set_last_error(int code, const char *msg) {
    t_last_error = msg;
    return code;
}
extern "C" const char *fga_version(void) { return "fgadmm-gb300 0.1 (sm_103a)"; }

// ---------------------------------------------------------------------------
// device buffers
// ---------------------------------------------------------------------------
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    cudaError_t alloc(size_t n) {
        release();
        bytes = n;
        if (n == 0) return cudaSuccess;
        return cudaMalloc(&p, n);
    }
    template <typename T>
    T *as() const { return static_cast<T *>(p); }
};

// ---------------------------------------------------------------------------
// the graph
// ---------------------------------------------------------------------------
struct FactorBatch {
    int type = 0;
    int64_t count = 0;
    int nv = 0;
    std::vector<int64_t> vars;     // count * nv
    std::vector<double> params;    // count * np, or np when shared
    int np = 0;
    bool shared = false;
    int64_t edge0 = 0;             // first creation-order edge
    int arity = 0;
    std::vector<int> dims;         // nv
    const double *param(int64_t f) const { return params.data() + (shared ? 0 : f * np); }
};

struct Bucket {
    int type = 0;
    std::vector<int> dims;
    int np = 0;
    int arity = 0;
    std::vector<std::pair<int, int64_t>> members;   // (batch, factor in batch), creation order
    int64_t ebase = 0, item0 = 0, nitems = 0;
    bool per_edge = false;
    bool aos = false;      // factor-major storage of the bucket's edges
    int prm_buf = -1;      // its parameters in bucket_bufs
};

// A bucket of a user-supplied operator: per edge (factor-major) its scalar
// variable and the slot of its rho m in the z-reduction's input.
struct UserBucket {
    int bucket = 0, user = 0;
    DevBuf var, dst;
};

struct fga_graph {
    int precision = FGA_F64;
    int device = 0;
    cudaStream_t stream = nullptr;
    int zorder = -1, store_m = -1, block = 0;

    std::vector<int32_t> vdim;
    std::vector<int64_t> voff;
    int64_t nz = 0;

    std::vector<FactorBatch> batches;
    int64_t nfac = 0, ne = 0;

    double rho_u = 1.0, alpha_u = 1.0;
    std::vector<double> rho_c, alpha_c;   // per edge, creation order (empty = uniform)

    bool finalized = false;
    bool initialized = false;

    // layout (host)
    std::vector<Bucket> buckets;
    std::vector<int64_t> s2c;       // storage -> creation (-1 for alignment padding)
    int64_t es = 0;                 // storage slots (edges + padding)
    std::vector<int32_t> svar;      // storage order
    int64_t nitems_f = 0;

    // device
    DevBuf x[2], m[2], u, rho_e, alpha_e, d_svar, d_pos, pvm, z[2], srho, srho2, row;
    DevBuf small_vars, witems, hub_np, hub_off, hub_part, hub_ticket;
    DevBuf res_pri, res_dual, ctl, bar;
    std::vector<std::unique_ptr<DevBuf>> bucket_bufs;
    int n_small = 0, n_witems = 0, n_hubs = 0;
    DevBuf chunks, slot_var, ppos, lrow, lidx, part, prow;
    int nchunks = 0, smem = 0, bps = 0, kind = 0;
    // scatter order (zorder 4): per-edge variable | column words, the
    // overflow flags per variable, the column count and overflow entries
    DevBuf d_ev, zovf;
    int colw = 0;
    int64_t novf = 0;
    // disk-tile order (zorder 2): the plan and its device copies
    TilePlan tile;
    DevBuf t_cta, t_rowslot, t_colslot, t_mask, t_sv, t_zden, t_cptr, t_clist, t_loc, t_part, t_res, t_dsave;
    DevBuf t_dres, t_zprev, t_lres, t_dlive;
    // hinge bank (zorder 3)
    HingePlan hinge;
    HingeInput hin;
    DevBuf h_cta, h_X, h_meta, h_gsave, h_gres, h_l2save, h_l2res, h_acc;
    int64_t hinge_e0 = 0, l2_e0 = 0, l2_nf = 0;
    bool tile_resume = false;   // alpha = 1: the last call left its displacements to resume from
    int64_t tile_pair_ebase = 0;
    bool uniform_rho = true, uniform_alpha = true;
    int grid = 1, blk = 256;
    // shard mode (fga_shard_*): srho / srho2 hold the graph-wide sums; the
    // u-update of the last z-step is pending until the next x-step
    bool shard = false, shard_pending = false;
    // weight mode (FGA_OPT_WEIGHTS): 1 = three weights (canonical order)
    int weights = 0;
    DevBuf wcls, pwcls, prho;
    DevBuf shard_res;   // per-CTA dual partials of the z-step (fixed grid: equal on every rank)
    // user-supplied operators (fga_register_prox) and their buckets
    std::vector<UserProg> users;
    std::vector<std::unique_ptr<UserBucket>> ubk;
    bool has_user() const { return !ubk.empty(); }

    // state
    int64_t iters_done = 0;
    int xpar = 0, zpar = 0;
    double last_rp = std::numeric_limits<double>::quiet_NaN();
    double last_rd = std::numeric_limits<double>::quiet_NaN();
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;

    size_t rsize() const { return precision == FGA_F32 ? sizeof(float) : sizeof(double); }
};

static int set_device(const fga_graph *g) {
    CUDA_TRY(cudaSetDevice(g->device));
    return FGA_OK;
}

// Expected number of parameters for a factor of `type` with variable
// dimensions `dims` (-1 if the shape is invalid for the type).
static int expected_params(int type, const std::vector<int> &dims, int arity) {
    const int nv = (int)dims.size();
    switch (type) {
    case FGA_PACK_PAIR:
        return (nv == 4 && dims[0] == 2 && dims[1] == 1 && dims[2] == 2 && dims[3] == 1) ? 0 : -1;
    case FGA_PACK_WALL:
        return (nv == 2 && dims[0] == 2 && dims[1] == 1) ? 4 : -1;
    case FGA_PACK_RADIUS_LIN:
        return (nv == 1 && dims[0] == 1) ? 1 : -1;
    case FGA_PACK_RADIUS_QUAD:
        return (nv == 1 && dims[0] == 1) ? 0 : -1;
    case FGA_SVM_HINGE:
        return (nv == 2 && dims[1] == 1) ? dims[0] + 2 : -1;
    case FGA_SVM_L2:
        return nv == 1 ? 1 : -1;
    case FGA_MPC_DYN:
        return (nv == 3 && dims[0] == dims[2] && 2 * dims[0] + dims[1] <= 64) ? dims[0] * dims[0] + dims[0] * dims[1]
                                                                               : -1;
    case FGA_MPC_QUAD:
        return arity;
    case FGA_MPC_BOX:
        return 2;
    case FGA_FIX:
        return arity;
    case FGA_SVM_MARGIN:
        return (nv == 3 && dims[1] == 1 && dims[2] == 1) ? dims[0] + 1 : -1;
    case FGA_SVM_SLACK:
        return nv == 1 ? 1 : -1;
    case FGA_EQUAL:
        return (nv == 2 && dims[0] == dims[1]) ? 0 : -1;
    default:
        return -1;
    }
}

static bool is_per_edge(int type) {
    return type == FGA_PACK_RADIUS_LIN || type == FGA_PACK_RADIUS_QUAD || type == FGA_SVM_L2 ||
           type == FGA_MPC_QUAD || type == FGA_MPC_BOX || type == FGA_FIX || type == FGA_SVM_SLACK;
}

// ---------------------------------------------------------------------------
// C-ABI: building
// ---------------------------------------------------------------------------
extern "C" int fga_graph_create(fga_graph **out, int32_t precision, int32_t device, void *cuda_stream) {
    if (!out) return fail(FGA_EINVAL, "fga_graph_create: out is NULL");
    if (precision != FGA_F32 && precision != FGA_F64)
        return fail(FGA_EINVAL, "fga_graph_create: precision must be FGA_F32 or FGA_F64");
    if (device < 0) return fail(FGA_EINVAL, "fga_graph_create: bad device %d", device);
    fga_graph *g = new (std::nothrow) fga_graph();
    if (!g) return fail(FGA_ENOMEM, "fga_graph_create: out of host memory");
    g->precision = precision;
    g->device = device;
    g->stream = (cudaStream_t)cuda_stream;
    *out = g;
    return FGA_OK;
}

extern "C" int fga_set_stream(fga_graph *g, void *cuda_stream) {
    if (!g) return fail(FGA_EINVAL, "fga_set_stream: NULL graph");
    g->stream = (cudaStream_t)cuda_stream;
    return FGA_OK;
}

extern "C" int fga_set_option(fga_graph *g, int32_t option, int64_t value) {
    if (!g) return fail(FGA_EINVAL, "fga_set_option: NULL graph");
    if (g->finalized) return fail(FGA_ESTATE, "fga_set_option: graph already finalized");
    switch (option) {
    case FGA_OPT_ZORDER:
        if (value < 0 || value > 4) return fail(FGA_EINVAL, "FGA_OPT_ZORDER must be 0, 1, 2, 3 or 4");
        g->zorder = (int)value;
        return FGA_OK;
    case FGA_OPT_STORE_M:
        g->store_m = value ? 1 : 0;
        return FGA_OK;
    case FGA_OPT_WEIGHTS:
        if (value != 0 && value != 1) return fail(FGA_EINVAL, "FGA_OPT_WEIGHTS must be 0 or 1");
        g->weights = (int)value;
        return FGA_OK;
    case FGA_OPT_BLOCK:
        if (value != 0 && (value < 64 || value > 256 || value % 32))
            return fail(FGA_EINVAL, "FGA_OPT_BLOCK must be 0 or a multiple of 32 in [64, 256]");
        g->block = (int)value;
        return FGA_OK;
    default:
        return fail(FGA_EINVAL, "fga_set_option: unknown option %d", option);
    }
}

extern "C" int fga_add_variables(fga_graph *g, int64_t count, int32_t dim, int64_t *first_var_id) {
    if (!g) return fail(FGA_EINVAL, "fga_add_variables: NULL graph");
    if (g->finalized) return fail(FGA_ESTATE, "fga_add_variables: graph already finalized");
    if (count < 0 || dim < 1) return fail(FGA_EINVAL, "fga_add_variables: count %lld dim %d", (long long)count, dim);
    if (g->nz + count * (int64_t)dim > (int64_t)INT32_MAX - 1)
        return fail(FGA_EINVAL, "fga_add_variables: more than 2^31-2 scalar variables");
    const int64_t first = (int64_t)g->vdim.size();
    try {
        g->vdim.insert(g->vdim.end(), (size_t)count, dim);
        for (int64_t i = 0; i < count; ++i) {
            g->voff.push_back(g->nz);
            g->nz += dim;
        }
    } catch (...) {
        return fail(FGA_ENOMEM, "fga_add_variables: out of host memory");
    }
    if (first_var_id) *first_var_id = first;
    return FGA_OK;
}

extern "C" int fga_add_factors(fga_graph *g, int32_t type, int64_t count, int32_t n_vars_per_factor,
                               const int64_t *var_ids, const double *params, int32_t params_per_factor,
                               int32_t params_shared, int64_t *first_factor_id) {
    if (!g) return fail(FGA_EINVAL, "fga_add_factors: NULL graph");
    if (g->finalized) return fail(FGA_ESTATE, "fga_add_factors: graph already finalized");
    const bool user = type >= kUserType0;
    if (type < 0 || (type >= FGA_NUM_TYPES && !user) || (user && type - kUserType0 >= (int)g->users.size()))
        return fail(FGA_EINVAL, "fga_add_factors: unknown type %d", type);
    if (count < 0 || n_vars_per_factor < 1 || n_vars_per_factor > 64)
        return fail(FGA_EINVAL, "fga_add_factors: count %lld, %d variables per factor", (long long)count,
                    n_vars_per_factor);
    if (count == 0) {
        if (first_factor_id) *first_factor_id = g->nfac;
        return FGA_OK;
    }
    if (!var_ids) return fail(FGA_EINVAL, "fga_add_factors: var_ids is NULL");
    if (params_per_factor < 0 || (params_per_factor > 0 && !params))
        return fail(FGA_EINVAL, "fga_add_factors: params missing");
    FactorBatch b;
    b.type = type;
    b.count = count;
    b.nv = n_vars_per_factor;
    b.np = params_per_factor;
    b.shared = params_shared != 0;
    b.edge0 = g->ne;
    const int64_t nvar = (int64_t)g->vdim.size();
    // all factors of one call must share one variable shape
    for (int k = 0; k < b.nv; ++k) {
        const int64_t v = var_ids[k];
        if (v < 0 || v >= nvar) return fail(FGA_EINVAL, "fga_add_factors: variable id %lld out of range", (long long)v);
        b.dims.push_back(g->vdim[v]);
        b.arity += g->vdim[v];
    }
    for (int64_t f = 0; f < count; ++f) {
        for (int k = 0; k < b.nv; ++k) {
            const int64_t v = var_ids[f * b.nv + k];
            if (v < 0 || v >= nvar)
                return fail(FGA_EINVAL, "fga_add_factors: variable id %lld out of range (factor %lld)",
                            (long long)v, (long long)f);
            if (g->vdim[v] != b.dims[k])
                return fail(FGA_EINVAL, "fga_add_factors: factors of one call must have the same variable shape");
        }
    }
    const int want = !user ? expected_params(type, b.dims, b.arity)
                     : b.arity == g->users[type - kUserType0].arity ? g->users[type - kUserType0].np
                                                                    : -1;
    if (want < 0) return fail(FGA_EINVAL, "fga_add_factors: variable shape does not fit factor type %d", type);
    if (want != params_per_factor)
        return fail(FGA_EINVAL, "fga_add_factors: type %d takes %d parameters, got %d", type, want, params_per_factor);
    if (g->ne + count * (int64_t)b.arity > (int64_t)INT32_MAX - 1)
        return fail(FGA_EINVAL, "fga_add_factors: more than 2^31-2 scalar edges");
    try {
        b.vars.assign(var_ids, var_ids + count * b.nv);
        const int64_t np_total = b.shared ? b.np : count * b.np;
        if (np_total) b.params.assign(params, params + np_total);
    } catch (...) {
        return fail(FGA_ENOMEM, "fga_add_factors: out of host memory");
    }
    for (double v : b.params)
        if (!std::isfinite(v)) return fail(FGA_EINVAL, "fga_add_factors: non-finite parameter");
    if (type == FGA_MPC_BOX) {
        for (int64_t f = 0; f < (b.shared ? 1 : count); ++f)
            if (!(b.param(f)[0] <= b.param(f)[1])) return fail(FGA_EINVAL, "fga_add_factors: box with lo > hi");
    }
    if (type == FGA_SVM_HINGE) {
        for (int64_t f = 0; f < (b.shared ? 1 : count); ++f)
            if (!(b.param(f)[b.dims[0] + 1] >= 0.0)) return fail(FGA_EINVAL, "fga_add_factors: hinge weight c < 0");
    }
    if (type == FGA_SVM_L2 || type == FGA_SVM_SLACK) {
        for (int64_t f = 0; f < (b.shared ? 1 : count); ++f)
            if (!(b.param(f)[0] >= 0.0)) return fail(FGA_EINVAL, "fga_add_factors: lambda < 0");
    }
    if (type == FGA_MPC_QUAD) {
        for (double v : b.params)
            if (!(v >= 0.0)) return fail(FGA_EINVAL, "fga_add_factors: negative quadratic weight");
    }
    const int64_t first = g->nfac;
    g->ne += count * (int64_t)b.arity;
    g->nfac += count;
    try {
        g->batches.push_back(std::move(b));
    } catch (...) {
        return fail(FGA_ENOMEM, "fga_add_factors: out of host memory");
    }
    if (first_factor_id) *first_factor_id = first;
    return FGA_OK;
}

extern "C" int fga_register_prox(fga_graph *g, const char *cuda_source, const char *function_name, int32_t arity,
                                 int32_t params_per_factor, int32_t *type_out) {
    if (!g || !cuda_source || !function_name || !type_out) return fail(FGA_EINVAL, "fga_register_prox: NULL argument");
    if (g->finalized) return fail(FGA_ESTATE, "fga_register_prox: graph already finalized");
    if (arity < 1 || arity > kUserMaxArity)
        return fail(FGA_EINVAL, "fga_register_prox: arity %d outside [1, %d]", arity, kUserMaxArity);
    if (params_per_factor < 0 || params_per_factor > kUserMaxParams)
        return fail(FGA_EINVAL, "fga_register_prox: %d parameters per factor (at most %d)", params_per_factor,
                    kUserMaxParams);
    if ((int)g->users.size() == kMaxUserTypes)
        return fail(FGA_EINVAL, "fga_register_prox: more than %d user operators", kMaxUserTypes);
    int rc = set_device(g);
    if (rc) return rc;
    UserProg p;
    std::string log;
    if (!user_compile(cuda_source, function_name, arity, params_per_factor, g->precision == FGA_F64, p, log)) {
        if (log.size() > 1500) log.resize(1500);
        const bool env = log.rfind("NVRTC (", 0) == 0 || log.rfind("no CUDA", 0) == 0 ||
                         log.rfind("cudaLibrary", 0) == 0;
        t_last_error = "fga_register_prox: " + log;
        return env ? FGA_ECUDA : FGA_EINVAL;
    }
    try {
        g->users.push_back(p);
    } catch (...) {
        user_release(p);
        return fail(FGA_ENOMEM, "fga_register_prox: out of host memory");
    }
    *type_out = kUserType0 + (int)g->users.size() - 1;
    return FGA_OK;
}

extern "C" int fga_set_rho_alpha(fga_graph *g, double rho, double alpha) {
    if (!g) return fail(FGA_EINVAL, "fga_set_rho_alpha: NULL graph");
    if (g->finalized) return fail(FGA_ESTATE, "fga_set_rho_alpha: graph already finalized");
    if (!(rho > 0.0) || !(alpha > 0.0) || !std::isfinite(rho) || !std::isfinite(alpha))
        return fail(FGA_EINVAL, "fga_set_rho_alpha: rho and alpha must be finite and > 0");
    g->rho_u = rho;
    g->alpha_u = alpha;
    g->rho_c.clear();
    g->alpha_c.clear();
    return FGA_OK;
}

extern "C" int fga_set_edge_rho_alpha(fga_graph *g, const double *rho, const double *alpha) {
    if (!g) return fail(FGA_EINVAL, "fga_set_edge_rho_alpha: NULL graph");
    if (g->finalized) return fail(FGA_ESTATE, "fga_set_edge_rho_alpha: graph already finalized");
    for (int64_t e = 0; e < g->ne; ++e) {
        if (rho && (!(rho[e] > 0.0) || !std::isfinite(rho[e])))
            return fail(FGA_EINVAL, "fga_set_edge_rho_alpha: rho[%lld] not finite > 0", (long long)e);
        if (alpha && (!(alpha[e] > 0.0) || !std::isfinite(alpha[e])))
            return fail(FGA_EINVAL, "fga_set_edge_rho_alpha: alpha[%lld] not finite > 0", (long long)e);
    }
    if (rho) g->rho_c.assign(rho, rho + g->ne);
    if (alpha) g->alpha_c.assign(alpha, alpha + g->ne);
    return FGA_OK;
}

extern "C" int fga_graph_info(const fga_graph *g, int64_t *num_edges, int64_t *num_scalar_vars, int64_t *num_factors,
                              int64_t *num_vars) {
    if (!g) return fail(FGA_EINVAL, "fga_graph_info: NULL graph");
    if (num_edges) *num_edges = g->ne;
    if (num_scalar_vars) *num_scalar_vars = g->nz;
    if (num_factors) *num_factors = g->nfac;
    if (num_vars) *num_vars = (int64_t)g->vdim.size();
    return FGA_OK;
}

// ---------------------------------------------------------------------------
// finalize: layout + upload
// ---------------------------------------------------------------------------
static double edge_rho_c(const fga_graph *g, int64_t c) { return g->rho_c.empty() ? g->rho_u : g->rho_c[c]; }

// fast z-order layout built by build_chunks
struct FastLayout {
    std::vector<ChunkDev> chunks;
    std::vector<int32_t> slot_var, ppos, lrow, prow;
    std::vector<uint32_t> lidx;   // slot | padded buffer position << 16
    // scatter order: per storage edge variable | column << kEvColShift, and
    // per variable 1 when it has an overflow row (rows in prow)
    std::vector<uint32_t> ev;
    std::vector<unsigned char> zovf;
};

template <typename R>
static int upload_vec(DevBuf &buf, const std::vector<R> &v) {
    CUDA_TRY(buf.alloc(v.size() * sizeof(R)));
    if (!v.empty()) CUDA_TRY(cudaMemcpy(buf.p, v.data(), v.size() * sizeof(R), cudaMemcpyHostToDevice));
    return FGA_OK;
}

template <typename R>
static int finalize_typed(fga_graph *g, const std::vector<int32_t> &pos, const std::vector<int32_t> &rowp,
                          const std::vector<double> &srho_d, const std::vector<double> &srho2_d,
                          const FastLayout &fl) {
    const int64_t E = g->ne;
    int rc;
    // per-edge rho / alpha in storage order (only when not uniform)
    g->uniform_rho = g->rho_c.empty();
    g->uniform_alpha = g->alpha_c.empty();
    const int64_t ES = g->es;
    if (!g->uniform_rho) {
        std::vector<R> v((size_t)ES, R(1));
        for (int64_t s = 0; s < ES; ++s)
            if (g->s2c[s] >= 0) v[s] = (R)g->rho_c[g->s2c[s]];
        if ((rc = upload_vec(g->rho_e, v))) return rc;
    }
    if (!g->uniform_alpha) {
        std::vector<R> v((size_t)ES, R(1));
        for (int64_t s = 0; s < ES; ++s)
            if (g->s2c[s] >= 0) v[s] = (R)g->alpha_c[g->s2c[s]];
        if ((rc = upload_vec(g->alpha_e, v))) return rc;
    }
    {
        std::vector<R> v(srho_d.size());
        for (size_t i = 0; i < v.size(); ++i) v[i] = (R)srho_d[i];
        if ((rc = upload_vec(g->srho, v))) return rc;
    }
    if ((rc = upload_vec(g->srho2, srho2_d))) return rc;
    // 64 spare elements: a bulk copy may read up to 16 bytes past the last edge
    const size_t eb = (size_t)(std::max<int64_t>(ES, 1) + 64) * sizeof(R);
    (void)E;
    if (g->zorder == 3) {
        const HingePlan &H = g->hinge;
        if ((rc = upload_vec(g->h_cta, H.cta))) return rc;
        if ((rc = upload_vec(g->h_X, H.X))) return rc;
        if ((rc = upload_vec(g->h_meta, H.meta))) return rc;
        const size_t n = (size_t)std::max<int64_t>(g->hin.N, 1) * sizeof(float);
        CUDA_TRY(g->h_gsave.alloc(2 * n));
        CUDA_TRY(g->h_gres.alloc(n));
        CUDA_TRY(g->h_l2save.alloc((size_t)kHingeMaxL2 * kHingeD * sizeof(float)));
        CUDA_TRY(g->h_l2res.alloc((size_t)kHingeMaxL2 * kHingeD * sizeof(float)));
        CUDA_TRY(cudaMemset(g->h_l2res.p, 0, g->h_l2res.bytes));
        CUDA_TRY(g->h_acc.alloc((size_t)2 * (g->hin.D + 1) * kHingeAccStride * sizeof(unsigned long long)));
        CUDA_TRY(cudaMemset(g->h_acc.p, 0, g->h_acc.bytes));
        CUDA_TRY(g->t_zprev.alloc((size_t)std::max<int64_t>(g->nz, 1) * sizeof(float)));
    } else if (g->zorder == 2) {
        const TilePlan &T = g->tile;
        if ((rc = upload_vec(g->t_cta, T.cta))) return rc;
        if ((rc = upload_vec(g->t_rowslot, T.rowslot))) return rc;
        if ((rc = upload_vec(g->t_colslot, T.colslot))) return rc;
        if ((rc = upload_vec(g->t_mask, T.mask))) return rc;
        if ((rc = upload_vec(g->t_sv, T.sv))) return rc;
        if ((rc = upload_vec(g->t_zden, T.zden))) return rc;
        if ((rc = upload_vec(g->t_cptr, T.cptr))) return rc;
        if ((rc = upload_vec(g->t_clist, T.clist))) return rc;
        if ((rc = upload_vec(g->t_loc, T.loc))) return rc;
        CUDA_TRY(g->t_part.alloc((size_t)2 * T.ptot * sizeof(unsigned long long)));
        CUDA_TRY(cudaMemset(g->t_part.p, 0, g->t_part.bytes));
        CUDA_TRY(g->t_dsave.alloc((size_t)T.U * (kUnitEdges / 2) * sizeof(float)));
        CUDA_TRY(g->t_dres.alloc((size_t)T.U * (kUnitEdges / 2) * sizeof(float)));
        if (T.W > T.warps) CUDA_TRY(g->t_dlive.alloc((size_t)T.U * (kUnitEdges / 2) * sizeof(float)));
        CUDA_TRY(g->t_lres.alloc((size_t)std::max<size_t>(T.loc.size(), 1) * sizeof(float)));
        CUDA_TRY(g->t_zprev.alloc((size_t)std::max<int64_t>(g->nz, 1) * sizeof(float)));
    } else if (g->zorder == 0) {
        // canonical order: per-edge variable ids and positions in the
        // creation-ordered variable-major array
        if ((rc = upload_vec(g->d_svar, g->svar))) return rc;
        if ((rc = upload_vec(g->d_pos, pos))) return rc;
        if ((rc = upload_vec(g->row, rowp))) return rc;
        CUDA_TRY(g->pvm.alloc(eb));
        CUDA_TRY(cudaMemset(g->pvm.p, 0, eb));
        if (g->weights) {
            CUDA_TRY(g->wcls.alloc((size_t)std::max<int64_t>(ES, 1)));
            CUDA_TRY(g->pwcls.alloc((size_t)std::max<int64_t>(g->ne, 1)));
            if (!g->uniform_rho) {
                std::vector<R> pr((size_t)std::max<int64_t>(g->ne, 1), R(1));
                for (int64_t s2 = 0; s2 < ES; ++s2)
                    if (g->s2c[s2] >= 0) pr[pos[s2]] = (R)g->rho_c[g->s2c[s2]];
                if ((rc = upload_vec(g->prho, pr))) return rc;
            }
        }
    } else if (g->zorder == 4) {
        // scatter order: per-edge words, overflow positions and rows, the
        // zeroed column table (entries past a variable's degree stay 0)
        if ((rc = upload_vec(g->d_ev, fl.ev))) return rc;
        if ((rc = upload_vec(g->d_pos, pos))) return rc;
        if ((rc = upload_vec(g->prow, fl.prow))) return rc;
        if ((rc = upload_vec(g->zovf, fl.zovf))) return rc;
        const size_t pb = (size_t)std::max<int64_t>((int64_t)g->colw * g->nz + g->novf, 1) * sizeof(R);
        CUDA_TRY(g->pvm.alloc(pb));
        CUDA_TRY(cudaMemset(g->pvm.p, 0, pb));
    } else {
        if ((rc = upload_vec(g->chunks, fl.chunks))) return rc;
        if ((rc = upload_vec(g->slot_var, fl.slot_var))) return rc;
        if ((rc = upload_vec(g->ppos, fl.ppos))) return rc;
        if ((rc = upload_vec(g->lrow, fl.lrow))) return rc;
        if ((rc = upload_vec(g->lidx, fl.lidx))) return rc;
        if ((rc = upload_vec(g->prow, fl.prow))) return rc;
        const size_t pb = std::max<size_t>(fl.slot_var.size(), 1) * sizeof(R);
        CUDA_TRY(g->part.alloc(pb));
        CUDA_TRY(cudaMemset(g->part.p, 0, pb));
    }
    CUDA_TRY(g->x[0].alloc(eb));
    CUDA_TRY(g->x[1].alloc(eb));
    CUDA_TRY(g->u.alloc(eb));
    CUDA_TRY(cudaMemset(g->x[0].p, 0, eb));
    CUDA_TRY(cudaMemset(g->x[1].p, 0, eb));
    CUDA_TRY(cudaMemset(g->u.p, 0, eb));
    if (g->store_m) {
        CUDA_TRY(g->m[0].alloc(eb));
        CUDA_TRY(g->m[1].alloc(eb));
        CUDA_TRY(cudaMemset(g->m[0].p, 0, eb));
        CUDA_TRY(cudaMemset(g->m[1].p, 0, eb));
    }
    const size_t zb = (size_t)std::max<int64_t>(g->nz, 1) * sizeof(R);
    CUDA_TRY(g->z[0].alloc(zb));
    CUDA_TRY(g->z[1].alloc(zb));
    CUDA_TRY(cudaMemset(g->z[0].p, 0, zb));
    CUDA_TRY(cudaMemset(g->z[1].p, 0, zb));

    // per-bucket parameters (SoA) and MPC projection matrices
    g->bucket_bufs.clear();
    g->ubk.clear();
    for (auto &bk : g->buckets) {
        const int64_t nf = (int64_t)bk.members.size();
        std::vector<R> prm((size_t)bk.np * nf);
        for (int64_t f = 0; f < nf; ++f) {
            const FactorBatch &b = g->batches[bk.members[f].first];
            const double *p = b.param(bk.members[f].second);
            // hinge and margin parameters factor-major (a factor's data
            // point read contiguously); every other type edge-major
            const bool fmaj = bk.type == FGA_SVM_HINGE || bk.type == FGA_SVM_MARGIN || bk.type >= kUserType0;
            for (int j = 0; j < bk.np; ++j) prm[fmaj ? (size_t)f * bk.np + j : (size_t)j * nf + f] = (R)p[j];
        }
        auto pb = std::make_unique<DevBuf>();
        if ((rc = upload_vec(*pb, prm))) return rc;
        bk.prm_buf = (int)g->bucket_bufs.size();
        g->bucket_bufs.push_back(std::move(pb));
        if (bk.type >= kUserType0) {
            // per edge of the bucket: its scalar variable and where its rho m
            // goes (the canonical rows, or the scatter columns / overflow)
            auto ub = std::make_unique<UserBucket>();
            ub->bucket = (int)(&bk - g->buckets.data());
            ub->user = bk.type - kUserType0;
            const int64_t n = nf * bk.arity;
            std::vector<int32_t> var((size_t)std::max<int64_t>(n, 1), 0);
            std::vector<uint32_t> dst((size_t)std::max<int64_t>(n, 1), 0u);
            for (int64_t l = 0; l < n; ++l) {
                const int64_t st = bk.ebase + l;
                var[l] = g->svar[st];
                if (g->zorder == 4) {
                    const uint32_t ev = fl.ev[st], c = ev >> kEvColShift, b = ev & kEvVarMask;
                    dst[l] = c != kEvOverflow ? c * (uint32_t)g->nz + b
                                              : (uint32_t)((int64_t)g->colw * g->nz) + (uint32_t)pos[st];
                } else {
                    dst[l] = (uint32_t)pos[st];
                }
            }
            if ((rc = upload_vec(ub->var, var))) return rc;
            if ((rc = upload_vec(ub->dst, dst))) return rc;
            g->ubk.push_back(std::move(ub));
        }
        if (bk.type == FGA_MPC_DYN) {
            const int nx = bk.dims[0], nu = bk.dims[1], n = bk.arity;
            std::map<std::vector<double>, int> seen;
            std::vector<R> mats;
            std::vector<int32_t> pidx((size_t)nf);
            std::vector<double> key, rho((size_t)n), P;
            for (int64_t f = 0; f < nf; ++f) {
                const FactorBatch &b = g->batches[bk.members[f].first];
                const int64_t fi = bk.members[f].second;
                const double *p = b.param(fi);
                const int64_t c0 = b.edge0 + fi * b.arity;
                key.assign(p, p + bk.np);
                for (int k = 0; k < n; ++k) {
                    rho[k] = edge_rho_c(g, c0 + k);
                    key.push_back(rho[k]);
                }
                auto it = seen.find(key);
                if (it == seen.end()) {
                    if (!dyn_projector(nx, nu, p, p + nx * nx, rho.data(), P))
                        return fail(FGA_EINVAL, "fga_finalize: singular dynamics constraint");
                    const int id = (int)seen.size();
                    seen.emplace(key, id);
                    for (double v : P) mats.push_back((R)v);
                    pidx[f] = id;
                } else {
                    pidx[f] = it->second;
                }
            }
            auto mb = std::make_unique<DevBuf>();
            if ((rc = upload_vec(*mb, mats))) return rc;
            g->bucket_bufs.push_back(std::move(mb));
            auto ib = std::make_unique<DevBuf>();
            if ((rc = upload_vec(*ib, pidx))) return rc;
            g->bucket_bufs.push_back(std::move(ib));
        }
    }
    return FGA_OK;
}

// ---------------------------------------------------------------------------
// fast z-order layout
// ---------------------------------------------------------------------------
// Cuts every bucket into chunks of consecutive work items (at most
// kChunkItems items, kChunkEdges scalar edges and kChunkSlots distinct scalar
// variables each), numbers each chunk's variables ("slots") in order of first
// appearance, and gives every edge its slot and its position in the chunk's
// slot-sorted buffer.  The per-slot partial sums are laid out variable-major
// (chunk order inside a row).
static int build_chunks(fga_graph *g, FastLayout &fl, int64_t items_per_chunk) {
    const int64_t Z = g->nz;
    try {
        fl.lidx.assign((size_t)g->es + 64, 0);   // spare tail for bulk copies
    } catch (...) {
        return fail(FGA_ENOMEM, "fga_finalize: out of host memory");
    }
    std::vector<int32_t> mark((size_t)Z, -1), slot_of((size_t)Z, 0);
    std::vector<int32_t> cnt;
    std::vector<int64_t> edges;
    int chunk_id = 0;
    for (int bi = 0; bi < (int)g->buckets.size(); ++bi) {
        const Bucket &bk = g->buckets[bi];
        const int64_t nf = (int64_t)bk.members.size();
        if (bk.arity > kChunkEdges) return fail(FGA_EINVAL, "fga_finalize: factor arity %d too large", bk.arity);
        auto item_edges = [&](int64_t i, std::vector<int64_t> &out) {
            out.clear();
            if (bk.per_edge) {
                out.push_back(bk.ebase + i);
            } else if (bk.type == FGA_EQUAL) {
                // item i = component j of factor f, i = j * nf + f
                const int64_t j = i / nf, f = i % nf;
                out.push_back(bk.ebase + j * nf + f);
                out.push_back(bk.ebase + (j + bk.arity / 2) * nf + f);
            } else {
                for (int k = 0; k < bk.arity; ++k)
                    out.push_back(bk.aos ? bk.ebase + i * bk.arity + k : bk.ebase + (int64_t)k * nf + i);
            }
        };
        std::vector<int64_t> ie;
        int64_t i = 0;
        while (i < bk.nitems) {
            ChunkDev ch;
            std::memset(&ch, 0, sizeof ch);
            ch.bucket = bi;
            ch.f0 = i;
            ch.sbase = (int)fl.slot_var.size();
            ch.lrbase = (int)fl.lrow.size();
            edges.clear();
            int nslots = 0;
            // disk-pair chunks start at even factors (16-byte aligned bulk copies)
            const int64_t unit = bk.type == FGA_PACK_PAIR ? 2 : 1;
            while (i < bk.nitems && i - ch.f0 < items_per_chunk) {
                item_edges(i, ie);
                if (unit == 2 && i + 1 < bk.nitems) {
                    std::vector<int64_t> ie2;
                    item_edges(i + 1, ie2);
                    ie.insert(ie.end(), ie2.begin(), ie2.end());
                }
                int fresh = 0;
                for (int64_t e : ie) {
                    const int32_t v = g->svar[e];
                    if (mark[v] != chunk_id) {
                        // count distinct new variables of this item once
                        bool dup = false;
                        for (int64_t e2 : ie) {
                            if (e2 == e) break;
                            if (g->svar[e2] == v) { dup = true; break; }
                        }
                        if (!dup) ++fresh;
                    }
                }
                if (i == ch.f0 && fresh > kChunkSlots)
                    return fail(FGA_EINVAL, "fga_finalize: a factor touches more than %d scalar variables",
                                kChunkSlots);
                if (i > ch.f0 && ((int64_t)edges.size() + (int64_t)ie.size() > kChunkEdges ||
                                  nslots + fresh > kChunkSlots))
                    break;
                for (int64_t e : ie) {
                    const int32_t v = g->svar[e];
                    if (mark[v] != chunk_id) {
                        mark[v] = chunk_id;
                        slot_of[v] = nslots++;
                        fl.slot_var.push_back(v);
                    }
                    edges.push_back(e);
                }
                i += (unit == 2 && i + 1 < bk.nitems) ? 2 : 1;
            }
            ch.nitems = (int)(i - ch.f0);
            ch.nslots = nslots;
            cnt.assign((size_t)nslots + 1, 0);
            for (int64_t e : edges) cnt[slot_of[g->svar[e]] + 1]++;
            for (int k = 0; k < nslots; ++k) cnt[k + 1] += cnt[k];
            for (int k = 0; k <= nslots; ++k) fl.lrow.push_back(cnt[k]);
            for (int64_t e : edges) {
                // segments are padded by one element each (slot sl starts at
                // cnt[sl] + sl) so that lanes writing to different slots hit
                // different shared-memory banks
                const int sl = slot_of[g->svar[e]];
                const uint32_t pos = (uint32_t)(cnt[sl]++ + sl);
                fl.lidx[e] = (uint32_t)sl | (pos << 16);
            }
            fl.chunks.push_back(ch);
            ++chunk_id;
        }
    }
    // variable-major partials: row of variable b = its (chunk, slot) entries in chunk order
    fl.prow.assign((size_t)Z + 1, 0);
    for (int32_t v : fl.slot_var) fl.prow[v + 1]++;
    for (int64_t b = 0; b < Z; ++b) fl.prow[b + 1] += fl.prow[b];
    std::vector<int32_t> fill(fl.prow.begin(), fl.prow.end() - 1);
    fl.ppos.resize(fl.slot_var.size());
    for (size_t k = 0; k < fl.slot_var.size(); ++k) fl.ppos[k] = fill[fl.slot_var[k]]++;
    g->nchunks = (int)fl.chunks.size();
    return FGA_OK;
}

// Work lists of the fast z-update over rows `rowp`: low-degree rows one
// thread each, others one warp each, hub rows split into kPiece pieces.
// Scatter order (overflow = true): only the overflow rows, each a warp item
// or hub pieces (the columns are summed one thread per variable).
static int build_zlists(fga_graph *g, const std::vector<int32_t> &rowp, bool overflow) {
    int rc;
    std::vector<int32_t> small, hub_np, hub_off;
    std::vector<int4> witems, med;
    int off = 0;
    for (int64_t b = 0; b < g->nz; ++b) {
        const int deg = rowp[b + 1] - rowp[b];
        if (overflow && deg == 0) continue;
        if (!overflow && deg <= kSmallDeg) {
            small.push_back((int32_t)b);
        } else if (deg <= kPiece) {
            med.push_back(make_int4((int)b, rowp[b], deg, -1));
        } else {
            const int h = (int)hub_np.size();
            const int np = (deg + kPiece - 1) / kPiece;
            hub_np.push_back(np);
            hub_off.push_back(off);
            off += np;
            for (int p = 0; p < np; ++p)
                witems.push_back(make_int4((int)b, rowp[b] + p * kPiece, std::min(kPiece, deg - p * kPiece), h));
        }
    }
    witems.insert(witems.end(), med.begin(), med.end());
    g->n_small = (int)small.size();
    g->n_witems = (int)witems.size();
    g->n_hubs = (int)hub_np.size();
    if ((rc = upload_vec(g->small_vars, small))) return rc;
    if ((rc = upload_vec(g->witems, witems))) return rc;
    if ((rc = upload_vec(g->hub_np, hub_np))) return rc;
    if ((rc = upload_vec(g->hub_off, hub_off))) return rc;
    CUDA_TRY(g->hub_part.alloc((size_t)std::max(off, 1) * g->rsize()));
    CUDA_TRY(g->hub_ticket.alloc((size_t)std::max(g->n_hubs, 1) * sizeof(unsigned int)));
    CUDA_TRY(cudaMemset(g->hub_ticket.p, 0, g->hub_ticket.bytes));
    return FGA_OK;
}

// Disk-tile order: checks that the graph is a circle-packing graph the tile
// kernel can run (FP32, one rho and alpha, only disk-pair / wall / radius
// factors, m not kept) and builds the plan.  0: planned; 1: not suitable
// (reason in `why`); < 0: error.
static int try_tile_plan(fga_graph *g, std::string &why) {
    if (!g->rho_c.empty() || !g->alpha_c.empty()) {
        why = "rho or alpha set per edge";
        return 1;
    }
    if (g->store_m == 1) {
        why = "m is kept (FGA_OPT_STORE_M)";
        return 1;
    }
    int npair_buckets = 0;
    for (const Bucket &bk : g->buckets) {
        if (bk.type == FGA_PACK_PAIR) ++npair_buckets;
        else if (bk.type != FGA_PACK_WALL && bk.type != FGA_PACK_RADIUS_LIN && bk.type != FGA_PACK_RADIUS_QUAD) {
            why = "factor types other than disk pairs, walls and radius rewards";
            return 1;
        }
    }
    if (npair_buckets != 1) {
        why = "no disk pairs";
        return 1;
    }
    TileInput in;
    in.nz = g->nz;
    try {
        in.deg.assign((size_t)g->nz, 0.0);
        const double rho = g->rho_u;
        for (const Bucket &bk : g->buckets) {
            for (int64_t f = 0; f < (int64_t)bk.members.size(); ++f) {
                const FactorBatch &b = g->batches[bk.members[f].first];
                const int64_t fi = bk.members[f].second;
                const int64_t *v = b.vars.data() + fi * b.nv;
                const double *p = b.param(fi);
                if (bk.type == FGA_PACK_PAIR) {
                    const int32_t c1 = (int32_t)g->voff[v[0]], r1 = (int32_t)g->voff[v[1]];
                    const int32_t c2 = (int32_t)g->voff[v[2]], r2 = (int32_t)g->voff[v[3]];
                    in.c1.push_back(c1);
                    in.r1.push_back(r1);
                    in.c2.push_back(c2);
                    in.r2.push_back(r2);
                    for (int32_t s : {c1, c1 + 1, r1, c2, c2 + 1, r2}) in.deg[s] += 1.0;
                } else {
                    TileInput::Local L;
                    std::memset(&L, 0, sizeof L);
                    L.type = bk.type;
                    L.member = f;
                    if (bk.type == FGA_PACK_WALL) {
                        L.c = (int32_t)g->voff[v[0]];
                        L.r = (int32_t)g->voff[v[1]];
                        for (int k = 0; k < 4; ++k) L.p[k] = (float)p[k];
                        L.p[4] = (float)(1.0 / (p[0] * p[0] + p[1] * p[1] + 1.0));
                        for (int32_t s : {L.c, L.c + 1, L.r}) in.deg[s] += 1.0;
                    } else {
                        L.c = -1;
                        L.r = (int32_t)g->voff[v[0]];
                        L.p[0] = bk.type == FGA_PACK_RADIUS_LIN ? (float)(p[0] / rho) : (float)(1.0 / (rho - 1.0));
                        in.deg[L.r] += 1.0;
                    }
                    in.locs.push_back(L);
                }
            }
        }
    } catch (...) {
        return fail(FGA_ENOMEM, "fga_finalize: out of host memory");
    }
    CUDA_TRY(cudaDeviceGetAttribute(&in.sms, cudaDevAttrMultiProcessorCount, g->device));
    in.wmax = tile_max_warps();
    if (g->block) in.wmax = std::min(in.wmax, g->block / 32);   // FGA_OPT_BLOCK caps the warps per CTA
    int rc;
    try {
        rc = tile_plan(in, g->tile, why);
    } catch (...) {
        return fail(FGA_ENOMEM, "fga_finalize: out of host memory");
    }
    if (rc) return rc;
    int optin = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, g->device));
    if (tile_smem_bytes(g->tile) > optin) {
        why = "the z table of a CTA does not fit in shared memory";
        return 1;
    }
    return 0;
}

// Hinge bank: checks that the graph is a linear SVM the hinge kernel can
// run (FP32, one rho, alpha = 1, m not kept, hinge factors on one shared
// (w, b) and L2 factors on that w only) and builds the plan.  0: planned;
// 1: not suitable (reason in `why`); < 0: error.
static int try_hinge_plan(fga_graph *g, std::string &why) {
    if (!g->rho_c.empty() || !g->alpha_c.empty() || g->alpha_u != 1.0) {
        why = "rho or alpha set per edge, or alpha other than 1";
        return 1;
    }
    if (g->store_m == 1) {
        why = "m is kept (FGA_OPT_STORE_M)";
        return 1;
    }
    const Bucket *hb = nullptr, *lb = nullptr;
    for (const Bucket &bk : g->buckets) {
        if (bk.type == FGA_SVM_HINGE && !hb) hb = &bk;
        else if (bk.type == FGA_SVM_L2 && !lb) lb = &bk;
        else {
            why = "factor types other than one hinge bank and its L2 factors";
            return 1;
        }
    }
    if (!hb) {
        why = "no hinge factors";
        return 1;
    }
    HingeInput &in = g->hin;
    in = HingeInput();
    const int D = hb->dims[0];
    in.D = D;
    in.N = (int64_t)hb->members.size();
    int64_t w = -1, b = -1;
    try {
        in.X.resize((size_t)in.N * D);
        in.yl.resize((size_t)in.N);
        in.cl.resize((size_t)in.N);
        for (int64_t f = 0; f < in.N; ++f) {
            const FactorBatch &fb = g->batches[hb->members[f].first];
            const int64_t fi = hb->members[f].second;
            const int64_t *v = fb.vars.data() + fi * fb.nv;
            if (f == 0) {
                w = v[0];
                b = v[1];
            } else if (v[0] != w || v[1] != b) {
                why = "hinge factors on different variables";
                return 1;
            }
            const double *pp = fb.param(fi);
            for (int j = 0; j < D; ++j) in.X[(size_t)f * D + j] = (float)pp[j];
            in.yl[f] = (float)pp[D];
            in.cl[f] = (float)pp[D + 1];
        }
        if (lb) {
            for (int64_t f = 0; f < (int64_t)lb->members.size(); ++f) {
                const FactorBatch &fb = g->batches[lb->members[f].first];
                const int64_t fi = lb->members[f].second;
                if (fb.vars[fi * fb.nv] != w) {
                    why = "an L2 factor on a variable other than the hinges' w";
                    return 1;
                }
                in.lam.push_back((float)fb.param(fi)[0]);
            }
        }
    } catch (...) {
        return fail(FGA_ENOMEM, "fga_finalize: out of host memory");
    }
    in.vw = (int)g->voff[w];
    in.vb = (int)g->voff[b];
    in.rho = g->rho_u;
    CUDA_TRY(cudaDeviceGetAttribute(&in.sms, cudaDevAttrMultiProcessorCount, g->device));
    CUDA_TRY(cudaDeviceGetAttribute(&in.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, g->device));
    int rc;
    try {
        rc = hinge_plan(in, g->hinge, why);
    } catch (...) {
        return fail(FGA_ENOMEM, "fga_finalize: out of host memory");
    }
    return rc;
}

// Scatter order: the number of columns W (1..kColMax) for the degrees of
// the scalar variables, the one that minimises the values phase Z reads
// (W per variable) plus twice the overflow entries (each also costs a
// position read and a warp item); returns the overflow entry count.
static int64_t choose_columns(const std::vector<int32_t> &deg, int &W) {
    std::vector<int64_t> cnt((size_t)kColMax + 1, 0);
    int64_t big_n = 0, big_sum = 0;
    for (int32_t d : deg) {
        if (d <= kColMax) cnt[d]++;
        else {
            big_n++;
            big_sum += d;
        }
    }
    const int64_t nz = (int64_t)deg.size();
    int64_t best = -1, best_ovf = 0;
    W = 1;
    for (int w = 1; w <= kColMax; ++w) {
        int64_t ovf = big_sum - big_n * w;
        for (int d = w + 1; d <= kColMax; ++d) ovf += cnt[d] * (d - w);
        const int64_t cost = (int64_t)w * nz + 2 * ovf;
        if (best < 0 || cost < best) {
            best = cost;
            best_ovf = ovf;
            W = w;
        }
    }
    return best_ovf;
}

extern "C" int fga_finalize(fga_graph *g) {
    if (!g) return fail(FGA_EINVAL, "fga_finalize: NULL graph");
    if (g->finalized) return fail(FGA_ESTATE, "fga_finalize: graph already finalized");
    int rc = set_device(g);
    if (rc) return rc;
    if (g->weights) {
        // three weights run in the canonical order
        if (g->zorder > 0) return fail(FGA_EINVAL, "fga_finalize: FGA_OPT_WEIGHTS 1 needs FGA_OPT_ZORDER 0");
        g->zorder = 0;
    }
    const int zreq = g->zorder;   // -1: library choice
    bool user = false;
    for (const FactorBatch &b : g->batches) user = user || b.type >= kUserType0;
    if (user && (g->weights || (zreq >= 1 && zreq <= 3)))
        return fail(FGA_EINVAL, "fga_finalize: user operators run with fixed weights in the canonical (0) or "
                                "scatter (4) z-order");
    if (zreq == 2 && g->precision != FGA_F32)
        return fail(FGA_EINVAL, "fga_finalize: FGA_OPT_ZORDER 2 (disk tiles) needs FGA_F32");
    if (g->zorder < 0) g->zorder = g->precision == FGA_F64 ? 0 : 1;
    if (g->store_m < 0) g->store_m = g->precision == FGA_F64 ? 1 : 0;
    const int64_t E = g->ne;

    // rho checks that the prox formulas rely on
    for (const FactorBatch &b : g->batches) {
        for (int64_t f = 0; f < b.count; ++f) {
            const int64_t c0 = b.edge0 + f * b.arity;
            if ((b.type == FGA_PACK_PAIR || b.type == FGA_PACK_WALL) && edge_rho_c(g, c0) != edge_rho_c(g, c0 + 1))
                return fail(FGA_EINVAL, "fga_finalize: the two centre coordinates of a disk need one rho");
            if (b.type == FGA_PACK_PAIR && edge_rho_c(g, c0 + 3) != edge_rho_c(g, c0 + 4))
                return fail(FGA_EINVAL, "fga_finalize: the two centre coordinates of a disk need one rho");
            if (b.type == FGA_PACK_RADIUS_QUAD && !(edge_rho_c(g, c0) > 1.0))
                return fail(FGA_EINVAL, "fga_finalize: the area reward needs rho > 1 on its edge");
        }
    }

    // 1. buckets: factors grouped by (type, variable shape), creation order kept
    g->buckets.clear();
    for (int bi = 0; bi < (int)g->batches.size(); ++bi) {
        const FactorBatch &b = g->batches[bi];
        int found = -1;
        for (int k = 0; k < (int)g->buckets.size(); ++k)
            if (g->buckets[k].type == b.type && g->buckets[k].dims == b.dims) found = k;
        if (found < 0) {
            if ((int)g->buckets.size() == kMaxBuckets)
                return fail(FGA_EINVAL, "fga_finalize: more than %d distinct (type, shape) groups", kMaxBuckets);
            Bucket nb;
            nb.type = b.type;
            nb.dims = b.dims;
            nb.np = b.np;
            nb.arity = b.arity;
            nb.per_edge = is_per_edge(b.type);
            nb.aos = b.type == FGA_PACK_PAIR || b.type == FGA_PACK_WALL || b.type == FGA_MPC_DYN ||
                     b.type == FGA_SVM_HINGE || b.type == FGA_SVM_MARGIN || b.type >= kUserType0;
            g->buckets.push_back(nb);
            found = (int)g->buckets.size() - 1;
        }
        for (int64_t f = 0; f < b.count; ++f) g->buckets[found].members.emplace_back(bi, f);
    }
    // 1a. disk-tile order when the graph suits it (FP32 default) or when asked
    if (g->precision == FGA_F32 && !user && (zreq < 0 || zreq == 2)) {
        std::string why;
        const int r = try_tile_plan(g, why);
        if (r < 0) return r;
        if (r == 0) g->zorder = 2;
        else if (zreq == 2)
            return fail(FGA_EINVAL, "fga_finalize: the disk-tile order does not apply: %s", why.c_str());
    }
    // 1a'. hinge bank for a linear SVM (FP32 default when it qualifies)
    if (g->precision == FGA_F32 && !user && g->zorder != 2 && (zreq < 0 || zreq == 3)) {
        std::string why;
        const int r = try_hinge_plan(g, why);
        if (r < 0) return r;
        if (r == 0) g->zorder = 3;
        else if (zreq == 3)
            return fail(FGA_EINVAL, "fga_finalize: the hinge-bank order does not apply: %s", why.c_str());
    }
    if (zreq == 3 && g->precision != FGA_F32)
        return fail(FGA_EINVAL, "fga_finalize: FGA_OPT_ZORDER 3 (hinge bank) needs FGA_F32");
    // 1a''. scatter order: per-variable columns when most edges fit in them
    // (FP32 default over the chunked order for graphs of low-degree
    // variables) or when asked
    if (zreq == 4 || (zreq < 0 && g->zorder == 1)) {
        std::vector<int32_t> deg((size_t)g->nz, 0);
        for (const FactorBatch &b : g->batches)
            for (int64_t f = 0; f < b.count; ++f)
                for (int v = 0; v < b.nv; ++v) {
                    const int64_t var = b.vars[f * b.nv + v];
                    for (int d = 0; d < b.dims[v]; ++d) deg[(size_t)(g->voff[var] + d)]++;
                }
        int W = 1;
        const int64_t ovf = choose_columns(deg, W);
        const bool fits = g->nz < (int64_t)kEvVarMask && (int64_t)W * g->nz + ovf < (int64_t)UINT32_MAX;
        if (zreq == 4 && !fits)
            return fail(FGA_EINVAL, "fga_finalize: the scatter order (FGA_OPT_ZORDER 4) takes fewer than 2^28 "
                                    "scalar variables and 2^32 column entries");
        if (zreq == 4 || (fits && 4 * ovf <= g->ne && (int64_t)W * g->nz <= 2 * g->ne)) {
            g->zorder = 4;
            g->colw = W;
            g->novf = ovf;
        }
    }
    // user operators: the canonical order when the scatter order does not
    // apply (their kernels write each edge's rho m to one slot)
    if (user && g->zorder == 1) g->zorder = 0;
    // the scatter order stores every bucket factor-major (consecutive work
    // items touch consecutive components of a variable block), except the
    // dynamics factors, one thread each: edge-major, so that a warp's loads
    // and stores of its factors' k-th edges are contiguous
    if (g->zorder == 4)
        for (Bucket &bk : g->buckets) bk.aos = bk.type != FGA_MPC_DYN;
    const bool tile = g->zorder == 2;
    const bool hinge = g->zorder == 3;
    const int64_t tile_span = (int64_t)g->tile.U * kUnitEdges;
    // 1b. fast order: inside a bucket, factors that touch nearby variables
    // are stored together (stable sort by the blocks of the first and last
    // variable), so that a chunk of consecutive factors touches few variables
    if (g->zorder == 1) {
        for (Bucket &bk : g->buckets) {
            auto key = [&](const std::pair<int, int64_t> &m) {
                const FactorBatch &b = g->batches[m.first];
                const int64_t v0 = b.vars[m.second * b.nv], v1 = b.vars[m.second * b.nv + b.nv - 1];
                const int64_t first = g->voff[v0], last = g->voff[v1] + g->vdim[v1] - 1;
                return std::make_pair(first / kLocalityBlock, last / kLocalityBlock);
            };
            std::stable_sort(bk.members.begin(), bk.members.end(),
                             [&](const std::pair<int, int64_t> &a, const std::pair<int, int64_t> &b) {
                                 return key(a) < key(b);
                             });
        }
    }
    // 2. storage order: bucket by bucket (each base a multiple of 4),
    // factor-major or edge-major inside a bucket
    int64_t es = 0;
    for (const Bucket &bk : g->buckets)
        es = ((es + 3) & ~int64_t(3)) +
             (tile && bk.type == FGA_PACK_PAIR ? tile_span : (int64_t)bk.members.size() * bk.arity);
    if (es > (int64_t)INT32_MAX - 8) return fail(FGA_EINVAL, "fga_finalize: more than 2^31 edges with padding");
    std::vector<int64_t> c2s;
    try {
        g->s2c.assign((size_t)es, -1);
        g->svar.assign((size_t)es, 0);
        c2s.assign((size_t)E, 0);
    } catch (...) {
        return fail(FGA_ENOMEM, "fga_finalize: out of host memory");
    }
    int64_t ebase = 0, item = 0;
    for (Bucket &bk : g->buckets) {
        const int64_t nf = (int64_t)bk.members.size();
        const bool tp = tile && bk.type == FGA_PACK_PAIR;
        ebase = (ebase + 3) & ~int64_t(3);
        bk.ebase = ebase;
        bk.item0 = item;
        // per-edge types: one item per scalar edge; equality: one item per
        // component pair; every other type: one item per factor
        bk.nitems = bk.per_edge ? nf * bk.arity : bk.type == FGA_EQUAL ? nf * (bk.arity / 2) : nf;
        if (tp) g->tile_pair_ebase = ebase;
        for (int64_t f = 0; f < nf; ++f) {
            const FactorBatch &b = g->batches[bk.members[f].first];
            const int64_t fi = bk.members[f].second;
            const int64_t c0 = b.edge0 + fi * b.arity;
            // disk-tile order: pair slot (unit, column, lane), edge k at
            // unit * kUnitEdges + (column * 6 + k) * 32 + lane
            const int64_t tpos = tp ? (int64_t)g->tile.pair_pos[f] : 0;
            const int64_t tbase = (tpos / 256) * kUnitEdges + ((tpos % 256) / 32) * 6 * 32 + tpos % 32;
            int k = 0;
            for (int v = 0; v < b.nv; ++v) {
                const int64_t var = b.vars[fi * b.nv + v];
                for (int d = 0; d < b.dims[v]; ++d, ++k) {
                    const int64_t s = tp ? ebase + tbase + (int64_t)k * 32
                                         : bk.aos ? ebase + f * bk.arity + k : ebase + (int64_t)k * nf + f;
                    g->s2c[s] = c0 + k;
                    c2s[c0 + k] = s;
                    g->svar[s] = (int32_t)(g->voff[var] + d);
                }
            }
        }
        ebase += tp ? tile_span : nf * bk.arity;
        item += bk.nitems;
    }
    g->es = es;
    if (tile) {
        // storage of the walls' and rewards' first edges
        for (size_t i = 0; i < g->tile.loc.size(); ++i) {
            for (const Bucket &bk : g->buckets) {
                if (bk.type != g->tile.loc_bucket_type[i]) continue;
                const int64_t f = g->tile.loc_member[i];
                g->tile.loc[i].e0 = (int)(bk.aos ? bk.ebase + f * bk.arity : bk.ebase + f);
            }
        }
    }
    g->nitems_f = item;
    // 3. variable-major rows, each in ascending creation order
    const int64_t Z = g->nz;
    std::vector<int32_t> rowp((size_t)Z + 1, 0), pos((size_t)es, 0), fill((size_t)Z, 0);
    std::vector<double> srho_d((size_t)Z, 0.0), srho2_d((size_t)Z, 0.0);
    for (int64_t c = 0; c < E; ++c) rowp[g->svar[c2s[c]] + 1]++;
    for (int64_t b = 0; b < Z; ++b) rowp[b + 1] += rowp[b];
    for (int64_t b = 0; b < Z; ++b) fill[b] = rowp[b];
    for (int64_t c = 0; c < E; ++c) {
        const int64_t s = c2s[c];
        const int32_t b = g->svar[s];
        pos[s] = fill[b]++;
        const double r = edge_rho_c(g, c);
        srho_d[b] += r;        // sequential, ascending creation order
        srho2_d[b] += r * r;
    }
    // 3a. scatter order: an edge of rank k (creation order) in its
    // variable's row goes to column k while k < W, else to the variable's
    // overflow row (its position there replaces pos)
    FastLayout fl;
    if (g->zorder == 4) {
        const int W = g->colw;
        try {
            fl.ev.assign((size_t)es, 0u);
            fl.prow.assign((size_t)Z + 1, 0);
            fl.zovf.assign((size_t)std::max<int64_t>(Z, 1), 0);
        } catch (...) {
            return fail(FGA_ENOMEM, "fga_finalize: out of host memory");
        }
        for (int64_t b = 0; b < Z; ++b) {
            const int d = rowp[b + 1] - rowp[b];
            fl.prow[b + 1] = fl.prow[b] + std::max(0, d - W);
            fl.zovf[b] = d > W ? 1 : 0;
        }
        if ((int64_t)fl.prow[Z] != g->novf) return fail(FGA_EINVAL, "fga_finalize: scatter layout mismatch");
        for (int64_t s = 0; s < es; ++s) {
            if (g->s2c[s] < 0) continue;
            const int32_t b = g->svar[s];
            const int k = pos[s] - rowp[b];
            if (k < W) {
                fl.ev[s] = (uint32_t)b | ((uint32_t)k << kEvColShift);
            } else {
                fl.ev[s] = (uint32_t)b | (kEvOverflow << kEvColShift);
                pos[s] = fl.prow[b] + (k - W);
            }
        }
    }
    // 4. fast z-order: chunks, their slots, and the variable-major partials
    int dev_sms = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, g->device));
    g->blk = g->block ? g->block : 256;
    g->smem = g->zorder == 1   ? chunk_smem((int)g->rsize()).total
              : g->zorder == 4 ? 0
                               : canonical_z_smem((int)g->rsize());
    // kernel variant: 1 = neither hinge / dynamics nor margin / equality
    // paths, 2 = margin / equality paths only, 3 = dynamics of at most 9
    // edges and elementwise paths, 0 = every path
    bool has_hinge = false, dyn = false, dyn_big = false, me = false;
    for (const Bucket &bk : g->buckets) {
        has_hinge = has_hinge || bk.type == FGA_SVM_HINGE;
        dyn = dyn || bk.type == FGA_MPC_DYN;
        dyn_big = dyn_big || (bk.type == FGA_MPC_DYN && bk.arity > 9);
        me = me || bk.type == FGA_SVM_MARGIN || bk.type == FGA_EQUAL;
    }
    g->kind = (has_hinge || dyn_big || (dyn && me)) ? 0 : dyn ? 3 : me ? 2 : 1;
    if (g->zorder == 4) g->kind |= kKindScatter;
    if (tile) {
        g->blk = g->tile.warps * 32;
        g->smem = tile_smem_bytes(g->tile);
    }
    if (hinge) {
        g->blk = kHingeWarps * 32;
        g->smem = hinge_smem_bytes(g->hinge.rows_max);
        for (const Bucket &bk : g->buckets) {
            if (bk.type == FGA_SVM_HINGE) g->hinge_e0 = bk.ebase;
            if (bk.type == FGA_SVM_L2) {
                g->l2_e0 = bk.ebase;
                g->l2_nf = (int64_t)bk.members.size();
            }
        }
        if (es > (int64_t)INT32_MAX / 2) return fail(FGA_EINVAL, "fga_finalize: too many edges for the hinge bank");
    }
    const int bps = (tile || hinge) ? 1
                    : g->precision == FGA_F32 ? sweep_max_blocks_per_sm<float>(g->blk, g->smem, g->kind)
                                              : sweep_max_blocks_per_sm<double>(g->blk, g->smem, g->kind);
    if (bps < 1) return fail(FGA_ECUDA, "fga_finalize: the sweep kernel cannot be resident at %d threads", g->blk);
    g->bps = bps;
    const int64_t full = (int64_t)bps * dev_sms;
    if (g->zorder == 1) {
        // about one chunk per resident CTA, so that phase F is balanced: the
        // smallest chunk size whose chunk count (buckets are cut separately)
        // does not exceed the resident grid
        auto count_chunks = [&](int64_t per) {
            int64_t n = 0;
            for (const Bucket &bk : g->buckets) n += (bk.nitems + per - 1) / per;
            return n;
        };
        int64_t per = std::max<int64_t>(32, (g->nitems_f + full - 1) / full);
        per += per & 1;
        while (per < kChunkItems && count_chunks(per) > full) per += 2 * std::max<int64_t>(1, per / 128);
        per = std::min<int64_t>(kChunkItems, per);
        if ((rc = build_chunks(g, fl, per))) return rc;
        if ((rc = build_zlists(g, fl.prow, false))) return rc;
    } else if (g->zorder == 4) {
        if ((rc = build_zlists(g, fl.prow, true))) return rc;
    }
    // 5. upload
    rc = g->precision == FGA_F32 ? finalize_typed<float>(g, pos, rowp, srho_d, srho2_d, fl)
                                 : finalize_typed<double>(g, pos, rowp, srho_d, srho2_d, fl);
    if (rc) return rc;
    // 6. launch shape: co-resident CTAs, no more than the work needs
    int64_t work;
    if (tile)
        work = (int64_t)g->tile.G * g->blk;
    else if (hinge)
        work = (int64_t)g->hinge.G * g->blk;
    else if (g->zorder == 1)
        work = std::max<int64_t>(std::max<int64_t>((int64_t)g->nchunks * g->blk, g->n_small),
                                 (int64_t)g->n_witems * 32);
    else
        work = std::max<int64_t>(g->nitems_f, Z);
    g->grid = (int)std::max<int64_t>(1, std::min<int64_t>(full, (work + g->blk - 1) / g->blk));
    if (tile || hinge) {
        g->grid = tile ? g->tile.G : g->hinge.G;
        CUDA_TRY(g->t_res.alloc((size_t)4 * g->grid * sizeof(double)));
        CUDA_TRY(cudaMemset(g->t_res.p, 0, g->t_res.bytes));
    }
    CUDA_TRY(g->res_pri.alloc((size_t)g->grid * sizeof(double)));
    CUDA_TRY(g->res_dual.alloc((size_t)2 * g->grid * sizeof(double)));
    CUDA_TRY(cudaMemset(g->res_pri.p, 0, g->res_pri.bytes));
    CUDA_TRY(cudaMemset(g->res_dual.p, 0, g->res_dual.bytes));
    CUDA_TRY(g->ctl.alloc(sizeof(Ctl)));
    CUDA_TRY(g->bar.alloc(sizeof(Barrier)));
    CUDA_TRY(cudaEventCreate(&g->ev0));
    CUDA_TRY(cudaEventCreate(&g->ev1));
    CUDA_TRY(cudaDeviceSynchronize());
    g->finalized = true;
    return FGA_OK;
}

// ---------------------------------------------------------------------------
// host/device pointer helpers
// ---------------------------------------------------------------------------
static bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Copies n doubles from a host-or-device pointer into a host vector.
static int fetch_doubles(const double *src, int64_t n, std::vector<double> &dst, cudaStream_t s) {
    dst.resize((size_t)n);
    if (n == 0) return FGA_OK;
    if (is_device_ptr(src)) {
        CUDA_TRY(cudaMemcpyAsync(dst.data(), src, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
    } else {
        std::memcpy(dst.data(), src, (size_t)n * sizeof(double));
    }
    return FGA_OK;
}

static int deliver_doubles(double *dst, const std::vector<double> &src, cudaStream_t s) {
    if (src.empty()) return FGA_OK;
    if (is_device_ptr(dst)) {
        CUDA_TRY(cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(double), cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaStreamSynchronize(s));
    } else {
        std::memcpy(dst, src.data(), src.size() * sizeof(double));
    }
    return FGA_OK;
}

template <typename R>
static int download(const DevBuf &b, int64_t n, std::vector<R> &out, cudaStream_t s) {
    out.resize((size_t)n);
    if (n == 0) return FGA_OK;
    CUDA_TRY(cudaMemcpyAsync(out.data(), b.p, (size_t)n * sizeof(R), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return FGA_OK;
}

// ---------------------------------------------------------------------------
// init
// ---------------------------------------------------------------------------
template <typename R>
static int init_typed(fga_graph *g, const std::vector<double> &z0, const std::vector<double> &u0) {
    cudaStream_t st = g->stream;
    std::vector<R> zr, ur;
    if (g->nz) {
        if (z0.empty()) {
            CUDA_TRY(cudaMemsetAsync(g->z[0].p, 0, (size_t)g->nz * sizeof(R), st));
        } else {
            zr.resize((size_t)g->nz);
            for (int64_t b = 0; b < g->nz; ++b) zr[b] = (R)z0[b];
            CUDA_TRY(cudaMemcpyAsync(g->z[0].p, zr.data(), zr.size() * sizeof(R), cudaMemcpyHostToDevice, st));
        }
    }
    if (g->es) {
        if (u0.empty()) {
            CUDA_TRY(cudaMemsetAsync(g->u.p, 0, (size_t)g->es * sizeof(R), st));
        } else {
            ur.assign((size_t)g->es, R(0));
            for (int64_t s = 0; s < g->es; ++s)
                if (g->s2c[s] >= 0) ur[s] = (R)u0[g->s2c[s]];
            CUDA_TRY(cudaMemcpyAsync(g->u.p, ur.data(), ur.size() * sizeof(R), cudaMemcpyHostToDevice, st));
        }
        CUDA_TRY(cudaMemsetAsync(g->x[0].p, 0, (size_t)g->es * sizeof(R), st));
        if (g->store_m) CUDA_TRY(cudaMemsetAsync(g->m[0].p, 0, (size_t)g->es * sizeof(R), st));
    }
    if (g->weights) {   // every message starts with standard weight
        CUDA_TRY(cudaMemsetAsync(g->wcls.p, 1, g->wcls.bytes, st));
        CUDA_TRY(cudaMemsetAsync(g->pwcls.p, 1, g->pwcls.bytes, st));
    }
    CUDA_TRY(cudaStreamSynchronize(st));
    return FGA_OK;
}

extern "C" int fga_init(fga_graph *g, const double *z0, const double *u0) {
    if (!g) return fail(FGA_EINVAL, "fga_init: NULL graph");
    if (!g->finalized) return fail(FGA_ESTATE, "fga_init: call fga_finalize first");
    int rc = set_device(g);
    if (rc) return rc;
    std::vector<double> zh, uh;
    if (z0 && (rc = fetch_doubles(z0, g->nz, zh, g->stream))) return rc;
    if (u0 && (rc = fetch_doubles(u0, g->ne, uh, g->stream))) return rc;
    for (double v : zh)
        if (!std::isfinite(v)) return fail(FGA_EINVAL, "fga_init: non-finite z0");
    for (double v : uh)
        if (!std::isfinite(v)) return fail(FGA_EINVAL, "fga_init: non-finite u0");
    rc = g->precision == FGA_F32 ? init_typed<float>(g, zh, uh) : init_typed<double>(g, zh, uh);
    if (rc) return rc;
    g->iters_done = 0;
    g->xpar = 0;
    g->zpar = 0;
    g->tile_resume = false;
    g->shard_pending = false;
    g->last_rp = g->last_rd = std::numeric_limits<double>::quiet_NaN();
    g->initialized = true;
    return FGA_OK;
}

// ---------------------------------------------------------------------------
// iterate
// ---------------------------------------------------------------------------
template <typename R>
static void fill_args(const fga_graph *g, SweepArgs<R> &a) {
    std::memset(&a, 0, sizeof a);
    a.nb = (int)g->buckets.size();
    int pb = 0;
    for (int i = 0; i < a.nb; ++i) {
        const Bucket &bk = g->buckets[i];
        BucketDev<R> &d = a.bk[i];
        d.type = bk.type;
        d.arity = bk.arity;
        d.nprm = bk.np;
        d.per_edge = bk.per_edge ? 1 : 0;
        d.aos = bk.aos ? 1 : 0;
        for (int k = 0; k < 4; ++k) d.dims[k] = k < (int)bk.dims.size() ? bk.dims[k] : 0;
        d.nf = (int)bk.members.size();
        d.ebase = (int)bk.ebase;
        d.item0 = (int)bk.item0;
        d.nitems = (int)bk.nitems;
        d.prm = g->bucket_bufs[pb++]->as<R>();
        if (bk.type == FGA_MPC_DYN) {
            d.pmat = g->bucket_bufs[pb++]->as<R>();
            d.pidx = g->bucket_bufs[pb++]->as<int>();
        }
    }
    a.nitems_f = (int)g->nitems_f;
    a.E = g->ne;
    a.nz = (int)g->nz;
    a.x[0] = g->x[0].as<R>();
    a.x[1] = g->x[1].as<R>();
    a.m[0] = g->store_m ? g->m[0].as<R>() : nullptr;
    a.m[1] = g->store_m ? g->m[1].as<R>() : nullptr;
    a.u = g->u.as<R>();
    a.rho_e = g->uniform_rho ? nullptr : g->rho_e.as<R>();
    a.alpha_e = g->uniform_alpha ? nullptr : g->alpha_e.as<R>();
    a.rho_u = (R)g->rho_u;
    a.alpha_u = (R)g->alpha_u;
    a.svar = g->d_svar.as<int>();
    a.pos = g->d_pos.as<int>();
    a.pvm = g->pvm.as<R>();
    a.z[0] = g->z[0].as<R>();
    a.z[1] = g->z[1].as<R>();
    a.srho = g->srho.as<R>();
    a.srho2 = g->srho2.as<double>();
    a.row = g->row.as<int>();
    a.nchunks = g->nchunks;
    a.chunks = g->chunks.as<ChunkDev>();
    a.slot_var = g->slot_var.as<int>();
    a.ppos = g->ppos.as<int>();
    a.lrow = g->lrow.as<int>();
    a.lidx = g->lidx.as<unsigned>();
    a.part = g->part.as<R>();
    a.prow = g->prow.as<int>();
    a.zorder = g->zorder;
    a.ev = g->zorder == 4 ? g->d_ev.as<unsigned>() : nullptr;
    a.ovf0 = (unsigned)((int64_t)g->colw * g->nz);
    a.colw = g->colw;
    a.zovf = g->zovf.as<unsigned char>();
    a.n_small = g->n_small;
    a.small_vars = g->small_vars.as<int>();
    a.n_witems = g->n_witems;
    a.witems = g->witems.as<int4>();
    a.hub_npieces = g->hub_np.as<int>();
    a.hub_off = g->hub_off.as<int>();
    a.hub_part = g->hub_part.as<R>();
    a.hub_ticket = g->hub_ticket.as<unsigned int>();
    a.wcls = g->weights ? g->wcls.as<unsigned char>() : nullptr;
    a.pwcls = g->weights ? g->pwcls.as<unsigned char>() : nullptr;
    a.prho = g->weights && !g->uniform_rho ? g->prho.as<R>() : nullptr;
    a.res_pri = g->res_pri.as<double>();
    a.res_dual = g->res_dual.as<double>();
    a.gmax = g->grid;
    a.ctl = g->ctl.as<Ctl>();
    a.bar = g->bar.as<Barrier>();
}

// Disk-tile order: one cooperative launch for the whole call (FP32).
static void fill_tile_args(const fga_graph *g, TileArgs &a) {
    const TilePlan &T = g->tile;
    std::memset(&a, 0, sizeof a);
    a.G = T.G;
    a.U = T.U;
    a.smax = T.smax;
    a.stgmax = T.stgmax;
    a.svmax = T.svmax;
    a.locmax = T.locmax;
    a.clmax = T.clmax;
    a.cta = g->t_cta.as<TileCta>();
    a.rowslot = g->t_rowslot.as<unsigned short>();
    a.colslot = g->t_colslot.as<unsigned short>();
    a.mask = g->t_mask.as<unsigned char>();
    a.sv = g->t_sv.as<int4>();
    a.zden = g->t_zden.as<float>();
    a.cptr = g->t_cptr.as<int>();
    a.clist = g->t_clist.as<int>();
    a.loc = g->t_loc.as<TileLocal>();
    a.srho2 = g->srho2.as<double>();
    a.u = g->u.as<float>();
    a.dsave = g->t_dsave.as<float>();
    a.dres = g->t_dres.as<float>();
    a.dlive = T.W > T.warps ? g->t_dlive.as<float>() : nullptr;
    a.lres = g->t_lres.as<float>();
    a.zpin = g->t_zprev.as<float>();
    a.zpout = g->t_zprev.as<float>();
    a.resume = g->tile_resume ? 1 : 0;
    a.xw = g->xpar ^ 1;
    a.zw = g->zpar ^ 1;
    a.xout = g->x[a.xw].as<float>();
    a.zin = g->z[g->zpar].as<float>();
    a.zout = g->z[a.zw].as<float>();
    a.acc = g->t_part.as<unsigned long long>();
    a.ptot = T.ptot;
    a.res = g->t_res.as<double>();
    a.pair_ebase = (int)g->tile_pair_ebase;
    a.alpha = (float)g->alpha_u;
    a.E = g->ne;
    a.ctl = g->ctl.as<Ctl>();
    a.sync = g->bar.as<TileSync>();
}

static int iterate_tile(fga_graph *g, const fga_iter_opts &o, fga_iter_result &res) {
    TileArgs a;
    fill_tile_args(g, a);
    a.k0 = g->iters_done;
    a.K = o.max_iters;
    a.check_every = o.check_every;
    a.tol_pri = o.tol_pri;
    a.tol_dual = o.tol_dual;
    a.timeout_ns = o.barrier_timeout_ns > 0 ? o.barrier_timeout_ns : 2000000000LL;
    a.skip_block = o.fault_skip_block;
    cudaStream_t s = g->stream;
    if (a.K <= 0) {
        res.iters = 0;
        res.r_pri = g->last_rp;
        res.r_dual = g->last_rd;
        res.status = FGA_OK;
        res.ms = 0.f;
        return FGA_OK;
    }
    CUDA_TRY(cudaMemsetAsync(g->ctl.p, 0, sizeof(Ctl), s));
    CUDA_TRY(cudaMemsetAsync(g->bar.p, 0, sizeof(TileSync), s));
    CUDA_TRY(cudaMemsetAsync(g->t_part.p, 0, g->t_part.bytes, s));   // the count-and-sum words
    // z of variables outside every tile (none in a qualifying graph) keep
    // their value in the buffer the call writes
    CUDA_TRY(cudaMemcpyAsync(a.zout, a.zin, (size_t)g->nz * sizeof(float), cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaEventRecord(g->ev0, s));
    CUDA_TRY(tile_sweep_launch(a, g->blk, g->smem, s));
    CUDA_TRY(cudaEventRecord(g->ev1, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, g->ev0, g->ev1));
    Ctl c;
    TileSync b;
    CUDA_TRY(cudaMemcpy(&c, g->ctl.p, sizeof c, cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(&b, g->bar.p, sizeof b, cudaMemcpyDeviceToHost));
    res.ms = ms;
    if (b.error) {
        g->initialized = false;
        res.iters = 0;
        res.r_pri = res.r_dual = std::numeric_limits<double>::quiet_NaN();
        res.status = b.error;
        return fail(b.error, "fga_iterate: a grid-wide wait timed out (status %d)", b.error);
    }
    if (!c.done) return fail(FGA_ECUDA, "fga_iterate: the sweep ended without reporting");
    g->iters_done += c.iters;
    g->xpar = c.xpar;
    g->zpar = c.zpar;
    g->last_rp = c.r_pri;
    g->last_rd = c.r_dual;
    g->tile_resume = a.alpha == 1.0f;
    res.iters = c.iters;
    res.r_pri = c.r_pri;
    res.r_dual = c.r_dual;
    res.status = c.status;
    if (c.status == FGA_ENONFINITE) return fail(FGA_ENONFINITE, "fga_iterate: residual became non-finite");
    return FGA_OK;
}

static void fill_hinge_args(const fga_graph *g, HingeArgs &a) {
    const HingePlan &H = g->hinge;
    const HingeInput &in = g->hin;
    std::memset(&a, 0, sizeof a);
    a.G = H.G;
    a.N = (int)in.N;
    a.D = in.D;
    a.nl2 = (int)in.lam.size();
    a.cta = g->h_cta.as<HingeCta>();
    a.X = g->h_X.as<float>();
    a.meta = g->h_meta.as<float4>();
    for (int f = 0; f < a.nl2; ++f) a.lam[f] = in.lam[f];
    a.rho = (float)g->rho_u;
    a.inv_rho = (float)(1.0 / g->rho_u);
    a.deg_w = (int)(in.N + (int64_t)in.lam.size());
    a.deg_b = (int)in.N;
    a.rows_max = H.rows_max;
    a.u = g->u.as<float>();
    a.xw = g->xpar ^ 1;
    a.zw = g->zpar ^ 1;
    a.xout = g->x[a.xw].as<float>();
    a.zin = g->z[g->zpar].as<float>();
    a.zout = g->z[a.zw].as<float>();
    a.zpin = g->t_zprev.as<float>();
    a.zpout = g->t_zprev.as<float>();
    a.vw = in.vw;
    a.vb = in.vb;
    a.hb_e0 = (int)g->hinge_e0;
    a.l2_e0 = (int)g->l2_e0;
    a.l2_nf = (int)g->l2_nf;
    a.acc = g->h_acc.as<unsigned long long>();
    a.gsave = g->h_gsave.as<float>();
    a.gres = g->h_gres.as<float>();
    a.l2save = g->h_l2save.as<float>();
    a.l2res = g->h_l2res.as<float>();
    a.resume = g->tile_resume ? 1 : 0;
    a.res = g->t_res.as<double>();
    a.E = g->ne;
    a.ctl = g->ctl.as<Ctl>();
    a.sync = g->bar.as<TileSync>();
}

// Hinge bank: one cooperative launch for the whole call (FP32, alpha = 1).
static int iterate_hinge(fga_graph *g, const fga_iter_opts &o, fga_iter_result &res) {
    HingeArgs a;
    fill_hinge_args(g, a);
    a.k0 = g->iters_done;
    a.K = o.max_iters;
    a.check_every = o.check_every;
    a.tol_pri = o.tol_pri;
    a.tol_dual = o.tol_dual;
    a.timeout_ns = o.barrier_timeout_ns > 0 ? o.barrier_timeout_ns : 2000000000LL;
    a.skip_block = o.fault_skip_block;
    cudaStream_t s = g->stream;
    if (a.K <= 0) {
        res.iters = 0;
        res.r_pri = g->last_rp;
        res.r_dual = g->last_rd;
        res.status = FGA_OK;
        res.ms = 0.f;
        return FGA_OK;
    }
    CUDA_TRY(cudaMemsetAsync(g->ctl.p, 0, sizeof(Ctl), s));
    CUDA_TRY(cudaMemsetAsync(g->bar.p, 0, sizeof(TileSync), s));
    CUDA_TRY(cudaMemsetAsync(g->h_acc.p, 0, g->h_acc.bytes, s));   // the count-and-sum words
    CUDA_TRY(cudaMemcpyAsync(a.zout, a.zin, (size_t)g->nz * sizeof(float), cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaEventRecord(g->ev0, s));
    CUDA_TRY(hinge_sweep_launch(a, g->smem, s));
    CUDA_TRY(cudaEventRecord(g->ev1, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, g->ev0, g->ev1));
    Ctl c;
    TileSync b;
    CUDA_TRY(cudaMemcpy(&c, g->ctl.p, sizeof c, cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(&b, g->bar.p, sizeof b, cudaMemcpyDeviceToHost));
    res.ms = ms;
    if (b.error) {
        g->initialized = false;
        res.iters = 0;
        res.r_pri = res.r_dual = std::numeric_limits<double>::quiet_NaN();
        res.status = b.error;
        return fail(b.error, "fga_iterate: a grid-wide wait timed out (status %d)", b.error);
    }
    if (!c.done) return fail(FGA_ECUDA, "fga_iterate: the sweep ended without reporting");
    g->iters_done += c.iters;
    g->xpar = c.xpar;
    g->zpar = c.zpar;
    g->last_rp = c.r_pri;
    g->last_rd = c.r_dual;
    g->tile_resume = true;
    res.iters = c.iters;
    res.r_pri = c.r_pri;
    res.r_dual = c.r_dual;
    res.status = c.status;
    if (c.status == FGA_ENONFINITE) return fail(FGA_ENONFINITE, "fga_iterate: residual became non-finite");
    return FGA_OK;
}

// The x-update of every bucket of a user operator, in phase-F mode `mode`,
// after the built-in types' phase F of the same iteration (same stream).
template <typename R>
static int user_xsteps(fga_graph *g, const SweepArgs<R> &a, int mode, int xp, int zp, cudaStream_t s) {
    for (const auto &ub : g->ubk) {
        const Bucket &bk = g->buckets[ub->bucket];
        UserLaunch L;
        L.mode = mode;
        L.nf = (int)bk.members.size();
        L.ebase = (int)bk.ebase;
        L.var = ub->var.as<int>();
        L.dst = ub->dst.as<unsigned>();
        L.zc = a.z[zp];
        L.xin = a.x[xp];
        L.xout = a.x[xp ^ 1];
        L.u = a.u;
        L.mout = a.m[xp ^ 1];
        L.pvm = a.pvm;
        L.rho_e = a.rho_e;
        L.rho_u = g->rho_u;
        L.alpha_e = a.alpha_e;
        L.alpha_u = g->alpha_u;
        L.prm = g->bucket_bufs[bk.prm_buf]->p;
        L.res_pri = a.res_pri;
        L.done = reinterpret_cast<const int *>(reinterpret_cast<const char *>(a.ctl) + offsetof(Ctl, done));
        CUDA_TRY(user_launch(g->users[ub->user], g->precision == FGA_F64, L, g->grid, g->blk, s));
    }
    return FGA_OK;
}

template <typename R>
static int iterate_typed(fga_graph *g, const fga_iter_opts &o, fga_iter_result &res) {
    SweepArgs<R> a;
    fill_args(g, a);
    a.k0 = g->iters_done;
    a.K = o.max_iters;
    a.check_every = o.check_every;
    a.tol_pri = o.tol_pri;
    a.tol_dual = o.tol_dual;
    a.timeout_ns = o.barrier_timeout_ns > 0 ? o.barrier_timeout_ns : 2000000000LL;
    a.skip_block = o.fault_skip_block;
    a.xpar0 = g->xpar;
    a.zpar0 = g->zpar;
    cudaStream_t s = g->stream;
    CUDA_TRY(cudaMemsetAsync(g->ctl.p, 0, sizeof(Ctl), s));
    CUDA_TRY(cudaMemsetAsync(g->bar.p, 0, sizeof(Barrier), s));
    if (g->n_hubs) CUDA_TRY(cudaMemsetAsync(g->hub_ticket.p, 0, g->hub_ticket.bytes, s));
    CUDA_TRY(cudaEventRecord(g->ev0, s));
    int rc;
    if (o.fused && !g->has_user()) {
        CUDA_TRY(sweep_persistent<R>(a, g->grid, g->blk, g->smem, g->kind, s));
    } else {
        // one launch per phase (and the graph's user operators run their
        // own kernels between phase F and the check)
        int xp = g->xpar, zp = g->zpar;
        for (long long it = 1; it <= a.K; ++it) {
            const bool pend = it > 1;
            const bool chk = pend && ((a.k0 + it - 1) % a.check_every == 0);
            const int mode = !pend ? F_PROX : chk ? F_U_PROX_CHK : F_U_PROX;
            CUDA_TRY(sweep_phase_f<R>(a, mode, xp, zp, g->grid, g->blk, g->smem, g->kind, s));
            if ((rc = user_xsteps<R>(g, a, mode, xp, zp, s))) return rc;
            if (chk) CUDA_TRY(sweep_check<R>(a, it - 1, xp, zp, 0, g->grid, s));
            xp ^= 1;
            const bool chkz = ((a.k0 + it) % a.check_every == 0) || it == a.K;
            CUDA_TRY(sweep_phase_z<R>(a, zp, it, chkz ? 1 : 0, g->grid, g->blk, s));
            zp ^= 1;
        }
        if (a.K > 0) {
            CUDA_TRY(sweep_phase_f<R>(a, F_U_ONLY, xp, zp, g->grid, g->blk, g->smem, g->kind, s));
            if ((rc = user_xsteps<R>(g, a, F_U_ONLY, xp, zp, s))) return rc;
            CUDA_TRY(sweep_check<R>(a, a.K, xp, zp, 1, g->grid, s));
        }
    }
    CUDA_TRY(cudaEventRecord(g->ev1, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, g->ev0, g->ev1));
    Ctl c;
    Barrier b;
    CUDA_TRY(cudaMemcpy(&c, g->ctl.p, sizeof c, cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(&b, g->bar.p, sizeof b, cudaMemcpyDeviceToHost));
    res.ms = ms;
    if (b.error) {
        // the state is undefined after an aborted launch; a new fga_init is needed
        g->initialized = false;
        res.iters = 0;
        res.r_pri = res.r_dual = std::numeric_limits<double>::quiet_NaN();
        res.status = b.error;
        return fail(b.error, "fga_iterate: a grid-wide wait timed out (status %d)", b.error);
    }
    if (a.K <= 0) {
        res.iters = 0;
        res.r_pri = g->last_rp;
        res.r_dual = g->last_rd;
        res.status = FGA_OK;
        return FGA_OK;
    }
    if (!c.done) return fail(FGA_ECUDA, "fga_iterate: the sweep ended without reporting");
    g->iters_done += c.iters;
    g->xpar = c.xpar;
    g->zpar = c.zpar;
    g->last_rp = c.r_pri;
    g->last_rd = c.r_dual;
    res.iters = c.iters;
    res.r_pri = c.r_pri;
    res.r_dual = c.r_dual;
    res.status = c.status;
    if (c.status == FGA_ENONFINITE) return fail(FGA_ENONFINITE, "fga_iterate: residual became non-finite");
    return FGA_OK;
}

extern "C" int fga_iterate(fga_graph *g, const fga_iter_opts *opts, fga_iter_result *result) {
    if (!g || !opts || !result) return fail(FGA_EINVAL, "fga_iterate: NULL argument");
    if (!g->finalized || !g->initialized) return fail(FGA_ESTATE, "fga_iterate: call fga_finalize and fga_init first");
    if (opts->max_iters < 0 || opts->check_every < 1 || opts->tol_pri < 0 || opts->tol_dual < 0)
        return fail(FGA_EINVAL, "fga_iterate: bad options");
    if (opts->fault_skip_block >= 0 && (!opts->fused || g->has_user()))
        return fail(FGA_EINVAL, "fga_iterate: fault_skip_block needs the fused kernel (graphs with user operators "
                                "run one launch per phase)");
    if (g->shard) return fail(FGA_ESTATE, "fga_iterate: the graph is a shard (use fga_shard_xstep / zstep)");
    if ((g->zorder == 2 || g->zorder == 3) && !opts->fused)
        return fail(FGA_EINVAL, "fga_iterate: the disk-tile and hinge-bank orders run as one persistent launch "
                                "(fused = 1); set FGA_OPT_ZORDER 1 for one launch per phase");
    int rc = set_device(g);
    if (rc) return rc;
    fga_iter_result r;
    std::memset(&r, 0, sizeof r);
    rc = g->zorder == 2                ? iterate_tile(g, *opts, r)
         : g->zorder == 3              ? iterate_hinge(g, *opts, r)
         : g->precision == FGA_F32 ? iterate_typed<float>(g, *opts, r)
                                   : iterate_typed<double>(g, *opts, r);
    *result = r;   // also on timeout / non-finite, so the caller sees the status
    return rc;
}

// ---------------------------------------------------------------------------
// shard mode: one rank's slice of the factors of a graph split across GPUs
// ---------------------------------------------------------------------------
extern "C" int fga_shard_rho_chain(const fga_graph *g, const double *srho_in, const double *srho2_in,
                                   double *srho_out, double *srho2_out) {
    if (!g || !srho_out || !srho2_out) return fail(FGA_EINVAL, "fga_shard_rho_chain: NULL argument");
    if (!g->finalized) return fail(FGA_ESTATE, "fga_shard_rho_chain: call fga_finalize first");
    const int64_t Z = g->nz;
    std::vector<double> r((size_t)Z, 0.0), r2((size_t)Z, 0.0);
    for (int64_t b = 0; b < Z; ++b) {
        if (srho_in) r[b] = srho_in[b];
        if (srho2_in) r2[b] = srho2_in[b];
    }
    // this shard's edges in creation order, onto the incoming sums one by one
    std::vector<int64_t> c2s((size_t)g->ne, -1);
    for (int64_t s2 = 0; s2 < g->es; ++s2)
        if (g->s2c[s2] >= 0) c2s[g->s2c[s2]] = s2;
    for (int64_t c = 0; c < g->ne; ++c) {
        const int32_t b = g->svar[c2s[c]];
        const double v = edge_rho_c(g, c);
        r[b] += v;
        r2[b] += v * v;
    }
    std::memcpy(srho_out, r.data(), (size_t)Z * sizeof(double));
    std::memcpy(srho2_out, r2.data(), (size_t)Z * sizeof(double));
    return FGA_OK;
}

// The z-step's launch shape depends only on the number of variables, never
// on the shard: every rank then sums the (graph-wide) dual residual in the
// same order and takes the same stop decision.
constexpr int kShardZGrid = 1024, kShardZBlock = 256;

template <typename R>
static int shard_begin_typed(fga_graph *g, const double *srho, const double *srho2) {
    std::vector<R> v((size_t)g->nz);
    for (int64_t b = 0; b < g->nz; ++b) v[b] = (R)srho[b];
    std::vector<double> v2(srho2, srho2 + g->nz);
    int rc;
    if ((rc = upload_vec(g->srho, v))) return rc;
    if ((rc = upload_vec(g->srho2, v2))) return rc;
    CUDA_TRY(g->shard_res.alloc(kShardZGrid * sizeof(double)));
    CUDA_TRY(cudaMemset(g->ctl.p, 0, sizeof(Ctl)));
    // the uploads and the memset ran on the legacy stream, which a
    // non-blocking caller stream does not wait for
    CUDA_TRY(cudaDeviceSynchronize());
    return FGA_OK;
}

extern "C" int fga_shard_begin(fga_graph *g, const double *srho_total, const double *srho2_total) {
    if (!g || !srho_total || !srho2_total) return fail(FGA_EINVAL, "fga_shard_begin: NULL argument");
    if (!g->finalized) return fail(FGA_ESTATE, "fga_shard_begin: call fga_finalize first");
    if (g->zorder != 0 && g->zorder != 1)
        return fail(FGA_EINVAL, "fga_shard_begin: shards run the canonical or the fast z-order (FGA_OPT_ZORDER 0 "
                                "or 1), not the disk-tile or hinge-bank kernels");
    if (g->weights) return fail(FGA_EINVAL, "fga_shard_begin: shards run fixed weights (FGA_OPT_WEIGHTS 0)");
    if (g->has_user()) return fail(FGA_EINVAL, "fga_shard_begin: shards run the built-in factor types only");
    for (int64_t b = 0; b < g->nz; ++b)
        if (!std::isfinite(srho_total[b]) || srho_total[b] < 0.0 || !std::isfinite(srho2_total[b]))
            return fail(FGA_EINVAL, "fga_shard_begin: bad graph-wide rho sum at variable %lld", (long long)b);
    int rc = set_device(g);
    if (rc) return rc;
    rc = g->precision == FGA_F32 ? shard_begin_typed<float>(g, srho_total, srho2_total)
                                 : shard_begin_typed<double>(g, srho_total, srho2_total);
    if (rc) return rc;
    g->shard = true;
    g->shard_pending = false;
    return FGA_OK;
}

template <typename R>
static int shard_xstep_typed(fga_graph *g, int check_prev, const void *s_in, void *s_out, double *pri_out) {
    SweepArgs<R> a;
    fill_args(g, a);
    cudaStream_t s = g->stream;
    const int mode = !g->shard_pending ? F_PROX : check_prev ? F_U_PROX_CHK : F_U_PROX;
    CUDA_TRY(sweep_phase_f<R>(a, mode, g->xpar, g->zpar, g->grid, g->blk, g->smem, g->kind, s));
    if (mode == F_U_PROX_CHK) CUDA_TRY(shard_total<R>(a.res_pri, g->grid, pri_out, s));
    // the shard touches only some variables: the others pass s_in through
    if (g->zorder == 1) {
        if (s_in) CUDA_TRY(cudaMemcpyAsync(s_out, s_in, (size_t)g->nz * sizeof(R), cudaMemcpyDeviceToDevice, s));
        else CUDA_TRY(cudaMemsetAsync(s_out, 0, (size_t)g->nz * sizeof(R), s));
    }
    CUDA_TRY(shard_sums<R>(a, static_cast<const R *>(s_in), static_cast<R *>(s_out), g->grid, g->blk, s));
    g->shard_pending = false;
    return FGA_OK;
}

extern "C" int fga_shard_xstep(fga_graph *g, int32_t check_prev, const void *s_in, void *s_out, double *pri_out) {
    if (!g || !s_out) return fail(FGA_EINVAL, "fga_shard_xstep: NULL argument");
    if (!g->shard || !g->initialized) return fail(FGA_ESTATE, "fga_shard_xstep: call fga_shard_begin and fga_init");
    if (check_prev && (!g->shard_pending || !pri_out))
        return fail(FGA_EINVAL, "fga_shard_xstep: no pending iteration to check, or NULL pri_out");
    int rc = set_device(g);
    if (rc) return rc;
    return g->precision == FGA_F32 ? shard_xstep_typed<float>(g, check_prev, s_in, s_out, pri_out)
                                   : shard_xstep_typed<double>(g, check_prev, s_in, s_out, pri_out);
}

extern "C" int fga_shard_add_parts(fga_graph *g, const void *parts, int32_t n_shards, void *total) {
    if (!g || !parts || !total || n_shards < 1) return fail(FGA_EINVAL, "fga_shard_add_parts: bad argument");
    if (!g->shard) return fail(FGA_ESTATE, "fga_shard_add_parts: call fga_shard_begin first");
    int rc = set_device(g);
    if (rc) return rc;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(1024, (g->nz + 255) / 256));
    if (g->precision == FGA_F32)
        CUDA_TRY(shard_add_parts<float>(static_cast<const float *>(parts), n_shards, g->nz, static_cast<float *>(total),
                                        grid, g->stream));
    else
        CUDA_TRY(shard_add_parts<double>(static_cast<const double *>(parts), n_shards, g->nz,
                                         static_cast<double *>(total), grid, g->stream));
    return FGA_OK;
}

template <typename R>
static int shard_zstep_typed(fga_graph *g, const void *total, int check, double *dual_out) {
    SweepArgs<R> a;
    fill_args(g, a);
    cudaStream_t s = g->stream;
    const int xp = g->xpar ^ 1;   // the x of the x-step just run
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(kShardZGrid, (g->nz + kShardZBlock - 1) /
                                                                                  kShardZBlock));
    a.res_dual = g->shard_res.as<double>();
    CUDA_TRY(shard_z<R>(a, static_cast<const R *>(total), g->zpar, check, grid, kShardZBlock, s));
    if (check) CUDA_TRY(shard_total<R>(a.res_dual, grid, dual_out, s));
    g->xpar = xp;
    g->zpar ^= 1;
    g->iters_done += 1;
    g->shard_pending = true;
    return FGA_OK;
}

extern "C" int fga_shard_zstep(fga_graph *g, const void *total, int32_t check, double *dual_out) {
    if (!g || !total || (check && !dual_out)) return fail(FGA_EINVAL, "fga_shard_zstep: NULL argument");
    if (!g->shard || !g->initialized) return fail(FGA_ESTATE, "fga_shard_zstep: call fga_shard_begin and fga_init");
    int rc = set_device(g);
    if (rc) return rc;
    return g->precision == FGA_F32 ? shard_zstep_typed<float>(g, total, check, dual_out)
                                   : shard_zstep_typed<double>(g, total, check, dual_out);
}

template <typename R>
static int shard_finish_typed(fga_graph *g, double *pri_out) {
    SweepArgs<R> a;
    fill_args(g, a);
    CUDA_TRY(sweep_phase_f<R>(a, F_U_ONLY, g->xpar, g->zpar, g->grid, g->blk, g->smem, g->kind, g->stream));
    CUDA_TRY(shard_total<R>(a.res_pri, g->grid, pri_out, g->stream));
    g->shard_pending = false;
    return FGA_OK;
}

extern "C" int fga_shard_finish(fga_graph *g, double *pri_out) {
    if (!g || !pri_out) return fail(FGA_EINVAL, "fga_shard_finish: NULL argument");
    if (!g->shard || !g->initialized) return fail(FGA_ESTATE, "fga_shard_finish: call fga_shard_begin and fga_init");
    if (!g->shard_pending) return fail(FGA_ESTATE, "fga_shard_finish: no pending u-update");
    int rc = set_device(g);
    if (rc) return rc;
    return g->precision == FGA_F32 ? shard_finish_typed<float>(g, pri_out) : shard_finish_typed<double>(g, pri_out);
}

extern "C" int fga_shard_stop_rule(const double *pri_parts, int32_t n_shards, double dual, int64_t num_edges,
                                   double tol_pri, double tol_dual, double *r_pri, double *r_dual, int32_t *stop) {
    if (!pri_parts || n_shards < 1 || num_edges < 0 || !r_pri || !r_dual || !stop)
        return fail(FGA_EINVAL, "fga_shard_stop_rule: bad argument");
    double sp = 0.0;
    for (int32_t r = 0; r < n_shards; ++r) sp += pri_parts[r];   // rank order
    const double E = num_edges > 0 ? (double)num_edges : 1.0;
    *r_pri = std::sqrt(sp / E);
    *r_dual = std::sqrt(dual / E);
    const bool finite = std::isfinite(*r_pri) && std::isfinite(*r_dual);
    *stop = !finite || (*r_pri <= tol_pri && *r_dual <= tol_dual);
    return FGA_OK;
}

extern "C" int fga_latency_floor(fga_graph *g, int64_t iters, int32_t mode, float *ms) {
    if (!g || !ms || iters < 1 || (mode != 0 && mode != 1)) return fail(FGA_EINVAL, "fga_latency_floor: bad argument");
    if (!g->finalized) return fail(FGA_ESTATE, "fga_latency_floor: call fga_finalize first");
    if (g->zorder != 2 && g->zorder != 3)
        return fail(FGA_EINVAL, "fga_latency_floor: the disk-tile and hinge-bank orders only");
    int rc = set_device(g);
    if (rc) return rc;
    cudaStream_t s = g->stream;
    CUDA_TRY(cudaMemsetAsync(g->bar.p, 0, sizeof(TileSync), s));
    if (g->zorder == 2) {
        TileArgs a;
        fill_tile_args(g, a);
        a.timeout_ns = 2000000000LL;
        CUDA_TRY(cudaMemsetAsync(g->t_part.p, 0, g->t_part.bytes, s));   // the next solve zeroes them again
        CUDA_TRY(cudaEventRecord(g->ev0, s));
        CUDA_TRY(tile_floor_launch(a, iters, mode, g->blk, g->smem, s));
    } else {
        HingeArgs a;
        fill_hinge_args(g, a);
        a.timeout_ns = 2000000000LL;
        CUDA_TRY(cudaMemsetAsync(g->h_acc.p, 0, g->h_acc.bytes, s));   // the next solve zeroes them again
        CUDA_TRY(cudaEventRecord(g->ev0, s));
        CUDA_TRY(hinge_floor_launch(a, iters, mode, s));
    }
    CUDA_TRY(cudaEventRecord(g->ev1, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    float t = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&t, g->ev0, g->ev1));
    TileSync b;
    CUDA_TRY(cudaMemcpy(&b, g->bar.p, sizeof b, cudaMemcpyDeviceToHost));
    if (b.error) return fail(b.error, "fga_latency_floor: a grid-wide wait timed out");
    *ms = t;
    return FGA_OK;
}

extern "C" int fga_launch_info(const fga_graph *g, int64_t *info, int32_t n) {
    if (!g || !info || n < 6) return fail(FGA_EINVAL, "fga_launch_info: need an array of 6");
    if (!g->finalized) return fail(FGA_ESTATE, "fga_launch_info: graph not finalized");
    info[0] = g->grid;
    info[1] = g->blk;
    info[2] = g->smem;
    info[3] = g->bps;
    info[4] = g->zorder == 1   ? g->nchunks
              : g->zorder == 2 ? g->tile.U
              : g->zorder == 3 ? g->hinge.G
              : g->zorder == 4 ? g->colw
                               : 0;
    info[5] = (int64_t)g->buckets.size();
    if (n >= 7) info[6] = g->zorder;
    return FGA_OK;
}

extern "C" int fga_residuals(const fga_graph *g, double *r_pri, double *r_dual) {
    if (!g) return fail(FGA_EINVAL, "fga_residuals: NULL graph");
    if (r_pri) *r_pri = g->last_rp;
    if (r_dual) *r_dual = g->last_rd;
    return FGA_OK;
}

// ---------------------------------------------------------------------------
// readout
// ---------------------------------------------------------------------------
template <typename R>
static int read_z_typed(fga_graph *g, double *out) {
    std::vector<R> zr;
    int rc = download(g->z[g->zpar], g->nz, zr, g->stream);
    if (rc) return rc;
    std::vector<double> zd(zr.begin(), zr.end());
    return deliver_doubles(out, zd, g->stream);
}

extern "C" int fga_read_z(fga_graph *g, double *out, int64_t n) {
    if (!g || (!out && n)) return fail(FGA_EINVAL, "fga_read_z: NULL argument");
    if (!g->finalized) return fail(FGA_ESTATE, "fga_read_z: graph not finalized");
    if (n != g->nz) return fail(FGA_EINVAL, "fga_read_z: n = %lld, graph has %lld scalar variables", (long long)n,
                                (long long)g->nz);
    int rc = set_device(g);
    if (rc) return rc;
    return g->precision == FGA_F32 ? read_z_typed<float>(g, out) : read_z_typed<double>(g, out);
}

template <typename R>
static int read_edge_typed(fga_graph *g, int which, double *out) {
    const int64_t ES = g->es;
    std::vector<R> v, u, z;
    int rc;
    std::vector<double> res((size_t)g->ne);
    if (which == FGA_EDGE_X || which == FGA_EDGE_M) {
        const DevBuf &b = which == FGA_EDGE_X ? g->x[g->xpar] : g->m[g->xpar];
        if ((rc = download(b, ES, v, g->stream))) return rc;
        for (int64_t s = 0; s < ES; ++s)
            if (g->s2c[s] >= 0) res[g->s2c[s]] = (double)v[s];
    } else if (which == FGA_EDGE_U) {
        if ((rc = download(g->u, ES, u, g->stream))) return rc;
        for (int64_t s = 0; s < ES; ++s)
            if (g->s2c[s] >= 0) res[g->s2c[s]] = (double)u[s];
    } else {
        // n = z_b - u, evaluated in the working precision as the sweep does
        if ((rc = download(g->u, ES, u, g->stream))) return rc;
        if ((rc = download(g->z[g->zpar], g->nz, z, g->stream))) return rc;
        for (int64_t s = 0; s < ES; ++s) {
            if (g->s2c[s] < 0) continue;
            const R n = z[g->svar[s]] - u[s];
            res[g->s2c[s]] = (double)n;
        }
    }
    return deliver_doubles(out, res, g->stream);
}

extern "C" int fga_read_edge_state(fga_graph *g, int32_t which, double *out, int64_t n) {
    if (!g || (!out && n)) return fail(FGA_EINVAL, "fga_read_edge_state: NULL argument");
    if (!g->finalized) return fail(FGA_ESTATE, "fga_read_edge_state: graph not finalized");
    if (which < FGA_EDGE_X || which > FGA_EDGE_N) return fail(FGA_EINVAL, "fga_read_edge_state: bad array %d", which);
    if (which == FGA_EDGE_M && !g->store_m)
        return fail(FGA_ESTATE, "fga_read_edge_state: m is not kept (set FGA_OPT_STORE_M before finalize)");
    if (n != g->ne) return fail(FGA_EINVAL, "fga_read_edge_state: n = %lld, graph has %lld edges", (long long)n,
                                (long long)g->ne);
    int rc = set_device(g);
    if (rc) return rc;
    return g->precision == FGA_F32 ? read_edge_typed<float>(g, which, out) : read_edge_typed<double>(g, which, out);
}

extern "C" int fga_destroy(fga_graph *g) {
    if (!g) return FGA_OK;
    if (g->finalized) {
        cudaSetDevice(g->device);
        cudaStreamSynchronize(g->stream);
        if (g->ev0) cudaEventDestroy(g->ev0);
        if (g->ev1) cudaEventDestroy(g->ev1);
    }
    if (!g->users.empty()) {
        cudaSetDevice(g->device);
        for (UserProg &p : g->users) user_release(p);
    }
    delete g;
    return FGA_OK;
}
