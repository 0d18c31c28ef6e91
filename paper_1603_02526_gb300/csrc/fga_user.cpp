// fga_user.cpp -- user-supplied proximal operators.
//
// The paper's addNode takes each factor's proximal operator as a function
// pointer (Sec. III).  A GPU kernel cannot call a host function pointer, so
// here the caller hands over the operator as CUDA source: a device function
// template fn<R>(arity, n, rho, params, x).  It is compiled at run time with
// NVRTC, together with a generated kernel that runs the x-update of every
// factor of that type: the deferred u- and n-update of the previous
// iteration on the factor's edges, the operator, then x, m = x + u and rho m
// into the z-reduction's input slot of each edge -- the same per-edge steps
// the built-in types take (Algorithm 2, Sec. II).  The kernel runs in the
// one-launch-per-phase sweep, after the built-in types' x-update.
//
// NVRTC is opened with dlopen on first use, so the library loads (and every
// other entry point works) where it is absent; registering an operator then
// fails with FGA_ECUDA.
#include <dlfcn.h>

#include <cctype>
#include <cstdlib>
#include <mutex>
#include <string>
#include <vector>

#include <nvrtc.h>

#include "user_internal.h"

namespace fga {

namespace {

struct Nvrtc {
    decltype(&nvrtcCreateProgram) create = nullptr;
    decltype(&nvrtcCompileProgram) compile = nullptr;
    decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
    decltype(&nvrtcGetProgramLog) log = nullptr;
    decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
    decltype(&nvrtcGetCUBIN) cubin = nullptr;
    decltype(&nvrtcDestroyProgram) destroy = nullptr;
    decltype(&nvrtcGetErrorString) error_string = nullptr;
    bool ok = false;
    std::string why;
};

const Nvrtc &nvrtc() {
    static Nvrtc n;
    static std::once_flag once;
    std::call_once(once, [] {
        std::vector<std::string> names = {"libnvrtc.so.13", "libnvrtc.so"};
        for (const char *env : {"CUDA_HOME", "CUDA_PATH"}) {
            const char *h = std::getenv(env);
            if (h && *h) names.push_back(std::string(h) + "/lib64/libnvrtc.so.13");
        }
        names.push_back("/usr/local/cuda/lib64/libnvrtc.so.13");
        void *h = nullptr;
        for (const std::string &s : names)
            if ((h = dlopen(s.c_str(), RTLD_NOW | RTLD_LOCAL))) break;
        if (!h) {
            n.why = "NVRTC (libnvrtc.so.13) not found";
            return;
        }
        n.create = (decltype(n.create))dlsym(h, "nvrtcCreateProgram");
        n.compile = (decltype(n.compile))dlsym(h, "nvrtcCompileProgram");
        n.log_size = (decltype(n.log_size))dlsym(h, "nvrtcGetProgramLogSize");
        n.log = (decltype(n.log))dlsym(h, "nvrtcGetProgramLog");
        n.cubin_size = (decltype(n.cubin_size))dlsym(h, "nvrtcGetCUBINSize");
        n.cubin = (decltype(n.cubin))dlsym(h, "nvrtcGetCUBIN");
        n.destroy = (decltype(n.destroy))dlsym(h, "nvrtcDestroyProgram");
        n.error_string = (decltype(n.error_string))dlsym(h, "nvrtcGetErrorString");
        n.ok = n.create && n.compile && n.log_size && n.log && n.cubin_size && n.cubin && n.destroy && n.error_string;
        if (!n.ok) n.why = "NVRTC library lacks an expected entry point";
    });
    return n;
}

// The generated x-update kernel (after the user's source).  Modes are the
// phase-F modes of the built-in sweep: 0 x-update only (first iteration of a
// call), 1 deferred u/n-update then x-update, 3 the same on a checked
// iteration (also the primal-residual partial), 2 u-update only (end of a
// call, with the partial).
const char *kKernel = R"(
extern "C" __global__ void __launch_bounds__(256) fga_user_xstep(
    int mode, int nf, int ebase, const int *__restrict__ var, const unsigned *__restrict__ dst,
    const fga_real *__restrict__ zc, const fga_real *__restrict__ xin, fga_real *__restrict__ xout,
    fga_real *__restrict__ u, fga_real *__restrict__ mout, fga_real *__restrict__ pvm,
    const fga_real *__restrict__ rho_e, fga_real rho_u, const fga_real *__restrict__ alpha_e, fga_real alpha_u,
    const fga_real *__restrict__ prm, double *__restrict__ res_pri, const int *done)
{
    if (*(volatile const int *)done) return;
    __shared__ double red[32];
    double pri = 0.0;
    const int stride = gridDim.x * blockDim.x;
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += stride) {
        fga_real n[FGA_ARITY], r[FGA_ARITY], x[FGA_ARITY], uu[FGA_ARITY];
        for (int k = 0; k < FGA_ARITY; ++k) {
            const int l = f * FGA_ARITY + k, e = ebase + l;
            const fga_real z = zc[var[l]];
            fga_real v = u[e];
            if (mode != 0) {
                const fga_real xo = xin[e];
                if (mode >= 2) {
                    const double dd = (double)xo - (double)z;
                    pri += dd * dd;
                }
                const fga_real al = alpha_e ? alpha_e[e] : alpha_u;
                const fga_real d = xo - z;
                v = v + al * d;
                u[e] = v;
            }
            uu[k] = v;
            n[k] = z - v;
            r[k] = rho_e ? rho_e[e] : rho_u;
            x[k] = n[k];
        }
        if (mode == 2) continue;
        FGA_USER_FN<fga_real>(FGA_ARITY, n, r, prm + (long long)f * FGA_NPARAM, x);
        for (int k = 0; k < FGA_ARITY; ++k) {
            const int l = f * FGA_ARITY + k, e = ebase + l;
            xout[e] = x[k];
            const fga_real m = x[k] + uu[k];
            if (mout) mout[e] = m;
            pvm[dst[l]] = r[k] * m;
        }
    }
    if (mode >= 2) {
        // this CTA's primal-residual partial by a fixed tree, added to the
        // built-in types' partial of the same CTA (written before, in stream
        // order)
        for (int o = 16; o > 0; o >>= 1) pri += __shfl_down_sync(0xffffffffu, pri, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = pri;
        __syncthreads();
        if (threadIdx.x < 32) {
            double s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            if (threadIdx.x == 0) res_pri[blockIdx.x] += s;
        }
    }
}
)";

bool valid_identifier(const std::string &s) {
    if (s.empty() || s.size() > 128 || std::isdigit((unsigned char)s[0])) return false;
    for (char c : s)
        if (!(std::isalnum((unsigned char)c) || c == '_')) return false;
    return true;
}

}  // namespace

bool user_compile(const std::string &source, const std::string &fn, int arity, int np, bool f64, UserProg &out,
                  std::string &log) {
    const Nvrtc &N = nvrtc();
    if (!N.ok) {
        log = N.why;
        return false;
    }
    if (!valid_identifier(fn)) {
        log = "function name must be a C identifier";
        return false;
    }
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) {
        log = "no CUDA device";
        return false;
    }
    std::string text = "#define FGA_ARITY " + std::to_string(arity) + "\n#define FGA_NPARAM " +
                       std::to_string(np > 0 ? np : 0) + "\n#define FGA_USER_FN " + fn + "\ntypedef " +
                       (f64 ? "double" : "float") + " fga_real;\n#line 1 \"user_prox.cu\"\n" + source + "\n" +
                       "#line 1 \"fga_user_xstep.cu\"\n" + kKernel;
    nvrtcProgram prog = nullptr;
    if (N.create(&prog, text.c_str(), "user_prox.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) {
        log = "nvrtcCreateProgram failed";
        return false;
    }
    const std::string arch = "--gpu-architecture=sm_" + std::to_string(major) + std::to_string(minor);
    // FP64: no contraction into fused multiply-adds, IEEE division and
    // square root, as the library's own FP64 sweep is built, so that an
    // operator written the same way as a host implementation gives the same
    // bits.  FP32: contraction allowed, as in the FP32 sweep.
    std::vector<const char *> opts = {arch.c_str(), "-std=c++17", "-default-device", "--prec-div=true",
                                      "--prec-sqrt=true", "--ftz=false", f64 ? "--fmad=false" : "--fmad=true"};
    const nvrtcResult cr = N.compile(prog, (int)opts.size(), opts.data());
    size_t ls = 0;
    N.log_size(prog, &ls);
    std::string clog(ls, '\0');
    if (ls) N.log(prog, &clog[0]);
    if (cr != NVRTC_SUCCESS) {
        log = std::string(N.error_string(cr)) + ": " + clog;
        N.destroy(&prog);
        return false;
    }
    size_t cs = 0;
    N.cubin_size(prog, &cs);
    std::vector<char> cubin(cs);
    if (!cs || N.cubin(prog, cubin.data()) != NVRTC_SUCCESS) {
        N.destroy(&prog);
        log = "NVRTC produced no device code";
        return false;
    }
    N.destroy(&prog);
    cudaLibrary_t lib = nullptr;
    cudaError_t e = cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e != cudaSuccess) {
        log = std::string("cudaLibraryLoadData: ") + cudaGetErrorString(e);
        return false;
    }
    cudaKernel_t k = nullptr;
    e = cudaLibraryGetKernel(&k, lib, "fga_user_xstep");
    if (e != cudaSuccess) {
        cudaLibraryUnload(lib);
        log = std::string("cudaLibraryGetKernel: ") + cudaGetErrorString(e);
        return false;
    }
    out.name = fn;
    out.arity = arity;
    out.np = np;
    out.lib = lib;
    out.kern = k;
    return true;
}

cudaError_t user_launch(const UserProg &p, bool f64, const UserLaunch &a, int grid, int block, cudaStream_t s) {
    int mode = a.mode, nf = a.nf, ebase = a.ebase;
    const void *var = a.var, *dst = a.dst, *zc = a.zc, *xin = a.xin, *rho_e = a.rho_e, *alpha_e = a.alpha_e,
               *prm = a.prm, *done = a.done;
    void *xout = a.xout, *u = a.u, *mout = a.mout, *pvm = a.pvm, *res = a.res_pri;
    double rd = a.rho_u, ad = a.alpha_u;
    float rf = (float)a.rho_u, af = (float)a.alpha_u;
    void *args[] = {&mode, &nf,   &ebase, &var,   &dst,
                    &zc,   &xin,  &xout,  &u,     &mout,
                    &pvm,  &rho_e, f64 ? (void *)&rd : (void *)&rf,
                    &alpha_e, f64 ? (void *)&ad : (void *)&af,
                    &prm,  &res,  &done};
    return cudaLaunchKernel((const void *)p.kern, dim3(grid), dim3(block), args, 0, s);
}

void user_release(UserProg &p) {
    if (p.lib) cudaLibraryUnload(p.lib);
    p.lib = nullptr;
    p.kern = nullptr;
}

}  // namespace fga
