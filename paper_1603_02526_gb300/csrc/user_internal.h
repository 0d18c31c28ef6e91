// user_internal.h -- user-supplied proximal operators: CUDA source compiled
// at run time (NVRTC) into one x-update kernel per type (not part of the
// public C-ABI).
#pragma once

#include <string>

#include <cuda_runtime.h>

#include "fga_internal.h"

namespace fga {

constexpr int kMaxUserTypes = 16;   // user operators per graph
constexpr int kUserMaxArity = 64;   // scalar edges of one user factor
constexpr int kUserMaxParams = 4096;

// One compiled user operator: the module and its x-update kernel.
struct UserProg {
    std::string name;
    int arity = 0, np = 0;
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kern = nullptr;
};

// Pointers and sizes of one launch over one bucket of a user type (plain
// values: the kernel takes them as separate arguments).
struct UserLaunch {
    int mode, nf, ebase;
    const int *var;         // [nf * arity] scalar variable of each edge
    const unsigned *dst;    // [nf * arity] slot of its rho * m in the z-reduction input
    const void *zc, *xin;
    void *xout, *u, *mout, *pvm;
    const void *rho_e;
    double rho_u;
    const void *alpha_e;
    double alpha_u;
    const void *prm;        // [nf * np] factor-major
    double *res_pri;
    const int *done;
};

// Compiles `source` with the generated x-update kernel around the user's
// function `fn` for the current device, FP64 (`f64`) or FP32; on failure
// returns false and `log` holds the compiler's or loader's message.
bool user_compile(const std::string &source, const std::string &fn, int arity, int np, bool f64, UserProg &out,
                  std::string &log);

// Launches the x-update kernel of `p` (grid x block threads) on stream s.
cudaError_t user_launch(const UserProg &p, bool f64, const UserLaunch &a, int grid, int block, cudaStream_t s);

void user_release(UserProg &p);

}  // namespace fga
