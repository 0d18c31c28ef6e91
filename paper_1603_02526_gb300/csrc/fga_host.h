// fga_host.h -- host-side helpers shared by the graph and batch layers of
// libfgadmm (not part of the public C-ABI).
#pragma once

#include <cmath>
#include <vector>

namespace fga {

// Projector onto {v : M v = 0}, M = [A B -I], in the metric diag(rho):
// P = I - W M^T (M W M^T)^{-1} M with W = diag(1/rho).  Gauss-Jordan with
// partial pivoting on the nx x nx matrix M W M^T.
inline bool dyn_projector(int nx, int nu, const double *A, const double *B, const double *rho, std::vector<double> &P) {
    const int n = 2 * nx + nu;
    std::vector<double> M((size_t)nx * n, 0.0);
    for (int i = 0; i < nx; ++i) {
        for (int j = 0; j < nx; ++j) M[(size_t)i * n + j] = A[i * nx + j];
        for (int j = 0; j < nu; ++j) M[(size_t)i * n + nx + j] = B[i * nu + j];
        M[(size_t)i * n + nx + nu + i] = -1.0;
    }
    std::vector<double> K((size_t)nx * 2 * nx, 0.0);   // [K | I]
    for (int i = 0; i < nx; ++i) {
        for (int k = 0; k < nx; ++k) {
            double t = 0.0;
            for (int j = 0; j < n; ++j) t += M[(size_t)i * n + j] * M[(size_t)k * n + j] / rho[j];
            K[(size_t)i * 2 * nx + k] = t;
        }
        K[(size_t)i * 2 * nx + nx + i] = 1.0;
    }
    for (int c = 0; c < nx; ++c) {
        int piv = c;
        for (int r = c + 1; r < nx; ++r)
            if (std::fabs(K[(size_t)r * 2 * nx + c]) > std::fabs(K[(size_t)piv * 2 * nx + c])) piv = r;
        if (!(std::fabs(K[(size_t)piv * 2 * nx + c]) > 0.0)) return false;
        if (piv != c)
            for (int j = 0; j < 2 * nx; ++j) std::swap(K[(size_t)c * 2 * nx + j], K[(size_t)piv * 2 * nx + j]);
        const double d = K[(size_t)c * 2 * nx + c];
        for (int j = 0; j < 2 * nx; ++j) K[(size_t)c * 2 * nx + j] /= d;
        for (int r = 0; r < nx; ++r) {
            if (r == c) continue;
            const double f = K[(size_t)r * 2 * nx + c];
            if (f == 0.0) continue;
            for (int j = 0; j < 2 * nx; ++j) K[(size_t)r * 2 * nx + j] -= f * K[(size_t)c * 2 * nx + j];
        }
    }
    // T = K^{-1} M  (nx x n)
    std::vector<double> T((size_t)nx * n, 0.0);
    for (int i = 0; i < nx; ++i)
        for (int j = 0; j < n; ++j) {
            double t = 0.0;
            for (int k = 0; k < nx; ++k) t += K[(size_t)i * 2 * nx + nx + k] * M[(size_t)k * n + j];
            T[(size_t)i * n + j] = t;
        }
    P.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double t = 0.0;
            for (int k = 0; k < nx; ++k) t += M[(size_t)k * n + i] * T[(size_t)k * n + j];
            P[(size_t)i * n + j] = (i == j ? 1.0 : 0.0) - t / rho[i];
        }
    return true;
}

}  // namespace fga
