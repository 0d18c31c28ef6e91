// fga_hinge.cpp -- host planner of the hinge-bank sweep (see
// hinge_internal.h): the hinge factors cut into contiguous slices, one per
// CTA, and the data rows padded to 64 values with their per-factor
// constants (label, weight, |x|^2 + 1).
#include <algorithm>
#include <cstring>

#include "hinge_internal.h"

namespace fga {

int hinge_plan(const HingeInput &in, HingePlan &P, std::string &why) {
    const int64_t N = in.N;
    if (N <= 0) {
        why = "no hinge factors";
        return 1;
    }
    if (in.D < 1 || in.D > kHingeD) {
        why = "dim(w) above 64";
        return 1;
    }
    if ((int)in.lam.size() > kHingeMaxL2) {
        why = "more than 4 L2 factors";
        return 1;
    }
    if (in.sms <= 0) {
        why = "no launch shape";
        return 1;
    }
    const int64_t G0 = std::min<int64_t>(in.sms, N);
    const int64_t rows = (N + G0 - 1) / G0;
    if (rows > (int64_t)kHingeGroups * kHingeK) {
        why = "more hinge factors per CTA than its groups hold";
        return 1;
    }
    if (hinge_smem_bytes((int)rows) > in.smem_optin) {
        why = "a CTA's data rows do not fit in shared memory";
        return 1;
    }
    if (N * (int64_t)kHingeD > (int64_t)INT32_MAX) {
        why = "too many data values";
        return 1;
    }
    const int G = (int)((N + rows - 1) / rows);
    if (G > kTileMaxHolders) {   // every CTA adds to every variable: the word counts at most 255
        why = "more CTAs than a count-and-sum word counts";
        return 1;
    }
    P.G = G;
    P.rows_max = (int)rows;
    P.cta.resize((size_t)G);
    for (int g = 0; g < G; ++g) {
        P.cta[g].f0 = (int)(g * rows);
        P.cta[g].nf = (int)std::min<int64_t>(rows, N - g * rows);
    }
    P.X.assign((size_t)N * kHingeD, 0.f);
    P.meta.resize((size_t)N);
    for (int64_t f = 0; f < N; ++f) {
        double s2 = 0.0;
        for (int j = 0; j < in.D; ++j) {
            const float v = in.X[(size_t)f * in.D + j];
            P.X[(size_t)f * kHingeD + j] = v;
            s2 += (double)v * (double)v;
        }
        P.meta[f] = make_float4(in.yl[f], in.cl[f], (float)(s2 + 1.0), (float)(in.rho / (s2 + 1.0)));
    }
    return 0;
}

}  // namespace fga
