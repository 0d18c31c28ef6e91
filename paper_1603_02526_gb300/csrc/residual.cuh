// residual.cuh -- the RMS residual test of the stopping rule without the
// FP64 pipe on the hot side: sums carried as unevaluated float pairs, the
// comparison against squared thresholds, the FP64 square root only near the
// threshold and for the reported values.  (A dependent FP64 addition costs
// about 64 cycles on this part; FP64 trees and square roots made a residual
// check several microseconds long.)
#pragma once

#include <cuda_runtime.h>

namespace fga {

// (h, l) += (h2, l2) for unevaluated float pairs h + l (TwoSum, then a fast
// renormalisation): the pair keeps about 44 significant bits, and the sum
// is commutative, so a butterfly leaves the same value in every lane.
__device__ __forceinline__ void ff_add(float &h, float &l, float h2, float l2) {
    const float s = h + h2;
    const float bb = s - h;
    float e = (h - (s - bb)) + (h2 - bb);
    e += l + l2;
    h = s + e;
    l = e - (h - s);
}

// A double as an unevaluated float pair (the double rounded to float, and
// the remainder rounded to float).
__device__ __forceinline__ void ff_from_double(double v, float &h, float &l) {
    h = __double2float_rn(v);
    l = __double2float_rn(v - (double)h);
}

// sqrt(t / E) <= tol (the RMS residual test), decided without the FP64
// divide and square root unless t lies close to tol^2 E, where the exact
// form decides: within a relative 2^-40 for an FP64 t, within 2^-20 for a
// float pair h + l (carried to about 2^-44), whose fast test compares h.
struct ResidualTest {
    double E, tol, lo, hi;
    float lo32, hi32;
    __device__ void init(double E_, double tol_) {
        E = E_;
        tol = tol_;
        if (!(tol_ > 0.0)) {
            lo = hi = 0.0;   // only t = 0 can pass
            lo32 = hi32 = 0.f;
        } else {
            const double t2 = tol_ * tol_ * E_;
            const bool normal = t2 > 1e-30 && t2 < 1e30;
            lo = normal ? t2 * (1.0 - 0x1p-40) : -INFINITY;   // else always the exact form
            hi = normal ? t2 * (1.0 + 0x1p-40) : INFINITY;
            lo32 = normal ? (float)(t2 * (1.0 - 0x1p-20)) : -INFINITY;
            hi32 = normal ? (float)(t2 * (1.0 + 0x1p-20)) : INFINITY;
        }
    }
    __device__ bool pass(double t) const {
        if (t < lo) return true;
        if (t > hi) return false;
        return sqrt(t / E) <= tol;
    }
    __device__ bool pass(float h, float l) const {
        if (h < lo32) return true;
        if (h > hi32) return false;
        return sqrt(((double)h + (double)l) / E) <= tol;
    }
};

// Warp sums of two float pairs by a fixed butterfly (every lane ends with
// the same bits).
__device__ __forceinline__ void warp_sum2_ff(float &ah, float &al, float &bh, float &bl) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float xh = __shfl_xor_sync(0xffffffffu, ah, o), xl = __shfl_xor_sync(0xffffffffu, al, o);
        const float yh = __shfl_xor_sync(0xffffffffu, bh, o), yl = __shfl_xor_sync(0xffffffffu, bl, o);
        ff_add(ah, al, xh, xl);
        ff_add(bh, bl, yh, yl);
    }
}

// The CTA's sums of two per-thread FP64 partials, as float pairs, in thread
// 0: each partial split into a pair, warps by warp_sum2_ff, the warps in
// order.  Deterministic.  Every thread of the CTA calls it.
__device__ __forceinline__ float4 block_sum2_ff(double a, double b) {
    __shared__ float4 s_w[32];
    float ah, al, bh, bl;
    ff_from_double(a, ah, al);
    ff_from_double(b, bh, bl);
    warp_sum2_ff(ah, al, bh, bl);
    const int w = threadIdx.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s_w[w] = make_float4(ah, al, bh, bl);
    __syncthreads();
    float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
    if (threadIdx.x == 0) {
        r = s_w[0];
        const int nw = (blockDim.x + 31) >> 5;
        for (int i = 1; i < nw; ++i) {
            const float4 v = s_w[i];
            ff_add(r.x, r.y, v.x, v.y);
            ff_add(r.z, r.w, v.z, v.w);
        }
    }
    return r;
}

// The sum of the n CTAs' pairs p[0..n) (x, y: first value; z, w: second),
// by one full warp in a fixed order; every lane obtains the same bits.  The
// two values are summed one after the other (fewer live registers).
__device__ __forceinline__ float2 warp_sum_partial_ff(const float4 *p, int n, int which) {
    const int l = threadIdx.x & 31;
    const float2 *q = reinterpret_cast<const float2 *>(p) + which;
    float h = 0.f, lo = 0.f;
    for (int i = l; i < n; i += 32) {
        const float2 v = __ldcg(q + 2 * i);
        ff_add(h, lo, v.x, v.y);
    }
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float xh = __shfl_xor_sync(0xffffffffu, h, o), xl = __shfl_xor_sync(0xffffffffu, lo, o);
        ff_add(h, lo, xh, xl);
    }
    return make_float2(h, lo);
}

}  // namespace fga
