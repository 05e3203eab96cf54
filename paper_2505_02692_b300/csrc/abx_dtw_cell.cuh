// DTW cell update and interval bound shared by the stand-alone DTW kernel and
// the fused tile kernel (fastabx Sec. 3.2 recurrence, shorter path on equal
// cost, near-optimal path-length range for the exact-value interval).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace abx {

#define ABX_INF __int_as_float(0x7f800000)

// |cos| above which a pair's interval is not derived (it gets [0, 1]).
constexpr float kCosMax = 0.999f;

__device__ __forceinline__ uint32_t dtw_pack3(uint32_t l, uint32_t lmin, uint32_t lmax) {
    return l | (lmin << 8) | (lmax << 16);
}

// Frame-distance error bound from a cosine error ec at |cos| <= m: either
// the slope of arccos or arccos(1 - w) <= 1.02 sqrt(2 w); divided by pi.
__device__ __forceinline__ float dtw_dist_err(float ec, float m) {
    const float e_sqrt = 1.02f * sqrtf(2.0f * ec);
    const float e_lin = m < 1.0f ? ec / sqrtf((1.0f - m) * (1.0f + m)) : ABX_INF;
    return fminf(e_sqrt, e_lin) * 0.318309886f;
}

// One cell from its three predecessors: cost = d + min, length of the
// lexicographic (cost, length) minimum, and the range of lengths over the
// predecessors within tau of the minimum (packed as len | lmin<<8 | lmax<<16).
__device__ __forceinline__ void dtw_cell(float dij, float uc, uint32_t ul, float lc, uint32_t ll,
                                         float dc, uint32_t dl, float tau, float &nc,
                                         uint32_t &info) {
    const float mc = fminf(uc, fminf(lc, dc));
    uint32_t len = 255, lmin = 255, lmax = 0;
    const float lim = mc + tau;
    if (uc == mc) len = min(len, ul & 0xffu);
    if (lc == mc) len = min(len, ll & 0xffu);
    if (dc == mc) len = min(len, dl & 0xffu);
    if (uc <= lim) { lmin = min(lmin, (ul >> 8) & 0xffu); lmax = max(lmax, ul >> 16); }
    if (lc <= lim) { lmin = min(lmin, (ll >> 8) & 0xffu); lmax = max(lmax, ll >> 16); }
    if (dc <= lim) { lmin = min(lmin, (dl >> 8) & 0xffu); lmax = max(lmax, dl >> 16); }
    info = dtw_pack3(len + 1, lmin + 1, lmax + 1);
    nc = dij + mc;
}

// Per-pair constants: tau for the near-optimal length range and the
// quantisation part of the frame-distance error.
struct DtwBound {
    float th, lam, gam, tau;
};

__device__ __forceinline__ DtwBound dtw_bound(int Tx, int Ty, float theta_x, float theta_y,
                                              float ec) {
    DtwBound b;
    const float u = 5.9604645e-8f;  // 2^-24
    b.th = (theta_x + theta_y) * 0.31830989f + 4e-7f;
    b.lam = (float)(Tx + Ty - 1);
    b.gam = b.lam * u / (1.0f - b.lam * u);
    const float delta0 = b.th + dtw_dist_err(ec, kCosMax + ec);
    b.tau = 2.5f * (b.lam * delta0 * (1.0f + b.gam) + 2.0f * b.gam * b.lam) + 8.0f * b.gam * b.lam;
    return b;
}

// Interval [lo, hi] holding the exact normalised distance, from the final
// cost, packed lengths and the largest |d - 1/2| met.
__device__ __forceinline__ void dtw_interval(const DtwBound &b, float cost, uint32_t info,
                                             float dev, float ec, int intervals, float D,
                                             float &lo, float &hi) {
    const uint32_t Lmin = (info >> 8) & 0xffu, Lmax = info >> 16;
    const float cmax = sinf(3.14159265f * fminf(dev, 0.5f)) * 1.000001f + 1e-7f;
    lo = 0.0f;
    hi = 1.0f;
    if (!intervals) {
        lo = hi = D;  // other distances: no error model, no recheck
    } else if (cmax <= kCosMax) {
        const float delta = b.th + dtw_dist_err(ec, cmax + ec);
        const float E = __fadd_ru(b.lam * delta * 1.0001f,
                                  2.0f * b.gam * (cost + b.lam * delta) + 1e-7f);
        lo = fmaxf(0.0f, __fdiv_rd(__fsub_rd(cost, E), (float)Lmax));
        hi = fminf(1.0f, __fdiv_ru(__fadd_ru(cost, E), (float)Lmin));
    }
}

}  // namespace abx
