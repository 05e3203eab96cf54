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

// dtw_bound for a pair whose largest |d - 1/2| (dev) is known before the
// pass: tau from the frame-distance error at the pair's own largest |cos|
// (plus the cosine error, as in dtw_interval) instead of at kCosMax.
__device__ __forceinline__ DtwBound dtw_bound_dev(int Tx, int Ty, float theta_x, float theta_y,
                                                  float ec, float dev) {
    DtwBound b = dtw_bound(Tx, Ty, theta_x, theta_y, ec);
    const float cmax = sinf(3.14159265f * fminf(dev, 0.5f)) * 1.000001f + 1e-7f;
    if (cmax <= kCosMax) {
        const float delta0 = b.th + dtw_dist_err(ec, cmax + ec);
        b.tau = 2.5f * (b.lam * delta0 * (1.0f + b.gam) + 2.0f * b.gam * b.lam) +
                8.0f * b.gam * b.lam;
    }
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

namespace abx {

// DTW of one pair by one thread, in place on the pair's block of a row-major
// distance table (d(i, j) at db[i * ld + j], 0 <= i < R, 0 <= j < C), for the
// fused tile kernel, whose shared-memory d tile leaves no room for row
// buffers of its own.  The cost of cell (i, j) overwrites d(i, j) once read;
// the packed lengths of row i go to the slots of row i - 1, whose costs no
// later cell reads (cell (i, j + 1) takes c(i - 1, j) from a register), and
// row 0's lengths are j + 1 (its only path), so they are not stored.  The
// same cell update on the same sums as the row-buffer walk, hence the same
// cost, lengths and largest |d - 1/2|.  The block is overwritten.
__device__ __forceinline__ void dtw_inplace(float *db, int ld, int R, int C, float tau,
                                            float &cost, uint32_t &info, float &dev) {
    float dv = 0.0f;
    float lc = 0.0f;
    for (int j = 0; j < C; ++j) {  // row 0: the left predecessor only
        const float d = db[j];
        dv = fmaxf(dv, fabsf(d - 0.5f));
        lc = j == 0 ? d : d + lc;
        db[j] = lc;
    }
    uint32_t ll = dtw_pack3((uint32_t)C, (uint32_t)C, (uint32_t)C);
    for (int i = 1; i < R; ++i) {
        float *up = db + (i - 1) * ld;                  // costs of row i - 1
        float *row = up + ld;                           // distances of row i
        const float *upl = db + (i >= 2 ? (i - 2) * ld : 0);  // lengths of row i - 1
        float lcst = ABX_INF, dcst = ABX_INF;
        uint32_t llen = 0, dlen = 0;
        int j = 0;
        for (; j + 4 <= C; j += 4) {
            float dq[4], uq[4];
            uint32_t lq[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                dq[q] = row[j + q];
                uq[q] = up[j + q];
                const uint32_t l1 = (uint32_t)(j + q + 1);
                lq[q] = i >= 2 ? __float_as_uint(upl[j + q]) : dtw_pack3(l1, l1, l1);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                dv = fmaxf(dv, fabsf(dq[q] - 0.5f));
                float nc;
                uint32_t ni;
                dtw_cell(dq[q], uq[q], lq[q], lcst, llen, dcst, dlen, tau, nc, ni);
                row[j + q] = nc;
                up[j + q] = __uint_as_float(ni);
                dcst = uq[q];
                dlen = lq[q];
                lcst = nc;
                llen = ni;
            }
        }
        for (; j < C; ++j) {
            const float d = row[j];
            const float uc = up[j];
            const uint32_t l1 = (uint32_t)(j + 1);
            const uint32_t ul = i >= 2 ? __float_as_uint(upl[j]) : dtw_pack3(l1, l1, l1);
            dv = fmaxf(dv, fabsf(d - 0.5f));
            float nc;
            uint32_t ni;
            dtw_cell(d, uc, ul, lcst, llen, dcst, dlen, tau, nc, ni);
            row[j] = nc;
            up[j] = __uint_as_float(ni);
            dcst = uc;
            dlen = ul;
            lcst = nc;
            llen = ni;
        }
        lc = lcst;
        ll = llen;
    }
    cost = lc;
    info = ll;
    dev = dv;
}

// Anti-diagonal wavefront DTW of one pair by a group of 8 consecutive lanes
// (the Sec. 3.2 recurrence, evaluated in the order of the paper's wavefront
// figure).  Lane g of the group owns row 8s + g of strip s; at step k it
// computes cell (8s + g, k - g).  The cell above is lane g - 1's result of
// the previous step (a shuffle), the diagonal one is what the lane received
// one step earlier, the left one its own previous result; cells of one
// anti-diagonal are computed in the same step.  Rows come in strips of 8;
// lane 7 keeps the strip's last row in rbc / rbl (C entries, the group's
// own) for lane 0 of the next strip.  dat(i, j) returns d(i, j) for
// 0 <= i < R, 0 <= j < C.  Every lane of the group receives the final cost,
// its packed lengths (dtw_pack3) and the largest |d - 1/2| of the pair.
// A group takes R / 8 rounded up strips of R_strip + C - 1 steps each, so a
// 25 x 25 pair needs 4 x 32 steps of a few dozen instructions instead of the
// 625 dependent cell updates of one thread.
template <class DAt>
__device__ __forceinline__ void dtw_wave8(const DAt dat, int R, int C, float tau, float *rbc,
                                          uint32_t *rbl, float &cost, uint32_t &info,
                                          float &dev) {
    const int lane = threadIdx.x & 31;
    const int g = lane & 7;
    const unsigned gmask = 0xffu << (lane & 24);
    float dv = 0.0f;
    float pc = ABX_INF;
    uint32_t pl = 0;
    const int strips = (R + 7) >> 3;
    for (int s = 0; s < strips; ++s) {
        const int i = 8 * s + g;
        const int rows = min(8, R - 8 * s);
        // own previous cell (left), received cell (becomes the diagonal), and
        // for lane 0 the previous strip's cell above-left
        pc = ABX_INF;
        pl = 0;
        float rc = ABX_INF, lastc = ABX_INF;
        uint32_t rl = 0, lastl = 0;
        const int steps = rows + C - 1;
        for (int k = 0; k < steps; ++k) {
            const int j = k - g;
            const float tc = __shfl_up_sync(gmask, pc, 1, 8);
            const uint32_t tl = __shfl_up_sync(gmask, pl, 1, 8);
            float uc, dc;
            uint32_t ul, dl;
            if (g == 0) {
                if (s > 0 && j < C) {
                    uc = rbc[j];
                    ul = rbl[j];
                } else {
                    uc = ABX_INF;
                    ul = 0;
                }
                dc = lastc;
                dl = lastl;
                lastc = uc;
                lastl = ul;
            } else {
                uc = tc;
                ul = tl;
                dc = rc;
                dl = rl;
                rc = tc;
                rl = tl;
            }
            if (j >= 0 && j < C && i < R) {
                const float d = dat(i, j);
                dv = fmaxf(dv, fabsf(d - 0.5f));
                float nc;
                uint32_t ni;
                if (i == 0 && j == 0) {
                    nc = d;
                    ni = dtw_pack3(1, 1, 1);
                } else {
                    dtw_cell(d, uc, ul, pc, pl, dc, dl, tau, nc, ni);
                }
                pc = nc;
                pl = ni;
                if (g == 7) {
                    rbc[j] = nc;
                    rbl[j] = ni;
                }
            }
        }
        __syncwarp(gmask);  // the strip's last row is visible to the next strip
    }
    const int src = (lane & 24) + ((R - 1) & 7);  // lane of row R - 1
    cost = __shfl_sync(gmask, pc, src);
    info = __shfl_sync(gmask, pl, src);
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) dv = fmaxf(dv, __shfl_xor_sync(gmask, dv, o));
    dev = dv;
}

}  // namespace abx
