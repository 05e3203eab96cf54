// DTW kernel (fastabx Sec. 3.2): for every needed item pair, the dynamic
// programme c(i,j) = d(i,j) + min(c(i-1,j), c(i,j-1), c(i-1,j-1)) over the
// pair's block of the frame-distance tile, normalised by the number of cells
// on the optimal path (shorter path on equal cost).
//
// One thread per pair.  The pairs are short (3..40 frames here) and number in
// the millions, so a whole-warp wavefront per pair would leave most lanes
// idle; instead each thread walks its pair row by row with the previous row
// in shared memory, laid out [column][thread] so that a warp's accesses fall
// on 32 distinct banks.  Pairs stay in tile order: the threads of a warp
// mostly share the x item of one tile, so their loads fall in the same tile
// rows (sorting by shape to remove divergence measured slower: it scatters
// those loads).
//
// Besides the distance the kernel emits an interval [lo, hi] that holds the
// exact distance.  With delta bounding every frame-distance error of the pair
// and Lambda = Tx + Ty - 1 the longest path, any path sum moves by at most
// Lambda * delta, plus FP32 rounding of the running sums (gamma_Lambda
// relative).  Because the result is divided by the optimal path's length,
// the kernel also tracks, per cell, the range [Lmin, Lmax] of lengths of
// paths whose cost is within tau of the optimum (tau = twice the cost error
// bound, with slack for rounding): every prefix of a near-optimal path is
// near-optimal at its own end cell, so the range propagates through the
// predecessors whose cost lies within tau of the minimum.  Then
//   exact distance in [(c - E) / Lmax, (c + E) / Lmin].
// tau is fixed before the pass from the bound the cosine error has while
// |cos| <= kCosMax; the pass records the largest |cos| it meets, the final
// E uses it, and a pair that exceeds kCosMax gets the interval [0, 1] (it is
// then always re-decided in FP64).
#include <cuda_runtime.h>

#include <algorithm>

#include "abx_dtw_cell.cuh"
#include "abx_internal.h"

namespace abx {
namespace {

#define kInf ABX_INF

__global__ void __launch_bounds__(128) dtw_kernel(DtwArgs a) {
    extern __shared__ float smem[];
    const int tid = threadIdx.x, nt = blockDim.x;
    float *rbc = smem;                                              // [max_len][nt]
    uint32_t *rbl = reinterpret_cast<uint32_t *>(smem + a.max_len * nt);
    const int64_t n_pairs = *a.n_pairs;
    const float ec = a.eps_c;
    for (int64_t p = (int64_t)blockIdx.x * nt + tid; p < n_pairs; p += (int64_t)gridDim.x * nt) {
        const int4 pr = a.pairs[p];
        const int x = pr.x, y = pr.y;
        const int rx = pr.w & 0xffff, cy = pr.w >> 16;
        const int Tx = a.len[x], Ty = a.len[y];
        const float *tb = a.tilebuf + (int64_t)pr.z * (kPanel * kPanel) + rx * kPanel + cy;
        const DtwBound bd = dtw_bound(Tx, Ty, a.theta_item[x], a.theta_item[y], ec);
        const float tau = bd.tau;

        float dev = 0.0f;  // largest |d - 1/2|, i.e. largest |cos|
        float lc = 0.0f;
        uint32_t ll = 0;
        for (int i = 0; i < Tx; ++i) {
            const float *drow = tb + i * kPanel;
            float dc, uc;
            uint32_t dl, ul;
            lc = kInf;
            ll = 0;
            dc = kInf;
            dl = 0;
            int j = 0;
            for (; j + 4 <= Ty; j += 4) {
                float dv[4], uv[4];
                uint32_t uw[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    dv[q] = drow[j + q];
                    uv[q] = i > 0 ? rbc[(j + q) * nt + tid] : kInf;
                    uw[q] = i > 0 ? rbl[(j + q) * nt + tid] : 0u;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    dev = fmaxf(dev, fabsf(dv[q] - 0.5f));
                    float nc;
                    uint32_t info;
                    if (i == 0 && j + q == 0) {
                        nc = dv[q];
                        info = dtw_pack3(1, 1, 1);
                    } else {
                        dtw_cell(dv[q], uv[q], uw[q], lc, ll, dc, dl, tau, nc, info);
                    }
                    dc = uv[q];
                    dl = uw[q];
                    lc = nc;
                    ll = info;
                    rbc[(j + q) * nt + tid] = nc;
                    rbl[(j + q) * nt + tid] = info;
                }
            }
            for (; j < Ty; ++j) {
                const float dij = drow[j];
                uc = i > 0 ? rbc[j * nt + tid] : kInf;
                ul = i > 0 ? rbl[j * nt + tid] : 0u;
                dev = fmaxf(dev, fabsf(dij - 0.5f));
                float nc;
                uint32_t info;
                if (i == 0 && j == 0) {
                    nc = dij;
                    info = dtw_pack3(1, 1, 1);
                } else {
                    dtw_cell(dij, uc, ul, lc, ll, dc, dl, tau, nc, info);
                }
                dc = uc;
                dl = ul;
                lc = nc;
                ll = info;
                rbc[j * nt + tid] = nc;
                rbl[j * nt + tid] = info;
            }
        }
        const float cost = lc;
        const uint32_t L = ll & 0xffu;
        const float D = __fdiv_rn(cost, (float)L);
        float lo, hi;
        dtw_interval(bd, cost, ll, dev, ec, a.intervals, D, lo, hi);

        const int4 gm = a.t.gmeta[a.t.item_g[x]];
        const int gb = gm.x;
        const int64_t ng = gm.y;
        const int64_t base = ((int64_t)(uint32_t)gm.w << 32) | (uint32_t)gm.z;
        const int64_t e1 = base + (int64_t)(x - gb) * ng + (y - gb);
        const int64_t e2 = base + (int64_t)(y - gb) * ng + (x - gb);
        const PairVal v{D, lo, hi, L};
        a.pv[e1] = v;
        a.pv[e2] = v;
    }
}

}  // namespace

cudaError_t launch_dtw(const DtwArgs &a, cudaStream_t s) {
    if (a.pair_cap == 0) return cudaSuccess;
    const int nt = 128;
    const size_t smem = (size_t)a.max_len * nt * 8;
    cudaError_t e = cudaFuncSetAttribute(dtw_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = (a.pair_cap + nt - 1) / nt;
    const int64_t cap = (int64_t)nsm * 16;
    if (blocks > cap) blocks = cap;
    {
        ProfScope ps_("dtw", s);
        dtw_kernel<<<(unsigned)blocks, nt, smem, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace abx
