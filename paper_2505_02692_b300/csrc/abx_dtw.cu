// DTW kernel (fastabx Sec. 3.2): for every needed item pair, the dynamic
// programme c(i,j) = d(i,j) + min(c(i-1,j), c(i,j-1), c(i-1,j-1)) over the
// pair's block of the frame-distance tile, normalised by the number of cells
// on the optimal path (shorter path on equal cost).
//
// One thread per pair.  The pairs are short (3..40 frames here) and number in
// the millions, so a whole-warp wavefront per pair would leave most lanes
// idle; instead each thread walks its pair row by row with the previous row
// in shared memory, laid out [column][thread] so that a warp's accesses fall
// on 32 distinct banks.
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
#include <cuda_runtime.h>

#include "abx_internal.h"

namespace abx {
namespace {

#define kInf __int_as_float(0x7f800000)

__device__ __forceinline__ uint32_t pack3(uint32_t l, uint32_t lmin, uint32_t lmax) {
    return l | (lmin << 8) | (lmax << 16);
}

__global__ void __launch_bounds__(128) dtw_kernel(DtwArgs a) {
    extern __shared__ float smem[];
    const int tid = threadIdx.x, nt = blockDim.x;
    float *rbc = smem;                                              // [max_len][nt]
    uint32_t *rbl = reinterpret_cast<uint32_t *>(smem + a.max_len * nt);
    const float u = 5.9604645e-8f;  // 2^-24
    const int64_t n_pairs = *a.n_pairs;
    for (int64_t p = (int64_t)blockIdx.x * nt + tid; p < n_pairs; p += (int64_t)gridDim.x * nt) {
        const int4 pr = a.pairs[p];
        const int x = pr.x, y = pr.y;
        const int rx = pr.w & 0xffff, cy = pr.w >> 16;
        const int Tx = a.len[x], Ty = a.len[y];
        const float *tb = a.tilebuf + (int64_t)pr.z * (kPanel * kPanel) + rx * kPanel + cy;

        // largest |cos| of the block: |cos(pi d)| = sin(pi |d - 1/2|)
        float dev = 0.0f;
        for (int i = 0; i < Tx; ++i)
            for (int j = 0; j < Ty; ++j) dev = fmaxf(dev, fabsf(tb[i * kPanel + j] - 0.5f));
        const float cmax = sinf(3.14159265f * fminf(dev, 0.5f)) * 1.000001f + 1e-7f;
        // frame-distance error: cosine error eps_c through arccos, either by
        // the slope at |cos| <= cmax + eps_c or by arccos(1 - w) <= 1.02 sqrt(2w)
        const float ec = a.eps_c;
        const float m = cmax + ec;
        const float e_sqrt = 1.02f * sqrtf(2.0f * ec);
        const float e_lin = m < 1.0f ? ec / sqrtf((1.0f - m) * (1.0f + m)) : kInf;
        const float e_d = fminf(e_sqrt, e_lin) * 0.318309886f;
        const float delta = (a.theta_item[x] + a.theta_item[y]) * 0.31830989f + e_d + 4e-7f;
        const float lam = (float)(Tx + Ty - 1);
        const float gam = lam * u / (1.0f - lam * u);
        const float tau = 2.5f * (lam * delta * (1.0f + gam) + 2.0f * gam * lam) + 8.0f * gam * lam;

        float lc = 0.0f;
        uint32_t ll = 0;
        for (int i = 0; i < Tx; ++i) {
            lc = kInf;
            ll = 0;
            float dc = kInf;
            uint32_t dl = 0;
            const float *drow = tb + i * kPanel;
            for (int j = 0; j < Ty; ++j) {
                const float dij = drow[j];
                float uc = kInf;
                uint32_t ul = 0;
                if (i > 0) {
                    uc = rbc[j * nt + tid];
                    ul = rbl[j * nt + tid];
                }
                float mc;
                uint32_t info;
                if (i == 0 && j == 0) {
                    mc = 0.0f;
                    info = pack3(1, 1, 1);
                } else {
                    mc = fminf(uc, fminf(lc, dc));
                    uint32_t len = 255, lmin = 255, lmax = 0;
                    const float lim = mc + tau;
                    // lexicographic (cost, length) minimum and near-optimal range
                    if (uc == mc) len = min(len, ul & 0xffu);
                    if (lc == mc) len = min(len, ll & 0xffu);
                    if (dc == mc) len = min(len, dl & 0xffu);
                    if (uc <= lim) { lmin = min(lmin, (ul >> 8) & 0xffu); lmax = max(lmax, ul >> 16); }
                    if (lc <= lim) { lmin = min(lmin, (ll >> 8) & 0xffu); lmax = max(lmax, ll >> 16); }
                    if (dc <= lim) { lmin = min(lmin, (dl >> 8) & 0xffu); lmax = max(lmax, dl >> 16); }
                    info = pack3(len + 1, lmin + 1, lmax + 1);
                }
                const float nc = dij + mc;
                dc = uc;
                dl = ul;
                lc = nc;
                ll = info;
                rbc[j * nt + tid] = nc;
                rbl[j * nt + tid] = info;
            }
        }
        const float cost = lc;
        const uint32_t L = ll & 0xffu, Lmin = (ll >> 8) & 0xffu, Lmax = ll >> 16;
        const float D = __fdiv_rn(cost, (float)L);
        const float E = __fadd_ru(lam * delta * 1.0001f, 2.0f * gam * (cost + lam * delta) + 1e-7f);
        const float lo = fmaxf(0.0f, __fdiv_rd(__fsub_rd(cost, E), (float)Lmax));
        const float hi = fminf(1.0f, __fdiv_ru(__fadd_ru(cost, E), (float)Lmin));

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
