// DTW kernel (fastabx Sec. 3.2): for every needed item pair, the dynamic
// programme c(i,j) = d(i,j) + min(c(i-1,j), c(i,j-1), c(i-1,j-1)) over the
// pair's block of the frame-distance tile, normalised by the number of cells
// on the optimal path (shorter path on equal cost).
//
// One thread per pair.  The pairs are short (3..40 frames here) and number in
// the millions, so a whole-warp wavefront per pair would leave most lanes
// idle; instead each thread walks its pair row by row with the previous row
// in shared memory, laid out [column][thread] so that a warp's accesses fall
// on 32 distinct banks.  The anti-diagonal wavefront is kept as variant 4
// (dtw_wave_kernel, one 8-lane group per pair): on the triphone-scale step
// it took 12.4 ms against 3.8 ms for this kernel (since 3.4 ms with the
// chunk claiming and one block per window below).
//
// A warp runs as long as its longest pair, so pairs of similar shape are
// dealt to the same warp: each block takes a window of kDtwWin consecutive
// pairs (tile order, about twenty tiles, so the reads stay local), sorts it
// by the Morton code of (Ty, Tx) in shared memory (bitonic network), and its
// warps claim chunks of 32 consecutive sorted positions from a shared
// counter, the largest shapes first.  Unsorted, a warp ran at about a
// quarter of its lanes; sorted windows of 2048 pairs measured 1.7x faster
// than unsorted (Morton order beat (Ty, Tx) order; 4096-pair windows lost
// occupancy).
//
// A pair's block of the tile buffer is stored column by column (Tx
// consecutive distances per frame of y; the columns back to back in the
// strip layout, 128 floats apart in a column-major tile), so the walk goes
// over the transposed table, outer index over y's frames, inner index over
// x's frames, reading contiguous columns.  The step set and the shorter-path rule are symmetric
// under transposition, so cost, path length and interval are those of the
// row-major walk.
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

// Morton (bit-interleaved) code of (Ty, Tx), 7 bits each: pairs of similar
// shape in both dimensions get close codes.
__device__ __forceinline__ uint32_t shape_code(uint32_t ty, uint32_t tx) {
    uint32_t code = 0;
#pragma unroll
    for (int b = 0; b < 7; ++b) code |= (((ty >> b) & 1u) << (2 * b + 1)) | (((tx >> b) & 1u) << (2 * b));
    return code;
}

// DTW of pair p by the calling thread (row buffers at column stride nt).
__device__ __forceinline__ void dtw_pair(const DtwArgs &a, int64_t p, int tid, int nt,
                                         float *rbc, uint32_t *rbl) {
    const int4 pr = a.pairs[p];
    const int x = pr.x, y = pr.y;
    const int rx = pr.w & 0xffff, cy = pr.w >> 16;
    const int Tx = a.len[x], Ty = a.len[y];
    // the pair's block: d(i, j) at tb[j * ld + i], in strips (tile_strip_offset,
    // ld = Tx: the block is contiguous) or a column-major tile (ld = 128)
    const int ld = a.strips ? Tx : kPanel;
    const float *tb = a.tilebuf + (int64_t)pr.z * (kPanel * kPanel) +
                      (a.strips ? tile_strip_offset(rx, Tx, rx, cy) : (int64_t)cy * kPanel + rx);
    const DtwBound bd = dtw_bound(Tx, Ty, a.theta_item[x], a.theta_item[y], a.eps_c);
    const float tau = bd.tau;

    float dev = 0.0f;  // largest |d - 1/2|, i.e. largest |cos|
    float lc = 0.0f;
    uint32_t ll = 0;
    for (int i = 0; i < Ty; ++i) {
        const float *drow = tb + i * ld;
        float dc, uc;
        uint32_t dl, ul;
        lc = kInf;
        ll = 0;
        dc = kInf;
        dl = 0;
        int j = 0;
        for (; j + 4 <= Tx; j += 4) {
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
        for (; j < Tx; ++j) {
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
    dtw_interval(bd, cost, ll, dev, a.eps_c, a.intervals, D, lo, hi);

    const int4 gm = a.t.gmeta[a.t.item_g[x]];
    const int gb = gm.x;
    const int64_t ng = gm.y;
    const int64_t base = ((int64_t)(uint32_t)gm.w << 32) | (uint32_t)gm.z;
    const PairVal v{D, lo, hi, L};
    a.pv[base + (int64_t)(x - gb) * ng + (y - gb)] = v;
    a.pv[base + (int64_t)(y - gb) * ng + (x - gb)] = v;
}

// NT threads: 256, or 128 when the row buffers of long items do not fit.
// NT threads per block, kDtwWin pairs per sorted window (default 256, 2048)
template <int NT, int kDtwWin>
__global__ void __launch_bounds__(NT) dtw_kernel(DtwArgs a) {
    extern __shared__ float smem[];
    __shared__ uint32_t key[kDtwWin];
    __shared__ int next_chunk;
    const int tid = threadIdx.x, nt = NT;
    float *rbc = smem;                                              // [max_len][nt]
    uint32_t *rbl = reinterpret_cast<uint32_t *>(smem + a.max_len * nt);
    const int64_t n_pairs = *a.n_pairs;
    for (int64_t p0 = (int64_t)blockIdx.x * kDtwWin; p0 < n_pairs;
         p0 += (int64_t)gridDim.x * kDtwWin) {
        // keys: shape code (14 bits) | window position (11 bits); absent pairs
        // sort last
#pragma unroll
        for (int k = 0; k < kDtwWin / NT; ++k) {
            const int i = tid + k * NT;
            uint32_t kv = 0xffffffffu;
            if (p0 + i < n_pairs) {
                const int4 pr = a.pairs[p0 + i];
                const uint32_t ty = a.len[pr.y], tx = a.len[pr.x];
                kv = (shape_code(ty, tx) << 11) | (uint32_t)i;
            }
            key[i] = kv;
        }
        if (tid == 0) next_chunk = 0;
        __syncthreads();
        for (int k = 2; k <= kDtwWin; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int q = tid; q < kDtwWin / 2; q += NT) {
                    const int i = ((q & ~(j - 1)) << 1) | (q & (j - 1));
                    const uint32_t u = key[i], w = key[i + j];
                    if ((u > w) == ((i & k) == 0)) {
                        key[i] = w;
                        key[i + j] = u;
                    }
                }
                __syncthreads();
            }
        // each warp claims the next chunk of 32 sorted positions until none
        // is left, largest shapes first, so the warps of the block reach the
        // end of the window together
        constexpr int kChunks = kDtwWin / 32;
#pragma unroll 1
        for (;;) {
            int c = 0;
            if ((tid & 31) == 0) c = atomicAdd(&next_chunk, 1);
            c = __shfl_sync(0xffffffffu, c, 0);
            if (c >= kChunks) break;
            const uint32_t kv = key[(kChunks - 1 - c) * 32 + (tid & 31)];
            if (kv != 0xffffffffu) dtw_pair(a, p0 + (kv & (kDtwWin - 1)), tid, nt, rbc, rbl);
        }
        __syncthreads();  // key and next_chunk are rewritten by the next window
    }
}

// Variant 4: the anti-diagonal wavefront (dtw_wave8) on the tile buffer, one
// 8-lane group per pair, x's frames on the rows so that a group's lanes read
// consecutive addresses of the pair's column-major block.  Pairs are taken in tile
// order, without sorting.
struct GlobalBlock {
    const float *tb;  // the pair's block: d(i, j) at tb[j * ld + i]
    int ld;
    __device__ __forceinline__ float operator()(int i, int j) const {
        return __ldg(tb + j * ld + i);
    }
};

constexpr int kWaveThreads = 256;
constexpr int kWaveGroups = kWaveThreads / 8;

__global__ void __launch_bounds__(kWaveThreads) dtw_wave_kernel(DtwArgs a) {
    __shared__ float rbc[kWaveGroups * kMaxItemLen];
    __shared__ uint32_t rbl[kWaveGroups * kMaxItemLen];
    const int lane = threadIdx.x & 31;
    const int grp = threadIdx.x >> 3;
    const int64_t n_pairs = *a.n_pairs;
    const int64_t stride = (int64_t)gridDim.x * kWaveGroups;
    for (int64_t p = (int64_t)blockIdx.x * kWaveGroups + grp; p < n_pairs; p += stride) {
        const int4 pr = a.pairs[p];
        const int x = pr.x, y = pr.y;
        const int rx = pr.w & 0xffff, cy = pr.w >> 16;
        const int Tx = a.len[x], Ty = a.len[y];
        const DtwBound bd = dtw_bound(Tx, Ty, a.theta_item[x], a.theta_item[y], a.eps_c);
        const GlobalBlock dat{a.tilebuf + (int64_t)pr.z * (kPanel * kPanel) +
                                  (a.strips ? tile_strip_offset(rx, Tx, rx, cy)
                                            : (int64_t)cy * kPanel + rx),
                              a.strips ? Tx : kPanel};
        float cost, dev;
        uint32_t info;
        dtw_wave8(dat, Tx, Ty, bd.tau, rbc + grp * kMaxItemLen, rbl + grp * kMaxItemLen, cost,
                  info, dev);
        if ((lane & 7) == 0) {
            const uint32_t L = info & 0xffu;
            const float D = __fdiv_rn(cost, (float)L);
            float lo, hi;
            dtw_interval(bd, cost, info, dev, a.eps_c, a.intervals, D, lo, hi);
            const int4 gm = a.t.gmeta[a.t.item_g[x]];
            const int gb = gm.x;
            const int64_t ng = gm.y;
            const int64_t base = ((int64_t)(uint32_t)gm.w << 32) | (uint32_t)gm.z;
            const PairVal v{D, lo, hi, L};
            a.pv[base + (int64_t)(x - gb) * ng + (y - gb)] = v;
            a.pv[base + (int64_t)(y - gb) * ng + (x - gb)] = v;
        }
    }
}

}  // namespace

template <int NT, int kDtwWin>
cudaError_t launch_dtw_nt(const DtwArgs &a, size_t smem, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(dtw_kernel<NT, kDtwWin>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dtw_kernel<NT, kDtwWin>, NT, smem);
    if (e != cudaSuccess) return e;
    // one block per window (blocks past the device-side pair count return at
    // once), so the block scheduler balances the SMs window by window; the
    // cap only bounds the grid of a very large pair capacity
    int64_t blocks = (a.pair_cap + kDtwWin - 1) / kDtwWin;
    const int64_t cap = (int64_t)nsm * (per_sm > 0 ? per_sm : 1) * 256;
    if (blocks > cap) blocks = cap;
    ProfScope ps_("dtw", s);
    dtw_kernel<NT, kDtwWin><<<(unsigned)blocks, NT, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_dtw(const DtwArgs &a, cudaStream_t s) {
    if (a.pair_cap == 0) return cudaSuccess;
    if (a.variant == 4) {  // wavefront groups (not among the autotuner's choices)
        int dev = 0, nsm = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        int64_t blocks = (a.pair_cap + kWaveGroups - 1) / kWaveGroups;
        blocks = std::min<int64_t>(blocks, (int64_t)nsm * 8);
        ProfScope ps_("dtw_wave", s);
        dtw_wave_kernel<<<(unsigned)blocks, kWaveThreads, 0, s>>>(a);
        return cudaGetLastError();
    }
    const size_t row = (size_t)a.max_len * 8;  // bytes of row buffer per thread
    // variants (autotuner): 0 = 256 threads / 2048-pair windows, 1 = 256 /
    // 1024, 2 = 128 / 2048, 3 = 128 / 1024; 128 threads when long items leave
    // no room for 256 row buffers
    const bool fits256 = row * 256 + 2048 * 4 <= 200 * 1024;
    switch (fits256 ? a.variant : (a.variant == 1 || a.variant == 3 ? 3 : 2)) {
    case 1: return launch_dtw_nt<256, 1024>(a, row * 256, s);
    case 2: return launch_dtw_nt<128, 2048>(a, row * 128, s);
    case 3: return launch_dtw_nt<128, 1024>(a, row * 128, s);
    default: return launch_dtw_nt<256, 2048>(a, row * 256, s);
    }
}

}  // namespace abx
