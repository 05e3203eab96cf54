// Pair planning: which item pairs of each 128 x 128 frame tile some triple
// of the task compares (fastabx Sec. 2 triple conditions), their count per
// tile, and the compact pair list the DTW kernel consumes.
#include <cuda_runtime.h>

#include "abx_internal.h"

namespace abx {
namespace {

__device__ __forceinline__ int blk_count(const TaskDev &t, int g, int p, int s) {
    return t.blk[((int64_t)g * t.K_on + p) * t.K_s + s].y;
}

// Unordered pair {x, y} (sorted indices, same group, x != y) is needed when
// one of them can be the X of a triple in which the other is A or B.
//   no across: same on -> needs some b of another on value in the group;
//              different on -> the X item needs a second item of its on value.
//   across:    across values must differ; same on -> the A item's across
//              value needs some b of another on value; different on -> the
//              B item's across value needs an a with the X item's on value.
__device__ __forceinline__ bool pair_needed(const TaskDev &t, int x, int y) {
    const int g = t.item_g[x];
    const int px = t.item_p[x], py = t.item_p[y];
    if (!t.across) {
        if (px == py) return t.tot[g] - blk_count(t, g, px, 0) > 0;
        return blk_count(t, g, px, 0) >= 2 || blk_count(t, g, py, 0) >= 2;
    }
    const int sx = t.item_s[x], sy = t.item_s[y];
    if (sx == sy) return false;
    if (px == py)
        return t.tot[(int64_t)g * t.K_s + sy] - blk_count(t, g, px, sy) > 0 ||
               t.tot[(int64_t)g * t.K_s + sx] - blk_count(t, g, px, sx) > 0;
    return blk_count(t, g, px, sy) > 0 || blk_count(t, g, py, sx) > 0;
}

// One warp per tile; candidates enumerated in (x, y) row-major order.
template <bool WRITE>
__global__ void plan_kernel(TaskDev t, TileList tl, const int32_t *len, const int32_t *row,
                            int32_t *tile_count, const int64_t *tile_base, int4 *pairs,
                            unsigned long long *frame_pairs) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= tl.n_tiles) return;
    const int2 pp = tl.tiles[w];
    const int ia = tl.panel_item[pp.x], ib = tl.panel_item[pp.x + 1];
    const int ja = tl.panel_item[pp.y], jb = tl.panel_item[pp.y + 1];
    const int mi = ib - ia, mj = jb - ja;
    const bool diag = pp.x == pp.y;
    const int r0 = tl.panel_row[pp.x], c0 = tl.panel_row[pp.y];
    const int64_t ncand = (int64_t)mi * mj;
    int64_t base = WRITE ? tile_base[w] : 0;
    int count = 0;
    unsigned long long fp = 0;
    for (int64_t c0i = 0; c0i < ncand; c0i += 32) {
        const int64_t c = c0i + lane;
        bool ok = false;
        int x = 0, y = 0;
        if (c < ncand) {
            x = ia + (int)(c / mj);
            y = ja + (int)(c % mj);
            ok = (!diag || y > x) && pair_needed(t, x, y);
        }
        const unsigned m = __ballot_sync(0xffffffffu, ok);
        if (WRITE && ok) {
            const int64_t pos = base + __popc(m & ((1u << lane) - 1u));
            const int rx = row[x] - r0, cy = row[y] - c0;
            pairs[pos] = make_int4(x, y, (int)w, rx | (cy << 16));
        }
        if (!WRITE && ok) fp += (unsigned long long)(len[x] * len[y]);
        base += __popc(m);
        count += __popc(m);
    }
    if (!WRITE) {
        for (int o = 16; o; o >>= 1) fp += __shfl_xor_sync(0xffffffffu, fp, o);
        if (lane == 0) {
            tile_count[w] = count;
            if (fp) atomicAdd(frame_pairs, fp);
        }
    }
}

// Exclusive scan of int32 counts into int64 offsets, single block.
__global__ void __launch_bounds__(1024) scan_kernel(const int32_t *in, int64_t *out, int64_t n,
                                                     int64_t *total, int64_t *accum) {
    __shared__ int64_t part[1024];
    const int tid = threadIdx.x;
    const int64_t per = (n + 1023) / 1024;
    const int64_t b = tid * per, e = b + per < n ? b + per : n;
    int64_t s = 0;
    for (int64_t i = b; i < e; ++i) s += in[i];
    part[tid] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        int64_t v = tid >= off ? part[tid - off] : 0;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    int64_t run = tid ? part[tid - 1] : 0;
    for (int64_t i = b; i < e; ++i) {
        out[i] = run;
        run += in[i];
    }
    if (tid == 1023) {
        out[n] = part[1023];
        *total = part[1023];
        *accum += part[1023];
    }
}

__global__ void gather_kernel(const PairVal *pv, const int64_t *ent, int64_t n, float *oD,
                              float *olo, float *ohi, int32_t *oL) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t e = ent[i];
    const float nan = __int_as_float(0x7fc00000);
    const PairVal v = e >= 0 ? pv[e] : PairVal{nan, nan, nan, 0u};
    const bool ok = v.len != 0;
    oD[i] = ok ? v.d : nan;
    olo[i] = ok ? v.lo : nan;
    ohi[i] = ok ? v.hi : nan;
    oL[i] = (int32_t)v.len;
}

}  // namespace

cudaError_t launch_plan_count(const TaskDev &t, const TileList &tl, const int32_t *len,
                              const int32_t *row, int32_t *tile_count, int64_t *frame_pairs,
                              cudaStream_t s) {
    if (tl.n_tiles == 0) return cudaSuccess;
    const int64_t threads = tl.n_tiles * 32;
    {
        ProfScope ps_("plan_count", s);
        plan_kernel<false><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
            t, tl, len, row, tile_count, nullptr, nullptr, (unsigned long long *)frame_pairs);
    }
    return cudaGetLastError();
}

cudaError_t launch_plan_write(const TaskDev &t, const TileList &tl, const int32_t *len,
                              const int32_t *row, const int64_t *tile_base, int4 *pairs,
                              cudaStream_t s) {
    if (tl.n_tiles == 0) return cudaSuccess;
    const int64_t threads = tl.n_tiles * 32;
    {
        ProfScope ps_("plan_write", s);
        plan_kernel<true><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
            t, tl, len, row, nullptr, tile_base, pairs, nullptr);
    }
    return cudaGetLastError();
}

cudaError_t launch_scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, int64_t *total,
                                   int64_t *accum, cudaStream_t s) {
    {
        ProfScope ps_("scan", s);
        scan_kernel<<<1, 1024, 0, s>>>(in, out, n, total, accum);
    }
    return cudaGetLastError();
}

cudaError_t launch_gather(const PairVal *pv, const int64_t *entries, int64_t n, float *oD,
                          float *olo, float *ohi, int32_t *oL, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    {
        ProfScope ps_("gather", s);
        gather_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pv, entries, n, oD, olo, ohi,
                                                                 oL);
    }
    return cudaGetLastError();
}

}  // namespace abx
