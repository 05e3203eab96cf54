// Pair planning: which item pairs of each 128 x 128 frame tile some triple
// of the task compares (fastabx Sec. 2 triple conditions), their count per
// tile, and the compact pair list the DTW kernel consumes.
#include <cuda_runtime.h>

#include <algorithm>

#include "abx_internal.h"

namespace abx {
namespace {

// Packed row -> sorted item: the rows of item k are row[k] .. row[k] +
// len[k] - 1 (items back to back, no gaps).  One thread per item.
__global__ void row_items_kernel(const int32_t *len, const int32_t *row, int64_t n_items,
                                 int32_t *row_item) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_items) return;
    const int32_t r0 = row[k], T = len[k];
    for (int32_t t = 0; t < T; ++t) row_item[r0 + t] = (int32_t)k;
}

__global__ void item_attrs_kernel(ItemAttrArgs a) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.n_items) return;
    const int32_t *lab = a.labels + (int64_t)a.item_id[k] * a.n_attr;
    int64_t code = 0;
    for (int b = 0; b < a.n_by; ++b) code = code * a.K_by[b] + lab[a.by[b]];
    a.item_g[k] = a.gtab[code];
    a.item_p[k] = lab[a.on];
    a.item_s[k] = a.across >= 0 ? lab[a.across] : 0;
}

// One warp per tile; candidates enumerated in (x, y) row-major order, the
// lane's (x, y) advanced by 32 candidates with a carry (no division per
// candidate).  The frame-pair total is summed over the block before its one
// atomic: one atomic per warp on a single counter serialised in L2.
// The count pass (WRITE = false) also writes the tile's store map for the
// tile kernels (launch_plan_count) when xmask / col_yo are given.
template <bool WRITE>
__global__ void __launch_bounds__(256) plan_kernel(TaskDev t, TileList tl, const int32_t *len,
                                                   const int32_t *row, int32_t *tile_count,
                                                   const int64_t *tile_base, int4 *pairs,
                                                   unsigned long long *frame_pairs,
                                                   uint64_t *xmask, uint8_t *col_yo,
                                                   const int32_t *row_item, int64_t n_rows) {
    __shared__ unsigned long long part[8];
    __shared__ unsigned long long msk[WRITE ? 1 : 8][kPanel];
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    unsigned long long fp = 0;
    if (w < tl.n_tiles) {
        const int2 pp = tl.tiles[w];
        const int ia = tl.panel_item[pp.x], ib = tl.panel_item[pp.x + 1];
        const int ja = tl.panel_item[pp.y], jb = tl.panel_item[pp.y + 1];
        const int mi = ib - ia, mj = jb - ja;
        const bool diag = pp.x == pp.y;
        const int r0 = tl.panel_row[pp.x], c0 = tl.panel_row[pp.y];
        const int ncand = mi * mj;  // <= 128 x 128
        const bool maps = !WRITE && xmask != nullptr && col_yo != nullptr;
        unsigned long long *wm = msk[WRITE ? 0 : (threadIdx.x >> 5)];
        if (maps) {
            // column -> column item (255 past the last), four columns per
            // lane in one 32-bit store; rows' masks cleared
            uint32_t word = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int64_t r = (int64_t)c0 + 4 * lane + k;
                const int y = r < n_rows ? row_item[r] : jb;
                word |= (uint32_t)(y < jb ? y - ja : 255) << (8 * k);
            }
            reinterpret_cast<uint32_t *>(col_yo + w * kPanel)[lane] = word;
            for (int c = lane; c < kPanel; c += 32) wm[c] = 0ull;
            __syncwarp();
        }
        int64_t base = WRITE ? tile_base[w] : 0;
        int count = 0;
        int xo = mj > 0 ? lane / mj : 0, yo = lane - xo * mj;  // lane's candidate
        const int dx = mj > 0 ? 32 / mj : 0, dy = 32 - dx * mj;
        for (int c0i = 0; c0i < ncand; c0i += 32) {
            const int c = c0i + lane;
            bool ok = false;
            const int x = ia + xo, y = ja + yo;
            if (c < ncand) ok = (!diag || y > x) && pair_needed(t, x, y);
            const unsigned m = __ballot_sync(0xffffffffu, ok);
            if (WRITE && ok) {
                const int64_t pos = base + __popc(m & ((1u << lane) - 1u));
                const int rx = row[x] - r0, cy = row[y] - c0;
                pairs[pos] = make_int4(x, y, (int)w, rx | (cy << 16));
            }
            if (!WRITE && ok) fp += (unsigned long long)(len[x] * len[y]);
            if (maps && ok && mj <= 64) atomicOr(&wm[xo], 1ull << yo);
            base += __popc(m);
            count += __popc(m);
            yo += dy;
            xo += dx;
            if (yo >= mj) {
                yo -= mj;
                ++xo;
            }
        }
        if (!WRITE && lane == 0) tile_count[w] = count;
        if (maps && mj <= 64) {
            __syncwarp();
            for (int i = lane; i < mi; i += 32) xmask[w * kPanel + i] = wm[i];
        }
    }
    if (!WRITE) {
        for (int o = 16; o; o >>= 1) fp += __shfl_xor_sync(0xffffffffu, fp, o);
        if (lane == 0) part[threadIdx.x >> 5] = fp;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long tot = 0;
            for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += part[i];
            if (tot) atomicAdd(frame_pairs, tot);
        }
    }
}

// Exclusive scan of int32 counts into int64 offsets in three kernels:
// per-block sums, a scan of the block sums, per-block scans plus offset.
// 128-thread blocks: the cell building's scans run on a high-priority stream
// beside a persistent tile kernel (576 threads x 96 registers per SM), and a
// block must fit in the registers that kernel leaves free (about 10k) to
// start before it ends; with 1024-thread blocks they waited for it.
constexpr int kScanBlock = 128;
constexpr int kScanItems = 8;                       // per thread
constexpr int kScanTile = kScanBlock * kScanItems;  // elements per block

__device__ __forceinline__ int64_t block_incl_scan(int64_t v, int64_t *sh) {
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        int64_t x = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        sh[lane] = x;
    }
    __syncthreads();
    const int64_t r = v + (w ? sh[w - 1] : 0);
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanBlock) scan_sums_kernel(const int32_t *in, int64_t n,
                                                                int64_t *sums) {
    __shared__ int64_t sh[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    int64_t v = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) v += in[base + i];
    const int64_t incl = block_incl_scan(v, sh);
    if (threadIdx.x == kScanBlock - 1) sums[blockIdx.x] = incl;
}

__global__ void __launch_bounds__(kScanBlock) scan_top_kernel(int64_t *sums, int64_t nb,
                                                               int64_t *total, int64_t *accum) {
    __shared__ int64_t sh[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b0 = 0; b0 < nb; b0 += kScanBlock) {
        const int64_t i = b0 + threadIdx.x;
        const int64_t v = i < nb ? sums[i] : 0;
        const int64_t incl = block_incl_scan(v, sh);
        if (i < nb) sums[i] = carry + incl - v;  // exclusive
        __syncthreads();
        if (threadIdx.x == kScanBlock - 1) carry += incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *total = carry;
        *accum += carry;
    }
}

__global__ void __launch_bounds__(kScanBlock) scan_apply_kernel(const int32_t *in, int64_t n,
                                                                 const int64_t *sums,
                                                                 int64_t *out, const int64_t *total) {
    __shared__ int64_t sh[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    int32_t x[kScanItems];
    int64_t v = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        x[i] = base + i < n ? in[base + i] : 0;
        v += x[i];
    }
    int64_t run = block_incl_scan(v, sh) - v + sums[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) {
            out[base + i] = run;
            run += x[i];
        }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = *total;
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
                              uint64_t *xmask, uint8_t *col_yo, const int32_t *row_item,
                              int64_t n_rows, cudaStream_t s) {
    if (tl.n_tiles == 0) return cudaSuccess;
    const int64_t threads = tl.n_tiles * 32;
    {
        ProfScope ps_("plan_count", s);
        plan_kernel<false><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
            t, tl, len, row, tile_count, nullptr, nullptr, (unsigned long long *)frame_pairs,
            xmask, col_yo, row_item, n_rows);
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
            t, tl, len, row, nullptr, tile_base, pairs, nullptr, nullptr, nullptr, nullptr, 0);
    }
    return cudaGetLastError();
}

cudaError_t launch_scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, int64_t *total,
                                   int64_t *accum, cudaStream_t s) {
    const int64_t nb = std::max<int64_t>(1, (n + kScanTile - 1) / kScanTile);
    int64_t *sums = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&sums, nb * sizeof(int64_t), s);
    if (e != cudaSuccess) return e;
    {
        ProfScope ps_("scan", s);
        scan_sums_kernel<<<(unsigned)nb, kScanBlock, 0, s>>>(in, n, sums);
    }
    {
        ProfScope ps_("scan", s);
        scan_top_kernel<<<1, kScanBlock, 0, s>>>(sums, nb, total, accum);
    }
    {
        ProfScope ps_("scan", s);
        scan_apply_kernel<<<(unsigned)nb, kScanBlock, 0, s>>>(in, n, sums, out, total);
    }
    e = cudaGetLastError();
    cudaFreeAsync(sums, s);
    return e;
}

cudaError_t launch_row_items(const int32_t *len, const int32_t *row, int64_t n_items,
                             int32_t *row_item, cudaStream_t s) {
    if (n_items == 0) return cudaSuccess;
    {
        ProfScope ps_("row_items", s);
        row_items_kernel<<<(unsigned)((n_items + 255) / 256), 256, 0, s>>>(len, row, n_items,
                                                                           row_item);
    }
    return cudaGetLastError();
}

cudaError_t launch_item_attrs(const ItemAttrArgs &a, cudaStream_t s) {
    if (a.n_items == 0) return cudaSuccess;
    {
        ProfScope ps_("item_attrs", s);
        item_attrs_kernel<<<(unsigned)((a.n_items + 255) / 256), 256, 0, s>>>(a);
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
