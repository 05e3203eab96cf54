// Cell building on the device (fastabx Sec. 2 task definition; Sec. 3.1
// Task): items sorted by (group, across value, on value), stable in item
// index, and the tables the distance and score kernels read.
//
//   groups     the distinct value combinations of the `by` attributes,
//              numbered in increasing mixed-radix code (presence flags and
//              an exclusive scan);
//   blocks     key (group, across, on): counts by atomics, offsets by a scan,
//              items scattered by atomics and each block's items then sorted
//              by item index (the order of a stable counting sort);
//   tables     block table [g][s][p] -> (first, count), per (group, across)
//              totals, group ranges and the offsets of the groups' item-pair
//              matrices (a scan of n_g^2);
//   candidates the number of cells the scorer enumerates, so that it can
//              size its cell arrays without reading a count back.
#include <cuda_runtime.h>

#include <algorithm>

#include "abx_internal.h"

namespace abx {
namespace {

__device__ __forceinline__ int64_t by_code(const CellBuildArgs &a, int64_t i) {
    const int32_t *lab = a.labels + i * a.n_attr;
    int64_t code = 0;
    for (int b = 0; b < a.n_by; ++b) code = code * a.K_by[b] + lab[a.by[b]];
    return code;
}

__global__ void cb_presence_kernel(CellBuildArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    a.flags[by_code(a, i)] = 1;
}

__global__ void cb_gtab_kernel(CellBuildArgs a) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.by_space) return;
    a.gtab[c] = a.flags[c] ? (int32_t)a.gpos[c] : -1;
}

__global__ void cb_key_kernel(CellBuildArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const int32_t *lab = a.labels + i * a.n_attr;
    const int64_t g = a.gtab[by_code(a, i)];
    const int64_t s = a.across >= 0 ? lab[a.across] : 0;
    const int64_t k = (g * a.K_s + s) * a.K_on + lab[a.on];
    a.key[i] = k;
    a.item_group[i] = (int32_t)g;
    atomicAdd(&a.counts[k], 1);
}

__global__ void cb_scatter_kernel(CellBuildArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const int64_t slot =
        (int64_t)atomicAdd((unsigned long long *)&a.cursor[a.key[i]], 1ull);
    a.item_id[slot] = (int32_t)i;
}

// Each block's items in increasing item index (insertion sort; blocks are
// small, a few items on average).
__global__ void cb_sort_kernel(CellBuildArgs a) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.nkeys) return;
    const int64_t b = a.pos[k], e = a.pos[k + 1];
    for (int64_t i = b + 1; i < e; ++i) {
        const int32_t v = a.item_id[i];
        int64_t j = i - 1;
        while (j >= b && a.item_id[j] > v) {
            a.item_id[j + 1] = a.item_id[j];
            --j;
        }
        a.item_id[j + 1] = v;
    }
}

// Block table, per (group, across) totals, group ranges and matrix sizes.
__global__ void cb_tables_kernel(CellBuildArgs a) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t G = *a.n_groups;
    const int64_t nkeys = G * a.K_s * a.K_on;
    if (k < nkeys) a.blk[k] = make_int2((int32_t)a.pos[k], (int32_t)(a.pos[k + 1] - a.pos[k]));
    if (k < G * a.K_s) a.tot[k] = (int32_t)(a.pos[(k + 1) * a.K_on] - a.pos[k * a.K_on]);
    if (k <= G) a.group_begin[k] = (int32_t)a.pos[k * a.K_s * a.K_on];
    if (k < G) {
        const int64_t ng = a.pos[(k + 1) * a.K_s * a.K_on] - a.pos[k * a.K_s * a.K_on];
        a.ng2[k] = (int32_t)ng;
    }
}

// Offsets of the groups' n_g x n_g matrices: an exclusive int64 scan of
// n_g^2 by one block (each thread a contiguous run of groups).
__global__ void __launch_bounds__(256) cb_dm_kernel(CellBuildArgs a) {
    __shared__ int64_t part[256];
    const int64_t G = *a.n_groups;
    const int t = threadIdx.x, nt = blockDim.x;
    const int64_t per = (G + nt - 1) / nt, g0 = std::min<int64_t>(G, t * per),
                  g1 = std::min<int64_t>(G, g0 + per);
    int64_t sum = 0;
    for (int64_t q = g0; q < g1; ++q) sum += (int64_t)a.ng2[q] * a.ng2[q];
    part[t] = sum;
    __syncthreads();
    if (t == 0) {
        int64_t run = 0;
        for (int i = 0; i < nt; ++i) {
            const int64_t v = part[i];
            part[i] = run;
            run += v;
        }
        *a.dm_total = run;
    }
    __syncthreads();
    int64_t dm = part[t];
    for (int64_t q = g0; q < g1; ++q) {
        const int64_t ng = a.ng2[q];
        a.group_dm[q] = dm;
        a.gmeta[q] = make_int4(a.group_begin[q], (int32_t)ng, (int32_t)(dm & 0xffffffff),
                               (int32_t)(dm >> 32));
        dm += ng * ng;
    }
}

// Non-empty blocks per (group, across value).
__global__ void cb_nz_kernel(CellBuildArgs a) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= *a.n_groups * a.K_s) return;
    const int2 *row = a.blk + k * a.K_on;
    int32_t n = 0;
    for (int p = 0; p < a.K_on; ++p) n += row[p].y > 0;
    a.nz_s[k] = n;
}

// Score candidates (group, P, Q, across_ab, across_x): the scorer keeps one
// per combination with P != Q whose blocks (P, across_ab), (Q, across_ab) and
// (P, across_x) are all non-empty, across_ab != across_x with an across
// attribute, and across_x = across_ab (the block of A) without one.  One
// thread per (group, P): with e(s) = [block (P, s) non-empty],
//   across:    (sum_s e(s) - 1) * sum_s e(s) (nz(s) - 1)
//   otherwise: e * (nz - 1),
// nz(s) the non-empty blocks of (group, s).  Summed per thread block, then
// one atomic add.
__global__ void __launch_bounds__(256) cb_cand_kernel(CellBuildArgs a) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long n = 0;
    if (k < *a.n_groups * a.K_on) {
        const int64_t g = k / a.K_on;
        const int p = (int)(k - g * a.K_on);
        int64_t ep = 0, sum = 0;
        for (int s = 0; s < a.K_s; ++s) {
            const int64_t gs = g * a.K_s + s;
            if (a.blk[gs * a.K_on + p].y > 0) {
                ++ep;
                sum += a.nz_s[gs] - 1;
            }
        }
        n = (unsigned long long)(a.across >= 0 ? (ep - 1) * sum : sum);
    }
    for (int o = 16; o; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    __shared__ unsigned long long part[8];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = n;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        if (t) atomicAdd((unsigned long long *)a.n_cand, t);
    }
}

unsigned grid(int64_t n) { return (unsigned)std::max<int64_t>(1, (n + 255) / 256); }

}  // namespace

cudaError_t launch_cell_build(const CellBuildArgs &a, int64_t nkeys_max, int64_t g_max,
                              int64_t *scratch, cudaStream_t s) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(a.flags, 0, a.by_space * sizeof(int32_t), s))) return e;
    {
        ProfScope ps_("build_cells", s);
        cb_presence_kernel<<<grid(a.n), 256, 0, s>>>(a);
    }
    if ((e = launch_scan_i32_to_i64(a.flags, a.gpos, a.by_space, a.n_groups, scratch, s)))
        return e;
    {
        ProfScope ps_("build_cells", s);
        cb_gtab_kernel<<<grid(a.by_space), 256, 0, s>>>(a);
    }
    if ((e = cudaMemsetAsync(a.counts, 0, nkeys_max * sizeof(int32_t), s))) return e;
    {
        ProfScope ps_("build_cells", s);
        cb_key_kernel<<<grid(a.n), 256, 0, s>>>(a);
    }
    // offsets over the largest key space (keys of absent groups count 0)
    if ((e = launch_scan_i32_to_i64(a.counts, a.pos, nkeys_max, scratch + 1, scratch + 2, s)))
        return e;
    if ((e = cudaMemcpyAsync(a.cursor, a.pos, nkeys_max * sizeof(int64_t),
                             cudaMemcpyDeviceToDevice, s)))
        return e;
    CellBuildArgs b = a;
    b.nkeys = nkeys_max;
    {
        ProfScope ps_("build_cells", s);
        cb_scatter_kernel<<<grid(a.n), 256, 0, s>>>(a);
    }
    {
        ProfScope ps_("build_cells", s);
        cb_sort_kernel<<<grid(nkeys_max), 256, 0, s>>>(b);
    }
    {
        ProfScope ps_("build_cells", s);
        cb_tables_kernel<<<grid(std::max(nkeys_max, g_max + 1)), 256, 0, s>>>(a);
    }
    {
        ProfScope ps_("build_cells", s);
        cb_dm_kernel<<<1, 256, 0, s>>>(a);
    }
    if ((e = cudaMemsetAsync(a.n_cand, 0, sizeof(int64_t), s))) return e;
    {
        ProfScope ps_("build_cells", s);
        cb_nz_kernel<<<grid(g_max * a.K_s), 256, 0, s>>>(a);
        cb_cand_kernel<<<grid(g_max * a.K_on), 256, 0, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace abx
