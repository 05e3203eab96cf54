// FP32 CUDA-core tile kernel: one CTA per 128 x 128 frame tile computes all
// frame cosines with FFMA and writes d = arccos(cos) / pi (fastabx Sec. 3.1
// angular distance) into the tile buffer.  Reference path for the tcgen05
// kernels and the ABX_FP32_SIMT precision.
#include <cuda_runtime.h>

#include "abx_internal.h"

namespace abx {
namespace {

constexpr int KC = 32;    // k per smem stage
constexpr int LDS = 132;  // padded row of the [k][row] stage

__global__ void __launch_bounds__(256) tile_simt_kernel(TileGemmArgs a) {
    const int64_t t = blockIdx.x;
    if (a.tile_count[t] == 0) return;
    const int2 pp = a.tiles[t];
    const int64_t r0 = a.panel_row[pp.x], c0 = a.panel_row[pp.y];
    __shared__ __align__(16) float As[KC][LDS];
    __shared__ __align__(16) float Bs[KC][LDS];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const float *P = reinterpret_cast<const float *>(a.packed);
    const int dp = a.dim_pad;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
    const int lr = tid >> 1, lk = (tid & 1) * 16;
    const int64_t ra = r0 + lr, rb = c0 + lr;
    const bool va = ra < a.n_rows, vb = rb < a.n_rows;
    for (int k0 = 0; k0 < dp; k0 += KC) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float4 x = va ? *reinterpret_cast<const float4 *>(P + ra * dp + k0 + lk + 4 * q)
                          : make_float4(0.f, 0.f, 0.f, 0.f);
            float4 y = vb ? *reinterpret_cast<const float4 *>(P + rb * dp + k0 + lk + 4 * q)
                          : make_float4(0.f, 0.f, 0.f, 0.f);
            As[lk + 4 * q + 0][lr] = x.x;
            As[lk + 4 * q + 1][lr] = x.y;
            As[lk + 4 * q + 2][lr] = x.z;
            As[lk + 4 * q + 3][lr] = x.w;
            Bs[lk + 4 * q + 0][lr] = y.x;
            Bs[lk + 4 * q + 1][lr] = y.y;
            Bs[lk + 4 * q + 2][lr] = y.z;
            Bs[lk + 4 * q + 3][lr] = y.w;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < KC; ++kk) {
            float av[8], bv[8];
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[kk][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[kk][ty * 8 + 4]);
            const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 8]);
            const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 8 + 4]);
            av[0] = a0.x; av[1] = a0.y; av[2] = a0.z; av[3] = a0.w;
            av[4] = a1.x; av[5] = a1.y; av[6] = a1.z; av[7] = a1.w;
            bv[0] = b0.x; bv[1] = b0.y; bv[2] = b0.z; bv[3] = b0.w;
            bv[4] = b1.x; bv[5] = b1.y; bv[6] = b1.z; bv[7] = b1.w;
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
    float *out = a.tilebuf + t * (int64_t)(kPanel * kPanel);
    const float inv_pi = 0.318309886183790671f;
    float ib[8], nb[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int64_t c = c0 + tx * 8 + j;
        ib[j] = c < a.n_rows ? a.inv_norm[c] : 0.0f;
        nb[j] = (a.distance == ABX_DIST_EUCLIDEAN && c < a.n_rows) ? a.nrm2[c] : 0.0f;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int row = ty * 8 + i;
        const bool rv = r0 + row < a.n_rows;
        const float ia = rv ? a.inv_norm[r0 + row] : 0.0f;
        const float na = (a.distance == ABX_DIST_EUCLIDEAN && rv) ? a.nrm2[r0 + row] : 0.0f;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float c = acc[i][j] * ia * ib[j];
            if (a.distance == ABX_DIST_EUCLIDEAN)
                acc[i][j] = sqrtf(fmaxf(0.0f, na + nb[j] - 2.0f * c));
            else if (a.distance == ABX_DIST_COSINE)
                acc[i][j] = 1.0f - fminf(1.0f, fmaxf(-1.0f, c));
            else
                acc[i][j] = acosf(fminf(1.0f, fmaxf(-1.0f, c))) * inv_pi;
        }
    }
    if (!a.strips) {  // column-major tile: element (row, col) at col * kPanel + row
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float4 *o = reinterpret_cast<float4 *>(out + (tx * 8 + j) * kPanel + ty * 8);
            o[0] = make_float4(acc[0][j], acc[1][j], acc[2][j], acc[3][j]);
            o[1] = make_float4(acc[4][j], acc[5][j], acc[6][j], acc[7][j]);
        }
        return;
    }
    // strips (tile_strip_offset): each row goes to its item's strip; rows
    // past the panel's last item are dropped
    const int32_t item_end = a.panel_item[pp.x + 1];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int row = ty * 8 + i;
        const int64_t r = r0 + row;
        const int x = r < a.n_rows ? a.row_item[r] : item_end;
        if (x >= item_end) continue;
        const int rx = (int)(a.row[x] - r0), Tx = a.len[x];
#pragma unroll
        for (int j = 0; j < 8; ++j) out[tile_strip_offset(rx, Tx, row, tx * 8 + j)] = acc[i][j];
    }
}

}  // namespace

cudaError_t launch_tile_simt(const TileGemmArgs &a, cudaStream_t s) {
    if (a.n_tiles == 0) return cudaSuccess;
    {
        ProfScope ps_("tile_simt", s);
        tile_simt_kernel<<<(unsigned)a.n_tiles, 256, 0, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace abx
