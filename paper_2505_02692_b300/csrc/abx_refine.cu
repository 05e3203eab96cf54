// Refined stage of the recheck: the DTW distance of every listed item pair
// recomputed from the raw FP32 features, with an interval that holds the
// exact distance (the angular frame distance of fastabx Sec. 3.1 and the
// Sec. 3.2 DTW, normalised by the optimal path's length).
//
// A low-precision distance matrix (FP8, BF16) leaves a triple undecided when
// the intervals of its two distances overlap; those intervals are wide
// because they must hold for every direction of the quantisation error.  The
// pairs of such triples are recomputed here first, at TF32 precision on the
// tensor cores; only the triples that these narrower intervals still cannot
// separate go to the FP64 kernel, whose double-word dot products cost far
// more per product.
//
// Stored vectors.  Every feature element is rounded to TF32 (10 fraction
// bits, round to nearest) in registers before the MMA, so the kernel computes
// the cosine of q_x = tf32(x) and q_y = tf32(y) exactly as a tensor-core dot
// product of those values.  A prep pass over the features (refine_prep)
// stores per frame 1 / |q| and the angle between the frame and its rounding,
// theta = asin(|q - x| / |x|) (an upper bound: a perturbation of relative
// size r turns a vector by at most asin(r)); the angle between two frames
// then moves by at most theta_x + theta_y, and the DTW interval adds each
// item's largest angle like the quantisation angle of the tile kernels.
//
// Dot products.  The Tx x Ty dot products of a pair are mma.sync m16n8k8
// tiles (x frames on the 16 rows, y frames on the 8 columns, FP32
// accumulation), one or two tiles (16 x 16 frames) per pass over the feature
// dimension, several accumulator chains taking the 16-dimension chunks in
// turn.  The k index of the MMA is a permutation of the feature dimension
// chosen so that each thread feeds two consecutive k-steps from one float4:
// for the 16 dimensions [b, b + 16), thread (g, t) = (lane / 4, lane % 4)
// takes dimensions b + 4t .. b + 4t + 3 of its rows, and k-step 0 takes
// k = t <-> b + 4t, k = t + 4 <-> b + 4t + 1, k-step 1 the other two.  The
// same permutation on both operands leaves every dot product unchanged, and
// each output lands in one thread's accumulator (no cross-lane reduction).
//
// Kernels.  For 16-byte feature rows (the usual case) two kernels:
// refine_fd_kernel, one warp per pair, the feature chunks staged in shared
// memory by cp.async (four chunks in flight per warp), the frame distances
// written to a buffer; then refine_dp_kernel, one thread per pair, the
// dynamic programme and the interval.  Otherwise refine_dtw_kernel does both
// in one: a warp takes four consecutive pairs per round, their distances go
// (one pair after another, loads four chunks deep) to four slices of shared
// memory, and each 8-lane group then runs one pair's dynamic programme as an
// anti-diagonal wavefront (dtw_wave8), the four at once.
//
// Error of a cosine of the stored vectors: the MMA accumulation is bounded
// with the same model as the tcgen05 kernels (each instruction of K = 8
// products adds at most (K + 2) 2^-23 of the sum of the magnitudes), over
// at most m = 2 ceil(dim / 16) instructions: gamma(10 m, 2^-23), relative
// to sum |q_x q_y| <= |q_x| |q_y| (the kernel's two or four chains are
// each a fraction of that long, and their sum adds at most three FP32
// roundings, well inside the bound).  The squared norms carry gamma_n with
// n = 4 ceil(dim / 128) + 5 (lane chains and a warp tree in refine_prep),
// and 1 / sqrt and the two products add 7u, u = 2^-24 (refine_cosine_bound).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>
#include <string.h>

#include "abx_dtw_cell.cuh"
#include "abx_internal.h"

namespace abx {

float refine_cosine_bound(int dim) {
    auto gamma = [](double n, double u) { return n * u / (1.0 - n * u); };
    const double u = std::ldexp(1.0, -24), u23 = std::ldexp(1.0, -23);
    const double m = 2.0 * ((dim + 15) / 16);
    const double n = 4.0 * ((dim + 127) / 128) + 5.0;
    return (float)((gamma(10.0 * m, u23) + gamma(n, u) + 7.0 * u) * 1.0001);
}

namespace {

constexpr int kRefineMaxWarps = 8;

__device__ __forceinline__ uint32_t tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mma_tf32(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, "
        "{%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Four consecutive features of row r at dimension c (zeros past the row
// count or the dimension).
template <bool V4>
__device__ __forceinline__ float4 load4(const float *F, int r, int rows, int c, int dim) {
    if (r >= rows) return make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    const float *p = F + (int64_t)r * dim + c;
    if (V4) {
        if (c < dim) return __ldg(reinterpret_cast<const float4 *>(p));
        return make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    float4 v;
    v.x = c < dim ? __ldg(p) : 0.0f;
    v.y = c + 1 < dim ? __ldg(p + 1) : 0.0f;
    v.z = c + 2 < dim ? __ldg(p + 2) : 0.0f;
    v.w = c + 3 < dim ? __ldg(p + 3) : 0.0f;
    return v;
}

// Dot products of x rows [0, nx) (nx <= 16 MT) with y rows [0, ny)
// (ny <= 8 NT) into dm (row stride ld), MT x NT m16n8k8 tiles.  NA
// accumulator sets take the 16-dimension chunks in turn (NA independent MMA
// chains instead of one; 4 for one tile, 2 for two) and are added at the
// end.
template <bool V4, int MT, int NT>
__device__ __forceinline__ void tile_dots(const float *X, int nx, const float *Y, int ny,
                                          int dim, int lane, float *dm, int ld) {
    constexpr int NA = NT == 1 ? 4 : 2;
    const int g = lane >> 2, t = lane & 3;
    float acc[NA][MT][NT][4];
#pragma unroll
    for (int q = 0; q < NA; ++q)
#pragma unroll
        for (int m = 0; m < MT; ++m)
#pragma unroll
            for (int n = 0; n < NT; ++n)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[q][m][n][e] = 0.0f;
    // this thread's rows (NULL: past the item, read as zero) at dimension 4t
    const float *xr[MT][2], *yr[NT];
#pragma unroll
    for (int m = 0; m < MT; ++m)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int r = 16 * m + 8 * h + g;
            xr[m][h] = r < nx ? X + (int64_t)r * dim + 4 * t : nullptr;
        }
#pragma unroll
    for (int n = 0; n < NT; ++n) {
        const int r = 8 * n + g;
        yr[n] = r < ny ? Y + (int64_t)r * dim + 4 * t : nullptr;
    }
    auto ld4 = [&](const float *p, int b) -> float4 {
        if (!p) return make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (V4) {
            if (b + 4 * t < dim) return __ldg(reinterpret_cast<const float4 *>(p + b));
            return make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
        const int c = b + 4 * t;
        float4 v;
        v.x = c < dim ? __ldg(p + b) : 0.0f;
        v.y = c + 1 < dim ? __ldg(p + b + 1) : 0.0f;
        v.z = c + 2 < dim ? __ldg(p + b + 2) : 0.0f;
        v.w = c + 3 < dim ? __ldg(p + b + 3) : 0.0f;
        return v;
    };
    const int nchunk = (dim + 15) >> 4;
    for (int k0 = 0; k0 < nchunk; k0 += NA) {
        // the loads of NA chunks first, so that they are in flight together
        uint32_t xa[NA][MT][2][4], yb[NA][NT][4];
#pragma unroll
        for (int q = 0; q < NA; ++q) {
            const int b = 16 * (k0 + q);
            const bool in = k0 + q < nchunk;
#pragma unroll
            for (int m = 0; m < MT; ++m)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float4 v = in ? ld4(xr[m][h], b) : make_float4(0.f, 0.f, 0.f, 0.f);
                    xa[q][m][h][0] = tf32(v.x);
                    xa[q][m][h][1] = tf32(v.y);
                    xa[q][m][h][2] = tf32(v.z);
                    xa[q][m][h][3] = tf32(v.w);
                }
#pragma unroll
            for (int n = 0; n < NT; ++n) {
                const float4 v = in ? ld4(yr[n], b) : make_float4(0.f, 0.f, 0.f, 0.f);
                yb[q][n][0] = tf32(v.x);
                yb[q][n][1] = tf32(v.y);
                yb[q][n][2] = tf32(v.z);
                yb[q][n][3] = tf32(v.w);
            }
        }
#pragma unroll
        for (int s2 = 0; s2 < 2; ++s2)
#pragma unroll
            for (int q = 0; q < NA; ++q)
#pragma unroll
                for (int m = 0; m < MT; ++m)
#pragma unroll
                    for (int n = 0; n < NT; ++n)
                        mma_tf32(acc[q][m][n], xa[q][m][0][2 * s2], xa[q][m][1][2 * s2],
                                 xa[q][m][0][2 * s2 + 1], xa[q][m][1][2 * s2 + 1],
                                 yb[q][n][2 * s2], yb[q][n][2 * s2 + 1]);
    }
#pragma unroll
    for (int m = 0; m < MT; ++m)
#pragma unroll
        for (int n = 0; n < NT; ++n)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                float v = acc[0][m][n][e];
#pragma unroll
                for (int q = 1; q < NA; ++q) v += acc[q][m][n][e];
                const int i = 16 * m + g + 8 * (e >> 1), j = 8 * n + 2 * t + (e & 1);
                if (i < nx && j < ny) dm[i * ld + j] = v;
            }
}

// Largest TF32 rounding angle of the n frames from f0 (by one thread).
__device__ __forceinline__ float item_theta(const float *theta_frame, int64_t f0, int n) {
    float t = 0.0f;
    for (int i = 0; i < n; ++i) t = fmaxf(t, __ldg(theta_frame + f0 + i));
    return t;
}

// The same by a warp (every lane gets it).
__device__ __forceinline__ float item_theta_warp(const float *theta_frame, int64_t f0, int n,
                                                 int lane) {
    float t = 0.0f;
    for (int i = lane; i < n; i += 32) t = fmaxf(t, __ldg(theta_frame + f0 + i));
    for (int o = 16; o; o >>= 1) t = fmaxf(t, __shfl_xor_sync(0xffffffffu, t, o));
    return t;
}

struct SmemMat {
    const float *m;
    int ld;
    __device__ __forceinline__ float operator()(int i, int j) const { return m[i * ld + j]; }
};

constexpr int kRefineGroup = 4;  // most pairs per warp and round: one DP per 8-lane group

template <bool V4>
__global__ void __launch_bounds__(kRefineMaxWarps * 32, 2) refine_dtw_kernel(RefineArgs a) {
    extern __shared__ float sm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int grp = lane >> 3;
    const int ML = a.max_len;
    // per warp and pair of the round: distances [ML * ML], row buffers of
    // the wavefront [2 * ML]
    const size_t per_pair = (size_t)ML * ML + 2 * ML;
    const int G = a.group;  // pairs per round (1, 2 or 4: what shared memory holds)
    float *wbuf = sm + (size_t)warp * G * per_pair;
    const int count = min(*a.count, a.capacity);
    const int64_t stride = (int64_t)gridDim.x * nw * G;
    for (int64_t q0 = ((int64_t)blockIdx.x * nw + warp) * G; q0 < count; q0 += stride) {
        // 1. frame distances of up to G consecutive pairs, one after
        // another, each into its own buffer
        float devs = 0.0f;  // lane-group p keeps pair p's largest |d - 1/2|
        float thx = 0.0f, thy = 0.0f;  // and its items' largest rounding angles
        for (int p = 0; p < G && q0 + p < count; ++p) {
            const int2 pr = a.list[q0 + p];
            const int64_t gx = a.item_id ? a.item_id[pr.x] : pr.x;
            const int64_t gy = a.item_id ? a.item_id[pr.y] : pr.y;
            const int64_t ox = a.offsets[gx], oy = a.offsets[gy];
            const int Tx = (int)(a.offsets[gx + 1] - ox), Ty = (int)(a.offsets[gy + 1] - oy);
            const float *X = a.feats + ox * (int64_t)a.dim;
            const float *Y = a.feats + oy * (int64_t)a.dim;
            float *dm = wbuf + p * per_pair;
            // passes of at most 16 x 16 frames (one or two tiles: few
            // registers, so that many warps share an SM)
            for (int ib = 0; ib < Tx; ib += 16) {
                const int nx = min(16, Tx - ib);
                for (int jb = 0; jb < Ty; jb += 16) {
                    const int ny = min(16, Ty - jb);
                    const float *Xb = X + (int64_t)ib * a.dim, *Yb = Y + (int64_t)jb * a.dim;
                    float *out = dm + ib * Ty + jb;
                    if (ny > 8)
                        tile_dots<V4, 1, 2>(Xb, nx, Yb, ny, a.dim, lane, out, Ty);
                    else
                        tile_dots<V4, 1, 1>(Xb, nx, Yb, ny, a.dim, lane, out, Ty);
                }
            }
            __syncwarp();
            float dev = 0.0f;  // largest |d - 1/2| of the pair, i.e. largest |cos|
            const float rTy = 1.0f / (float)Ty;
            for (int e = lane; e < Tx * Ty; e += 32) {
                // (i, j) of entry e: the float quotient is off by at most one
                int i = __float2int_rz((float)e * rTy);
                int j = e - i * Ty;
                if (j < 0) {
                    --i;
                    j += Ty;
                } else if (j >= Ty) {
                    ++i;
                    j -= Ty;
                }
                const float c = __fmul_rn(__fmul_rn(dm[e], __ldg(a.inv_q + ox + i)),
                                          __ldg(a.inv_q + oy + j));
                const float d = acosf(fminf(1.0f, fmaxf(-1.0f, c))) * 0.318309886183790671f;
                dm[e] = d;
                dev = fmaxf(dev, fabsf(d - 0.5f));
            }
            for (int o = 16; o; o >>= 1) dev = fmaxf(dev, __shfl_xor_sync(0xffffffffu, dev, o));
            const float tx = item_theta_warp(a.theta_frame, ox, Tx, lane);
            const float ty = item_theta_warp(a.theta_frame, oy, Ty, lane);
            if (grp == p) {
                devs = dev;
                thx = tx;
                thy = ty;
            }
            __syncwarp();
        }
        // 2. the dynamic programmes, 8-lane group p on pair p
        const int64_t q = q0 + grp;
        if (grp < G && q < count) {
            const int2 pr = a.list[q];
            const int64_t gx = a.item_id ? a.item_id[pr.x] : pr.x;
            const int64_t gy = a.item_id ? a.item_id[pr.y] : pr.y;
            const int Tx = (int)(a.offsets[gx + 1] - a.offsets[gx]);
            const int Ty = (int)(a.offsets[gy + 1] - a.offsets[gy]);
            float *dm = wbuf + grp * per_pair;
            float *rbc = dm + ML * ML;
            uint32_t *rbl = reinterpret_cast<uint32_t *>(rbc + ML);
            // the distances are known before the pass: tau from their own |cos|
            const DtwBound bd = dtw_bound_dev(Tx, Ty, thx, thy, a.eps_c, devs);
            float cost, dev;
            uint32_t info;
            dtw_wave8(SmemMat{dm, Ty}, Tx, Ty, bd.tau, rbc, rbl, cost, info, dev);
            if ((lane & 7) == 0) {
                const float D = __fdiv_rn(cost, (float)(info & 0xffu));
                float lo, hi;
                dtw_interval(bd, cost, info, dev, a.eps_c, 1, D, lo, hi);
                a.iv[q] = make_float2(lo, hi);
            }
        }
        __syncwarp();
    }
}

// ---------------------------------------------- two-kernel refined stage
// The frame distances of the listed pairs (refine_fd_kernel) and their
// dynamic programmes (refine_dp_kernel) as separate kernels: the distance
// kernel then holds no DP buffers, its warps only stream features, and the
// DP runs one thread per pair at full width.  Each warp of the distance
// kernel stages its feature chunks in shared memory with cp.async (16 bytes
// per thread and copy, kRingD chunks in flight), reads its own copies back
// and feeds the same m16n8k8 TF32 MMAs as tile_dots.  Distances go to a
// buffer in [x frame][y frame] order at a per-pair offset that each warp
// takes for its pairs with one atomicAdd; a pair that does not fit gets
// offset -1 and the interval [0, 1] (its triples then go to FP64).

constexpr int kRingD = 4;        // chunks in flight per warp
constexpr int kFdWarps = 8;      // warps per block of refine_fd_kernel
constexpr int kDpThreads = 128;  // threads per block of refine_dp_kernel

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// 16 bytes from src to shared dst, or zeros when !valid (src is then not
// read; it must still be a valid address).
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, bool valid) {
    const int n = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(n)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// One pass of at most 16 x 16 frames of pair rows X (nx) and Y (ny): dot
// products on the tensor cores from chunks staged in `ring` (this warp's
// kRingD x 4 x 32 float4), then frame distances into fd (row stride ld),
// returning this lane's largest |d - 1/2|.
template <int NT>
__device__ __forceinline__ float fd_pass(const float *X, int nx, const float *Y, int ny, int dim,
                                         int lane, float4 *ring, const float *ix,
                                         const float *iy, float *fd, int ld) {
    constexpr int NA = 2;
    const int g = lane >> 2, t = lane & 3;
    float acc[NA][NT][4];
#pragma unroll
    for (int q = 0; q < NA; ++q)
#pragma unroll
        for (int n = 0; n < NT; ++n)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[q][n][e] = 0.0f;
    // this thread's rows: x rows g, g + 8; y rows g, g + 8 (NT = 2)
    const float *src[4];
    bool ok[4];
    src[0] = X + (int64_t)g * dim + 4 * t;
    ok[0] = g < nx;
    src[1] = X + (int64_t)(g + 8) * dim + 4 * t;
    ok[1] = g + 8 < nx;
    src[2] = Y + (int64_t)g * dim + 4 * t;
    ok[2] = g < ny;
    src[3] = Y + (int64_t)(g + 8) * dim + 4 * t;
    ok[3] = NT == 2 && g + 8 < ny;
    const int nchunk = (dim + 15) >> 4;
    auto issue = [&](int k) {
        const int c = 16 * k;
        const bool in = c + 4 * t < dim;
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            if (f == 3 && NT == 1) continue;
            const bool v = ok[f] && in;
            cp_async16(smem_addr(ring + ((k % kRingD) * 4 + f) * 32 + lane), v ? src[f] + c : X, v);
        }
    };
#pragma unroll
    for (int k = 0; k < kRingD - 1; ++k) {
        if (k < nchunk) issue(k);
        cp_async_commit();
    }
    for (int k = 0; k < nchunk; ++k) {
        if (k + kRingD - 1 < nchunk) issue(k + kRingD - 1);
        cp_async_commit();
        cp_async_wait<kRingD - 1>();  // chunk k has landed (this thread's copies)
        const float4 *slot = ring + (k % kRingD) * 4 * 32 + lane;
        uint32_t xa[2][4], yb[NT][4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float4 v = slot[h * 32];
            xa[h][0] = tf32(v.x);
            xa[h][1] = tf32(v.y);
            xa[h][2] = tf32(v.z);
            xa[h][3] = tf32(v.w);
        }
#pragma unroll
        for (int n = 0; n < NT; ++n) {
            const float4 v = slot[(2 + n) * 32];
            yb[n][0] = tf32(v.x);
            yb[n][1] = tf32(v.y);
            yb[n][2] = tf32(v.z);
            yb[n][3] = tf32(v.w);
        }
        const int q = k & (NA - 1);
#pragma unroll
        for (int s2 = 0; s2 < 2; ++s2)
#pragma unroll
            for (int n = 0; n < NT; ++n)
                mma_tf32(acc[q][n], xa[0][2 * s2], xa[1][2 * s2], xa[0][2 * s2 + 1],
                         xa[1][2 * s2 + 1], yb[n][2 * s2], yb[n][2 * s2 + 1]);
    }
    cp_async_wait<0>();
    float dev = 0.0f;
#pragma unroll
    for (int n = 0; n < NT; ++n)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int i = g + 8 * (e >> 1), j = 8 * n + 2 * t + (e & 1);
            if (i < nx && j < ny) {
                float v = acc[0][n][e];
#pragma unroll
                for (int q = 1; q < NA; ++q) v += acc[q][n][e];
                const float c = __fmul_rn(__fmul_rn(v, __ldg(ix + i)), __ldg(iy + j));
                const float d = acosf(fminf(1.0f, fmaxf(-1.0f, c))) * 0.318309886183790671f;
                fd[i * ld + j] = d;
                dev = fmaxf(dev, fabsf(d - 0.5f));
            }
        }
    return dev;
}

constexpr size_t kFdSmem = (size_t)kFdWarps * kRingD * 4 * 32 * sizeof(float4);

__global__ void __launch_bounds__(kFdWarps * 32, 3) refine_fd_kernel(RefineArgs a) {
    extern __shared__ float4 ring_all[];  // [kFdWarps][kRingD * 4 * 32]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float4 *ring = ring_all + (size_t)warp * kRingD * 4 * 32;
    const int count = min(*a.count, a.capacity);
    const int64_t stride = (int64_t)gridDim.x * kFdWarps * kRefineGroup;
    for (int64_t q0 = ((int64_t)blockIdx.x * kFdWarps + warp) * kRefineGroup; q0 < count;
         q0 += stride) {
        // offsets for the round's pairs: one atomicAdd for their total size
        int64_t gx = 0, gy = 0, ox = 0, oy = 0;
        int Tx = 0, Ty = 0;
        if (lane < kRefineGroup && q0 + lane < count) {
            const int2 pr = a.list[q0 + lane];
            gx = a.item_id ? a.item_id[pr.x] : pr.x;
            gy = a.item_id ? a.item_id[pr.y] : pr.y;
            ox = a.offsets[gx];
            oy = a.offsets[gy];
            Tx = (int)(a.offsets[gx + 1] - ox);
            Ty = (int)(a.offsets[gy + 1] - oy);
        }
        const int64_t sz = (int64_t)Tx * Ty;
        int64_t incl = sz;
        for (int o = 1; o < kRefineGroup; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int64_t total = __shfl_sync(0xffffffffu, incl, kRefineGroup - 1);
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(a.fd_used, (unsigned long long)total);
        base = __shfl_sync(0xffffffffu, base, 0);
        const int64_t my_off = (int64_t)base + incl - sz;
        const bool fits = (int64_t)base + total <= a.fd_cap;  // the round fits or none of it
        if (lane < kRefineGroup && q0 + lane < count) a.fd_off[q0 + lane] = fits ? my_off : -1;
        if (!fits) continue;
        for (int p = 0; p < kRefineGroup && q0 + p < count; ++p) {
            const int64_t pox = __shfl_sync(0xffffffffu, ox, p), poy = __shfl_sync(0xffffffffu, oy, p);
            const int pTx = __shfl_sync(0xffffffffu, Tx, p), pTy = __shfl_sync(0xffffffffu, Ty, p);
            const int64_t off = __shfl_sync(0xffffffffu, my_off, p);
            const float *X = a.feats + pox * (int64_t)a.dim;
            const float *Y = a.feats + poy * (int64_t)a.dim;
            float *fd = a.fd + off;
            float dev = 0.0f;
            for (int ib = 0; ib < pTx; ib += 16) {
                const int nx = min(16, pTx - ib);
                for (int jb = 0; jb < pTy; jb += 16) {
                    const int ny = min(16, pTy - jb);
                    const float *Xb = X + (int64_t)ib * a.dim, *Yb = Y + (int64_t)jb * a.dim;
                    float *out = fd + ib * pTy + jb;
                    const float *ixb = a.inv_q + pox + ib, *iyb = a.inv_q + poy + jb;
                    const float dv = ny > 8
                        ? fd_pass<2>(Xb, nx, Yb, ny, a.dim, lane, ring, ixb, iyb, out, pTy)
                        : fd_pass<1>(Xb, nx, Yb, ny, a.dim, lane, ring, ixb, iyb, out, pTy);
                    dev = fmaxf(dev, dv);
                }
            }
            for (int o = 16; o; o >>= 1) dev = fmaxf(dev, __shfl_xor_sync(0xffffffffu, dev, o));
            if (lane == 0) a.dev[q0 + p] = dev;
        }
    }
}

// One thread per listed pair: the DP over its distances (rows = x frames,
// previous row in shared memory, laid out [column][thread]), the interval
// with tau from the pair's largest |cos|.
__global__ void __launch_bounds__(kDpThreads) refine_dp_kernel(RefineArgs a) {
    extern __shared__ float rb[];  // [ML][kDpThreads] costs, then [ML][kDpThreads] packed lengths
    const int tid = threadIdx.x;
    uint32_t *rl = reinterpret_cast<uint32_t *>(rb + (size_t)a.max_len * kDpThreads);
    const int count = min(*a.count, a.capacity);
    for (int64_t q = (int64_t)blockIdx.x * kDpThreads + tid; q < count;
         q += (int64_t)gridDim.x * kDpThreads) {
        const int64_t off = a.fd_off[q];
        if (off < 0) {
            a.iv[q] = make_float2(0.0f, 1.0f);
            continue;
        }
        const int2 pr = a.list[q];
        const int64_t gx = a.item_id ? a.item_id[pr.x] : pr.x;
        const int64_t gy = a.item_id ? a.item_id[pr.y] : pr.y;
        const int64_t ox = a.offsets[gx], oy = a.offsets[gy];
        const int Tx = (int)(a.offsets[gx + 1] - ox);
        const int Ty = (int)(a.offsets[gy + 1] - oy);
        const float devq = a.dev[q];
        const DtwBound bd = dtw_bound_dev(Tx, Ty, item_theta(a.theta_frame, ox, Tx),
                                          item_theta(a.theta_frame, oy, Ty), a.eps_c, devq);
        const float *fd = a.fd + off;
        float lc = 0.0f;
        uint32_t ll = 0;
        for (int i = 0; i < Tx; ++i) {
            const float *row = fd + (int64_t)i * Ty;
            float dc = ABX_INF;
            uint32_t dl = 0;
            lc = ABX_INF;
            ll = 0;
            for (int j = 0; j < Ty; ++j) {
                const float dij = row[j];
                const float uc = i > 0 ? rb[j * kDpThreads + tid] : ABX_INF;
                const uint32_t ul = i > 0 ? rl[j * kDpThreads + tid] : 0u;
                float nc;
                uint32_t info;
                if (i == 0 && j == 0) {
                    nc = dij;
                    info = dtw_pack3(1, 1, 1);
                } else {
                    dtw_cell(dij, uc, ul, lc, ll, dc, dl, bd.tau, nc, info);
                }
                dc = uc;
                dl = ul;
                lc = nc;
                ll = info;
                rb[j * kDpThreads + tid] = nc;
                rl[j * kDpThreads + tid] = info;
            }
        }
        const float D = __fdiv_rn(lc, (float)(ll & 0xffu));
        float lo, hi;
        dtw_interval(bd, lc, ll, devq, a.eps_c, 1, D, lo, hi);
        a.iv[q] = make_float2(lo, hi);
    }
}

// Per frame 1 / |tf32(x)| and the rounding angle asin(|tf32(x) - x| / |x|)
// (with slack for its FP32 evaluation); one warp per frame, lanes over the
// dimension.  Runs only if acc[gate] != 0 (acc NULL: always).
template <bool V4>
__device__ __forceinline__ void prep_frame(const RefinePrepArgs &a, int64_t f, int lane) {
    const float *x = a.feats + f * (int64_t)a.dim;
    float qq = 0.0f, dd = 0.0f, xx = 0.0f;
#pragma unroll 8
    for (int c = 4 * lane; c < a.dim; c += 128) {
        const float4 v = load4<V4>(x, 0, 1, c, a.dim);
        const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float qv = __uint_as_float(tf32(e[i]));
            const float d = qv - e[i];  // exact: qv is within 2^-11 |e| of e
            qq = fmaf(qv, qv, qq);
            dd = fmaf(d, d, dd);
            xx = fmaf(e[i], e[i], xx);
        }
    }
    for (int o = 16; o; o >>= 1) {
        qq += __shfl_xor_sync(0xffffffffu, qq, o);
        dd += __shfl_xor_sync(0xffffffffu, dd, o);
        xx += __shfl_xor_sync(0xffffffffu, xx, o);
    }
    if (lane == 0) {
        a.inv_q[f] = __fdiv_rn(1.0f, __fsqrt_rn(qq));
        a.theta_frame[f] =
            xx > 0.0f ? asinf(fminf(1.0f, sqrtf(dd / xx))) * 1.0001f + 1e-7f : 0.0f;
    }
}

// prep_frame for 16-byte aligned rows of at most 128 NV dimensions: the
// row's NV float4 loads per lane are issued before any is used (the loop
// form above waits for each in turn); the sums run in the same order, so
// the results are identical.
template <int NV>
__device__ __forceinline__ void prep_frame_nv(const RefinePrepArgs &a, int64_t f, int lane) {
    const float *x = a.feats + f * (int64_t)a.dim;
    float4 v[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = load4<true>(x, 0, 1, 4 * lane + 128 * k, a.dim);
    float qq = 0.0f, dd = 0.0f, xx = 0.0f;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const float e[4] = {v[k].x, v[k].y, v[k].z, v[k].w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float qv = __uint_as_float(tf32(e[i]));
            const float d = qv - e[i];
            qq = fmaf(qv, qv, qq);
            dd = fmaf(d, d, dd);
            xx = fmaf(e[i], e[i], xx);
        }
    }
    for (int o = 16; o; o >>= 1) {
        qq += __shfl_xor_sync(0xffffffffu, qq, o);
        dd += __shfl_xor_sync(0xffffffffu, dd, o);
        xx += __shfl_xor_sync(0xffffffffu, xx, o);
    }
    if (lane == 0) {
        a.inv_q[f] = __fdiv_rn(1.0f, __fsqrt_rn(qq));
        a.theta_frame[f] =
            xx > 0.0f ? asinf(fminf(1.0f, sqrtf(dd / xx))) * 1.0001f + 1e-7f : 0.0f;
    }
}

// NV = 0: the loop form (any dimension); NV >= 1: 16-byte aligned rows of at
// most 128 NV dimensions.
template <bool V4, int NV = 0>
__global__ void __launch_bounds__(256) refine_prep_kernel(RefinePrepArgs a) {
    if (a.acc && a.acc[a.gate] == 0) return;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t f = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; f < a.n_frames;
         f += nwarps) {
        if constexpr (NV > 0)
            prep_frame_nv<NV>(a, f, lane);
        else
            prep_frame<V4>(a, f, lane);
    }
}

template <bool V4>
cudaError_t launch_refine_v(const RefineArgs &a, int32_t capacity, cudaStream_t s) {
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const size_t ml = (size_t)a.max_len;
    // pairs per round and warps per block from the shared memory they take:
    // up to 4 pairs within 24 KB per warp, up to 8 warps within 110 KB
    const size_t per_pair = (ml * ml + 2 * ml) * sizeof(float);
    RefineArgs b = a;
    b.group = (int)std::max<size_t>(1, std::min<size_t>(kRefineGroup, (24u << 10) / per_pair));
    const size_t per_warp = per_pair * b.group;
    const int warps = (int)std::max<size_t>(1, std::min<size_t>(kRefineMaxWarps,
                                                                (110u << 10) / per_warp));
    const size_t smem = per_warp * warps;
    cudaError_t e = cudaFuncSetAttribute(refine_dtw_kernel<V4>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) {
        cudaGetLastError();  // leave no error behind for later launches
        return e;
    }
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, refine_dtw_kernel<V4>, warps * 32,
                                                      smem);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e;
    }
    const int64_t need = ((int64_t)capacity + warps * b.group - 1) / (warps * b.group);
    const int64_t full = (int64_t)nsm * std::max(per_sm, 1);
    const int blocks = (int)std::min(need, full);
    ProfScope ps_("recheck_refine", s);
    refine_dtw_kernel<V4><<<blocks, warps * 32, smem, s>>>(b);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_refine_prep(const RefinePrepArgs &a, cudaStream_t s) {
    if (a.n_items <= 0 || a.n_frames <= 0) return cudaSuccess;
    const bool v4 = (a.dim & 3) == 0 && (reinterpret_cast<uintptr_t>(a.feats) & 15) == 0;
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    // grid-stride over frames: a gated launch with nothing to do ends at once
    const int64_t blocks = std::min<int64_t>((a.n_frames + 7) / 8, (int64_t)nsm * 8);
    ProfScope ps_("recheck_refine_prep", s);
    const int nv = v4 ? (a.dim + 127) / 128 : 0;
    switch (nv > 8 ? 0 : nv) {
#define PREP_CASE(v) \
    case v: refine_prep_kernel<true, v><<<(unsigned)blocks, 256, 0, s>>>(a); break;
        PREP_CASE(1) PREP_CASE(2) PREP_CASE(3) PREP_CASE(4)
        PREP_CASE(5) PREP_CASE(6) PREP_CASE(7) PREP_CASE(8)
#undef PREP_CASE
    default:
        if (v4)
            refine_prep_kernel<true><<<(unsigned)blocks, 256, 0, s>>>(a);
        else
            refine_prep_kernel<false><<<(unsigned)blocks, 256, 0, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_refine(const RefineArgs &a, int32_t capacity, cudaStream_t s) {
    if (capacity <= 0) return cudaSuccess;
    const bool v4 = (a.dim & 3) == 0 && (reinterpret_cast<uintptr_t>(a.feats) & 15) == 0;
    if (!v4 || !a.fd) return v4 ? launch_refine_v<true>(a, capacity, s)
                                : launch_refine_v<false>(a, capacity, s);
    // two kernels: distances (cp.async-staged features), then the DPs
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaMemsetAsync(a.fd_used, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    {
        e = cudaFuncSetAttribute(refine_fd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kFdSmem);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e;
        }
        const int64_t need = ((int64_t)capacity + kFdWarps * kRefineGroup - 1) /
                             (kFdWarps * kRefineGroup);
        const int blocks = (int)std::min<int64_t>(need, (int64_t)nsm * 3);
        ProfScope ps_("recheck_refine", s);
        refine_fd_kernel<<<blocks, kFdWarps * 32, kFdSmem, s>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const size_t smem = (size_t)a.max_len * kDpThreads * 8;
    e = cudaFuncSetAttribute(refine_dp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e;
    }
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, refine_dp_kernel, kDpThreads, smem);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e;
    }
    const int64_t need = ((int64_t)capacity + kDpThreads - 1) / kDpThreads;
    const int blocks = (int)std::min<int64_t>(need, (int64_t)nsm * std::max(per_sm, 1));
    ProfScope ps_("recheck_refine_dp", s);
    refine_dp_kernel<<<blocks, kDpThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace abx

using namespace abx;

#define CU(call)                                                                   \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),      \
                      __FILE__, __LINE__);                                         \
            return e_ == cudaErrorMemoryAllocation ? ABX_E_OOM : ABX_E_CUDA;       \
        }                                                                          \
    } while (0)

#define REQUIRE(cond, code, ...)      \
    do {                              \
        if (!(cond)) {                \
            set_error(__VA_ARGS__);   \
            return (code);            \
        }                             \
    } while (0)

extern "C" {

int abx_refine_pairs(abx_ctx *ctx_, const abx_items *items_, int64_t n, const int64_t *x,
                     const int64_t *y, float *lo, float *hi, void *stream) {
    Ctx *ctx = reinterpret_cast<Ctx *>(ctx_);
    const Items *it = reinterpret_cast<const Items *>(items_);
    REQUIRE(ctx && it && (n == 0 || (x && y && lo && hi)), ABX_E_INVALID, "NULL argument");
    REQUIRE(it->ctx == ctx, ABX_E_STATE, "items belong to another context");
    REQUIRE(n >= 0 && n < (1LL << 31), ABX_E_INVALID, "bad pair count %lld", (long long)n);
    REQUIRE(it->max_len <= kMaxItemLen, ABX_E_UNSUPPORTED, "item longer than %d frames",
            kMaxItemLen);
    if (n == 0) return ABX_OK;
    std::vector<int2> h(n);
    for (int64_t q = 0; q < n; ++q) {
        REQUIRE(x[q] >= 0 && x[q] < it->n_items && y[q] >= 0 && y[q] < it->n_items,
                ABX_E_INVALID, "pair %lld out of range", (long long)q);
        h[q] = make_int2((int)x[q], (int)y[q]);
    }
    CU(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    CU(cudaStreamWaitEvent(s, it->ready, 0));
    int2 *d_list = nullptr;
    float2 *d_iv = nullptr;
    int32_t *d_count = nullptr;
    float *d_invq = nullptr, *d_theta = nullptr;
    CU(cudaMallocAsync((void **)&d_invq, std::max<int64_t>(it->n_frames, 1) * sizeof(float), s));
    CU(cudaMallocAsync((void **)&d_theta, std::max<int64_t>(it->n_frames, 1) * sizeof(float), s));
    RefinePrepArgs pa;
    pa.feats = it->d_feats;
    pa.offsets = it->d_offsets;
    pa.n_items = it->n_items;
    pa.n_frames = it->n_frames;
    pa.dim = it->dim;
    pa.inv_q = d_invq;
    pa.theta_frame = d_theta;
    pa.acc = nullptr;
    pa.gate = 0;
    CU(launch_refine_prep(pa, s));
    CU(cudaMallocAsync((void **)&d_list, n * sizeof(int2), s));
    CU(cudaMallocAsync((void **)&d_iv, n * sizeof(float2), s));
    CU(cudaMallocAsync((void **)&d_count, sizeof(int32_t), s));
    const int32_t cnt = (int32_t)n;
    CU(cudaMemcpyAsync(d_list, h.data(), n * sizeof(int2), cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(d_count, &cnt, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    const int64_t ml = it->max_len;
    const int64_t fd_cap = std::min<int64_t>(1LL << 28, n * ml * ml);
    float *d_fd = nullptr, *d_dev = nullptr;
    int64_t *d_fdoff = nullptr;
    unsigned long long *d_used = nullptr;
    CU(cudaMallocAsync((void **)&d_fd, fd_cap * sizeof(float), s));
    CU(cudaMallocAsync((void **)&d_fdoff, n * sizeof(int64_t), s));
    CU(cudaMallocAsync((void **)&d_dev, n * sizeof(float), s));
    CU(cudaMallocAsync((void **)&d_used, sizeof(unsigned long long), s));
    RefineArgs a;
    memset(&a, 0, sizeof(a));
    a.fd = d_fd;
    a.fd_cap = fd_cap;
    a.fd_off = d_fdoff;
    a.dev = d_dev;
    a.fd_used = d_used;
    a.feats = it->d_feats;
    a.offsets = it->d_offsets;
    a.item_id = nullptr;
    a.dim = it->dim;
    a.max_len = it->max_len;
    a.list = d_list;
    a.count = d_count;
    a.capacity = cnt;
    a.iv = d_iv;
    a.inv_q = d_invq;
    a.theta_frame = d_theta;
    a.eps_c = refine_cosine_bound(it->dim);
    CU(launch_refine(a, cnt, s));
    std::vector<float2> o(n);
    CU(cudaMemcpyAsync(o.data(), d_iv, n * sizeof(float2), cudaMemcpyDeviceToHost, s));
    cudaFreeAsync(d_list, s);
    cudaFreeAsync(d_iv, s);
    cudaFreeAsync(d_count, s);
    cudaFreeAsync(d_invq, s);
    cudaFreeAsync(d_theta, s);
    for (void *p : {(void *)d_fd, (void *)d_fdoff, (void *)d_dev, (void *)d_used})
        cudaFreeAsync(p, s);
    CU(cudaStreamSynchronize(s));
    for (int64_t q = 0; q < n; ++q) {
        lo[q] = o[q].x;
        hi[q] = o[q].y;
    }
    return ABX_OK;
}

}  // extern "C"
