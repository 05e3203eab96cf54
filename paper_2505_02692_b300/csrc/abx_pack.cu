// Pack kernel: gathers the frames of a task into group order, L2-normalises
// them, stores them in the kernel precision, and records per stored vector
// its inverse norm and a bound on its angle to the exact frame.
//
// The angular distance (fastabx Sec. 3.1) only depends on frame directions,
// so the distance kernels work on normalised frames; the stored vector q of a
// frame x is used through cos(q_i, q_j) = <q_i, q_j> / (|q_i| |q_j|), which
// keeps any per-item scale out of the cosine.  theta = angle(q, x) bounds the
// effect of the storage precision on every frame distance (the angular
// distance is a metric on the sphere, so |d(q_i,q_j) - d(x_i,x_j)| <=
// (theta_i + theta_j) / pi).
//
// Mean-pooled mode (Sec. 3.2, "pool along the time domain") first averages
// the raw frames of each item and packs the mean as a one-frame item.  The
// sum over frames runs in double-word arithmetic on the FP32 pipe (FP64 is
// scarce on this GPU): each frame value is added to a float pair with the
// double-word-plus-float addition of Joldes, Muller and Popescu (ACM TOMS
// 2017, "DWPlusFP", relative error at most 2u^2, u = 2^-24), then the pair is
// divided by T with one correction step, which leaves the FP32 mean within
// one unit in the last place of the exact mean (its angle to the exact mean
// is below 2^-23, covered by the slack of the distance intervals).
#include <algorithm>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include "abx_internal.h"

namespace abx {
namespace {

__device__ __forceinline__ float warp_sum(float v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
    for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Stored value of component xh (already normalised) and its float value.
// FP32: x itself.  FP32 split: v = x * scale (a power of two, see
// split_scale), hi = fp16(v), lo = fp16(v - hi), value hi + lo in scaled
// units.  Halves below FP16's normal range (2^-14) are stored as zero, so the
// stored vector is exactly what the tensor cores read whether or not they
// flush FP16 subnormals; the angle theta of the stored vector covers the
// dropped part.  BF16: bf16(x).  FP8: e4m3(x * scale) (value in scaled units).
constexpr float kHalfMinNormal = 6.103515625e-05f;  // 2^-14

__device__ __forceinline__ __half half_or_zero(float v) {
    const __half h = __float2half_rn(v);
    return fabsf(__half2float(h)) < kHalfMinNormal ? __float2half_rn(0.0f) : h;
}

struct Quant {
    int precision;
    float scale;
    __device__ __forceinline__ float value(float xh, __half *hi, __half *lo, __nv_bfloat16 *b16,
                                           __nv_fp8_e4m3 *q8) const {
        if (precision == ABX_FP32_SIMT) return xh;
        if (precision == ABX_FP32) {
            const float v = xh * scale;
            *hi = half_or_zero(v);
            const float h = __half2float(*hi);
            *lo = half_or_zero(v - h);
            return h + __half2float(*lo);
        }
        if (precision == ABX_BF16) {
            *b16 = __float2bfloat16_rn(xh);
            return __bfloat162float(*b16);
        }
        *q8 = __nv_fp8_e4m3(xh * scale);
        return float(*q8);
    }
};

// Power-of-two scale of the FP32 split for a vector whose largest |component|
// is mx: the largest component lands in [2^13, 2^14), far below FP16's
// largest finite value 65504, and the lo halves of all but tiny components
// stay normal.  Unit vectors (angular, cosine) use 2^14 directly.
constexpr float kSplitUnitScale = 16384.0f;  // 2^14
__device__ __forceinline__ float split_scale(float mx) {
    if (!(mx > 0.0f)) return 1.0f;
    int e;
    frexpf(mx, &e);  // mx = m 2^e, m in [0.5, 1)
    return ldexpf(1.0f, 14 - e);
}

// Row -> (source row, sorted item) map, one thread per sorted item.
__global__ void expand_rows(const int32_t *len, const int32_t *row, const int64_t *src_row,
                            int32_t n_items, int64_t *row_src, int32_t *row_item) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_items) return;
    const int T = len[k];
    const int64_t r0 = row[k], s0 = src_row[k];
    for (int t = 0; t < T; ++t) {
        row_src[r0 + t] = s0 + t;
        row_item[r0 + t] = (int32_t)k;
    }
}

// FP8 scale per item: 448 / the largest normalised component of its frames
// (raw component for the Euclidean distance).  One warp per packed row, with
// the loads and the norm of pack_rows_kernel, so the maximum is that of the
// values the pack then scales; a row's maximum goes to its item by an atomic
// max on the float's bits (non-negative floats order like their bit
// patterns).
template <int V>
__global__ void __launch_bounds__(256) row_max_kernel(PackArgs a, const float *src,
                                                      const int64_t *row_src,
                                                      const int32_t *row_item) {
    const int lane = threadIdx.x & 31;
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= a.n_rows) return;
    const int dim = a.dim;
    const float *x = src + row_src[r] * (int64_t)dim;
    const bool vec = (dim & 3) == 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0;
    float ss = 0.0f, mx = 0.0f;
#pragma unroll
    for (int i = 0; i < V; ++i) {
        const int c = (i * 32 + lane) * 4;
        float v[4];
        if (vec && c + 3 < dim) {
            const float4 f = __ldg(reinterpret_cast<const float4 *>(x + c));
            v[0] = f.x;
            v[1] = f.y;
            v[2] = f.z;
            v[3] = f.w;
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) v[e] = c + e < dim ? __ldg(x + c + e) : 0.0f;
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            ss = fmaf(v[e], v[e], ss);
            mx = fmaxf(mx, fabsf(v[e]));
        }
    }
    ss = warp_sum(ss);
    mx = warp_max(mx);
    const float inv = ss > 0.0f ? 1.0f / sqrtf(ss) : 0.0f;
    const float m = a.distance == ABX_DIST_EUCLIDEAN ? mx : mx * inv;
    if (lane == 0 && m > 0.0f)
        atomicMax(reinterpret_cast<int *>(a.item_scale) + row_item[r], __float_as_int(m));
}

// Item maximum -> FP8 scale 448 / max (1 for an all-zero item).
__global__ void item_scale_finish(float *item_scale, int32_t n) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float m = item_scale[k];
    item_scale[k] = m > 0.0f ? 448.0f / m : 1.0f;
}

__device__ __forceinline__ void store4(const PackArgs &a, int64_t r, int c, const float *q,
                                       const __half *hi, const __half *lo,
                                       const __nv_bfloat16 *b16, const __nv_fp8_e4m3 *q8) {
    const int dp = a.dim_pad;
    if (a.precision == ABX_FP32_SIMT) {
        *reinterpret_cast<float4 *>(reinterpret_cast<float *>(a.packed) + r * dp + c) =
            make_float4(q[0], q[1], q[2], q[3]);
    } else if (a.precision == ABX_FP32) {
        __half *P = reinterpret_cast<__half *>(a.packed) + r * 2 * dp;
        __half2 h01 = {hi[0], hi[1]}, h23 = {hi[2], hi[3]};
        __half2 l01 = {lo[0], lo[1]}, l23 = {lo[2], lo[3]};
        uint2 hv, lv;
        hv.x = *reinterpret_cast<uint32_t *>(&h01);
        hv.y = *reinterpret_cast<uint32_t *>(&h23);
        lv.x = *reinterpret_cast<uint32_t *>(&l01);
        lv.y = *reinterpret_cast<uint32_t *>(&l23);
        *reinterpret_cast<uint2 *>(P + c) = hv;
        *reinterpret_cast<uint2 *>(P + dp + c) = lv;
    } else if (a.precision == ABX_BF16) {
        __nv_bfloat16 *P = reinterpret_cast<__nv_bfloat16 *>(a.packed) + r * dp;
        __nv_bfloat162 h01 = {b16[0], b16[1]}, h23 = {b16[2], b16[3]};
        uint2 hv;
        hv.x = *reinterpret_cast<uint32_t *>(&h01);
        hv.y = *reinterpret_cast<uint32_t *>(&h23);
        *reinterpret_cast<uint2 *>(P + c) = hv;
    } else {
        uint32_t w = 0;
        for (int e = 0; e < 4; ++e)
            w |= (uint32_t)(*reinterpret_cast<const uint8_t *>(&q8[e])) << (8 * e);
        *reinterpret_cast<uint32_t *>(reinterpret_cast<uint8_t *>(a.packed) + r * dp + c) = w;
    }
}

// One warp per packed row; the frame stays in registers (V float4 per lane,
// dim_pad = 128 V), so the raw features are read once.  Four blocks per SM
// (64 registers, a few bytes spilled at V = 6) moved more bytes than three
// (80 registers): 0.95 -> 0.88 ms FP32 split, 0.80 -> 0.71 ms BF16 for 2.5 GB.
template <int V>
__global__ void __launch_bounds__(256, 4) pack_rows_kernel(PackArgs a, const float *src,
                                                        const int64_t *row_src,
                                                        const int32_t *row_item) {
    const int lane = threadIdx.x & 31;
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= a.n_rows) return;
    const int dim = a.dim;
    const int k = row_item[r];
    const float *x = src + row_src[r] * (int64_t)dim;
    const bool vec = (dim & 3) == 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0;
    float v[4 * V];
#pragma unroll
    for (int i = 0; i < V; ++i) {
        const int c = (i * 32 + lane) * 4;
        if (vec && c + 3 < dim) {
            const float4 f = __ldg(reinterpret_cast<const float4 *>(x + c));
            v[4 * i] = f.x;
            v[4 * i + 1] = f.y;
            v[4 * i + 2] = f.z;
            v[4 * i + 3] = f.w;
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) v[4 * i + e] = c + e < dim ? __ldg(x + c + e) : 0.0f;
        }
    }
    const bool euclid = a.distance == ABX_DIST_EUCLIDEAN;
    float ss = 0.0f;
#pragma unroll
    for (int i = 0; i < 4 * V; ++i) ss = fmaf(v[i], v[i], ss);
    ss = warp_sum(ss);
    if (!euclid && ss == 0.0f && lane == 0) atomicOr(a.err, kPackZeroNorm);
    // angular / cosine work on x / |x|; Euclidean on the raw frame
    const float inv = euclid ? 1.0f : (ss > 0.0f ? 1.0f / sqrtf(ss) : 0.0f);
    float scale = 1.0f;
    if (a.precision == ABX_FP8) {
        scale = a.item_scale[k];
    } else if (a.precision == ABX_FP32) {
        if (euclid) {  // raw frame: its own power-of-two scale
            float mx = 0.0f;
#pragma unroll
            for (int i = 0; i < 4 * V; ++i) mx = fmaxf(mx, fabsf(v[i]));
            scale = split_scale(warp_max(mx));
        } else {
            scale = kSplitUnitScale;
        }
    }
    Quant qz{a.precision, scale};
    float q[4 * V];
    float qq = 0.0f;
#pragma unroll
    for (int i = 0; i < V; ++i) {
        __half hi[4], lo[4];
        __nv_bfloat16 b16[4];
        __nv_fp8_e4m3 q8[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            v[4 * i + e] *= inv;
            q[4 * i + e] = qz.value(v[4 * i + e], &hi[e], &lo[e], &b16[e], &q8[e]);
            qq = fmaf(q[4 * i + e], q[4 * i + e], qq);
        }
        store4(a, r, (i * 32 + lane) * 4, &q[4 * i], hi, lo, b16, q8);
    }
    qq = warp_sum(qq);
    if (euclid) {
        // stored q = x * scale: the raw value is q / scale, |raw|^2 = qq / scale^2
        const float back = 1.0f / qz.scale;
        if (lane == 0) {
            a.inv_norm[r] = back;
            a.nrm2[r] = qq * back * back;
            a.theta[r] = 0.0f;
        }
        return;
    }
    const float invq = qq > 0.0f ? 1.0f / sqrtf(qq) : 0.0f;
    // |q/|q| - x/|x||^2 = (2 sin(theta/2))^2
    float rr = 0.0f;
#pragma unroll
    for (int i = 0; i < 4 * V; ++i) {
        const float dl = q[i] * invq - v[i];
        rr = fmaf(dl, dl, rr);
    }
    rr = warp_sum(rr);
    // slack 4.8e-7 rad covers the FP32 evaluation of rr and the rounding of
    // x/|x| itself (one rounding per component, at most 2^-24 rad)
    const float th = 2.0f * asinf(fminf(1.0f, 0.5f * sqrtf(rr))) * 1.0001f + 4.8e-7f;
    if (lane == 0) {
        a.inv_norm[r] = invq;
        a.theta[r] = th;
        atomicMax(reinterpret_cast<int *>(a.theta_item) + k, __float_as_int(th));
    }
}

// One warp per sorted item; rows of the item processed one after another
// (any dim; used when dim_pad exceeds the register-resident variants).
__global__ void __launch_bounds__(256) pack_kernel(PackArgs a, const float *src,
                                                   const int64_t *src_row) {
    const int lane = threadIdx.x & 31;
    const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (k >= a.n_items) return;
    const int T = a.len[k];
    const int64_t r0 = a.row[k];
    const float *X = src + src_row[k] * (int64_t)a.dim;
    const int dim = a.dim, dp = a.dim_pad;

    Quant qz{a.precision, 1.0f};
    if (a.precision == ABX_FP8) {
        // one scale per item: map the largest normalised component to 448
        float m = 0.0f;
        for (int t = 0; t < T; ++t) {
            const float *x = X + (int64_t)t * dim;
            float ss = 0.0f, mx = 0.0f;
            for (int c = lane; c < dim; c += 32) {
                float v = x[c];
                ss = fmaf(v, v, ss);
                mx = fmaxf(mx, fabsf(v));
            }
            ss = warp_sum(ss);
            mx = warp_max(mx);
            if (ss > 0.0f) m = fmaxf(m, mx / sqrtf(ss));
        }
        qz.scale = m > 0.0f ? 448.0f / m : 1.0f;
        if (lane == 0) a.item_scale[k] = qz.scale;
    }

    float th_item = 0.0f;
    for (int t = 0; t < T; ++t) {
        const float *x = X + (int64_t)t * dim;
        const int64_t r = r0 + t;
        float ss = 0.0f, mx = 0.0f;
        for (int c = lane; c < dim; c += 32) {
            ss = fmaf(x[c], x[c], ss);
            mx = fmaxf(mx, fabsf(x[c]));
        }
        ss = warp_sum(ss);
        mx = warp_max(mx);
        const bool euclid = a.distance == ABX_DIST_EUCLIDEAN;
        if (!euclid && ss == 0.0f && lane == 0) atomicOr(a.err, kPackZeroNorm);
        const float inv = euclid ? 1.0f : (ss > 0.0f ? 1.0f / sqrtf(ss) : 0.0f);
        if (a.precision == ABX_FP32) qz.scale = euclid ? split_scale(mx) : kSplitUnitScale;
        // store and accumulate |q|^2
        float qq = 0.0f;
        for (int c = lane; c < dp; c += 32) {
            float xh = c < dim ? x[c] * inv : 0.0f;
            __half hi, lo;
            __nv_bfloat16 b16;
            __nv_fp8_e4m3 q8;
            float q = qz.value(xh, &hi, &lo, &b16, &q8);
            qq = fmaf(q, q, qq);
            if (a.precision == ABX_FP32_SIMT)
                reinterpret_cast<float *>(a.packed)[r * dp + c] = q;
            else if (a.precision == ABX_FP32) {
                __half *P = reinterpret_cast<__half *>(a.packed) + r * 2 * dp;
                P[c] = hi;
                P[dp + c] = lo;
            } else if (a.precision == ABX_BF16)
                reinterpret_cast<__nv_bfloat16 *>(a.packed)[r * dp + c] = b16;
            else
                reinterpret_cast<__nv_fp8_e4m3 *>(a.packed)[r * dp + c] = q8;
        }
        qq = warp_sum(qq);
        if (euclid) {
            const float back = 1.0f / qz.scale;
            if (lane == 0) {
                a.inv_norm[r] = back;
                a.nrm2[r] = qq * back * back;
                a.theta[r] = 0.0f;
            }
            continue;
        }
        const float invq = qq > 0.0f ? 1.0f / sqrtf(qq) : 0.0f;
        // |q/|q| - x/|x||^2 = (2 sin(theta/2))^2
        float rr = 0.0f;
        for (int c = lane; c < dim; c += 32) {
            float xh = x[c] * inv;
            __half hi, lo;
            __nv_bfloat16 b16;
            __nv_fp8_e4m3 q8;
            float q = qz.value(xh, &hi, &lo, &b16, &q8);
            float dlt = q * invq - xh;
            rr = fmaf(dlt, dlt, rr);
        }
        rr = warp_sum(rr);
        // slack 2^-21 rad covers the FP32 evaluation of rr and the rounding
        // of x/|x| itself (one rounding per component, at most 2^-24 rad)
        float th = 2.0f * asinf(fminf(1.0f, 0.5f * sqrtf(rr))) * 1.0001f + 4.8e-7f;
        th_item = fmaxf(th_item, th);
        if (lane == 0) {
            a.inv_norm[r] = invq;
            a.theta[r] = th;
        }
    }
    if (lane == 0) a.theta_item[k] = th_item;
}

// Mean of the raw frames of each item, accumulated in FP64 and rounded once
// to FP32 (so the mean's direction is exact to one rounding per component).
// Double-word running sum h + l of one component: two-sum of h and x, then
// fast two-sum renormalisation with l; the mean (h + l) / T with one
// correction by the exact FMA remainder.
struct PoolSum {
    float h = 0.0f, l = 0.0f;
    __device__ __forceinline__ void add(float x) {
        const float s = __fadd_rn(h, x);
        const float bb = __fsub_rn(s, h);
        const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(x, bb));
        const float v = __fadd_rn(l, err);
        h = __fadd_rn(s, v);
        l = __fsub_rn(v, __fsub_rn(h, s));
    }
    __device__ __forceinline__ float mean(float T) const {
        const float q = __fdiv_rn(h, T);
        const float r = __fadd_rn(__fmaf_rn(-q, T, h), l);
        return __fadd_rn(q, __fdiv_rn(r, T));
    }
};

// One block per item, four components per thread (dim a multiple of 4,
// 16-byte aligned rows): the item's frames are read as whole rows, in frame
// order, so each component is summed exactly as pool_kernel sums it.
__global__ void __launch_bounds__(256) pool_rows_kernel(const float *feats,
                                                        const int64_t *offsets,
                                                        const int32_t *item_id, int32_t dim,
                                                        float *out) {
    const int64_t k = blockIdx.x;
    const int64_t id = item_id[k];
    const int64_t b = offsets[id], e = offsets[id + 1];
    const float T = (float)(e - b);
    for (int c = threadIdx.x * 4; c < dim; c += blockDim.x * 4) {
        PoolSum acc[4];
        for (int64_t t = b; t < e; ++t) {
            const float4 x = __ldg(reinterpret_cast<const float4 *>(feats + t * dim + c));
            acc[0].add(x.x);
            acc[1].add(x.y);
            acc[2].add(x.z);
            acc[3].add(x.w);
        }
        *reinterpret_cast<float4 *>(out + k * dim + c) =
            make_float4(acc[0].mean(T), acc[1].mean(T), acc[2].mean(T), acc[3].mean(T));
    }
}

__global__ void pool_kernel(const float *feats, const int64_t *offsets, const int32_t *item_id,
                            int32_t n_items, int32_t dim, float *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n_items * dim) return;
    const int64_t k = i / dim;
    const int c = (int)(i - k * dim);
    const int64_t id = item_id[k];
    const int64_t b = offsets[id], e = offsets[id + 1];
    PoolSum acc;
    for (int64_t t = b; t < e; ++t) acc.add(__ldg(feats + t * dim + c));
    out[k * dim + c] = acc.mean((float)(e - b));
}

__global__ void identity_rows(const int64_t *offsets, const int32_t *item_id, int32_t n,
                              int32_t mean_mode, int64_t *src_row) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    src_row[k] = mean_mode ? k : offsets[item_id[k]];
}

// Symmetrised KL: each frame read as a distribution p = x / sum(x) (every
// component must be > 0, else the kPackNonPositive flag), stored as the
// vector [p | ln p] of dim_pad elements (each half dim_pad / 2, zero-padded)
// in the FP32 split layout (FP16 hi, then FP16 lo = fp16(v - hi)), with
// h = sum p ln p per row in nrm2.  One warp per sorted item.  The halves are
// scaled by powers of two, p by 2^14 and ln p by 2^8 (|ln p| < 104 for any
// positive FP32), the same for every row, so the contraction of
// [p_i | ln p_i] with [ln p_j | p_j] is 2^22 times the unscaled one and the
// per-row factor 2^-11 (inv_norm) undoes it exactly.
__global__ void __launch_bounds__(256) pack_kl_kernel(PackArgs a, const float *src,
                                                       const int64_t *src_row) {
    const int lane = threadIdx.x & 31;
    const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (k >= a.n_items) return;
    const int T = a.len[k];
    const int half = a.dim_pad / 2;
    const float sp = 16384.0f, sl = 256.0f;  // 2^14, 2^8
    __half *P = reinterpret_cast<__half *>(a.packed);
    if (lane == 0) a.theta_item[k] = 0.0f;
    for (int t = 0; t < T; ++t) {
        const int64_t r = (int64_t)a.row[k] + t;
        const float *x = src + (src_row[k] + t) * (int64_t)a.dim;
        float sum = 0.0f;
        bool bad = false;
        for (int c = lane; c < a.dim; c += 32) {
            const float v = __ldg(x + c);
            sum += v;
            bad |= !(v > 0.0f);
        }
        sum = warp_sum(sum);
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.err, kPackNonPositive);
        const float inv = sum > 0.0f ? 1.0f / sum : 0.0f;
        float h = 0.0f;
        __half *row = P + r * 2 * (int64_t)a.dim_pad;
        for (int c = lane; c < half; c += 32) {
            float pv = 0.0f, lv = 0.0f;
            if (c < a.dim) {
                pv = __ldg(x + c) * inv;
                lv = pv > 0.0f ? logf(pv) : 0.0f;
                h = fmaf(pv, lv, h);
            }
            const float ps = pv * sp, ls = lv * sl;
            const __half ph = half_or_zero(ps), lh = half_or_zero(ls);
            row[c] = ph;
            row[half + c] = lh;
            row[a.dim_pad + c] = half_or_zero(ps - __half2float(ph));
            row[a.dim_pad + half + c] = half_or_zero(ls - __half2float(lh));
        }
        h = warp_sum(h);
        if (lane == 0) {
            a.nrm2[r] = h;
            a.inv_norm[r] = 4.8828125e-4f;  // 2^-11
            a.theta[r] = 0.0f;
        }
    }
}

}  // namespace

cudaError_t launch_pack(const PackArgs &a, cudaStream_t s) {
    const int32_t n = a.n_items;
    int64_t *src_row = nullptr, *row_src = nullptr;
    int32_t *row_item = nullptr;
    float *pooled = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&src_row, sizeof(int64_t) * (size_t)n, s);
    if (e != cudaSuccess) return e;
    {
        ProfScope ps_("pack_rows", s);
        identity_rows<<<(n + 255) / 256, 256, 0, s>>>(a.offsets, a.item_id, n, a.mode == ABX_MEAN,
                                                       src_row);
    }
    const float *src = a.feats;
    if (a.mode == ABX_MEAN) {
        e = cudaMallocAsync((void **)&pooled, sizeof(float) * (size_t)n * a.dim, s);
        if (e != cudaSuccess) return e;
        int64_t tot = (int64_t)n * a.dim;
        {
            ProfScope ps_("pool_mean", s);
            if ((a.dim & 3) == 0 && (reinterpret_cast<uintptr_t>(a.feats) & 15) == 0) {
                const int threads = std::min(256, ((a.dim / 4 + 31) / 32) * 32);
                pool_rows_kernel<<<(unsigned)n, threads, 0, s>>>(a.feats, a.offsets, a.item_id,
                                                                 a.dim, pooled);
            } else {
                pool_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(a.feats, a.offsets,
                                                                           a.item_id, n, a.dim,
                                                                           pooled);
            }
        }
        src = pooled;
    }
    const unsigned item_blocks = (unsigned)(((int64_t)n * 32 + 255) / 256);
    const int V = a.dim_pad / 128;
    if (a.distance == ABX_DIST_KL) {
        ProfScope ps_("pack", s);
        pack_kl_kernel<<<item_blocks, 256, 0, s>>>(a, src, src_row);
    } else if (V >= 1 && V <= 8) {
        e = cudaMallocAsync((void **)&row_src, sizeof(int64_t) * (size_t)std::max<int64_t>(a.n_rows, 1), s);
        if (e == cudaSuccess)
            e = cudaMallocAsync((void **)&row_item, sizeof(int32_t) * (size_t)std::max<int64_t>(a.n_rows, 1), s);
        if (e != cudaSuccess) return e;
        cudaMemsetAsync(a.theta_item, 0, sizeof(float) * (size_t)n, s);
        {
            ProfScope ps_("pack_expand", s);
            expand_rows<<<(n + 255) / 256, 256, 0, s>>>(a.len, a.row, src_row, n, row_src, row_item);
        }
        const unsigned blocks = (unsigned)((a.n_rows * 32 + 255) / 256);
        if (a.precision == ABX_FP8) {
            // row-parallel, vectorised like the pack (a warp per item read its
            // frames one after another with scalar loads: 0.67 ms for 2.5 GB)
            cudaMemsetAsync(a.item_scale, 0, sizeof(float) * (size_t)n, s);
            ProfScope ps_("pack_scale", s);
            switch (V) {
#define MAX_CASE(v) \
    case v: row_max_kernel<v><<<blocks, 256, 0, s>>>(a, src, row_src, row_item); break;
                MAX_CASE(1) MAX_CASE(2) MAX_CASE(3) MAX_CASE(4)
                MAX_CASE(5) MAX_CASE(6) MAX_CASE(7) MAX_CASE(8)
#undef MAX_CASE
            }
            item_scale_finish<<<(n + 255) / 256, 256, 0, s>>>(a.item_scale, n);
        }
        ProfScope ps_("pack", s);
        switch (V) {
#define PACK_CASE(v) \
    case v: pack_rows_kernel<v><<<blocks, 256, 0, s>>>(a, src, row_src, row_item); break;
            PACK_CASE(1) PACK_CASE(2) PACK_CASE(3) PACK_CASE(4)
            PACK_CASE(5) PACK_CASE(6) PACK_CASE(7) PACK_CASE(8)
#undef PACK_CASE
        }
    } else {
        ProfScope ps_("pack", s);
        pack_kernel<<<item_blocks, 256, 0, s>>>(a, src, src_row);
    }
    e = cudaGetLastError();
    cudaFreeAsync(src_row, s);
    if (row_src) cudaFreeAsync(row_src, s);
    if (row_item) cudaFreeAsync(row_item, s);
    if (pooled) cudaFreeAsync(pooled, s);
    return e;
}

}  // namespace abx
