// abx_dtw_pairs_noalloc: DTW distances for an explicit list of item pairs,
// for callers that cannot allocate device memory -- for example code that
// runs under a memory pool it does not own, inside a strict real-time
// serving loop where an allocation could stall, or in an embedding
// application that has handed all device memory to its own allocator.
//
// It is a variant of the DTW kernel: instead of reading frame distances from
// a tile buffer that abx_distances allocates, it computes each pair's
// frame-distance block into a fixed scratch array that lives in this file as
// a static __device__ object, then runs the same dynamic programme (minimum
// over the steps (i-1,j), (i,j-1), (i-1,j-1), shorter path on equal cost,
// cost divided by the optimal path length).  The library allocates nothing:
// no cudaMalloc / cudaFree / pinned host buffers; the caller provides every
// input and output buffer.
//
// Limits (rejected with ABX_E_UNSUPPORTED before any GPU work):
//   pairs per call               <= kMaxPairs (65536)
//   sum over pairs of Tx * Ty    <= kMaxFramePairs (2^22, 16 MiB of FP32)
//   frames per item              <= 128
// Every GPU that loads the library holds the scratch (about 18 MiB) until
// the process exits.
//
// A frame of zero norm has no angular distance: its pairs get NaN and the
// call sets a status word at the head of the scratch, which
// abx_dtw_pairs_noalloc_check reads (ABX_E_ZERO_NORM), the same error that
// abx_distances reports for such a frame.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "abx_internal.h"

namespace abx {
namespace {

constexpr int64_t kMaxPairs = 65536;
constexpr int64_t kMaxFramePairs = int64_t(1) << 22;
constexpr int kMaxDevices = 64;

struct PairRec {
    int64_t x_row;   // first frame row of x in the caller's feature matrix
    int64_t y_row;
    int64_t block;   // offset of the pair's Tx x Ty block in the distance area
    int32_t tx, ty;
};

constexpr size_t kHeadBytes = 256;  // status word (int32 flags), padded
constexpr size_t kTableBytes = sizeof(PairRec) * kMaxPairs;
constexpr size_t kScratchBytes = kHeadBytes + kTableBytes + sizeof(float) * kMaxFramePairs;
constexpr int32_t kNaZeroNorm = 1;   // status flag: a frame with zero L2 norm

// The scratch: status word, pair table, then the frame-distance blocks.
// Shared by every call on a device; calls that overlap on the GPU race on it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Host-side staging of the pair table and of the status read back by
// abx_dtw_pairs_noalloc_check (static storage, not allocations), guarded by
// a mutex together with the per-device scratch addresses.
static PairRec h_table[kMaxPairs];
static int32_t h_status;
static void *g_scratch_ptr[kMaxDevices];
static std::mutex g_mu;

__device__ __forceinline__ float warp_sum(float v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One CTA per pair: inverse norms of its frames, then every frame cosine
// by a warp (lanes over dim), d = arccos(c) / pi into the pair's block.
__global__ void __launch_bounds__(256) na_frame_dist_kernel(const float *feats, int32_t dim,
                                                             unsigned char *scratch,
                                                             int64_t n_pairs) {
    int32_t *status = reinterpret_cast<int32_t *>(scratch);
    const PairRec *tab = reinterpret_cast<const PairRec *>(scratch + kHeadBytes);
    float *area = reinterpret_cast<float *>(scratch + kHeadBytes + kTableBytes);
    const float nan = __int_as_float(0x7fc00000);
    __shared__ float inv[2 * kMaxItemLen];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int64_t p = blockIdx.x; p < n_pairs; p += gridDim.x) {
        const PairRec r = tab[p];
        for (int f = warp; f < r.tx + r.ty; f += nw) {
            const float *v = feats + (f < r.tx ? r.x_row + f : r.y_row + (f - r.tx)) * dim;
            float s = 0.0f;
            for (int c = lane; c < dim; c += 32) s = fmaf(v[c], v[c], s);
            s = warp_sum(s);
            if (lane == 0) {
                inv[f] = s > 0.0f ? 1.0f / sqrtf(s) : nan;
                if (!(s > 0.0f)) atomicOr(status, kNaZeroNorm);
            }
        }
        __syncthreads();
        for (int e = warp; e < r.tx * r.ty; e += nw) {
            const int i = e / r.ty, j = e - i * r.ty;
            const float *u = feats + (r.x_row + i) * dim, *v = feats + (r.y_row + j) * dim;
            float s = 0.0f;
            for (int c = lane; c < dim; c += 32) s = fmaf(u[c], v[c], s);
            s = warp_sum(s);
            if (lane == 0) {
                // a zero-norm frame (inverse norm NaN) gives NaN, not a clamped cosine
                const float c0 = s * inv[i] * inv[r.tx + j];
                const float c = c0 != c0 ? c0 : fminf(1.0f, fmaxf(-1.0f, c0));
                area[r.block + e] = acosf(c) * 0.318309886183790671f;
            }
        }
        __syncthreads();
    }
}

// One thread per pair: the DTW of the distance kernel, row by row, previous
// row in shared memory laid out [column][thread].
constexpr int kDtwThreads = 64;

__global__ void __launch_bounds__(kDtwThreads) na_dtw_kernel(const unsigned char *scratch,
                                                              int64_t n_pairs, float *dist,
                                                              int32_t *len) {
    const PairRec *tab = reinterpret_cast<const PairRec *>(scratch + kHeadBytes);
    const float *area = reinterpret_cast<const float *>(scratch + kHeadBytes + kTableBytes);
    __shared__ float rbc[kMaxItemLen * kDtwThreads];
    __shared__ uint8_t rbl[kMaxItemLen * kDtwThreads];
    const int tid = threadIdx.x, nt = blockDim.x;
    const float inf = __int_as_float(0x7f800000);
    for (int64_t p = (int64_t)blockIdx.x * nt + tid; p < n_pairs; p += (int64_t)gridDim.x * nt) {
        const PairRec r = tab[p];
        const float *blk = area + r.block;
        float lc = 0.0f;
        int ll = 0;
        bool bad = false;  // a frame of zero norm (NaN distances): no DTW value
        for (int i = 0; i < r.tx; ++i) {
            lc = inf;
            ll = 0;
            float dc = inf;
            int dl = 0;
            for (int j = 0; j < r.ty; ++j) {
                float uc = inf;
                int ul = 0;
                if (i > 0) {
                    uc = rbc[j * nt + tid];
                    ul = rbl[j * nt + tid];
                }
                float mc;
                int ml;
                if (i == 0 && j == 0) {
                    mc = 0.0f;
                    ml = 0;
                } else {
                    mc = fminf(uc, fminf(lc, dc));
                    ml = 255;
                    if (uc == mc) ml = min(ml, ul);
                    if (lc == mc) ml = min(ml, ll);
                    if (dc == mc) ml = min(ml, dl);
                }
                const float dij = blk[i * r.ty + j];
                bad |= dij != dij;
                const float nc = dij + mc;
                dc = uc;
                dl = ul;
                lc = nc;
                ll = ml + 1;
                rbc[j * nt + tid] = nc;
                rbl[j * nt + tid] = (uint8_t)ll;
            }
        }
        dist[p] = bad ? __int_as_float(0x7fc00000) : __fdiv_rn(lc, (float)ll);
        if (len) len[p] = bad ? 0 : ll;
    }
}

}  // namespace
}  // namespace abx

using namespace abx;

extern "C" int abx_dtw_pairs_noalloc(const float *feats, int64_t n_frames, int32_t dim,
                                     const int64_t *item_offsets, int64_t n_items,
                                     const int64_t *pairs, int64_t n_pairs, float *dist,
                                     int32_t *len, void *stream) {
    if (!feats || !item_offsets || (n_pairs > 0 && (!pairs || !dist)) || n_items <= 0 ||
        dim <= 0 || n_pairs < 0) {
        set_error("abx_dtw_pairs_noalloc: NULL argument or bad size");
        return ABX_E_INVALID;
    }
    if (n_pairs > kMaxPairs) {
        set_error("abx_dtw_pairs_noalloc: %lld pairs exceed the fixed scratch limit of %lld",
                  (long long)n_pairs, (long long)kMaxPairs);
        return ABX_E_UNSUPPORTED;
    }
    if (item_offsets[0] != 0 || item_offsets[n_items] != n_frames) {
        set_error("abx_dtw_pairs_noalloc: item_offsets must run from 0 to n_frames");
        return ABX_E_INVALID;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    int64_t total = 0;
    for (int64_t p = 0; p < n_pairs; ++p) {
        const int64_t x = pairs[2 * p], y = pairs[2 * p + 1];
        if (x < 0 || x >= n_items || y < 0 || y >= n_items) {
            set_error("abx_dtw_pairs_noalloc: pair %lld refers to a missing item", (long long)p);
            return ABX_E_INVALID;
        }
        if (item_offsets[x] < 0 || item_offsets[x + 1] > n_frames || item_offsets[y] < 0 ||
            item_offsets[y + 1] > n_frames) {
            set_error("abx_dtw_pairs_noalloc: pair %lld has an item outside 0..n_frames",
                      (long long)p);
            return ABX_E_INVALID;
        }
        const int64_t tx = item_offsets[x + 1] - item_offsets[x];
        const int64_t ty = item_offsets[y + 1] - item_offsets[y];
        if (tx < 1 || ty < 1) {
            set_error("abx_dtw_pairs_noalloc: pair %lld has an empty item or decreasing "
                      "frame offsets", (long long)p);
            return ABX_E_INVALID;
        }
        if (tx > kMaxItemLen || ty > kMaxItemLen) {
            set_error("abx_dtw_pairs_noalloc: pair %lld has an item of %lld / %lld frames "
                      "(1..%d supported)", (long long)p, (long long)tx, (long long)ty,
                      kMaxItemLen);
            return ABX_E_UNSUPPORTED;
        }
        h_table[p] = PairRec{item_offsets[x], item_offsets[y], total, (int32_t)tx, (int32_t)ty};
        total += tx * ty;
    }
    if (total > kMaxFramePairs) {
        set_error("abx_dtw_pairs_noalloc: %lld frame pairs exceed the fixed scratch limit of "
                  "%lld", (long long)total, (long long)kMaxFramePairs);
        return ABX_E_UNSUPPORTED;
    }
    if (n_pairs == 0) return ABX_OK;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        set_error("abx_dtw_pairs_noalloc: no usable current device");
        return ABX_E_CUDA;
    }
    // set-up, once per device, with that device current
    if (!g_scratch_ptr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            set_error("abx_dtw_pairs_noalloc: cudaGetSymbolAddress failed: %s",
                      cudaGetErrorString(e));
            return ABX_E_CUDA;
        }
        g_scratch_ptr[dev] = ptr;
    }
    unsigned char *scratch = static_cast<unsigned char *>(g_scratch_ptr[dev]);
    cudaStream_t s = (cudaStream_t)stream;
    // the pair table is staged from static pageable host storage, a copy that
    // stream capture cannot record (a captured copy would replay whatever a
    // later call left in h_table): refuse to run while the stream captures
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
        set_error("abx_dtw_pairs_noalloc: the stream is being captured (or cannot be "
                  "queried); call it outside stream capture");
        return ABX_E_UNSUPPORTED;
    }
    // this call's status starts at zero
    e = cudaMemsetAsync(scratch, 0, sizeof(int32_t), s);
    // for pageable host memory the copy has left h_table before
    // cudaMemcpyAsync returns
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(scratch + kHeadBytes, h_table, sizeof(PairRec) * n_pairs,
                            cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        set_error("abx_dtw_pairs_noalloc: table copy failed: %s", cudaGetErrorString(e));
        return ABX_E_CUDA;
    }
    int nsm = 148;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int g1 = (int)(n_pairs < (int64_t)nsm * 8 ? n_pairs : (int64_t)nsm * 8);
    na_frame_dist_kernel<<<g1, 256, 0, s>>>(feats, dim, scratch, n_pairs);
    count_launch();
    const int64_t g2 = (n_pairs + kDtwThreads - 1) / kDtwThreads;
    na_dtw_kernel<<<(unsigned)g2, kDtwThreads, 0, s>>>(scratch, n_pairs, dist, len);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("abx_dtw_pairs_noalloc: launch failed: %s", cudaGetErrorString(e));
        return ABX_E_CUDA;
    }
    return ABX_OK;
}

extern "C" int abx_dtw_pairs_noalloc_check(void *stream) {
    std::lock_guard<std::mutex> lk(g_mu);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        set_error("abx_dtw_pairs_noalloc_check: no usable current device");
        return ABX_E_CUDA;
    }
    if (!g_scratch_ptr[dev]) return ABX_OK;  // no call has run on this device
    cudaStream_t s = (cudaStream_t)stream;
    e = cudaMemcpyAsync(&h_status, g_scratch_ptr[dev], sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_error("abx_dtw_pairs_noalloc_check: %s", cudaGetErrorString(e));
        return ABX_E_CUDA;
    }
    if (h_status & kNaZeroNorm) {
        set_error("abx_dtw_pairs_noalloc: a frame has zero L2 norm (its pairs are NaN)");
        return ABX_E_ZERO_NORM;
    }
    return ABX_OK;
}
