// Host runtime of libabx: contexts, item registration, the task (cell)
// builder, and the orchestration of the distance kernels.
//
// Paper map (fastabx, arXiv 2505.02692):
//   abx_load_items   Sec. 3.1 Dataset (labels + representations)
//   abx_build_cells  Sec. 2 on/by/across conditions, Sec. 3.1 Task
//   abx_distances    Sec. 3.2 (DTW on angular frame distances, or pooling)
//
// Everything device-side is stream ordered: uploads go through pinned
// staging buffers from a per-context pool and stream-ordered allocations,
// objects are freed with cudaFreeAsync on their stream, and abx_distances
// never waits for the GPU (sizes it cannot know on the host are bounded from
// above and read back by the kernels themselves).
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "abx_internal.h"

namespace abx {

static thread_local std::string g_err;

void set_error(const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
}

TaskDev Cells::dev() const {
    TaskDev t;
    t.n_items = (int32_t)info.n_items;
    t.K_on = K_on;
    t.K_s = K_s;
    t.n_groups = n_groups;
    t.across = across >= 0 ? 1 : 0;
    t.item_id = d_item_id;
    t.item_g = d_item_g;
    t.item_p = d_item_p;
    t.item_s = d_item_s;
    t.group_begin = d_group_begin;
    t.group_dm = d_group_dm;
    t.blk = d_blk;
    t.tot = d_tot;
    t.gmeta = d_gmeta;
    return t;
}

void *PinnedPool::acquire(size_t n) {
    std::lock_guard<std::mutex> lk(mu);
    for (auto &b : bufs)
        if (!b.busy && b.n >= n && cudaEventQuery(b.ev) == cudaSuccess) {
            b.busy = true;
            return b.p;
        }
    size_t cap = 4096;
    while (cap < n) cap <<= 1;
    Buf b;
    if (cudaMallocHost(&b.p, cap) != cudaSuccess) return nullptr;
    if (cudaEventCreateWithFlags(&b.ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaFreeHost(b.p);
        return nullptr;
    }
    b.n = cap;
    b.busy = true;
    bufs.push_back(b);
    return b.p;
}

void PinnedPool::release(void *p, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(mu);
    for (auto &b : bufs)
        if (b.p == p) {
            cudaEventRecord(b.ev, s);
            b.busy = false;
            return;
        }
}

PinnedPool::~PinnedPool() {
    for (auto &b : bufs) {
        cudaEventSynchronize(b.ev);
        cudaEventDestroy(b.ev);
        cudaFreeHost(b.p);
    }
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

template <class T>
static cudaError_t dalloc(T **p, size_t n, cudaStream_t s) {
    *p = nullptr;
    if (n == 0) n = 1;
    return cudaMallocAsync((void **)p, n * sizeof(T), s);
}

template <class T>
static void dfree(T *&p, cudaStream_t s) {
    if (p) cudaFreeAsync((void *)p, s);
    p = nullptr;
}

// Upload from a pinned host buffer.  A copy engine serves the host-to-device
// copies of all streams in submission order, so a cudaMemcpyAsync of a few
// kilobytes issued while another stream's multi-gigabyte feature copy is
// queued would wait for all of it.  So while a feature copy of the context
// is pending, a kernel reads the host memory through the unified address
// space over the bus itself; otherwise the copy engine takes the upload
// (about 0.08 ms less per upload of a plan).
__global__ void upload_kernel(uint4 *__restrict__ dst, const uint4 *__restrict__ src, size_t n16) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16;
         i += (size_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

static cudaError_t upload(Ctx *ctx, void *dev, const void *pinned, size_t bytes,
                          cudaStream_t s) {
    const size_t n16 = (bytes + 15) / 16;  // both buffers are padded to 256 bytes
    if (n16 == 0) return cudaSuccess;
    // the copy engine while no feature copy of this context is pending (and
    // the stream is not being captured), else the kernel
    bool dma = true;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
        dma = false;
    if (dma) {
        std::lock_guard<std::mutex> g(ctx->copy_mu);
        if (ctx->feat_copy) {
            const cudaError_t q = cudaEventQuery(ctx->feat_copy);
            if (q == cudaErrorNotReady)
                dma = false;
            else if (q != cudaSuccess)
                return q;
        }
    }
    if (dma) return cudaMemcpyAsync(dev, pinned, n16 * 16, cudaMemcpyHostToDevice, s);
    const unsigned blocks = (unsigned)std::min<size_t>((n16 + 255) / 256, 1024);
    abx::ProfScope ps_("upload", s);
    upload_kernel<<<blocks, 256, 0, s>>>((uint4 *)dev, (const uint4 *)pinned, n16);
    return cudaGetLastError();
}

// Packs several host arrays into one pinned buffer from the context pool
// and one stream-ordered device block, uploaded at once.  Each array starts
// on a 256-byte boundary.
struct Staging {
    std::vector<std::pair<size_t, size_t>> parts;  // (offset, bytes)
    std::vector<const void *> srcs;
    size_t bytes = 0;
    uint8_t *dev = nullptr;
    template <class T>
    size_t add(const std::vector<T> &v) {
        return add_raw(v.data(), v.size() * sizeof(T));
    }
    size_t add_raw(const void *src, size_t b) {
        size_t off = bytes;
        parts.push_back({off, b});
        srcs.push_back(src);
        bytes += std::max<size_t>(256, (b + 255) / 256 * 256);
        return off;
    }
    template <class T>
    T *at(size_t off) const { return reinterpret_cast<T *>(dev + off); }
    cudaError_t commit(Ctx *ctx, cudaStream_t s) {
        void *pin = ctx->pinned.acquire(bytes);
        if (!pin) return cudaErrorMemoryAllocation;
        for (size_t i = 0; i < parts.size(); ++i)
            if (parts[i].second && srcs[i])
                memcpy((uint8_t *)pin + parts[i].first, srcs[i], parts[i].second);
        cudaError_t e = cudaMallocAsync((void **)&dev, bytes, s);
        if (e == cudaSuccess) e = upload(ctx, dev, pin, bytes, s);
        ctx->pinned.release(pin, s);
        return e;
    }
};

namespace abx {

// A non-blocking stream per (thread, device) for cell building, at the
// highest priority: its small kernels get SMs ahead of the queued blocks of
// earlier tasks' distance kernels, so the host's planning of the next task
// does not wait for them.
cudaStream_t build_stream(int device) {
    static thread_local std::map<int, cudaStream_t> m;
    auto f = m.find(device);
    if (f != m.end()) return f->second;
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    cudaStream_t s = nullptr;
    cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, hi);
    m[device] = s;
    return s;
}

Ctx::~Ctx() {
    if (feat_copy) cudaEventDestroy(feat_copy);
    for (ScratchSlot &sl : scratch) {
        if (sl.ev) {
            cudaEventSynchronize(sl.ev);
            cudaEventDestroy(sl.ev);
        }
        if (sl.p) cudaFree(sl.p);
    }
}

constexpr size_t kScratchSlots = 2;

void *scratch_acquire(Ctx *c, size_t n, cudaStream_t s, int *slot) {
    *slot = -1;
    std::lock_guard<std::mutex> lk(c->scratch_mu);
    // a free slot last used on this stream or whose last use has ended
    // (the smallest that fits), else a new slot, else a free slot whose
    // last use, on another stream, this stream then waits for
    int best = -1, other = -1;
    for (int i = 0; i < (int)c->scratch.size(); ++i) {
        const Ctx::ScratchSlot &sl = c->scratch[i];
        if (sl.busy || sl.n < n) continue;
        const bool ready = sl.last == s || cudaEventQuery(sl.ev) == cudaSuccess;
        int &b = ready ? best : other;
        if (b < 0 || sl.n < c->scratch[b].n) b = i;
    }
    if (best < 0 && c->scratch.size() < kScratchSlots) {
        // sized to the next power of two, so that a later, somewhat larger
        // request (the next job's) still fits
        size_t cap = 1;
        while (cap < n) cap <<= 1;
        n = cap;
        Ctx::ScratchSlot sl;
        if (cudaMalloc(&sl.p, n) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        if (cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaFree(sl.p);
            cudaGetLastError();
            return nullptr;
        }
        sl.n = n;
        c->scratch.push_back(sl);
        best = (int)c->scratch.size() - 1;
    }
    if (best < 0 && other >= 0) {
        if (cudaStreamWaitEvent(s, c->scratch[other].ev, 0) != cudaSuccess) return nullptr;
        best = other;
    }
    if (best < 0) return nullptr;
    c->scratch[best].busy = true;
    *slot = best;
    return c->scratch[best].p;
}

void scratch_release(Ctx *c, int slot, cudaStream_t s) {
    if (slot < 0) return;
    std::lock_guard<std::mutex> lk(c->scratch_mu);
    Ctx::ScratchSlot &sl = c->scratch[slot];
    cudaEventRecord(sl.ev, s);
    sl.last = s;
    sl.busy = false;
}

void ctx_retain(Ctx *c) {
    if (c) c->refs.fetch_add(1, std::memory_order_relaxed);
}

void ctx_release(Ctx *c) {
    if (c && c->refs.fetch_sub(1, std::memory_order_acq_rel) == 1) {
        cudaSetDevice(c->device);
        delete c;
    }
}

// Bound on |computed cosine - exact cosine of the stored vectors| for each
// precision, the cosine being <q_x, q_y> |q_x|^-1 |q_y|^-1 of the stored
// vectors q (their angle theta to the exact frames is bounded separately).
//
// Dot product, CUDA cores (ABX_FP32_SIMT): a chain of dim_pad fused
// multiply-adds rounded to nearest, gamma_n(u) with n = dim_pad, u = 2^-24
// (Higham, Accuracy and Stability of Numerical Algorithms, Sec. 3.1), times
// sum |q_xk q_yk| <= |q_x| |q_y|.
//
// Dot product, tensor cores: the products of two FP16, BF16 or E4M3 values
// are exact in FP32, but the rounding of tcgen05's FP32 accumulation is not
// documented.  Assumed model (conservative; it covers the behaviour measured
// on earlier tensor cores, Fasi, Higham, Mikaitis and Pranesh, "Numerical
// behavior of NVIDIA tensor cores", PeerJ Comput. Sci. 2021: addends aligned
// to the largest exponent and truncated, result truncated): one MMA
// instruction that adds its K products (K = 16 for kind::f16, 32 for
// kind::f8f6f4) to the accumulator commits an error of at most K + 2 units
// of 2^-23 times the sum of the magnitudes of the accumulator and its
// products.  With m instructions per dot product the error is then at most
// gamma_{(K+2) m}(2^-23) times the sum of |terms|.
//   ABX_BF16: m = dim_pad / 16.      ABX_FP8: m = dim_pad / 32.
//   ABX_FP32 (split v = hi + lo, FP16 halves, lo*lo dropped): hi*hi goes to
//   one accumulator (m = dim_pad / 16, sum |terms| <= (1 + 2^-9) |q_x||q_y|)
//   and hi*lo + lo*hi to another (m = 2 dim_pad / 16, sum |terms| <=
//   2^-10 (1 + 2^-9) |q_x||q_y| since |lo| <= 2^-11 (1 + 2^-11) |v|), added
//   once in FP32 (u); the dropped sum |lo_x lo_y| <= 2^-22 (1 + 2^-9)
//   |q_x||q_y|.
//
// Scaling (every precision): the inverse norms come from sum q^2 in FP32
// (per lane a chain of dim_pad / 32 terms, then a 5-level warp tree: relative
// error gamma_{dim_pad/32+5}(u)), a square root and a division, so each is
// within gamma_{dim_pad/32+5}(u) / 2 + 2u of 1/|q|; the epilogue's two
// products add 2u.  The cosine (|cos| <= 1) moves by at most
// gamma_{dim_pad/32+5}(u) + 6u.  The total is widened by 1e-4 relative, which
// covers the second-order terms and the FP32 evaluation of this formula.
float cosine_error_bound(int precision, int dim_pad) {
    auto gamma = [](double n, double u) { return n * u / (1.0 - n * u); };
    const double u = std::ldexp(1.0, -24), u23 = std::ldexp(1.0, -23);
    double e;
    if (precision == ABX_FP32_SIMT) {
        e = gamma(dim_pad, u);
    } else if (precision == ABX_FP32) {
        const double m = dim_pad / 16.0, w = 1.0 + std::ldexp(1.0, -9);
        e = gamma(18.0 * m, u23) * w + gamma(18.0 * 2.0 * m, u23) * std::ldexp(w, -10) + u +
            std::ldexp(w, -22);
    } else if (precision == ABX_BF16) {
        e = gamma(18.0 * (dim_pad / 16.0), u23);
    } else {
        e = gamma(34.0 * (dim_pad / 32.0), u23);
    }
    e += gamma(dim_pad / 32.0 + 5.0, u) + 6.0 * u;
    return (float)(e * 1.0001);
}

void packed_rows_release(const Items *it, PackedRows *pr, cudaStream_t s) {
    if (!pr) return;
    {
        std::lock_guard<std::mutex> g(it->pack_mu);
        if (--pr->refs > 0) return;
    }
    for (cudaEvent_t e : pr->uses) {
        cudaStreamWaitEvent(s, e, 0);
        cudaEventDestroy(e);
    }
    for (void *q : {(void *)pr->inv_norm, (void *)pr->nrm2, (void *)pr->theta, (void *)pr->scale,
                    (void *)pr->theta_item, (void *)pr->err, pr->packed})
        if (q) cudaFreeAsync(q, s);
    if (pr->ready) cudaEventDestroy(pr->ready);
    delete pr;
}

int dist_plan_build_rows(Ctx *ctx, const Items *it, const Cells *c, int32_t mode,
                         int32_t distance, int32_t precision, cudaStream_t s, DistPlan *pp) {
    DistPlan &p = *pp;
    REQUIRE(mode == ABX_DTW || mode == ABX_MEAN, ABX_E_INVALID, "bad mode %d", mode);
    REQUIRE(distance >= ABX_DIST_ANGULAR && distance <= ABX_DIST_KL, ABX_E_INVALID,
            "bad distance %d", distance);
    REQUIRE(precision >= ABX_FP32_SIMT && precision <= ABX_FP8, ABX_E_INVALID,
            "bad precision %d", precision);
    REQUIRE(precision == ABX_FP32_SIMT || umma_supported(precision), ABX_E_UNSUPPORTED,
            "precision %d not available in this build", precision);
    Trace tr("dist_plan");
    p.ctx = ctx;
    p.it = it;
    p.c = c;
    p.mode = mode;
    p.distance = distance;
    p.precision = precision;
    const int64_t n = c->info.n_items;
    p.n = n;
    p.dim = it->dim;
    p.dim_pad = (p.dim + 127) / 128 * 128;
    // KL: each packed row holds [p | ln p], a k extent of twice the padded dim
    REQUIRE(distance != ABX_DIST_KL || precision == ABX_FP32, ABX_E_UNSUPPORTED,
            "the KL distance is built for precision ABX_FP32 only");
    if (distance == ABX_DIST_KL) p.dim_pad *= 2;

    // ---- packed rows: items in task order, one row per frame (or per item)
    std::vector<int32_t> &len = p.h_len, &row = p.h_row;
    len.resize(n);
    row.resize(n);
    int64_t rows = 0;
    int32_t max_len = 1;
    for (int64_t k = 0; k < n; ++k) {
        int64_t id = c->item_id[k];
        int32_t T = mode == ABX_MEAN ? 1 : (int32_t)(it->h_offsets[id + 1] - it->h_offsets[id]);
        len[k] = T;
        row[k] = (int32_t)rows;
        rows += T;
        max_len = std::max(max_len, T);
    }
    p.rows = rows;
    p.max_len = max_len;
    tr.mark("lengths");
    Staging st_keep;
    size_t o_len = st_keep.add(len), o_row = st_keep.add(row);
    CU(cudaStreamWaitEvent(s, c->ready, 0));
    CU(st_keep.commit(ctx, s));
    p.keep_block = st_keep.dev;
    p.d_len = st_keep.at<int32_t>(o_len);
    p.d_row = st_keep.at<int32_t>(o_row);
    tr.mark("keep upload");
    CU(dalloc(&p.d_err, 4, s));
    CU(dalloc(&p.d_count, 2, s));
    p.elem = precision == ABX_FP32_SIMT ? 4 : precision == ABX_FP32 ? 4 : precision == ABX_BF16 ? 2 : 1;
    if (p.share_pack) {
        std::lock_guard<std::mutex> g(it->pack_mu);
        PackedRows *e = it->pack;
        if (e && e->mode == mode && e->distance == distance && e->precision == precision &&
            e->dim_pad == p.dim_pad && (int64_t)e->order.size() == n &&
            memcmp(e->order.data(), c->item_id.data(), (size_t)n * sizeof(int32_t)) == 0) {
            ++e->refs;
            p.shared = e;
            p.pack_hit = true;
            p.packed = e->packed;
            p.inv_norm = e->inv_norm;
            p.nrm2 = e->nrm2;
            p.theta = e->theta;
            p.scale = e->scale;
            p.theta_item = e->theta_item;
        }
    }
    if (!p.shared) {
        CU(cudaMallocAsync(&p.packed, (size_t)std::max<int64_t>(rows, 1) * p.dim_pad * p.elem, s));
        CU(dalloc(&p.inv_norm, rows, s));
        CU(dalloc(&p.nrm2, rows, s));
        CU(dalloc(&p.theta, rows, s));
        CU(dalloc(&p.scale, n, s));
        CU(dalloc(&p.theta_item, n, s));
    }
    tr.mark("rows");
    return ABX_OK;
}

int dist_plan_build_tiles(cudaStream_t s, DistPlan *pp) {
    DistPlan &p = *pp;
    Trace tr("dist_plan");
    const Cells *c = p.c;
    const Ctx *ctx = p.ctx;
    const int64_t n = p.n;
    const std::vector<int32_t> &len = p.h_len, &row = p.h_row;
    const int32_t max_len = p.max_len;
    const int32_t precision = p.precision;
    // per group: panels by greedy packing of whole items (the fewest panels
    // of consecutive items), then the upper triangle of panel pairs; group
    // offsets from prefix sums
    const int32_t G = c->n_groups;
    std::vector<int64_t> g_np(G + 1, 0), g_nt(G + 1, 0);
    for (int32_t g = 0; g < G; ++g) {
        const int32_t b = c->group_begin[g], e = c->group_begin[g + 1];
        int64_t np = 0;
        int32_t used = kPanel;
        for (int32_t k = b; k < e; ++k) {
            if (used + len[k] > kPanel) {
                ++np;
                used = 0;
            }
            used += len[k];
        }
        g_np[g + 1] = np;
        g_nt[g + 1] = e - b < 2 ? 0 : np * (np + 1) / 2;
    }
    for (int32_t g = 0; g < G; ++g) {
        g_np[g + 1] += g_np[g];
        g_nt[g + 1] += g_nt[g];
    }
    tr.mark("panel counts");
    std::vector<int32_t> panel_row(g_np[G]), panel_item(g_np[G] + 1);
    std::vector<int2> tiles(g_nt[G]);
    std::vector<int64_t> tile_cand(g_nt[G]);  // candidate pairs per tile (upper bound)
    tr.mark("tile vectors");
    for (int32_t g = 0; g < G; ++g) {
        const int32_t b = c->group_begin[g], e = c->group_begin[g + 1];
        const int32_t p0 = (int32_t)g_np[g], p1 = (int32_t)g_np[g + 1];
        int32_t q = p0, used = kPanel;
        for (int32_t k = b; k < e; ++k) {
            if (used + len[k] > kPanel) {
                panel_row[q] = row[k];
                panel_item[q] = k;
                ++q;
                used = 0;
            }
            used += len[k];
        }
        if (e - b < 2) continue;
        int64_t t = g_nt[g];
        for (int32_t pi = p0; pi < p1; ++pi) {
            const int64_t mi = (pi + 1 < p1 ? panel_item[pi + 1] : e) - panel_item[pi];
            for (int32_t pj = pi; pj < p1; ++pj, ++t) {
                const int64_t mj = (pj + 1 < p1 ? panel_item[pj + 1] : e) - panel_item[pj];
                tiles[t] = make_int2(pi, pj);
                tile_cand[t] = pi == pj ? mi * (mi - 1) / 2 : mi * mj;
            }
        }
    }
    panel_item[g_np[G]] = (int32_t)n;
    p.n_tiles = (int64_t)tiles.size();
    tr.mark("panels+tiles");

    // Fused tile + DTW kernel (tcgen05 path, items of at most
    // umma_fuse_max_len() frames): the DTWs run on the tile in shared memory,
    // so there is no tile buffer and one chunk takes every tile.  ABX_FUSE=1:
    // a thread per pair, in place on the d tile; ABX_FUSE=2: 8-lane
    // wavefronts.  Not the default: on the triphone-scale step the two took
    // 22.9 and 25.4 ms against 10.8-11.4 ms for the tile kernel +
    // stand-alone DTW kernel.  A tile's DTW waits for its longest pair's
    // serial chain, which the few warps of one tile cannot hide, so it no
    // longer fits under the next tile's MMAs.
    const char *fz = getenv("ABX_FUSE");
    p.fused = precision != ABX_FP32_SIMT && max_len <= umma_fuse_max_len() && fz &&
              (fz[0] == '1' || fz[0] == '2');
    p.fuse_form = p.fused && fz[0] == '2' ? 1 : 0;
    // chunks of tiles under the tile-buffer budget; pair capacity per chunk
    const char *env = getenv("ABX_TILE_BUDGET_MB");
    const int64_t budget_mb = env ? atoll(env) : 8192;
    int64_t chunk = p.fused ? std::max<int64_t>(p.n_tiles, 1)
                            : std::max<int64_t>(1, budget_mb * (1LL << 20) / (kPanel * kPanel * 4));
    // at most 2^17 tiles (8 GiB) per chunk: the tile kernels index a chunk's
    // buffer with 32-bit offsets
    chunk = std::min<int64_t>(chunk, (int64_t)1 << 17);
    chunk = std::min<int64_t>(chunk, std::max<int64_t>(p.n_tiles, 1));
    p.chunk = chunk;
    p.chunk_cap.clear();
    p.cap_max = p.cap_total = 0;
    for (int64_t t0 = 0; t0 < p.n_tiles; t0 += chunk) {
        int64_t cap = 0;
        for (int64_t t = t0; t < std::min(p.n_tiles, t0 + chunk); ++t) cap += tile_cand[t];
        p.chunk_cap.push_back(cap);
        p.cap_max = std::max(p.cap_max, cap);
        p.cap_total += cap;
    }
    // default kernel variants of the unfused path (the batch autotuner may
    // change them): 3 = for BF16 / FP8 the wide tcgen05 kernel with 16
    // epilogue warps (BF16 4.6 -> 3.5 ms per triphone-scale step against the
    // narrow kernel), for the FP32 split the narrow kernel with 16 epilogue
    // warps
    const char *uv = getenv("ABX_UMMA_VARIANT");
    p.umma_variant = uv ? atoi(uv) : 3;
    const char *dv = getenv("ABX_DTW_VARIANT");
    p.dtw_variant = dv ? atoi(dv) : 0;
    // tile buffer layout and the narrow / pair kernels' store rule.  Default:
    // column-major tiles, only the listed pairs' blocks stored (FP32 split
    // tile kernel 7.3 -> 6.8 ms per triphone-scale step).  ABX_TILE_LAYOUT=1
    // puts each item's rows in a strip, so that a pair's block is contiguous:
    // it halved the DTW's DRAM reads (11 -> 6 B per cell) but not its time
    // (3.85 -> 3.9 ms), and is kept as a measured option.  The wide kernel
    // (BF16 / FP8 default) always writes whole column-major tiles.
    const char *tlay = getenv("ABX_TILE_LAYOUT");
    p.strips = tlay ? (atoi(tlay) != 0) : 0;
    const char *tst = getenv("ABX_TILE_STORE");
    p.listed_only = tst ? (atoi(tst) != 0) : 1;

    tr.mark("chunks");
    // work items of the wide tile kernel: a tile and the next tile of the
    // same panel row (adjacent column panel) of the same chunk, tile indices
    // relative to the chunk
    // (built for the kernels that take them: the BF16 / FP8 wide kernel, which
    // the autotuner may also choose, and the FP32 split's cluster-pair
    // variant; the narrow kernel does without)
    std::vector<int2> work;
    const bool need_work = precision != ABX_FP32 || p.umma_variant == 4;
    if (need_work) work.reserve(p.n_tiles / 2 + 16);
    const int64_t n_chunks = (p.n_tiles + chunk - 1) / chunk;
    p.work_off.assign(n_chunks + 1, 0);
    for (int64_t t = 0; need_work && t < p.n_tiles;) {
        const int64_t ci = t / chunk, t0 = ci * chunk;
        const bool pair = t + 1 < p.n_tiles && (t + 1) / chunk == ci &&
                          tiles[t + 1].x == tiles[t].x && tiles[t + 1].y == tiles[t].y + 1;
        work.push_back(make_int2((int)(t - t0), pair ? (int)(t + 1 - t0) : -1));
        ++p.work_off[ci + 1];
        t += pair ? 2 : 1;
    }
    for (int64_t ci = 0; ci < n_chunks; ++ci) p.work_off[ci + 1] += p.work_off[ci];
    Staging st_plan;
    size_t o_pr = st_plan.add(panel_row), o_pi = st_plan.add(panel_item), o_t = st_plan.add(tiles);
    size_t o_w = st_plan.add(work);
    tr.mark("work list");
    CU(st_plan.commit(const_cast<Ctx *>(ctx), s));
    p.plan_block = st_plan.dev;
    tr.mark("upload");
    p.d_panel_row = st_plan.at<int32_t>(o_pr);
    p.d_panel_item = st_plan.at<int32_t>(o_pi);
    p.d_tiles = st_plan.at<int2>(o_t);
    p.d_work = need_work ? st_plan.at<int2>(o_w) : nullptr;

    // ---- device buffers
    p.dm = std::max<int64_t>(c->dm_entries, 1);
    CU(dalloc(&p.pv, p.dm, s));
    CU(dalloc(&p.tile_count, chunk, s));
    CU(dalloc(&p.tile_base, chunk + 1, s));
    CU(dalloc(&p.chunk_total, 1, s));
    p.tilebuf = nullptr;
    if (p.use_scratch && !p.fused)
        p.tilebuf = static_cast<float *>(scratch_acquire(
            p.ctx, (size_t)chunk * kPanel * kPanel * sizeof(float), s, &p.scratch_slot));
    if (!p.tilebuf) CU(dalloc(&p.tilebuf, p.fused ? 1 : (size_t)chunk * kPanel * kPanel, s));
    CU(dalloc(&p.d_row_item, p.fused ? 1 : std::max<int64_t>(p.rows, 1), s));
    CU(dalloc(&p.d_xmask, p.fused ? 1 : (size_t)chunk * kPanel, s));
    CU(dalloc(&p.d_col_yo, p.fused ? 1 : (size_t)chunk * kPanel, s));
    CU(dalloc(&p.pairs, std::max<int64_t>(p.cap_max, 1), s));
    tr.mark("buffers");
    return ABX_OK;
}

int dist_plan_build(Ctx *ctx, const Items *it, const Cells *c, int32_t mode, int32_t distance,
                    int32_t precision, cudaStream_t s, DistPlan *p) {
    int rc = dist_plan_build_rows(ctx, it, c, mode, distance, precision, s, p);
    return rc ? rc : dist_plan_build_tiles(s, p);
}

int dist_plan_exec(const DistPlan &p, cudaStream_t s) {
    int rc = dist_plan_exec_pack(p, s);
    return rc ? rc : dist_plan_exec_tiles(p, s);
}

int dist_plan_exec_pack(const DistPlan &p, cudaStream_t s) {
    const Cells *c = p.c;
    const Items *it = p.it;
    CU(cudaMemsetAsync(p.d_err, 0, 4 * sizeof(int32_t), s));
    CU(cudaMemsetAsync(p.d_count, 0, 2 * sizeof(int64_t), s));

    if (p.pack_hit) {  // packed by an earlier call: wait for it, take its flags
        CU(cudaStreamWaitEvent(s, p.shared->ready, 0));
        CU(cudaMemcpyAsync(p.d_err, p.shared->err, sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        return ABX_OK;
    }
    // ---- pack: normalise, quantise, gather into task order
    PackArgs pa;
    pa.feats = it->d_feats;
    pa.offsets = it->d_offsets;
    pa.item_id = c->d_item_id;
    pa.row = p.d_row;
    pa.len = p.d_len;
    pa.n_items = (int32_t)p.n;
    pa.dim = p.dim;
    pa.dim_pad = p.dim_pad;
    pa.mode = p.mode;
    pa.precision = p.precision;
    pa.distance = p.distance;
    pa.nrm2 = p.nrm2;
    pa.n_rows = p.rows;
    pa.packed = p.packed;
    pa.inv_norm = p.inv_norm;
    pa.theta = p.theta;
    pa.theta_item = p.theta_item;
    pa.item_scale = p.scale;
    pa.err = p.d_err;
    CU(launch_pack(pa, s));
    return ABX_OK;
}

int dist_plan_exec_tiles(const DistPlan &p, cudaStream_t s) {
    Trace tr("dist_exec");
    const Cells *c = p.c;
    // ---- group matrices: len 0 = not computed
    CU(cudaMemsetAsync(p.pv, 0, p.dm * sizeof(PairVal), s));

    // ---- chunks of tiles: plan pairs, tile distances, DTW (no host sync)
    TaskDev td = c->dev();
    const float eps_c = cosine_error_bound(p.precision, p.dim_pad);
    const int intervals = p.distance == ABX_DIST_ANGULAR ? 1 : 0;
    // the narrow and pair tcgen05 kernels read the store map and the packed
    // row -> item map; the wide, fused and CUDA-core kernels do not (the
    // CUDA-core kernel reads the row -> item map for the strip layout)
    const bool wide = p.precision != ABX_FP32_SIMT && umma_wide(p.precision, p.umma_variant) &&
                      p.d_work != nullptr;
    const bool maps = !p.fused && !wide && p.precision != ABX_FP32_SIMT;
    const int32_t strips = p.strips && !wide;
    if (maps || (strips && !p.fused))
        CU(launch_row_items(p.d_len, p.d_row, p.n, p.d_row_item, s));
    for (int64_t t0 = 0, ci = 0; t0 < p.n_tiles; t0 += p.chunk, ++ci) {
        const int64_t nt = std::min(p.chunk, p.n_tiles - t0);
        if (p.chunk_cap[ci] == 0) continue;
        TileList tl{p.d_tiles + t0, p.d_panel_row, p.d_panel_item, nt};
        CU(launch_plan_count(td, tl, p.d_len, p.d_row, p.tile_count, p.d_count + 1,
                             maps ? p.d_xmask : nullptr, maps ? p.d_col_yo : nullptr,
                             p.d_row_item, p.rows, s));
        CU(launch_scan_i32_to_i64(p.tile_count, p.tile_base, nt, p.chunk_total, p.d_count, s));
        CU(launch_plan_write(td, tl, p.d_len, p.d_row, p.tile_base, p.pairs, s));
        TileGemmArgs ga;
        ga.packed = p.packed;
        ga.inv_norm = p.inv_norm;
        ga.n_rows = p.rows;
        ga.dim_pad = p.dim_pad;
        ga.tiles = p.d_tiles + t0;
        ga.panel_row = p.d_panel_row;
        ga.tile_count = p.tile_count;
        ga.n_tiles = nt;
        ga.tilebuf = p.tilebuf;
        ga.err = p.d_err + 1;
        ga.distance = p.distance;
        ga.nrm2 = p.nrm2;
        ga.b_rot = p.distance == ABX_DIST_KL ? p.dim_pad / 2 : 0;
        ga.fused = p.fused ? 1 + p.fuse_form : 0;
        ga.pairs = p.pairs;
        ga.tile_base = p.tile_base;
        ga.len = p.d_len;
        ga.theta_item = p.theta_item;
        ga.eps_c = eps_c;
        ga.intervals = intervals;
        ga.item_g = td.item_g;
        ga.gmeta = td.gmeta;
        ga.pv = p.pv;
        ga.variant = p.umma_variant;
        ga.work = p.d_work ? p.d_work + p.work_off[ci] : nullptr;
        ga.n_work = p.work_off[ci + 1] - p.work_off[ci];
        ga.row_item = p.d_row_item;
        ga.row = p.d_row;
        ga.panel_item = p.d_panel_item;
        ga.xmask = p.d_xmask;
        ga.col_yo = p.d_col_yo;
        ga.strips = strips;
        ga.listed_only = p.listed_only;
        if (p.precision == ABX_FP32_SIMT)
            CU(launch_tile_simt(ga, s));
        else
            CU(launch_tile_umma(ga, p.precision, p.ctx->n_sm, s));
        if (p.fused) continue;  // the tile kernel ran the DTWs
        DtwArgs da;
        da.t = td;
        da.pairs = p.pairs;
        da.n_pairs = p.chunk_total;
        da.pair_cap = p.chunk_cap[ci];
        da.tilebuf = p.tilebuf;
        da.strips = strips;
        da.len = p.d_len;
        da.theta_item = p.theta_item;
        da.eps_c = eps_c;
        da.intervals = intervals;
        da.max_len = p.max_len;
        da.pv = p.pv;
        da.variant = p.dtw_variant;
        CU(launch_dtw(da, s));
    }
    tr.mark("enqueued");
    return ABX_OK;
}

int64_t dist_plan_bytes(const DistPlan &p) {
    const int64_t rows = std::max<int64_t>(p.rows, 1);
    return rows * p.dim_pad * (int64_t)p.elem      // packed rows
           + rows * 12 + p.n * 24                  // norms, angles, lengths, rows
           + p.dm * (int64_t)sizeof(PairVal)       // group matrices
           + (p.fused ? 0 : p.chunk * kPanel * (kPanel * 4 + 9) + rows * 4)  // tile buffer, maps
           + std::max<int64_t>(p.cap_max, 1) * 16  // pair list
           + p.chunk * 12 + (int64_t)p.n_tiles * 8 + (int64_t)p.n * 8;
}

void dist_plan_free(DistPlan *p, cudaStream_t s, bool all) {
    dfree(p->pairs, s);
    if (p->scratch_slot >= 0) {
        scratch_release(p->ctx, p->scratch_slot, s);
        p->scratch_slot = -1;
        p->tilebuf = nullptr;
    } else {
        dfree(p->tilebuf, s);
    }
    dfree(p->d_row_item, s);
    dfree(p->d_xmask, s);
    dfree(p->d_col_yo, s);
    dfree(p->tile_count, s);
    dfree(p->tile_base, s);
    dfree(p->chunk_total, s);
    dfree(p->plan_block, s);
    if (p->shared) {  // the packing belongs to the items' cache
        packed_rows_release(p->it, p->shared, s);
        p->shared = nullptr;
        p->packed = nullptr;
        p->inv_norm = p->nrm2 = p->theta = p->scale = p->theta_item = nullptr;
    } else {
        if (p->packed) cudaFreeAsync(p->packed, s);
        p->packed = nullptr;
        dfree(p->inv_norm, s);
        dfree(p->nrm2, s);
        dfree(p->theta, s);
        dfree(p->scale, s);
        dfree(p->theta_item, s);
    }
    if (all) {
        dfree(p->keep_block, s);
        dfree(p->pv, s);
        dfree(p->d_err, s);
        dfree(p->d_count, s);
    }
}

// Adds the plan's freshly packed rows to the items' cache (replacing the
// previous packing); the plan then holds one reference to them.
static int publish_pack(const Items *it, const Cells *c, DistPlan &p, cudaStream_t s) {
    std::unique_ptr<PackedRows> e(new (std::nothrow) PackedRows);
    REQUIRE(e, ABX_E_OOM, "host allocation failed");
    e->mode = p.mode;
    e->distance = p.distance;
    e->precision = p.precision;
    e->dim_pad = p.dim_pad;
    e->order = c->item_id;
    CU(dalloc(&e->err, 1, s));
    CU(cudaMemcpyAsync(e->err, p.d_err, sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    CU(cudaEventCreateWithFlags(&e->ready, cudaEventDisableTiming));
    CU(cudaEventRecord(e->ready, s));
    e->packed = p.packed;
    e->inv_norm = p.inv_norm;
    e->nrm2 = p.nrm2;
    e->theta = p.theta;
    e->scale = p.scale;
    e->theta_item = p.theta_item;
    e->refs = 2;  // the cache and this plan
    PackedRows *old;
    {
        std::lock_guard<std::mutex> g(it->pack_mu);
        old = it->pack;
        it->pack = e.get();
    }
    p.shared = e.release();
    packed_rows_release(it, old, s);
    return ABX_OK;
}

// Records that the plan's kernels on s use its shared packing (its buffers
// are freed only after them); completed records are dropped.
static int note_pack_use(const Items *it, PackedRows *e, cudaStream_t s) {
    cudaEvent_t ev;
    CU(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    CU(cudaEventRecord(ev, s));
    std::lock_guard<std::mutex> g(it->pack_mu);
    std::vector<cudaEvent_t> keep;
    for (cudaEvent_t u : e->uses) {
        if (cudaEventQuery(u) == cudaSuccess) cudaEventDestroy(u);
        else keep.push_back(u);
    }
    keep.push_back(ev);
    e->uses.swap(keep);
    return ABX_OK;
}

}  // namespace abx

extern "C" {

const char *abx_last_error(void) { return g_err.c_str(); }

const char *abx_version(void) { return "abx-b300 0.4 (sm_103a)"; }

double abx_cosine_error_bound(int32_t precision, int32_t dim) {
    if (precision < ABX_FP32_SIMT || precision > ABX_FP8 || dim <= 0) return -1.0;
    return (double)cosine_error_bound(precision, (dim + 127) / 128 * 128);
}

int abx_ctx_create(int device, abx_ctx **out) {
    REQUIRE(out, ABX_E_INVALID, "out is NULL");
    *out = nullptr;
    int n = 0;
    CU(cudaGetDeviceCount(&n));
    REQUIRE(device >= 0 && device < n, ABX_E_INVALID, "device %d out of range (%d)", device, n);
    cudaDeviceProp prop;
    CU(cudaGetDeviceProperties(&prop, device));
    REQUIRE(prop.major == 10 && prop.minor == 3, ABX_E_UNSUPPORTED,
            "device %d is sm_%d%d; this build targets sm_103a", device, prop.major, prop.minor);
    CU(cudaSetDevice(device));
    // Keep freed stream-ordered allocations in the device's default pool so
    // repeated calls do not go back to the driver for memory.
    cudaMemPool_t pool;
    CU(cudaDeviceGetDefaultMemPool(&pool, device));
    uint64_t keep = UINT64_MAX;
    CU(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
    Ctx *c = new (std::nothrow) Ctx;
    REQUIRE(c, ABX_E_OOM, "host allocation failed");
    c->device = device;
    c->n_sm = prop.multiProcessorCount;
    *out = reinterpret_cast<abx_ctx *>(c);
    return ABX_OK;
}

int abx_ctx_destroy(abx_ctx *ctx) {
    ctx_release(reinterpret_cast<Ctx *>(ctx));
    return ABX_OK;
}

// ------------------------------------------------------------------ items

int abx_load_items(abx_ctx *ctx_, const float *feats, int64_t n_frames, int32_t dim,
                   const int64_t *item_offsets, int64_t n_items, const int32_t *labels,
                   int32_t n_attr, int32_t mem, void *stream, abx_items **out) {
    Ctx *ctx = reinterpret_cast<Ctx *>(ctx_);
    REQUIRE(ctx && out && item_offsets && labels, ABX_E_INVALID, "NULL argument");
    *out = nullptr;
    REQUIRE(n_items > 0 && n_frames > 0 && dim > 0 && n_attr > 0, ABX_E_INVALID,
            "empty input (n_items=%lld n_frames=%lld dim=%d n_attr=%d)", (long long)n_items,
            (long long)n_frames, dim, n_attr);
    REQUIRE(feats, ABX_E_INVALID, "feats is NULL");
    REQUIRE(mem >= ABX_MEM_HOST && mem <= ABX_MEM_DEVICE_BORROW, ABX_E_INVALID, "bad mem %d", mem);
    REQUIRE(n_items < (1LL << 31) - 1 && n_frames < (1LL << 31) - 1, ABX_E_UNSUPPORTED,
            "more than 2^31 items or frames");
    REQUIRE(dim <= 8192, ABX_E_UNSUPPORTED, "dim %d > 8192", dim);
    REQUIRE(item_offsets[0] == 0 && item_offsets[n_items] == n_frames, ABX_E_INVALID,
            "item_offsets must start at 0 and end at n_frames");
    Trace tr("load_items");
    // range checks as branch-free min/max passes (vectorisable); the slow
    // search for the offending entry runs only when one fails
    int64_t t_min = INT64_MAX, t_max = 0;
    for (int64_t i = 0; i < n_items; ++i) {
        const int64_t T = item_offsets[i + 1] - item_offsets[i];
        t_min = std::min(t_min, T);
        t_max = std::max(t_max, T);
    }
    if (t_min < 1 || t_max > kMaxItemLen)
        for (int64_t i = 0; i < n_items; ++i) {
            const int64_t T = item_offsets[i + 1] - item_offsets[i];
            REQUIRE(T >= 1, ABX_E_INVALID, "item %lld is empty", (long long)i);
            REQUIRE(T <= kMaxItemLen, ABX_E_UNSUPPORTED, "item %lld has %lld frames (> %d)",
                    (long long)i, (long long)T, kMaxItemLen);
        }
    const int32_t max_len = (int32_t)t_max;
    std::vector<int32_t> label_max(n_attr, 0);
    int32_t l_min = INT32_MAX;
    const int64_t n_lab = n_items * n_attr;
    for (int64_t i = 0; i < n_lab; ++i) l_min = std::min(l_min, labels[i]);
    if (l_min < 0)
        for (int64_t i = 0; i < n_lab; ++i)
            REQUIRE(labels[i] >= 0, ABX_E_INVALID, "negative label code at %lld", (long long)i);
    for (int32_t k = 0; k < n_attr; ++k) {
        int32_t m = 0;
        for (int64_t i = k; i < n_lab; i += n_attr) m = std::max(m, labels[i]);
        label_max[k] = m;
    }
    tr.mark("validate");
    cudaStream_t s = (cudaStream_t)stream;
    CU(cudaSetDevice(ctx->device));
    if (mem != ABX_MEM_HOST) {
        cudaPointerAttributes pa;
        CU(cudaPointerGetAttributes(&pa, feats));
        REQUIRE(pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged,
                ABX_E_INVALID, "mem says device but feats is not device memory");
    }
    std::unique_ptr<Items> it(new (std::nothrow) Items);
    REQUIRE(it, ABX_E_OOM, "host allocation failed");
    it->ctx = ctx;
    it->stream = s;
    it->n_items = n_items;
    it->n_frames = n_frames;
    it->dim = dim;
    it->n_attr = n_attr;
    it->max_len = max_len;
    it->label_max.swap(label_max);
    it->h_offsets.assign(item_offsets, item_offsets + n_items + 1);
    tr.mark("host copy");
    size_t fbytes = (size_t)n_frames * dim * sizeof(float);
    if (mem == ABX_MEM_DEVICE_BORROW) {
        it->d_feats = feats;
        it->owns_feats = false;
    } else {
        float *buf = nullptr;
        CU(cudaMallocAsync((void **)&buf, fbytes, s));
        // copied in pieces: a copy engine serves the queued copies of all
        // streams in turn, so the small uploads of kernels running meanwhile
        // on other streams wait for one piece, not for the whole feature set
        const size_t piece = (size_t)32 << 20;
        cudaError_t e = cudaSuccess;
        for (size_t o = 0; o < fbytes && e == cudaSuccess; o += piece)
            e = cudaMemcpyAsync((uint8_t *)buf + o, (const uint8_t *)feats + o,
                                std::min(piece, fbytes - o),
                                mem == ABX_MEM_HOST ? cudaMemcpyHostToDevice
                                                    : cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess && mem == ABX_MEM_HOST) {
            std::lock_guard<std::mutex> g(ctx->copy_mu);
            if (!ctx->feat_copy)
                e = cudaEventCreateWithFlags(&ctx->feat_copy, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventRecord(ctx->feat_copy, s);
        }
        if (e != cudaSuccess) {
            cudaFreeAsync(buf, s);
            set_error("feature copy failed: %s", cudaGetErrorString(e));
            return ABX_E_CUDA;
        }
        it->d_feats = buf;
        it->owns_feats = true;
    }
    Staging st;
    // the labels go to the device straight from the caller's buffer (the
    // host keeps only their code ranges)
    size_t o_off = st.add(it->h_offsets),
           o_lab = st.add_raw(labels, (size_t)n_lab * sizeof(int32_t));
    CU(st.commit(ctx, s));
    tr.mark("upload");
    it->d_offsets = st.at<int64_t>(o_off);
    it->d_labels = st.at<int32_t>(o_lab);
    CU(cudaEventCreateWithFlags(&it->ready, cudaEventDisableTiming));
    CU(cudaEventRecord(it->ready, s));
    tr.mark("event");
    ctx_retain(ctx);
    *out = reinterpret_cast<abx_items *>(it.release());
    return ABX_OK;
}

int abx_items_free(abx_items *items_) {
    Items *it = reinterpret_cast<Items *>(items_);
    if (!it) return ABX_OK;
    cudaSetDevice(it->ctx->device);
    PackedRows *pr = it->pack;
    it->pack = nullptr;
    packed_rows_release(it, pr, it->stream);
    if (it->owns_feats && it->d_feats) cudaFreeAsync((void *)it->d_feats, it->stream);
    if (it->d_offsets) cudaFreeAsync(it->d_offsets, it->stream);
    if (it->ready) cudaEventDestroy(it->ready);
    Ctx *ctx = it->ctx;
    delete it;
    ctx_release(ctx);
    return ABX_OK;
}

// ------------------------------------------------------------------ cells

int abx_build_cells(abx_ctx *ctx_, const abx_items *items_, int32_t on_attr, const int32_t *by,
                    int32_t n_by, int32_t across_attr, abx_cells **out) {
    Ctx *ctx = reinterpret_cast<Ctx *>(ctx_);
    const Items *it = reinterpret_cast<const Items *>(items_);
    REQUIRE(ctx && it && out, ABX_E_INVALID, "NULL argument");
    REQUIRE(it->ctx == ctx, ABX_E_STATE, "items belong to another context");
    *out = nullptr;
    REQUIRE(n_by >= 0 && n_by <= 8 && (n_by == 0 || by), ABX_E_INVALID, "bad by list");
    const int A = it->n_attr;
    REQUIRE(on_attr >= 0 && on_attr < A, ABX_E_INVALID, "on attribute %d out of range", on_attr);
    REQUIRE(across_attr >= -1 && across_attr < A, ABX_E_INVALID, "across attribute out of range");
    REQUIRE(across_attr != on_attr, ABX_E_INVALID, "across equals on");
    for (int i = 0; i < n_by; ++i) {
        REQUIRE(by[i] >= 0 && by[i] < A, ABX_E_INVALID, "by attribute %d out of range", by[i]);
        REQUIRE(by[i] != on_attr && by[i] != across_attr, ABX_E_INVALID,
                "by attribute %d repeats on/across", by[i]);
        for (int j = 0; j < i; ++j)
            REQUIRE(by[i] != by[j], ABX_E_INVALID, "by attribute %d listed twice", by[i]);
    }
    Trace tr("build_cells");
    std::unique_ptr<Cells> c(new (std::nothrow) Cells);
    REQUIRE(c, ABX_E_OOM, "host allocation failed");
    c->ctx = ctx;
    c->items = it;
    c->stream = it->stream;
    c->on = on_attr;
    c->across = across_attr;
    c->by.assign(by, by + n_by);
    const int64_t n = it->n_items;
    // code ranges of the attributes (largest codes, from abx_load_items)
    const std::vector<int32_t> &mx = it->label_max;
    c->K_on = mx[on_attr] + 1;
    c->K_s = across_attr >= 0 ? mx[across_attr] + 1 : 1;
    c->by_space = 1;
    for (int i = 0; i < n_by; ++i) {
        c->K_by.push_back(mx[by[i]] + 1);
        c->by_space *= c->K_by.back();
        REQUIRE(c->by_space <= (1LL << 26), ABX_E_UNSUPPORTED,
                "product of by-attribute code ranges exceeds 2^26");
    }
    const int64_t K_on = c->K_on, K_s = c->K_s;
    const int64_t g_max = std::min<int64_t>(c->by_space, n);
    const int64_t nkeys_max = g_max * K_s * K_on;
    REQUIRE(nkeys_max <= (1LL << 28), ABX_E_UNSUPPORTED,
            "groups x on codes x across codes exceeds 2^28");
    tr.mark("ranges");
    CU(cudaSetDevice(ctx->device));
    // the tables are built on the device on a stream of this thread, apart
    // from the caller's stream (which may be busy with earlier tasks)
    cudaStream_t bs = build_stream(ctx->device);
    CU(cudaStreamWaitEvent(bs, it->ready, 0));
    // kept block: sorted-item arrays and tables
    auto al = [](int64_t b) { return (b + 255) / 256 * 256; };
    const int64_t o_id = 0, o_ig = o_id + al(n * 4), o_ip = o_ig + al(n * 4),
                  o_is = o_ip + al(n * 4), o_gb = o_is + al(n * 4),
                  o_dm = o_gb + al((g_max + 1) * 4), o_blk = o_dm + al(g_max * 8),
                  o_tot = o_blk + al(nkeys_max * 8), o_gt = o_tot + al(g_max * K_s * 4),
                  o_gm = o_gt + al(c->by_space * 4), o_end = o_gm + al(g_max * 16);
    CU(cudaMallocAsync((void **)&c->d_block, o_end, bs));
    uint8_t *kb = c->d_block;
    c->d_item_id = reinterpret_cast<int32_t *>(kb + o_id);
    c->d_item_g = reinterpret_cast<int32_t *>(kb + o_ig);
    c->d_item_p = reinterpret_cast<int32_t *>(kb + o_ip);
    c->d_item_s = reinterpret_cast<int32_t *>(kb + o_is);
    c->d_group_begin = reinterpret_cast<int32_t *>(kb + o_gb);
    c->d_group_dm = reinterpret_cast<int64_t *>(kb + o_dm);
    c->d_blk = reinterpret_cast<int2 *>(kb + o_blk);
    c->d_tot = reinterpret_cast<int32_t *>(kb + o_tot);
    c->d_gtab = reinterpret_cast<int32_t *>(kb + o_gt);
    c->d_gmeta = reinterpret_cast<int4 *>(kb + o_gm);
    // scratch block
    const int64_t s_fl = 0, s_gp = s_fl + al(c->by_space * 4), s_cn = s_gp + al((c->by_space + 1) * 8),
                  s_ps = s_cn + al(nkeys_max * 4), s_cu = s_ps + al((nkeys_max + 1) * 8),
                  s_ky = s_cu + al(nkeys_max * 8), s_n2 = s_ky + al(n * 8),
                  s_ig = s_n2 + al(g_max * 4), s_sc = s_ig + al(n * 4), s_nz = s_sc + al(8 * 8),
                  s_end = s_nz + al(g_max * K_s * 4);
    uint8_t *sb = nullptr;
    CU(cudaMallocAsync((void **)&sb, s_end, bs));
    CellBuildArgs ca;
    memset(&ca, 0, sizeof(ca));
    ca.labels = it->d_labels;
    ca.n = n;
    ca.n_attr = A;
    ca.on = on_attr;
    ca.across = across_attr;
    ca.n_by = n_by;
    for (int i = 0; i < n_by; ++i) {
        ca.by[i] = by[i];
        ca.K_by[i] = c->K_by[i];
    }
    ca.K_on = (int32_t)K_on;
    ca.K_s = (int32_t)K_s;
    ca.by_space = c->by_space;
    ca.flags = reinterpret_cast<int32_t *>(sb + s_fl);
    ca.gpos = reinterpret_cast<int64_t *>(sb + s_gp);
    ca.counts = reinterpret_cast<int32_t *>(sb + s_cn);
    ca.pos = reinterpret_cast<int64_t *>(sb + s_ps);
    ca.cursor = reinterpret_cast<int64_t *>(sb + s_cu);
    ca.key = reinterpret_cast<int64_t *>(sb + s_ky);
    ca.ng2 = reinterpret_cast<int32_t *>(sb + s_n2);
    ca.item_group = reinterpret_cast<int32_t *>(sb + s_ig);
    ca.nz_s = reinterpret_cast<int32_t *>(sb + s_nz);
    // scalars: [0] groups, [1] matrix total, [2..4] scan scratch, [5] candidates
    int64_t *scal = reinterpret_cast<int64_t *>(sb + s_sc);
    ca.n_groups = scal;
    ca.dm_total = scal + 1;
    ca.n_cand = scal + 5;
    ca.gtab = c->d_gtab;
    ca.item_id = c->d_item_id;
    ca.blk = c->d_blk;
    ca.tot = c->d_tot;
    ca.group_begin = c->d_group_begin;
    ca.group_dm = c->d_group_dm;
    ca.gmeta = c->d_gmeta;
    CU(launch_cell_build(ca, nkeys_max, g_max, scal + 2, bs));
    ItemAttrArgs ia;
    ia.item_id = c->d_item_id;
    ia.labels = it->d_labels;
    ia.gtab = c->d_gtab;
    ia.n_items = (int32_t)n;
    ia.n_attr = A;
    ia.on = on_attr;
    ia.across = across_attr;
    ia.n_by = n_by;
    for (int b = 0; b < n_by; ++b) {
        ia.by[b] = by[b];
        ia.K_by[b] = c->K_by[b];
    }
    ia.item_g = c->d_item_g;
    ia.item_p = c->d_item_p;
    ia.item_s = c->d_item_s;
    CU(launch_item_attrs(ia, bs));
    // what the host plans with: group count, matrix total, group ranges,
    // sorted order, group of each item
    const size_t hs = 6 * sizeof(int64_t);
    const size_t hb = hs + (size_t)(g_max + 1) * 4 + (size_t)n * 8;
    uint8_t *pin = (uint8_t *)ctx->pinned.acquire(hb);
    REQUIRE(pin, ABX_E_OOM, "pinned host allocation failed");
    CU(cudaMemcpyAsync(pin, scal, hs, cudaMemcpyDeviceToHost, bs));
    CU(cudaMemcpyAsync(pin + hs, c->d_group_begin, (g_max + 1) * 4, cudaMemcpyDeviceToHost, bs));
    CU(cudaMemcpyAsync(pin + hs + (g_max + 1) * 4, c->d_item_id, n * 4, cudaMemcpyDeviceToHost,
                       bs));
    CU(cudaMemcpyAsync(pin + hs + (g_max + 1) * 4 + n * 4, ca.item_group, n * 4,
                       cudaMemcpyDeviceToHost, bs));
    CU(cudaEventCreateWithFlags(&c->ready, cudaEventDisableTiming));
    CU(cudaEventRecord(c->ready, bs));
    cudaFreeAsync(sb, bs);
    CU(cudaStreamSynchronize(bs));
    tr.mark("device build");
    const int64_t *sc = reinterpret_cast<const int64_t *>(pin);
    const int32_t G = (int32_t)sc[0];
    c->n_groups = G;
    c->dm_entries = sc[1];
    c->n_cand = sc[5];
    const int32_t *gb = reinterpret_cast<const int32_t *>(pin + hs);
    c->group_begin.assign(gb, gb + G + 1);
    const int32_t *ids = reinterpret_cast<const int32_t *>(pin + hs + (g_max + 1) * 4);
    c->item_id.assign(ids, ids + n);
    const int32_t *igp = ids + n;
    c->item_group.assign(igp, igp + n);
    ctx->pinned.release(pin, bs);
    c->group_dm.resize(G);
    int64_t dm = 0;
    for (int32_t g = 0; g < G; ++g) {
        const int64_t ng = c->group_begin[g + 1] - c->group_begin[g];
        c->group_dm[g] = dm;
        dm += ng * ng;
    }
    c->info.n_items = n;
    c->info.n_groups = G;
    c->stream = it->stream;  // later work and the frees follow the caller's stream
    tr.mark("host tables");
    ctx_retain(ctx);
    *out = reinterpret_cast<abx_cells *>(c.release());
    return ABX_OK;
}

}  // extern "C"

// Counts of blocks, cells and triples from the block table (Sec. 2
// definitions), computed on first request: O(groups x on x across codes)
// with per-(group, across) and per-(group, on) totals and non-empty counts.
void abx::Cells::compute_info() {
    if (info_done) return;
    if (blk.empty()) {  // the block table lives on the device; fetch it once
        cudaSetDevice(ctx->device);
        cudaEventSynchronize(ready);
        blk.resize((size_t)n_groups * K_s * K_on);
        tot.resize((size_t)n_groups * K_s);
        cudaMemcpy(blk.data(), d_blk, blk.size() * sizeof(int2), cudaMemcpyDeviceToHost);
        cudaMemcpy(tot.data(), d_tot, tot.size() * sizeof(int32_t), cudaMemcpyDeviceToHost);
    }
    const int64_t K_on = this->K_on, K_s = this->K_s;
    int64_t n_cells = 0, n_trip = 0, nblocks = 0, maxg = 0;
    std::vector<int64_t> nz_s(K_s), tot_p(K_on), nz_p(K_on);
    for (int32_t g = 0; g < n_groups; ++g) {
        maxg = std::max<int64_t>(maxg, group_begin[g + 1] - group_begin[g]);
        const int2 *bg = &blk[(size_t)g * K_on * K_s];
        std::fill(nz_s.begin(), nz_s.end(), 0);
        std::fill(tot_p.begin(), tot_p.end(), 0);
        std::fill(nz_p.begin(), nz_p.end(), 0);
        for (int64_t s = 0; s < K_s; ++s)
            for (int64_t p = 0; p < K_on; ++p) {
                const int64_t a = bg[s * K_on + p].y;
                nblocks += a > 0;
                nz_s[s] += a > 0;
                tot_p[p] += a;
                nz_p[p] += a > 0;
            }
        const int32_t *tg = &tot[(size_t)g * K_s];
        for (int64_t s = 0; s < K_s; ++s)
            for (int64_t p = 0; p < K_on; ++p) {
                const int64_t a = bg[s * K_on + p].y;
                if (!a) continue;
                if (across < 0) {
                    if (a < 2) continue;
                    n_cells += nz_s[s] - 1;                 // b from any other on value
                    n_trip += a * (a - 1) * (tg[s] - a);
                } else {
                    n_cells += (nz_s[s] - 1) * (nz_p[p] - 1);   // other on same s, same on other s
                    n_trip += a * (tg[s] - a) * (tot_p[p] - a);
                }
            }
    }
    info.n_blocks = nblocks;
    info.n_cells = n_cells;
    info.n_triplets = n_trip;
    info.max_group = maxg;
    info_done = true;
}

extern "C" {

int abx_cells_get_info(const abx_cells *cells, abx_cells_info *info) {
    REQUIRE(cells && info, ABX_E_INVALID, "NULL argument");
    Cells *c = const_cast<Cells *>(reinterpret_cast<const Cells *>(cells));
    c->compute_info();
    *info = c->info;
    return ABX_OK;
}

int abx_cells_set_subsampler(abx_cells *cells_, int32_t max_size_group, int32_t max_x_across,
                             uint64_t seed) {
    Cells *c = reinterpret_cast<Cells *>(cells_);
    REQUIRE(c, ABX_E_INVALID, "NULL argument");
    REQUIRE(max_size_group >= 0 && max_size_group <= kMaxSubCap, ABX_E_INVALID,
            "max_size_group must be 0..%d", kMaxSubCap);
    REQUIRE(max_x_across >= 0, ABX_E_INVALID, "negative max_x_across");
    c->sub_cap = max_size_group;
    c->sub_xmax = max_x_across;
    c->sub_seed = seed;
    return ABX_OK;
}

int abx_cells_free(abx_cells *cells_) {
    Cells *c = reinterpret_cast<Cells *>(cells_);
    if (!c) return ABX_OK;
    REQUIRE(c->jobs.load() == 0, ABX_E_STATE, "a submitted score of these cells is not waited for");
    cudaSetDevice(c->ctx->device);
    if (c->d_block) cudaFreeAsync(c->d_block, c->stream);
    if (c->ready) cudaEventDestroy(c->ready);
    Ctx *ctx = c->ctx;
    delete c;
    ctx_release(ctx);
    return ABX_OK;
}

// -------------------------------------------------------------- distances

int abx_distances(abx_ctx *ctx_, const abx_items *items_, const abx_cells *cells_, int32_t mode,
                  int32_t precision, void *stream, abx_dist **out) {
    return abx_distances_ex(ctx_, items_, cells_, mode, ABX_DIST_ANGULAR, precision, stream, out);
}

int abx_distances_ex(abx_ctx *ctx_, const abx_items *items_, const abx_cells *cells_,
                     int32_t mode, int32_t distance, int32_t precision, void *stream,
                     abx_dist **out) {
    Ctx *ctx = reinterpret_cast<Ctx *>(ctx_);
    const Items *it = reinterpret_cast<const Items *>(items_);
    const Cells *c = reinterpret_cast<const Cells *>(cells_);
    REQUIRE(ctx && it && c && out, ABX_E_INVALID, "NULL argument");
    REQUIRE(it->ctx == ctx && c->ctx == ctx && c->items == it, ABX_E_STATE,
            "objects from different contexts or items");
    *out = nullptr;
    Trace tr("distances");
    cudaStream_t s = (cudaStream_t)stream;
    CU(cudaSetDevice(ctx->device));
    std::unique_ptr<Dist> d(new (std::nothrow) Dist);
    REQUIRE(d, ABX_E_OOM, "host allocation failed");
    // the pack is enqueued before the tile planning, so it runs while the
    // host plans panels and tiles; its result is kept with the items for
    // later tasks of the same item order
    DistPlan p;
    p.share_pack = true;
    p.use_scratch = true;
    int rc = dist_plan_build_rows(ctx, it, c, mode, distance, precision, s, &p);
    if (!rc) rc = dist_plan_exec_pack(p, s);
    if (!rc && !p.pack_hit) rc = publish_pack(it, c, p, s);
    tr.mark(p.pack_hit ? "rows (packed)" : "rows+pack");
    if (!rc) rc = dist_plan_build_tiles(s, &p);
    tr.mark("plan+upload");
    if (!rc) rc = dist_plan_exec_tiles(p, s);
    if (!rc && p.shared) rc = note_pack_use(it, p.shared, s);
    if (rc) {
        dist_plan_free(&p, s, true);
        return rc;
    }
    d->ctx = ctx;
    d->items = it;
    d->cells = c;
    d->stream = s;
    d->mode = mode;
    d->precision = precision;
    d->distance = distance;
    d->max_len = p.max_len;
    d->pair_cap = p.cap_total;
    d->info.n_tiles = p.n_tiles;
    d->info.n_frames = p.rows;
    d->info.mode = mode;
    d->info.precision = precision;
    d->info.distance = distance;
    // the persistent buffers move to the Dist
    d->d_block = p.keep_block;
    d->d_len = p.d_len;
    d->d_row = p.d_row;
    d->d_pv = p.pv;
    d->d_err = p.d_err;
    d->d_count = p.d_count;
    p.keep_block = nullptr;
    p.pv = nullptr;
    p.d_err = nullptr;
    p.d_count = nullptr;
    dist_plan_free(&p, s, false);
    d->h_mirror = ctx->pinned.acquire(64);
    REQUIRE(d->h_mirror, ABX_E_OOM, "pinned host allocation failed");
    d->h_err = reinterpret_cast<int32_t *>(d->h_mirror);
    d->h_count = reinterpret_cast<int64_t *>((uint8_t *)d->h_mirror + 16);
    CU(cudaMemcpyAsync(d->h_err, d->d_err, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(d->h_count, d->d_count, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CU(cudaEventCreateWithFlags(&d->done, cudaEventDisableTiming));
    CU(cudaEventRecord(d->done, s));
    tr.mark("enqueue");
    CU(cudaGetLastError());
    ctx_retain(ctx);
    *out = reinterpret_cast<abx_dist *>(d.release());
    return ABX_OK;
}

int abx_dist_sync(abx_dist *dist_) {
    Dist *d = reinterpret_cast<Dist *>(dist_);
    REQUIRE(d, ABX_E_INVALID, "NULL argument");
    CU(cudaSetDevice(d->ctx->device));
    // the distance work only (the event follows the counters' copies), not
    // whatever the caller enqueued on the stream since
    CU(cudaEventSynchronize(d->done));
    if (!d->synced) {
        d->synced = true;
        d->n_pairs = d->h_count[0];
        d->info.n_pairs = d->h_count[0];
        d->info.n_frame_pairs = d->h_count[1];
    }
    REQUIRE(!(d->h_err[0] & kPackNonPositive), ABX_E_INVALID,
            "the KL distance needs every frame component > 0");
    REQUIRE(!(d->h_err[0] & kPackZeroNorm), ABX_E_ZERO_NORM,
            "a frame has zero L2 norm (angle undefined)");
    REQUIRE(d->h_err[1] == 0, ABX_E_CUDA, "tile kernel pipeline wait expired (code %d)",
            d->h_err[1]);
    return ABX_OK;
}

int abx_dist_get_info(abx_dist *dist_, abx_dist_info *info) {
    Dist *d = reinterpret_cast<Dist *>(dist_);
    REQUIRE(d && info, ABX_E_INVALID, "NULL argument");
    int rc = abx_dist_sync(dist_);
    *info = d->info;
    return rc;
}

int abx_dist_lookup(abx_dist *dist_, int64_t n, const int64_t *x, const int64_t *y, float *dv,
                    float *lov, float *hiv, int32_t *lenv) {
    Dist *d = reinterpret_cast<Dist *>(dist_);
    REQUIRE(d && (n == 0 || (x && y)), ABX_E_INVALID, "NULL argument");
    int rc = abx_dist_sync(dist_);
    if (rc) return rc;
    if (n == 0) return ABX_OK;
    const Cells *c = d->cells;
    std::vector<int32_t> pos(c->info.n_items);
    for (int64_t k = 0; k < c->info.n_items; ++k) pos[c->item_id[k]] = (int32_t)k;
    std::vector<int64_t> ent(n);
    for (int64_t q = 0; q < n; ++q) {
        REQUIRE(x[q] >= 0 && x[q] < c->info.n_items && y[q] >= 0 && y[q] < c->info.n_items,
                ABX_E_INVALID, "pair %lld out of range", (long long)q);
        int32_t kx = pos[x[q]], ky = pos[y[q]];
        int32_t g = c->item_group[x[q]];
        ent[q] = -1;
        if (g == c->item_group[y[q]] && kx != ky) {
            int64_t ng = c->group_begin[g + 1] - c->group_begin[g];
            ent[q] = c->group_dm[g] + (int64_t)(kx - c->group_begin[g]) * ng + (ky - c->group_begin[g]);
        }
    }
    int64_t *d_ent = nullptr;
    float *o = nullptr;
    int32_t *oL = nullptr;
    cudaStream_t s = d->stream;
    CU(cudaMallocAsync((void **)&d_ent, n * sizeof(int64_t), s));
    CU(cudaMallocAsync((void **)&o, 3 * n * sizeof(float), s));
    CU(cudaMallocAsync((void **)&oL, n * sizeof(int32_t), s));
    CU(cudaMemcpyAsync(d_ent, ent.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    CU(launch_gather(d->d_pv, d_ent, n, o, o + n, o + 2 * n, oL, s));
    std::vector<float> h(3 * n);
    std::vector<int32_t> hL(n);
    CU(cudaMemcpyAsync(h.data(), o, 3 * n * sizeof(float), cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(hL.data(), oL, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    cudaFreeAsync(d_ent, s);
    cudaFreeAsync(o, s);
    cudaFreeAsync(oL, s);
    CU(cudaStreamSynchronize(s));
    for (int64_t q = 0; q < n; ++q) {
        if (dv) dv[q] = h[q];
        if (lov) lov[q] = h[n + q];
        if (hiv) hiv[q] = h[2 * n + q];
        if (lenv) lenv[q] = hL[q];
    }
    return ABX_OK;
}

int abx_dist_free(abx_dist *dist_) {
    Dist *d = reinterpret_cast<Dist *>(dist_);
    if (!d) return ABX_OK;
    REQUIRE(d->jobs.load() == 0, ABX_E_STATE,
            "a submitted score of these distances is not waited for");
    cudaSetDevice(d->ctx->device);
    cudaStream_t s = d->stream;
    for (void *p : {(void *)d->d_block, (void *)d->d_pv,
                    (void *)d->d_err, (void *)d->d_count})
        if (p) cudaFreeAsync(p, s);
    if (d->h_mirror) d->ctx->pinned.release(d->h_mirror, s);
    if (d->done) cudaEventDestroy(d->done);
    Ctx *ctx = d->ctx;
    delete d;
    ctx_release(ctx);
    return ABX_OK;
}

}  // extern "C"
