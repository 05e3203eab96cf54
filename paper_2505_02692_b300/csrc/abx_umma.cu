// tcgen05 tensor-core kernels for the frame distances (fastabx Sec. 3.1
// "angular", Sec. 3.2): every 128 x 128 tile of frame cosines
// <q_i, q_j> |q_i|^-1 |q_j|^-1 is accumulated in TMEM by M = 128 UMMAs and
// turned into d = arccos(c) / pi by an epilogue.
//
// Precisions (operands K-major, staged by TMA with 128-byte swizzle):
//   ABX_FP32  frames (scaled by a power of two) split as hi + lo, two FP16
//             halves; per k step one N = 256 kind::f16 MMA of A_hi against
//             [B_hi | B_lo] (hi*hi into the main accumulator, hi*lo into the
//             cross accumulator beside it) and one N = 128 MMA of A_lo against
//             B_hi (lo*hi into the cross accumulator); FP32 accumulation; the
//             epilogue adds the two (the dropped lo*lo term is at most 2^-22
//             of |u||v|).
//   ABX_BF16  one kind::f16 MMA per k step (BF16 operands, FP32 accumulation).
//   ABX_FP8   one kind::f8f6f4 MMA per k step (E4M3 operands, FP32 accumulation).
//
// Kernels, all persistent with one CTA per SM:
//   umma_tile_kernel   ("narrow"; the FP32 split's default) writes the
//       blocks of the pairs the planner listed (its per-tile store map,
//       launch_plan_count) of each 128 x 128 distance tile to a global tile
//       buffer for the stand-alone DTW kernel, column-major or, with
//       ABX_TILE_LAYOUT=1, in strips (tile_strip_offset: each pair's block
//       contiguous); 16 epilogue warps (8 in the split's variant 2).
//   umma_wide_kernel   (BF16 / FP8; variant 3, the default, with 16
//       epilogue warps, variant 2 with 8) a tile and its neighbour in the
//       panel row as one N = 256 MMA, every entry written to column-major
//       tiles (its epilogue sets its pace, so it does no store-map work).
//   umma_pair_kernel   (FP32 split, variant 4) narrow tiles on clusters of
//       two CTAs that share their row panel by TMA multicast.
//   umma_fused_kernel  (opt-in, items of up to kFuseMaxLen frames) the
//       tile's frame distances go to a shared-memory d tile and the CTA's 16
//       epilogue warps run the DTW of every needed item pair of the tile on
//       it while the MMAs of the next tile run: no tile buffer in global
//       memory.  ABX_FUSE=1: a thread per pair, in place (dtw_inplace);
//       ABX_FUSE=2: 8-lane anti-diagonal wavefronts (dtw_wave8).  Both
//       measured slower than the two-kernel path: the serial chain of a
//       tile's longest pair, not the MMAs, sets their pace.
// Warp roles: warp 0 the TMA producer (one lane), warp 1 the TMEM owner and
// MMA issuer (one lane), the rest epilogue warps (tcgen05.ld of the TMEM lane
// quarter their warp index allows).  Two TMEM accumulators let the epilogue
// of one tile run under the MMAs of the next.  Every mbarrier wait is
// bounded; on expiry the kernel records an error code, stops issuing work
// and still releases TMEM.
#include <cuda.h>
#include <algorithm>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "abx_dtw_cell.cuh"
#include "abx_internal.h"

namespace abx {
namespace {


constexpr int kFuseWarps = 16;                  // fused kernel: epilogue + DTW warps
constexpr int kFuseEpiThreads = 32 * kFuseWarps;
constexpr int kFuseThreads = 32 * (2 + kFuseWarps);
constexpr int kFuseGroups = 4 * kFuseWarps;     // 8-lane DTW groups
constexpr int kFuseMaxLen = 40;                 // longest item the fused kernel takes
// Row stride of the shared d tile (floats).  Even, so that a group's lanes,
// which walk an anti-diagonal (row + 1, column - 1 per lane), hit addresses
// kDS - 1 (odd) apart, i.e. distinct banks, and float2 stores stay aligned.
constexpr int kDS = kPanel + 2;
constexpr int kTileBytes = kPanel * 128;        // one 128-row x 128-byte operand tile
// TMEM columns: two buffers of one 128-column FP32 accumulator, or for the
// FP32 split two (hi*hi and hi*lo + lo*hi) per buffer
template <int PREC>
constexpr uint32_t tmem_cols() { return PREC == ABX_FP32 ? 512u : 256u; }
template <int PREC>
constexpr uint32_t acc_stride() { return PREC == ABX_FP32 ? 256u : 128u; }
constexpr long long kWaitCycles = 4000000000LL; // ~2 s at 2 GHz

struct UmmaParams {
    const float *inv_norm;
    int64_t n_rows;
    int32_t n_kchunks;     // 128-byte k-chunks per row
    int32_t lo_offset;     // element offset of the lo half (FP32 split), else 0
    int32_t b_rot;         // B operand's k offset in elements, modulo k_elems (KL)
    int32_t k_elems;       // elements of k per row (the hi half for the split)
    const int2 *tiles;
    const int32_t *panel_row;
    const int32_t *tile_count;
    int64_t n_tiles;
    float *tilebuf;
    int32_t *err;
    int32_t distance;
    const float *nrm2;
    // DTW of the fused kernel
    const int4 *pairs;
    const int64_t *tile_base;
    const int32_t *len;
    const float *theta_item;
    float eps_c;
    int32_t intervals;
    const int32_t *item_g;
    const int4 *gmeta;
    PairVal *pv;
    // wide kernel: work items (tile, adjacent tile or -1)
    const int2 *work;
    int64_t n_work;
    // tile buffer strips: packed row -> item, item -> first row, panel ->
    // first item, and the per-tile store map (launch_plan_count)
    const int32_t *row_item;
    const int32_t *row;
    const int32_t *panel_item;
    const uint64_t *xmask;
    const uint8_t *col_yo;
    int32_t strips;        // tile buffer layout: 1 strips, 0 column-major tiles
    int32_t listed_only;   // 1: store only the listed pairs' blocks, 0: every entry
};

// Named barrier 1 over the NT epilogue threads only; returns the OR of `flag`.
template <int NT>
__device__ __forceinline__ bool epi_bar_or(bool flag) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n"
        " bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}"
        : "=r"(r)
        : "r"((uint32_t)flag), "r"(NT)
        : "memory");
    return r != 0;
}

template <int NT>
__device__ __forceinline__ void epi_bar() {
    asm volatile("bar.sync 1, %0;" ::"r"(NT) : "memory");
}

// ------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: returns false (and records `code`) if the phase never completes.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int32_t *err,
                                          int code) {
    if (mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try(bar, parity)) {
        if (clock64() - t0 > kWaitCycles) {
            atomicCAS(err, 0, code);
            return false;
        }
        if (*(volatile int32_t *)err) return false;
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int32_t x, int32_t y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// The same load delivered to the CTAs of the cluster in ctaMask: the tile
// lands at this shared-memory offset in each of them and completes the
// transaction bytes of the barrier at this offset in each.
__device__ __forceinline__ void tma_load_2d_mc(void *dst, const CUtensorMap *map, uint64_t *bar,
                                               int32_t x, int32_t y, uint16_t mask) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        ".multicast::cluster [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar)), "h"(mask)
        : "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_id() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_count() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}
// Every thread of every CTA of the cluster (release / acquire).
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release;\nbarrier.cluster.wait.acquire;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row
// atoms 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;              // leading byte offset (unused for SW128 K-major)
    d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset
    d |= (uint64_t)1 << 46;              // version
    d |= (uint64_t)2 << 61;              // 128-byte swizzle
    return d;
}

template <int KIND>  // 0 = kind::f16, 1 = kind::f8f6f4
__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                     uint32_t accumulate) {
    if (KIND == 0)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
            "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
    else
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
            "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

// Arrives on the barrier at this offset in each CTA of ctaMask once the
// MMAs this thread issued before are complete.
__device__ __forceinline__ void umma_commit_mc(uint64_t *bar, uint16_t mask) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
        " [%0], %1;" ::"r"(smem_u32(bar)),
        "h"(mask)
        : "memory");
}

__device__ __forceinline__ void fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Frame distance from x = <q_a, q_b> |q_a|^-1 |q_b|^-1 (Euclidean: the raw
// inner product; KL: the rotated contraction <p_a, ln p_b> + <ln p_a, p_b>)
// and, for Euclidean and KL, the rows' squared norms or sums p ln p na, nb.
template <int DIST>
__device__ __forceinline__ float frame_dist(float x, float na, float nb) {
    if (DIST == ABX_DIST_KL) return fmaxf(0.0f, 0.5f * (na + nb - x));
    if (DIST == ABX_DIST_EUCLIDEAN) return sqrtf(fmaxf(0.0f, na + nb - 2.0f * x));
    if (DIST == ABX_DIST_COSINE) return 1.0f - fminf(1.0f, fmaxf(-1.0f, x));
    return acosf(fminf(1.0f, fmaxf(-1.0f, x))) * 0.318309886183790671f;
}

// 8 consecutive columns of the warp's TMEM lane quarter (one per lane row).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float *v) {
    uint32_t r[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Epilogue of the wide kernel: NC accumulator columns of one row, dot
// products -> frame distances, every entry stored in the column-major tile
// (out[c * 128]).  ia: the row's 1/|a| (1/scale for Euclidean); na: its
// squared norm or sum p ln p; columns cb.. with their 1/|b| and nb.  With the
// BF16 / FP8 products the epilogue, not the MMAs, sets this kernel's pace,
// and any work added to it (the narrow kernel's store map below) measured
// slower: 3.5 -> 4.8 ms per triphone-scale step.
template <int DIST, int NC>
__device__ __forceinline__ void epi_row(const float (&v)[NC], float ia, float na, int64_t cb,
                                        int64_t n_rows, const float *__restrict__ inv_norm,
                                        const float *__restrict__ nrm2, float *out) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const bool cv = cb + c < n_rows;
        const float ib = cv ? __ldg(inv_norm + cb + c) : 0.0f;
        const float nb = (DIST == ABX_DIST_KL || DIST == ABX_DIST_EUCLIDEAN) && cv
                             ? __ldg(nrm2 + cb + c)
                             : 0.0f;
        out[c * kPanel] = frame_dist<DIST>(v[c] * ia * ib, na, nb);
    }
}

// One accumulator row of a tile in the tile buffer (narrow and pair
// kernels): out indexes the row's entry of tile column 0 (kNoRow for a row
// past the panel's last item) and ld is the distance between its columns, in
// a column-major tile (ld = 128) or in the strip of its item x
// (tile_strip_offset: ld = Tx); mask has bit yo set for each column item yo
// whose block with x is stored (all set when every entry is stored, or when
// the column panel has more than 64 items); ia / na are the row's 1/|a|
// (1/scale for Euclidean) and squared norm or sum p ln p.
struct StripRow {
    uint32_t out;  // tile buffer index of (row, column 0), or kNoRow
    int ld;
    uint64_t mask;
    float ia, na;
};
constexpr uint32_t kNoRow = 0xffffffffu;  // a chunk holds fewer than 2^32 / 16384 tiles

__device__ __forceinline__ StripRow strip_row(const UmmaParams &p, int64_t t, int2 pp, int row) {
    StripRow r{kNoRow, kPanel, 0ull, 0.0f, 0.0f};
    const int64_t ra = p.panel_row[pp.x] + row;
    if (ra >= p.n_rows) return r;
    const int x = __ldg(p.row_item + ra);
    const int xa = __ldg(p.panel_item + pp.x);
    if (x >= __ldg(p.panel_item + pp.x + 1)) return r;
    const int mj = __ldg(p.panel_item + pp.y + 1) - __ldg(p.panel_item + pp.y);
    if (p.strips) {
        const int rx = __ldg(p.row + x) - p.panel_row[pp.x];
        r.ld = __ldg(p.len + x);
        r.out = (uint32_t)(t * (int64_t)(kPanel * kPanel) + tile_strip_offset(rx, r.ld, row, 0));
    } else {
        r.ld = kPanel;
        r.out = (uint32_t)(t * (int64_t)(kPanel * kPanel) + row);
    }
    r.mask = p.listed_only && mj <= 64 ? __ldg(p.xmask + t * kPanel + (x - xa)) : ~0ull;
    r.ia = p.inv_norm[ra];
    r.na = (p.distance == ABX_DIST_KL || p.distance == ABX_DIST_EUCLIDEAN) ? p.nrm2[ra] : 0.0f;
    return r;
}

// A tile's column -> column item bytes for NC columns from tile column c0
// (one 16-byte load per 16 columns, the same address for every lane).
template <int NC>
struct ColMap {
    uint4 w[NC / 16];
};

template <int NC>
__device__ __forceinline__ ColMap<NC> col_map(const UmmaParams &p, int64_t t, int c0) {
    ColMap<NC> m;
    const uint4 *cm = reinterpret_cast<const uint4 *>(p.col_yo + t * kPanel + c0);
#pragma unroll
    for (int i = 0; i < NC / 16; ++i) m.w[i] = __ldg(cm + i);
    return m;
}

// Epilogue of NC accumulator columns of one row (tile columns c0 ..,
// packed rows cb ..) of the narrow and pair kernels: dot products -> frame
// distances, computed and stored only in the blocks of the tile's listed
// pairs (the only blocks the DTW reads) unless every entry is stored.  The
// kernels fetch the row's StripRow and the column map before they wait for
// the accumulator, so that these loads overlap the MMAs.  (With the column's
// norm load and distance outside the branch and only the store predicated,
// the FP32 split step measured 0.3 ms slower.)
template <int DIST, int NC>
__device__ __forceinline__ void epi_strip(const float (&v)[NC], const StripRow &r,
                                          const ColMap<NC> &m, int64_t cb, int c0,
                                          const UmmaParams &p) {
    if (r.out == kNoRow) return;
    float *out = p.tilebuf + r.out;
#pragma unroll
    for (int c16 = 0; c16 < NC; c16 += 16) {
        const uint4 m4 = m.w[c16 / 16];
        const uint32_t mw[4] = {m4.x, m4.y, m4.z, m4.w};
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int c = c16 + k;
            const uint32_t yo = (mw[k >> 2] >> (8 * (k & 3))) & 0xffu;
            if (yo != 255u && ((r.mask >> (yo & 63u)) & 1ull)) {
                const float ib = __ldg(p.inv_norm + cb + c);
                const float nb = (DIST == ABX_DIST_KL || DIST == ABX_DIST_EUCLIDEAN)
                                     ? __ldg(p.nrm2 + cb + c)
                                     : 0.0f;
                out[(c0 + c) * r.ld] = frame_dist<DIST>(v[c] * r.ia * ib, r.na, nb);
            }
        }
    }
}

// epi_strip with the distance chosen once per tile
template <int NC>
__device__ __forceinline__ void epi_strip_any(const float (&v)[NC], const StripRow &r,
                                              const ColMap<NC> &m, int64_t cb, int c0,
                                              const UmmaParams &p) {
    if (p.distance == ABX_DIST_KL)
        epi_strip<ABX_DIST_KL, NC>(v, r, m, cb, c0, p);
    else if (p.distance == ABX_DIST_EUCLIDEAN)
        epi_strip<ABX_DIST_EUCLIDEAN, NC>(v, r, m, cb, c0, p);
    else if (p.distance == ABX_DIST_COSINE)
        epi_strip<ABX_DIST_COSINE, NC>(v, r, m, cb, c0, p);
    else
        epi_strip<ABX_DIST_ANGULAR, NC>(v, r, m, cb, c0, p);
}

// NC columns (a multiple of 32) of the accumulator at TMEM address ta; for
// the FP32 split the cross-term accumulator `cross` columns further is added.
template <int PREC, int NC>
__device__ __forceinline__ void acc_load(uint32_t ta, float (&v)[NC],
                                         uint32_t cross = kPanel) {
#pragma unroll
    for (int c = 0; c < NC; c += 32) tmem_ld32(ta + c, v + c);
    if (PREC == ABX_FP32) {  // 8 columns at a time: few registers beyond v
#pragma unroll
        for (int c = 0; c < NC; c += 8) {
            float w[8];
            tmem_ld8(ta + cross + c, w);
#pragma unroll
            for (int i = 0; i < 8; ++i) v[c + i] += w[i];
        }
    }
}

// ------------------------------------------- producer and MMA issuer (one lane)

// TMA producer of the narrow and fused kernels: for each of the CTA's tiles
// with a needed pair, the k-chunks of its row panel (A) and column panel (B),
// hi and lo halves for the FP32 split.  Stage layout: A, B (BF16, FP8) or
// A hi, A lo, B hi, B lo (FP32 split: B hi and B lo adjacent, one N = 256
// operand).
template <int PREC, int STAGES>
__device__ __forceinline__ void produce_tiles(const CUtensorMap *tmap, const UmmaParams &p,
                                              uint8_t *smem, uint64_t *full, uint64_t *empty) {
    constexpr int kOps = PREC == ABX_FP32 ? 4 : 2;
    constexpr uint32_t kStageBytes = kOps * kTileBytes;
    int s = 0;
    uint32_t ph = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < p.n_tiles && ok; t += gridDim.x) {
        if (p.tile_count[t] == 0) continue;
        const int2 pp = p.tiles[t];
        const int32_t ra = p.panel_row[pp.x], rb = p.panel_row[pp.y];
        for (int kc = 0; kc < p.n_kchunks && ok; ++kc) {
            if (!(ok = mbar_wait(&empty[s], ph ^ 1u, p.err, 11))) break;
            uint8_t *st = smem + s * kStageBytes;
            mbar_expect_tx(&full[s], kStageBytes);
            const int32_t x = kc * (PREC == ABX_FP8 ? 128 : 64);
            int32_t xb = x + p.b_rot;
            if (xb >= p.k_elems) xb -= p.k_elems;
            tma_load_2d(st, tmap, &full[s], x, ra);
            if (PREC == ABX_FP32) {
                tma_load_2d(st + kTileBytes, tmap, &full[s], x + p.lo_offset, ra);
                tma_load_2d(st + 2 * kTileBytes, tmap, &full[s], xb, rb);
                tma_load_2d(st + 3 * kTileBytes, tmap, &full[s], xb + p.lo_offset, rb);
            } else {
                tma_load_2d(st + kTileBytes, tmap, &full[s], xb, rb);
            }
            if (++s == STAGES) {
                s = 0;
                ph ^= 1u;
            }
        }
    }
}

// MMA issuer of the narrow and fused kernels.  FP32 split: hi*hi into the
// main accumulator d, hi*lo + lo*hi into a second one (d + kPanel).  The
// cross terms are about 2^-10 of the main ones, so their accumulator stays
// small and loses almost nothing to the accumulation's rounding: only
// dim / 16 additions reach full magnitude instead of 3 dim / 16.  Per k step
// one N = 256 MMA, A hi x [B hi | B lo], writes both hi*hi (columns 0..127)
// and hi*lo (128..255), and one N = 128 MMA adds lo*hi to the cross columns:
// 20 KB of operands read from shared memory per k step instead of 24 KB for
// three N = 128 MMAs, which bound the kernel.
template <int PREC, int STAGES>
__device__ __forceinline__ void mma_tiles(const UmmaParams &p, uint8_t *smem, uint64_t *full,
                                          uint64_t *empty, uint64_t *acc_full,
                                          uint64_t *acc_empty, uint32_t tmem) {
    constexpr int kOps = PREC == ABX_FP32 ? 4 : 2;
    constexpr uint32_t kStageBytes = kOps * kTileBytes;
    constexpr int KIND = PREC == ABX_FP8 ? 1 : 0;
    // instruction descriptor: D = F32 (bits 4-5), A/B = F16 (0, the FP32
    // split), BF16 (1) or E4M3 (0 of kind::f8f6f4) (bits 7-9, 10-12), both
    // K-major, N >> 3 at bits 17-22, M >> 4 at 24-28
    constexpr uint32_t kFmt = PREC == ABX_BF16 ? 1u : 0u;
    constexpr uint32_t kIdesc = (1u << 4) | (kFmt << 7) | (kFmt << 10) |
                                ((uint32_t)(kPanel >> 3) << 17) | ((uint32_t)(kPanel >> 4) << 24);
    constexpr uint32_t kIdesc256 = (1u << 4) | (kFmt << 7) | (kFmt << 10) |
                                   ((uint32_t)(2 * kPanel >> 3) << 17) |
                                   ((uint32_t)(kPanel >> 4) << 24);
    int s = 0;
    uint32_t ph = 0;
    int local = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < p.n_tiles && ok; t += gridDim.x) {
        if (p.tile_count[t] == 0) continue;
        const int b = local & 1;
        const uint32_t aph = (uint32_t)(local >> 1) & 1u;
        if (!(ok = mbar_wait(&acc_empty[b], aph ^ 1u, p.err, 12))) break;
        fence_after();
        const uint32_t d = tmem + (uint32_t)(b * acc_stride<PREC>());
        const uint32_t dx = d + (uint32_t)kPanel;
        for (int kc = 0; kc < p.n_kchunks && ok; ++kc) {
            if (!(ok = mbar_wait(&full[s], ph, p.err, 13))) break;
            fence_after();
            const uint32_t base = smem_u32(smem + s * kStageBytes);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const uint32_t off = kk * 32;  // 32 bytes = one MMA's k extent
                const uint32_t acc0 = (kc | kk) ? 1u : 0u;
                const uint64_t ah = sdesc(base + off);
                if (PREC == ABX_FP32) {
                    const uint64_t al = sdesc(base + kTileBytes + off);
                    const uint64_t bhl = sdesc(base + 2 * kTileBytes + off);  // [B hi | B lo]
                    umma<KIND>(d, ah, bhl, kIdesc256, acc0);
                    umma<KIND>(dx, al, bhl, kIdesc, 1u);                     // B hi rows
                } else {
                    umma<KIND>(d, ah, sdesc(base + kTileBytes + off), kIdesc, acc0);
                }
            }
            umma_commit(&empty[s]);
            if (++s == STAGES) {
                s = 0;
                ph ^= 1u;
            }
        }
        if (ok) umma_commit(&acc_full[b]);
        ++local;
    }
}

// Barriers and TMEM of the narrow and fused kernels: STAGES full / empty
// pairs, two accumulator full / empty pairs (empty counted by the NEPI
// epilogue warps), TMEM allocated by warp 1.
template <int PREC, int STAGES, int NEPI>
__device__ __forceinline__ uint32_t tile_setup(uint64_t *full, uint32_t *tmem_slot) {
    uint64_t *empty = full + STAGES, *acc_full = empty + STAGES, *acc_empty = acc_full + 2;
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], NEPI);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(tmem_cols<PREC>())
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    return *tmem_slot;
}

template <int PREC>
__device__ __forceinline__ void tile_teardown(uint32_t tmem) {
    fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 1) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(tmem_cols<PREC>())
                     : "memory");
    }
}

// --------------------------------------------------------- the narrow kernel

// PREC: ABX_FP32 (split), ABX_BF16, ABX_FP8.  STAGES: smem ring depth.
// EW epilogue warps (8 or 16), warps 2.. : each 32 rows (its TMEM lane
// quarter) x 128 / (EW / 4) columns of the tile.
template <int PREC, int STAGES, int EW>
__global__ void __launch_bounds__(32 * (2 + EW), 1)
    umma_tile_kernel(const __grid_constant__ CUtensorMap tmap, UmmaParams p) {
    constexpr int kNC = kPanel / (EW / 4);
    constexpr int kOps = PREC == ABX_FP32 ? 4 : 2;  // operand tiles per stage
    constexpr uint32_t kStageBytes = kOps * kTileBytes;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * kStageBytes);
    uint64_t *empty = full + STAGES;
    uint64_t *acc_full = empty + STAGES;
    uint64_t *acc_empty = acc_full + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_empty + 2);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t tmem = tile_setup<PREC, STAGES, EW>(full, tmem_slot);

    if (warp == 0) {
        if (lane == 0) produce_tiles<PREC, STAGES>(&tmap, p, smem, full, empty);
    } else if (warp == 1) {
        if (lane == 0) mma_tiles<PREC, STAGES>(p, smem, full, empty, acc_full, acc_empty, tmem);
        __syncwarp();
    } else {
        const int ew = warp - 2;
        const int q = warp & 3;            // TMEM lane quarter this warp may access
        const int slice = ew >> 2;         // column slice
        const int row = q * 32 + lane;
        int local = 0;
        bool ok = true;
        for (int64_t t = blockIdx.x; t < p.n_tiles && ok; t += gridDim.x) {
            if (p.tile_count[t] == 0) continue;
            const int2 pp = p.tiles[t];
            const StripRow sr = strip_row(p, t, pp, row);
            const ColMap<kNC> cmap = col_map<kNC>(p, t, slice * kNC);
            const int b = local & 1;
            const uint32_t aph = (uint32_t)(local >> 1) & 1u;
            ok = mbar_wait(&acc_full[b], aph, p.err, 14);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            fence_after();
            float v[kNC];
            acc_load<PREC, kNC>(tmem + ((uint32_t)(q * 32) << 16) +
                                    (uint32_t)(b * acc_stride<PREC>() + slice * kNC),
                                v);
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[b]);
            epi_strip_any<kNC>(v, sr, cmap, p.panel_row[pp.y] + slice * kNC, slice * kNC, p);
            ++local;
        }
    }
    tile_teardown<PREC>(tmem);
}

// ------------------------------------------------- the cluster-pair kernel

// Work item of the pair kernel: rank r's tile (or -1) and the cluster's
// mask of ranks with a tile that has a needed pair.
__device__ __forceinline__ uint32_t pair_item(const UmmaParams &p, int64_t w, uint32_t rank,
                                              int *mine, int *any_tile) {
    const int2 wk = p.work[w];
    const bool h0 = p.tile_count[wk.x] > 0;
    const bool h1 = wk.y >= 0 && p.tile_count[wk.y] > 0;
    *mine = rank == 0 ? wk.x : wk.y;
    *any_tile = h0 ? wk.x : wk.y;
    return (h0 ? 1u : 0u) | (h1 ? 2u : 0u);
}

// FP32 split on a cluster of two CTAs (two SMs).  A work item is a tile and
// the next tile of its panel row (as for the wide kernel); rank 0 computes
// the first, rank 1 the second, each with its own double-buffered pair of
// TMEM accumulators as in the narrow kernel.  The two tiles share their row
// panel A: the lowest rank with a tile loads A's k-chunks once and TMA
// multicasts them into both CTAs' stages, each rank loads its own column
// panel B.  A stage is refilled only once both CTAs' MMAs are done with it:
// every MMA issuer's commit arrives on the stage's empty barrier in both
// CTAs (two arrivals per phase).  Per pair of tiles the operands read from
// L2 drop from four panels (hi and lo) to three (the narrow kernel moves
// about 13 TB/s from L2); it measured no faster than the narrow kernel, whose
// limit is the latency its three 64 KB stages can cover.  A rank without a
// tile in an item still steps through the item's stages (zero bytes
// expected, commits only) so that both CTAs fill and drain the same stage in
// the same order.
template <int PREC, int STAGES, int EW>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(32 * (2 + EW), 1)
    umma_pair_kernel(const __grid_constant__ CUtensorMap tmap, UmmaParams p) {
    static_assert(PREC == ABX_FP32, "the pair kernel serves the FP32 split");
    constexpr int kNC = kPanel / (EW / 4);
    constexpr uint32_t kStageBytes = 4 * kTileBytes;  // A hi, A lo, B hi, B lo
    constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(kPanel >> 3) << 17) |
                                ((uint32_t)(kPanel >> 4) << 24);  // F16 x F16 -> F32
    constexpr uint32_t kIdesc256 = (1u << 4) | ((uint32_t)(2 * kPanel >> 3) << 17) |
                                   ((uint32_t)(kPanel >> 4) << 24);
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * kStageBytes);
    uint64_t *empty = full + STAGES;
    uint64_t *acc_full = empty + STAGES;
    uint64_t *acc_empty = acc_full + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_empty + 2);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const int64_t cid = cluster_id(), ncl = cluster_count();
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 2);  // one commit from each CTA's MMA issuer
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], EW);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(tmem_cols<PREC>())
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    cluster_sync();  // both CTAs' barriers exist before either signals the other's
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            bool ok = true;
            for (int64_t w = cid; w < p.n_work && ok; w += ncl) {
                int mine, any;
                const uint32_t mask = pair_item(p, w, rank, &mine, &any);
                if (!mask) continue;
                const bool has = (mask >> rank) & 1u;
                const bool loader = rank == (uint32_t)__ffs(mask) - 1u;
                const int32_t ra = p.panel_row[p.tiles[any].x];
                const int32_t rb = has ? p.panel_row[p.tiles[mine].y] : 0;
                for (int kc = 0; kc < p.n_kchunks && ok; ++kc) {
                    if (!(ok = mbar_wait(&empty[s], ph ^ 1u, p.err, 11))) break;
                    uint8_t *st = smem + s * kStageBytes;
                    mbar_expect_tx(&full[s], has ? kStageBytes : 0u);
                    const int32_t x = kc * 64;
                    if (loader) {
                        tma_load_2d_mc(st, &tmap, &full[s], x, ra, (uint16_t)mask);
                        tma_load_2d_mc(st + kTileBytes, &tmap, &full[s], x + p.lo_offset, ra,
                                       (uint16_t)mask);
                    }
                    if (has) {
                        tma_load_2d(st + 2 * kTileBytes, &tmap, &full[s], x, rb);
                        tma_load_2d(st + 3 * kTileBytes, &tmap, &full[s], x + p.lo_offset, rb);
                    }
                    if (++s == STAGES) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
            }
            // tail: every stage released once more by both CTAs, i.e. the
            // other CTA's last commits have landed on this CTA's barriers
            for (int k = 0; k < STAGES && ok; ++k) {
                ok = mbar_wait(&empty[s], ph ^ 1u, p.err, 16);
                if (++s == STAGES) {
                    s = 0;
                    ph ^= 1u;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            int local = 0;
            bool ok = true;
            for (int64_t w = cid; w < p.n_work && ok; w += ncl) {
                int mine, any;
                const uint32_t mask = pair_item(p, w, rank, &mine, &any);
                if (!mask) continue;
                const bool has = (mask >> rank) & 1u;
                const int b = local & 1;
                const uint32_t aph = (uint32_t)(local >> 1) & 1u;
                if (has && !(ok = mbar_wait(&acc_empty[b], aph ^ 1u, p.err, 12))) break;
                fence_after();
                const uint32_t d = tmem + (uint32_t)(b * acc_stride<PREC>());
                const uint32_t dx = d + (uint32_t)kPanel;
                for (int kc = 0; kc < p.n_kchunks && ok; ++kc) {
                    if (!(ok = mbar_wait(&full[s], ph, p.err, 13))) break;
                    fence_after();
                    if (has) {
                        const uint32_t base = smem_u32(smem + s * kStageBytes);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint32_t off = kk * 32;
                            const uint32_t acc0 = (kc | kk) ? 1u : 0u;
                            const uint64_t ah = sdesc(base + off);
                            const uint64_t al = sdesc(base + kTileBytes + off);
                            const uint64_t bhl = sdesc(base + 2 * kTileBytes + off);
                            umma<0>(d, ah, bhl, kIdesc256, acc0);  // hi*hi | hi*lo
                            umma<0>(dx, al, bhl, kIdesc, 1u);      // lo*hi
                        }
                    }
                    umma_commit_mc(&empty[s], 3);  // both CTAs' stage s
                    if (++s == STAGES) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
                if (has) {
                    if (ok) umma_commit(&acc_full[b]);
                    ++local;
                }
            }
        }
        __syncwarp();
    } else {
        const int ew = warp - 2;
        const int q = warp & 3;
        const int slice = ew >> 2;
        const int row = q * 32 + lane;
        int local = 0;
        bool ok = true;
        for (int64_t w = cid; w < p.n_work && ok; w += ncl) {
            int t, any;
            const uint32_t mask = pair_item(p, w, rank, &t, &any);
            if (!((mask >> rank) & 1u)) continue;
            const int2 pp = p.tiles[t];
            const StripRow sr = strip_row(p, t, pp, row);
            const ColMap<kNC> cmap = col_map<kNC>(p, t, slice * kNC);
            const int b = local & 1;
            const uint32_t aph = (uint32_t)(local >> 1) & 1u;
            ok = mbar_wait(&acc_full[b], aph, p.err, 14);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            fence_after();
            float v[kNC];
            acc_load<PREC, kNC>(tmem + ((uint32_t)(q * 32) << 16) +
                                    (uint32_t)(b * acc_stride<PREC>() + slice * kNC),
                                v);
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[b]);
            epi_strip_any<kNC>(v, sr, cmap, p.panel_row[pp.y] + slice * kNC, slice * kNC, p);
            ++local;
        }
    }
    fence_before();
    __syncthreads();
    // neither CTA leaves while the other may still multicast into it or
    // arrive on its barriers
    cluster_sync();
    if (warp == 1) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(tmem_cols<PREC>())
                     : "memory");
    }
}

// ---------------------------------------------------------- the fused kernel

// d(i, j) of one pair's block in the shared d tile; rows of the DTW are the
// shorter item (tr: the column panel's item y), which keeps the wavefront's
// strips few.  The DTW is symmetric under transposition (same step set, same
// shorter-path rule on the same sums), so the result is the pair's.
struct SmemBlock {
    const float *db;  // d tile at (rx, cy)
    bool tr;
    __device__ __forceinline__ float operator()(int i, int j) const {
        return tr ? db[j * kDS + i] : db[i * kDS + j];
    }
};

// Distances of the 32 columns cb.. of one accumulator row into the d tile
// (row-major, stride kDS), two per 8-byte store.
template <int DIST>
__device__ __forceinline__ void epi_smem(const float (&v)[32], float ia, float na, int64_t cb,
                                         int64_t n_rows, const float *__restrict__ inv_norm,
                                         const float *__restrict__ nrm2, float *out) {
#pragma unroll
    for (int c = 0; c < 32; c += 2) {
        float o[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const bool cv = cb + c + e < n_rows;
            const float ib = cv ? __ldg(inv_norm + cb + c + e) : 0.0f;
            const float nb = (DIST == ABX_DIST_KL || DIST == ABX_DIST_EUCLIDEAN) && cv
                                 ? __ldg(nrm2 + cb + c + e)
                                 : 0.0f;
            o[e] = frame_dist<DIST>(v[c + e] * ia * ib, na, nb);
        }
        *reinterpret_cast<float2 *>(out + c) = make_float2(o[0], o[1]);
    }
}

// Fused tile + DTW kernel (items of at most kFuseMaxLen frames).  Per tile:
// the 16 epilogue warps load the accumulator (warp w: rows of TMEM quarter
// w % 4, 32 columns), release it to the MMA issuer, write the frame
// distances to the shared d tile, then run the DTW of every needed pair of
// the tile on the d tile and write distance, interval and path length to
// both orientations of the group matrix.  FORM 0 (the default form): one
// thread per pair, in place on the pair's block (dtw_inplace), pairs dealt
// to consecutive threads, so the ~100 pairs of a typical tile fill about
// four warps, one per SM sub-partition.  FORM 1: one 8-lane group per pair
// (64 groups, pairs dealt round-robin) running an anti-diagonal wavefront
// with row buffers of its own.  The MMAs of the next tile (other
// accumulator) run meanwhile.
template <int PREC, int STAGES, int FORM>
__global__ void __launch_bounds__(kFuseThreads, 1)
    umma_fused_kernel(const __grid_constant__ CUtensorMap tmap, UmmaParams p) {
    constexpr int kOps = PREC == ABX_FP32 ? 4 : 2;
    constexpr uint32_t kStageBytes = kOps * kTileBytes;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    float *dtile = reinterpret_cast<float *>(smem + STAGES * kStageBytes);  // kPanel x kDS
    float *rbc = dtile + kPanel * kDS;                                     // per group
    uint32_t *rbl = reinterpret_cast<uint32_t *>(rbc + kFuseGroups * kFuseMaxLen);
    uint64_t *full = reinterpret_cast<uint64_t *>(rbl + kFuseGroups * kFuseMaxLen);
    uint64_t *empty = full + STAGES;
    uint64_t *acc_full = empty + STAGES;
    uint64_t *acc_empty = acc_full + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_empty + 2);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t tmem = tile_setup<PREC, STAGES, kFuseWarps>(full, tmem_slot);

    if (warp == 0) {
        if (lane == 0) produce_tiles<PREC, STAGES>(&tmap, p, smem, full, empty);
    } else if (warp == 1) {
        if (lane == 0) mma_tiles<PREC, STAGES>(p, smem, full, empty, acc_full, acc_empty, tmem);
        __syncwarp();
    } else {
        const int ew = warp - 2;
        const int q = warp & 3;            // TMEM lane quarter this warp may access
        const int slice = ew >> 2;         // 32-column slice of the tile
        const int row = q * 32 + lane;
        const int grp = ew * 4 + (lane >> 3);
        float *grb = rbc + grp * kFuseMaxLen;
        uint32_t *grl = rbl + grp * kFuseMaxLen;
        int local = 0;
        for (int64_t t = blockIdx.x; t < p.n_tiles; t += gridDim.x) {
            if (p.tile_count[t] == 0) continue;
            const int b = local & 1;
            const uint32_t aph = (uint32_t)(local >> 1) & 1u;
            const bool ok = mbar_wait(&acc_full[b], aph, p.err, 14);
            if (epi_bar_or<kFuseEpiThreads>(!ok)) break;  // all warps take the same decision
            fence_after();
            float v[32];
            acc_load<PREC, 32>(tmem + ((uint32_t)(q * 32) << 16) +
                                   (uint32_t)(b * acc_stride<PREC>() + slice * 32),
                               v);
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[b]);
            const int2 pp = p.tiles[t];
            const int64_t ra = p.panel_row[pp.x] + row;
            const int64_t cb = p.panel_row[pp.y] + slice * 32;
            const float ia = ra < p.n_rows ? p.inv_norm[ra] : 0.0f;
            const float na = (p.distance == ABX_DIST_KL || p.distance == ABX_DIST_EUCLIDEAN) &&
                                     ra < p.n_rows
                                 ? p.nrm2[ra]
                                 : 0.0f;
            float *out = dtile + row * kDS + slice * 32;
            if (p.distance == ABX_DIST_KL)
                epi_smem<ABX_DIST_KL>(v, ia, na, cb, p.n_rows, p.inv_norm, p.nrm2, out);
            else if (p.distance == ABX_DIST_EUCLIDEAN)
                epi_smem<ABX_DIST_EUCLIDEAN>(v, ia, na, cb, p.n_rows, p.inv_norm, p.nrm2, out);
            else if (p.distance == ABX_DIST_COSINE)
                epi_smem<ABX_DIST_COSINE>(v, ia, 0.0f, cb, p.n_rows, p.inv_norm, p.nrm2, out);
            else
                epi_smem<ABX_DIST_ANGULAR>(v, ia, 0.0f, cb, p.n_rows, p.inv_norm, p.nrm2, out);
            epi_bar<kFuseEpiThreads>();  // the d tile is complete
            const int64_t pe = p.tile_base[t + 1];
            if (FORM == 0) {
                for (int64_t pi = p.tile_base[t] + (threadIdx.x - 64); pi < pe;
                     pi += kFuseEpiThreads) {
                    const int4 pr = p.pairs[pi];
                    const int x = pr.x, y = pr.y;
                    const int rx = pr.w & 0xffff, cy = pr.w >> 16;
                    const int Tx = p.len[x], Ty = p.len[y];
                    // the planner never sends these; refuse, do not overrun
                    if (Tx > kFuseMaxLen || Ty > kFuseMaxLen || rx + Tx > kPanel ||
                        cy + Ty > kPanel) {
                        atomicCAS(p.err, 0, 15);
                        continue;
                    }
                    const DtwBound bd =
                        dtw_bound(Tx, Ty, p.theta_item[x], p.theta_item[y], p.eps_c);
                    float cost, dev;
                    uint32_t info;
                    dtw_inplace(dtile + rx * kDS + cy, kDS, Tx, Ty, bd.tau, cost, info, dev);
                    const uint32_t L = info & 0xffu;
                    const float D = __fdiv_rn(cost, (float)L);
                    float lo, hi;
                    dtw_interval(bd, cost, info, dev, p.eps_c, p.intervals, D, lo, hi);
                    const int4 gm = p.gmeta[p.item_g[x]];
                    const int gb = gm.x;
                    const int64_t ng = gm.y;
                    const int64_t base = ((int64_t)(uint32_t)gm.w << 32) | (uint32_t)gm.z;
                    const PairVal pvv{D, lo, hi, L};
                    p.pv[base + (int64_t)(x - gb) * ng + (y - gb)] = pvv;
                    p.pv[base + (int64_t)(y - gb) * ng + (x - gb)] = pvv;
                }
            } else
            for (int64_t pi = p.tile_base[t] + grp; pi < pe; pi += kFuseGroups) {
                const int4 pr = p.pairs[pi];
                const int x = pr.x, y = pr.y;
                const int rx = pr.w & 0xffff, cy = pr.w >> 16;
                const int Tx = p.len[x], Ty = p.len[y];
                const bool tr = Tx > Ty;
                const int R = tr ? Ty : Tx, C = tr ? Tx : Ty;
                if (C > kFuseMaxLen) {  // the planner never sends these; refuse, do not overrun
                    if ((lane & 7) == 0) atomicCAS(p.err, 0, 15);
                    continue;
                }
                const DtwBound bd = dtw_bound(Tx, Ty, p.theta_item[x], p.theta_item[y], p.eps_c);
                const SmemBlock dat{dtile + rx * kDS + cy, tr};
                float cost, dev;
                uint32_t info;
                dtw_wave8(dat, R, C, bd.tau, grb, grl, cost, info, dev);
                if ((lane & 7) == 0) {
                    const uint32_t L = info & 0xffu;
                    const float D = __fdiv_rn(cost, (float)L);
                    float lo, hi;
                    dtw_interval(bd, cost, info, dev, p.eps_c, p.intervals, D, lo, hi);
                    const int4 gm = p.gmeta[p.item_g[x]];
                    const int gb = gm.x;
                    const int64_t ng = gm.y;
                    const int64_t base = ((int64_t)(uint32_t)gm.w << 32) | (uint32_t)gm.z;
                    const PairVal pvv{D, lo, hi, L};
                    p.pv[base + (int64_t)(x - gb) * ng + (y - gb)] = pvv;
                    p.pv[base + (int64_t)(y - gb) * ng + (x - gb)] = pvv;
                }
            }
            __syncwarp();
            epi_bar<kFuseEpiThreads>();  // every group is done with the d tile
            ++local;
        }
    }
    tile_teardown<PREC>(tmem);
}

// ------------------------------------------------------- the wide kernel

// A work item is a tile and, when it has one, the next tile of the same panel
// row: the A panel is loaded once for both and one N = 256 MMA covers them,
// which cuts the operand bytes per MMA from shared memory by a quarter (the
// narrow kernel measured bound by the operand feed, not the tensor pipe).
// Returns the number of tiles the item computes (tiles without a needed pair
// are dropped; a lone remaining tile runs as N = 128).
__device__ __forceinline__ int wide_item(const UmmaParams &p, int64_t w, int *t0, int *t1) {
    const int2 wk = p.work[w];
    const bool c0 = p.tile_count[wk.x] > 0;
    const bool c1 = wk.y >= 0 && p.tile_count[wk.y] > 0;
    *t0 = c0 ? wk.x : wk.y;
    *t1 = wk.y;
    return (int)c0 + (int)c1;
}

// EW epilogue warps (8 or 16): each reads 32 rows x (128 / (EW / 4)) columns
// of each tile of the item.
template <int PREC, int STAGES, int EW>
__global__ void __launch_bounds__(32 * (2 + EW), 1)
    umma_wide_kernel(const __grid_constant__ CUtensorMap tmap, UmmaParams p) {
    static_assert(PREC != ABX_FP32, "the FP32 split runs on the narrow kernel");
    constexpr int kNC = kPanel / (EW / 4);  // columns per epilogue thread and tile
    // stage: A, B (two panels)
    constexpr uint32_t kA = 0, kB = kTileBytes;
    constexpr uint32_t kStageBytes = 3 * kTileBytes;
    constexpr int KIND = PREC == ABX_FP8 ? 1 : 0;
    constexpr uint32_t kFmt = PREC == ABX_BF16 ? 1u : 0u;  // F16 / BF16 / E4M3
    constexpr uint32_t kIdescBase = (1u << 4) | (kFmt << 7) | (kFmt << 10) |
                                    ((uint32_t)(kPanel >> 4) << 24);
    constexpr uint32_t kCols = 512;  // two 256-column FP32 accumulators
    constexpr int kBufs = 2;

    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * kStageBytes);
    uint64_t *empty = full + STAGES;
    uint64_t *acc_full = empty + STAGES;
    uint64_t *acc_empty = acc_full + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_empty + 2);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], EW);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    const int nk = p.n_kchunks;

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            bool ok = true;
            for (int64_t w = blockIdx.x; w < p.n_work && ok; w += gridDim.x) {
                int t0, t1;
                const int nb = wide_item(p, w, &t0, &t1);
                if (nb == 0) continue;
                const int32_t ra = p.panel_row[p.tiles[t0].x];
                const int32_t rb0 = p.panel_row[p.tiles[t0].y];
                const int32_t rb1 = nb == 2 ? p.panel_row[p.tiles[t1].y] : 0;
                const uint32_t bytes = (1u + (uint32_t)nb) * kTileBytes;
                for (int kc = 0; kc < nk && ok; ++kc) {
                    if (!(ok = mbar_wait(&empty[s], ph ^ 1u, p.err, 11))) break;
                    uint8_t *st = smem + s * kStageBytes;
                    mbar_expect_tx(&full[s], bytes);
                    const int32_t x = kc * (PREC == ABX_FP8 ? 128 : 64);
                    int32_t xb = x + p.b_rot;
                    if (xb >= p.k_elems) xb -= p.k_elems;
                    tma_load_2d(st + kA, &tmap, &full[s], x, ra);
                    tma_load_2d(st + kB, &tmap, &full[s], xb, rb0);
                    if (nb == 2) tma_load_2d(st + kB + kTileBytes, &tmap, &full[s], xb, rb1);
                    if (++s == STAGES) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            int local = 0;
            bool ok = true;
            for (int64_t w = blockIdx.x; w < p.n_work && ok; w += gridDim.x) {
                int t0, t1;
                const int nb = wide_item(p, w, &t0, &t1);
                if (nb == 0) continue;
                const uint32_t idesc = kIdescBase | ((uint32_t)((nb * kPanel) >> 3) << 17);
                const int b = local % kBufs;
                const uint32_t aph = (uint32_t)(local / kBufs) & 1u;
                if (!(ok = mbar_wait(&acc_empty[b], aph ^ 1u, p.err, 12))) break;
                fence_after();
                const uint32_t d = tmem + (uint32_t)(b * 2 * kPanel);
                for (int kc = 0; kc < nk && ok; ++kc) {
                    if (!(ok = mbar_wait(&full[s], ph, p.err, 13))) break;
                    fence_after();
                    const uint32_t base = smem_u32(smem + s * kStageBytes);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint32_t off = kk * 32;  // 32 bytes = one MMA's k extent
                        const uint64_t ah = sdesc(base + kA + off), bh = sdesc(base + kB + off);
                        const uint32_t acc0 = (kc | kk) ? 1u : 0u;
                        umma<KIND>(d, ah, bh, idesc, acc0);
                    }
                    umma_commit(&empty[s]);
                    if (++s == STAGES) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
                if (ok) umma_commit(&acc_full[b]);
                ++local;
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: each warp 32 rows x kNC columns of each tile
        const int ew = warp - 2;
        const int q = warp & 3;            // TMEM lane quarter this warp may access
        const int slice = ew >> 2;         // column slice of each tile
        const int row = q * 32 + lane;
        int local = 0;
        bool ok = true;
        for (int64_t w = blockIdx.x; w < p.n_work && ok; w += gridDim.x) {
            int t0, t1;
            const int nb = wide_item(p, w, &t0, &t1);
            if (nb == 0) continue;
            const int b = local % kBufs;
            const uint32_t aph = (uint32_t)(local / kBufs) & 1u;
            ok = mbar_wait(&acc_full[b], aph, p.err, 14);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            fence_after();
            for (int j = 0; j < nb; ++j) {
                const int t = j ? t1 : t0;
                float v[kNC];
                const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) +
                                    (uint32_t)(b * 2 * kPanel + j * kPanel + slice * kNC);
#pragma unroll
                for (int c = 0; c < kNC; c += 32) tmem_ld32(ta + c, v + c);
                const int2 pp = p.tiles[t];
                const int64_t ra = p.panel_row[pp.x] + row;
                const int64_t cb = p.panel_row[pp.y] + slice * kNC;
                const float ia = ra < p.n_rows ? p.inv_norm[ra] : 0.0f;
                // column-major tile (the host plans this layout for the wide kernel)
                float *out =
                    p.tilebuf + t * (int64_t)(kPanel * kPanel) + slice * kNC * kPanel + row;
                if (p.distance == ABX_DIST_KL)
                    epi_row<ABX_DIST_KL, kNC>(v, ia, ra < p.n_rows ? p.nrm2[ra] : 0.0f,
                                              cb, p.n_rows, p.inv_norm, p.nrm2, out);
                else if (p.distance == ABX_DIST_EUCLIDEAN)
                    epi_row<ABX_DIST_EUCLIDEAN, kNC>(v, ia, ra < p.n_rows ? p.nrm2[ra] : 0.0f,
                                                     cb, p.n_rows, p.inv_norm, p.nrm2, out);
                else if (p.distance == ABX_DIST_COSINE)
                    epi_row<ABX_DIST_COSINE, kNC>(v, ia, 0.0f, cb, p.n_rows, p.inv_norm,
                                                  p.nrm2, out);
                else
                    epi_row<ABX_DIST_ANGULAR, kNC>(v, ia, 0.0f, cb, p.n_rows, p.inv_norm,
                                                   p.nrm2, out);
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[b]);
            ++local;
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kCols)
                     : "memory");
    }
}

// ------------------------------------------------------------- host side

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *ptr = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    }
    return fn;
}

// Tensor map over the packed rows (2-D: elements of a row x rows; boxes of
// 128 bytes x 128 rows, 128-byte swizzle) and the kernel parameters.
template <int PREC>
cudaError_t make_args(const TileGemmArgs &a, int32_t *err, CUtensorMap *map, UmmaParams *pp) {
    auto fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    const int elem = PREC == ABX_FP8 ? 1 : 2;
    const int64_t width = PREC == ABX_FP32 ? 2 * (int64_t)a.dim_pad : a.dim_pad;  // elements
    cuuint64_t gdim[2] = {(cuuint64_t)width, (cuuint64_t)a.n_rows};
    cuuint64_t gstride[1] = {(cuuint64_t)(width * elem)};
    cuuint32_t box[2] = {(cuuint32_t)(128 / elem), (cuuint32_t)kPanel};
    cuuint32_t estride[2] = {1, 1};
    CUresult r = fn(map, PREC == ABX_FP8    ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                         : PREC == ABX_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                            : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
                    2, const_cast<void *>(a.packed), gdim, gstride, box, estride,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    UmmaParams &p = *pp;
    p.inv_norm = a.inv_norm;
    p.n_rows = a.n_rows;
    p.n_kchunks = (int32_t)(a.dim_pad * elem / 128);
    p.lo_offset = PREC == ABX_FP32 ? a.dim_pad : 0;
    p.b_rot = a.b_rot;
    p.k_elems = a.dim_pad;
    p.tiles = a.tiles;
    p.panel_row = a.panel_row;
    p.tile_count = a.tile_count;
    p.n_tiles = a.n_tiles;
    p.tilebuf = a.tilebuf;
    p.err = err;
    p.distance = a.distance;
    p.nrm2 = a.nrm2;
    p.pairs = a.pairs;
    p.tile_base = a.tile_base;
    p.len = a.len;
    p.theta_item = a.theta_item;
    p.eps_c = a.eps_c;
    p.intervals = a.intervals;
    p.item_g = a.item_g;
    p.gmeta = a.gmeta;
    p.pv = a.pv;
    p.work = a.work;
    p.n_work = a.n_work;
    p.row_item = a.row_item;
    p.row = a.row;
    p.panel_item = a.panel_item;
    p.xmask = a.xmask;
    p.col_yo = a.col_yo;
    p.strips = a.strips;
    p.listed_only = a.listed_only;
    return cudaSuccess;
}

const char *kernel_name(int prec, bool fused) {
    if (fused)
        return prec == ABX_FP32 ? "tile_dtw_umma_fp32split"
               : prec == ABX_BF16 ? "tile_dtw_umma_bf16"
                                  : "tile_dtw_umma_fp8";
    return prec == ABX_FP32 ? "tile_umma_fp32split"
           : prec == ABX_BF16 ? "tile_umma_bf16"
                              : "tile_umma_fp8";
}

// WIDE = 0: narrow kernel with NARROW_EW epilogue warps; 8 or 16: wide kernel
// with that many epilogue warps
template <int PREC, int STAGES, int WIDE = 0, int NARROW_EW = 16>
cudaError_t launch_prec(const TileGemmArgs &a, int n_sm, int32_t *err, cudaStream_t s) {
    CUtensorMap map;
    UmmaParams p;
    cudaError_t e = make_args<PREC>(a, err, &map, &p);
    if (e != cudaSuccess) return e;
    constexpr int kOps = WIDE ? 3 : (PREC == ABX_FP32 ? 4 : 2);
    const size_t smem = 1024 + (size_t)STAGES * kOps * kTileBytes + 256;
    auto kern = [] {
        if constexpr (WIDE != 0)
            return umma_wide_kernel<PREC, STAGES, WIDE>;
        else
            return umma_tile_kernel<PREC, STAGES, NARROW_EW>;
    }();
    const int threads = 32 * (2 + (WIDE ? WIDE : NARROW_EW));
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t items = WIDE ? a.n_work : a.n_tiles;
    const int grid = (int)(items < n_sm ? items : n_sm);
    if (grid == 0) return cudaSuccess;
    {
        ProfScope ps_(kernel_name(PREC, false), s);
        kern<<<grid, threads, smem, s>>>(map, p);
    }
    return cudaGetLastError();
}

// Cluster-pair kernel: as many clusters of two CTAs as can be resident at
// once (the work is dealt round-robin over clusters, so a second wave of
// clusters would run after the first one's whole share).
template <int PREC, int STAGES, int EW>
cudaError_t launch_pair(const TileGemmArgs &a, int n_sm, int32_t *err, cudaStream_t s) {
    CUtensorMap map;
    UmmaParams p;
    cudaError_t e = make_args<PREC>(a, err, &map, &p);
    if (e != cudaSuccess) return e;
    const size_t smem = 1024 + (size_t)STAGES * 4 * kTileBytes + 256;
    auto kern = umma_pair_kernel<PREC, STAGES, EW>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int threads = 32 * (2 + EW);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(n_sm & ~1));
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = 2;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int ncl = 0;
    e = cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg);
    if (e != cudaSuccess) return e;
    if (ncl < 1) return cudaErrorNotSupported;
    const int64_t clusters = std::min<int64_t>(ncl, std::max<int64_t>(a.n_work, 1));
    {
        ProfScope ps_(kernel_name(PREC, false), s);
        kern<<<(unsigned)(2 * clusters), threads, smem, s>>>(map, p);
    }
    return cudaGetLastError();
}

template <int PREC, int STAGES, int FORM>
cudaError_t launch_fused(const TileGemmArgs &a, int n_sm, int32_t *err, cudaStream_t s) {
    CUtensorMap map;
    UmmaParams p;
    cudaError_t e = make_args<PREC>(a, err, &map, &p);
    if (e != cudaSuccess) return e;
    constexpr int kOps = PREC == ABX_FP32 ? 4 : 2;
    const size_t smem = 1024 + (size_t)STAGES * kOps * kTileBytes +
                        (size_t)kPanel * kDS * 4 + (size_t)kFuseGroups * kFuseMaxLen * 8 + 256;
    e = cudaFuncSetAttribute(umma_fused_kernel<PREC, STAGES, FORM>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = (int)(a.n_tiles < n_sm ? a.n_tiles : n_sm);
    if (grid == 0) return cudaSuccess;
    {
        ProfScope ps_(kernel_name(PREC, true), s);
        umma_fused_kernel<PREC, STAGES, FORM><<<grid, kFuseThreads, smem, s>>>(map, p);
    }
    return cudaGetLastError();
}

}  // namespace

bool umma_supported(int precision) {
    return (precision == ABX_FP32 || precision == ABX_BF16 || precision == ABX_FP8) &&
           encode_fn() != nullptr;
}

cudaError_t launch_tile_umma(const TileGemmArgs &a, int precision, int n_sm, cudaStream_t s) {
    if (a.n_tiles == 0) return cudaSuccess;
    if (a.fused == 1) {  // 128 KB of operand stages next to the d tile; thread per pair
        if (precision == ABX_FP32) return launch_fused<ABX_FP32, 2, 0>(a, n_sm, a.err, s);
        if (precision == ABX_BF16) return launch_fused<ABX_BF16, 4, 0>(a, n_sm, a.err, s);
        if (precision == ABX_FP8) return launch_fused<ABX_FP8, 4, 0>(a, n_sm, a.err, s);
        return cudaErrorNotSupported;
    }
    if (a.fused == 2) {  // 8-lane wavefronts
        if (precision == ABX_FP32) return launch_fused<ABX_FP32, 2, 1>(a, n_sm, a.err, s);
        if (precision == ABX_BF16) return launch_fused<ABX_BF16, 4, 1>(a, n_sm, a.err, s);
        if (precision == ABX_FP8) return launch_fused<ABX_FP8, 4, 1>(a, n_sm, a.err, s);
        return cudaErrorNotSupported;
    }
    // variants (autotuner): 0 = the default ring depth, 1 = a shallower ring,
    // 2 = wide work items (two tiles of a panel row, N = 256), 3 = wide with
    // 16 epilogue warps.  The FP32 split keeps two accumulators per tile:
    // 0, 1 and 3 = the narrow kernel, 2 = narrow with 8 epilogue warps, 4 =
    // the cluster-pair kernel (narrow tiles, row panel multicast to two CTAs;
    // measured no faster: 7.7 against 7.4 ms per triphone-scale step).
    if (umma_wide(precision, a.variant) && a.work) {
        if (a.variant == 2) {
            if (precision == ABX_BF16) return launch_prec<ABX_BF16, 4, 8>(a, n_sm, a.err, s);
            if (precision == ABX_FP8) return launch_prec<ABX_FP8, 4, 8>(a, n_sm, a.err, s);
        } else {
            if (precision == ABX_BF16) return launch_prec<ABX_BF16, 4, 16>(a, n_sm, a.err, s);
            if (precision == ABX_FP8) return launch_prec<ABX_FP8, 4, 16>(a, n_sm, a.err, s);
        }
        return cudaErrorNotSupported;
    }
    if (precision == ABX_FP32 && a.variant == 2)  // 8 epilogue warps, 64 columns each
        return launch_prec<ABX_FP32, 3, 0, 8>(a, n_sm, a.err, s);
    if (precision == ABX_FP32 && a.variant == 4 && a.work)  // cluster pairs, shared A
        return launch_pair<ABX_FP32, 3, 16>(a, n_sm, a.err, s);
    if (a.variant == 1) {
        if (precision == ABX_FP32) return launch_prec<ABX_FP32, 2>(a, n_sm, a.err, s);
        if (precision == ABX_BF16) return launch_prec<ABX_BF16, 4>(a, n_sm, a.err, s);
        if (precision == ABX_FP8) return launch_prec<ABX_FP8, 4>(a, n_sm, a.err, s);
        return cudaErrorNotSupported;
    }
    if (precision == ABX_FP32) return launch_prec<ABX_FP32, 3>(a, n_sm, a.err, s);
    if (precision == ABX_BF16) return launch_prec<ABX_BF16, 6>(a, n_sm, a.err, s);
    if (precision == ABX_FP8) return launch_prec<ABX_FP8, 6>(a, n_sm, a.err, s);
    return cudaErrorNotSupported;
}

int umma_fuse_max_len() { return kFuseMaxLen; }

bool umma_wide(int precision, int variant) {
    return precision != ABX_FP32 && (variant == 2 || variant == 3);
}

}  // namespace abx
