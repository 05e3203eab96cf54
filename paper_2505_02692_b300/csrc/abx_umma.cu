// tcgen05 tensor-core tile kernel for the angular frame distances
// (fastabx Sec. 3.1 "angular"): every 128 x 128 tile of frame cosines
// <q_i, q_j> |q_i|^-1 |q_j|^-1 is one M=128, N=128 UMMA accumulation in TMEM,
// followed by an epilogue d = arccos(c) / pi written to the tile buffer.
//
// Precisions (operands K-major, staged by TMA with 128-byte swizzle):
//   ABX_FP32  frames split as hi + lo (two BF16 halves); three kind::f16 MMAs
//             per k step, hi*hi + hi*lo + lo*hi, FP32 accumulation in TMEM.
//   ABX_BF16  one kind::f16 MMA per k step (BF16 operands, FP32 accumulation).
//   ABX_FP8   one kind::f8f6f4 MMA per k step (E4M3 operands, FP32 accumulation).
//
// Persistent kernel, one CTA per SM, tiles taken round-robin.  Warp roles:
//   warp 0      TMA producer (one lane): k-chunks into a ring of smem stages
//   warp 1      TMEM owner and MMA issuer (one lane)
//   warps 2..9  epilogue: tcgen05.ld of a 32-lane quarter x 64 columns,
//               scale by the inverse norms, arccos / pi, store.
// Two TMEM accumulators (2 x 128 columns) let the epilogue of one tile run
// under the MMAs of the next.  Every mbarrier wait is bounded; on expiry the
// kernel records an error code, stops issuing work and still releases TMEM.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "abx_dtw_cell.cuh"
#include "abx_internal.h"

namespace abx {
namespace {

constexpr int kEpiWarps = 8;
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kFuseMaxLen = 32;                 // longest item the fused path takes
constexpr int kDLd = kPanel + 1;                // row stride of the shared d tile
constexpr int kThreads = 32 * (2 + kEpiWarps);
constexpr int kTileBytes = kPanel * 128;        // one 128-row x 128-byte operand tile
constexpr uint32_t kTmemCols = 256;             // two 128-column FP32 accumulators
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
    // fused DTW (FUSED = true)
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
};

// Named barrier over the epilogue warps only; returns the OR of `flag`.
__device__ __forceinline__ bool epi_bar_or(bool flag) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n"
        " bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}"
        : "=r"(r)
        : "r"((uint32_t)flag), "r"(kEpiThreads)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void epi_bar() {
    asm volatile("bar.sync 1, %0;" ::"r"(kEpiThreads) : "memory");
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

// Epilogue of one accumulator row half: 64 dot products -> frame distances.
// ia: the row's 1/|a| (1/scale for Euclidean); na: the row's squared norm
// (Euclidean only); columns cb.. with their 1/|b| and squared norms.  Column c
// goes to out[c] in the fused shared-memory tile (row-major) and to
// out[c * kPanel] in the global tile buffer, which is column-major so that a
// warp's 32 rows of one column form one 128-byte store.
template <int DIST, bool FUSED, int NC = 64>
__device__ __forceinline__ void epi_row(const float (&v)[NC], float ia, float na, int64_t cb,
                                        int64_t n_rows, const float *__restrict__ inv_norm,
                                        const float *__restrict__ nrm2, float *out) {
    const float inv_pi = 0.318309886183790671f;
#pragma unroll
    for (int c4 = 0; c4 < NC / 4; ++c4) {
        float o[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int c = c4 * 4 + e;
            const bool cv = cb + c < n_rows;
            const float ib = cv ? __ldg(inv_norm + cb + c) : 0.0f;
            const float x = v[c] * ia * ib;
            if (DIST == ABX_DIST_KL) {
                // (h_i + h_j - <p_i, ln p_j> - <ln p_i, p_j>) / 2, h = sum p ln p
                const float nb = cv ? __ldg(nrm2 + cb + c) : 0.0f;
                o[e] = fmaxf(0.0f, 0.5f * (na + nb - x));
            } else if (DIST == ABX_DIST_EUCLIDEAN) {
                const float nb = cv ? __ldg(nrm2 + cb + c) : 0.0f;
                o[e] = sqrtf(fmaxf(0.0f, na + nb - 2.0f * x));
            } else if (DIST == ABX_DIST_COSINE) {
                o[e] = 1.0f - fminf(1.0f, fmaxf(-1.0f, x));
            } else {
                o[e] = acosf(fminf(1.0f, fmaxf(-1.0f, x))) * inv_pi;
            }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) out[(c4 * 4 + e) * (FUSED ? 1 : kPanel)] = o[e];
    }
}

// --------------------------------------------------------------- the kernel

// PREC: ABX_FP32 (split), ABX_BF16, ABX_FP8.  STAGES: smem ring depth.
// FUSED: the epilogue runs the tile's DTWs from a shared-memory d tile
// instead of writing the tile to global memory.
template <int PREC, int STAGES, bool FUSED>
__global__ void __launch_bounds__(kThreads, 1)
    umma_tile_kernel(const __grid_constant__ CUtensorMap tmap, UmmaParams p) {
    constexpr int kOps = PREC == ABX_FP32 ? 4 : 2;            // operand tiles per stage
    constexpr uint32_t kStageBytes = kOps * kTileBytes;
    constexpr int KIND = PREC == ABX_FP8 ? 1 : 0;
    // instruction descriptor: D = F32 (bits 4-5), A/B = BF16 (1) or E4M3 (0)
    // (bits 7-9, 10-12), both K-major, N >> 3 at bits 17-22, M >> 4 at 24-28
    constexpr uint32_t kFmt = PREC == ABX_FP8 ? 0u : 1u;
    constexpr uint32_t kIdesc = (1u << 4) | (kFmt << 7) | (kFmt << 10) |
                                ((uint32_t)(kPanel >> 3) << 17) | ((uint32_t)(kPanel >> 4) << 24);

    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    float *dtile = reinterpret_cast<float *>(smem + STAGES * kStageBytes);     // FUSED
    uint32_t *lenbuf = reinterpret_cast<uint32_t *>(dtile + kPanel * kDLd);     // FUSED
    uint64_t *full = reinterpret_cast<uint64_t *>(
        smem + STAGES * kStageBytes +
        (FUSED ? (size_t)kPanel * kDLd * 4 + (size_t)kFuseMaxLen * kEpiThreads * 4 : 0));
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
            mbar_init(&acc_empty[b], kEpiWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(kTmemCols)
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
            for (int64_t t = blockIdx.x; t < p.n_tiles && ok; t += gridDim.x) {
                if (p.tile_count[t] == 0) continue;
                const int2 pp = p.tiles[t];
                const int32_t ra = p.panel_row[pp.x], rb = p.panel_row[pp.y];
                for (int kc = 0; kc < nk && ok; ++kc) {
                    if (!(ok = mbar_wait(&empty[s], ph ^ 1u, p.err, 11))) break;
                    uint8_t *st = smem + s * kStageBytes;
                    mbar_expect_tx(&full[s], kStageBytes);
                    const int32_t x = kc * (PREC == ABX_FP8 ? 128 : 64);
                    int32_t xb = x + p.b_rot;
                    if (xb >= p.k_elems) xb -= p.k_elems;
                    tma_load_2d(st, &tmap, &full[s], x, ra);
                    tma_load_2d(st + kTileBytes, &tmap, &full[s], xb, rb);
                    if (PREC == ABX_FP32) {
                        tma_load_2d(st + 2 * kTileBytes, &tmap, &full[s], x + p.lo_offset, ra);
                        tma_load_2d(st + 3 * kTileBytes, &tmap, &full[s], xb + p.lo_offset, rb);
                    }
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
            for (int64_t t = blockIdx.x; t < p.n_tiles && ok; t += gridDim.x) {
                if (p.tile_count[t] == 0) continue;
                const int b = local & 1;
                const uint32_t aph = (uint32_t)(local >> 1) & 1u;
                if (!(ok = mbar_wait(&acc_empty[b], aph ^ 1u, p.err, 12))) break;
                fence_after();
                const uint32_t d = tmem + (uint32_t)(b * kPanel);
                for (int kc = 0; kc < nk && ok; ++kc) {
                    if (!(ok = mbar_wait(&full[s], ph, p.err, 13))) break;
                    fence_after();
                    const uint32_t base = smem_u32(smem + s * kStageBytes);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint32_t off = kk * 32;  // 32 bytes = one MMA's k extent
                        const uint64_t ah = sdesc(base + off), bh = sdesc(base + kTileBytes + off);
                        const uint32_t acc0 = (kc | kk) ? 1u : 0u;
                        umma<KIND>(d, ah, bh, kIdesc, acc0);
                        if (PREC == ABX_FP32) {
                            const uint64_t al = sdesc(base + 2 * kTileBytes + off);
                            const uint64_t bl = sdesc(base + 3 * kTileBytes + off);
                            umma<KIND>(d, ah, bl, kIdesc, 1u);
                            umma<KIND>(d, al, bh, kIdesc, 1u);
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
        __syncwarp();
    } else {
        // ---------------- epilogue
        const int ew = warp - 2;
        const int q = warp & 3;            // TMEM lane quarter this warp may access
        const int half = ew >> 2;          // column half
        const int row = q * 32 + lane;
        int local = 0;
        bool ok = true;
        const int etid = threadIdx.x - 64;  // 0..255 over the epilogue warps
        for (int64_t t = blockIdx.x; t < p.n_tiles && ok; t += gridDim.x) {
            if (p.tile_count[t] == 0) continue;
            const int b = local & 1;
            const uint32_t aph = (uint32_t)(local >> 1) & 1u;
            ok = mbar_wait(&acc_full[b], aph, p.err, 14);
            if (FUSED) {
                // all epilogue warps take the same decision
                if (epi_bar_or(!ok)) break;
            } else {
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) break;
            }
            fence_after();
            float v[64];
            const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * kPanel + half * 64);
            tmem_ld32(ta, v);
            tmem_ld32(ta + 32, v + 32);
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[b]);
            const int2 pp = p.tiles[t];
            const int64_t ra = p.panel_row[pp.x] + row;
            const int64_t cb = p.panel_row[pp.y] + half * 64;
            const float ia = ra < p.n_rows ? p.inv_norm[ra] : 0.0f;
            float *out = FUSED ? dtile + row * kDLd + half * 64
                               : p.tilebuf + t * (int64_t)(kPanel * kPanel) + half * 64 * kPanel + row;
            // one unrolled store loop per distance, chosen once per tile
            if (p.distance == ABX_DIST_KL)
                epi_row<ABX_DIST_KL, FUSED>(v, ia, ra < p.n_rows ? p.nrm2[ra] : 0.0f, cb,
                                            p.n_rows, p.inv_norm, p.nrm2, out);
            else if (p.distance == ABX_DIST_EUCLIDEAN)
                epi_row<ABX_DIST_EUCLIDEAN, FUSED>(v, ia, ra < p.n_rows ? p.nrm2[ra] : 0.0f, cb,
                                                   p.n_rows, p.inv_norm, p.nrm2, out);
            else if (p.distance == ABX_DIST_COSINE)
                epi_row<ABX_DIST_COSINE, FUSED>(v, ia, 0.0f, cb, p.n_rows, p.inv_norm, p.nrm2, out);
            else
                epi_row<ABX_DIST_ANGULAR, FUSED>(v, ia, 0.0f, cb, p.n_rows, p.inv_norm, p.nrm2, out);
            if (FUSED) {
                epi_bar();
                // every needed pair of this tile: DTW in place on its block
                const int64_t pe = p.tile_base[t + 1];
                for (int64_t pi = p.tile_base[t] + etid; pi < pe; pi += kEpiThreads) {
                    const int4 pr = p.pairs[pi];
                    const int x = pr.x, y = pr.y;
                    const int rx = pr.w & 0xffff, cy = pr.w >> 16;
                    const int Tx = p.len[x], Ty = p.len[y];
                    const DtwBound bd = dtw_bound(Tx, Ty, p.theta_item[x], p.theta_item[y],
                                                  p.eps_c);
                    float dev = 0.0f, lc = 0.0f;
                    uint32_t ll = 0;
                    for (int i = 0; i < Tx; ++i) {
                        float *rw = dtile + (rx + i) * kDLd + cy;
                        const float *up = rw - kDLd;
                        float dc = ABX_INF;
                        uint32_t dl = 0;
                        lc = ABX_INF;
                        ll = 0;
                        for (int j = 0; j < Ty; ++j) {
                            const float dij = rw[j];
                            const float uc = i > 0 ? up[j] : ABX_INF;
                            const uint32_t ul = i > 0 ? lenbuf[j * kEpiThreads + etid] : 0u;
                            dev = fmaxf(dev, fabsf(dij - 0.5f));
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
                            rw[j] = nc;
                            lenbuf[j * kEpiThreads + etid] = info;
                        }
                    }
                    const uint32_t L = ll & 0xffu;
                    const float D = __fdiv_rn(lc, (float)L);
                    float lo, hi;
                    dtw_interval(bd, lc, ll, dev, p.eps_c, p.intervals, D, lo, hi);
                    const int4 gm = p.gmeta[p.item_g[x]];
                    const int gb = gm.x;
                    const int64_t ng = gm.y;
                    const int64_t base = ((int64_t)(uint32_t)gm.w << 32) | (uint32_t)gm.z;
                    const PairVal pvv{D, lo, hi, L};
                    p.pv[base + (int64_t)(x - gb) * ng + (y - gb)] = pvv;
                    p.pv[base + (int64_t)(y - gb) * ng + (x - gb)] = pvv;
                }
                epi_bar();
            }
            ++local;
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols)
                     : "memory");
    }
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
    constexpr bool kSplit = PREC == ABX_FP32;
    constexpr int kNC = kPanel / (EW / 4);  // columns per epilogue thread and tile
    // stage: A (hi), [A lo], B (two panels, hi), [B lo (two panels)]
    constexpr uint32_t kA = 0, kAlo = kTileBytes, kB = kSplit ? 2 * kTileBytes : kTileBytes;
    constexpr uint32_t kBlo = kB + 2 * kTileBytes;
    constexpr uint32_t kStageBytes = (kSplit ? 6 : 3) * kTileBytes;
    constexpr int KIND = PREC == ABX_FP8 ? 1 : 0;
    constexpr uint32_t kFmt = PREC == ABX_FP8 ? 0u : 1u;
    constexpr uint32_t kIdescBase = (1u << 4) | (kFmt << 7) | (kFmt << 10) |
                                    ((uint32_t)(kPanel >> 4) << 24);
    constexpr uint32_t kCols = 512;  // two 256-column FP32 accumulators

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
                const uint32_t bytes = (kSplit ? 2u : 1u) * (1u + (uint32_t)nb) * kTileBytes;
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
                    if (kSplit) {
                        tma_load_2d(st + kAlo, &tmap, &full[s], x + p.lo_offset, ra);
                        tma_load_2d(st + kBlo, &tmap, &full[s], xb + p.lo_offset, rb0);
                        if (nb == 2)
                            tma_load_2d(st + kBlo + kTileBytes, &tmap, &full[s], xb + p.lo_offset,
                                        rb1);
                    }
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
                const int b = local & 1;
                const uint32_t aph = (uint32_t)(local >> 1) & 1u;
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
                        if (kSplit) {
                            const uint64_t al = sdesc(base + kAlo + off);
                            const uint64_t bl = sdesc(base + kBlo + off);
                            umma<KIND>(d, ah, bl, idesc, 1u);
                            umma<KIND>(d, al, bh, idesc, 1u);
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
            const int b = local & 1;
            const uint32_t aph = (uint32_t)(local >> 1) & 1u;
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
                float *out =
                    p.tilebuf + t * (int64_t)(kPanel * kPanel) + slice * kNC * kPanel + row;
                if (p.distance == ABX_DIST_KL)
                    epi_row<ABX_DIST_KL, false, kNC>(v, ia, ra < p.n_rows ? p.nrm2[ra] : 0.0f,
                                                     cb, p.n_rows, p.inv_norm, p.nrm2, out);
                else if (p.distance == ABX_DIST_EUCLIDEAN)
                    epi_row<ABX_DIST_EUCLIDEAN, false, kNC>(v, ia,
                                                            ra < p.n_rows ? p.nrm2[ra] : 0.0f, cb,
                                                            p.n_rows, p.inv_norm, p.nrm2, out);
                else if (p.distance == ABX_DIST_COSINE)
                    epi_row<ABX_DIST_COSINE, false, kNC>(v, ia, 0.0f, cb, p.n_rows, p.inv_norm,
                                                         p.nrm2, out);
                else
                    epi_row<ABX_DIST_ANGULAR, false, kNC>(v, ia, 0.0f, cb, p.n_rows, p.inv_norm,
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

// WIDE = 0: narrow kernel; 8 or 16: wide kernel with that many epilogue warps
template <int PREC, int STAGES, bool FUSED, int WIDE = 0>
cudaError_t launch_prec(const TileGemmArgs &a, int n_sm, int32_t *err, cudaStream_t s) {
    auto fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    const int elem = PREC == ABX_FP8 ? 1 : 2;
    const int64_t width = PREC == ABX_FP32 ? 2 * (int64_t)a.dim_pad : a.dim_pad;  // elements
    CUtensorMap map;
    cuuint64_t gdim[2] = {(cuuint64_t)width, (cuuint64_t)a.n_rows};
    cuuint64_t gstride[1] = {(cuuint64_t)(width * elem)};
    cuuint32_t box[2] = {(cuuint32_t)(128 / elem), (cuuint32_t)kPanel};
    cuuint32_t estride[2] = {1, 1};
    CUresult r = fn(&map, PREC == ABX_FP8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                          : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                    2, const_cast<void *>(a.packed), gdim, gstride, box, estride,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    UmmaParams p;
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
    constexpr int kOps = WIDE ? (PREC == ABX_FP32 ? 6 : 3) : (PREC == ABX_FP32 ? 4 : 2);
    const size_t smem = 1024 + (size_t)STAGES * kOps * kTileBytes + 256 +
                        (FUSED ? (size_t)kPanel * kDLd * 4 + (size_t)kFuseMaxLen * kEpiThreads * 4
                               : 0);
    auto kern = [] {
        if constexpr (WIDE != 0)
            return umma_wide_kernel<PREC, STAGES, WIDE>;
        else
            return umma_tile_kernel<PREC, STAGES, FUSED>;
    }();
    const int threads = WIDE ? 32 * (2 + WIDE) : kThreads;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t items = WIDE ? a.n_work : a.n_tiles;
    const int grid = (int)(items < n_sm ? items : n_sm);
    if (grid == 0) return cudaSuccess;
    {
        ProfScope ps_(FUSED ? (PREC == ABX_FP32 ? "tile_dtw_umma_fp32split"
                                                : PREC == ABX_BF16 ? "tile_dtw_umma_bf16"
                                                                   : "tile_dtw_umma_fp8")
                            : (PREC == ABX_FP32 ? "tile_umma_fp32split"
                                                : PREC == ABX_BF16 ? "tile_umma_bf16"
                                                                   : "tile_umma_fp8"),
                      s);
        kern<<<grid, threads, smem, s>>>(map, p);
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
    if (a.fused) {
        if (precision == ABX_FP32) return launch_prec<ABX_FP32, 2, true>(a, n_sm, a.err, s);
        if (precision == ABX_BF16) return launch_prec<ABX_BF16, 4, true>(a, n_sm, a.err, s);
        if (precision == ABX_FP8) return launch_prec<ABX_FP8, 4, true>(a, n_sm, a.err, s);
        return cudaErrorNotSupported;
    }
    // variants (autotuner): 0 = the default ring depth, 1 = a shallower ring,
    // 2 = wide work items (two tiles of a panel row, N = 256)
    if (a.variant == 2 && a.work) {
        if (precision == ABX_FP32) return launch_prec<ABX_FP32, 2, false, 8>(a, n_sm, a.err, s);
        if (precision == ABX_BF16) return launch_prec<ABX_BF16, 4, false, 8>(a, n_sm, a.err, s);
        if (precision == ABX_FP8) return launch_prec<ABX_FP8, 4, false, 8>(a, n_sm, a.err, s);
        return cudaErrorNotSupported;
    }
    // 3 = wide work items with 16 epilogue warps
    if (a.variant == 3 && a.work) {
        if (precision == ABX_FP32) return launch_prec<ABX_FP32, 2, false, 16>(a, n_sm, a.err, s);
        if (precision == ABX_BF16) return launch_prec<ABX_BF16, 4, false, 16>(a, n_sm, a.err, s);
        if (precision == ABX_FP8) return launch_prec<ABX_FP8, 4, false, 16>(a, n_sm, a.err, s);
        return cudaErrorNotSupported;
    }
    if (a.variant == 1) {
        if (precision == ABX_FP32) return launch_prec<ABX_FP32, 2, false>(a, n_sm, a.err, s);
        if (precision == ABX_BF16) return launch_prec<ABX_BF16, 4, false>(a, n_sm, a.err, s);
        if (precision == ABX_FP8) return launch_prec<ABX_FP8, 4, false>(a, n_sm, a.err, s);
        return cudaErrorNotSupported;
    }
    if (precision == ABX_FP32) return launch_prec<ABX_FP32, 3, false>(a, n_sm, a.err, s);
    if (precision == ABX_BF16) return launch_prec<ABX_BF16, 6, false>(a, n_sm, a.err, s);
    if (precision == ABX_FP8) return launch_prec<ABX_FP8, 6, false>(a, n_sm, a.err, s);
    return cudaErrorNotSupported;
}

int umma_fuse_max_len() { return kFuseMaxLen; }

}  // namespace abx
