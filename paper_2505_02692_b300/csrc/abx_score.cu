// Scoring kernels (fastabx Sec. 2): per-cell triple counts
//   N_C = sum over (a, b, x) of 2 * 1[d(x,a) < d(x,b)] + 1[d(x,a) = d(x,b)],
// the level-by-level collapse, and the FP64 recheck of undecided triples.
//
// Cells are never materialised.  A cell key is the tuple (on_ax, on_b, by
// values, across pair); the collapse averages over the attributes of each
// level in a fixed order.  The first kernel runs one thread per key of the
// first level's result (all key digits except the level-1 attributes) and
// loops over the level-1 attribute values in increasing order, looking up the
// cell's three item blocks in the dense (group, on, across) table.  The
// result array is dense in mixed radix with the next level's digits
// innermost, so each further level is a contiguous segmented mean.  All sums
// run in a fixed order, so the FP64 result does not depend on scheduling.
#include <cuda_runtime.h>

#include <algorithm>

#include "abx_internal.h"

namespace abx {
namespace {

enum { PASS_MARK = 0, PASS_SCORE = 1, PASS_COUNT = 2, PASS_EMIT = 3 };

__device__ __forceinline__ int decide(float a, float b) { return a < b ? 2 : (a == b ? 1 : 0); }

// 2 (win) / 0 (loss) when the stored values settle the triple, -1 when the
// FP64 values are needed: intervals overlap (mode 1) or the margin is below
// the stated bound (mode 2).
__device__ __forceinline__ int settled(const ScoreArgs &a, const PairVal &va, const PairVal &vb) {
    if (a.recheck == 2) {
        // strict: with margin 0 an exact tie still goes to FP64
        if (va.d + a.margin < vb.d) return 2;
        if (vb.d + a.margin < va.d) return 0;
        return -1;
    }
    if (va.hi < vb.lo) return 2;
    if (vb.hi < va.lo) return 0;
    return -1;
}
__device__ __forceinline__ int decide64(double a, double b) { return a < b ? 2 : (a == b ? 1 : 0); }

// Subsampler draw (Sec. 3.1 Subsampler): SplitMix64's output function
// (Steele, Lea & Flood 2014) on state x; a sequence is hashed by
// h <- mix64(h xor v).  Per cell and role, the kept items are the cap items
// with the smallest mix64(h_role xor item id) (ties by id); for across tasks
// the kept across_x values of a (by, on_ax, on_b, across_ab) are the ones
// with the smallest mix64(h xor across_x).
__device__ __forceinline__ uint64_t mix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// h of (seed, role, by values..., on_ax, on_b, across_ab[, across_x])
__device__ __forceinline__ uint64_t cell_hash(const ScoreArgs &a, const int32_t *cv, int role,
                                              int P, int Q, int s_ab, int s_x, bool with_x) {
    uint64_t h = mix64(a.sub_seed);
    h = mix64(h ^ (uint64_t)role);
    for (int b = 0; b < a.n_by; ++b) h = mix64(h ^ (uint64_t)(uint32_t)cv[2 + b]);
    h = mix64(h ^ (uint64_t)P);
    h = mix64(h ^ (uint64_t)Q);
    h = mix64(h ^ (uint64_t)s_ab);
    if (with_x) h = mix64(h ^ (uint64_t)s_x);
    return h;
}

// Is this across cell's across_x among the sub_xmax kept ones?
__device__ __forceinline__ bool x_kept(const ScoreArgs &a, const int32_t *cv, int g, int P, int Q,
                                       int s_ab, int s_x) {
    const TaskDev &t = a.t;
    const uint64_t h = cell_hash(a, cv, 3, P, Q, s_ab, 0, false);
    const uint64_t mine = mix64(h ^ (uint64_t)s_x);
    int better = 0;
    for (int v = 0; v < t.K_s; ++v) {
        if (v == s_ab || v == s_x) continue;
        if (t.blk[((int64_t)g * t.K_s + v) * t.K_on + P].y == 0) continue;  // no such cell
        const uint64_t k = mix64(h ^ (uint64_t)v);
        better += (k < mine) || (k == mine && v < s_x);
    }
    return better < a.sub_xmax;
}

// Flag the unordered pair {x, y} (local indices) for the recheck; slots are
// assigned afterwards in entry order (launch_recheck_compact).
__device__ __forceinline__ void mark_pair(const ScoreArgs &a, int64_t base, int64_t ng, int gb,
                                          int lx, int ly) {
    int32_t *e = &a.rc_idx[base + (int64_t)min(lx, ly) * ng + max(lx, ly)];
    if (*e == -1) *e = -2;
}

__device__ __forceinline__ int slot_of(const ScoreArgs &a, int64_t base, int64_t ng, int lx,
                                       int ly) {
    return a.rc_idx[base + (int64_t)min(lx, ly) * ng + max(lx, ly)];
}

// List slot q for the FP64 stage (once).
__device__ __forceinline__ void mark_exact(const ScoreArgs &a, int q) {
    if (q < 0) return;  // not listed: the overflow flag is already set
    if (atomicCAS(&a.rc_state[q], 0, 1) == 0) a.rc64_list[atomicAdd(a.rc64_count, 1)] = q;
}

__device__ __forceinline__ double exact_at(const ScoreArgs &a, int q) {
    // every undecided pair was marked; a missing slot (list overflow, which
    // the host reports) yields NaN instead of an out-of-range read
    return q >= 0 ? a.rc_exact[q] : __longlong_as_double(0x7ff8000000000000ll);
}

// A triple (x, a, b) that the stored values leave undecided, at the current
// recheck stage: its decision (2 / 1 / 0), or -1 when it waits for a later
// stage, whose pairs are then marked.  Stage 0 marks both pairs for the
// refined recomputation (or directly for FP64 when there is no refined
// stage); stage 1 decides from the refined intervals when they do not
// overlap and lists the pairs for FP64 otherwise; stage 2 takes the same
// refined decision or the FP64 one.  A refined interval holds the exact
// distance, so either way the decision is that of the exact distances.
__device__ __forceinline__ int undecided_triple(const ScoreArgs &a, int64_t base, int64_t ng,
                                                int gb, int lx, int la, int lb) {
    if (a.stage == 0) {
        mark_pair(a, base, ng, gb, lx, la);
        mark_pair(a, base, ng, gb, lx, lb);
        return -1;
    }
    const int qa = slot_of(a, base, ng, lx, la), qb = slot_of(a, base, ng, lx, lb);
    if (a.rc_iv) {
        const float2 ia = qa >= 0 ? a.rc_iv[qa] : make_float2(0.0f, 1.0f);
        const float2 ib = qb >= 0 ? a.rc_iv[qb] : make_float2(0.0f, 1.0f);
        if (ia.y < ib.x) return 2;
        if (ib.y < ia.x) return 0;
        if (a.stage == 1) {
            mark_exact(a, qa);
            mark_exact(a, qb);
            return -1;
        }
    }
    return decide64(exact_at(a, qa), exact_at(a, qb));
}

// Digits of x in the mixed radix of ds[0..n-1] (last digit fastest) into
// cv[ds[d].comp]; divisions by the radices as multiply-high and shifts.
__device__ __forceinline__ void decode_digits(uint32_t x, const CollapseDigit *ds, int n,
                                              int32_t *cv) {
    for (int d = n - 1; d >= 0; --d) {
        const uint32_t q = fast_div(x, ds[d].fd);
        cv[ds[d].comp] = (int32_t)(x - q * (uint32_t)ds[d].radix);
        x = q;
    }
}

// Across pair code v = s_ab * K_s + s_x.
__device__ __forceinline__ void split_across(const ScoreArgs &a, int v, int &s_ab, int &s_x) {
    s_ab = (int)fast_div((uint32_t)v, a.ks_div);
    s_x = v - s_ab * a.t.K_s;
}

__global__ void __launch_bounds__(128) score_kernel(ScoreArgs a) {
    const int64_t seg = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (seg >= a.n_seg) return;
    if (a.gate && *(volatile unsigned long long *)&a.acc[a.gate] == 0) return;
    int32_t cv[2 + kMaxDims];
    decode_digits((uint32_t)seg, a.seg, a.n_seg_digits, cv);
    const int P = cv[0], Q = cv[1];
    const TaskDev &t = a.t;
    const int sc = 2 + a.n_by;  // component of the across pair
    double sum = 0.0;
    int32_t n = 0;
    unsigned long long s_num = 0, s_den = 0, s_cells = 0, s_trip = 0, s_und = 0, s_flip = 0;
    int64_t emit = (a.pass == PASS_EMIT) ? a.cell_count[seg] : 0;
    int64_t ncell = 0;
    bool dirty = false;

    // one cell: the level-1 digits come from loop index l
    auto cell = [&](int64_t l) {
        decode_digits((uint32_t)l, a.loop, a.n_loop_digits, cv);
        int s_ab = 0, s_x = 0;
        if (t.across) {
            split_across(a, cv[sc], s_ab, s_x);
            if (s_ab == s_x) return;
        }
        int64_t code = 0;
        for (int b = 0; b < a.n_by; ++b) code = code * a.by_radix[b] + cv[2 + b];
        const int g = a.gtab[code];
        if (g < 0) return;
        const int64_t ga = ((int64_t)g * t.K_s + s_ab) * t.K_on;
        const int2 A = t.blk[ga + P];
        const int2 B = t.blk[ga + Q];
        const int2 X = t.across ? t.blk[((int64_t)g * t.K_s + s_x) * t.K_on + P] : A;
        const int4 gm = t.gmeta[g];
        if (A.y == 0 || (!t.across && A.y < 2) || B.y == 0 || X.y == 0) return;
        const int gb = gm.x;
        const int64_t ng = gm.y;
        const int64_t base = ((int64_t)(uint32_t)gm.w << 32) | (uint32_t)gm.z;
        long long num2 = 0, cnt = 0;
        for (int xi = 0; xi < X.y; ++xi) {
            const int lx = X.x + xi - gb;
            const PairVal *rowx = a.pv + base + (int64_t)lx * ng;
            for (int ai = 0; ai < A.y; ++ai) {
                const int la = A.x + ai - gb;
                if (la == lx) continue;
                const PairVal va = rowx[la];
                for (int bi = 0; bi < B.y; ++bi) {
                    const int lb = B.x + bi - gb;
                    const PairVal vb = rowx[lb];
                    int dec;
                    const int st = a.recheck ? settled(a, va, vb) : -2;
                    if (st == -2) {
                        dec = decide(va.d, vb.d);
                    } else if (st >= 0) {
                        dec = st;
                    } else {
                        // not decidable from the stored values: a later
                        // stage of the recheck decides it, and the segment
                        // is then scored again
                        dec = undecided_triple(a, base, ng, gb, lx, la, lb);
                        if (dec < 0) {
                            dirty = true;
                            continue;
                        }
                        ++s_und;
                        s_flip += decide(va.d, vb.d) != dec;
                    }
                    num2 += dec;
                    ++cnt;
                }
            }
        }
        if (a.pass == PASS_SCORE) {
            sum += (double)num2 / (2.0 * (double)cnt);
            ++n;
            s_num += num2;
            s_den += 2 * cnt;
            ++s_cells;
            s_trip += cnt;
        } else if (a.pass == PASS_COUNT) {
            ++ncell;
        } else if (a.pass == PASS_EMIT) {
            int32_t *k = a.cell_keys + emit * a.key_width;
            k[0] = P;
            k[1] = Q;
            k[2] = s_ab;
            k[3] = s_x;
            for (int b = 0; b < a.n_by; ++b) k[4 + b] = cv[2 + b];
            a.cell_num2[emit] = num2;
            a.cell_cnt[emit] = cnt;
            ++emit;
        }
    };

    if (P != Q) {
        if (a.bits) {
            // level-1 values where all three blocks exist, in increasing order
            int s_ab = 0, s_x = 0;
            bool ok = true;
            if (t.across) {
                split_across(a, cv[sc], s_ab, s_x);
                ok = s_ab != s_x;
            }
            if (ok) {
                int64_t rest = 0;
                for (int i = 0; i < a.n_rest; ++i) {
                    const int b = a.rest_by[i];
                    rest = rest * a.by_radix[b] + cv[2 + b];
                }
                const int W = a.bits_words;
                const uint32_t *ra = a.bits + (((int64_t)P * t.K_s + s_ab) * a.rest_radix + rest) * W;
                const uint32_t *rb = a.bits + (((int64_t)Q * t.K_s + s_ab) * a.rest_radix + rest) * W;
                const uint32_t *rx = a.bits + (((int64_t)P * t.K_s + s_x) * a.rest_radix + rest) * W;
                for (int w = 0; w < W; ++w) {
                    uint32_t m = __ldg(ra + w) & __ldg(rb + w) & __ldg(rx + w);
                    while (m) {
                        const int bit = __ffs(m) - 1;
                        m &= m - 1;
                        cell((int64_t)w * 32 + bit);
                    }
                }
            }
        } else {
            for (int64_t l = 0; l < a.loop_len; ++l) cell(l);
        }
    }
    if (dirty) atomicAdd(&a.acc[a.dirty_slot], 1ull);
    if (a.pass == PASS_SCORE) {
        a.res[seg] = n ? sum / (double)n : 0.0;
        a.res_n[seg] = n;
        if (s_cells) {
            atomicAdd(&a.acc[0], s_num);
            atomicAdd(&a.acc[1], s_den);
            atomicAdd(&a.acc[2], s_cells);
            atomicAdd(&a.acc[3], s_trip);
        }
        if (s_und) atomicAdd(&a.acc[4], s_und);
        if (s_flip) atomicAdd(&a.acc[5], s_flip);
    } else if (a.pass == PASS_COUNT) {
        a.cell_count[seg] = ncell;
    }
}

// ------------------------------------------------- materialised-cell path
// Used when the level-1 attributes are by attributes only (presence bitsets
// available).  Each cell becomes one thread, so the chain of dependent loads
// of one cell (group table, blocks, pair records) no longer serialises
// within a segment; the per-segment means then sum contiguous, ordered cell
// ranges.

__device__ __forceinline__ void decode_seg(const ScoreArgs &a, int64_t seg, int32_t *cv) {
    decode_digits((uint32_t)seg, a.seg, a.n_seg_digits, cv);
}

// Bitset rows of the three blocks of a segment; false if it has no cell.
__device__ __forceinline__ bool seg_rows(const ScoreArgs &a, const int32_t *cv,
                                         const uint32_t **ra, const uint32_t **rb,
                                         const uint32_t **rx) {
    const TaskDev &t = a.t;
    const int P = cv[0], Q = cv[1];
    if (P == Q) return false;
    int s_ab = 0, s_x = 0;
    if (t.across) {
        split_across(a, cv[2 + a.n_by], s_ab, s_x);
        if (s_ab == s_x) return false;
    }
    int64_t rest = 0;
    for (int i = 0; i < a.n_rest; ++i) {
        const int b = a.rest_by[i];
        rest = rest * a.by_radix[b] + cv[2 + b];
    }
    const int W = a.bits_words;
    *ra = a.bits + (((int64_t)P * t.K_s + s_ab) * a.rest_radix + rest) * W;
    *rb = a.bits + (((int64_t)Q * t.K_s + s_ab) * a.rest_radix + rest) * W;
    *rx = a.bits + (((int64_t)P * t.K_s + s_x) * a.rest_radix + rest) * W;
    return true;
}

__global__ void __launch_bounds__(256) seg_count_kernel(ScoreArgs a) {
    const int64_t seg = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (seg >= a.n_seg) return;
    int32_t cv[2 + kMaxDims];
    decode_seg(a, seg, cv);
    const uint32_t *ra, *rb, *rx;
    int n = 0;
    if (seg_rows(a, cv, &ra, &rb, &rx))
        for (int w = 0; w < a.bits_words; ++w) n += __popc(__ldg(ra + w) & __ldg(rb + w) & __ldg(rx + w));
    a.seg_n[seg] = n;
}

__global__ void __launch_bounds__(256) cell_enum_kernel(ScoreArgs a) {
    const int64_t seg = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (seg >= a.n_seg || a.seg_n[seg] == 0) return;
    int32_t cv[2 + kMaxDims];
    decode_seg(a, seg, cv);
    const uint32_t *ra, *rb, *rx;
    seg_rows(a, cv, &ra, &rb, &rx);
    int64_t o = a.seg_base[seg];
    for (int w = 0; w < a.bits_words; ++w) {
        uint32_t m = __ldg(ra + w) & __ldg(rb + w) & __ldg(rx + w);
        while (m) {
            const int bit = __ffs(m) - 1;
            m &= m - 1;
            // the arrays hold cell_cap cells; a larger device total is
            // reported by the host check and nothing is stored past the end
            if (o < a.cell_cap) a.cell_id[o] = make_int2((int32_t)seg, w * 32 + bit);
            ++o;
        }
    }
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Small cells, one thread per cell: N and |C| (|C| = 0 marks a candidate
// without a triple, a within-style block of one item).  A cell with more than
// kBigCell candidate triples goes to the big-cell list instead, which one warp
// per cell evaluates next (cell_eval_big_kernel): cells range from one triple
// to thousands, and one thread per cell would leave warps waiting on their
// largest cell, while one warp per cell would waste lanes on the many tiny
// cells.
constexpr int kBigCell = 32;

__global__ void __launch_bounds__(256) cell_eval_kernel(ScoreArgs a) {
    if (a.gate && *(volatile unsigned long long *)&a.acc[a.gate] == 0) return;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = min(*a.n_cells_dev, a.cell_cap);
    long long num2 = 0, cnt = 0;
    unsigned long long und = 0, flip = 0;
    bool dirty = false;
    if (c < total) {
        const TaskDev &t = a.t;
        const int2 id = a.cell_id[c];
        int32_t cv[2 + kMaxDims];
        decode_seg(a, id.x, cv);
        decode_digits((uint32_t)id.y, a.loop, a.n_loop_digits, cv);
        const int P = cv[0], Q = cv[1];
        int s_ab = 0, s_x = 0;
        if (t.across) split_across(a, cv[2 + a.n_by], s_ab, s_x);
        int64_t code = 0;
        for (int b = 0; b < a.n_by; ++b) code = code * a.by_radix[b] + cv[2 + b];
        const int g = a.gtab[code];
        const int64_t ga = ((int64_t)g * t.K_s + s_ab) * t.K_on;
        const int2 A = t.blk[ga + P];
        const int2 B = t.blk[ga + Q];
        const int2 X = t.across ? t.blk[((int64_t)g * t.K_s + s_x) * t.K_on + P] : A;
        const int4 gm = t.gmeta[g];
        const bool capped = a.sub_cap > 0 && (X.y > a.sub_cap || A.y > a.sub_cap || B.y > a.sub_cap);
        if (a.sub_xmax > 0 && t.across && !x_kept(a, cv, g, P, Q, s_ab, s_x)) {
            // dropped by the across_x limit: no triple
        } else if (capped || (int64_t)X.y * A.y * B.y > kBigCell) {
            a.big[atomicAdd((unsigned long long *)a.big_count, 1ull)] = c;
        } else if (!(!t.across && A.y < 2)) {
            const int gb = gm.x;
            const int64_t ng = gm.y;
            const int64_t base = ((int64_t)(uint32_t)gm.w << 32) | (uint32_t)gm.z;
            for (int xi = 0; xi < X.y; ++xi) {
                const int lx = X.x + xi - gb;
                const PairVal *rowx = a.pv + base + (int64_t)lx * ng;
                for (int ai = 0; ai < A.y; ++ai) {
                    const int la = A.x + ai - gb;
                    if (la == lx) continue;
                    const PairVal va = rowx[la];
                    for (int bi = 0; bi < B.y; ++bi) {
                        const int lb = B.x + bi - gb;
                        const PairVal vb = rowx[lb];
                        int dec;
                        const int st = a.recheck ? settled(a, va, vb) : -2;
                        if (st == -2) {
                            dec = decide(va.d, vb.d);
                        } else if (st >= 0) {
                            dec = st;
                        } else {
                            dec = undecided_triple(a, base, ng, gb, lx, la, lb);
                            if (dec < 0) {
                                dirty = true;
                                continue;
                            }
                            ++und;
                            flip += decide(va.d, vb.d) != dec;
                        }
                        num2 += dec;
                        ++cnt;
                    }
                }
            }
        }
        a.cell_num2[c] = num2;
        a.cell_cnt[c] = cnt;
    }
    // statistics summed over the block first: every block adding to the same
    // few counters would serialise on them in L2
    __shared__ unsigned long long part[8][7];
    unsigned long long v[7] = {(unsigned long long)num2, 2ull * (unsigned long long)cnt,
                               (unsigned long long)(cnt > 0), (unsigned long long)cnt, und,
                               flip, (unsigned long long)dirty};
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        v[i] = warp_sum_u64(v[i]);
        if (lane == 0) part[wid][i] = v[i];
    }
    __syncthreads();
    if (threadIdx.x < 7) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w][threadIdx.x];
        // counters 0-3: sums of N, 2|C|, cells, triples; 4-5: undecided and
        // flipped triples; 6 -> acc[dirty_slot]: cells that met a deferred triple
        if (t) atomicAdd(&a.acc[threadIdx.x == 6 ? a.dirty_slot : threadIdx.x], t);
    }
}

// Big cells, one warp per cell: the lanes walk the cell's (x, a, b) index
// space flattened with b fastest, so the lanes of one step read consecutive
// entries of x's row of the group matrix.
__global__ void __launch_bounds__(256, 4) cell_eval_big_kernel(ScoreArgs a) {
    if (a.gate && *(volatile unsigned long long *)&a.acc[a.gate] == 0) return;
    // per warp: kept positions of A, B, X (dynamic shared memory, 8 warps x
    // 3 x sub_cap entries; none without the subsampler)
    extern __shared__ int32_t s_sel[];
    const int lane = threadIdx.x & 31;
    int32_t *sel_w = s_sel + ((threadIdx.x >> 5) & 7) * 3 * (a.sub_cap > 0 ? a.sub_cap : 1);
    auto sel = [&](int r, int i) -> int32_t & { return sel_w[r * a.sub_cap + i]; };
    const int64_t total = *a.big_count;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    unsigned long long s_num = 0, s_den = 0, s_cells = 0, s_trip = 0, s_und = 0, s_flip = 0,
                       s_dirty = 0;
    const TaskDev &t = a.t;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < total;
         w += warps) {
        const int64_t c = a.big[w];
        const int2 id = a.cell_id[c];
        int32_t cv[2 + kMaxDims];
        decode_seg(a, id.x, cv);
        decode_digits((uint32_t)id.y, a.loop, a.n_loop_digits, cv);
        const int P = cv[0], Q = cv[1];
        int s_ab = 0, s_x = 0;
        if (t.across) split_across(a, cv[2 + a.n_by], s_ab, s_x);
        int64_t code = 0;
        for (int b = 0; b < a.n_by; ++b) code = code * a.by_radix[b] + cv[2 + b];
        const int g = a.gtab[code];
        const int64_t ga = ((int64_t)g * t.K_s + s_ab) * t.K_on;
        const int2 A = t.blk[ga + P];
        const int2 B = t.blk[ga + Q];
        const int2 X = t.across ? t.blk[((int64_t)g * t.K_s + s_x) * t.K_on + P] : A;
        const int4 gm = t.gmeta[g];
        long long num2 = 0, cnt = 0;
        unsigned long long und = 0, flip = 0;
        bool dirty = false;
        if (!(!t.across && A.y < 2)) {
            const int gb = gm.x;
            const int64_t ng = gm.y;
            const int64_t base = ((int64_t)(uint32_t)gm.w << 32) | (uint32_t)gm.z;
            // one triple from its two pair records (loaded by the caller)
            auto decide_triple = [&](int lx, int la, int lb, const PairVal &va, const PairVal &vb) {
                int dec;
                const int st = a.recheck ? settled(a, va, vb) : -2;
                if (st == -2) {
                    dec = decide(va.d, vb.d);
                } else if (st >= 0) {
                    dec = st;
                } else {
                    dec = undecided_triple(a, base, ng, gb, lx, la, lb);
                    if (dec < 0) {
                        dirty = true;
                        return;
                    }
                    ++und;
                    flip += decide(va.d, vb.d) != dec;
                }
                num2 += dec;
                ++cnt;
            };
            auto visit = [&](int xi, int ai, int bi) {
                const int lx = X.x + xi - gb, la = A.x + ai - gb;
                if (la == lx) return;
                const int lb = B.x + bi - gb;
                const PairVal *rowx = a.pv + base + (int64_t)lx * ng;
                decide_triple(lx, la, lb, rowx[la], rowx[lb]);
            };
            // subsampler: positions kept in each role (identity when off)
            int mA = A.y, mB = B.y, mX = X.y;
            bool subA = false, subB = false, subX = false;
            if (a.sub_cap > 0) {
                auto pick = [&](int r, int2 blk, int &mr, bool &sr) {
                    const int n = blk.y;
                    if (n <= a.sub_cap) return;
                    const uint64_t h = cell_hash(a, cv, r, P, Q, s_ab, s_x, true);
                    for (int i = lane; i < n; i += 32) {
                        const uint64_t id_i = (uint64_t)t.item_id[blk.x + i];
                        const uint64_t k_i = mix64(h ^ id_i);
                        int rank = 0;
                        for (int j = 0; j < n; ++j) {
                            const uint64_t id_j = (uint64_t)t.item_id[blk.x + j];
                            const uint64_t k_j = mix64(h ^ id_j);
                            rank += (k_j < k_i) || (k_j == k_i && id_j < id_i);
                        }
                        if (rank < a.sub_cap) sel(r, rank) = i;
                    }
                    mr = a.sub_cap;
                    sr = true;
                };
                pick(0, A, mA, subA);
                pick(1, B, mB, subB);
                pick(2, X, mX, subX);
                __syncwarp();
            }
            const uint32_t nb = (uint32_t)mB, nab = (uint32_t)mA * nb;
            const bool any_sub = subA || subB || subX;
            // lane q of the flattened (x, a, b) space, b fastest, in steps of
            // 32: the three counters advance by the digits of 32 with carries
            // (the divisions run once per cell, not per triple)
            // lane q of the flattened (x, a, b) space, b fastest, in steps of
            // 32: the three counters advance by the digits of 32 with carries
            // (the divisions run once per cell, not per triple)
            auto walk = [&](auto &&fn) {
                const uint32_t n = (uint32_t)mX * nab;
                uint32_t xi = lane / nab, r = lane - xi * nab;
                uint32_t ai = r / nb, bi = r - ai * nb;
                const uint32_t dx = 32u / nab, r32 = 32u - dx * nab;
                const uint32_t da = r32 / nb, db = r32 - da * nb;
                for (uint32_t q = lane; q < n; q += 32) {
                    fn((int)xi, (int)ai, (int)bi);
                    bi += db;
                    ai += da;
                    xi += dx;
                    if (bi >= nb) {
                        bi -= nb;
                        ++ai;
                    }
                    if (ai >= (uint32_t)mA) {
                        ai -= (uint32_t)mA;
                        ++xi;
                    }
                }
            };
            if (!any_sub && (uint64_t)mX * nab < (1ull << 31)) {
                // no subsampling (the common case): positions are block offsets
                walk(visit);
            } else {
                auto visit_kept = [&](int xi, int ai, int bi) {
                    visit(subX ? sel(2, xi) : xi, subA ? sel(0, ai) : ai, subB ? sel(1, bi) : bi);
                };
                if ((uint64_t)mX * nab < (1ull << 31)) {
                    walk(visit_kept);
                } else {  // very large cells: x outer, (a, b) over the lanes
                    for (int xi = 0; xi < mX; ++xi)
                        for (uint32_t q = lane; q < nab; q += 32) {
                            const uint32_t ai = q / nb;
                            visit_kept(xi, (int)ai, (int)(q - ai * nb));
                        }
                }
            }
            __syncwarp();  // sel is rewritten by the warp's next cell
        }
        num2 = (long long)warp_sum_u64((unsigned long long)num2);
        cnt = (long long)warp_sum_u64((unsigned long long)cnt);
        const bool any_dirty = __any_sync(0xffffffffu, dirty);
        if (lane == 0) {
            a.cell_num2[c] = num2;
            a.cell_cnt[c] = cnt;
            if (cnt > 0) {
                s_num += (unsigned long long)num2;
                s_den += 2ull * (unsigned long long)cnt;
                s_cells += 1;
                s_trip += (unsigned long long)cnt;
            }
            s_dirty += any_dirty ? 1 : 0;
        }
        s_und += und;
        s_flip += flip;
    }
    // one set of atomics per warp
    s_und = warp_sum_u64(s_und);
    s_flip = warp_sum_u64(s_flip);
    if (lane == 0) {
        if (s_cells) {
            atomicAdd(&a.acc[0], s_num);
            atomicAdd(&a.acc[1], s_den);
            atomicAdd(&a.acc[2], s_cells);
            atomicAdd(&a.acc[3], s_trip);
        }
        if (s_und) atomicAdd(&a.acc[4], s_und);
        if (s_flip) atomicAdd(&a.acc[5], s_flip);
        if (s_dirty) atomicAdd(&a.acc[a.dirty_slot], s_dirty);
    }
}

// num / den for a den >= 1; a power-of-two den divides exactly by scaling,
// which is the correctly rounded quotient FP64 division would return.
__device__ __forceinline__ double div_exact_pow2(double num, long long den) {
    if ((den & (den - 1)) == 0)
        return num * __longlong_as_double((long long)(1023 - (__ffsll(den) - 1)) << 52);
    return num / (double)den;
}

// Ordered mean of D_C = N / (2 |C|) over each segment's contiguous cell
// range (cells are loaded four at a time; the sum keeps its order).  A warp
// per segment, the lanes loading 32 cells at a time with an ordered shuffle
// sum, measured slower: 32 segments per warp in parallel beat one segment's
// coalesced loads.
__global__ void __launch_bounds__(256) seg_reduce_kernel(ScoreArgs a) {
    const int64_t seg = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (seg >= a.n_seg) return;
    const int64_t b = min(a.seg_base[seg], a.cell_cap), e = min(a.seg_base[seg + 1], a.cell_cap);
    double sum = 0.0;
    int32_t n = 0;
    for (int64_t c0 = b; c0 < e; c0 += 4) {
        long long cnt[4], num2[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            cnt[i] = c0 + i < e ? a.cell_cnt[c0 + i] : 0;
            num2[i] = c0 + i < e ? a.cell_num2[c0 + i] : 0;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (cnt[i]) {
                sum += div_exact_pow2((double)num2[i], 2 * cnt[i]);
                ++n;
            }
    }
    a.res[seg] = n ? div_exact_pow2(sum, n) : 0.0;
    a.res_n[seg] = n;
}

// Keys of every candidate cell (|C| = 0 rows are dropped by the host).
__global__ void __launch_bounds__(256) cell_emit_kernel(ScoreArgs a) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= min(*a.n_cells_dev, a.cell_cap)) return;
    const int2 id = a.cell_id[c];
    int32_t cv[2 + kMaxDims];
    decode_seg(a, id.x, cv);
    decode_digits((uint32_t)id.y, a.loop, a.n_loop_digits, cv);
    int32_t *k = a.cell_keys + c * a.key_width;
    k[0] = cv[0];
    k[1] = cv[1];
    int s_ab = 0, s_x = 0;
    if (a.t.across) split_across(a, cv[2 + a.n_by], s_ab, s_x);
    k[2] = s_ab;
    k[3] = s_x;
    for (int b = 0; b < a.n_by; ++b) k[4 + b] = cv[2 + b];
}

// Adds the present entries among a warp's 32 values to s in lane order; every
// lane performs the same additions, so s is the sequential sum.
__device__ __forceinline__ void warp_ordered_add(double v, bool present, double &s, int64_t &n) {
    const unsigned m = __ballot_sync(0xffffffffu, present);
    n += __popc(m);
    // all 32 values first (independent shuffles), then the dependent adds
    double e[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) e[i] = __shfl_sync(0xffffffffu, v, i);
#pragma unroll
    for (int i = 0; i < 32; ++i)
        if (m & (1u << i)) s += e[i];
}

// Ordered sum of the present entries at in[at(k)], k < n, by one warp: each
// chunk of 32 entries is loaded (coalesced where at is) while the previous
// chunk is added.
template <class At>
__device__ __forceinline__ void warp_ordered_sum(const double *in, const int32_t *in_n, int64_t n,
                                                 At at, double &s, int64_t &cnt) {
    const int lane = threadIdx.x & 31;
    s = 0.0;
    cnt = 0;
    double v = 0.0;
    int32_t c = 0;
    if (lane < n) {
        v = in[at(lane)];
        c = in_n[at(lane)];
    }
    for (int64_t k0 = 0; k0 < n; k0 += 32) {
        const int64_t k = k0 + 32 + lane;
        double vn = 0.0;
        int32_t cn = 0;
        if (k < n) {
            vn = in[at(k)];
            cn = in_n[at(k)];
        }
        warp_ordered_add(v, c != 0, s, cnt);
        v = vn;
        c = cn;
    }
}

// Mean over the `radix` innermost entries of each key, existing ones only,
// summed in increasing order: one thread per key for short runs, one warp
// per key (collapse_warp_kernel) for runs of 32 and more.  One lane per key
// with the chunks transposed through shared memory (32 keys per warp, one
// FP64 addition per entry) measured slower on the triphone-scale step (0.42
// and, with NaN marking absent entries, 1.64 ms per step against 0.27).
__global__ void collapse_kernel(const double *in, const int32_t *in_n, int64_t n_out,
                                int64_t radix, double *out, int32_t *out_n) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_out) return;
    double s = 0.0;
    int32_t n = 0;
    const double *pin = in + k * radix;
    const int32_t *pn = in_n + k * radix;
    for (int64_t r = 0; r < radix; ++r)
        if (pn[r]) {
            s += pin[r];
            ++n;
        }
    out[k] = n ? div_exact_pow2(s, n) : 0.0;
    out_n[k] = n;
}

__global__ void collapse_warp_kernel(const double *in, const int32_t *in_n, int64_t n_out,
                                     int64_t radix, double *out, int32_t *out_n) {
    const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (k >= n_out) return;
    double s;
    int64_t n;
    const int64_t base = k * radix;
    warp_ordered_sum(in, in_n, radix, [&](int64_t r) { return base + r; }, s, n);
    if ((threadIdx.x & 31) == 0) {
        out[k] = n ? div_exact_pow2(s, n) : 0.0;
        out_n[k] = (int32_t)n;
    }
}

// Final mean over all existing entries in index order (one warp: the order
// of the FP64 sum is part of the result's definition).
__global__ void final_kernel(const double *in, const int32_t *in_n, int64_t n, double *out,
                             int64_t *out_n) {
    if (blockIdx.x) return;
    double s;
    int64_t c;
    warp_ordered_sum(in, in_n, n, [](int64_t k) { return k; }, s, c);
    if (threadIdx.x == 0) {
        *out = c ? div_exact_pow2(s, c) : 0.0;
        *out_n = c;
    }
}

// ---------------------------------------------------------------- recheck
// Distance of one item pair recomputed to FP64 accuracy from the raw FP32
// features: the angular frame distance arccos(<u,v> / (|u| |v|)) / pi and the
// DTW with the shorter-path rule (or the angular distance of the FP64 means).
//
// FP64 arithmetic is scarce on this GPU (about 1/64 of the FP32 rate), so the
// dot products, which are almost all of the work, run on the FP32 pipe in
// double-word arithmetic: each product u_k v_k is split exactly into two
// floats with an FMA (Dekker's product), and the running sums are float pairs
// added with the accurate double-word addition of Joldes, Muller and Popescu
// (ACM TOMS 2017, "AccurateDWPlusDW"; relative error at most 3u^2/(1-4u),
// u = 2^-24, per addition).  A pair sum h + l has at most 48 significant bits
// and converts exactly to a double.  Over the 24 + 5 additions of a lane sum
// and the warp tree the error stays below 3.2e-13 * sum |u_k v_k|, the same
// order as a sequential FP64 sum of 768 terms (768 * 2^-53 = 8.5e-14).  The
// norms, the division, arccos and the dynamic programme are FP64.

struct DW {
    float h, l;
};

// Knuth's two-sum: s + e = a + b exactly.
__device__ __forceinline__ DW two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

// Dekker's fast two-sum (|a| >= |b|): s + e = a + b exactly.
__device__ __forceinline__ DW fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// p + e = a * b exactly (barring underflow).
__device__ __forceinline__ DW two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

// Accurate double-word addition (two two-sums, two renormalisations).
__device__ __forceinline__ DW dw_add(DW a, DW b) {
    const DW s = two_sum(a.h, b.h);
    const DW t = two_sum(a.l, b.l);
    const DW v = fast_two_sum(s.h, __fadd_rn(s.l, t.h));
    return fast_two_sum(v.h, __fadd_rn(t.l, v.l));
}

// dw_add is commutative, so every lane ends with the same pair.
__device__ __forceinline__ DW dw_warp_sum(DW v) {
    for (int o = 16; o; o >>= 1) {
        const DW w{__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)};
        v = dw_add(v, w);
    }
    return v;
}

__device__ __forceinline__ double dw_to_double(DW v) { return (double)v.h + (double)v.l; }

// <u, v> of two feature rows by one warp, as a double-word sum.
__device__ __forceinline__ DW dw_dot(const float *__restrict__ u, const float *__restrict__ v,
                                     int dim, bool vec4, int lane) {
    DW acc{0.0f, 0.0f};
    if (vec4) {
        const float4 *u4 = reinterpret_cast<const float4 *>(u);
        const float4 *v4 = reinterpret_cast<const float4 *>(v);
        for (int c = lane; c < (dim >> 2); c += 32) {
            const float4 a = __ldg(u4 + c), b = __ldg(v4 + c);
            acc = dw_add(acc, two_prod(a.x, b.x));
            acc = dw_add(acc, two_prod(a.y, b.y));
            acc = dw_add(acc, two_prod(a.z, b.z));
            acc = dw_add(acc, two_prod(a.w, b.w));
        }
    } else {
        for (int c = lane; c < dim; c += 32) acc = dw_add(acc, two_prod(__ldg(u + c), __ldg(v + c)));
    }
    return dw_warp_sum(acc);
}

__device__ __forceinline__ double warp_sum_d(double v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Mean mode: one block per pair, FP64 means (few pairs, cheap).
__global__ void __launch_bounds__(256) recheck_mean_kernel(RecheckArgs a) {
    extern __shared__ double sm[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int count = min(*a.count, a.capacity);
    for (int k = blockIdx.x; k < count; k += gridDim.x) {
        const int q = a.slots ? a.slots[k] : k;
        const int2 pr = a.list[q];
        const int64_t ix = a.item_id[pr.x], iy = a.item_id[pr.y];
        const float *X = a.feats + a.offsets[ix] * (int64_t)a.dim;
        const float *Y = a.feats + a.offsets[iy] * (int64_t)a.dim;
        const int Tx = (int)(a.offsets[ix + 1] - a.offsets[ix]);
        const int Ty = (int)(a.offsets[iy + 1] - a.offsets[iy]);
        double *mx = sm, *my = sm + a.dim;
        for (int c = tid; c < a.dim; c += blockDim.x) {
            double s = 0.0;
            for (int t = 0; t < Tx; ++t) s += (double)X[(int64_t)t * a.dim + c];
            mx[c] = s / (double)Tx;
            s = 0.0;
            for (int t = 0; t < Ty; ++t) s += (double)Y[(int64_t)t * a.dim + c];
            my[c] = s / (double)Ty;
        }
        __syncthreads();
        if (warp == 0) {
            double uv = 0, uu = 0, vv = 0;
            for (int c = lane; c < a.dim; c += 32) {
                uv += mx[c] * my[c];
                uu += mx[c] * mx[c];
                vv += my[c] * my[c];
            }
            uv = warp_sum_d(uv);
            uu = warp_sum_d(uu);
            vv = warp_sum_d(vv);
            if (lane == 0) {
                double c = uv / (sqrt(uu) * sqrt(vv));
                c = fmin(1.0, fmax(-1.0, c));
                a.exact[q] = acos(c) / 3.141592653589793;
            }
        }
        __syncthreads();
    }
}

// DTW mode: one block of kRecheckThreads per pair; warp per dot product
// (frame norms and frame pairs), thread per frame distance, then the dynamic
// programme by one warp along anti-diagonals.
constexpr int kRecheckThreads = 128;

__global__ void __launch_bounds__(kRecheckThreads) recheck_dtw_kernel(RecheckArgs a) {
    extern __shared__ double sm[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int count = min(*a.count, a.capacity);
    const int ML = a.max_len;
    double *dm = sm;                       // [ML * ML]
    double *nrm = sm + (size_t)ML * ML;    // [2 * ML]
    short *ln = reinterpret_cast<short *>(nrm + 2 * ML);
    const bool vec4 = (a.dim & 3) == 0 && (reinterpret_cast<uintptr_t>(a.feats) & 15) == 0;
    for (int k = blockIdx.x; k < count; k += gridDim.x) {
        const int q = a.slots ? a.slots[k] : k;
        const int2 pr = a.list[q];
        const int64_t ix = a.item_id[pr.x], iy = a.item_id[pr.y];
        const float *X = a.feats + a.offsets[ix] * (int64_t)a.dim;
        const float *Y = a.feats + a.offsets[iy] * (int64_t)a.dim;
        const int Tx = (int)(a.offsets[ix + 1] - a.offsets[ix]);
        const int Ty = (int)(a.offsets[iy + 1] - a.offsets[iy]);
        auto frame = [&](int f) -> const float * {
            return f < Tx ? X + (int64_t)f * a.dim : Y + (int64_t)(f - Tx) * a.dim;
        };
        // 1. squared norms and cross dot products, warp per value (FP32 pipe)
        for (int w = warp; w < Tx + Ty + Tx * Ty; w += nw) {
            const float *u, *v;
            if (w < Tx + Ty) {
                u = v = frame(w);
            } else {
                const int e = w - Tx - Ty, i = e / Ty, j = e - i * Ty;
                u = frame(i);
                v = frame(Tx + j);
            }
            const DW r = dw_dot(u, v, a.dim, vec4, lane);
            // the pair (h, l) parks in the 8 bytes of its double slot
            if (lane == 0)
                *reinterpret_cast<float2 *>(w < Tx + Ty ? nrm + w : dm + (w - Tx - Ty)) =
                    make_float2(r.h, r.l);
        }
        __syncthreads();
        // 2. norms, then frame distances, thread per value (FP64, all lanes busy)
        for (int f = tid; f < Tx + Ty; f += blockDim.x) {
            const float2 r = *reinterpret_cast<const float2 *>(nrm + f);
            nrm[f] = sqrt(dw_to_double({r.x, r.y}));
        }
        __syncthreads();
        for (int e = tid; e < Tx * Ty; e += blockDim.x) {
            const int i = e / Ty, j = e - i * Ty;
            const float2 r = *reinterpret_cast<const float2 *>(dm + e);
            double c = dw_to_double({r.x, r.y}) / (nrm[i] * nrm[Tx + j]);
            c = fmin(1.0, fmax(-1.0, c));
            dm[e] = acos(c) / 3.141592653589793;
        }
        __syncthreads();
        // 3. the dynamic programme by warp 0 over anti-diagonals i + j = k: a
        // cell's predecessors lie on diagonals k - 1 and k - 2
        if (warp == 0) {
            for (int k = 0; k < Tx + Ty - 1; ++k) {
                const int i_lo = max(0, k - (Ty - 1)), i_hi = min(k, Tx - 1);
                for (int i = i_lo + lane; i <= i_hi; i += 32) {
                    const int j = k - i;
                    double bc = 0.0;
                    int bl = 0;
                    if (i || j) {
                        bool have = false;
                        const int pi[3] = {i - 1, i, i - 1}, pj[3] = {j, j - 1, j - 1};
                        for (int m = 0; m < 3; ++m) {
                            if (pi[m] < 0 || pj[m] < 0) continue;
                            const double pc = dm[pi[m] * Ty + pj[m]];
                            const int pl = ln[pi[m] * Ty + pj[m]];
                            if (!have || pc < bc || (pc == bc && pl < bl)) {
                                bc = pc;
                                bl = pl;
                                have = true;
                            }
                        }
                    }
                    dm[i * Ty + j] += bc;
                    ln[i * Ty + j] = (short)(bl + 1);
                }
                __syncwarp();
            }
            if (lane == 0) a.exact[q] = dm[Tx * Ty - 1] / (double)ln[Tx * Ty - 1];
        }
        __syncthreads();
    }
}

// One thread per (by code, on value, across value): set the presence bit of
// a non-empty block.
__global__ void bits_kernel(BitsArgs b) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per = (int64_t)b.K_on * b.K_s;
    if (i >= b.by_space * per) return;
    const int64_t code = i / per;
    const int32_t r = (int32_t)(i - code * per);
    const int32_t p = r % b.K_on, s = r / b.K_on;
    const int32_t g = b.gtab[code];
    if (g < 0 || b.blk[((int64_t)g * b.K_s + s) * b.K_on + p].y == 0) return;
    int32_t val[kMaxDims];
    int64_t rem = code;
    for (int k = b.n_by - 1; k >= 0; --k) {
        val[k] = (int32_t)(rem % b.by_radix[k]);
        rem /= b.by_radix[k];
    }
    int64_t l = 0, rest = 0, rest_radix = 1;
    for (int k = 0; k < b.n_loop; ++k) l = l * b.by_radix[b.loop_by[k]] + val[b.loop_by[k]];
    for (int k = 0; k < b.n_rest; ++k) {
        rest = rest * b.by_radix[b.rest_by[k]] + val[b.rest_by[k]];
        rest_radix *= b.by_radix[b.rest_by[k]];
    }
    const int64_t row = ((int64_t)p * b.K_s + s) * rest_radix + rest;
    atomicOr(&b.bits[row * b.words + l / 32], 1u << (l % 32));
}

// Slot assignment of the flagged pairs in entry order: group by group, and
// within a group row by row, so that the recheck kernels, which take the
// slots in order, work on one group's items at a time (they stay in L2).
// Each block covers kCompactPer consecutive entries, 16 per thread.
constexpr int kCompactThreads = 256;
constexpr int kCompactPer = kCompactThreads * 16;

__global__ void __launch_bounds__(kCompactThreads) compact_count_kernel(CompactArgs c,
                                                                        int64_t nb) {
    if (c.acc[c.gate] == 0) return;  // nothing flagged: the scan writes a zero count
    __shared__ int32_t part[kCompactThreads / 32];
    for (int64_t vb = blockIdx.x; vb < nb; vb += gridDim.x) {
        int n = 0;
        const int64_t e0 = vb * kCompactPer + threadIdx.x * 16;
        for (int k = 0; k < 16; ++k) n += e0 + k < c.dm && c.rc_idx[e0 + k] == -2;
        for (int o = 16; o; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
        if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = n;
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
            for (int w = 0; w < kCompactThreads / 32; ++w) t += part[w];
            c.block_n[vb] = t;
        }
        __syncthreads();
    }
}

// Exclusive scan of the block counts (one block); the total is the list size.
__global__ void __launch_bounds__(1024) compact_scan_kernel(CompactArgs c, int32_t nb) {
    __shared__ int32_t sh[32];
    __shared__ int32_t carry;
    if (c.acc[c.gate] == 0) {
        if (threadIdx.x == 0) *c.rc_count = 0;
        return;
    }
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int32_t b0 = 0; b0 < nb; b0 += 1024) {
        const int32_t i = b0 + threadIdx.x;
        const int32_t v = i < nb ? c.block_n[i] : 0;
        int32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) sh[w] = x;
        __syncthreads();
        if (w == 0) {
            int32_t z = sh[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(0xffffffffu, z, o);
                if (lane >= o) z += y;
            }
            sh[lane] = z;
        }
        __syncthreads();
        const int32_t incl = x + (w ? sh[w - 1] : 0);
        if (i < nb) c.block_n[i] = carry + incl - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *c.rc_count = carry;
        if (carry > c.capacity) atomicOr(&c.acc[6], 1ull);
    }
}

__device__ __forceinline__ void compact_write_block(const CompactArgs &c, int64_t vb) {
    __shared__ int32_t part[kCompactThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t e0 = vb * kCompactPer + threadIdx.x * 16;
    int32_t v[16];
    int n = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        v[k] = e0 + k < c.dm ? c.rc_idx[e0 + k] : -1;
        n += v[k] == -2;
    }
    int x = n;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) part[w] = x;
    __syncthreads();
    int before = 0;
    for (int i = 0; i < w; ++i) before += part[i];
    __syncthreads();  // part is rewritten by the next virtual block
    int32_t slot = c.block_n[vb] + before + x - n;
    const TaskDev &t = c.t;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        if (v[k] != -2) continue;
        const int64_t e = e0 + k;
        if (slot < c.capacity) {
            // the group holding entry e: last g with group_dm[g] <= e
            int lo = 0, hi = t.n_groups - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (t.group_dm[mid] <= e) lo = mid; else hi = mid - 1;
            }
            const int4 gm = t.gmeta[lo];
            const int64_t local = e - t.group_dm[lo];
            const int r = (int)(local / gm.y), col = (int)(local - (int64_t)r * gm.y);
            c.rc_list[slot] = make_int2(gm.x + r, gm.x + col);
            c.rc_idx[e] = slot;
        }
        ++slot;
    }
}

__global__ void __launch_bounds__(kCompactThreads) compact_write_kernel(CompactArgs c,
                                                                        int64_t nb) {
    if (c.acc[c.gate] == 0) return;
    for (int64_t vb = blockIdx.x; vb < nb; vb += gridDim.x) compact_write_block(c, vb);
}

// Before a pass that scores again: clear the sums of the previous pass if
// acc[gate] says that it met deferred triples (the pass then runs).
__global__ void reset_if_dirty_kernel(unsigned long long *acc, int gate) {
    if (threadIdx.x < 6 && acc[gate] != 0) acc[threadIdx.x] = 0;
}

// One warp per group: mean of the existing entries of the group in index
// order (outer, then inner).
__global__ void final_group_kernel(const double *in, const int32_t *in_n, int64_t n_outer,
                                   int32_t n_group, int64_t inner, double *out, int64_t *out_n) {
    const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (g >= n_group) return;
    double s;
    int64_t c;
    auto at = [&](int64_t k) { return ((k / inner) * n_group + g) * inner + k % inner; };
    warp_ordered_sum(in, in_n, n_outer * inner, at, s, c);
    if ((threadIdx.x & 31) == 0) {
        out[g] = c ? div_exact_pow2(s, c) : 0.0;
        out_n[g] = c;
    }
}

// Per-block partial sums in shared memory (n_group <= kGroupSmem), one
// global atomic per group and block.
constexpr int kGroupSmem = 1024;

__global__ void cell_group_sums_kernel(ScoreArgs a, FastDiv by_seg_div, FastDiv by_group,
                                       int32_t n_group, unsigned long long *num2,
                                       unsigned long long *cnt) {
    __shared__ unsigned long long sn[kGroupSmem], sc[kGroupSmem];
    const bool local = n_group <= kGroupSmem;
    if (local)
        for (int i = threadIdx.x; i < n_group; i += blockDim.x) sn[i] = sc[i] = 0;
    __syncthreads();
    const int64_t total = min(*a.n_cells_dev, a.cell_cap);
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < total;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = a.cell_cnt[c];
        if (k == 0) continue;
        const uint32_t q = fast_div((uint32_t)a.cell_id[c].x, by_seg_div);
        const int g = (int)(q - fast_div(q, by_group) * (uint32_t)n_group);
        if (local) {
            atomicAdd(&sn[g], (unsigned long long)a.cell_num2[c]);
            atomicAdd(&sc[g], (unsigned long long)k);
        } else {
            atomicAdd(&num2[g], (unsigned long long)a.cell_num2[c]);
            atomicAdd(&cnt[g], (unsigned long long)k);
        }
    }
    __syncthreads();
    if (local)
        for (int i = threadIdx.x; i < n_group; i += blockDim.x)
            if (sc[i]) {
                atomicAdd(&num2[i], sn[i]);
                atomicAdd(&cnt[i], sc[i]);
            }
}

}  // namespace

cudaError_t launch_score(const ScoreArgs &a, cudaStream_t s) {
    if (a.n_seg == 0) return cudaSuccess;
    {
        ProfScope ps_("score", s);
        score_kernel<<<(unsigned)((a.n_seg + 127) / 128), 128, 0, s>>>(a);
    }
    return cudaGetLastError();
}

static unsigned grid_of(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t launch_seg_count(const ScoreArgs &a, cudaStream_t s) {
    if (a.n_seg == 0) return cudaSuccess;
    ProfScope ps_("score_count", s);
    seg_count_kernel<<<grid_of(a.n_seg, 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_cell_enum(const ScoreArgs &a, cudaStream_t s) {
    if (a.n_seg == 0) return cudaSuccess;
    ProfScope ps_("score_enum", s);
    cell_enum_kernel<<<grid_of(a.n_seg, 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_cell_eval(const ScoreArgs &a, cudaStream_t s) {
    if (a.cell_cap == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(a.big_count, 0, sizeof(int64_t), s);
    if (e != cudaSuccess) return e;
    {
        ProfScope ps_("score_cells", s);
        cell_eval_kernel<<<grid_of(a.cell_cap, 256), 256, 0, s>>>(a);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // big cells: one warp each, grid-stride over at most 148 x 16 blocks
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const unsigned blocks = (unsigned)std::min<int64_t>((a.cell_cap + 7) / 8, (int64_t)nsm * 16);
    const size_t smem = a.sub_cap > 0 ? (size_t)8 * 3 * a.sub_cap * sizeof(int32_t) : 0;
    {
        ProfScope ps_("score_cells_big", s);
        cell_eval_big_kernel<<<blocks, 256, smem, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_seg_reduce(const ScoreArgs &a, cudaStream_t s) {
    if (a.n_seg == 0) return cudaSuccess;
    ProfScope ps_("score_reduce", s);
    seg_reduce_kernel<<<grid_of(a.n_seg, 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_cell_emit(const ScoreArgs &a, cudaStream_t s) {
    if (a.cell_cap == 0) return cudaSuccess;
    ProfScope ps_("score_emit", s);
    cell_emit_kernel<<<grid_of(a.cell_cap, 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_collapse_level(const double *in, const int32_t *in_n, int64_t n_out,
                                  int64_t radix, double *out, int32_t *out_n, cudaStream_t s) {
    if (n_out == 0) return cudaSuccess;
    {
        ProfScope ps_("collapse_level", s);
        if (radix >= 32)
            collapse_warp_kernel<<<(unsigned)((n_out * 32 + 255) / 256), 256, 0, s>>>(
                in, in_n, n_out, radix, out, out_n);
        else
            collapse_kernel<<<(unsigned)((n_out + 255) / 256), 256, 0, s>>>(in, in_n, n_out,
                                                                           radix, out, out_n);
    }
    return cudaGetLastError();
}

cudaError_t launch_final_mean(const double *in, const int32_t *in_n, int64_t n, double *out,
                              int64_t *out_n, cudaStream_t s) {
    {
        ProfScope ps_("collapse_final", s);
        final_kernel<<<1, 32, 0, s>>>(in, in_n, n, out, out_n);
    }
    return cudaGetLastError();
}

cudaError_t launch_bits(const BitsArgs &b, cudaStream_t s) {
    const int64_t n = b.by_space * (int64_t)b.K_on * b.K_s;
    if (n == 0) return cudaSuccess;
    {
        ProfScope ps_("score_bits", s);
        bits_kernel<<<grid_of(n, 256), 256, 0, s>>>(b);
    }
    return cudaGetLastError();
}

cudaError_t launch_recheck_compact(const CompactArgs &c, cudaStream_t s) {
    const int64_t nb = (c.dm + kCompactPer - 1) / kCompactPer;
    if (nb == 0) return cudaSuccess;
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    // grid-stride over the entry blocks: a gated launch ends at once
    const unsigned grid = (unsigned)std::min<int64_t>(nb, (int64_t)nsm * 8);
    ProfScope ps_("recheck_compact", s);
    compact_count_kernel<<<grid, kCompactThreads, 0, s>>>(c, nb);
    compact_scan_kernel<<<1, 1024, 0, s>>>(c, (int32_t)nb);
    compact_write_kernel<<<grid, kCompactThreads, 0, s>>>(c, nb);
    return cudaGetLastError();
}

cudaError_t launch_reset_if_dirty(unsigned long long *acc, int gate, cudaStream_t s) {
    {
        ProfScope ps_("score_reset", s);
        reset_if_dirty_kernel<<<1, 32, 0, s>>>(acc, gate);
    }
    return cudaGetLastError();
}

cudaError_t launch_final_group(const double *in, const int32_t *in_n, int64_t n_outer,
                               int32_t n_group, int64_t inner, double *out, int64_t *out_n,
                               cudaStream_t s) {
    if (n_group <= 0) return cudaSuccess;
    {
        ProfScope ps_("collapse_final", s);
        final_group_kernel<<<(unsigned)(((int64_t)n_group * 32 + 255) / 256), 256, 0, s>>>(
            in, in_n, n_outer, n_group, inner, out, out_n);
    }
    return cudaGetLastError();
}

cudaError_t launch_cell_group_sums(const ScoreArgs &a, int64_t seg_div, int32_t n_group,
                                   unsigned long long *num2, unsigned long long *cnt,
                                   cudaStream_t s) {
    if (a.cell_cap == 0) return cudaSuccess;
    {
        ProfScope ps_("score_group_sums", s);
        int dev = 0, nsm = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        const unsigned blocks = (unsigned)std::min<int64_t>(grid_of(a.cell_cap, 256), nsm * 4);
        cell_group_sums_kernel<<<blocks, 256, 0, s>>>(a, make_fastdiv((uint32_t)seg_div),
                                                      make_fastdiv((uint32_t)n_group), n_group,
                                                      num2, cnt);
    }
    return cudaGetLastError();
}

cudaError_t launch_recheck(const RecheckArgs &a, int32_t capacity, cudaStream_t s) {
    if (capacity <= 0) return cudaSuccess;
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (a.mode == ABX_MEAN) {
        const size_t smem = (size_t)a.dim * 2 * 8;
        cudaError_t e = cudaFuncSetAttribute(recheck_mean_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        const int blocks = capacity < nsm * 4 ? capacity : nsm * 4;
        ProfScope ps_("recheck_fp64", s);
        recheck_mean_kernel<<<blocks, 256, smem, s>>>(a);
        return cudaGetLastError();
    }
    const size_t ml = a.max_len;
    const size_t smem = ml * ml * 8 + 2 * ml * 8 + ml * ml * 2;
    cudaError_t e = cudaFuncSetAttribute(recheck_dtw_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, recheck_dtw_kernel, kRecheckThreads,
                                                      smem);
    if (e != cudaSuccess) return e;
    const int64_t full = (int64_t)nsm * (per_sm > 0 ? per_sm : 1);
    const int blocks = (int)(capacity < full ? capacity : full);
    ProfScope ps_("recheck_fp64", s);
    recheck_dtw_kernel<<<blocks, kRecheckThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace abx
