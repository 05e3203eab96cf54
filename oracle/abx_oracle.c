/*
 * abx_oracle.c -- plain FP64 CPU oracle for the ABX distance path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and
 * bench.py's cpu_baseline / reference leg may load or call this code; the
 * product library never links, imports or executes it, and the two share no
 * source, header, table or helper.
 *
 * What it computes (fastabx, arXiv 2505.02692):
 *   - angular frame distance  d(u,v) = arccos(<u,v> / (|u| |v|)) / pi, the
 *     "angular" distance named for Score in Sec. 3.1; the clamp of the cosine
 *     to [-1, 1] only guards rounding.
 *   - DTW cost by the dynamic programme of Sec. 3.2:
 *        c(i,j) = d(i,j) + min(c(i-1,j), c(i,j-1), c(i-1,j-1)),
 *     with c(0,0) = d(0,0) and the first row / column as running sums (the
 *     recurrence is only stated for i,j >= 1, so row 0 and column 0 are the
 *     only paths that reach them).
 *   - normalisation by path length: the result is c(Tx-1,Ty-1) / L where L is
 *     the number of cells on the optimal path.  Among predecessors of equal
 *     cost the one with the shorter path is taken, i.e. the minimum is the
 *     lexicographic minimum of (cost, length).  The paper states neither the
 *     normalisation nor a tie rule; this is the reading used throughout.
 *   - mean-pooled mode (Sec. 3.2, "pool along the time domain"): the frame
 *     distance between the arithmetic means of the raw frames.
 *   - other frame distances (Sec. 3.1 names "angular", "euclidean", etc.):
 *     cosine distance 1 - cos and the Euclidean distance, the latter from
 *     coordinate differences.
 *
 * Every loop is the definition written out: full Tx x Ty table, no blocking,
 * no reordering.  FP64 throughout; inputs are the caller's FP32 features.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC abx_oracle.c -lm
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_MODE_DTW 0
#define ORACLE_MODE_MEAN 1

/* Frame distances (Sec. 3.1: Score takes "angular", "euclidean", etc.). */
#define ORACLE_DIST_ANGULAR 0   /* arccos(cos) / pi                     */
#define ORACLE_DIST_COSINE 1    /* 1 - cos                              */
#define ORACLE_DIST_EUCLIDEAN 2 /* sqrt(sum_k (u_k - v_k)^2)            */
#define ORACLE_DIST_KL 3        /* symmetrised KL of the frames as
                                   distributions (components > 0, each frame
                                   divided by its sum): (KL(p|q) + KL(q|p)) / 2
                                   = 1/2 sum_k (p_k - q_k)(ln p_k - ln q_k)  */

/* Distance between two FP64 vectors: angular (Sec. 3.1) or one of the
 * other named distances. */
static double dist_d(const double *u, const double *v, int64_t dim, int distance) {
    if (distance == ORACLE_DIST_KL) {
        double su = 0.0, sv = 0.0;
        for (int64_t k = 0; k < dim; ++k) {
            if (!(u[k] > 0.0) || !(v[k] > 0.0)) return NAN;
            su += u[k];
            sv += v[k];
        }
        double s = 0.0;
        for (int64_t k = 0; k < dim; ++k) {
            const double p = u[k] / su, q = v[k] / sv;
            s += (p - q) * (log(p) - log(q));
        }
        return 0.5 * s;
    }
    if (distance == ORACLE_DIST_EUCLIDEAN) {
        double s = 0.0;
        for (int64_t k = 0; k < dim; ++k) s += (u[k] - v[k]) * (u[k] - v[k]);
        return sqrt(s);
    }
    double uv = 0.0, uu = 0.0, vv = 0.0;
    for (int64_t k = 0; k < dim; ++k) {
        uv += u[k] * v[k];
        uu += u[k] * u[k];
        vv += v[k] * v[k];
    }
    double c = uv / (sqrt(uu) * sqrt(vv));
    if (c > 1.0) c = 1.0;
    if (c < -1.0) c = -1.0;
    return distance == ORACLE_DIST_COSINE ? 1.0 - c : acos(c) / M_PI;
}

/* Distance between two FP32 frames, evaluated in FP64. */
double abxo_distance(const float *u, const float *v, int64_t dim, int distance) {
    double *a = (double *)malloc(sizeof(double) * (size_t)dim);
    double *b = (double *)malloc(sizeof(double) * (size_t)dim);
    if (!a || !b) {
        free(a);
        free(b);
        return NAN;
    }
    for (int64_t k = 0; k < dim; ++k) {
        a[k] = (double)u[k];
        b[k] = (double)v[k];
    }
    double d = dist_d(a, b, dim, distance);
    free(a);
    free(b);
    return d;
}

/* Angular distance between two FP32 frames, evaluated in FP64. */
double abxo_angular(const float *u, const float *v, int64_t dim) {
    double uv = 0.0, uu = 0.0, vv = 0.0;
    for (int64_t k = 0; k < dim; ++k) {
        double a = (double)u[k], b = (double)v[k];
        uv += a * b;
        uu += a * a;
        vv += b * b;
    }
    double c = uv / (sqrt(uu) * sqrt(vv));
    if (c > 1.0) c = 1.0;
    if (c < -1.0) c = -1.0;
    return acos(c) / M_PI;
}

/* Frame-distance matrix out[i*ty + j] = d(X_i, Y_j); X rows, Y columns. */
void abxo_frame_dists(const float *X, int64_t tx, const float *Y, int64_t ty,
                      int64_t dim, double *out) {
    for (int64_t i = 0; i < tx; ++i)
        for (int64_t j = 0; j < ty; ++j)
            out[i * ty + j] = abxo_angular(X + i * dim, Y + j * dim, dim);
}

/* DTW over a given distance matrix d[i*ty + j] (Sec. 3.2 recurrence).
 * Writes the optimal cost and the length (cells) of the optimal path; among
 * equal-cost predecessors the shorter path wins.  Returns 0, or -1 on bad
 * sizes / allocation failure. */
int abxo_dtw(const double *d, int64_t tx, int64_t ty, double *cost_out,
             int64_t *len_out) {
    if (tx <= 0 || ty <= 0) return -1;
    double *c = (double *)malloc(sizeof(double) * (size_t)(tx * ty));
    int64_t *l = (int64_t *)malloc(sizeof(int64_t) * (size_t)(tx * ty));
    if (!c || !l) {
        free(c);
        free(l);
        return -1;
    }
    for (int64_t i = 0; i < tx; ++i) {
        for (int64_t j = 0; j < ty; ++j) {
            double best_c;
            int64_t best_l;
            if (i == 0 && j == 0) {
                best_c = 0.0;
                best_l = 0;
            } else {
                int have = 0;
                best_c = 0.0;
                best_l = 0;
                /* the three predecessors of Sec. 3.2, those that exist */
                int64_t pi[3] = {i - 1, i, i - 1};
                int64_t pj[3] = {j, j - 1, j - 1};
                for (int p = 0; p < 3; ++p) {
                    if (pi[p] < 0 || pj[p] < 0) continue;
                    double pc = c[pi[p] * ty + pj[p]];
                    int64_t pl = l[pi[p] * ty + pj[p]];
                    if (!have || pc < best_c || (pc == best_c && pl < best_l)) {
                        best_c = pc;
                        best_l = pl;
                        have = 1;
                    }
                }
            }
            c[i * ty + j] = d[i * ty + j] + best_c;
            l[i * ty + j] = best_l + 1;
        }
    }
    *cost_out = c[tx * ty - 1];
    *len_out = l[tx * ty - 1];
    free(c);
    free(l);
    return 0;
}

/* Item-pair distance for one ordered pair (x rows, y columns).
 * DTW mode: cost / length of the optimal path.  Mean mode: the frame
 * distance of the FP64 means of the raw frames (length reported as 1). */
static int pair_distance(const float *X, int64_t tx, const float *Y, int64_t ty,
                         int64_t dim, int mode, int distance, double *dist, double *cost,
                         int64_t *len) {
    if (mode == ORACLE_MODE_MEAN) {
        double *mx = (double *)calloc((size_t)dim, sizeof(double));
        double *my = (double *)calloc((size_t)dim, sizeof(double));
        if (!mx || !my) {
            free(mx);
            free(my);
            return -1;
        }
        for (int64_t t = 0; t < tx; ++t)
            for (int64_t k = 0; k < dim; ++k) mx[k] += (double)X[t * dim + k];
        for (int64_t t = 0; t < ty; ++t)
            for (int64_t k = 0; k < dim; ++k) my[k] += (double)Y[t * dim + k];
        for (int64_t k = 0; k < dim; ++k) {
            mx[k] /= (double)tx;
            my[k] /= (double)ty;
        }
        double dd = dist_d(mx, my, dim, distance);
        free(mx);
        free(my);
        *dist = dd;
        *cost = dd;
        *len = 1;
        return 0;
    }
    double *d = (double *)malloc(sizeof(double) * (size_t)(tx * ty));
    if (!d) return -1;
    if (distance == ORACLE_DIST_ANGULAR)
        abxo_frame_dists(X, tx, Y, ty, dim, d);
    else
        for (int64_t i = 0; i < tx; ++i)
            for (int64_t j = 0; j < ty; ++j)
                d[i * ty + j] = abxo_distance(X + i * dim, Y + j * dim, dim, distance);
    int rc = abxo_dtw(d, tx, ty, cost, len);
    free(d);
    if (rc) return rc;
    *dist = *cost / (double)(*len);
    return 0;
}

/* Batch of ordered item pairs (px[k], py[k]) over CSR items
 * feats[offsets[i] .. offsets[i+1]) x dim.  OpenMP over pairs; each pair is
 * independent.  Returns 0 or -1 if any pair failed. */
int abxo_pair_distances(const float *feats, const int64_t *offsets, int64_t dim,
                        int64_t npairs, const int64_t *px, const int64_t *py,
                        int mode, int distance, double *dist, double *cost, int64_t *len,
                        int nthreads) {
    int failed = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 16) reduction(| : failed)
    for (int64_t k = 0; k < npairs; ++k) {
        int64_t x = px[k], y = py[k];
        const float *X = feats + offsets[x] * dim;
        const float *Y = feats + offsets[y] * dim;
        int64_t tx = offsets[x + 1] - offsets[x];
        int64_t ty = offsets[y + 1] - offsets[y];
        if (pair_distance(X, tx, Y, ty, dim, mode, distance, &dist[k], &cost[k], &len[k]))
            failed = 1;
    }
    return failed ? -1 : 0;
}

/* Threads the OpenMP runtime would use for a parallel region. */
int abxo_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
