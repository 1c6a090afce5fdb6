/*
 * CPU oracle for the MG-sketch local-moving sweep (arXiv 2411.02268).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, single-threaded
 * restatement of what the method computes.  It shares no code with the CUDA
 * path; only the tests, the smoke check and the benchmark's CPU-baseline leg
 * may load it.
 *
 * All arithmetic is exact integer arithmetic: weights are uint32, weighted
 * degrees and community totals uint64, modularity gains signed 128-bit.
 *
 * Notation follows Section 3 of the paper:
 *   K_i        weighted degree, sum of w over row i (self-loop entry included)
 *   K_{i->c}   sum of w over entries (i, j) of row i with j != i and C_j = c
 *   Sigma_c    sum of K_i over members of c
 *   sigma_c    sum of w over entries (i, j) with C_i = C_j = c
 *   2m         sum of K_i over all vertices
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;
typedef unsigned __int128 u128;

#define EMPTY_KEY 0xFFFFFFFFu

enum { MODE_LOUVAIN = 0, MODE_LPA = 1, MODE_REFINE = 2 };

/* ---------------------------------------------------------------------------
 * Weighted degree and community totals (Section 3).
 * ------------------------------------------------------------------------- */
void or_degrees(int64_t n, const int64_t* off, const uint32_t* w, uint64_t* K) {
    for (int64_t i = 0; i < n; ++i) {
        uint64_t s = 0;
        for (int64_t e = off[i]; e < off[i + 1]; ++e) s += w[e];
        K[i] = s;
    }
}

void or_community_totals(int64_t n, const uint32_t* labels, const uint64_t* K,
                         uint64_t* Sigma, uint32_t* size) {
    memset(Sigma, 0, sizeof(uint64_t) * (size_t)n);
    memset(size, 0, sizeof(uint32_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        Sigma[labels[i]] += K[i];
        size[labels[i]] += 1;
    }
}

/* ---------------------------------------------------------------------------
 * Modularity, Eq. 1:  Q = sum_c [ sigma_c/2m - (Sigma_c/2m)^2 ]
 *                       = (2m * sum_c sigma_c - sum_c Sigma_c^2) / (2m)^2.
 * Returns the integer parts: sum_c sigma_c, sum_c Sigma_c^2 (as two 64-bit
 * halves) and 2m.  Labels must be < n.
 * ------------------------------------------------------------------------- */
void or_modularity_parts(int64_t n, const int64_t* off, const int32_t* cols, const uint32_t* w,
                         const uint32_t* labels, uint64_t* sigma_in, uint64_t* sq_lo,
                         uint64_t* sq_hi, uint64_t* two_m) {
    uint64_t* Sig = (uint64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(uint64_t));
    uint64_t sin_ = 0, tm = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t e = off[i]; e < off[i + 1]; ++e) {
            tm += w[e];
            Sig[labels[i]] += w[e];
            if (labels[cols[e]] == labels[i]) sin_ += w[e];
        }
    }
    u128 sq = 0;
    for (int64_t c = 0; c < n; ++c) sq += (u128)Sig[c] * (u128)Sig[c];
    free(Sig);
    *sigma_in = sin_;
    *sq_lo = (uint64_t)sq;
    *sq_hi = (uint64_t)(sq >> 64);
    *two_m = tm;
}

/* ---------------------------------------------------------------------------
 * Weighted Misra-Gries sketch, Algorithm 1 (Appendix A.1), stated as a rule.
 *
 * A sketch is k slots (keys[p], vals[p]); a slot whose value is 0 is free,
 * and a free slot keeps whatever key it last held.  The initial state is
 * keys = EMPTY_KEY, vals = 0.  Feeding (c, w):
 *   - if some slot holds the key c, that slot gains w (a freed slot that
 *     still holds c comes back to life);
 *   - otherwise the paper's conditional rule takes the free slot with the
 *     largest index for (c, w), and when there is none it lowers every value
 *     by w (never below 0) and forgets c.
 * uncond = 1 (Section 4.1, unconditional subtraction): a c that no slot holds
 * first lowers every value by w (never below 0), then takes the free slot
 * with the largest index if one exists.  uncond = 2 selects the weighted
 * Misra-Gries summary of the literature instead (below).
 * Keys are never duplicated: c is placed only when no slot holds it.
 * ------------------------------------------------------------------------- */
static int slot_holding(const uint32_t* keys, int k, uint32_t c) {
    for (int p = 0; p < k; ++p)
        if (keys[p] == c) return p;
    return -1;
}

static int largest_free_slot(const uint64_t* vals, int k) {
    for (int p = k - 1; p >= 0; --p)
        if (vals[p] == 0) return p;
    return -1;
}

static void lower_all(uint64_t* vals, int k, uint64_t by) {
    for (int p = 0; p < k; ++p) vals[p] = vals[p] > by ? vals[p] - by : 0;
}

static uint64_t smallest_value(const uint64_t* vals, int k) {
    uint64_t m = vals[0];
    for (int p = 1; p < k; ++p)
        if (vals[p] < m) m = vals[p];
    return m;
}

void or_sketch_update(uint32_t* keys, uint64_t* vals, int k, uint32_t c, uint64_t w, int uncond) {
    const int held = slot_holding(keys, k, c);
    if (held >= 0) {
        vals[held] += w;
        return;
    }
    int f;
    switch (uncond) {
        case 0: /* Algorithm 1 */
            f = largest_free_slot(vals, k);
            if (f < 0) {
                lower_all(vals, k, w);
                return;
            }
            break;
        case 1: /* unconditional subtraction */
            lower_all(vals, k, w);
            f = largest_free_slot(vals, k);
            if (f < 0) return;
            break;
        default: {
            /* the weighted Misra-Gries summary of the literature (not the
             * paper's rule): with no free slot every value drops by
             * d = min(w, smallest value) and whatever is left of w, if
             * anything, is placed in the largest-index slot that freed up */
            f = largest_free_slot(vals, k);
            if (f < 0) {
                const uint64_t m = smallest_value(vals, k);
                const uint64_t d = w < m ? w : m;
                lower_all(vals, k, d);
                if (w == d) return;
                w -= d;
                f = largest_free_slot(vals, k);
            }
            break;
        }
    }
    keys[f] = c;
    vals[f] = w;
}

/* merge(A, B): every live slot of B, in slot order, is fed to A as one
 * update.  (The paper streams one vertex per thread and needs no merge; the
 * merge defines how partial sketches of one row are combined.) */
void or_sketch_merge(uint32_t* akeys, uint64_t* avals, const uint32_t* bkeys, const uint64_t* bvals,
                     int k, int uncond) {
    for (int p = 0; p < k; ++p)
        if (bvals[p] > 0) or_sketch_update(akeys, avals, k, bkeys[p], bvals[p], uncond);
}

/* ---------------------------------------------------------------------------
 * Stream partition of a row.  A schedule maps the row length to a number of
 * streams L (a power of two); entry e (global CSR index) of the row belongs
 * to stream (e / V) mod L and each stream takes its entries in increasing e.
 * The L partial sketches are combined by a tree: for o = L/2, L/4, ..., 1,
 * S[s] = merge(S[s], S[s + o]) for every s < o; the result is S[0].
 * ------------------------------------------------------------------------- */
typedef struct {
    int nbuckets;
    const int64_t* deg_max; /* ascending; bucket b takes rows with length <= deg_max[b] */
    const int32_t* lanes;   /* streams per row in bucket b */
    int vec;                /* V */
} or_sched;

static int64_t streams_for(const or_sched* s, int64_t deg) {
    for (int b = 0; b < s->nbuckets; ++b)
        if (deg <= s->deg_max[b]) return s->lanes[b];
    return s->lanes[s->nbuckets - 1];
}

/* Build the sketch of row i (self-loops skipped; in the refine mode only
 * entries with bound[j] == bound[i] are taken, Algorithm 1 lines 2-3). */
static void row_sketch(int64_t i, const int64_t* off, const int32_t* cols, const uint32_t* w,
                       const uint32_t* labels, const uint32_t* bound, int k, int uncond,
                       const or_sched* sched, uint32_t* keys_out, uint64_t* vals_out) {
    int64_t deg = off[i + 1] - off[i];
    int64_t L = streams_for(sched, deg);
    int64_t V = sched->vec;
    uint32_t* SK = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(L * k));
    uint64_t* SV = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(L * k));
    for (int64_t x = 0; x < L * k; ++x) { SK[x] = EMPTY_KEY; SV[x] = 0; }
    for (int64_t e = off[i]; e < off[i + 1]; ++e) {
        int64_t j = cols[e];
        if (j == i) continue;
        if (bound && bound[j] != bound[i]) continue;
        int64_t s = (e / V) % L;
        or_sketch_update(SK + s * k, SV + s * k, k, labels[j], w[e], uncond);
    }
    for (int64_t o = L / 2; o >= 1; o /= 2)
        for (int64_t s = 0; s < o; ++s)
            or_sketch_merge(SK + s * k, SV + s * k, SK + (s + o) * k, SV + (s + o) * k, k, uncond);
    memcpy(keys_out, SK, sizeof(uint32_t) * (size_t)k);
    memcpy(vals_out, SV, sizeof(uint64_t) * (size_t)k);
    free(SK);
    free(SV);
}

/* Exact K_{i->c} by a second scan of row i (self-loops excluded). */
static uint64_t link_weight(int64_t i, uint32_t c, const int64_t* off, const int32_t* cols,
                            const uint32_t* w, const uint32_t* labels, const uint32_t* bound) {
    uint64_t s = 0;
    for (int64_t e = off[i]; e < off[i + 1]; ++e) {
        int64_t j = cols[e];
        if (j == i) continue;
        if (bound && bound[j] != bound[i]) continue;
        if (labels[j] == c) s += w[e];
    }
    return s;
}

/* Colour class of vertex v among `colors` classes: the 32-bit integer hash
 * "lowbias32" (C. Wellons) of v, modulo the number of classes. */
static uint32_t color_of(uint32_t v, int colors) {
    if (colors <= 1) return 0u;
    uint32_t x = v;
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x % (uint32_t)colors;
}

/* Scaled delta-modularity, Eq. 2 multiplied by 2m^2:
 *   gain = 2m (K_{i->c} - K_{i->d}) - K_i (K_i + Sigma_c - Sigma_d). */
static i128 dq_gain(uint64_t two_m, uint64_t Kic, uint64_t Kid, uint64_t Ki, uint64_t Sc, uint64_t Sd) {
    return (i128)two_m * ((i128)Kic - (i128)Kid) - (i128)Ki * ((i128)Ki + (i128)Sc - (i128)Sd);
}

/* ---------------------------------------------------------------------------
 * One synchronous sweep (every decision reads the sweep-start state).
 *
 * k > 0: candidates are the live keys of the row's MG sketch (value > 0),
 *        exact K_{i->c} from a second scan (Section 4.1, Fig. 2).
 * k = 0: exact: candidates are all distinct neighbour communities.
 * The current community d is never a candidate; K_{i->d} is always exact.
 *
 * Louvain (and refine): gain as above; a singleton vertex may not join another
 * singleton community with a larger id whose id has colour `sub_color` among
 * `colors` (that is, whose vertex decides in the same sub-sweep: this stops
 * pairwise swaps of simultaneous moves; colors = 1, a fully synchronous
 * sweep, bars every such target); best gain wins, ties to the smaller id;
 * moves iff gain > 0.
 * LPA: largest K_{i->c} wins, ties to the smaller id; moves iff it exceeds
 * K_{i->d}.
 * Refine (Leiden, Section 3.4): both scans are restricted to neighbours with
 * bound[j] == bound[i]; only vertices whose community is a singleton move;
 * the singleton rule above is replaced by: a singleton community whose
 * vertex has colour `sub_color` (the colour class deciding in this
 * sub-sweep, among `colors`) is not a candidate, so that no vertex joins a
 * community whose only member may leave in the same sub-sweep.
 *
 * Vertices in [v0, v1) with active[i] != 0 (or all, active == NULL) are
 * decided; the others copy their label.  gains_out (optional) receives the
 * chosen gain for movers and 0 otherwise, as two 64-bit halves.
 * ------------------------------------------------------------------------- */
void or_sweep(int64_t n, const int64_t* off, const int32_t* cols, const uint32_t* w,
              const uint32_t* labels, const uint64_t* K, const uint64_t* Sigma, const uint32_t* size,
              uint64_t two_m, const uint32_t* bound, const uint8_t* active, int mode, int k, int uncond,
              int nbuckets, const int64_t* deg_max, const int32_t* lanes, int vec,
              int64_t v0, int64_t v1, uint32_t* labels_out, uint64_t* gain_lo, uint64_t* gain_hi,
              int colors, int sub_color, int one_scan) {
    or_sched sched = {nbuckets, deg_max, lanes, vec};
    (void)n;
    int kk = k > 0 ? k : 1;
    uint32_t* keys = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)kk);
    uint64_t* vals = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)kk);
    const uint32_t* bnd = (mode == MODE_REFINE) ? bound : NULL;
    for (int64_t i = v0; i < v1; ++i) {
        uint32_t d = labels[i];
        labels_out[i] = d;
        if (gain_lo) { gain_lo[i] = 0; gain_hi[i] = 0; }
        if (active && !active[i]) continue;
        if (mode == MODE_REFINE && size[d] != 1) continue;
        /* candidate list */
        int64_t deg = off[i + 1] - off[i];
        uint32_t* cand;
        int64_t ncand = 0;
        if (k > 0) {
            row_sketch(i, off, cols, w, labels, bnd, k, uncond, &sched, keys, vals);
            cand = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)k);
            for (int p = 0; p < k; ++p)
                if (vals[p] > 0 && keys[p] != d) cand[ncand++] = keys[p];
        } else {
            cand = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(deg > 0 ? deg : 1));
            for (int64_t e = off[i]; e < off[i + 1]; ++e) {
                int64_t j = cols[e];
                if (j == i) continue;
                if (bnd && bnd[j] != bnd[i]) continue;
                uint32_t c = labels[j];
                if (c == d) continue;
                int seen = 0;
                for (int64_t q = 0; q < ncand; ++q)
                    if (cand[q] == c) { seen = 1; break; }
                if (!seen) cand[ncand++] = c;
            }
        }
        /* LPA 1-scan variant (Section 4.3): the sketch values stand in for the
         * linking weights and no second scan is made */
        const int sketch_weights = one_scan && k > 0 && mode == MODE_LPA;
        uint64_t Kid = 0;
        if (sketch_weights) {
            for (int p = 0; p < k; ++p)
                if (keys[p] == d) Kid = vals[p];
        } else {
            Kid = link_weight(i, d, off, cols, w, labels, bnd);
        }
        uint32_t best = d;
        i128 best_gain = 0;
        uint64_t best_k = Kid;
        int have = 0;
        for (int64_t q = 0; q < ncand; ++q) {
            uint32_t c = cand[q];
            uint64_t Kic = 0;
            if (sketch_weights) {
                for (int p = 0; p < k; ++p)
                    if (keys[p] == c) Kic = vals[p];
            } else {
                Kic = link_weight(i, c, off, cols, w, labels, bnd);
            }
            if (mode == MODE_LPA) {
                if (Kic > Kid && (Kic > best_k || (Kic == best_k && c < best))) {
                    best = c; best_k = Kic; have = 1;
                }
            } else {
                if (mode == MODE_LOUVAIN && size[d] == 1 && size[c] == 1 && c > d &&
                    (int)color_of(c, colors) == sub_color)
                    continue;
                if (mode == MODE_REFINE && size[c] == 1 && (int)color_of(c, colors) == sub_color) continue;
                i128 g = dq_gain(two_m, Kic, Kid, K[i], Sigma[c], Sigma[d]);
                if (g > 0 && (g > best_gain || (g == best_gain && c < best))) {
                    best = c; best_gain = g; have = 1;
                }
            }
        }
        free(cand);
        if (have) {
            labels_out[i] = best;
            if (gain_lo) {
                u128 g = (mode == MODE_LPA) ? (u128)(best_k - Kid) : (u128)best_gain;
                gain_lo[i] = (uint64_t)g;
                gain_hi[i] = (uint64_t)(g >> 64);
            }
        }
    }
    free(keys);
    free(vals);
}

/* The MG sketch of one row on its own (for tests of the stream partition). */
void or_row_sketch(int64_t i, const int64_t* off, const int32_t* cols, const uint32_t* w,
                   const uint32_t* labels, const uint32_t* bound, int k, int uncond, int nbuckets,
                   const int64_t* deg_max, const int32_t* lanes, int vec, uint32_t* keys,
                   uint64_t* vals) {
    or_sched sched = {nbuckets, deg_max, lanes, vec};
    row_sketch(i, off, cols, w, labels, bound, k, uncond, &sched, keys, vals);
}

/* Linking weights of row i to every neighbouring community (self-loops
 * excluded): the row's (C_j, w_ij) pairs sorted by community and summed per
 * community.  Writes the distinct communities other than d to cand[] with
 * their weights in wsum[] (ascending id), returns their number, and stores
 * K_{i->d} in *kid.  The same sums as link_weight() for each community, in
 * O(deg log deg) instead of O(deg^2): used by the sequential exact sweep on
 * rows with hundreds of thousands of entries. */
typedef struct { uint32_t c; uint32_t w; } or_pair;

static int cmp_pair(const void* a, const void* b) {
    const uint32_t x = ((const or_pair*)a)->c, y = ((const or_pair*)b)->c;
    return x < y ? -1 : (x > y ? 1 : 0);
}

static int64_t row_community_weights(int64_t i, uint32_t d, const int64_t* off, const int32_t* cols,
                                     const uint32_t* w, const uint32_t* labels, uint32_t* cand,
                                     uint64_t* wsum, uint64_t* kid) {
    int64_t deg = off[i + 1] - off[i];
    or_pair* pr = (or_pair*)malloc(sizeof(or_pair) * (size_t)(deg > 0 ? deg : 1));
    int64_t np = 0;
    for (int64_t e = off[i]; e < off[i + 1]; ++e) {
        if (cols[e] == i) continue;
        pr[np].c = labels[cols[e]];
        pr[np].w = w[e];
        ++np;
    }
    qsort(pr, (size_t)np, sizeof(or_pair), cmp_pair);
    int64_t ncand = 0;
    *kid = 0;
    for (int64_t a = 0; a < np;) {
        uint64_t s = 0;
        int64_t b = a;
        while (b < np && pr[b].c == pr[a].c) s += pr[b++].w;
        if (pr[a].c == d) {
            *kid = s;
        } else {
            cand[ncand] = pr[a].c;
            wsum[ncand] = s;
            ++ncand;
        }
        a = b;
    }
    free(pr);
    return ncand;
}

/* ---------------------------------------------------------------------------
 * Sequential (Gauss-Seidel) local-moving phase, one vertex at a time in id
 * order, each move updating Sigma at once (the paper's per-thread loop with
 * a single thread).  Sketches are one stream per row in CSR order.
 * Louvain: repeats sweeps until the sweep's summed delta-modularity is at
 * most tol (compared as gain_sum <= tol * 2m^2), or max_sweeps.
 * LPA: repeats until at most tol * n vertices changed label, or max_sweeps.
 * labels is updated in place; returns the number of sweeps.
 * ------------------------------------------------------------------------- */
int or_local_move_seq(int64_t n, const int64_t* off, const int32_t* cols, const uint32_t* w,
                      uint32_t* labels, int mode, int k, int uncond, double tol, int max_sweeps) {
    uint64_t* K = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
    uint64_t* Sig = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
    uint32_t* size = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    or_degrees(n, off, w, K);
    or_community_totals(n, labels, K, Sig, size);
    uint64_t two_m = 0;
    for (int64_t i = 0; i < n; ++i) two_m += K[i];
    int kk = k > 0 ? k : 1;
    uint32_t* keys = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)kk);
    uint64_t* vals = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)kk);
    int64_t one_stream_deg = INT64_MAX;
    int32_t one_lane = 1;
    or_sched sched = {1, &one_stream_deg, &one_lane, 1};
    int sweeps = 0;
    for (; sweeps < max_sweeps;) {
        ++sweeps;
        u128 gain_sum = 0;
        int64_t moved = 0;
        for (int64_t i = 0; i < n; ++i) {
            uint32_t d = labels[i];
            int64_t deg = off[i + 1] - off[i];
            uint32_t* cand = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(deg > kk ? deg : kk));
            uint64_t* wsum = NULL;
            uint64_t Kid = 0;
            int64_t ncand = 0;
            if (k == 0) {
                /* exact: every neighbouring community, weights by sorting */
                wsum = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(deg > 0 ? deg : 1));
                ncand = row_community_weights(i, d, off, cols, w, labels, cand, wsum, &Kid);
            } else if (k > 0) {
                row_sketch(i, off, cols, w, labels, NULL, k, uncond, &sched, keys, vals);
                for (int p = 0; p < k; ++p)
                    if (vals[p] > 0 && keys[p] != d) cand[ncand++] = keys[p];
            }
            if (k > 0) Kid = link_weight(i, d, off, cols, w, labels, NULL);
            uint32_t best = d;
            i128 best_gain = 0;
            uint64_t best_k = Kid;
            int have = 0;
            for (int64_t q = 0; q < ncand; ++q) {
                uint32_t c = cand[q];
                uint64_t Kic = k == 0 ? wsum[q] : link_weight(i, c, off, cols, w, labels, NULL);
                if (mode == MODE_LPA) {
                    if (Kic > Kid && (Kic > best_k || (Kic == best_k && c < best))) {
                        best = c; best_k = Kic; have = 1;
                    }
                } else {
                    i128 g = dq_gain(two_m, Kic, Kid, K[i], Sig[c], Sig[d]);
                    if (g > 0 && (g > best_gain || (g == best_gain && c < best))) {
                        best = c; best_gain = g; have = 1;
                    }
                }
            }
            free(cand);
            free(wsum);
            if (have) {
                Sig[d] -= K[i]; size[d] -= 1;
                Sig[best] += K[i]; size[best] += 1;
                labels[i] = best;
                moved += 1;
                gain_sum += (u128)best_gain;
            }
        }
        if (mode == MODE_LPA) {
            if ((double)moved <= tol * (double)n) break;
        } else {
            double dq = (double)gain_sum / ((double)two_m * (double)two_m / 2.0);
            if (dq <= tol) break;
        }
    }
    free(K); free(Sig); free(size); free(keys); free(vals);
    return sweeps;
}

/* ---------------------------------------------------------------------------
 * MG aggregation (Section 4.1, "aggregation phase", Fig. 3): the super-vertex
 * of community c keeps the k-majority neighbouring communities of c found by
 * one MG sketch over the edges of all members of c, with the sketch values
 * as (approximate) weights and no second pass.  Members are taken in
 * ascending vertex id, the edges of each in CSR order; self-loops are kept
 * (the "exclude self" rule is for the local-moving and refinement phases).
 * The stream partition follows the schedule by the community's total entry
 * count: entry e (global CSR index) goes to stream (e / V) mod L, streams
 * merged by the same tree as the sweep.
 * members: vertex ids grouped by community (ascending within a community),
 * member_off[nc+1].  keys_out, vals_out: nc * k.
 * ------------------------------------------------------------------------- */
void or_aggregate_mg_sketch(int64_t n, const int64_t* off, const int32_t* cols, const uint32_t* w,
                            const uint32_t* dense, int64_t nc, const int64_t* member_off,
                            const uint32_t* members, int k, int uncond, int nbuckets,
                            const int64_t* deg_max, const int32_t* lanes, int vec,
                            uint32_t* keys_out, uint64_t* vals_out) {
    or_sched sched = {nbuckets, deg_max, lanes, vec};
    (void)n;
    for (int64_t c = 0; c < nc; ++c) {
        int64_t total = 0;
        for (int64_t q = member_off[c]; q < member_off[c + 1]; ++q) {
            uint32_t i = members[q];
            total += off[i + 1] - off[i];
        }
        int64_t L = streams_for(&sched, total);
        int64_t V = sched.vec;
        uint32_t* SK = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(L * k));
        uint64_t* SV = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(L * k));
        for (int64_t x = 0; x < L * k; ++x) { SK[x] = EMPTY_KEY; SV[x] = 0; }
        for (int64_t q = member_off[c]; q < member_off[c + 1]; ++q) {
            uint32_t i = members[q];
            for (int64_t e = off[i]; e < off[i + 1]; ++e) {
                int64_t s = (e / V) % L;
                or_sketch_update(SK + s * k, SV + s * k, k, dense[cols[e]], w[e], uncond);
            }
        }
        for (int64_t o = L / 2; o >= 1; o /= 2)
            for (int64_t s = 0; s < o; ++s)
                or_sketch_merge(SK + s * k, SV + s * k, SK + (s + o) * k, SV + (s + o) * k, k, uncond);
        memcpy(keys_out + c * k, SK, sizeof(uint32_t) * (size_t)k);
        memcpy(vals_out + c * k, SV, sizeof(uint64_t) * (size_t)k);
        free(SK);
        free(SV);
    }
}
