/*
 * Seeded synthetic graph generators and CSR builder.
 *
 * This file is the input side shared by the CUDA path and the CPU oracle.
 * It holds none of the community-detection arithmetic: it only draws
 * edges, symmetrises them, removes self-loops and duplicates, sorts each
 * row by column and attaches integer weights.
 *
 * Every random number is counter-based (splitmix64 applied to a tuple of
 * seed, stream and index), so the output depends only on the arguments and
 * never on the thread count or the machine.  The only floating-point step is
 * the geometric skip of the SBM generator; it uses a logarithm written here
 * from basic IEEE operations (no libm), built with -ffp-contract=off, so the
 * same graph comes out on x86-64 and aarch64.
 *
 * The graphs are undirected (Section 3: w_ij = w_ji, reverse edges inserted;
 * Section 5.1.3 makes every input undirected the same way).  Weights are
 * unsigned integers: w = 1 + H(seed, min(u,v), max(u,v)) mod wmax, a function
 * of the unordered pair, so both directions carry the same weight.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct gg_csr {
    int64_t n;
    int64_t nnz;
    int64_t* offsets; /* n+1 */
    int32_t* cols;    /* nnz */
    uint32_t* w;      /* nnz */
} gg_csr;

enum { GG_OK = 0, GG_EINVAL = -1, GG_ENOMEM = -2 };

/* ---- counter-based RNG ------------------------------------------------- */

static inline uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* rng(seed, stream, a, b): splitmix64 chained over the tuple. */
static inline uint64_t rng4(uint64_t seed, uint64_t stream, uint64_t a, uint64_t b) {
    return mix64(mix64(mix64(mix64(seed) + stream) + a) + b);
}

uint64_t gg_rng(uint64_t seed, uint64_t stream, uint64_t a, uint64_t b) {
    return rng4(seed, stream, a, b);
}

enum {
    S_RMAT = 1, S_WEIGHT = 2, S_SBM_IN = 3, S_SBM_OUT = 4,
    S_GRID = 5, S_PERM = 6, S_GRID_END = 7, S_GRID_V = 8
};

/* uniform double in (0, 1] from 53 random bits */
static inline double u01(uint64_t r) { return ((double)(r >> 11) + 1.0) * (1.0 / 9007199254740992.0); }

/* Natural logarithm of x in (0, 1], from frexp-free exponent extraction and
 * the atanh series log(m) = 2 * sum t^(2n+1)/(2n+1), t = (m-1)/(m+1).
 * Only +, -, *, / are used, so the result is the same on every IEEE machine
 * when contraction into fma is disabled. */
static double det_log(double x) {
    int e = 0;
    while (x < 0.5) { x *= 2.0; e -= 1; }
    /* x in [0.5, 1] */
    double t = (x - 1.0) / (x + 1.0);
    double t2 = t * t, term = t, sum = 0.0;
    for (int k = 1; k < 80; k += 2) {
        sum += term / (double)k;
        term *= t2;
    }
    return 2.0 * sum + (double)e * 0.69314718055994530942;
}

static inline uint32_t edge_weight(uint64_t seed, uint32_t wmax, int64_t u, int64_t v) {
    if (wmax <= 1) return 1u;
    uint64_t lo = (uint64_t)(u < v ? u : v), hi = (uint64_t)(u < v ? v : u);
    return 1u + (uint32_t)(rng4(seed, S_WEIGHT, lo, hi) % (uint64_t)wmax);
}

/* ---- CSR assembly -------------------------------------------------------- */

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/* Given counts -> offsets and scattered (unsorted, possibly duplicated)
 * columns, sort every row, drop duplicates, compact in place. */
static int finish_csr(gg_csr* g) {
    int64_t n = g->n;
    int64_t* newdeg = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!newdeg) return GG_ENOMEM;
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < n; ++i) {
        int32_t* row = g->cols + g->offsets[i];
        int64_t d = g->offsets[i + 1] - g->offsets[i];
        if (d > 1) qsort(row, (size_t)d, sizeof(int32_t), cmp_i32);
        int64_t u = 0;
        for (int64_t e = 0; e < d; ++e)
            if (u == 0 || row[u - 1] != row[e]) row[u++] = row[e];
        newdeg[i] = u;
    }
    /* compact left, row by row (new start <= old start, so forward copy is safe) */
    int64_t pos = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t s = g->offsets[i], d = newdeg[i];
        if (pos != s) memmove(g->cols + pos, g->cols + s, sizeof(int32_t) * (size_t)d);
        g->offsets[i] = pos;
        pos += d;
    }
    g->offsets[n] = pos;
    g->nnz = pos;
    free(newdeg);
    int32_t* c2 = (int32_t*)realloc(g->cols, sizeof(int32_t) * (size_t)(pos > 0 ? pos : 1));
    if (c2) g->cols = c2;
    g->w = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(pos > 0 ? pos : 1));
    if (!g->w) return GG_ENOMEM;
    return GG_OK;
}

static void fill_weights(gg_csr* g, uint64_t seed, uint32_t wmax) {
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < g->n; ++i)
        for (int64_t e = g->offsets[i]; e < g->offsets[i + 1]; ++e)
            g->w[e] = edge_weight(seed, wmax, i, g->cols[e]);
}

void gg_free(gg_csr* g) {
    if (!g) return;
    free(g->offsets); free(g->cols); free(g->w);
    g->offsets = NULL; g->cols = NULL; g->w = NULL;
}

/* Generic two-phase builder: an edge source is called once to count and once
 * to scatter.  It emits undirected pairs (u, v), u != v; both directions are
 * stored. */
typedef void (*emit_fn)(void* ctx, int64_t u, int64_t v);
typedef void (*source_fn)(void* src_ctx, int64_t chunk, emit_fn emit, void* emit_ctx);

typedef struct { int64_t* cnt; } count_ctx;
static void emit_count(void* c, int64_t u, int64_t v) {
    count_ctx* cc = (count_ctx*)c;
    __atomic_fetch_add(&cc->cnt[u], 1, __ATOMIC_RELAXED);
    __atomic_fetch_add(&cc->cnt[v], 1, __ATOMIC_RELAXED);
}
typedef struct { int64_t* cur; int32_t* cols; } scat_ctx;
static void emit_scatter(void* c, int64_t u, int64_t v) {
    scat_ctx* sc = (scat_ctx*)c;
    int64_t pu = __atomic_fetch_add(&sc->cur[u], 1, __ATOMIC_RELAXED);
    int64_t pv = __atomic_fetch_add(&sc->cur[v], 1, __ATOMIC_RELAXED);
    sc->cols[pu] = (int32_t)v;
    sc->cols[pv] = (int32_t)u;
}

static int build_from_source(int64_t n, int64_t nchunks, source_fn src, void* sctx,
                             uint64_t seed, uint32_t wmax, gg_csr* out) {
    memset(out, 0, sizeof(*out));
    out->n = n;
    int64_t* cnt = (int64_t*)calloc((size_t)(n + 1), sizeof(int64_t));
    if (!cnt) return GG_ENOMEM;
    count_ctx cc = {cnt};
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t ch = 0; ch < nchunks; ++ch) src(sctx, ch, emit_count, &cc);
    out->offsets = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!out->offsets) { free(cnt); return GG_ENOMEM; }
    int64_t s = 0;
    for (int64_t i = 0; i < n; ++i) { out->offsets[i] = s; s += cnt[i]; cnt[i] = out->offsets[i]; }
    out->offsets[n] = s;
    out->cols = (int32_t*)malloc(sizeof(int32_t) * (size_t)(s > 0 ? s : 1));
    if (!out->cols) { free(cnt); gg_free(out); return GG_ENOMEM; }
    scat_ctx sc = {cnt, out->cols};
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t ch = 0; ch < nchunks; ++ch) src(sctx, ch, emit_scatter, &sc);
    free(cnt);
    int rc = finish_csr(out);
    if (rc) { gg_free(out); return rc; }
    fill_weights(out, seed, wmax);
    return GG_OK;
}

/* ---- R-MAT ---------------------------------------------------------------- */

typedef struct {
    int scale; int64_t nedges; uint64_t seed;
    uint32_t ta, tab, tabc;
    const int32_t* perm;
} rmat_ctx;

#define RMAT_CHUNK 65536

static void rmat_source(void* c, int64_t chunk, emit_fn emit, void* ectx) {
    rmat_ctx* r = (rmat_ctx*)c;
    int64_t t0 = chunk * RMAT_CHUNK, t1 = t0 + RMAT_CHUNK;
    if (t1 > r->nedges) t1 = r->nedges;
    for (int64_t t = t0; t < t1; ++t) {
        int64_t u = 0, v = 0;
        uint64_t bits = 0;
        for (int l = 0; l < r->scale; ++l) {
            if ((l & 1) == 0) bits = rng4(r->seed, S_RMAT, (uint64_t)t, (uint64_t)(l >> 1));
            uint32_t x = (l & 1) ? (uint32_t)(bits >> 32) : (uint32_t)bits;
            int bu, bv;
            if (x < r->ta) { bu = 0; bv = 0; }
            else if (x < r->tab) { bu = 0; bv = 1; }
            else if (x < r->tabc) { bu = 1; bv = 0; }
            else { bu = 1; bv = 1; }
            u = (u << 1) | bu;
            v = (v << 1) | bv;
        }
        if (r->perm) { u = r->perm[u]; v = r->perm[v]; }
        if (u != v) emit(ectx, u, v);
    }
}

static uint32_t frac32(double p) {
    if (p <= 0.0) return 0u;
    if (p >= 1.0) return 0xFFFFFFFFu;
    return (uint32_t)(p * 4294967296.0);
}

/* R-MAT (Chakrabarti et al.) with quadrant probabilities (a, b, c, 1-a-b-c),
 * 2^scale vertices and edge_factor * 2^scale drawn edges.  With permute != 0
 * the vertex ids are relabelled by a seeded Fisher-Yates permutation. */
int gg_rmat(int scale, int64_t edge_factor, double a, double b, double c, uint32_t wmax,
            uint64_t seed, int permute, gg_csr* out) {
    if (scale < 1 || scale > 30 || edge_factor < 0 || wmax < 1 || !out) return GG_EINVAL;
    rmat_ctx r;
    r.scale = scale; r.seed = seed;
    r.nedges = edge_factor << scale;
    r.ta = frac32(a); r.tab = frac32(a + b); r.tabc = frac32(a + b + c);
    r.perm = NULL;
    int32_t* perm = NULL;
    int64_t n = (int64_t)1 << scale;
    if (permute) {
        perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
        if (!perm) return GG_ENOMEM;
        for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
        for (int64_t i = n - 1; i > 0; --i) {
            int64_t j = (int64_t)(rng4(seed, S_PERM, (uint64_t)i, 0) % (uint64_t)(i + 1));
            int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
        }
        r.perm = perm;
    }
    int64_t nchunks = (r.nedges + RMAT_CHUNK - 1) / RMAT_CHUNK;
    int rc = build_from_source(n, nchunks, rmat_source, &r, seed, wmax, out);
    free(perm);
    return rc;
}

/* ---- planted-partition SBM ------------------------------------------------ */

typedef struct {
    int64_t n, nblocks; uint64_t seed;
    double p_in, p_out, lq_in, lq_out;
} sbm_ctx;

#define SBM_CHUNK 256

/* block b holds vertices [ceil(b n / B), ceil((b+1) n / B)) */
static inline int64_t sbm_block_end(const sbm_ctx* s, int64_t u) {
    int64_t b = (u * s->nblocks) / s->n;
    /* smallest v with v * B / n >= b + 1 */
    int64_t bn = (b + 1) * s->n;
    return (bn + s->nblocks - 1) / s->nblocks;
}

/* Draw the Bernoulli(p) successes among positions [lo, hi) by geometric
 * skipping; emits (u, v) for each success v. */
static void sbm_range(const sbm_ctx* s, int64_t u, int64_t lo, int64_t hi, double p, double lq,
                      uint64_t stream, emit_fn emit, void* ectx) {
    if (hi <= lo || p <= 0.0) return;
    if (p >= 1.0) { for (int64_t v = lo; v < hi; ++v) emit(ectx, u, v); return; }
    int64_t pos = lo - 1;
    for (uint64_t t = 0;; ++t) {
        double q = det_log(u01(rng4(s->seed, stream, (uint64_t)u, t))) / lq;
        if (q >= (double)(hi - pos)) break;
        pos += (int64_t)q + 1;
        if (pos >= hi) break;
        emit(ectx, u, pos);
    }
}

static void sbm_source(void* c, int64_t chunk, emit_fn emit, void* ectx) {
    sbm_ctx* s = (sbm_ctx*)c;
    int64_t u0 = chunk * SBM_CHUNK, u1 = u0 + SBM_CHUNK;
    if (u1 > s->n) u1 = s->n;
    for (int64_t u = u0; u < u1; ++u) {
        int64_t be = sbm_block_end(s, u);
        sbm_range(s, u, u + 1, be, s->p_in, s->lq_in, S_SBM_IN, emit, ectx);
        sbm_range(s, u, be, s->n, s->p_out, s->lq_out, S_SBM_OUT, emit, ectx);
    }
}

/* Planted-partition stochastic block model: nblocks contiguous blocks, each
 * unordered pair joined with p_in inside a block and p_out across blocks. */
int gg_sbm(int64_t n, int64_t nblocks, double p_in, double p_out, uint32_t wmax, uint64_t seed,
           gg_csr* out) {
    if (n < 1 || n > 0x7FFFFFFF || nblocks < 1 || nblocks > n || wmax < 1 || !out) return GG_EINVAL;
    sbm_ctx s;
    s.n = n; s.nblocks = nblocks; s.seed = seed; s.p_in = p_in; s.p_out = p_out;
    s.lq_in = (p_in > 0.0 && p_in < 1.0) ? det_log(1.0 - p_in) : -1.0;
    s.lq_out = (p_out > 0.0 && p_out < 1.0) ? det_log(1.0 - p_out) : -1.0;
    int64_t nchunks = (n + SBM_CHUNK - 1) / SBM_CHUNK;
    return build_from_source(n, nchunks, sbm_source, &s, seed, wmax, out);
}

/* ---- 2-D grid with random rewiring ---------------------------------------- */

typedef struct { int64_t rows, cols, n, nedges; uint64_t seed; uint64_t thr; } grid_ctx;

#define GRID_CHUNK 65536

static void grid_source(void* c, int64_t chunk, emit_fn emit, void* ectx) {
    grid_ctx* g = (grid_ctx*)c;
    int64_t horiz = g->rows * (g->cols - 1);
    int64_t t0 = chunk * GRID_CHUNK, t1 = t0 + GRID_CHUNK;
    if (t1 > g->nedges) t1 = g->nedges;
    for (int64_t t = t0; t < t1; ++t) {
        int64_t u, v;
        if (t < horiz) { int64_t r = t / (g->cols - 1), cc = t % (g->cols - 1); u = r * g->cols + cc; v = u + 1; }
        else { int64_t q = t - horiz; u = q; v = q + g->cols; }
        if (rng4(g->seed, S_GRID, (uint64_t)t, 0) < g->thr) {
            /* rewire: replace one endpoint by a uniform vertex, redrawing self-loops */
            int which = (int)(rng4(g->seed, S_GRID_END, (uint64_t)t, 0) & 1);
            int64_t keep = which ? v : u, x = keep;
            for (uint64_t k = 0; x == keep; ++k)
                x = (int64_t)(rng4(g->seed, S_GRID_V, (uint64_t)t, k) % (uint64_t)g->n);
            u = keep; v = x;
        }
        emit(ectx, u, v);
    }
}

/* rows x cols 4-neighbour grid (no wrap-around); each edge is rewired with
 * probability p by replacing one endpoint with a uniform vertex.  Rewired
 * edges that land on an existing edge collapse into it. */
int gg_grid(int64_t rows, int64_t cols, double p, uint32_t wmax, uint64_t seed, gg_csr* out) {
    if (rows < 1 || cols < 1 || rows * cols > 0x7FFFFFFF || wmax < 1 || !out) return GG_EINVAL;
    grid_ctx g;
    g.rows = rows; g.cols = cols; g.n = rows * cols; g.seed = seed;
    g.nedges = rows * (cols - 1) + (rows - 1) * cols;
    g.thr = (p <= 0.0) ? 0ULL : (p >= 1.0 ? ~0ULL : (uint64_t)(p * 18446744073709551616.0));
    int64_t nchunks = (g.nedges + GRID_CHUNK - 1) / GRID_CHUNK;
    if (g.nedges == 0) nchunks = 0;
    return build_from_source(g.n, nchunks, grid_source, &g, seed, wmax, out);
}

/* ---- misc ------------------------------------------------------------------ */

/* 64-bit checksum of a CSR (n, nnz, offsets, cols, weights). */
uint64_t gg_checksum(int64_t n, int64_t nnz, const int64_t* offsets, const int32_t* cols,
                     const uint32_t* w) {
    uint64_t h = mix64((uint64_t)n) ^ mix64((uint64_t)nnz + 17);
    for (int64_t i = 0; i <= n; ++i) h = mix64(h ^ (uint64_t)offsets[i]);
    for (int64_t e = 0; e < nnz; ++e)
        h = mix64(h ^ ((uint64_t)(uint32_t)cols[e] | ((uint64_t)w[e] << 32)));
    return h;
}

/* Deterministic natural log, exposed so that seeded parameter draws made on
 * the host (log-uniform sizes) are the same on every machine. */
double gg_det_log(double x) { return det_log(x); }

int gg_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
