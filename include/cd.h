/*
 * cd.h - C ABI of the GB300 MG-sketch community-detection library.
 *
 * The library implements the local-moving sweep of Louvain, Leiden and LPA
 * with the weighted Misra-Gries (MG) sketch of arXiv 2411.02268 (Section 4,
 * Algorithm 1 in Appendix A.1) in hand-written sm_103a CUDA kernels, with an
 * exact per-vertex hashtable variant beside it (the paper's "Default",
 * Section 4, Fig. 1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Graph: undirected, both directions stored, CSR (Section 3: G = (V, E, w),
 *   w_ij = w_ji > 0).  offsets int64[n+1], cols int32[nnz], weights
 *   uint32[nnz].  Rows need not be sorted, but every result that depends on
 *   the order of a row (the MG sketch) follows the stored order.  A
 *   self-loop entry (i, i) counts in K_i and is skipped by the sweep
 *   (Algorithm 1, "exclude self").  n must be below 2^31 - 1 and every
 *   weight at least 1.
 * Memory: `memory` = CD_MEM_DEVICE means every array argument of the call
 *   (graph, labels, masks, outputs) is a device pointer of the current
 *   device; CD_MEM_HOST means they are host pointers and the library copies
 *   them in and out inside the call.  Device cols and weights must be 16-byte
 *   aligned (cudaMalloc memory is).  The caller owns every buffer it passes;
 *   the library only reads inputs and writes outputs.
 * Streams: `stream` is a cudaStream_t (NULL = the legacy default stream).
 *   Kernels are enqueued on it.  Calls that return host scalars (counts,
 *   modularity) synchronise the stream before returning.
 * Scratch: device scratch is allocated with cudaMallocAsync on the stream and
 *   freed before the call returns; its peak size is in cd_last_stats().
 *   The library raises the release threshold of the device's default memory
 *   pool (for this process) so that freed scratch stays mapped for the next
 *   call: to at least 16 GiB and twice the largest scratch of one call, at
 *   most a quarter of the device's memory.  A caller that needs that memory
 *   back trims the pool (cudaMemPoolTrimTo on cudaDeviceGetDefaultMemPool).
 *   Fault injection (for tests of callers' error paths): when the
 *   environment variable CD_FAIL_ALLOC holds n >= 1, the n-th scratch
 *   allocation of every call fails with CD_ENOMEM on the host, before the
 *   device is asked for it; what the call took before is released as on any
 *   error.
 * Errors: every entry point returns CD_OK (0) or a negative code; it never
 *   aborts or traps.  cd_strerror() names the code.  After CD_ECUDA the
 *   CUDA error string is in cd_last_stats()->cuda_error.
 * Threads: entry points may be called from several host threads; the
 *   statistics of the last call are kept per thread.
 */
#ifndef CD_H
#define CD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define CD_OK 0
#define CD_EINVAL (-1)    /* bad graph, labels or parameters */
#define CD_ENOMEM (-2)    /* device or host allocation failed */
#define CD_ECUDA (-3)     /* a CUDA call or kernel launch failed */
#define CD_ETIMEOUT (-4)  /* a bounded device wait gave up */
#define CD_EOVERFLOW (-5) /* a weight sum does not fit the integer type */
#define CD_ENOTIMPL (-6)  /* entry point or option not available */
#define CD_ESIZE (-7)     /* input larger than an entry point's fixed scratch holds */

/* sweep modes */
#define CD_MODE_LOUVAIN 0 /* delta-modularity, Eq. 2 (Section 3.3, 4.1) */
#define CD_MODE_LPA 1     /* maximum linking weight (Section 3.5, 4.3) */
#define CD_MODE_REFINE 2  /* Leiden refinement (Section 3.4, 4.2) */

/* memory kinds */
#define CD_MEM_DEVICE 0
#define CD_MEM_HOST 1

typedef struct cd_csr {
    int64_t n;
    int64_t nnz;
    const int64_t* offsets; /* n+1 entries, offsets[0] = 0, nondecreasing */
    const int32_t* cols;    /* nnz entries in [0, n) */
    const uint32_t* weights;/* nnz entries >= 1 */
    int32_t memory;         /* CD_MEM_DEVICE or CD_MEM_HOST */
} cd_csr;

/*
 * Stream schedule of the MG sketch (no counterpart in the paper, which
 * streams every row on one thread; this fixes how a row is split so that the
 * result is deterministic).  A row of length deg falls in the first bucket b
 * with deg <= deg_max[b] (the last bucket takes the rest) and is split into
 * lanes[b] streams: entry e of the row (e = global CSR index) belongs to
 * stream (e / vec) mod lanes[b], each stream feeds Algorithm 1 in increasing
 * e, and the partial sketches are combined by the tree
 * S[s] <- merge(S[s], S[s + o]) for o = lanes/2, ..., 1 and all s < o, where
 * merge(A, B) feeds every slot of B with a positive value, in slot order, to
 * A as one Algorithm 1 update.  lanes[b] is a power of two in [1, 256];
 * deg_max ascending; vec must be 4.  blocks_per_sm (launch shape only, no
 * effect on any result): 0 = the MG sweep kernel gets one 256-thread block
 * per group of rows ("virtual block"); n in [1, 8] = it gets n blocks per SM,
 * which stay resident and take the virtual blocks in turn, longest rows
 * first (a persistent launch).
 */
#define CD_MAX_BUCKETS 16
typedef struct cd_schedule {
    int32_t nbuckets;
    int32_t vec;
    int64_t deg_max[CD_MAX_BUCKETS];
    int32_t lanes[CD_MAX_BUCKETS];
    int32_t blocks_per_sm;
} cd_schedule;

/* Learned skip proposal (an addition to the paper's method, which has no
 * learned part): a perceptron 8 -> 32 (ReLU) -> 1 (sigmoid) on per-vertex
 * features predicting whether the vertex moves in the coming sweep.  float32
 * master weights; the kernels read them rounded to float16 (W1, w2) and
 * accumulate in float32.  Parameter order W1 (row j = hidden unit j), b1,
 * w2, b2. */
typedef struct cd_mlp {
    float W1[32][8];
    float b1[32];
    float w2[32];
    float b2;
} cd_mlp;

typedef struct cd_params {
    int32_t k;            /* MG slots: 1, 2, 4, 8, 16, 32 or 64; 0 = exact hashtable.  With
                             32 or 64 slots (the paper's Leiden uses 64, Section 5.3) a
                             schedule may give a row at most 32 streams */
    int32_t subtract;     /* 0 = conditional (Algorithm 1), 1 = unconditional (Section 4.1),
                             2 = the weighted Misra-Gries summary of the literature (no free
                             slot: every slot loses min(w, smallest value) and the rest of w
                             is inserted; not the paper's rule, offered for comparison; k <= 8
                             and agg_k = 0 only) */
    double tolerance;     /* Louvain: stop a pass when the sweep's summed delta-Q <= tolerance;
                             LPA: stop when at most tolerance * n labels changed (Section 3.5) */
    double tolerance_drop;/* Louvain: tolerance divided by this after each pass (>= 1) */
    double aggregation_tolerance; /* stop when |V'| > aggregation_tolerance * |V| */
    int32_t max_sweeps;   /* sweeps per pass (LPA: iterations) */
    int32_t max_passes;   /* Louvain/Leiden passes */
    const cd_schedule* sched; /* NULL = cd_default_schedule(k) */
    void* stream;         /* cudaStream_t */
    int32_t timing;       /* nonzero: time the sweep kernel with CUDA events on `stream`
                             (adds one event pair per sweep; see cd_stats) */
    int32_t colors;       /* drivers: each sweep is `colors` sub-sweeps, sub-sweep p deciding
                             the vertices i with lowbias32(i) mod colors = p from the state
                             left by the previous sub-sweeps (1 = fully synchronous sweeps,
                             0 = default 8, at most 16).  cd_sweep: the classes of a
                             sub-sweep (refine mode: 0 = 8; Louvain mode: 0 = 1, one class) */
    int32_t sub_color;    /* cd_sweep: the colour class deciding in this sweep (pass the
                             vertices of that class as `active`); the rules that guard
                             against simultaneous moves read it (see cd_sweep).  Must be
                             below the sweep's number of classes (CD_EINVAL otherwise) */
    int32_t one_scan;     /* LPA only (cd_sweep mode LPA, cd_lpa): the "1-scan" variant of
                             Section 4.3, deciding on the sketch values without the second
                             scan (needs k > 0) */
    int32_t agg_k;        /* drivers: 0 = exact aggregation (sort + segmented sum); 1..16
                             (power of two) = MG aggregation with agg_k slots (Section 4.1;
                             Leiden uses its symmetric form, Section 4.2), see cd_aggregate_mg */
    int32_t skip_rule;    /* Louvain and LPA drivers, sweeps after the first of a pass:
                             0 = every vertex decides; 1 = learned: only vertices whose
                             predicted move probability (skip_model) is >= skip_threshold;
                             2 = only movers of the previous sweep and their neighbours.
                             A sweep that skipped and then moved nobody or gained at most
                             the tolerance is followed by a full sweep, which decides
                             convergence. */
    float skip_threshold;
    const cd_mlp* skip_model; /* host memory, read during the call */
    int32_t capture;      /* drivers: nonzero = record the launches of one sweep (its
                             sub-sweeps, commits and, batched, the per-graph stopping rule)
                             once per level as a CUDA graph and replay it every sweep;
                             ignored with timing, skip rules or exact rows too long for
                             shared memory.  Results are the same either way. */
} cd_params;

typedef struct cd_stats {
    int64_t sweeps;          /* sweeps run by the last call (all passes) */
    int64_t passes;          /* passes (levels) of the last Louvain/Leiden call */
    int64_t moved;           /* vertices that changed label in the last sweep */
    uint64_t gain_lo, gain_hi;  /* last sweep: sum of scaled gains of movers (128-bit) */
    int64_t communities;     /* communities in the result */
    int64_t scratch_bytes;   /* peak device scratch of the last call */
    double sweep_kernel_ms;  /* total sweep-kernel time (timing != 0), CUDA events */
    int64_t sweep_kernel_launches;
    double modularity;       /* last modularity computed */
    int64_t entries_scanned; /* CSR entries of the vertices that decided (MG sweeps, all sweeps) */
    int64_t full_sweeps;     /* sweeps in which every vertex decided */
    char cuda_error[128];
    int64_t kernel_launches; /* kernels of this library launched by the last call (a CUDA-graph
                                replay counts the kernels recorded in the graph) */
    int64_t candidates;      /* MG sweeps (all sweeps): candidate communities evaluated by the
                                vertices that decided (the live sketch slots other than d); each
                                costs one gather of Sigma_c and of |c| */
    double phase_ms[4];      /* cd_sweep, host wall clock from the call's start to the end of:
                                [0] staging (device allocations, host inputs' copies enqueued),
                                [1] the O(n) checks of host inputs, [2] degrees, buckets and
                                totals (waits for offsets, labels and weights to arrive), [3]
                                the call (sweep, labels copied out, statistics read) */
} cd_stats;

/* Modularity parts (Eq. 1): Q = (two_m * sigma_in - sum_Sigma2) / two_m^2
 * where sigma_in = sum_c sigma_c and sum_Sigma2 = sum_c Sigma_c^2. */
typedef struct cd_modularity_parts {
    uint64_t sigma_in;
    uint64_t sum_sq_lo, sum_sq_hi;
    uint64_t two_m;
} cd_modularity_parts;

/* Name of a status code (static string). */
const char* cd_strerror(int code);

/* Statistics of the calling thread's last entry-point call. */
int cd_last_stats(cd_stats* out);

/* The schedule used when cd_params.sched is NULL, for sketch size k. */
int cd_default_schedule(int k, cd_schedule* out);

/*
 * One synchronous local-moving sweep (Section 4.1, Fig. 2; Section 4.3 for
 * LPA; Section 4.2 for refinement).  Every vertex decides from the state at
 * the start of the sweep:
 *   K_i, Sigma_c and community sizes are computed from labels_in;
 *   candidates: the slots of the row's MG sketch (k > 0) with a positive
 *   value, or every neighbouring community (k = 0), except the current
 *   community d = labels_in[i];
 *   K_{i->c} for every candidate and for d from a second scan of the row
 *   (self-loops skipped; in refine mode only neighbours j with
 *   bound[j] == bound[i]);
 *   Louvain/refine: gain(c) = 2m (K_{i->c} - K_{i->d}) - K_i (K_i + Sigma_c - Sigma_d)
 *   (Eq. 2 times 2m^2, exact 128-bit integers); a vertex whose community is
 *   a singleton may not join another singleton community with a larger id
 *   whose id is in the deciding colour class (lowbias32(c) mod colors =
 *   sub_color; with one class, every such community: no two singletons
 *   swap);
 *   the largest gain wins, ties to the smaller id; the vertex moves iff the
 *   gain is positive.  Refine additionally moves only vertices whose
 *   community is a singleton.
 *   LPA: the largest K_{i->c} wins, ties to the smaller id; the vertex moves
 *   iff it exceeds K_{i->d}.
 * labels_in: n labels in [0, n).  active: NULL or n bytes (0 = keep label).
 * bound: n labels (refine mode only, else NULL).  labels_out: n labels
 * (must not alias labels_in).  moved_out, gain_out (host, may be NULL):
 * number of movers and the 128-bit sum of their gains (LPA: of
 * K_{i->c} - K_{i->d}) as gain_out[0] (low) and gain_out[1] (high).
 * Returns CD_EOVERFLOW if 2m does not fit 63 bits.
 */
int cd_sweep(const cd_csr* g, const cd_params* p, int mode, const uint32_t* labels_in,
             const uint8_t* active, const uint32_t* bound, uint32_t* labels_out,
             int64_t* moved_out, uint64_t* gain_out);

/* Modularity of `labels` (Eq. 1, Section 3.2) from exact integer parts.
 * labels: n labels in [0, n).  q_out, parts (host, either may be NULL). */
int cd_modularity(const cd_csr* g, const uint32_t* labels, void* stream, double* q_out,
                  cd_modularity_parts* parts);

/* Louvain (Section 3.3, 4.1): passes of synchronous local-moving sweeps
 * followed by aggregation into the super-vertex graph (renumbering by
 * prefix scan, super-edges by sort and segmented sum), until a pass moves
 * nobody, |V'| > aggregation_tolerance |V|, or max_passes.  labels_out: n
 * dense community ids (ascending order of first appearance by id);
 * q_out (host, may be NULL): modularity of the result on the input graph. */
int cd_louvain(const cd_csr* g, const cd_params* p, uint32_t* labels_out, double* q_out);

/* Batched Louvain: `ngraphs` independent graphs detected together (the paper
 * runs one graph at a time; batching is an addition to its method that
 * changes none of its arithmetic).  The graphs are packed into one disjoint
 * union whose every graph starts its CSR entries on a multiple of 1024, so
 * that the sketch kernels give each graph the stream partition of a run on
 * its own; each sweep of the union is one launch per colour class over all
 * graphs, with 2m, the stopping rule (moved nobody, summed delta-Q <=
 * tolerance, max_sweeps) and the pass rule (|V'| = |V| or > aggregation_
 * tolerance |V|) applied per graph.  Every graph's labels, modularity and
 * sweep count equal those of cd_louvain on that graph alone with the same
 * parameters.
 * graphs: ngraphs CSRs, all in the same memory space (each n < 2^31 - 1,
 * the sum of n + 1 below 2^31 - 1).  labels_out[g]: graphs[g].n dense
 * community ids, same memory space as the graphs (may be NULL when n = 0).
 * q_out, sweeps_out (host, may be NULL): ngraphs modularities and sweep
 * counts (all passes).  skip_rule and one_scan must be 0.  cd_stats counts
 * the sweeps and passes of the union. */
int cd_louvain_batched(const cd_csr* graphs, int ngraphs, const cd_params* p, uint32_t* const* labels_out,
                       double* q_out, int64_t* sweeps_out);

#define CD_TUNE_MAX_K 8

typedef struct cd_tune_report {
    double default_ms;                  /* one full sweep of the packed batch, default schedule, k = ks[0] */
    double sweep_ms[CD_TUNE_MAX_K];     /* candidate i: one full sweep with its tuned schedule */
    double run_ms[CD_TUNE_MAX_K];       /* candidate i: the whole batched Louvain with that schedule */
    double q_mean[CD_TUNE_MAX_K];       /* candidate i: mean modularity over the graphs */
    int32_t trials;                     /* timed sweeps */
    int32_t chosen;                     /* index of the chosen candidate */
} cd_tune_report;

/* Autotuner of the batched form (an addition to the paper's method; it
 * changes no arithmetic, only the schedule and k): packs the graphs as
 * cd_louvain_batched does, then for every candidate sketch size ks[i] (nks
 * <= CD_TUNE_MAX_K, each a valid k) tunes the schedule (p->sched or the
 * default) by coordinate descent on timed sweeps of the whole batch from
 * singleton labels, keeping a change only when it is at least 2% faster
 * (median of 3 CUDA-event timings): the streams per degree band (each band,
 * longest rows first, tries half and twice its streams), then the band
 * thresholds (each deg_max tries 3/4 and 3/2 of its value, order kept), then
 * the launch shape (blocks_per_sm 0, 4, 2); and runs batched Louvain with
 * the tuned schedule.  The choice is the fastest
 * candidate whose mean modularity is within q_tol (relative) of the best
 * candidate's.  sched_out, k_out (host) receive it; report (host, may be
 * NULL) the timings.  Timings vary from run to run, so the choice may too;
 * the results of a given (schedule, k) do not. */
int cd_autotune(const cd_csr* graphs, int ngraphs, const cd_params* p, const int* ks, int nks, double q_tol,
                cd_schedule* sched_out, int* k_out, cd_tune_report* report);

/* LPA (Section 3.5, 4.3): synchronous iterations from singleton labels until
 * at most tolerance * n labels change or max_sweeps.  Same outputs. */
int cd_lpa(const cd_csr* g, const cd_params* p, uint32_t* labels_out, double* q_out);

/* Leiden (Section 3.4, 4.2).  Same outputs. */
int cd_leiden(const cd_csr* g, const cd_params* p, uint32_t* labels_out, double* q_out);

/* Aggregation step on its own (Section 3.3): labels (n, any ids < n) are
 * renumbered densely in ascending id order (dense_out, n entries) and the
 * super-vertex graph is written to offsets_out (n+1 capacity), cols_out and
 * weights_out (nnz capacity each); *n_out and *nnz_out (host) receive its
 * size.  Rows are sorted by column; the self-loop of c holds the summed
 * weight of both directions of c's internal edges.  Device memory only. */
int cd_aggregate(const cd_csr* g, const uint32_t* labels, void* stream, uint32_t* dense_out,
                 int64_t* offsets_out, int32_t* cols_out, uint32_t* weights_out,
                 int64_t* n_out, int64_t* nnz_out);

/* MG aggregation (Section 4.1, "aggregation phase", Fig. 3): like
 * cd_aggregate, but super-vertex c links only to the communities left in one
 * k-slot MG sketch (Algorithm 1, subtract as in cd_params) fed with the edges
 * of all members of c (ascending vertex id, each row in stored order,
 * self-loops kept), streams and merge tree as in the sweep (schedule by the
 * community's total entry count; NULL = default), with the sketch values as
 * weights and no second pass.  symmetric = 0: row c = the live slots of
 * sketch(c), sorted by column (may be asymmetric, as in the paper's Louvain).
 * symmetric = 1 (Leiden, Section 4.2): every live slot (c, d, v) yields
 * (c, d) and (d, c); when sketch(c) holds d and sketch(d) holds c, the value
 * of the smaller community's sketch is kept.  k: 1, 2, 4, 8 or 16.  Device
 * memory only; outputs as cd_aggregate (cols_out and weights_out hold nnz
 * entries, which bounds the result for an undirected input; CD_EINVAL if the
 * result would not fit); CD_EOVERFLOW if a value exceeds 32 bits. */
int cd_aggregate_mg(const cd_csr* g, const uint32_t* labels, int k, int subtract, int symmetric,
                    const cd_schedule* sched, void* stream, uint32_t* dense_out, int64_t* offsets_out,
                    int32_t* cols_out, uint32_t* weights_out, int64_t* n_out, int64_t* nnz_out);

/* Features of the learned skip proposal for every vertex (n x 8 float16,
 * device): log2(1 + deg) / 16; moved in the previous sweep; min(sweeps since
 * its last move, 8) / 8; log2(1 + |community|) / 24; sqrt(Sigma_d / 2m);
 * K_i / Sigma_d; K_{i->C_i} / K_i at the vertex's last decision (attach,
 * 0 before any); 1.  labels: n community ids; moved_last, since_move: n bytes
 * each, attach: n floats (NULL = zeros).  Device memory only. */
int cd_features(const cd_csr* g, const uint32_t* labels, const uint8_t* moved_last, const uint8_t* since_move,
                const float* attach, uint16_t* x_out, void* stream);

/* Forward pass of the skip model on n feature rows (device x, n x 8 float16):
 * p_out[i] (device, float32) = predicted move probability. */
int cd_mlp_forward(const uint16_t* x, int64_t n, const cd_mlp* model, float* p_out, void* stream);

/* Mean binary cross-entropy of the model on (x, y) (y: n bytes, 0/1, device)
 * and its gradient (host cd_mlp with the parameter layout), summed in a
 * fixed order (deterministic). */
int cd_mlp_gradient(const uint16_t* x, const uint8_t* y, int64_t n, const cd_mlp* model, cd_mlp* grad_out,
                    double* loss_out, void* stream);

/* `steps` full-batch Adam steps (learning rate lr) on (x, y) with the
 * gradient kernel above, starting from *model (updated in place); loss_out
 * (host, may be NULL) receives the loss before the last step. */
int cd_mlp_train(const uint16_t* x, const uint8_t* y, int64_t n, int steps, double lr, cd_mlp* model,
                 double* loss_out, void* stream);

/* Move traces of the plain method: runs the first local-moving phase of
 * Louvain on g (every vertex deciding in every sweep, parameters as
 * cd_louvain) and records, for sweeps after the first, the features of a
 * sample of the vertices with edges (each with probability sample_rate,
 * chosen by a hash of (vertex, sweep)) at the start of the sweep and whether
 * the vertex moved in it.  x_out: capacity x 8 float16, y_out: capacity bytes
 * (device); *count_out (host) = samples written (at most capacity). */
int cd_trace(const cd_csr* g, const cd_params* p, double sample_rate, uint16_t* x_out, uint8_t* y_out,
             int64_t capacity, int64_t* count_out);

/*
 * Modularity without any device allocation.  The paper has no counterpart:
 * this is an interface for callers that cannot allocate device memory while
 * they call the library - for example code whose device memory is owned by a
 * framework's caching allocator (a raw cudaMalloc/cudaFree there would
 * synchronise the device or fragment the pool), or services that must keep a
 * fixed device-memory budget.  It computes exactly what cd_modularity
 * computes (same kernels, same integer parts), but its scratch (weighted
 * degrees, community totals and sizes of up to 2^20 vertices, 20 MiB plus
 * 256 bytes) is one fixed array inside the library, which every GPU that
 * loads the library holds until the process exits.  It calls no cudaMalloc,
 * cudaFree or other allocating routine.
 * The first call on a device looks up the array's device address (with that
 * device current) and caches it.  Like the other entry points that return
 * host results, every call copies its result to the host and synchronises
 * `stream`.  All calls share the array and each call starts by
 * clearing what it reads: calls whose work overlaps on the GPU (several
 * streams, several host threads) race on it and must be serialised by the
 * caller.  Device memory only (CD_EINVAL for CD_MEM_HOST); n > 2^20 returns
 * CD_ESIZE.  Other arguments and results as cd_modularity; the call
 * synchronises `stream`.
 */
int cd_modularity_noalloc(const cd_csr* g, const uint32_t* labels, void* stream, double* q_out,
                          cd_modularity_parts* parts);

#ifdef __cplusplus
}
#endif

#endif /* CD_H */
