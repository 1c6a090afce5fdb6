// Internal declarations shared by the CUDA translation units of the library.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "cd.h"

namespace cdk {

constexpr uint32_t kEmpty = 0xFFFFFFFFu;  // key of a never-used sketch slot
constexpr int kBlock = 256;               // threads per block of the sweep kernels

// Kernels launched on this host thread since the current API call began
// (cd_stats.kernel_launches); every launch site calls note_launch() as it
// launches.
extern thread_local int64_t g_kernel_launches;
inline void note_launch(int64_t count = 1) { g_kernel_launches += count; }

typedef __int128 i128;
typedef unsigned __int128 u128;

// Device-side scalars of one call.
struct Globals {
    unsigned long long two_m;    // sum of K_i
    unsigned long long max_k;    // max K_i
    unsigned long long moved;    // movers in the last sweep
    unsigned long long gain_lo;  // 128-bit sum of movers' gains
    unsigned long long gain_hi;
    unsigned long long scanned;  // CSR entries of the vertices that decided
    unsigned long long cands;    // MG sweeps: candidates evaluated by the vertices that decided
    unsigned long long sigma_in; // modularity: sum_c sigma_c
    unsigned long long sq_lo;    // modularity: sum_c Sigma_c^2
    unsigned long long sq_hi;
    unsigned long long count;    // generic counter (renumbering)
    unsigned long long mark;     // movers before the current sub-sweep
    unsigned int err;            // nonzero: a device-side check failed
    unsigned int pad;
};

// Buckets of vertices by row length; bucket b holds verts[vbegin[b], vbegin[b+1])
// and is processed by grid blocks [bbegin[b], bbegin[b+1]).
struct BucketTable {
    int nb;
    int qmul;      // lanes per stream: k / 8 for the slot form of k >= 32, else 1 (0 reads as 1)
    int resident;  // MG sweep launch: blocks per SM that stride over the virtual blocks (0 = one each)
    int lanes[CD_MAX_BUCKETS];
    int64_t deg_max[CD_MAX_BUCKETS];
    int64_t vbegin[CD_MAX_BUCKETS + 1];
    int64_t bbegin[CD_MAX_BUCKETS + 1];
};

// Bucket ranges of one colour class after the skip mask has removed the
// vertices that do not decide (written on the device, see launch_compact).
struct DevRanges {
    int64_t vbegin[CD_MAX_BUCKETS + 1];
    int64_t bbegin[CD_MAX_BUCKETS + 1];
};

struct SweepArgs {
    const int64_t* off;
    const int32_t* cols;
    const uint32_t* w;
    const uint32_t* labels;   // sweep-start labels
    const uint64_t* K;
    const uint64_t* Sigma;
    const uint32_t* size;
    const uint8_t* active;    // may be null
    const uint32_t* bound;    // refine mode only
    uint32_t* labels_out;
    uint32_t* movers;         // optional list of movers (driver), capacity n
    float* attach;            // optional: K_{i->C_i} after the decision, as a float (skip features)
    // batched form (a disjoint union of graphs); null for a single graph
    const uint32_t* gid;      // graph of every vertex
    const unsigned long long* two_m_g;  // 2m of every graph
    const uint8_t* gdone;     // graphs whose local-moving phase has stopped
    unsigned long long* g_moved;        // per graph: movers, 128-bit gain sum
    unsigned long long* g_gain_lo;
    unsigned long long* g_gain_hi;
    Globals* glob;
    const uint32_t* verts;    // bucket-ordered vertex ids
    const DevRanges* dr;      // MG sweeps: ranges of verts on the device (blocks past them exit); null = bt
    int64_t n;
    int64_t nnz;
    int mode;
    int uncond;
    int one_scan;             // LPA: decide on sketch values, no second scan
    int out_all;              // 1: labels_out for every listed vertex; 0: only for the deciding ones
                              // (the drivers read labels_out of movers only)
    int colors;               // colour classes of the driver (1: a fully synchronous sweep)
    int sub_color;            // colour class deciding in this sub-sweep
    const uint32_t* cid;      // colour id of every vertex (its id inside its graph); null = the vertex id
    uint32_t* elab;           // k <= 16: label of every CSR entry as the first scan saw it (kEmpty =
                              // skipped), read back by the second scan; null = re-gather
    BucketTable bt;
};

// MG aggregation: communities are the rows (buckets over communities in
// a.verts/a.bt, member ranges in moff/members, dense ids in a.labels).
struct AggArgs {
    SweepArgs a;
    const int64_t* moff;      // nc + 1
    const uint32_t* members;  // vertex ids grouped by community, ascending
    uint32_t* out_keys;       // nc * k
    unsigned long long* out_vals;
};

// Colour class of vertex v among `colors` classes: the 32-bit integer hash
// "lowbias32" (C. Wellons) of v, modulo the number of classes.
__host__ __device__ __forceinline__ uint32_t color_of(uint32_t v, int colors) {
    if (colors <= 1) return 0u;
    uint32_t x = v;
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x % (uint32_t)colors;
}

// Whether vertex i decides in this sweep (the skip mask and, batched, its
// graph still moving).
__device__ __forceinline__ bool vertex_decides(const SweepArgs& a, uint32_t i) {
    if (a.active && !a.active[i]) return false;
    if (a.gdone && a.gdone[a.gid[i]]) return false;
    return true;
}

// 2m of vertex i's graph.
__device__ __forceinline__ unsigned long long two_m_of(const SweepArgs& a, uint32_t i) {
    return a.gid ? a.two_m_g[a.gid[i]] : a.glob->two_m;
}

// Per-graph statistics of a mover (batched form).
__device__ __forceinline__ void graph_stats(const SweepArgs& a, uint32_t i, u128 gain) {
    const uint32_t g = a.gid[i];
    atomicAdd(&a.g_moved[g], 1ull);
    const unsigned long long lo = (unsigned long long)gain, hi = (unsigned long long)(gain >> 64);
    const unsigned long long old = atomicAdd(&a.g_gain_lo[g], lo);
    const unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
    if (hi + carry) atomicAdd(&a.g_gain_hi[g], hi + carry);
}

// Whether the singleton community c may be left by its vertex in the
// deciding sub-sweep: its id has the sub-sweep's colour.
__device__ __forceinline__ bool deciding_colour(const SweepArgs& a, uint32_t c) {
    return (int)color_of(a.cid ? a.cid[c] : c, a.colors) == a.sub_color;
}
// Refine mode (Leiden): a singleton community whose vertex has the colour of
// the deciding sub-sweep is not a candidate (its only member may leave in the
// same sub-sweep).  Louvain: a singleton may not join a larger-id singleton
// that decides in the same sub-sweep (no pairwise swaps of simultaneous
// moves; with one colour class that is every singleton).
__device__ __forceinline__ bool barred(const SweepArgs& a, uint32_t c, uint32_t d, bool d_single) {
    if (a.mode == CD_MODE_REFINE) return a.size[c] == 1 && deciding_colour(a, c);
    return d_single && c > d && a.size[c] == 1 && deciding_colour(a, c);
}
// barred() with |c| already loaded.
__device__ __forceinline__ bool barred_n(const SweepArgs& a, uint32_t c, uint32_t d, bool d_single,
                                         uint32_t size_c) {
    if (a.mode == CD_MODE_REFINE) return size_c == 1 && deciding_colour(a, c);
    return d_single && c > d && size_c == 1 && deciding_colour(a, c);
}

// Lanes per stream of the MG sweep kernel for sketch size k (the slot form
// spreads k >= 32 slots over k / 8 lanes), and the threads of one row.
__host__ __device__ __forceinline__ int slot_lanes(int k) { return k >= 32 ? k / 8 : 1; }
__host__ __device__ __forceinline__ int threads_per_row(const BucketTable& bt, int b) {
    return bt.lanes[b] * (bt.qmul > 1 ? bt.qmul : 1);
}

// Host-side launchers (sweep.cu).
cudaError_t launch_degrees(const int64_t* off, const uint32_t* w, int64_t n, int64_t nnz,
                           uint64_t* K, Globals* glob, cudaStream_t s);
// Sigma_c and |c| from labels (null: singletons), 2m and max K_i into glob.
cudaError_t launch_totals(const uint32_t* labels, const uint64_t* K, int64_t n, uint64_t* Sigma,
                          uint32_t* size, Globals* glob, cudaStream_t s);
// Bucketing by (colour class, bucket): tile_counts / tile_offsets need
// colors * nb * bucket_tiles(n) entries; bucket_starts (colors * nb + 1 int64)
// receives the first index of every (colour, bucket) range in verts and the
// total.  Rows of length 0 are not listed; their label is
// copied from labels_in to labels_out when labels_out is not null.  The
// colour class of vertex v is that of cid[v] (of v when cid is null).
int64_t bucket_tiles(int64_t n);
cudaError_t launch_bucket(const int64_t* off, int64_t n, int64_t nnz, const BucketTable& bt, int colors,
                          const uint32_t* cid, uint32_t* tile_counts, uint32_t* tile_offsets, int64_t* bucket_starts,
                          uint32_t* verts, const uint32_t* labels_in, uint32_t* labels_out,
                          Globals* glob, cudaStream_t s, unsigned long long* scan_scratch = nullptr);
cudaError_t launch_sweep_mg(const SweepArgs& a, int k, bool wide, int64_t nblocks, cudaStream_t s);
// Compaction of the bucketed vertex list to the vertices whose active byte is
// set, order kept: cverts (n_listed), per colour class the new ranges in
// dr[colors].  starts: the (colour, bucket) range starts of verts on the
// device (colors * bt.nb + 1); flags/pos: n_listed scratch; tiles: scan
// scratch; total: one device counter.
cudaError_t launch_compact(const uint32_t* verts, int64_t n_listed, const uint8_t* active, const int64_t* starts,
                           const BucketTable& bt, int colors, uint32_t* flags, uint32_t* pos,
                           unsigned long long* tiles, unsigned long long* total, uint32_t* cverts, DevRanges* dr,
                           cudaStream_t s);
// K_i for the rows of one bucket table (vbegin ranges; bbegin is recomputed).
cudaError_t launch_row_sums(const int64_t* off, const uint32_t* w, int64_t n, int64_t nnz, const uint32_t* verts,
                            const BucketTable& bt, uint64_t* K, Globals* glob, cudaStream_t s);
cudaError_t launch_agg_mg(const AggArgs& g, int k, bool wide, int64_t nblocks, cudaStream_t s);
// Movers [mark, moved) of the last sub-sweep: Sigma and sizes moved from
// labels[i] to labels_out[i], then labels[i] = labels_out[i].
cudaError_t launch_commit(const uint32_t* movers, uint32_t* labels, const uint32_t* labels_out, const uint64_t* K,
                          int64_t n, uint64_t* Sigma, uint32_t* size, Globals* glob, cudaStream_t s);

// sweep_exact.cu
size_t exact_group_smem(int G, uint32_t T);
cudaError_t launch_exact_group(const SweepArgs& a, int bucket, int G, uint32_t T, cudaStream_t s);
cudaError_t launch_exact_block(const SweepArgs& a, int bucket, uint32_t T_smem, uint32_t* gkeys,
                               unsigned long long* gvals, const int64_t* table_off, cudaStream_t s);
cudaError_t launch_exact_table_sizes(const SweepArgs& a, int bucket, int64_t* sizes, cudaStream_t s);

// modularity.cu: Sigma_scratch and sizes_scratch hold n entries; glob->two_m,
// sigma_in, sq_lo and sq_hi must be zero on entry.
cudaError_t launch_modularity(const int64_t* off, const int32_t* cols, const uint32_t* w,
                              const uint32_t* labels, int64_t n, int64_t nnz, const uint64_t* K,
                              uint64_t* Sigma_scratch, uint32_t* sizes_scratch, Globals* glob,
                              cudaStream_t s);

// scan.cu
int64_t scan_tiles(int64_t n);
cudaError_t launch_exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n,
                                      unsigned long long* tile_scratch, unsigned long long* total_dev,
                                      cudaStream_t s);
cudaError_t launch_exclusive_scan_u32_to_i64(const uint32_t* in, int64_t* out, int64_t n,
                                             unsigned long long* tile_scratch, unsigned long long* total_dev,
                                             cudaStream_t s);

// aggregate.cu
cudaError_t launch_renumber(const uint32_t* labels, int64_t n, uint32_t* dense, uint32_t* scratch_n,
                            unsigned long long* tile_scratch, unsigned long long* count_dev, Globals* glob,
                            cudaStream_t s);
cudaError_t launch_compose(uint32_t* top, int64_t n0, const uint32_t* dense, cudaStream_t s);
cudaError_t launch_iota(uint32_t* x, int64_t n, cudaStream_t s);
cudaError_t launch_scatter_bound(const uint32_t* sub, const uint32_t* bound, int64_t n, uint32_t* next_init,
                                 cudaStream_t s);
int64_t radix_tiles(int64_t n);
struct AggScratch {
    uint32_t *src, *dst, *w, *src2, *dst2, *w2, *hist, *heads;
    unsigned long long *wsum, *tiles;
};
cudaError_t launch_expand(const int64_t* off, const int32_t* cols, int64_t n, int64_t nnz, const uint32_t* dense,
                          uint32_t* src, uint32_t* dst, Globals* glob, cudaStream_t s);
cudaError_t radix_sort_pairs(AggScratch& a, int64_t nnz, int64_t nc, Globals* glob, cudaStream_t s);
cudaError_t radix_sort_keys(AggScratch& a, int64_t nnz, int bits_src, int bits_dst, Globals* glob, cudaStream_t s);
int bits_for(int64_t nc);
cudaError_t launch_community_counts(const int64_t* off, const uint32_t* dense, int64_t n, uint32_t* cnt,
                                    uint32_t* ecnt, cudaStream_t s);
cudaError_t launch_mg_sort_rows(uint32_t* keys, unsigned long long* vals, int64_t nc, int k, uint32_t* count,
                                uint32_t* self_less, cudaStream_t s);
cudaError_t launch_mg_write_rows(const uint32_t* keys, const unsigned long long* vals, int64_t nc, int k,
                                 const int64_t* roff, int32_t* cols_out, uint32_t* w_out, Globals* glob,
                                 cudaStream_t s);
cudaError_t launch_mg_candidates(const uint32_t* keys, const unsigned long long* vals, int64_t nc, int k,
                                 const int64_t* fpos, const int64_t* rpos, int64_t R0, AggScratch& a, Globals* glob,
                                 cudaStream_t s);
cudaError_t launch_mg_select(const AggScratch& a, int64_t m, uint32_t* keep, cudaStream_t s);
cudaError_t launch_mg_compact(const AggScratch& a, const uint32_t* keep, const uint32_t* pos, int64_t m,
                              int32_t* cols_out, uint32_t* w_out, uint32_t* rowcnt, cudaStream_t s);
cudaError_t launch_heads(const AggScratch& a, int64_t nnz, cudaStream_t s);
cudaError_t launch_segsum(const AggScratch& a, const uint32_t* uidx, int64_t nnz, int32_t* cols_out,
                          uint32_t* rowcnt, cudaStream_t s);
cudaError_t launch_narrow(const unsigned long long* wsum, int64_t m, uint32_t* w_out, Globals* glob,
                          cudaStream_t s);

// mlp.cu (learned skip proposal)
cudaError_t launch_features(const int64_t* off, const uint64_t* K, const uint32_t* labels, const uint64_t* Sigma,
                            const uint32_t* size, unsigned long long two_m, const uint8_t* moved_last,
                            const uint8_t* since_move, const float* attach, bool attach_raw, int64_t n, void* x,
                            cudaStream_t s);
// Features and forward pass in one kernel (attach holds raw K_{i->C_i}):
// active[i] = (predicted move probability >= thr).
cudaError_t launch_propose(const int64_t* off, const uint64_t* K, const uint32_t* labels, const uint64_t* Sigma,
                           const uint32_t* size, unsigned long long two_m, const uint8_t* moved_last,
                           const uint8_t* since_move, const float* attach, int64_t n, const float* param, float thr,
                           uint8_t* active, cudaStream_t s);
cudaError_t launch_mlp_forward(const void* x, int64_t n, const float* param, float* p, uint8_t* active, float thr,
                               cudaStream_t s);
int64_t mlp_grad_blocks(int64_t n);
int mlp_param_count();
cudaError_t launch_mlp_grad(const void* x, const uint8_t* y, int64_t n, const float* param, float* partial,
                            float* loss_partial, float* grad, float* loss, cudaStream_t s);
cudaError_t launch_adam(float* param, const float* grad, float* m1, float* m2, int step, float lr, cudaStream_t s);
cudaError_t launch_move_state(const uint32_t* before, const uint32_t* after, int64_t n, uint8_t* moved_last,
                              uint8_t* since_move, cudaStream_t s);
cudaError_t launch_mark_neighbours(const int64_t* off, const int32_t* cols, const uint32_t* movers,
                                   const Globals* glob, uint8_t* active, cudaStream_t s);
cudaError_t launch_trace_flags(const int64_t* off, int64_t n, int sweep, uint32_t thr32, uint32_t* flags,
                               cudaStream_t s);
cudaError_t launch_trace_write(const void* x, const uint8_t* moved_last, const uint32_t* flags, const uint32_t* pos,
                               int64_t n, int64_t base, void* xo, uint8_t* yo, int64_t cap, cudaStream_t s);

// Device-side error flags (Globals::err bits).
constexpr unsigned kErrBadOffsets = 1u;
constexpr unsigned kErrBadCol = 2u;
constexpr unsigned kErrZeroWeight = 4u;
constexpr unsigned kErrBadLabel = 8u;
constexpr unsigned kErrWeightOverflow = 16u;

}  // namespace cdk
