// Batched form (batch.cu): packing of a disjoint union of graphs and the
// per-graph bookkeeping of its local-moving phase.
#pragma once

#include "cd_internal.cuh"

namespace cdk {

constexpr int64_t kPackAlign = 1024;  // entry alignment of every graph in the union (4 x 256 streams)

// One graph's rows [vsrc0, vsrc0 + n) of a source CSR, placed at destination
// vertices [vbase, vbase + n) and entries [ebase, ebase + nnz), followed by
// its padding vertex vbase + n with pad self-loops.  Source columns plus
// col_shift must fall in [vbase, vbase + n).
struct PackGraph {
    const int64_t* off;
    const int32_t* cols;
    const uint32_t* w;
    int64_t vsrc0, n, nnz;
    int64_t vbase, ebase, pad;
    int64_t col_shift;
    int64_t check_first;  // source offsets must start at 0
};

int64_t pack_tiles(const PackGraph& p);
// tstart: G + 1 prefix sums of pack_tiles; writes uoff[0, n_total], ucols,
// uw, gid (sentinel G for padding vertices) and lid (id inside the graph).
cudaError_t launch_pack(const PackGraph* pg, const int64_t* tstart, int G, int64_t tiles, int64_t* uoff,
                        int32_t* ucols, uint32_t* uw, uint32_t* gid, uint32_t* lid, int64_t n_total,
                        int64_t nnz_total, Globals* glob, cudaStream_t s);
cudaError_t launch_graph_two_m(const uint64_t* K, const int64_t* vb, const int64_t* nv, int G,
                               unsigned long long* two_m_g, cudaStream_t s);
cudaError_t launch_batch_converge(int G, const unsigned long long* two_m_g, const unsigned long long* g_moved,
                                  const unsigned long long* g_gain_lo, const unsigned long long* g_gain_hi,
                                  double tol, int64_t max_sweeps, uint32_t* gsweeps, uint8_t* gdone, Globals* glob,
                                  cudaStream_t s);
cudaError_t launch_gather_u32(const uint32_t* x, const int64_t* idx, int G, uint32_t* out, cudaStream_t s);
cudaError_t launch_gather_i64(const int64_t* x, const int64_t* idx, int count, int64_t* out, cudaStream_t s);
cudaError_t launch_batch_labels(const uint32_t* top, const uint32_t* gid, int64_t n, int G, const int64_t* vb0,
                                const int64_t* cb, uint32_t* loc, uint32_t* qlab, cudaStream_t s);
cudaError_t launch_batch_modularity(const int64_t* off, const int32_t* cols, const uint32_t* w,
                                    const uint32_t* labels, const uint64_t* Sigma, const int64_t* vb,
                                    const int64_t* nv, int G, unsigned long long* acc, cudaStream_t s);

}  // namespace cdk
