// Batched form: many independent graphs detected together as one disjoint
// union (an addition to the paper's method, which runs one graph at a time).
//
// Layout of the union at every level: graph g owns the vertex range
// [vbase_g, vbase_g + n_g] and the entry range [ebase_g, ebase_g + nnz_g +
// pad_g).  Vertex vbase_g + n_g is a padding vertex whose row holds pad_g
// self-loops of weight 1, so that the next graph's first entry starts on a
// multiple of kPackAlign.  The sketch kernels assign entry e to stream
// (e / 4) mod L with L <= 256, so with aligned bases every graph is scanned
// with the same stream partition as when it is detected on its own, and the
// union's sweeps give every graph exactly the labels of its own run.
// Padding vertices belong to the sentinel graph G, which never decides.
#include "cd_internal.cuh"
#include "batch.cuh"

namespace cdk {

constexpr int kPackTile = 2048;

__device__ __forceinline__ int graph_of_tile(const int64_t* __restrict__ tstart, int G, int64_t t) {
    int lo = 0, hi = G;  // tstart[lo] <= t < tstart[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (tstart[mid] <= t) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void k_pack(const PackGraph* __restrict__ pg, const int64_t* __restrict__ tstart, int G,
                       int64_t* __restrict__ uoff, int32_t* __restrict__ ucols, uint32_t* __restrict__ uw,
                       uint32_t* __restrict__ gid, uint32_t* __restrict__ lid, Globals* glob) {
    const int64_t t = blockIdx.x;
    const int g = graph_of_tile(tstart, G, t);
    const PackGraph p = pg[g];
    const int64_t local = t - tstart[g];
    const int64_t vt = (p.n + 1 + kPackTile - 1) / kPackTile;
    if (local < vt) {
        const int64_t o0 = p.n > 0 ? p.off[p.vsrc0] : 0;
        for (int64_t i = local * kPackTile + threadIdx.x; i < (local + 1) * kPackTile && i <= p.n; i += blockDim.x) {
            const int64_t v = p.vbase + i;
            if (i < p.n) {
                const int64_t a = p.off[p.vsrc0 + i], b = p.off[p.vsrc0 + i + 1];
                if (b < a || (p.check_first && i == 0 && a != 0) || (i == p.n - 1 && b - o0 != p.nnz))
                    atomicOr(&glob->err, kErrBadOffsets);
                uoff[v] = p.ebase + (a - o0);
                gid[v] = (uint32_t)g;
                lid[v] = (uint32_t)i;
            } else {
                uoff[v] = p.ebase + p.nnz;
                gid[v] = (uint32_t)G;
                lid[v] = 0;
            }
        }
        return;
    }
    const int64_t et = local - vt;
    const int64_t e0 = p.n > 0 ? p.off[p.vsrc0] : 0;
    const int64_t total = p.nnz + p.pad;
    for (int64_t e = et * kPackTile + threadIdx.x; e < (et + 1) * kPackTile && e < total; e += blockDim.x) {
        const int64_t d = p.ebase + e;
        if (e < p.nnz) {
            const int64_t c = (int64_t)p.cols[e0 + e] + p.col_shift;
            const uint32_t w = p.w[e0 + e];
            const bool ok = c >= p.vbase && c < p.vbase + p.n;
            if (!ok) atomicOr(&glob->err, kErrBadCol);
            if (w == 0) atomicOr(&glob->err, kErrZeroWeight);
            ucols[d] = ok ? (int32_t)c : (int32_t)(p.vbase + p.n);
            uw[d] = w;
        } else {
            ucols[d] = (int32_t)(p.vbase + p.n);
            uw[d] = 1u;
        }
    }
}

__global__ void k_set_i64(int64_t* p, int64_t v) { *p = v; }

int64_t pack_tiles(const PackGraph& p) {
    return (p.n + 1 + kPackTile - 1) / kPackTile + (p.nnz + p.pad + kPackTile - 1) / kPackTile;
}

cudaError_t launch_pack(const PackGraph* pg, const int64_t* tstart, int G, int64_t tiles, int64_t* uoff,
                        int32_t* ucols, uint32_t* uw, uint32_t* gid, uint32_t* lid, int64_t n_total,
                        int64_t nnz_total, Globals* glob, cudaStream_t s) {
    if (tiles > 0) {
        note_launch();
        k_pack<<<(unsigned)tiles, 256, 0, s>>>(pg, tstart, G, uoff, ucols, uw, gid, lid, glob);
    }
    note_launch();
    k_set_i64<<<1, 1, 0, s>>>(uoff + n_total, nnz_total);  // closing offset
    return cudaGetLastError();
}

// 2m of every graph: the sum of K over its vertex range (one block per graph).
__global__ void k_graph_two_m(const uint64_t* __restrict__ K, const int64_t* __restrict__ vb,
                              const int64_t* __restrict__ nv, unsigned long long* __restrict__ two_m_g) {
    const int g = blockIdx.x;
    unsigned long long s = 0;
    for (int64_t i = threadIdx.x; i < nv[g]; i += blockDim.x) s += K[vb[g] + i];
    __shared__ unsigned long long part[32];
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < blockDim.x / 32 ? part[threadIdx.x] : 0ull;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) two_m_g[g] = s;
    }
}

cudaError_t launch_graph_two_m(const uint64_t* K, const int64_t* vb, const int64_t* nv, int G,
                               unsigned long long* two_m_g, cudaStream_t s) {
    if (G > 0) {
        note_launch();
        k_graph_two_m<<<G, 256, 0, s>>>(K, vb, nv, two_m_g);
    }
    return cudaGetLastError();
}

// End of a sweep of the union: every graph still moving counts one sweep and
// stops when nobody of it moved, when its summed delta-Q is at most tol, or
// at max_sweeps (the single-graph driver's rule, per graph).  glob->count
// receives the number of graphs still moving.
__global__ void k_batch_converge(int G, const unsigned long long* __restrict__ two_m_g,
                                 const unsigned long long* __restrict__ g_moved,
                                 const unsigned long long* __restrict__ g_gain_lo,
                                 const unsigned long long* __restrict__ g_gain_hi, double tol,
                                 int64_t max_sweeps, uint32_t* __restrict__ gsweeps, uint8_t* __restrict__ gdone,
                                 Globals* glob) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G || gdone[g]) return;
    const uint32_t sw = gsweeps[g] + 1;
    gsweeps[g] = sw;
    bool done = g_moved[g] == 0;
    if (!done) {
        const double gain = (double)g_gain_hi[g] * 18446744073709551616.0 + (double)g_gain_lo[g];
        const double tm = (double)two_m_g[g];
        done = gain / (tm * tm / 2.0) <= tol;
    }
    if ((int64_t)sw >= max_sweeps) done = true;
    if (done) gdone[g] = 1;
    else atomicAdd(&glob->count, 1ull);
}

cudaError_t launch_batch_converge(int G, const unsigned long long* two_m_g, const unsigned long long* g_moved,
                                  const unsigned long long* g_gain_lo, const unsigned long long* g_gain_hi,
                                  double tol, int64_t max_sweeps, uint32_t* gsweeps, uint8_t* gdone, Globals* glob,
                                  cudaStream_t s) {
    if (G > 0) {
        note_launch();
        k_batch_converge<<<(G + 255) / 256, 256, 0, s>>>(G, two_m_g, g_moved, g_gain_lo, g_gain_hi, tol,
                                                         max_sweeps, gsweeps, gdone, glob);
    }
    return cudaGetLastError();
}

// out[g] = x[idx[g]]
__global__ void k_gather_u32(const uint32_t* __restrict__ x, const int64_t* __restrict__ idx, int G,
                             uint32_t* __restrict__ out) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < G) out[g] = x[idx[g]];
}

cudaError_t launch_gather_u32(const uint32_t* x, const int64_t* idx, int G, uint32_t* out, cudaStream_t s) {
    if (G > 0) {
        note_launch();
        k_gather_u32<<<(G + 255) / 256, 256, 0, s>>>(x, idx, G, out);
    }
    return cudaGetLastError();
}

__global__ void k_gather_i64(const int64_t* __restrict__ x, const int64_t* __restrict__ idx, int count,
                             int64_t* __restrict__ out) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < count) out[g] = x[idx[g]];
}

cudaError_t launch_gather_i64(const int64_t* x, const int64_t* idx, int count, int64_t* out, cudaStream_t s) {
    if (count > 0) {
        note_launch();
        k_gather_i64<<<(count + 255) / 256, 256, 0, s>>>(x, idx, count, out);
    }
    return cudaGetLastError();
}

// Final labels of every input vertex: loc[v] = top[v] - cb_g (dense id
// inside its graph) and qlab[v] = vb0_g + loc[v] (the same partition in the
// graph's input id range); padding vertices get qlab[v] = v.
__global__ void k_batch_labels(const uint32_t* __restrict__ top, const uint32_t* __restrict__ gid, int64_t n,
                               int G, const int64_t* __restrict__ vb0, const int64_t* __restrict__ cb,
                               uint32_t* __restrict__ loc, uint32_t* __restrict__ qlab) {
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= n) return;
    const uint32_t g = gid[v];
    if (g < (uint32_t)G) {
        const uint32_t l = (uint32_t)((int64_t)top[v] - cb[g]);
        loc[v] = l;
        qlab[v] = (uint32_t)(vb0[g] + l);
    } else {
        loc[v] = 0;
        qlab[v] = (uint32_t)v;
    }
}

cudaError_t launch_batch_labels(const uint32_t* top, const uint32_t* gid, int64_t n, int G, const int64_t* vb0,
                                const int64_t* cb, uint32_t* loc, uint32_t* qlab, cudaStream_t s) {
    if (n > 0) {
        note_launch();
        k_batch_labels<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(top, gid, n, G, vb0, cb, loc, qlab);
    }
    return cudaGetLastError();
}

// Per-graph modularity parts: sum_c sigma_c over the CSR entries of the
// graph's rows and sum_c Sigma_c^2 over the community ids of its id range.
// Grid (G, slices): block (g, y) takes slice y of graph g's rows, one warp per
// row; acc[g] = {sigma_in, sq_lo, sq_hi} (zero on entry).
__global__ void k_batch_modularity(const int64_t* __restrict__ off, const int32_t* __restrict__ cols,
                                   const uint32_t* __restrict__ w, const uint32_t* __restrict__ labels,
                                   const uint64_t* __restrict__ Sigma, const int64_t* __restrict__ vb,
                                   const int64_t* __restrict__ nv, unsigned long long* __restrict__ acc) {
    const int g = blockIdx.x;
    const int64_t v0 = vb[g], n = nv[g];
    const int64_t r0 = v0 + n * blockIdx.y / gridDim.y, r1 = v0 + n * (blockIdx.y + 1) / gridDim.y;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    unsigned long long sig = 0;
    for (int64_t r = r0 + warp; r < r1; r += nwarps) {
        const uint32_t lr = labels[r];
        const int64_t a = off[r], b = off[r + 1];
        for (int64_t e = a + lane; e < b; e += 32)
            if (labels[cols[e]] == lr) sig += w[e];
    }
    u128 sq = 0;
    for (int64_t c = r0 + threadIdx.x; c < r1; c += blockDim.x) {
        const unsigned long long x = Sigma[c];
        sq += (u128)x * (u128)x;
    }
    __shared__ unsigned long long ps[256], pl[256], ph[256];
    ps[threadIdx.x] = sig;
    pl[threadIdx.x] = (unsigned long long)sq;
    ph[threadIdx.x] = (unsigned long long)(sq >> 64);
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long s1 = 0;
        u128 s2 = 0;
        for (int t = 0; t < (int)blockDim.x; ++t) {
            s1 += ps[t];
            s2 += ((u128)ph[t] << 64) | (u128)pl[t];
        }
        if (s1) atomicAdd(&acc[3 * g], s1);
        const unsigned long long lo = (unsigned long long)s2, hi = (unsigned long long)(s2 >> 64);
        const unsigned long long old = atomicAdd(&acc[3 * g + 1], lo);
        const unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
        if (hi + carry) atomicAdd(&acc[3 * g + 2], hi + carry);
    }
}

cudaError_t launch_batch_modularity(const int64_t* off, const int32_t* cols, const uint32_t* w,
                                    const uint32_t* labels, const uint64_t* Sigma, const int64_t* vb,
                                    const int64_t* nv, int G, unsigned long long* acc, cudaStream_t s) {
    if (G > 0) {
        note_launch();
        k_batch_modularity<<<dim3(G, 16), 256, 0, s>>>(off, cols, w, labels, Sigma, vb, nv, acc);
    }
    return cudaGetLastError();
}

}  // namespace cdk
