// Per-pass kernels around the local-moving sweep: weighted degrees and
// community totals (Section 3), degree bucketing, the dispatch of the MG
// sweep by sketch size, and the commit of moves into Sigma and sizes.
#include <cstdio>

#include "cd_internal.cuh"
#include "csr_walk.cuh"

namespace cdk {

// ---------------------------------------------------------------------------
// K_i = sum of w over row i (Section 3), over the whole CSR (the modularity
// path; the sweeps sum the rows by bucket, k_row_sums below).
// ---------------------------------------------------------------------------
constexpr int64_t kDegTile = 4096;  // CSR entries per warp

// K_i = sum of w over row i: one warp per 4096-entry tile walks the entries
// with their rows (csr_walk.cuh); each step's lanes of one row are summed by a
// segmented shuffle reduction and the row's first lane adds the sum to K.
__global__ void k_degrees(const int64_t* __restrict__ off, const uint32_t* __restrict__ w,
                          int64_t n, int64_t nnz, unsigned long long* __restrict__ K, Globals* glob) {
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t e0 = warp * kDegTile;
    if (e0 >= nnz) return;  // the whole warp
    const int64_t e1 = e0 + kDegTile < nnz ? e0 + kDegTile : nnz;
    const int lane = threadIdx.x & 31;
    bool zero = false;
    const bool ok = warp_walk<true>(off, n, e0, e1, [&](int64_t e, int64_t r, bool valid) {
        unsigned long long v = 0;
        if (valid) {
            const uint32_t x = __ldg(w + e);
            zero |= x == 0;
            v = x;
        }
        const int64_t row = valid ? r : -1;
        // lanes of one row are consecutive: sum each lane's run to the right
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long v2 = __shfl_down_sync(0xffffffffu, v, o);
            const int64_t r2 = __shfl_down_sync(0xffffffffu, row, o);
            if (lane + o < 32 && r2 == row) v += v2;
        }
        const int64_t prev = __shfl_up_sync(0xffffffffu, row, 1);
        if (valid && (lane == 0 || prev != row) && v) atomicAdd(&K[row], v);
    });
    if (lane == 0 && !ok) atomicOr(&glob->err, kErrBadOffsets);
    if (zero) atomicOr(&glob->err, kErrZeroWeight);
}

// Offsets in order, starting at 0 and ending at nnz (kErrBadOffsets).
__global__ void k_check_offsets(const int64_t* __restrict__ off, int64_t n, int64_t nnz, Globals* glob) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t a = off[i], b = off[i + 1];
    if (b < a || (i == 0 && a != 0) || (i == n - 1 && b != nnz)) atomicOr(&glob->err, kErrBadOffsets);
}

cudaError_t launch_degrees(const int64_t* off, const uint32_t* w, int64_t n, int64_t nnz,
                           uint64_t* K, Globals* glob, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(K, 0, sizeof(uint64_t) * (size_t)(n > 0 ? n : 1), s);
    if (e != cudaSuccess) return e;
    if (n > 0) {
        note_launch();
        k_check_offsets<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(off, n, nnz, glob);
    }
    if (nnz == 0) return cudaGetLastError();
    const int64_t warps = (nnz + kDegTile - 1) / kDegTile;
    note_launch();
    k_degrees<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(off, w, n, nnz, (unsigned long long*)K, glob);
    return cudaGetLastError();
}

// Sigma_c and |c| from labels; 2m and max K_i into the globals.
__global__ void k_totals(const uint32_t* __restrict__ labels, const unsigned long long* __restrict__ K,
                         int64_t n, unsigned long long* __restrict__ Sigma, uint32_t* __restrict__ size,
                         Globals* glob) {
    // a grid of a few blocks per SM strides over the vertices, so that the
    // two global atomics per block (2m and max K_i, one address each) stay
    // few: one block per 256 vertices made them serialise on those
    // addresses
    unsigned long long s = 0, m = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = K[i];
        s += k;
        m = k > m ? k : m;
        if (!labels) {
            // singleton communities (labels = vertex ids): plain stores
            Sigma[i] = k;
            size[i] = 1u;
        } else {
            uint32_t c = labels[i];
            if ((int64_t)c < n) {
                if (k) atomicAdd(&Sigma[c], k);
                atomicAdd(&size[c], 1u);
            } else {
                atomicOr(&glob->err, kErrBadLabel);
            }
        }
    }
    // block reduction, then one atomic per block
    __shared__ unsigned long long ss[8], sm[8];
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, o);
        unsigned long long mo = __shfl_down_sync(0xffffffffu, m, o);
        m = mo > m ? mo : m;
    }
    if ((threadIdx.x & 31) == 0) {
        ss[threadIdx.x >> 5] = s;
        sm[threadIdx.x >> 5] = m;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) {
            s += ss[q];
            m = sm[q] > m ? sm[q] : m;
        }
        if (s) atomicAdd(&glob->two_m, s);
        if (m) atomicMax(&glob->max_k, m);
    }
}

// K_i = sum of w over row i for the rows listed in the bucket table.  Rows of
// a bucket with L <= 32 streams are summed by L threads of a warp (one thread
// per row for the short rows), rows of the wider buckets by a whole block;
// 16-byte loads, four of them in flight per thread (the rows are otherwise
// latency-bound), then a shuffle (and shared-memory) reduction.
// Each row's sum is written once; rows of length 0 are not listed and keep
// K = 0.
__device__ __forceinline__ uint4 load_w4(const uint32_t* __restrict__ w, int64_t ch, int64_t nnz) {
    const int64_t e0 = ch * 4;
    if (e0 + 4 <= nnz) return __ldg(reinterpret_cast<const uint4*>(w) + ch);
    uint4 v;
    v.x = e0 < nnz ? w[e0] : 0u;
    v.y = e0 + 1 < nnz ? w[e0 + 1] : 0u;
    v.z = e0 + 2 < nnz ? w[e0 + 2] : 0u;
    v.w = e0 + 3 < nnz ? w[e0 + 3] : 0u;
    return v;
}

__device__ __forceinline__ void add_w4(uint4 v, int64_t ch, int64_t start, int64_t end, unsigned long long& sum,
                                       bool& zero) {
    const int64_t e0 = ch * 4;
    const uint32_t xs[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const bool in = e0 + u >= start && e0 + u < end;
        zero |= in && xs[u] == 0;
        sum += in ? xs[u] : 0u;
    }
}

__device__ __forceinline__ int row_sum_lanes(int lanes) { return lanes <= 32 ? lanes : kBlock; }

__global__ void __launch_bounds__(256) k_row_sums(const int64_t* __restrict__ off, const uint32_t* __restrict__ w,
                                                  int64_t nnz, const uint32_t* __restrict__ verts, BucketTable bt,
                                                  unsigned long long* __restrict__ K, Globals* glob) {
    const int64_t blk = blockIdx.x;
    int b = 0;
#pragma unroll
    for (int q = 1; q < CD_MAX_BUCKETS; ++q)
        if (q < bt.nb && blk >= bt.bbegin[q]) b = q;
    const int L = row_sum_lanes(bt.lanes[b]);
    const int64_t vi = bt.vbegin[b] + (blk - bt.bbegin[b]) * (kBlock / L) + threadIdx.x / L;
    const bool valid = vi < bt.vbegin[b + 1];
    const int lane = threadIdx.x % L;
    unsigned long long sum = 0;
    bool zero = false;
    uint32_t i = 0;
    if (valid) {
        i = verts[vi];
        const int64_t start = off[i], end = off[i + 1];
        const int64_t c0 = start >> 2, c1 = (end + 3) >> 2;
        // four loads in flight per trip, each guarded (a lane's last trip is
        // usually partial)
        for (int64_t ch = c0 + lane; ch < c1; ch += 4 * (int64_t)L) {
            uint4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t cu = ch + u * (int64_t)L;
                v[u] = cu < c1 ? load_w4(w, cu, nnz) : make_uint4(0u, 0u, 0u, 0u);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) add_w4(v[u], ch + u * (int64_t)L, start, end, sum, zero);
        }
    }
    if (L > 1) {
        const int G = L < 32 ? L : 32;
        const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
        for (int o = G / 2; o >= 1; o >>= 1) sum += __shfl_down_sync(gmask, sum, o, G);
    }
    if (L == kBlock) {
        __shared__ unsigned long long part[kBlock / 32];
        if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = sum;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int q = 1; q < kBlock / 32; ++q) sum += part[q];
        }
    }
    if (valid && lane == 0) K[i] = sum;
    if (zero) atomicOr(&glob->err, kErrZeroWeight);
}

cudaError_t launch_row_sums(const int64_t* off, const uint32_t* w, int64_t n, int64_t nnz, const uint32_t* verts,
                            const BucketTable& bt_in, uint64_t* K, Globals* glob, cudaStream_t s) {
    // geometry: the sweep's L <= 32 threads per row, or a block per row for
    // wider buckets (more threads per row for the short-row buckets measured
    // slower: 1.573 against 1.517 ms per R-MAT 22 sweep step)
    BucketTable bt = bt_in;
    int64_t blk = 0;
    for (int b = 0; b < bt.nb; ++b) {
        bt.bbegin[b] = blk;
        const int L = bt.lanes[b] <= 32 ? bt.lanes[b] : kBlock;
        const int64_t nv = bt.vbegin[b + 1] - bt.vbegin[b];
        blk += (nv + (kBlock / L) - 1) / (kBlock / L);
    }
    bt.bbegin[bt.nb] = blk;
    (void)n;
    if (blk == 0) return cudaSuccess;
    note_launch();
    k_row_sums<<<(unsigned)blk, kBlock, 0, s>>>(off, w, nnz, verts, bt, (unsigned long long*)K, glob);
    return cudaGetLastError();
}

cudaError_t launch_totals(const uint32_t* labels, const uint64_t* K, int64_t n, uint64_t* Sigma,
                          uint32_t* size, Globals* glob, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    if (labels) {  // null labels: singletons, every entry is stored
        e = cudaMemsetAsync(Sigma, 0, sizeof(uint64_t) * (size_t)(n > 0 ? n : 1), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(size, 0, sizeof(uint32_t) * (size_t)(n > 0 ? n : 1), s);
    }
    if (e != cudaSuccess || n == 0) return e;
    int dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int64_t want = (n + 255) / 256, cap = (int64_t)sms * 8;
    note_launch();
    k_totals<<<(unsigned)(want < cap ? want : cap), 256, 0, s>>>(labels, (const unsigned long long*)K, n,
                                                                  (unsigned long long*)Sigma, size, glob);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Degree bucketing.  Rows of length 0 never move (their label is copied);
// the others are listed by (colour class, bucket) in ascending vertex id, so
// that neighbouring groups of a warp get rows of similar length and every
// colour class (one sub-sweep of the driver) is a contiguous range.
// ---------------------------------------------------------------------------
constexpr int kBucketTile = 2048;  // vertices per block, 8 rounds of 256
constexpr int kMaxKeys = 256;      // colours x buckets

__device__ __forceinline__ int bucket_of(int64_t deg, const BucketTable& bt) {
    if (deg == 0) return -1;
#pragma unroll
    for (int b = 0; b < CD_MAX_BUCKETS; ++b)
        if (b < bt.nb && deg <= bt.deg_max[b]) return b;
    return bt.nb - 1;
}

__device__ __forceinline__ int key_of(const int64_t* __restrict__ off, int64_t v, int64_t n, int64_t nnz,
                                      const BucketTable& bt, int colors, const uint32_t* __restrict__ cid,
                                      Globals* glob) {
    int64_t o0 = off[v], o1 = off[v + 1];
    bool bad = o1 < o0 || o0 < 0 || o1 > nnz || (v == 0 && o0 != 0) || (v == n - 1 && o1 != nnz);
    if (bad) {
        if (glob) atomicOr(&glob->err, kErrBadOffsets);
        return -1;
    }
    int b = bucket_of(o1 - o0, bt);
    if (b < 0) return -1;
    return (int)color_of(cid ? cid[v] : (uint32_t)v, colors) * bt.nb + b;
}

int64_t bucket_tiles(int64_t n) { return (n + kBucketTile - 1) / kBucketTile; }

// Also sets glob->pad when some label differs from its vertex id (labels
// not null), so that the caller can take the singleton path of the totals.
__global__ void k_bucket_count(const int64_t* __restrict__ off, int64_t n, int64_t nnz, BucketTable bt, int colors,
                               const uint32_t* __restrict__ cid, const uint32_t* __restrict__ labels,
                               uint32_t* __restrict__ tile_counts, int64_t ntiles, Globals* glob) {
    __shared__ uint32_t cnt[kMaxKeys];
    const int nkeys = colors * bt.nb;
    cnt[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kBucketTile;
    bool other = false;
    for (int r = 0; r < kBucketTile / 256; ++r) {
        int64_t v = base + r * 256 + threadIdx.x;
        if (v < n) {
            int key = key_of(off, v, n, nnz, bt, colors, cid, glob);
            if (key >= 0) atomicAdd(&cnt[key], 1u);
            if (labels && labels[v] != (uint32_t)v) other = true;
        }
    }
    if (__syncthreads_or(other) && threadIdx.x == 0) atomicOr(&glob->pad, 1u);
    if ((int)threadIdx.x < nkeys) tile_counts[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

// Single-block exclusive scan of a moderate array (tile counts); also writes
// the total to *total.
__global__ void k_scan_small(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int64_t m,
                             unsigned long long* total) {
    __shared__ unsigned long long part[1024];
    int64_t per = (m + blockDim.x - 1) / blockDim.x;
    int64_t a = threadIdx.x * per, b = a + per < m ? a + per : m;
    unsigned long long s = 0;
    for (int64_t x = a; x < b; ++x) s += in[x];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
        unsigned long long v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0ull;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    unsigned long long run = part[threadIdx.x] - s;
    for (int64_t x = a; x < b; ++x) {
        uint32_t v = in[x];
        out[x] = (uint32_t)run;
        run += v;
    }
    if (threadIdx.x == blockDim.x - 1 && total) *total = part[threadIdx.x];
}

__global__ void k_bucket_scatter(const int64_t* __restrict__ off, int64_t n, int64_t nnz, BucketTable bt,
                                 int colors, const uint32_t* __restrict__ cid,
                                 const uint32_t* __restrict__ tile_offsets, int64_t ntiles,
                                 uint32_t* __restrict__ verts, const uint32_t* __restrict__ labels_in,
                                 uint32_t* __restrict__ labels_out) {
    __shared__ uint32_t wc[8][kMaxKeys];
    __shared__ uint32_t run[kMaxKeys];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    run[threadIdx.x] = 0;
    int64_t base = (int64_t)blockIdx.x * kBucketTile;
    for (int r = 0; r < kBucketTile / 256; ++r) {
#pragma unroll
        for (int q = 0; q < 8; ++q) wc[q][threadIdx.x] = 0;
        __syncthreads();
        int64_t v = base + r * 256 + threadIdx.x;
        int key = -1;
        if (v < n) {
            key = key_of(off, v, n, nnz, bt, colors, cid, nullptr);
            if (key < 0 && labels_out) labels_out[v] = labels_in[v];
        }
        unsigned peers = __match_any_sync(0xffffffffu, key);
        unsigned rank = __popc(peers & ((1u << lane) - 1u));
        if (key >= 0 && rank == 0) wc[warp][key] = __popc(peers);
        __syncthreads();
        if (key >= 0) {
            uint32_t pos = tile_offsets[(int64_t)key * ntiles + blockIdx.x] + run[key] + rank;
            for (int q = 0; q < warp; ++q) pos += wc[q][key];
            verts[pos] = (uint32_t)v;
        }
        __syncthreads();
        uint32_t t = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) t += wc[q][threadIdx.x];
        run[threadIdx.x] += t;
        __syncthreads();
    }
}

__global__ void k_bucket_starts(const uint32_t* __restrict__ tile_offsets, int64_t ntiles, int nkeys,
                                const unsigned long long* __restrict__ total, int64_t* __restrict__ starts) {
    for (int b = threadIdx.x; b <= nkeys; b += blockDim.x) {
        if (b < nkeys) starts[b] = tile_offsets[(int64_t)b * ntiles];
        else starts[nkeys] = (int64_t)*total;
    }
}

cudaError_t launch_bucket(const int64_t* off, int64_t n, int64_t nnz, const BucketTable& bt, int colors,
                          const uint32_t* cid, uint32_t* tile_counts, uint32_t* tile_offsets, int64_t* bucket_starts,
                          uint32_t* verts, const uint32_t* labels_in, uint32_t* labels_out,
                          Globals* glob, cudaStream_t s, unsigned long long* scan_scratch) {
    const int nkeys = colors * bt.nb;
    if (nkeys > kMaxKeys) return cudaErrorInvalidValue;
    if (n == 0) return cudaMemsetAsync(bucket_starts, 0, sizeof(int64_t) * (nkeys + 1), s);
    int64_t ntiles = bucket_tiles(n);
    note_launch();
    k_bucket_count<<<(unsigned)ntiles, 256, 0, s>>>(off, n, nnz, bt, colors, cid, labels_in, tile_counts, ntiles,
                                                     glob);
    const int64_t m = ntiles * nkeys;
    if (scan_scratch && m > 4096) {
        // larger tables: the tiled scan (one block took 24 us at 28K entries)
        cudaError_t e = launch_exclusive_scan_u32(tile_counts, tile_offsets, m, scan_scratch, &glob->count, s);
        if (e != cudaSuccess) return e;
    } else {
        note_launch();
        k_scan_small<<<1, 1024, 0, s>>>(tile_counts, tile_offsets, m, &glob->count);
    }
    note_launch();
    k_bucket_scatter<<<(unsigned)ntiles, 256, 0, s>>>(off, n, nnz, bt, colors, cid, tile_offsets, ntiles, verts,
                                                      labels_in, labels_out);
    note_launch();
    k_bucket_starts<<<1, 256, 0, s>>>(tile_offsets, ntiles, nkeys, &glob->count, bucket_starts);
    return cudaGetLastError();
}

template <int K>
cudaError_t launch_k(const SweepArgs& a, bool wide, int64_t nblocks, cudaStream_t s);
extern template cudaError_t launch_k<1>(const SweepArgs&, bool, int64_t, cudaStream_t);
extern template cudaError_t launch_k<2>(const SweepArgs&, bool, int64_t, cudaStream_t);
extern template cudaError_t launch_k<4>(const SweepArgs&, bool, int64_t, cudaStream_t);
extern template cudaError_t launch_k<8>(const SweepArgs&, bool, int64_t, cudaStream_t);
extern template cudaError_t launch_k<16>(const SweepArgs&, bool, int64_t, cudaStream_t);
extern template cudaError_t launch_k<32>(const SweepArgs&, bool, int64_t, cudaStream_t);
extern template cudaError_t launch_k<64>(const SweepArgs&, bool, int64_t, cudaStream_t);
template <int K>
cudaError_t launch_agg_k(const AggArgs& g, bool wide, int64_t nblocks, cudaStream_t s);
extern template cudaError_t launch_agg_k<1>(const AggArgs&, bool, int64_t, cudaStream_t);
extern template cudaError_t launch_agg_k<2>(const AggArgs&, bool, int64_t, cudaStream_t);
extern template cudaError_t launch_agg_k<4>(const AggArgs&, bool, int64_t, cudaStream_t);
extern template cudaError_t launch_agg_k<8>(const AggArgs&, bool, int64_t, cudaStream_t);
extern template cudaError_t launch_agg_k<16>(const AggArgs&, bool, int64_t, cudaStream_t);

cudaError_t launch_agg_mg(const AggArgs& g, int k, bool wide, int64_t nblocks, cudaStream_t s) {
    switch (k) {
        case 1: return launch_agg_k<1>(g, wide, nblocks, s);
        case 2: return launch_agg_k<2>(g, wide, nblocks, s);
        case 4: return launch_agg_k<4>(g, wide, nblocks, s);
        case 8: return launch_agg_k<8>(g, wide, nblocks, s);
        case 16: return launch_agg_k<16>(g, wide, nblocks, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_sweep_mg(const SweepArgs& a, int k, bool wide, int64_t nblocks, cudaStream_t s) {
    if (nblocks == 0) return cudaSuccess;
    // a compacted list needs at most its full-list block count, and a few
    // resident waves stride over it
    if (a.dr && nblocks > 152 * 8) nblocks = 152 * 8;
    if (k >= 32)  // these sketch sizes merge inside one warp
        for (int b = 0; b < a.bt.nb; ++b)
            if (a.bt.lanes[b] > 32) return cudaErrorInvalidValue;
    switch (k) {
        case 1: return launch_k<1>(a, wide, nblocks, s);
        case 2: return launch_k<2>(a, wide, nblocks, s);
        case 4: return launch_k<4>(a, wide, nblocks, s);
        case 8: return launch_k<8>(a, wide, nblocks, s);
        case 16: return launch_k<16>(a, wide, nblocks, s);
        case 32: return launch_k<32>(a, wide, nblocks, s);
        case 64: return launch_k<64>(a, wide, nblocks, s);
        default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------------------
// Compaction of the bucketed vertex list to the deciding vertices (skip
// sweeps): flags, exclusive scan, scatter, and per colour class the new
// (bucket range, block range) table, all on the device.
// ---------------------------------------------------------------------------
__global__ void k_active_flags(const uint32_t* __restrict__ verts, int64_t m, const uint8_t* __restrict__ active,
                               uint32_t* __restrict__ flags) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j < m) flags[j] = active[verts[j]] ? 1u : 0u;
}

__global__ void k_active_scatter(const uint32_t* __restrict__ verts, int64_t m, const uint32_t* __restrict__ flags,
                                 const uint32_t* __restrict__ pos, uint32_t* __restrict__ cverts) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j < m && flags[j]) cverts[pos[j]] = verts[j];
}

__global__ void k_active_ranges(const int64_t* __restrict__ starts, int64_t m, const uint32_t* __restrict__ pos,
                                const unsigned long long* __restrict__ total, BucketTable bt, int colors,
                                DevRanges* __restrict__ dr) {
    const int c = threadIdx.x;
    if (c >= colors) return;
    auto at = [&](int64_t j) -> int64_t { return j < m ? (int64_t)pos[j] : (int64_t)*total; };
    int64_t blk = 0;
    for (int b = 0; b < bt.nb; ++b) {
        const int64_t v0 = at(starts[(int64_t)c * bt.nb + b]), v1 = at(starts[(int64_t)c * bt.nb + b + 1]);
        dr[c].vbegin[b] = v0;
        dr[c].bbegin[b] = blk;
        const int L = threads_per_row(bt, b);
        const int vpb = L >= kBlock ? 1 : kBlock / L;
        blk += (v1 - v0 + vpb - 1) / vpb;
    }
    dr[c].vbegin[bt.nb] = at(starts[(int64_t)c * bt.nb + bt.nb]);
    dr[c].bbegin[bt.nb] = blk;
}

cudaError_t launch_compact(const uint32_t* verts, int64_t m, const uint8_t* active, const int64_t* starts,
                           const BucketTable& bt, int colors, uint32_t* flags, uint32_t* pos,
                           unsigned long long* tiles, unsigned long long* total, uint32_t* cverts, DevRanges* dr,
                           cudaStream_t s) {
    if (colors < 1 || colors > 32) return cudaErrorInvalidValue;
    if (m > 0) {
        const unsigned g = (unsigned)((m + 255) / 256);
        note_launch();
        k_active_flags<<<g, 256, 0, s>>>(verts, m, active, flags);
        cudaError_t e = launch_exclusive_scan_u32(flags, pos, m, tiles, total, s);
        if (e != cudaSuccess) return e;
        note_launch();
        k_active_scatter<<<g, 256, 0, s>>>(verts, m, flags, pos, cverts);
    } else {
        cudaError_t e = cudaMemsetAsync(total, 0, sizeof(unsigned long long), s);
        if (e != cudaSuccess) return e;
    }
    note_launch();
    k_active_ranges<<<1, 32, 0, s>>>(starts, m, pos, total, bt, colors, dr);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Commit: apply the moves of the last (sub-)sweep to Sigma and sizes (after
// every decision of it has been taken from its start state), and copy the
// movers' new labels into the running labels for the next sub-sweep.  Each
// mover reads its old label and then overwrites it itself, so one kernel
// does both.
// ---------------------------------------------------------------------------
__global__ void k_commit(const uint32_t* __restrict__ movers, uint32_t* __restrict__ labels,
                         const uint32_t* __restrict__ labels_out, const unsigned long long* __restrict__ K,
                         unsigned long long* __restrict__ Sigma, uint32_t* __restrict__ size,
                         const Globals* __restrict__ glob) {
    const unsigned long long cnt = glob->moved;
    for (unsigned long long t = glob->mark + blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < cnt;
         t += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t i = movers[t];
        const uint32_t d = labels[i], c = labels_out[i];
        const unsigned long long k = K[i];
        atomicAdd(&Sigma[c], k);
        atomicAdd(&Sigma[d], ~k + 1ull);
        atomicAdd(&size[c], 1u);
        atomicSub(&size[d], 1u);
        labels[i] = c;
    }
}

cudaError_t launch_commit(const uint32_t* movers, uint32_t* labels, const uint32_t* labels_out, const uint64_t* K,
                          int64_t n, uint64_t* Sigma, uint32_t* size, Globals* glob, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    note_launch();
    k_commit<<<(unsigned)blocks, 256, 0, s>>>(movers, labels, labels_out, (const unsigned long long*)K,
                                              (unsigned long long*)Sigma, size, glob);
    return cudaGetLastError();
}

}  // namespace cdk
