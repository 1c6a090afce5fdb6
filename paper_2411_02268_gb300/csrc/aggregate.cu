// Aggregation phase (Section 3.3 and Section 4.1, "aggregation phase"):
// communities are renumbered densely by a prefix scan over the ids in use,
// and the super-vertex graph is built by sorting the CSR entries by
// (community of the row, community of the column) with a stable LSD radix
// sort and summing equal keys.  Entry (i, j, w) of G contributes w to entry
// (C'_i, C'_j) of G', so the self-loop of c' holds sigma_c (both directions of
// every internal edge) and every weighted degree and 2m are preserved.
//
// The paper builds each super-vertex row with one more MG sketch and no
// second pass (approximate weights); this is the exact construction.
#include <utility>

#include "cd_internal.cuh"

namespace cdk {

// ---- renumbering --------------------------------------------------------------

__global__ void k_mark_used(const uint32_t* __restrict__ labels, int64_t n, uint32_t* __restrict__ used,
                            Globals* glob) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t c = labels[i];
    if ((int64_t)c < n) used[c] = 1u;
    else atomicOr(&glob->err, kErrBadLabel);
}

__global__ void k_apply_ids(const uint32_t* __restrict__ labels, int64_t n, const uint32_t* __restrict__ newid,
                            uint32_t* __restrict__ dense) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t c = labels[i];
    dense[i] = (int64_t)c < n ? newid[c] : 0u;
}

// dense[i] = rank of labels[i] among the ids in use; *count_dev = number of ids.
cudaError_t launch_renumber(const uint32_t* labels, int64_t n, uint32_t* dense, uint32_t* scratch_n,
                            unsigned long long* tile_scratch, unsigned long long* count_dev, Globals* glob,
                            cudaStream_t s) {
    if (n == 0) return cudaMemsetAsync(count_dev, 0, sizeof(unsigned long long), s);
    cudaError_t e = cudaMemsetAsync(scratch_n, 0, sizeof(uint32_t) * n, s);
    if (e != cudaSuccess) return e;
    unsigned nb = (unsigned)((n + 255) / 256);
    k_mark_used<<<nb, 256, 0, s>>>(labels, n, scratch_n, glob);
    e = launch_exclusive_scan_u32(scratch_n, scratch_n, n, tile_scratch, count_dev, s);
    if (e != cudaSuccess) return e;
    k_apply_ids<<<nb, 256, 0, s>>>(labels, n, scratch_n, dense);
    return cudaGetLastError();
}

// map[i] = dense[map[i]] (composition of the per-pass label maps)
__global__ void k_compose(uint32_t* __restrict__ top, int64_t n0, const uint32_t* __restrict__ dense) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n0) top[i] = dense[top[i]];
}

cudaError_t launch_compose(uint32_t* top, int64_t n0, const uint32_t* dense, cudaStream_t s) {
    if (n0 == 0) return cudaSuccess;
    k_compose<<<(unsigned)((n0 + 255) / 256), 256, 0, s>>>(top, n0, dense);
    return cudaGetLastError();
}

__global__ void k_iota(uint32_t* __restrict__ x, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) x[i] = (uint32_t)i;
}

cudaError_t launch_iota(uint32_t* x, int64_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_iota<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, n);
    return cudaGetLastError();
}

// next_init[sub[v]] = bound[v]: the community of every sub-community (all
// members of a sub-community share one bound, so the writes agree).
__global__ void k_scatter_bound(const uint32_t* __restrict__ sub, const uint32_t* __restrict__ bound, int64_t n,
                                uint32_t* __restrict__ next_init) {
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v < n) next_init[sub[v]] = bound[v];
}

cudaError_t launch_scatter_bound(const uint32_t* sub, const uint32_t* bound, int64_t n, uint32_t* next_init,
                                 cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_scatter_bound<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(sub, bound, n, next_init);
    return cudaGetLastError();
}

// ---- super-vertex graph ----------------------------------------------------------

constexpr int kExpandChunk = 64;

// src[e] = dense[row(e)], dst[e] = dense[cols[e]]; rows found by binary search
// at the start of each 64-entry chunk.
__global__ void k_expand(const int64_t* __restrict__ off, const int32_t* __restrict__ cols, int64_t n,
                         int64_t nnz, const uint32_t* __restrict__ dense, uint32_t* __restrict__ src,
                         uint32_t* __restrict__ dst) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t e0 = t * kExpandChunk;
    if (e0 >= nnz) return;
    int64_t e1 = e0 + kExpandChunk < nnz ? e0 + kExpandChunk : nnz;
    int64_t lo = 0, hi = n;
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) >> 1;
        if (off[mid] <= e0) lo = mid; else hi = mid;
    }
    int64_t r = lo, rend = off[r + 1];
    uint32_t cr = dense[r];
    for (int64_t e = e0; e < e1; ++e) {
        while (e >= rend && r + 1 < n) {
            ++r;
            rend = off[r + 1];
            cr = dense[r];
        }
        uint32_t j = (uint32_t)cols[e];
        src[e] = cr;
        dst[e] = j < (uint32_t)n ? dense[j] : 0u;
    }
}

// Stable LSD radix sort pass on 8-bit digits of key (shift), carrying two
// payload arrays.  Tiles of 8192 entries; digit counts per tile are scanned in
// digit-major order so that equal digits keep their tile order.
constexpr int kRadixThreads = 256;
constexpr int kRadixRounds = 32;
constexpr int kRadixTile = kRadixThreads * kRadixRounds;

int64_t radix_tiles(int64_t n) { return (n + kRadixTile - 1) / kRadixTile; }

__global__ void k_radix_hist(const uint32_t* __restrict__ key, int64_t n, int shift,
                             uint32_t* __restrict__ hist, int64_t ntiles) {
    __shared__ uint32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kRadixTile;
    for (int r = 0; r < kRadixRounds; ++r) {
        int64_t i = base + (int64_t)r * kRadixThreads + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(key[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void k_radix_scatter(const uint32_t* __restrict__ key, const uint32_t* __restrict__ p1,
                                const uint32_t* __restrict__ p2, int64_t n, int shift,
                                const uint32_t* __restrict__ offs, int64_t ntiles, uint32_t* __restrict__ key_o,
                                uint32_t* __restrict__ p1_o, uint32_t* __restrict__ p2_o) {
    __shared__ uint32_t wc[8][256];
    __shared__ uint32_t run[256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    run[threadIdx.x] = 0;
    int64_t base = (int64_t)blockIdx.x * kRadixTile;
    for (int r = 0; r < kRadixRounds; ++r) {
#pragma unroll
        for (int q = 0; q < 8; ++q) wc[q][threadIdx.x] = 0;
        __syncthreads();
        int64_t i = base + (int64_t)r * kRadixThreads + threadIdx.x;
        bool ok = i < n;
        uint32_t k = ok ? key[i] : 0u;
        int dgt = ok ? (int)((k >> shift) & 255u) : -1;
        unsigned peers = __match_any_sync(0xffffffffu, dgt);
        unsigned rank = __popc(peers & ((1u << lane) - 1u));
        if (ok && rank == 0) wc[warp][dgt] = __popc(peers);
        __syncthreads();
        if (ok) {
            uint32_t pos = offs[(int64_t)dgt * ntiles + blockIdx.x] + run[dgt] + rank;
            for (int q = 0; q < warp; ++q) pos += wc[q][dgt];
            key_o[pos] = k;
            p1_o[pos] = p1[i];
            p2_o[pos] = p2[i];
        }
        __syncthreads();
        uint32_t t = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) t += wc[q][threadIdx.x];
        run[threadIdx.x] += t;
        __syncthreads();
    }
}

// heads[e] = 1 where (src, dst) differs from entry e-1.
__global__ void k_heads(const uint32_t* __restrict__ src, const uint32_t* __restrict__ dst, int64_t n,
                        uint32_t* __restrict__ heads) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    heads[e] = (e == 0 || src[e] != src[e - 1] || dst[e] != dst[e - 1]) ? 1u : 0u;
}

// uidx = exclusive scan of heads; unique entry u = uidx[e] for its first e.
__global__ void k_segsum(const uint32_t* __restrict__ src, const uint32_t* __restrict__ dst,
                         const uint32_t* __restrict__ w, const uint32_t* __restrict__ heads,
                         const uint32_t* __restrict__ uidx, int64_t n, int32_t* __restrict__ cols_out,
                         unsigned long long* __restrict__ wsum, uint32_t* __restrict__ rowcnt) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    uint32_t u = uidx[e] + heads[e] - 1u;  // index of this entry's unique key
    atomicAdd(&wsum[u], (unsigned long long)w[e]);
    if (heads[e]) {
        cols_out[u] = (int32_t)dst[e];
        atomicAdd(&rowcnt[src[e]], 1u);
    }
}

__global__ void k_narrow(const unsigned long long* __restrict__ wsum, int64_t m, uint32_t* __restrict__ w_out,
                         Globals* glob) {
    int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (u >= m) return;
    unsigned long long v = wsum[u];
    if (v >> 32) atomicOr(&glob->err, kErrWeightOverflow);
    w_out[u] = (uint32_t)v;
}

int bits_for(int64_t nc) {
    int b = 0;
    while (b < 32 && ((int64_t)1 << b) < nc) ++b;
    return b;
}

// Sorts (src, dst, w) by (src, dst).  On return the sorted arrays are in
// (src, dst, w) (the buffers may have been swapped with the *2 ones).
cudaError_t radix_sort_pairs(AggScratch& a, int64_t nnz, int64_t nc, Globals* glob, cudaStream_t s) {
    int bits = bits_for(nc);
    int64_t nt = radix_tiles(nnz);
    int64_t hn = nt * 256;
    // by dst, then by src: key passes
    for (int which = 0; which < 2; ++which) {
        for (int shift = 0; shift < bits; shift += 8) {
            uint32_t* key = which == 0 ? a.dst : a.src;
            uint32_t* p1 = which == 0 ? a.src : a.dst;
            uint32_t* key_o = which == 0 ? a.dst2 : a.src2;
            uint32_t* p1_o = which == 0 ? a.src2 : a.dst2;
            k_radix_hist<<<(unsigned)nt, kRadixThreads, 0, s>>>(key, nnz, shift, a.hist, nt);
            cudaError_t e = launch_exclusive_scan_u32(a.hist, a.hist, hn, a.tiles, &glob->count, s);
            if (e != cudaSuccess) return e;
            k_radix_scatter<<<(unsigned)nt, kRadixThreads, 0, s>>>(key, p1, a.w, nnz, shift, a.hist, nt, key_o,
                                                                    p1_o, a.w2);
            std::swap(a.src, a.src2);
            std::swap(a.dst, a.dst2);
            std::swap(a.w, a.w2);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_expand(const int64_t* off, const int32_t* cols, int64_t n, int64_t nnz, const uint32_t* dense,
                          uint32_t* src, uint32_t* dst, cudaStream_t s) {
    if (nnz == 0) return cudaSuccess;
    int64_t threads = (nnz + kExpandChunk - 1) / kExpandChunk;
    k_expand<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(off, cols, n, nnz, dense, src, dst);
    return cudaGetLastError();
}

cudaError_t launch_heads(const AggScratch& a, int64_t nnz, cudaStream_t s) {
    if (nnz == 0) return cudaSuccess;
    k_heads<<<(unsigned)((nnz + 255) / 256), 256, 0, s>>>(a.src, a.dst, nnz, a.heads);
    return cudaGetLastError();
}

cudaError_t launch_segsum(const AggScratch& a, const uint32_t* uidx, int64_t nnz, int32_t* cols_out,
                          uint32_t* rowcnt, cudaStream_t s) {
    if (nnz == 0) return cudaSuccess;
    k_segsum<<<(unsigned)((nnz + 255) / 256), 256, 0, s>>>(a.src, a.dst, a.w, a.heads, uidx, nnz, cols_out,
                                                            a.wsum, rowcnt);
    return cudaGetLastError();
}

cudaError_t launch_narrow(const unsigned long long* wsum, int64_t m, uint32_t* w_out, Globals* glob,
                          cudaStream_t s) {
    if (m == 0) return cudaSuccess;
    k_narrow<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(wsum, m, w_out, glob);
    return cudaGetLastError();
}

}  // namespace cdk
