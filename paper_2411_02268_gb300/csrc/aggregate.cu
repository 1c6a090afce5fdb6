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
#include "csr_walk.cuh"
#include "warp_vote.cuh"

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
    note_launch();
    k_mark_used<<<nb, 256, 0, s>>>(labels, n, scratch_n, glob);
    e = launch_exclusive_scan_u32(scratch_n, scratch_n, n, tile_scratch, count_dev, s);
    if (e != cudaSuccess) return e;
    note_launch();
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
    note_launch();
    k_compose<<<(unsigned)((n0 + 255) / 256), 256, 0, s>>>(top, n0, dense);
    return cudaGetLastError();
}

__global__ void k_iota(uint32_t* __restrict__ x, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) x[i] = (uint32_t)i;
}

cudaError_t launch_iota(uint32_t* x, int64_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    note_launch();
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
    note_launch();
    k_scatter_bound<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(sub, bound, n, next_init);
    return cudaGetLastError();
}

// ---- super-vertex graph ----------------------------------------------------------

constexpr int64_t kWalkTile = 4096;  // CSR entries per warp

// src[e] = dense[row(e)], dst[e] = dense[cols[e]]: one warp per 4096-entry
// tile, coalesced (csr_walk.cuh).
__global__ void k_expand(const int64_t* __restrict__ off, const int32_t* __restrict__ cols, int64_t n,
                         int64_t nnz, const uint32_t* __restrict__ dense, uint32_t* __restrict__ src,
                         uint32_t* __restrict__ dst, Globals* glob) {
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t e0 = warp * kWalkTile;
    if (e0 >= nnz) return;  // the whole warp
    const int64_t e1 = e0 + kWalkTile < nnz ? e0 + kWalkTile : nnz;
    const bool ok = warp_walk(off, n, e0, e1, [&](int64_t e, int64_t r) {
        src[e] = dense[r];
        const uint32_t j = (uint32_t)cols[e];
        dst[e] = j < (uint32_t)n ? dense[j] : 0u;
    });
    if (!ok && (threadIdx.x & 31) == 0) atomicOr(&glob->err, kErrBadOffsets);
}

// Stable LSD radix sort pass on 8-bit digits of key (shift), carrying two
// payload arrays.  Tiles of 4096 entries; digit counts per tile are scanned in
// digit-major order so that equal digits keep their tile order.
constexpr int kRadixThreads = 256;
constexpr int kRadixRounds = 16;
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

// The tile's entries are first placed in shared memory in their sorted order
// (digit, then original order), then written out so that consecutive threads
// write consecutive positions of one digit's run: the global writes coalesce
// (placing every entry straight at its global position scattered 4 bytes per
// 32-byte sector over three arrays).  Each of the 8 warps owns a contiguous
// slice of 512 entries of the tile, whose keys it loads into registers at
// once (16 per lane): it counts its digits, a prefix over the warps gives
// each warp where its entries of every digit start, and the warp then places
// its slice in order (rank among equal digits of a step, steps in order), so
// the sort stays stable with four block-wide barriers per tile.  The tile's
// digit counts and output starts come from the scanned histogram
// (consecutive exclusive offsets in digit-major order).  Four 256-thread
// blocks per SM (54 KB of shared memory each): the loads are latency-bound;
// 32 warps per SM measured faster than 16 warps holding twice the keys, and
// four small blocks 4% faster than two 512-thread blocks on 8192-entry
// tiles.
constexpr int kRadixSmem = 3 * kRadixTile * (int)sizeof(uint32_t);

constexpr int kScatterThreads = 256;
constexpr int kRadixWarps = kScatterThreads / 32;
constexpr int kRadixSlice = kRadixTile / kRadixWarps;  // entries per warp
constexpr int kSteps = kRadixSlice / 32;                // keys per lane, held in registers
constexpr int kBatch = 4;                               // payload loads in flight per lane

__global__ void __launch_bounds__(kScatterThreads, 4) k_radix_scatter(
    const uint32_t* __restrict__ key, const uint32_t* __restrict__ p1, const uint32_t* __restrict__ p2, int64_t n,
    int shift, const uint32_t* __restrict__ offs, int64_t ntiles, uint32_t* __restrict__ key_o,
    uint32_t* __restrict__ p1_o, uint32_t* __restrict__ p2_o) {
    extern __shared__ __align__(16) uint32_t tile_buf[];  // keys, p1, p2 of the tile in sorted order
    uint32_t* sk = tile_buf;
    uint32_t* s1 = tile_buf + kRadixTile;
    uint32_t* s2 = tile_buf + 2 * kRadixTile;
    __shared__ uint16_t wcnt[kRadixWarps][256];  // per warp: count, then the running start, of each digit
    __shared__ uint32_t tstart[256];  // where each digit's run starts in the tile
    __shared__ uint32_t gbase[256];   // where it starts in the output
    __shared__ uint32_t wsum[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t tile = blockIdx.x;
    const int64_t base = tile * kRadixTile;
    const int tn = (int)((n - base) < kRadixTile ? (n - base) : kRadixTile);
    const int j0 = warp * kRadixSlice;
    // the slice's keys: all loads in flight at once
    uint32_t kr[kSteps];
#pragma unroll
    for (int t = 0; t < kSteps; ++t) {
        const int j = j0 + t * 32 + lane;
        kr[t] = j < tn ? key[base + j] : 0u;
    }
    // digit d (threads 0..255, whole warps): output start and count of this
    // tile, and the digit's start in the tile
    const int d = threadIdx.x;
    uint32_t x = 0, cnt = 0;
    if (d < 256) {
        const int64_t idx = (int64_t)d * ntiles + tile;
        const uint32_t g0 = offs[idx];
        const uint32_t g1 = idx + 1 < 256 * ntiles ? offs[idx + 1] : (uint32_t)n;
        gbase[d] = g0;
        cnt = g1 - g0;
        x = cnt;  // inclusive scan of the counts over the digits
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
#pragma unroll
        for (int q = 0; q < kRadixWarps; ++q) wcnt[q][d] = 0;
    }
    __syncthreads();
    if (d < 256) {
        uint32_t before = 0;
        for (int q = 0; q < warp; ++q) before += wsum[q];
        tstart[d] = before + x - cnt;
    }
    // count the digits of this warp's slice
#pragma unroll
    for (int t = 0; t < kSteps; ++t) {
        const bool ok = j0 + t * 32 + lane < tn;
        const int dgt = ok ? (int)((kr[t] >> shift) & 255u) : -1;
        const unsigned peers = byte_peers(ok, (unsigned)dgt);
        if (ok && (peers & ((1u << lane) - 1u)) == 0) wcnt[warp][dgt] += (uint16_t)__popc(peers);
        __syncwarp();
    }
    __syncthreads();
    if (d < 256) {
        // per digit: exclusive prefix over the warps, from the digit's tile start
        uint32_t run = tstart[d];
#pragma unroll
        for (int q = 0; q < kRadixWarps; ++q) {
            const uint32_t c = wcnt[q][d];
            wcnt[q][d] = (uint16_t)run;
            run += c;
        }
    }
    __syncthreads();
    // place the slice in order, payloads loaded kBatch steps at a time
#pragma unroll
    for (int t0 = 0; t0 < kSteps; t0 += kBatch) {
        uint32_t a1[kBatch], a2[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int j = j0 + (t0 + u) * 32 + lane;
            a1[u] = j < tn ? p1[base + j] : 0u;
            a2[u] = j < tn ? p2[base + j] : 0u;
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int t = t0 + u;
            const bool ok = j0 + t * 32 + lane < tn;
            const uint32_t k = kr[t];
            const int dgt = ok ? (int)((k >> shift) & 255u) : -1;
            const unsigned peers = byte_peers(ok, (unsigned)dgt);
            const unsigned below = peers & ((1u << lane) - 1u);
            if (ok) {
                const uint32_t pos = wcnt[warp][dgt] + __popc(below);
                sk[pos] = k;
                s1[pos] = a1[u];
                s2[pos] = a2[u];
            }
            __syncwarp();
            if (ok && below == 0) wcnt[warp][dgt] += (uint16_t)__popc(peers);
            __syncwarp();
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < tn; j += kScatterThreads) {
        const uint32_t k = sk[j];
        const int dg = (int)((k >> shift) & 255u);
        const uint32_t pos = gbase[dg] + (uint32_t)j - tstart[dg];
        key_o[pos] = k;
        p1_o[pos] = s1[j];
        p2_o[pos] = s2[j];
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
// The sorted entries of one key are consecutive, so the lanes of a warp sum
// their runs with a segmented shuffle reduction and the first lane of each
// run piece adds it to wsum[u]: one atomic per run and warp instead of one
// per entry (after a pass most entries of a community fall into a few long
// runs, whose per-entry atomics would serialise on one address).  Integer
// sums: the order does not matter.
__global__ void k_segsum(const uint32_t* __restrict__ src, const uint32_t* __restrict__ dst,
                         const uint32_t* __restrict__ w, const uint32_t* __restrict__ heads,
                         const uint32_t* __restrict__ uidx, int64_t n, int32_t* __restrict__ cols_out,
                         unsigned long long* __restrict__ wsum, uint32_t* __restrict__ rowcnt) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool valid = e < n;
    uint32_t head = 0, u = 0xFFFFFFFFu;  // past the end: a key of its own
    unsigned long long v = 0;
    if (valid) {
        head = heads[e];
        u = uidx[e] + head - 1u;  // index of this entry's unique key
        v = w[e];
    }
    // sum each lane's run to its right within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long v2 = __shfl_down_sync(0xffffffffu, v, o);
        const uint32_t u2 = __shfl_down_sync(0xffffffffu, u, o);
        if (lane + o < 32 && u2 == u) v += v2;
    }
    const uint32_t uprev = __shfl_up_sync(0xffffffffu, u, 1);
    // distinct keys per row: the heads of one row are consecutive too, so
    // they are counted the same way (a hub community has millions of
    // distinct neighbour communities, one atomic each would serialise)
    const uint32_t r = valid ? src[e] : 0xFFFFFFFFu;
    uint32_t c = head;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t c2 = __shfl_down_sync(0xffffffffu, c, o);
        const uint32_t r2 = __shfl_down_sync(0xffffffffu, r, o);
        if (lane + o < 32 && r2 == r) c += c2;
    }
    const uint32_t rprev = __shfl_up_sync(0xffffffffu, r, 1);
    if (!valid) return;
    if (lane == 0 || uprev != u) atomicAdd(&wsum[u], v);
    if (head) cols_out[u] = (int32_t)dst[e];
    if ((lane == 0 || rprev != r) && c) atomicAdd(&rowcnt[r], c);
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

// Stable LSD sort of (src, dst, w): passes over the low `bits_dst` bits of dst,
// then the low `bits_src` bits of src, so the result is ordered by (src, dst)
// with ties in input order.  On return the sorted arrays are in (src, dst, w)
// (the buffers may have been swapped with the *2 ones).
cudaError_t radix_sort_keys(AggScratch& a, int64_t nnz, int bits_src, int bits_dst, Globals* glob, cudaStream_t s) {
    if (nnz == 0) return cudaSuccess;  // nothing to order (and no tile to launch)
    {
        cudaError_t e = cudaFuncSetAttribute(k_radix_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, kRadixSmem);
        if (e != cudaSuccess) return e;
    }
    int64_t nt = radix_tiles(nnz);
    int64_t hn = nt * 256;
    for (int which = 0; which < 2; ++which) {
        const int bits = which == 0 ? bits_dst : bits_src;
        for (int shift = 0; shift < bits; shift += 8) {
            uint32_t* key = which == 0 ? a.dst : a.src;
            uint32_t* p1 = which == 0 ? a.src : a.dst;
            uint32_t* key_o = which == 0 ? a.dst2 : a.src2;
            uint32_t* p1_o = which == 0 ? a.src2 : a.dst2;
            note_launch();
            k_radix_hist<<<(unsigned)nt, kRadixThreads, 0, s>>>(key, nnz, shift, a.hist, nt);
            cudaError_t e = launch_exclusive_scan_u32(a.hist, a.hist, hn, a.tiles, &glob->count, s);
            if (e != cudaSuccess) return e;
            note_launch();
            k_radix_scatter<<<(unsigned)nt, kScatterThreads, kRadixSmem, s>>>(key, p1, a.w, nnz, shift, a.hist, nt,
                                                                             key_o, p1_o, a.w2);
            std::swap(a.src, a.src2);
            std::swap(a.dst, a.dst2);
            std::swap(a.w, a.w2);
        }
    }
    return cudaGetLastError();
}

cudaError_t radix_sort_pairs(AggScratch& a, int64_t nnz, int64_t nc, Globals* glob, cudaStream_t s) {
    const int b = bits_for(nc);
    return radix_sort_keys(a, nnz, b, b, glob, s);
}

// ---- MG aggregation support ---------------------------------------------------------

// cnt[dense[i]] += 1 and ecnt[dense[i]] += deg(i)
__global__ void k_community_counts(const int64_t* __restrict__ off, const uint32_t* __restrict__ dense, int64_t n,
                                   uint32_t* __restrict__ cnt, uint32_t* __restrict__ ecnt) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t c = dense[i];
    atomicAdd(&cnt[c], 1u);
    const uint32_t d = (uint32_t)(off[i + 1] - off[i]);
    if (d) atomicAdd(&ecnt[c], d);
}

cudaError_t launch_community_counts(const int64_t* off, const uint32_t* dense, int64_t n, uint32_t* cnt,
                                    uint32_t* ecnt, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    note_launch();
    k_community_counts<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(off, dense, n, cnt, ecnt);
    return cudaGetLastError();
}

// Sketch slots of community c -> live entries sorted by key (in place), count.
template <int K>
__device__ void sort_slots(uint32_t* keys, unsigned long long* vals, uint32_t* count) {
    uint32_t k[K];
    unsigned long long v[K];
    int m = 0;
    for (int p = 0; p < K; ++p) {
        if (vals[p] > 0) { k[m] = keys[p]; v[m] = vals[p]; ++m; }
    }
    for (int x = 1; x < m; ++x) {  // insertion sort (K <= 16)
        uint32_t kk = k[x];
        unsigned long long vv = v[x];
        int y = x - 1;
        while (y >= 0 && k[y] > kk) { k[y + 1] = k[y]; v[y + 1] = v[y]; --y; }
        k[y + 1] = kk;
        v[y + 1] = vv;
    }
    for (int p = 0; p < K; ++p) {
        keys[p] = p < m ? k[p] : kEmpty;
        vals[p] = p < m ? v[p] : 0ull;
    }
    *count = (uint32_t)m;
}

__global__ void k_mg_sort_rows(uint32_t* __restrict__ keys, unsigned long long* __restrict__ vals, int64_t nc, int k,
                               uint32_t* __restrict__ count, uint32_t* __restrict__ self_less) {
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= nc) return;
    uint32_t* kk = keys + c * k;
    unsigned long long* vv = vals + c * k;
    switch (k) {
        case 1: sort_slots<1>(kk, vv, &count[c]); break;
        case 2: sort_slots<2>(kk, vv, &count[c]); break;
        case 4: sort_slots<4>(kk, vv, &count[c]); break;
        case 8: sort_slots<8>(kk, vv, &count[c]); break;
        default: sort_slots<16>(kk, vv, &count[c]); break;
    }
    if (self_less) {  // live entries other than the self-loop (reverse copies)
        uint32_t r = 0;
        for (int p = 0; p < k; ++p)
            if (vv[p] > 0 && kk[p] != (uint32_t)c) ++r;
        self_less[c] = r;
    }
}

// Louvain form: row c of G' = the live slots of sketch(c), sorted by key.
__global__ void k_mg_write_rows(const uint32_t* __restrict__ keys, const unsigned long long* __restrict__ vals,
                                int64_t nc, int k, const int64_t* __restrict__ roff, int32_t* __restrict__ cols_out,
                                uint32_t* __restrict__ w_out, Globals* glob) {
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= nc) return;
    int64_t o = roff[c];
    const int64_t m = roff[c + 1] - o;
    for (int64_t p = 0; p < m; ++p) {
        unsigned long long v = vals[c * k + p];
        if (v >> 32) atomicOr(&glob->err, kErrWeightOverflow);
        cols_out[o + p] = (int32_t)keys[c * k + p];
        w_out[o + p] = (uint32_t)v;
    }
}

// Leiden form, step 1: candidate entries; forward (c, d, v) of every live slot
// at fpos[c].., then reverse (d, c, v) of every live slot with d != c at
// R0 + rpos[c]..
__global__ void k_mg_candidates(const uint32_t* __restrict__ keys, const unsigned long long* __restrict__ vals,
                                int64_t nc, int k, const int64_t* __restrict__ fpos,
                                const int64_t* __restrict__ rpos, int64_t R0, uint32_t* __restrict__ src,
                                uint32_t* __restrict__ dst, uint32_t* __restrict__ w, Globals* glob) {
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= nc) return;
    int64_t f = fpos[c], r = R0 + rpos[c];
    for (int p = 0; p < k; ++p) {
        const unsigned long long v = vals[c * k + p];
        if (v == 0) continue;
        if (v >> 32) atomicOr(&glob->err, kErrWeightOverflow);
        const uint32_t d = keys[c * k + p];
        src[f] = (uint32_t)c; dst[f] = d; w[f] = (uint32_t)v; ++f;
        if (d != (uint32_t)c) { src[r] = d; dst[r] = (uint32_t)c; w[r] = (uint32_t)v; ++r; }
    }
}

// Leiden form, step 2 (entries sorted by (src, dst), forward before reverse for
// equal keys): keep one entry per pair, the one taken from the smaller
// community's sketch.
__global__ void k_mg_select(const uint32_t* __restrict__ src, const uint32_t* __restrict__ dst, int64_t m,
                            uint32_t* __restrict__ keep) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= m) return;
    const bool same_prev = e > 0 && src[e - 1] == src[e] && dst[e - 1] == dst[e];
    const bool same_next = e + 1 < m && src[e + 1] == src[e] && dst[e + 1] == dst[e];
    uint32_t k = 1;
    if (same_next) k = src[e] < dst[e] ? 1u : 0u;       // first of a pair
    else if (same_prev) k = src[e] > dst[e] ? 1u : 0u;  // second of a pair
    keep[e] = k;
}

__global__ void k_mg_compact(const uint32_t* __restrict__ src, const uint32_t* __restrict__ dst,
                             const uint32_t* __restrict__ w, const uint32_t* __restrict__ keep,
                             const uint32_t* __restrict__ pos, int64_t m, int32_t* __restrict__ cols_out,
                             uint32_t* __restrict__ w_out, uint32_t* __restrict__ rowcnt) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= m || !keep[e]) return;
    cols_out[pos[e]] = (int32_t)dst[e];
    w_out[pos[e]] = w[e];
    atomicAdd(&rowcnt[src[e]], 1u);
}

cudaError_t launch_mg_sort_rows(uint32_t* keys, unsigned long long* vals, int64_t nc, int k, uint32_t* count,
                                uint32_t* self_less, cudaStream_t s) {
    if (nc == 0) return cudaSuccess;
    note_launch();
    k_mg_sort_rows<<<(unsigned)((nc + 127) / 128), 128, 0, s>>>(keys, vals, nc, k, count, self_less);
    return cudaGetLastError();
}

cudaError_t launch_mg_write_rows(const uint32_t* keys, const unsigned long long* vals, int64_t nc, int k,
                                 const int64_t* roff, int32_t* cols_out, uint32_t* w_out, Globals* glob,
                                 cudaStream_t s) {
    if (nc == 0) return cudaSuccess;
    note_launch();
    k_mg_write_rows<<<(unsigned)((nc + 255) / 256), 256, 0, s>>>(keys, vals, nc, k, roff, cols_out, w_out, glob);
    return cudaGetLastError();
}

cudaError_t launch_mg_candidates(const uint32_t* keys, const unsigned long long* vals, int64_t nc, int k,
                                 const int64_t* fpos, const int64_t* rpos, int64_t R0, AggScratch& a, Globals* glob,
                                 cudaStream_t s) {
    if (nc == 0) return cudaSuccess;
    note_launch();
    k_mg_candidates<<<(unsigned)((nc + 255) / 256), 256, 0, s>>>(keys, vals, nc, k, fpos, rpos, R0, a.src, a.dst,
                                                                  a.w, glob);
    return cudaGetLastError();
}

cudaError_t launch_mg_select(const AggScratch& a, int64_t m, uint32_t* keep, cudaStream_t s) {
    if (m == 0) return cudaSuccess;
    note_launch();
    k_mg_select<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(a.src, a.dst, m, keep);
    return cudaGetLastError();
}

cudaError_t launch_mg_compact(const AggScratch& a, const uint32_t* keep, const uint32_t* pos, int64_t m,
                              int32_t* cols_out, uint32_t* w_out, uint32_t* rowcnt, cudaStream_t s) {
    if (m == 0) return cudaSuccess;
    note_launch();
    k_mg_compact<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(a.src, a.dst, a.w, keep, pos, m, cols_out, w_out,
                                                              rowcnt);
    return cudaGetLastError();
}

cudaError_t launch_expand(const int64_t* off, const int32_t* cols, int64_t n, int64_t nnz, const uint32_t* dense,
                          uint32_t* src, uint32_t* dst, Globals* glob, cudaStream_t s) {
    if (nnz == 0) return cudaSuccess;
    const int64_t warps = (nnz + kWalkTile - 1) / kWalkTile;
    note_launch();
    k_expand<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(off, cols, n, nnz, dense, src, dst, glob);
    return cudaGetLastError();
}

cudaError_t launch_heads(const AggScratch& a, int64_t nnz, cudaStream_t s) {
    if (nnz == 0) return cudaSuccess;
    note_launch();
    k_heads<<<(unsigned)((nnz + 255) / 256), 256, 0, s>>>(a.src, a.dst, nnz, a.heads);
    return cudaGetLastError();
}

cudaError_t launch_segsum(const AggScratch& a, const uint32_t* uidx, int64_t nnz, int32_t* cols_out,
                          uint32_t* rowcnt, cudaStream_t s) {
    if (nnz == 0) return cudaSuccess;
    note_launch();
    k_segsum<<<(unsigned)((nnz + 255) / 256), 256, 0, s>>>(a.src, a.dst, a.w, a.heads, uidx, nnz, cols_out,
                                                            a.wsum, rowcnt);
    return cudaGetLastError();
}

cudaError_t launch_narrow(const unsigned long long* wsum, int64_t m, uint32_t* w_out, Globals* glob,
                          cudaStream_t s) {
    if (m == 0) return cudaSuccess;
    note_launch();
    k_narrow<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(wsum, m, w_out, glob);
    return cudaGetLastError();
}

}  // namespace cdk
