// Exact-hashtable local-moving sweep: the comparator of the MG sketch.
//
// Paper: Section 4 and Fig. 1 describe the "Default" per-thread collision-free
// hashtables (a keys list and a |V|-sized values array per thread, 8T|V| to
// 16T|V| bytes).  On the GPU the same exact K_{i->c} for every neighbouring
// community is kept in an open-addressing table per vertex: in shared memory
// for rows up to 4096 entries, and in device scratch for longer rows (the
// memory cost the MG sketch avoids).  The decision rules are those of the MG
// sweep (Eq. 2 for Louvain, the maximum weight for LPA).
#include "cd_internal.cuh"

namespace cdk {

__device__ __forceinline__ uint32_t hash32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

// Best candidate of one lane, reduced across lanes afterwards.
struct Best {
    i128 gain;          // Louvain: scaled gain; LPA: K_{i->c}
    uint32_t c;
};

__device__ __forceinline__ bool better(const Best& x, const Best& y) {
    // x better than y: larger gain, ties to the smaller id; c == kEmpty is none.
    if (x.c == kEmpty) return false;
    if (y.c == kEmpty) return true;
    return x.gain > y.gain || (x.gain == y.gain && x.c < y.c);
}

__device__ __forceinline__ Best shfl_best(unsigned mask, const Best& b, int src_delta, int width) {
    Best o;
    unsigned long long lo = (unsigned long long)(u128)b.gain;
    unsigned long long hi = (unsigned long long)((u128)b.gain >> 64);
    lo = __shfl_down_sync(mask, lo, src_delta, width);
    hi = __shfl_down_sync(mask, hi, src_delta, width);
    o.gain = (i128)(((u128)hi << 64) | (u128)lo);
    o.c = __shfl_down_sync(mask, b.c, src_delta, width);
    return o;
}

// Insert (c, w) into a table of T slots (power of two) with linear probing.
__device__ __forceinline__ void table_add(uint32_t* keys, unsigned long long* vals, uint32_t T,
                                          uint32_t c, unsigned long long w) {
    uint32_t h = hash32(c) & (T - 1);
    for (uint32_t probe = 0; probe < T; ++probe) {
        uint32_t k = keys[h];
        if (k == kEmpty) {
            k = atomicCAS(&keys[h], kEmpty, c);
            if (k == kEmpty) k = c;
        }
        if (k == c) {
            atomicAdd(&vals[h], w);
            return;
        }
        h = (h + 1) & (T - 1);
    }
}

__device__ __forceinline__ unsigned long long table_get(const uint32_t* keys, const unsigned long long* vals,
                                                        uint32_t T, uint32_t c) {
    uint32_t h = hash32(c) & (T - 1);
    for (uint32_t probe = 0; probe < T; ++probe) {
        uint32_t k = keys[h];
        if (k == c) return vals[h];
        if (k == kEmpty) return 0;
        h = (h + 1) & (T - 1);
    }
    return 0;
}

// Evaluates the slots [s0, T) step `stride` of a filled table for vertex i.
__device__ __forceinline__ Best scan_table(const SweepArgs& a, const uint32_t* keys,
                                           const unsigned long long* vals, uint32_t T, uint32_t s0,
                                           uint32_t stride, uint32_t i, uint32_t d,
                                           unsigned long long kid) {
    Best best{0, kEmpty};
    const bool lpa = a.mode == CD_MODE_LPA;
    const unsigned long long two_m = two_m_of(a, i);
    const unsigned long long Ki = a.K[i];
    const unsigned long long Sd = lpa ? 0ull : a.Sigma[d];
    const bool sd1 = lpa ? false : a.size[d] == 1;
    for (uint32_t s = s0; s < T; s += stride) {
        uint32_t c = keys[s];
        if (c == kEmpty || c == d) continue;
        unsigned long long kic = vals[s];
        Best cur{0, c};
        if (lpa) {
            if (kic <= kid) continue;
            cur.gain = (i128)kic;
        } else {
            if (barred(a, c, d, sd1)) continue;
            i128 g = (i128)two_m * ((i128)kic - (i128)kid) - (i128)Ki * ((i128)Ki + (i128)a.Sigma[c] - (i128)Sd);
            if (g <= 0) continue;
            cur.gain = g;
        }
        if (better(cur, best)) best = cur;
    }
    return best;
}

// Warp-local statistics and the mover list (same contract as the MG sweep).
__device__ __forceinline__ void exact_epilogue(const SweepArgs& a, bool moved, u128 gain, uint32_t v) {
    const int lane = threadIdx.x & 31;
    unsigned mm = __ballot_sync(0xffffffffu, moved);
    if (mm == 0) return;
    unsigned long long lo = moved ? (unsigned long long)gain : 0ull;
    unsigned long long hi = moved ? (unsigned long long)(gain >> 64) : 0ull;
#pragma unroll
    for (int q = 16; q >= 1; q >>= 1) {
        unsigned long long l2 = __shfl_down_sync(0xffffffffu, lo, q);
        unsigned long long h2 = __shfl_down_sync(0xffffffffu, hi, q);
        unsigned long long nl = lo + l2;
        hi = hi + h2 + (nl < lo ? 1ull : 0ull);
        lo = nl;
    }
    if (moved && a.gid) graph_stats(a, v, gain);
    unsigned long long base = 0;
    if (lane == 0) {
        base = atomicAdd(&a.glob->moved, (unsigned long long)__popc(mm));
        unsigned long long old = atomicAdd(&a.glob->gain_lo, lo);
        unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
        if (hi + carry) atomicAdd(&a.glob->gain_hi, hi + carry);
    }
    base = __shfl_sync(0xffffffffu, base, 0);
    if (moved && a.movers) a.movers[base + __popc(mm & ((1u << lane) - 1u))] = v;
}

__device__ __forceinline__ void finish(const SweepArgs& a, uint32_t i, uint32_t d, unsigned long long kid,
                                       const Best& b, unsigned long long kbest, bool& moved, u128& gain) {
    moved = b.c != kEmpty;
    if (a.attach) a.attach[i] = (float)(moved ? kbest : kid);
    if (moved) {
        a.labels_out[i] = b.c;
        gain = a.mode == CD_MODE_LPA ? (u128)((unsigned long long)b.gain - kid) : (u128)b.gain;
    } else {
        a.labels_out[i] = d;
        gain = 0;
    }
}

// G lanes per vertex (G <= 32), one shared-memory table of T slots per group.
__global__ void __launch_bounds__(kBlock) k_sweep_exact_group(const SweepArgs a, int bucket, int G,
                                                              uint32_t T) {
    extern __shared__ unsigned long long smem_u64[];
    const int groups = kBlock / G;
    const int gi = threadIdx.x / G;
    const int lane = threadIdx.x % G;
    unsigned long long* vals = smem_u64 + (size_t)gi * T;
    uint32_t* keys = reinterpret_cast<uint32_t*>(smem_u64 + (size_t)groups * T) + (size_t)gi * T;
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
    const int64_t vi = a.bt.vbegin[bucket] + ((int64_t)blockIdx.x * groups + gi);
    const bool valid = vi < a.bt.vbegin[bucket + 1];
    uint32_t i = 0, d = 0, bi = 0;
    int64_t start = 0, end = 0;
    bool act = valid;
    if (valid) {
        i = a.verts[vi];
        start = a.off[i];
        end = a.off[i + 1];
        d = a.labels[i];
        if (a.active && !a.active[i]) act = false;
        if (a.gdone && a.gdone[a.gid[i]]) act = false;
        if (a.bound) {
            bi = a.bound[i];
            if (a.size[d] != 1) act = false;  // refine: only singletons move
        }
    }
    for (uint32_t s = lane; s < T; s += G) { keys[s] = kEmpty; vals[s] = 0; }
    __syncwarp(gmask);
    if (act) {
        for (int64_t e = start + lane; e < end; e += G) {
            uint32_t j = (uint32_t)a.cols[e];
            if (j >= (uint32_t)a.n) { atomicOr(&a.glob->err, kErrBadCol); continue; }
            if (j == i) continue;
            if (a.bound && __ldg(a.bound + j) != bi) continue;
            table_add(keys, vals, T, __ldg(a.labels + j), a.w[e]);
        }
    }
    __syncwarp(gmask);
    Best b{0, kEmpty};
    unsigned long long kid = 0;
    if (act) {
        kid = table_get(keys, vals, T, d);
        b = scan_table(a, keys, vals, T, lane, G, i, d, kid);
    }
    for (int o = G / 2; o >= 1; o >>= 1) {
        Best ob = shfl_best(gmask, b, o, G);
        if (better(ob, b)) b = ob;
    }
    bool moved = false;
    u128 gain = 0;
    if (valid && lane == 0) {
        if (act) finish(a, i, d, kid, b, b.c != kEmpty ? table_get(keys, vals, T, b.c) : 0ull, moved, gain);
        else a.labels_out[i] = d;
    }
    exact_epilogue(a, moved, gain, i);
}

// One block per vertex; the table lives in shared memory (T <= 4096) or in a
// per-vertex region of device scratch (table_off[vi - vbegin] slots).
__global__ void __launch_bounds__(kBlock) k_sweep_exact_block(const SweepArgs a, int bucket, uint32_t T_smem,
                                                              uint32_t* gkeys, unsigned long long* gvals,
                                                              const int64_t* table_off) {
    extern __shared__ unsigned long long smem_u64[];
    __shared__ Best wbest[kBlock / 32];
    __shared__ unsigned long long s_kid;
    const int64_t vi = a.bt.vbegin[bucket] + blockIdx.x;
    if (vi >= a.bt.vbegin[bucket + 1]) return;  // whole block exits together
    const uint32_t i = a.verts[vi];
    const int64_t start = a.off[i], end = a.off[i + 1];
    const uint32_t d = a.labels[i];
    const uint32_t bi = a.bound ? a.bound[i] : 0u;
    const bool act = !(a.active && !a.active[i]) && !(a.bound && a.size[d] != 1) &&
                     !(a.gdone && a.gdone[a.gid[i]]);
    uint32_t T;
    uint32_t* keys;
    unsigned long long* vals;
    if (table_off) {
        int64_t o0 = table_off[vi - a.bt.vbegin[bucket]];
        T = (uint32_t)(table_off[vi - a.bt.vbegin[bucket] + 1] - o0);
        keys = gkeys + o0;
        vals = gvals + o0;
    } else {
        T = T_smem;
        vals = smem_u64;
        keys = reinterpret_cast<uint32_t*>(smem_u64 + T);
    }
    for (uint32_t s = threadIdx.x; s < T; s += kBlock) { keys[s] = kEmpty; vals[s] = 0; }
    __syncthreads();
    if (act) {
        for (int64_t e = start + threadIdx.x; e < end; e += kBlock) {
            uint32_t j = (uint32_t)a.cols[e];
            if (j >= (uint32_t)a.n) { atomicOr(&a.glob->err, kErrBadCol); continue; }
            if (j == i) continue;
            if (a.bound && __ldg(a.bound + j) != bi) continue;
            table_add(keys, vals, T, __ldg(a.labels + j), a.w[e]);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) s_kid = act ? table_get(keys, vals, T, d) : 0ull;
    __syncthreads();
    const unsigned long long kid = s_kid;
    Best b{0, kEmpty};
    if (act) b = scan_table(a, keys, vals, T, threadIdx.x, kBlock, i, d, kid);
    for (int o = 16; o >= 1; o >>= 1) {
        Best ob = shfl_best(0xffffffffu, b, o, 32);
        if (better(ob, b)) b = ob;
    }
    if ((threadIdx.x & 31) == 0) wbest[threadIdx.x >> 5] = b;
    __syncthreads();
    bool moved = false;
    u128 gain = 0;
    if (threadIdx.x == 0) {
        for (int q = 1; q < kBlock / 32; ++q)
            if (better(wbest[q], b)) b = wbest[q];
        if (act) finish(a, i, d, kid, b, b.c != kEmpty ? table_get(keys, vals, T, b.c) : 0ull, moved, gain);
        else a.labels_out[i] = d;
    }
    if (threadIdx.x < 32) exact_epilogue(a, moved, gain, i);
}

// Table slots for a row of length deg: the smallest power of two >= 2 deg (>= 8).
__host__ __device__ inline uint32_t exact_slots(int64_t deg) {
    uint32_t t = 8;
    while ((int64_t)t < 2 * deg) t <<= 1;
    return t;
}

__global__ void k_exact_table_sizes(const SweepArgs a, int bucket, int64_t* sizes) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t vi = a.bt.vbegin[bucket] + t;
    if (vi >= a.bt.vbegin[bucket + 1]) return;
    uint32_t i = a.verts[vi];
    sizes[t] = exact_slots(a.off[i + 1] - a.off[i]);
}

size_t exact_group_smem(int G, uint32_t T) {
    return (size_t)(kBlock / G) * T * (sizeof(unsigned long long) + sizeof(uint32_t));
}

cudaError_t launch_exact_group(const SweepArgs& a, int bucket, int G, uint32_t T, cudaStream_t s) {
    int64_t nv = a.bt.vbegin[bucket + 1] - a.bt.vbegin[bucket];
    if (nv == 0) return cudaSuccess;
    int groups = kBlock / G;
    size_t smem = exact_group_smem(G, T);
    cudaError_t e = cudaFuncSetAttribute(k_sweep_exact_group, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    note_launch();
    k_sweep_exact_group<<<(unsigned)((nv + groups - 1) / groups), kBlock, smem, s>>>(a, bucket, G, T);
    return cudaGetLastError();
}

cudaError_t launch_exact_block(const SweepArgs& a, int bucket, uint32_t T_smem, uint32_t* gkeys,
                               unsigned long long* gvals, const int64_t* table_off, cudaStream_t s) {
    int64_t nv = a.bt.vbegin[bucket + 1] - a.bt.vbegin[bucket];
    if (nv == 0) return cudaSuccess;
    size_t smem = table_off ? 0 : (size_t)T_smem * (sizeof(unsigned long long) + sizeof(uint32_t));
    cudaError_t e = cudaFuncSetAttribute(k_sweep_exact_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    note_launch();
    k_sweep_exact_block<<<(unsigned)nv, kBlock, smem, s>>>(a, bucket, T_smem, gkeys, gvals, table_off);
    return cudaGetLastError();
}

cudaError_t launch_exact_table_sizes(const SweepArgs& a, int bucket, int64_t* sizes, cudaStream_t s) {
    int64_t nv = a.bt.vbegin[bucket + 1] - a.bt.vbegin[bucket];
    if (nv == 0) return cudaSuccess;
    note_launch();
    k_exact_table_sizes<<<(unsigned)((nv + 255) / 256), 256, 0, s>>>(a, bucket, sizes);
    return cudaGetLastError();
}

}  // namespace cdk
