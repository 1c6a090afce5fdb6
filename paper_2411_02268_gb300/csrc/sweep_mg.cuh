// MG-sketch sweep kernel template, instantiated once per sketch size k in
// sweep_k*.cu so that the translation units compile in parallel.
//
// Paper: Section 4.1 and Fig. 2 (two scans per vertex: populate a k-slot
// weighted Misra-Gries sketch of neighbour communities, then compute the exact
// linking weight of every sketch candidate and move by Eq. 2); Algorithm 1
// (Appendix A.1) for the sketch update; Section 4.3 for LPA.
#pragma once

#include "cd_internal.cuh"

namespace cdk {

// ---------------------------------------------------------------------------
// Algorithm 1 on a register-resident sketch of K slots.
// ---------------------------------------------------------------------------
template <int K, typename VT>
__device__ __forceinline__ void mg_update(uint32_t (&key)[K], VT (&val)[K], uint32_t c, VT w,
                                          bool uncond) {
    bool has = false;
#pragma unroll
    for (int p = 0; p < K; ++p) {
        bool m = key[p] == c;
        val[p] += m ? w : (VT)0;
        has |= m;
    }
    if (!has) {
        if (uncond) {
#pragma unroll
            for (int p = 0; p < K; ++p) val[p] = val[p] > w ? val[p] - w : (VT)0;
        }
        int e = -1;
#pragma unroll
        for (int p = 0; p < K; ++p)
            if (val[p] == 0) e = p;
        if (e >= 0) {
#pragma unroll
            for (int p = 0; p < K; ++p)
                if (p == e) { key[p] = c; val[p] = w; }
        } else if (!uncond) {
#pragma unroll
            for (int p = 0; p < K; ++p) val[p] = val[p] > w ? val[p] - w : (VT)0;
        }
    }
}

// Per-vertex decision (Eq. 2 / LPA rule); acc[p] = K_{i->cand[p]}, kid = K_{i->d}.
template <int K, typename VT>
__device__ __forceinline__ bool decide(const SweepArgs& a, uint32_t i, uint32_t d,
                                       const uint32_t (&cand)[K], const VT (&acc)[K], VT kid,
                                       uint32_t& best_out, u128& gain_out) {
    uint32_t best = d;
    bool have = false;
    if (a.mode == CD_MODE_LPA) {
        VT bk = kid;
#pragma unroll
        for (int p = 0; p < K; ++p) {
            uint32_t c = cand[p];
            if (c == kEmpty) continue;
            VT v = acc[p];
            if (v > kid && (v > bk || (v == bk && c < best))) { best = c; bk = v; have = true; }
        }
        gain_out = have ? (u128)(bk - kid) : (u128)0;
    } else {
        const unsigned long long two_m = a.glob->two_m;
        const unsigned long long Ki = a.K[i];
        const unsigned long long Sd = a.Sigma[d];
        const bool sd1 = a.size[d] == 1;
        i128 bg = 0;
#pragma unroll
        for (int p = 0; p < K; ++p) {
            uint32_t c = cand[p];
            if (c == kEmpty) continue;
            if (sd1 && c > d && a.size[c] == 1) continue;
            i128 g = (i128)two_m * ((i128)acc[p] - (i128)kid) -
                     (i128)Ki * ((i128)Ki + (i128)a.Sigma[c] - (i128)Sd);
            if (g > 0 && (g > bg || (g == bg && c < best))) { best = c; bg = g; have = true; }
        }
        gain_out = have ? (u128)bg : (u128)0;
    }
    best_out = best;
    return have;
}

// Loads chunk ch (4 entries, 16-byte aligned) of the row [start, end) and calls
// f(col, w) for entries inside the row that are not self-loops.
template <typename F>
__device__ __forceinline__ void for_chunk(const SweepArgs& a, int64_t ch, int64_t start, int64_t end,
                                          uint32_t i, F&& f) {
    int64_t e0 = ch * 4;
    int cs[4];
    uint32_t ws[4];
    if (e0 + 4 <= a.nnz) {
        int4 cv = __ldg(reinterpret_cast<const int4*>(a.cols) + ch);
        uint4 wv = __ldg(reinterpret_cast<const uint4*>(a.w) + ch);
        cs[0] = cv.x; cs[1] = cv.y; cs[2] = cv.z; cs[3] = cv.w;
        ws[0] = wv.x; ws[1] = wv.y; ws[2] = wv.z; ws[3] = wv.w;
    } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            bool ok = e0 + u < a.nnz;
            cs[u] = ok ? a.cols[e0 + u] : -1;
            ws[u] = ok ? a.w[e0 + u] : 0u;
        }
    }
    uint32_t labs[4];
    bool ok[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        int64_t e = e0 + u;
        const bool in_row = e >= start && e < end;
        const bool in_range = (uint32_t)cs[u] < (uint32_t)a.n;
        if (in_row && !in_range) atomicOr(&a.glob->err, kErrBadCol);
        ok[u] = in_row && in_range && (uint32_t)cs[u] != i;
        labs[u] = ok[u] ? __ldg(a.labels + cs[u]) : kEmpty;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
        if (ok[u]) f(labs[u], ws[u]);
}

// Per-thread statistics handed to the block epilogue.
struct Outcome {
    bool moved;
    u128 gain;
    uint32_t vertex;
};

// ---------------------------------------------------------------------------
// G streams per vertex inside one warp (G = 1, 2, ..., 32).
// ---------------------------------------------------------------------------
template <int G, int K, typename VT>
__device__ __forceinline__ Outcome group_body(const SweepArgs& a, int64_t vi, bool valid) {
    const int lane = threadIdx.x & (G - 1);
    const unsigned gmask = (G == 32) ? 0xffffffffu
                                     : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
    Outcome out{false, 0, 0};
    uint32_t i = 0, d = 0;
    int64_t start = 0, end = 0;
    bool act = valid;
    if (valid) {
        i = a.verts[vi];
        start = a.off[i];
        end = a.off[i + 1];
        d = a.labels[i];
        if (a.active && !a.active[i]) act = false;
    }
    uint32_t key[K];
    VT val[K];
#pragma unroll
    for (int p = 0; p < K; ++p) { key[p] = kEmpty; val[p] = 0; }
    const bool unc = a.uncond != 0;
    const int64_t c0 = start >> 2, c1 = (end + 3) >> 2;
    const int64_t first = c0 + (int64_t)((lane - (int)(c0 & (G - 1))) & (G - 1));
    if (act) {
        for (int64_t ch = first; ch < c1; ch += G)
            for_chunk(a, ch, start, end, i, [&](uint32_t c, uint32_t w) {
                mg_update<K, VT>(key, val, c, (VT)w, unc);
            });
    }
    // merge tree: S[s] <- merge(S[s], S[s+o]), o = G/2 .. 1
#pragma unroll 1
    for (int o = G / 2; o >= 1; o >>= 1) {
#pragma unroll
        for (int p = 0; p < K; ++p) {
            uint32_t ok = __shfl_down_sync(gmask, key[p], o, G);
            VT ov = __shfl_down_sync(gmask, val[p], o, G);
            if (lane < o && ov > 0) mg_update<K, VT>(key, val, ok, ov, unc);
        }
    }
    uint32_t cand[K];
#pragma unroll
    for (int p = 0; p < K; ++p) {
        uint32_t kk = val[p] > 0 ? key[p] : kEmpty;
        kk = __shfl_sync(gmask, kk, 0, G);
        cand[p] = kk == d ? kEmpty : kk;
    }
    // second scan: exact K_{i->c} for the candidates and for d
    VT acc[K];
    VT kid = 0;
#pragma unroll
    for (int p = 0; p < K; ++p) acc[p] = 0;
    if (act) {
        for (int64_t ch = first; ch < c1; ch += G)
            for_chunk(a, ch, start, end, i, [&](uint32_t c, uint32_t w) {
                kid += c == d ? (VT)w : (VT)0;
#pragma unroll
                for (int p = 0; p < K; ++p) acc[p] += c == cand[p] ? (VT)w : (VT)0;
            });
    }
#pragma unroll
    for (int o = G / 2; o >= 1; o >>= 1) {
        kid += __shfl_down_sync(gmask, kid, o, G);
#pragma unroll
        for (int p = 0; p < K; ++p) acc[p] += __shfl_down_sync(gmask, acc[p], o, G);
    }
    if (act && lane == 0) {
        uint32_t best;
        u128 g;
        bool mv = decide<K, VT>(a, i, d, cand, acc, kid, best, g);
        a.labels_out[i] = best;
        out.moved = mv;
        out.gain = g;
        out.vertex = i;
    } else if (valid && !act && lane == 0) {
        a.labels_out[i] = d;
    }
    return out;
}

// ---------------------------------------------------------------------------
// L = 64, 128 or 256 streams per vertex: L/32 warps (a sub-block of the
// 256-thread block, synchronised by a named barrier).
// ---------------------------------------------------------------------------
template <int K, typename VT>
struct BlockSmem {
    uint32_t k[128][K];
    VT v[128][K];
    VT acc[8][K + 1];
    uint32_t cand[4][K];
};

__device__ __forceinline__ void sub_barrier(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

template <int L, int K, typename VT>
__device__ __forceinline__ Outcome block_body(const SweepArgs& a, int64_t vi, bool valid,
                                              BlockSmem<K, VT>& sm) {
    constexpr int W = L / 32;
    const int sb = threadIdx.x / L;
    const int s = threadIdx.x % L;
    const int bar = 1 + sb;
    const int wl = s >> 5;          // warp within sub-block
    const int lane = s & 31;
    Outcome out{false, 0, 0};
    uint32_t i = 0, d = 0;
    int64_t start = 0, end = 0;
    bool act = valid;
    if (valid) {
        i = a.verts[vi];
        start = a.off[i];
        end = a.off[i + 1];
        d = a.labels[i];
        if (a.active && !a.active[i]) act = false;
    }
    uint32_t key[K];
    VT val[K];
#pragma unroll
    for (int p = 0; p < K; ++p) { key[p] = kEmpty; val[p] = 0; }
    const bool unc = a.uncond != 0;
    const int64_t c0 = start >> 2, c1 = (end + 3) >> 2;
    const int64_t first = c0 + (int64_t)((s - (int)(c0 & (L - 1))) & (L - 1));
    if (act) {
        for (int64_t ch = first; ch < c1; ch += L)
            for_chunk(a, ch, start, end, i, [&](uint32_t c, uint32_t w) {
                mg_update<K, VT>(key, val, c, (VT)w, unc);
            });
    }
    // cross-warp rounds through shared memory (o = L/2 .. 32)
    const int slot_base = sb * (L / 2);  // (256/L) sub-blocks x L/2 slots = 128
#pragma unroll 1
    for (int o = L / 2; o >= 32; o >>= 1) {
        if (s >= o && s < 2 * o) {
#pragma unroll
            for (int p = 0; p < K; ++p) {
                sm.k[slot_base + s - o][p] = key[p];
                sm.v[slot_base + s - o][p] = val[p];
            }
        }
        sub_barrier(bar, L);
        if (s < o) {
#pragma unroll
            for (int p = 0; p < K; ++p) {
                VT ov = sm.v[slot_base + s][p];
                if (ov > 0) mg_update<K, VT>(key, val, sm.k[slot_base + s][p], ov, unc);
            }
        }
        sub_barrier(bar, L);
    }
    // in-warp rounds (o = 16 .. 1) in the first warp of the sub-block
    if (wl == 0) {
#pragma unroll 1
        for (int o = 16; o >= 1; o >>= 1) {
#pragma unroll
            for (int p = 0; p < K; ++p) {
                uint32_t ok = __shfl_down_sync(0xffffffffu, key[p], o);
                VT ov = __shfl_down_sync(0xffffffffu, val[p], o);
                if (lane < o && ov > 0) mg_update<K, VT>(key, val, ok, ov, unc);
            }
        }
        if (lane == 0) {
#pragma unroll
            for (int p = 0; p < K; ++p) {
                uint32_t kk = val[p] > 0 ? key[p] : kEmpty;
                sm.cand[sb][p] = kk == d ? kEmpty : kk;
            }
        }
    }
    sub_barrier(bar, L);
    uint32_t cand[K];
#pragma unroll
    for (int p = 0; p < K; ++p) cand[p] = sm.cand[sb][p];
    VT acc[K];
    VT kid = 0;
#pragma unroll
    for (int p = 0; p < K; ++p) acc[p] = 0;
    if (act) {
        for (int64_t ch = first; ch < c1; ch += L)
            for_chunk(a, ch, start, end, i, [&](uint32_t c, uint32_t w) {
                kid += c == d ? (VT)w : (VT)0;
#pragma unroll
                for (int p = 0; p < K; ++p) acc[p] += c == cand[p] ? (VT)w : (VT)0;
            });
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        kid += __shfl_down_sync(0xffffffffu, kid, o);
#pragma unroll
        for (int p = 0; p < K; ++p) acc[p] += __shfl_down_sync(0xffffffffu, acc[p], o);
    }
    const int wbase = sb * W;  // this sub-block's rows of sm.acc
    if (lane == 0) {
#pragma unroll
        for (int p = 0; p < K; ++p) sm.acc[wbase + wl][p] = acc[p];
        sm.acc[wbase + wl][K] = kid;
    }
    sub_barrier(bar, L);
    if (s == 0) {
        for (int q = 1; q < W; ++q) {
#pragma unroll
            for (int p = 0; p < K; ++p) acc[p] += sm.acc[wbase + q][p];
            kid += sm.acc[wbase + q][K];
        }
        if (act) {
            uint32_t best;
            u128 g;
            bool mv = decide<K, VT>(a, i, d, cand, acc, kid, best, g);
            a.labels_out[i] = best;
            out.moved = mv;
            out.gain = g;
            out.vertex = i;
        } else if (valid) {
            a.labels_out[i] = d;
        }
    }
    sub_barrier(bar, L);  // sm is reused by nothing after this, but keep phases clean
    return out;
}

// Warp-level statistics and mover list; every lane of the warp must call it.
__device__ __forceinline__ void epilogue(const SweepArgs& a, const Outcome& o) {
    const int lane = threadIdx.x & 31;
    unsigned mm = __ballot_sync(0xffffffffu, o.moved);
    if (mm == 0) return;
    unsigned long long lo = o.moved ? (unsigned long long)o.gain : 0ull;
    unsigned long long hi = o.moved ? (unsigned long long)(o.gain >> 64) : 0ull;
#pragma unroll
    for (int q = 16; q >= 1; q >>= 1) {
        unsigned long long l2 = __shfl_down_sync(0xffffffffu, lo, q);
        unsigned long long h2 = __shfl_down_sync(0xffffffffu, hi, q);
        unsigned long long nl = lo + l2;
        hi = hi + h2 + (nl < lo ? 1ull : 0ull);
        lo = nl;
    }
    unsigned long long base = 0;
    if (lane == 0) {
        base = atomicAdd(&a.glob->moved, (unsigned long long)__popc(mm));
        unsigned long long old = atomicAdd(&a.glob->gain_lo, lo);
        unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
        if (hi + carry) atomicAdd(&a.glob->gain_hi, hi + carry);
    }
    base = __shfl_sync(0xffffffffu, base, 0);
    if (o.moved && a.movers) a.movers[base + __popc(mm & ((1u << lane) - 1u))] = o.vertex;
}

template <int K, typename VT>
__global__ void __launch_bounds__(kBlock) k_sweep_mg(const SweepArgs a) {
    __shared__ BlockSmem<K, VT> sm;
    int b = 0;
#pragma unroll
    for (int q = 1; q < CD_MAX_BUCKETS; ++q)
        if (q < a.bt.nb && (int64_t)blockIdx.x >= a.bt.bbegin[q]) b = q;
    const int L = a.bt.lanes[b];
    const int64_t lb = (int64_t)blockIdx.x - a.bt.bbegin[b];
    const int vpb = L >= kBlock ? 1 : kBlock / L;
    const int64_t vi = a.bt.vbegin[b] + lb * vpb + threadIdx.x / L;
    const bool valid = vi < a.bt.vbegin[b + 1];
    Outcome o;
    switch (L) {
        case 1: o = group_body<1, K, VT>(a, vi, valid); break;
        case 2: o = group_body<2, K, VT>(a, vi, valid); break;
        case 4: o = group_body<4, K, VT>(a, vi, valid); break;
        case 8: o = group_body<8, K, VT>(a, vi, valid); break;
        case 16: o = group_body<16, K, VT>(a, vi, valid); break;
        case 32: o = group_body<32, K, VT>(a, vi, valid); break;
        case 64: o = block_body<64, K, VT>(a, vi, valid, sm); break;
        case 128: o = block_body<128, K, VT>(a, vi, valid, sm); break;
        default: o = block_body<256, K, VT>(a, vi, valid, sm); break;
    }
    epilogue(a, o);
}

template <int K>
cudaError_t launch_k(const SweepArgs& a, bool wide, int64_t nblocks, cudaStream_t s) {
    if (wide) k_sweep_mg<K, unsigned long long><<<(unsigned)nblocks, kBlock, 0, s>>>(a);
    else k_sweep_mg<K, uint32_t><<<(unsigned)nblocks, kBlock, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace cdk
