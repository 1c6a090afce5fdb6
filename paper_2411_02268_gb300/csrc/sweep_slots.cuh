// Large MG sketches (k = 32, 64) with the slots of one stream spread over a
// group of Q = k / 8 lanes: lane q of the group holds slots 8q .. 8q+7 in
// registers, every lane of the group sees every entry of the stream, and the
// group agrees on the outcome of each Algorithm 1 update by warp votes:
//   - the lane holding c (keys are unique across the whole sketch) adds w;
//   - a miss takes the largest free slot of the group: the highest lane that
//     has a free slot inserts into its own largest free slot, which is the
//     largest free index of the whole sketch;
//   - a miss with no free slot lowers every slot of every lane (clamped).
// This gives exactly the sequential update of a k-slot sketch (Section 4.1,
// Algorithm 1 in Appendix A.1) at the register cost of an 8-slot one, so the
// kernel keeps four 256-thread blocks per SM instead of one.  The second scan
// splits the candidates the same way (each lane counts its 8), and each lane
// evaluates the gains of its own candidates before a group argmax.
#pragma once

#include "cd_internal.cuh"

namespace cdk {

constexpr unsigned kFullWarp = 0xffffffffu;

// Slots 8q .. 8q+7 of a stream's sketch (value 0 = free; a freed slot keeps
// its key, which still matches and revives).
template <typename VT>
struct SlotPart {
    uint32_t key[8];
    VT t[8];

    __device__ __forceinline__ void init() {
#pragma unroll
        for (int p = 0; p < 8; ++p) { key[p] = kEmpty; t[p] = 0; }
    }
    __device__ __forceinline__ void lower_all(VT w) {
#pragma unroll
        for (int p = 0; p < 8; ++p) t[p] = (t[p] > w ? t[p] : w) - w;
    }
    // (c, w) into this lane's largest free slot (the caller knows one exists)
    __device__ __forceinline__ void take_top(uint32_t c, VT w) {
        bool done = false;
#pragma unroll
        for (int p = 7; p >= 0; --p) {
            const bool z = !done && t[p] == 0;
            key[p] = z ? c : key[p];
            t[p] = z ? w : t[p];
            done |= z;
        }
    }
};

// The Q lanes of one stream inside a warp.
template <int Q>
struct SlotGroup {
    int q;       // this lane's part of the sketch
    int shift;   // the group's first lane within the warp
    __device__ __forceinline__ unsigned bits(unsigned ballot) const { return (ballot >> shift) & ((1u << Q) - 1u); }
};

// One Algorithm 1 update of the group's sketch with (c, w); `on` is uniform
// over the group (false: the group skips this step).  Must be called by every
// lane of the warp together (warp votes).  Returns whether the sketch lost
// weight (a subtraction happened).
template <int Q, typename VT>
__device__ __forceinline__ bool slot_update(SlotPart<VT>& s, uint32_t c, VT w, bool on, int uncond,
                                            const SlotGroup<Q>& g) {
    bool hit = false;
#pragma unroll
    for (int p = 0; p < 8; ++p) {
        const bool m = on && s.key[p] == c;
        s.t[p] += m ? w : (VT)0;
        hit |= m;
    }
    // every lane votes (the vote must not sit behind a short-circuit of `on`)
    const unsigned hits = __ballot_sync(kFullWarp, hit);
    const bool miss = on && g.bits(hits) == 0;
    bool lost = false;
    const bool any_miss = __any_sync(kFullWarp, miss);
    if (any_miss) {
        if (miss && uncond) {  // unconditional: lower every slot first
            s.lower_all(w);
            lost = true;
        }
        bool fr = false;
#pragma unroll
        for (int p = 0; p < 8; ++p) fr |= s.t[p] == 0;
        const unsigned frees = __ballot_sync(kFullWarp, miss && fr);
        const unsigned fb = g.bits(frees);
        if (miss) {
            if (fb) {
                if (g.q == 31 - __clz(fb)) s.take_top(c, w);
            } else if (!uncond) {
                s.lower_all(w);
                lost = true;
            }
        }
    }
    return lost;
}

// scan_chunks with a warp-uniform trip count, so that f (which votes) is
// called by all lanes of the warp together; f(c, w, ok) with ok = false for
// lanes that have no entry at this step.
template <typename F>
__device__ __forceinline__ void scan_chunks_sync(const SweepArgs& a, int64_t first, int64_t c1, int step,
                                                 int64_t start, int64_t end, uint32_t i, uint32_t bi, bool act,
                                                 F&& f) {
    for (int64_t ch = first;; ch += step) {
        const bool more = act && ch < c1;
        if (!__any_sync(kFullWarp, more)) break;
        uint32_t labs[4], ws[4];
        bool ok[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) { labs[u] = kEmpty; ws[u] = 0; ok[u] = false; }
        if (more) {
            const Chunk cur = load_chunk(a, ch);
            const int64_t e0 = ch * 4;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t e = e0 + u;
                const bool in_row = e >= start && e < end;
                const bool in_range = (uint32_t)cur.c[u] < (uint32_t)a.n;
                if (in_row && !in_range) atomicOr(&a.glob->err, kErrBadCol);
                ok[u] = in_row && in_range && (uint32_t)cur.c[u] != i;
                labs[u] = ok[u] ? __ldg(a.labels + cur.c[u]) : kEmpty;
                ws[u] = cur.w[u];
            }
            if (a.bound) {
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (ok[u]) ok[u] = __ldg(a.bound + cur.c[u]) == bi;
            }
        }
        // one copy of f for the four entries (f holds the votes: a smaller
        // body keeps the instruction cache warm)
#pragma unroll 1
        for (int u = 0; u < 4; ++u) {
            f(labs[0], ws[0], ok[0]);
            labs[0] = labs[1]; labs[1] = labs[2]; labs[2] = labs[3];
            ws[0] = ws[1]; ws[1] = ws[2]; ws[2] = ws[3];
            ok[0] = ok[1]; ok[1] = ok[2]; ok[2] = ok[3];
        }
    }
}

// Shared memory of the slot form: one staging column per thread (merges,
// candidate broadcast, second-scan sums), slot-major so that the lanes of a
// warp touch consecutive words.
template <typename VT>
struct SlotSmem {
    uint32_t k[8][kBlock];
    VT v[8][kBlock];
    VT x[kBlock];
    int lossy[kBlock];
};

// Synchronises the T threads of one row (T <= 32: the warp, whose lanes run
// the same steps together; T > 32: a named barrier per sub-block).
template <int T>
__device__ __forceinline__ void row_sync() {
    if constexpr (T <= 32) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(1 + (int)threadIdx.x / T), "r"(T) : "memory");
    }
}

// Best move among one lane's 8 candidates (Eq. 2 for Louvain and refine, the
// largest linking weight for LPA), then the argmax over the group's Q lanes
// (largest gain, ties to the smaller id).  Called by every lane of the warp
// together; only lanes with `use` set contribute.
template <int Q, typename VT>
__device__ __forceinline__ bool slot_decide(const SweepArgs& a, bool use, uint32_t i, uint32_t d,
                                            const uint32_t (&cand)[8], const VT (&acc)[8], VT kid,
                                            uint32_t& best_out, u128& gain_out, VT& bw_out) {
    uint32_t best = d;
    VT best_w = kid;
    bool have = false;
    i128 bg = 0;
    if (a.mode == CD_MODE_LPA) {
        if (use) {
#pragma unroll
            for (int p = 0; p < 8; ++p) {
                const uint32_t c = cand[p];
                if (c == kEmpty) continue;
                const VT v = acc[p];
                if (v > kid && (v > best_w || (v == best_w && c < best))) { best = c; best_w = v; have = true; }
            }
        }
        bg = have ? (i128)(best_w - kid) : (i128)0;
    } else if (use) {
        const unsigned long long two_m = two_m_of(a, i);
        const unsigned long long Ki = __ldg(a.K + i);
        const unsigned long long Sd = __ldg(a.Sigma + d);
        const bool sd1 = __ldg(a.size + d) == 1;
#pragma unroll
        for (int b = 0; b < 8; b += 4) {
            unsigned long long sig[4];
            uint32_t siz[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t c = cand[b + u];
                const bool ok = c != kEmpty;
                sig[u] = ok ? __ldg(a.Sigma + c) : 0ull;
                siz[u] = ok ? __ldg(a.size + c) : 0u;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t c = cand[b + u];
                if (c == kEmpty) continue;
                if (barred_n(a, c, d, sd1, siz[u])) continue;
                const i128 gn = (i128)two_m * ((i128)acc[b + u] - (i128)kid) -
                                (i128)Ki * ((i128)Ki + (i128)sig[u] - (i128)Sd);
                if (gn > 0 && (gn > bg || (gn == bg && c < best))) {
                    best = c;
                    bg = gn;
                    have = true;
                    best_w = acc[b + u];
                }
            }
        }
    }
    // argmax over the group (both modes rank by bg: the gain, or for LPA the
    // weight above K_{i->d}, which orders the candidates like their weights)
#pragma unroll
    for (int off = 1; off < Q; off <<= 1) {
        const unsigned long long lo = (unsigned long long)(u128)bg, hi = (unsigned long long)((u128)bg >> 64);
        const unsigned long long plo = __shfl_xor_sync(kFullWarp, lo, off);
        const unsigned long long phi = __shfl_xor_sync(kFullWarp, hi, off);
        const uint32_t pb = __shfl_xor_sync(kFullWarp, best, off);
        const bool ph = __shfl_xor_sync(kFullWarp, (int)have, off) != 0;
        VT pw;
        if constexpr (sizeof(VT) == 8) pw = __shfl_xor_sync(kFullWarp, (unsigned long long)best_w, off);
        else pw = __shfl_xor_sync(kFullWarp, (uint32_t)best_w, off);
        const i128 pg = (i128)(((u128)phi << 64) | (u128)plo);
        if (ph && (!have || pg > bg || (pg == bg && pb < best))) {
            bg = pg;
            best = pb;
            have = true;
            best_w = pw;
        }
    }
    best_out = best;
    gain_out = have ? (u128)bg : (u128)0;
    bw_out = best_w;
    return have;
}

// One row per T = L * Q threads: L streams, each a group of Q lanes.
template <int L, int K, typename VT, typename U>
__device__ __forceinline__ Outcome slot_body(const SweepArgs& a, int64_t vi, bool valid, SlotSmem<VT>& sm) {
    constexpr int Q = K / 8;
    constexpr int T = L * Q;
    const int u = threadIdx.x % T;       // thread within the row
    const int s = u / Q;                 // stream
    const int q = u % Q;                 // part of the sketch
    const int rowbase = threadIdx.x - u;
    SlotGroup<Q> g{q, (int)(threadIdx.x & 31) & ~(Q - 1)};
    Outcome out{false, 0, 0, 0, 0};
    uint32_t i = 0, d = 0, bi = 0;
    int64_t start = 0, end = 0;
    bool act = valid;
    if (valid) {
        i = a.verts[vi];
        act = vertex_decides(a, i);
        if (act || a.out_all) d = a.labels[i];
        if (act) {
            start = a.off[i];
            end = a.off[i + 1];
            if (a.bound) {
                bi = a.bound[i];
                if (a.size[d] != 1) act = false;  // refine: only singletons move
            }
        }
    }
    const U unc = mode_of<U>(a);
    SlotPart<VT> sk;
    sk.init();
    bool lossy = false;
    const int64_t c0 = start >> 2, c1 = (end + 3) >> 2;
    const int64_t first = c0 + (int64_t)((s - (int)(c0 & (L - 1))) & (L - 1));
    scan_chunks_sync(a, first, c1, L, start, end, i, bi, act, [&](uint32_t c, uint32_t w, bool ok) {
        lossy |= slot_update<Q, VT>(sk, c, (VT)w, ok, unc, g);
    });
    // merge tree: stream s <- merge(stream s, stream s + o), o = L/2 .. 1; the
    // partner's slots go in slot order (part q2, slot p) as updates
#pragma unroll 1
    for (int o = L / 2; o >= 1; o >>= 1) {
        if (s >= o && s < 2 * o) {
#pragma unroll
            for (int p = 0; p < 8; ++p) {
                sm.k[p][threadIdx.x] = sk.key[p];
                sm.v[p][threadIdx.x] = sk.t[p];
            }
            sm.lossy[threadIdx.x] = (int)lossy;
        }
        row_sync<T>();
        const bool recv = s < o;
        // the partner group's first thread (lanes that do not receive read
        // their own column, which is in range, and ignore it)
        const int src0 = recv ? (int)threadIdx.x - q + o * Q : (int)threadIdx.x - q;
#pragma unroll 1
        for (int j = 0; j < 8 * Q; ++j) {  // the partner's slots in slot order: part j / 8, slot j % 8
            const uint32_t bk = sm.k[j & 7][src0 + (j >> 3)];
            const VT bv = sm.v[j & 7][src0 + (j >> 3)];
            lossy |= slot_update<Q, VT>(sk, bk, bv, recv && bv > 0, unc, g);
        }
        if (recv) lossy |= sm.lossy[src0] != 0;
        row_sync<T>();
    }
    // the row's candidates (stream 0's sketch) to every stream of the row
    if (s == 0) {
#pragma unroll
        for (int p = 0; p < 8; ++p) {
            sm.k[p][threadIdx.x] = sk.t[p] > 0 ? sk.key[p] : kEmpty;
            sm.v[p][threadIdx.x] = sk.t[p];
        }
        if (q == 0) sm.lossy[threadIdx.x] = (int)lossy;
    }
    row_sync<T>();
    uint32_t cand[8];
    VT acc[8];
    VT kid = 0;
#pragma unroll
    for (int p = 0; p < 8; ++p) {
        const uint32_t kk = sm.k[p][rowbase + q];
        const VT v = sm.v[p][rowbase + q];
        cand[p] = kk == d ? kEmpty : kk;
        acc[p] = kk == d ? (VT)0 : v;  // exact when the sketch never subtracted
        kid += kk == d ? v : (VT)0;
    }
    // no second scan when the sketch never subtracted (its values are the
    // exact linking weights) or in the LPA 1-scan variant (Section 4.3)
    const bool exact = sm.lossy[rowbase] == 0 || a.one_scan;
    row_sync<T>();
    // K_{i->d} from the sketch sits in at most one lane of the group (summed
    // by every lane of the warp: rows of one warp may differ in `exact`)
#pragma unroll
    for (int off = 1; off < Q; off <<= 1) {
        if constexpr (sizeof(VT) == 8) kid += __shfl_xor_sync(kFullWarp, (unsigned long long)kid, off);
        else kid += __shfl_xor_sync(kFullWarp, (uint32_t)kid, off);
    }
    if (!exact) {
        // second scan: every lane counts its own 8 candidates (and d) over
        // its stream, then stream 0 adds up the streams
#pragma unroll
        for (int p = 0; p < 8; ++p) acc[p] = 0;
        kid = 0;
        if (act) {
            scan_chunks(a, first, c1, L, start, end, i, bi, [&](uint32_t c, uint32_t w) {
                kid += c == d ? (VT)w : (VT)0;
#pragma unroll
                for (int p = 0; p < 8; ++p) acc[p] += c == cand[p] ? (VT)w : (VT)0;
            });
        }
    }
    if (L > 1) {
        // (run for exact rows too: rows of one warp share its barriers)
#pragma unroll
        for (int p = 0; p < 8; ++p) sm.v[p][threadIdx.x] = acc[p];
        sm.x[threadIdx.x] = kid;
        row_sync<T>();
        if (s == 0 && !exact) {
#pragma unroll 1
            for (int s2 = 1; s2 < L; ++s2) {
                const int src = threadIdx.x + s2 * Q;
#pragma unroll
                for (int p = 0; p < 8; ++p) acc[p] += sm.v[p][src];
                kid += sm.x[src];
            }
        }
        row_sync<T>();
    }
    // candidates of the row (each lane holds 8 of them), summed over the group
    int nc = 0;
#pragma unroll
    for (int p = 0; p < 8; ++p) nc += cand[p] != kEmpty ? 1 : 0;
#pragma unroll
    for (int off = 1; off < Q; off <<= 1) nc += __shfl_xor_sync(kFullWarp, nc, off);
    uint32_t best;
    u128 gain;
    VT bw;
    const bool use = act && s == 0;
    const bool mv = slot_decide<Q, VT>(a, use, i, d, cand, acc, kid, best, gain, bw);
    if (u == 0) {
        if (act) {
            a.labels_out[i] = best;
            if (a.attach) a.attach[i] = (float)bw;
            out.moved = mv;
            out.gain = gain;
            out.vertex = i;
            out.scanned = (uint32_t)(end - start);
            out.ncand = (uint32_t)nc;
        } else if (valid && a.out_all) {
            a.labels_out[i] = d;
        }
    }
    return out;
}

}  // namespace cdk
