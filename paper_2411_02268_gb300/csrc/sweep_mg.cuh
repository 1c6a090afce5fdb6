// MG-sketch sweep kernel template, instantiated once per sketch size k in
// sweep_k*.cu so that the translation units compile in parallel.
//
// Paper: Section 4.1 and Fig. 2 (two scans per vertex: populate a k-slot
// weighted Misra-Gries sketch of neighbour communities, then compute the exact
// linking weight of every sketch candidate and move by Eq. 2); Algorithm 1
// (Appendix A.1) for the sketch update; Section 4.3 for LPA.
#pragma once

#include <type_traits>

#include "cd_internal.cuh"

namespace cdk {

// ---------------------------------------------------------------------------
// Algorithm 1 on a register-resident sketch of K slots: key[p], value t[p]
// (0 = empty).  `lossy` records whether anything was ever subtracted: a
// sketch that never subtracted holds every community it saw with its exact
// weight, so the second scan can be skipped.  (Keeping the values against a
// running subtraction total turned a subtraction into one add but made every
// accumulation dearer; on R-MAT 22 it was 15% slower overall.)
// ---------------------------------------------------------------------------
// Tag selecting the weighted Misra-Gries of the literature (subtract = 2).
struct TextbookMG {};

template <typename U>
__device__ __forceinline__ U mode_of(const SweepArgs& a);
template <>
__device__ __forceinline__ int mode_of<int>(const SweepArgs& a) { return a.uncond; }
template <>
__device__ __forceinline__ TextbookMG mode_of<TextbookMG>(const SweepArgs&) { return TextbookMG{}; }

template <int K, typename VT>
struct Sketch {
    uint32_t key[K];
    VT t[K];
    bool lossy;

    __device__ __forceinline__ void init() {
#pragma unroll
        for (int p = 0; p < K; ++p) { key[p] = kEmpty; t[p] = 0; }
        lossy = false;
    }

    __device__ __forceinline__ VT value(int p) const { return t[p]; }

    // Algorithm 1 for one (c, w): add w to the slot holding c (a slot whose
    // value fell to 0 keeps its key and revives); otherwise (unconditional,
    // mode 1: after subtracting w from every slot) put c into the
    // largest-index empty slot (value 0), found by a downward search; with no
    // empty slot (conditional, mode 0) subtract w from every slot, clamping
    // at 0.
    __device__ __forceinline__ void update(uint32_t c, VT w, int mode) {
        // is c held?  (compares only; the slot gets w on the hit path)
        bool has = false;
#pragma unroll
        for (int p = 0; p < K; ++p) has |= key[p] == c;
        if (has) {
#pragma unroll
            for (int p = 0; p < K; ++p) t[p] += key[p] == c ? w : (VT)0;
            return;
        }
        if (mode) {
#pragma unroll
            for (int p = 0; p < K; ++p) t[p] = (t[p] > w ? t[p] : w) - w;
            lossy = true;
        }
        // a free slot takes c; with none, the conditional rule lowers every
        // slot (the downward search runs only when it will succeed)
        bool free = false;
#pragma unroll
        for (int p = 0; p < K; ++p) free |= t[p] == 0;
        if (free) {
            insert_top(c, w);
        } else if (!mode) {
#pragma unroll
            for (int p = 0; p < K; ++p) t[p] = (t[p] > w ? t[p] : w) - w;
            lossy = true;
        }
    }

    // The weighted Misra-Gries summary of the literature (subtract = 2, not
    // the paper's rule): with no empty slot every slot loses d = min(w,
    // smallest value) and the rest of w, if any, goes into the largest-index
    // slot that fell to 0.  A separate overload (selected at compile time), so
    // that the paper's modes keep their code.
    __device__ __forceinline__ void update(uint32_t c, VT w, TextbookMG) {
        bool has = false;
#pragma unroll
        for (int p = 0; p < K; ++p) {
            const bool m = key[p] == c;
            t[p] += m ? w : (VT)0;
            has |= m;
        }
        if (!has && !insert_top(c, w)) {
            VT d = w;
#pragma unroll
            for (int p = 0; p < K; ++p) d = t[p] < d ? t[p] : d;
#pragma unroll
            for (int p = 0; p < K; ++p) t[p] -= d;
            lossy = true;
            if (d < w) insert_top(c, w - d);
        }
    }

    // (c, w) into the largest-index empty slot, if any.
    __device__ __forceinline__ bool insert_top(uint32_t c, VT w) {
        bool done = false;
#pragma unroll
        for (int p = K - 1; p >= 0; --p) {
            const bool z = !done && t[p] == 0;
            key[p] = z ? c : key[p];
            t[p] = z ? w : t[p];
            done |= z;
        }
        return done;
    }
};

// Per-vertex decision (Eq. 2 / LPA rule); acc[p] = K_{i->cand[p]}, kid = K_{i->d}.
template <int K, typename VT>
__device__ __forceinline__ bool decide(const SweepArgs& a, uint32_t i, uint32_t d,
                                       const uint32_t (&cand)[K], const VT (&acc)[K], VT kid,
                                       uint32_t& best_out, u128& gain_out) {
    uint32_t best = d;
    VT best_w = kid;  // K_{i->c} of the chosen community
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
        best_w = bk;
    } else {
        const unsigned long long two_m = two_m_of(a, i);
        const unsigned long long Ki = __ldg(a.K + i);
        const unsigned long long Sd = __ldg(a.Sigma + d);
        const bool sd1 = __ldg(a.size + d) == 1;
        // the candidates' totals and sizes are requested four at a time before
        // any is used, so that those gathers are in flight together (Sigma and
        // size are read-only during a sweep; eight at a time spilled registers)
        constexpr int kB = K < 4 ? K : 4;
        i128 bg = 0;
#pragma unroll
        for (int b = 0; b < K; b += kB) {
            unsigned long long sig[kB];
            uint32_t siz[kB];
#pragma unroll
            for (int q = 0; q < kB; ++q) {
                const uint32_t c = cand[b + q];
                const bool ok = c != kEmpty;
                sig[q] = ok ? __ldg(a.Sigma + c) : 0ull;
                siz[q] = ok ? __ldg(a.size + c) : 0u;
            }
#pragma unroll
            for (int q = 0; q < kB; ++q) {
                const uint32_t c = cand[b + q];
                if (c == kEmpty) continue;
                if (barred_n(a, c, d, sd1, siz[q])) continue;
                const i128 g = (i128)two_m * ((i128)acc[b + q] - (i128)kid) -
                               (i128)Ki * ((i128)Ki + (i128)sig[q] - (i128)Sd);
                if (g > 0 && (g > bg || (g == bg && c < best))) {
                    best = c;
                    bg = g;
                    have = true;
                    best_w = acc[b + q];
                }
            }
        }
        gain_out = have ? (u128)bg : (u128)0;
    }
    best_out = best;
    if (a.attach) a.attach[i] = (float)best_w;
    return have;
}

// Chunk ch of the CSR: 4 entries, 16-byte aligned.
struct Chunk {
    int c[4];
    uint32_t w[4];
};

__device__ __forceinline__ Chunk load_chunk(const SweepArgs& a, int64_t ch) {
    Chunk k;
    const int64_t e0 = ch * 4;
    if (e0 + 4 <= a.nnz) {
        const int4 cv = __ldg(reinterpret_cast<const int4*>(a.cols) + ch);
        const uint4 wv = __ldg(reinterpret_cast<const uint4*>(a.w) + ch);
        k.c[0] = cv.x; k.c[1] = cv.y; k.c[2] = cv.z; k.c[3] = cv.w;
        k.w[0] = wv.x; k.w[1] = wv.y; k.w[2] = wv.z; k.w[3] = wv.w;
    } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const bool ok = e0 + u < a.nnz;
            k.c[u] = ok ? a.cols[e0 + u] : -1;
            k.w[u] = ok ? a.w[e0 + u] : 0u;
        }
    }
    return k;
}

// Scans the chunks first, first + step, ... < c1 of the row [start, end) and
// calls f(label of col, w) for entries inside the row that are not self-loops
// (in refine mode only for neighbours inside the vertex's bound), in order.
// Two copies of f per chunk: entries 0 and 1, then 2 and 3 shifted down
// (four copies cost registers, one copy costs shifts; two measured fastest).
template <bool kSave = false, typename F>
__device__ __forceinline__ void scan_chunks(const SweepArgs& a, int64_t first, int64_t c1, int step,
                                            int64_t start, int64_t end, uint32_t i, uint32_t bi, F&& f) {
    const uint32_t len = (uint32_t)(end - start);
    for (int64_t ch = first; ch < c1; ch += step) {
        Chunk cur = load_chunk(a, ch);
        // entry offsets within the row, wrapping below 0 for entries before it
        const uint32_t rel = (uint32_t)(ch * 4 - start);
        uint32_t labs[4];
        bool ok[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const bool in_row = rel + (uint32_t)u < len;
            const bool in_range = (uint32_t)cur.c[u] < (uint32_t)a.n;
            if (in_row && !in_range) atomicOr(&a.glob->err, kErrBadCol);
            ok[u] = in_row && in_range && (uint32_t)cur.c[u] != i;
            labs[u] = ok[u] ? __ldg(a.labels + cur.c[u]) : kEmpty;
        }
        if (a.bound) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (ok[u]) ok[u] = __ldg(a.bound + cur.c[u]) == bi;
        }
        if (kSave && a.elab) {
            // the row's entries of this chunk as the second scan will read them
            const uint32_t l0 = ok[0] ? labs[0] : kEmpty, l1 = ok[1] ? labs[1] : kEmpty;
            const uint32_t l2 = ok[2] ? labs[2] : kEmpty, l3 = ok[3] ? labs[3] : kEmpty;
            if (rel < len && rel + 3u < len && rel + 3u > rel) {
                reinterpret_cast<uint4*>(a.elab)[ch] = make_uint4(l0, l1, l2, l3);
            } else {
                const uint32_t lv[4] = {l0, l1, l2, l3};
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (rel + (uint32_t)u < len) a.elab[ch * 4 + u] = lv[u];
            }
        }
#pragma unroll 1
        for (int u = 0; u < 2; ++u) {
            if (ok[0]) f(labs[0], cur.w[0]);
            if (ok[1]) f(labs[1], cur.w[1]);
            ok[0] = ok[2]; ok[1] = ok[3];
            labs[0] = labs[2]; labs[1] = labs[3];
            cur.w[0] = cur.w[2]; cur.w[1] = cur.w[3];
        }
    }
}

// The second scan over the labels saved by the first (a.elab): the same
// chunks, no column loads and no label gathers; f(label, w) for the row's
// entries the first scan took.
template <typename F>
__device__ __forceinline__ void scan_saved(const SweepArgs& a, int64_t first, int64_t c1, int step, int64_t start,
                                           int64_t end, F&& f) {
    const uint32_t len = (uint32_t)(end - start);
    for (int64_t ch = first; ch < c1; ch += step) {
        const int64_t e0 = ch * 4;
        const uint32_t rel = (uint32_t)(e0 - start);
        uint32_t lv[4], wv[4];
        if (e0 + 4 <= a.nnz) {
            const uint4 l4 = reinterpret_cast<const uint4*>(a.elab)[ch];
            const uint4 w4 = __ldg(reinterpret_cast<const uint4*>(a.w) + ch);
            lv[0] = l4.x; lv[1] = l4.y; lv[2] = l4.z; lv[3] = l4.w;
            wv[0] = w4.x; wv[1] = w4.y; wv[2] = w4.z; wv[3] = w4.w;
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool in = e0 + u < a.nnz;
                lv[u] = in ? a.elab[e0 + u] : kEmpty;
                wv[u] = in ? a.w[e0 + u] : 0u;
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (rel + (uint32_t)u < len && lv[u] != kEmpty) f(lv[u], wv[u]);
    }
}

// Entry-by-entry scan of a row on one thread (single-stream rows are short:
// no alignment waste at the row's ends).
template <typename F>
__device__ __forceinline__ void for_row(const SweepArgs& a, int64_t start, int64_t end, uint32_t i, uint32_t bi,
                                        F&& f) {
#pragma unroll 4
    for (int64_t e = start; e < end; ++e) {
        const uint32_t j = (uint32_t)__ldg(a.cols + e);
        const uint32_t w = __ldg(a.w + e);
        if (j >= (uint32_t)a.n) {
            atomicOr(&a.glob->err, kErrBadCol);
            continue;
        }
        if (j == i) continue;
        if (a.bound && __ldg(a.bound + j) != bi) continue;
        f(__ldg(a.labels + j), w);
    }
}

// Per-thread statistics handed to the block epilogue.
struct Outcome {
    bool moved;
    u128 gain;
    uint32_t vertex;
    uint32_t scanned;  // entries of the row, when the vertex decided
    uint32_t ncand;    // candidates it evaluated (each costs a Sigma_c and a size gather)
};

// Feeds the live slots of a partner sketch (keys pk, values pv) to s.
template <int K, typename VT, typename U>
__device__ __forceinline__ void merge_into(Sketch<K, VT>& s, const uint32_t (&pk_in)[K], const VT (&pv_in)[K],
                                           bool plossy, U unc) {
    if constexpr (K >= 16) {
        // one copy of the update: the partner's slots rotate through slot 0
        uint32_t pk[K];
        VT pv[K];
#pragma unroll
        for (int p = 0; p < K; ++p) { pk[p] = pk_in[p]; pv[p] = pv_in[p]; }
#pragma unroll 1
        for (int p = 0; p < K; ++p) {
            if (pv[0] > 0) s.update(pk[0], pv[0], unc);
#pragma unroll
            for (int q = 0; q + 1 < K; ++q) { pk[q] = pk[q + 1]; pv[q] = pv[q + 1]; }
        }
    } else {
#pragma unroll
        for (int p = 0; p < K; ++p)
            if (pv_in[p] > 0) s.update(pk_in[p], pv_in[p], unc);
    }
    s.lossy |= plossy;
}

// Merge tree over the G streams of a group inside one warp: S[s] <- merge(S[s],
// S[s+o]) for o = G/2 .. 1; lane 0 ends with the row's sketch.
template <int G, int K, typename VT, typename U>
__device__ __forceinline__ void group_merge(Sketch<K, VT>& sk, int lane, unsigned gmask, U unc) {
#pragma unroll 1
    for (int o = G / 2; o >= 1; o >>= 1) {
        uint32_t pk[K];
        VT pv[K];
#pragma unroll
        for (int p = 0; p < K; ++p) {
            pk[p] = __shfl_down_sync(gmask, sk.key[p], o, G);
            pv[p] = __shfl_down_sync(gmask, sk.value(p), o, G);
        }
        const bool pl = __shfl_down_sync(gmask, (int)sk.lossy, o, G) != 0;
        if (lane < o) merge_into(sk, pk, pv, pl, unc);
    }
}

// Second-scan tables for groups of G >= 4 streams and k >= 16 (for k = 8 the
// compares in registers were faster: 1.16 against 1.35 ms on R-MAT 22; for
// k = 16 the tables won, 3.1 against 4.0 ms): d and the candidates in a
// 32-slot open-addressing table per group in shared memory (Fibonacci
// hashing: the key times 2^32 / golden ratio, top five bits; linear probing),
// so that an entry of the second scan costs a hash and one or two probes
// instead of k + 1 compares.  Weights are added with shared-memory atomics
// (integers: the sums do not depend on the order).
constexpr int kTabSlots = 32;
template <typename VT>
struct PassTwoTabs {
    uint32_t key[kBlock / 4][kTabSlots];
    VT val[kBlock / 4][kTabSlots];
};

__device__ __forceinline__ int tab_hash(uint32_t c) { return (int)((c * 0x9E3779B1u) >> 27); }

// Slot of key c in table tk, or -1 (bounded probe).
__device__ __forceinline__ int tab_find(const uint32_t* tk, uint32_t c) {
    int h = tab_hash(c);
    for (int t = 0; t < kTabSlots; ++t) {
        const uint32_t k2 = tk[h];
        if (k2 == c) return h;
        if (k2 == kEmpty) return -1;
        h = (h + 1) & (kTabSlots - 1);
    }
    return -1;
}

// ---------------------------------------------------------------------------
// G streams per vertex inside one warp (G = 1, 2, ..., 32).
// ---------------------------------------------------------------------------
template <int G, int K, typename VT, typename U>
__device__ __forceinline__ Outcome group_body(const SweepArgs& a, int64_t vi, bool valid, PassTwoTabs<VT>* tabs) {
    const int lane = threadIdx.x & (G - 1);
    const unsigned gmask = (G == 32) ? 0xffffffffu
                                     : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
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
    Sketch<K, VT> sk;
    sk.init();
    const U unc = mode_of<U>(a);
    const int64_t c0 = start >> 2, c1 = (end + 3) >> 2;
    const int64_t first = c0 + (int64_t)((lane - (int)(c0 & (G - 1))) & (G - 1));
    if (act) {
        if (G == 1) {
            scan_chunks<true>(a, first, c1, G, start, end, i, bi, [&](uint32_t c, uint32_t w) { sk.update(c, (VT)w, unc); });
        } else {
            scan_chunks<true>(a, first, c1, G, start, end, i, bi, [&](uint32_t c, uint32_t w) { sk.update(c, (VT)w, unc); });
        }
    }
    group_merge<G, K, VT>(sk, lane, gmask, unc);
    // candidates (and, if the sketch never subtracted, their exact weights)
    uint32_t cand[K];
    VT acc[K];
    VT kid = 0;
    // no second scan when the sketch never subtracted (its values are then the
    // exact linking weights) or in the LPA 1-scan variant (Section 4.3)
    const bool exact = __shfl_sync(gmask, (int)sk.lossy, 0, G) == 0 || a.one_scan;
#pragma unroll
    for (int p = 0; p < K; ++p) {
        const VT v = sk.value(p);
        uint32_t kk = v > 0 ? sk.key[p] : kEmpty;
        kk = __shfl_sync(gmask, kk, 0, G);
        cand[p] = kk == d ? kEmpty : kk;
        acc[p] = kk == d ? (VT)0 : v;  // lane 0: exact when the sketch never subtracted
        kid += kk == d ? v : (VT)0;
    }
    if (!exact && G >= 4 && K >= 16) {
        // second scan through the group's table: exact K_{i->c} for the
        // candidates and for d
        uint32_t* tk = tabs->key[threadIdx.x / G];
        VT* tv = tabs->val[threadIdx.x / G];
        if (lane == 0) {
            for (int t = 0; t < kTabSlots; ++t) {
                tk[t] = kEmpty;
                tv[t] = 0;
            }
            auto put = [&](uint32_t c) {
                int h = tab_hash(c);
                for (int t = 0; t < kTabSlots && tk[h] != kEmpty; ++t) h = (h + 1) & (kTabSlots - 1);
                tk[h] = c;
            };
            put(d);
#pragma unroll
            for (int p = 0; p < K; ++p)
                if (cand[p] != kEmpty) put(cand[p]);
        }
        __syncwarp(gmask);
        if (act) {
            auto addt = [&](uint32_t c, uint32_t w) {
                const int h = tab_find(tk, c);
                if (h >= 0) atomicAdd(&tv[h], (VT)w);
            };
            if (a.elab) scan_saved(a, first, c1, G, start, end, addt);
            else scan_chunks(a, first, c1, G, start, end, i, bi, addt);
        }
        __syncwarp(gmask);
        if (lane == 0) {
            const int hd = tab_find(tk, d);
            kid = hd >= 0 ? tv[hd] : (VT)0;
#pragma unroll
            for (int p = 0; p < K; ++p) {
                const int h = cand[p] != kEmpty ? tab_find(tk, cand[p]) : -1;
                acc[p] = h >= 0 ? tv[h] : (VT)0;
            }
        }
        __syncwarp(gmask);  // the table is reused by the next virtual block
    } else if (!exact) {
        // second scan: exact K_{i->c} for the candidates and for d
#pragma unroll
        for (int p = 0; p < K; ++p) acc[p] = 0;
        kid = 0;
        if (act) {
            auto add = [&](uint32_t c, uint32_t w) {
                kid += c == d ? (VT)w : (VT)0;
#pragma unroll
                for (int p = 0; p < K; ++p) acc[p] += c == cand[p] ? (VT)w : (VT)0;
            };
            if (a.elab) scan_saved(a, first, c1, G, start, end, add);
            else scan_chunks(a, first, c1, G, start, end, i, bi, add);
        }
#pragma unroll
        for (int o = G / 2; o >= 1; o >>= 1) {
            kid += __shfl_down_sync(gmask, kid, o, G);
#pragma unroll
            for (int p = 0; p < K; ++p) acc[p] += __shfl_down_sync(gmask, acc[p], o, G);
        }
    }
    if (act && lane == 0) {
        uint32_t best;
        u128 g;
        bool mv = decide<K, VT>(a, i, d, cand, acc, kid, best, g);
        a.labels_out[i] = best;
        out.moved = mv;
        out.gain = g;
        out.vertex = i;
        out.scanned = (uint32_t)(end - start);
#pragma unroll
        for (int p = 0; p < K; ++p) out.ncand += cand[p] != kEmpty ? 1u : 0u;
    } else if (valid && !act && lane == 0 && a.out_all) {
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
    int lossy[128];
    VT acc[8][K + 1];
    uint32_t cand[4][K];
    VT cval[4][K];
    int exact[4];
};

__device__ __forceinline__ void sub_barrier(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Merge tree over the L = 64..256 streams of a sub-block: cross-warp rounds
// (o = L/2 .. 32) through shared memory, then in-warp rounds (o = 16 .. 1) in
// the sub-block's first warp; thread s = 0 ends with the row's sketch.
template <int L, int K, typename VT, typename U>
__device__ __forceinline__ void block_merge(Sketch<K, VT>& sk, int s, int sb, int bar, BlockSmem<K, VT>& sm,
                                            U unc) {
    const int slot_base = sb * (L / 2);  // (256/L) sub-blocks x L/2 slots = 128
#pragma unroll 1
    for (int o = L / 2; o >= 32; o >>= 1) {
        if (s >= o && s < 2 * o) {
#pragma unroll
            for (int p = 0; p < K; ++p) {
                sm.k[slot_base + s - o][p] = sk.key[p];
                sm.v[slot_base + s - o][p] = sk.value(p);
            }
            sm.lossy[slot_base + s - o] = (int)sk.lossy;
        }
        sub_barrier(bar, L);
        if (s < o) {
            uint32_t pk[K];
            VT pv[K];
#pragma unroll
            for (int p = 0; p < K; ++p) {
                pk[p] = sm.k[slot_base + s][p];
                pv[p] = sm.v[slot_base + s][p];
            }
            merge_into(sk, pk, pv, sm.lossy[slot_base + s] != 0, unc);
        }
        sub_barrier(bar, L);
    }
    if ((s >> 5) == 0) group_merge<32, K, VT, U>(sk, s & 31, 0xffffffffu, unc);
}

template <int L, int K, typename VT, typename U>
__device__ __forceinline__ Outcome block_body(const SweepArgs& a, int64_t vi, bool valid,
                                              BlockSmem<K, VT>& sm) {
    constexpr int W = L / 32;
    const int sb = threadIdx.x / L;
    const int s = threadIdx.x % L;
    const int bar = 1 + sb;
    const int wl = s >> 5;          // warp within sub-block
    const int lane = s & 31;
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
    Sketch<K, VT> sk;
    sk.init();
    const U unc = mode_of<U>(a);
    const int64_t c0 = start >> 2, c1 = (end + 3) >> 2;
    const int64_t first = c0 + (int64_t)((s - (int)(c0 & (L - 1))) & (L - 1));
    if (act) {
        scan_chunks<true>(a, first, c1, L, start, end, i, bi, [&](uint32_t c, uint32_t w) { sk.update(c, (VT)w, unc); });
    }
    block_merge<L, K, VT, U>(sk, s, sb, bar, sm, unc);
    if (wl == 0 && lane == 0) {
#pragma unroll
        for (int p = 0; p < K; ++p) {
            const VT v = sk.value(p);
            sm.cand[sb][p] = v > 0 ? sk.key[p] : kEmpty;
            sm.cval[sb][p] = v;
        }
        sm.exact[sb] = sk.lossy ? 0 : 1;
    }
    sub_barrier(bar, L);
    uint32_t cand[K];
    VT acc[K];
    VT kid = 0;
#pragma unroll
    for (int p = 0; p < K; ++p) {
        const uint32_t kk = sm.cand[sb][p];
        const VT v = sm.cval[sb][p];
        cand[p] = kk == d ? kEmpty : kk;
        acc[p] = kk == d ? (VT)0 : v;
        kid += kk == d ? v : (VT)0;
    }
    const bool exact = sm.exact[sb] != 0 || a.one_scan;
    if (!exact) {
#pragma unroll
        for (int p = 0; p < K; ++p) acc[p] = 0;
        kid = 0;
        if (act) {
            auto addb = [&](uint32_t c, uint32_t w) {
                kid += c == d ? (VT)w : (VT)0;
#pragma unroll
                for (int p = 0; p < K; ++p) acc[p] += c == cand[p] ? (VT)w : (VT)0;
            };
            if (a.elab) scan_saved(a, first, c1, L, start, end, addb);
            else scan_chunks(a, first, c1, L, start, end, i, bi, addb);
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
        }
    }
    if (s == 0) {
        if (act) {
            uint32_t best;
            u128 g;
            bool mv = decide<K, VT>(a, i, d, cand, acc, kid, best, g);
            a.labels_out[i] = best;
            out.moved = mv;
            out.gain = g;
            out.vertex = i;
            out.scanned = (uint32_t)(end - start);
#pragma unroll
            for (int p = 0; p < K; ++p) out.ncand += cand[p] != kEmpty ? 1u : 0u;
        } else if (valid && a.out_all) {
            a.labels_out[i] = d;
        }
    }
    sub_barrier(bar, L);
    return out;
}

// Block totals of the epilogue: movers, their 128-bit gain, entries scanned,
// and the block's first slot in the mover list.
struct EpiSmem {
    unsigned cnt;
    unsigned long long lo, hi, scanned, cands, base;
};

// Block-level statistics and mover list: warp sums go to shared memory and
// one thread adds the block's totals to the globals (one set of global
// atomics per block instead of per warp).  Every thread of the block must
// call it.
__device__ __forceinline__ void block_epilogue(const SweepArgs& a, const Outcome& o, EpiSmem& e) {
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) { e.cnt = 0; e.lo = 0; e.hi = 0; e.scanned = 0; e.cands = 0; }
    __syncthreads();
    const unsigned sc = __reduce_add_sync(0xffffffffu, o.scanned);
    const unsigned nc = __reduce_add_sync(0xffffffffu, o.ncand);
    const unsigned mm = __ballot_sync(0xffffffffu, o.moved);
    unsigned woff = 0;
    if (mm) {
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
        if (lane == 0) {
            woff = atomicAdd(&e.cnt, (unsigned)__popc(mm));
            unsigned long long old = atomicAdd(&e.lo, lo);
            hi += (old + lo < old) ? 1ull : 0ull;
            if (hi) atomicAdd(&e.hi, hi);
        }
        woff = __shfl_sync(0xffffffffu, woff, 0);
        if (o.moved && a.gid) graph_stats(a, o.vertex, o.gain);
    }
    if (lane == 0 && sc) atomicAdd(&e.scanned, (unsigned long long)sc);
    if (lane == 0 && nc) atomicAdd(&e.cands, (unsigned long long)nc);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (e.scanned) atomicAdd(&a.glob->scanned, e.scanned);
        if (e.cands) atomicAdd(&a.glob->cands, e.cands);
        if (e.cnt) {
            e.base = atomicAdd(&a.glob->moved, (unsigned long long)e.cnt);
            unsigned long long old = atomicAdd(&a.glob->gain_lo, e.lo);
            unsigned long long carry = (old + e.lo < old) ? 1ull : 0ull;
            if (e.hi + carry) atomicAdd(&a.glob->gain_hi, e.hi + carry);
        }
    }
    __syncthreads();
    if (o.moved && a.movers) a.movers[e.base + woff + __popc(mm & ((1u << lane) - 1u))] = o.vertex;
}

}  // namespace cdk

#include "sweep_slots.cuh"

namespace cdk {

// Shared memory of the sub-block merges (k <= 16; larger sketches use the
// slot form of sweep_slots.cuh).
struct NoTabs {};
template <int K, typename VT>
union SmallSketchSmem {
    BlockSmem<K, VT> b;    // sub-block merges (L >= 64)
    typename std::conditional<(K >= 16), PassTwoTabs<VT>, NoTabs>::type t;  // second-scan tables
};
template <int K, typename VT>
using SweepSmem = typename std::conditional<(K <= 16), SmallSketchSmem<K, VT>, SlotSmem<VT>>::type;

template <int K, typename VT>
__device__ __forceinline__ PassTwoTabs<VT>* tabs_of(SmallSketchSmem<K, VT>& sm) {
    if constexpr (K >= 16) return &sm.t;
    else return nullptr;
}

template <int K, typename VT>
constexpr int sweep_min_blocks() {
    return K >= 32 ? 4 : ((K >= 16 || sizeof(VT) == 8) ? 2 : 4);
}

template <int K, typename VT, typename U>
__global__ void __launch_bounds__(kBlock, sweep_min_blocks<K, VT>()) k_sweep_mg(const SweepArgs a) {
    __shared__ SweepSmem<K, VT> sm;
    __shared__ EpiSmem esm;
    // Virtual blocks, the longest rows first, so that they start at once and
    // overlap with the many short rows instead of trailing the launch.  A
    // full sweep runs one virtual block per grid block unless the schedule
    // asks for a resident grid; a skip sweep over the compacted list (ranges
    // on the device) runs a smaller grid; both stride over the virtual
    // blocks.
    const int64_t nvirt = a.dr ? a.dr->bbegin[a.bt.nb] : a.bt.bbegin[a.bt.nb];
    for (int64_t j = blockIdx.x; j < nvirt; j += gridDim.x) {
        if (j != (int64_t)blockIdx.x) __syncthreads();  // the previous virtual block is done with shared memory
        const int64_t blk = nvirt - 1 - j;
        int b = 0;
        int64_t vb0, vb1, bb0;
        if (a.dr) {
#pragma unroll
            for (int q = 1; q < CD_MAX_BUCKETS; ++q)
                if (q < a.bt.nb && blk >= a.dr->bbegin[q]) b = q;
            bb0 = a.dr->bbegin[b];
            vb0 = a.dr->vbegin[b];
            vb1 = a.dr->vbegin[b + 1];
        } else {
#pragma unroll
            for (int q = 1; q < CD_MAX_BUCKETS; ++q)
                if (q < a.bt.nb && blk >= a.bt.bbegin[q]) b = q;
            bb0 = a.bt.bbegin[b];
            vb0 = a.bt.vbegin[b];
            vb1 = a.bt.vbegin[b + 1];
        }
        const int L = a.bt.lanes[b];
        const int64_t lb = blk - bb0;
        // threads per row: L streams, each of Q = k/8 lanes for k >= 32
        const int T = K >= 32 ? L * (K / 8) : L;
        const int vpb = T >= kBlock ? 1 : kBlock / T;
        const int64_t vi = vb0 + lb * vpb + threadIdx.x / T;
        const bool valid = vi < vb1;
        Outcome o;
        if constexpr (K >= 32) {
            switch (L) {  // the host caps L at 32 for these sketch sizes
                case 1: o = slot_body<1, K, VT, U>(a, vi, valid, sm); break;
                case 2: o = slot_body<2, K, VT, U>(a, vi, valid, sm); break;
                case 4: o = slot_body<4, K, VT, U>(a, vi, valid, sm); break;
                case 8: o = slot_body<8, K, VT, U>(a, vi, valid, sm); break;
                case 16: o = slot_body<16, K, VT, U>(a, vi, valid, sm); break;
                default: o = slot_body<32, K, VT, U>(a, vi, valid, sm); break;
            }
        } else {
            switch (L) {
                case 1: o = group_body<1, K, VT, U>(a, vi, valid, tabs_of(sm)); break;
                case 2: o = group_body<2, K, VT, U>(a, vi, valid, tabs_of(sm)); break;
                case 4: o = group_body<4, K, VT, U>(a, vi, valid, tabs_of(sm)); break;
                case 8: o = group_body<8, K, VT, U>(a, vi, valid, tabs_of(sm)); break;
                case 16: o = group_body<16, K, VT, U>(a, vi, valid, tabs_of(sm)); break;
                case 32: o = group_body<32, K, VT, U>(a, vi, valid, tabs_of(sm)); break;
                case 64: o = block_body<64, K, VT, U>(a, vi, valid, sm.b); break;
                case 128: o = block_body<128, K, VT, U>(a, vi, valid, sm.b); break;
                default: o = block_body<256, K, VT, U>(a, vi, valid, sm.b); break;
            }
        }
        block_epilogue(a, o, esm);
    }
}

// ---------------------------------------------------------------------------
// MG aggregation (Section 4.1, "aggregation phase"; Fig. 3): one sketch per
// community over the edges of all its members (ascending vertex id, each row
// in CSR order, self-loops kept), streams and merge tree as in the sweep;
// no second pass.  The community's sketch is written to out_keys/out_vals
// (K slots per community).  a.labels holds the dense community ids; the
// buckets list communities, a.off gives their member ranges in `members`.
// ---------------------------------------------------------------------------
template <int K, typename VT, typename F>
__device__ __forceinline__ void for_members(const AggArgs& g, uint32_t c, int lane, int L, F&& f) {
    for (int64_t q = g.moff[c]; q < g.moff[c + 1]; ++q) {
        const uint32_t m = g.members[q];
        const int64_t start = g.a.off[m], end = g.a.off[m + 1];
        if (L == 1) {
            for_row(g.a, start, end, kEmpty, 0u, f);
        } else {
            const int64_t c0 = start >> 2, c1 = (end + 3) >> 2;
            const int64_t first = c0 + (int64_t)((lane - (int)(c0 & (L - 1))) & (L - 1));
            scan_chunks(g.a, first, c1, L, start, end, kEmpty, 0u, f);
        }
    }
}

template <int K, typename VT>
__device__ __forceinline__ void agg_store(const AggArgs& g, uint32_t c, const Sketch<K, VT>& sk) {
#pragma unroll
    for (int p = 0; p < K; ++p) {
        const VT v = sk.value(p);
        g.out_keys[(size_t)c * K + p] = v > 0 ? sk.key[p] : kEmpty;
        g.out_vals[(size_t)c * K + p] = (unsigned long long)v;
    }
}

template <int G, int K, typename VT>
__device__ __forceinline__ void agg_group(const AggArgs& g, int64_t vi, bool valid) {
    const int lane = threadIdx.x & (G - 1);
    const unsigned gmask = (G == 32) ? 0xffffffffu
                                     : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
    const int unc = g.a.uncond;
    Sketch<K, VT> sk;
    sk.init();
    uint32_t c = 0;
    if (valid) {
        c = g.a.verts[vi];
        for_members<K, VT>(g, c, lane, G, [&](uint32_t key, uint32_t w) { sk.update(key, (VT)w, unc); });
    }
    group_merge<G, K, VT>(sk, lane, gmask, unc);
    if (valid && lane == 0) agg_store(g, c, sk);
}

template <int L, int K, typename VT>
__device__ __forceinline__ void agg_block(const AggArgs& g, int64_t vi, bool valid, BlockSmem<K, VT>& sm) {
    const int sb = threadIdx.x / L;
    const int s = threadIdx.x % L;
    const int unc = g.a.uncond;
    Sketch<K, VT> sk;
    sk.init();
    uint32_t c = 0;
    if (valid) {
        c = g.a.verts[vi];
        for_members<K, VT>(g, c, s, L, [&](uint32_t key, uint32_t w) { sk.update(key, (VT)w, unc); });
    }
    block_merge<L, K, VT, int>(sk, s, sb, 1 + sb, sm, unc);
    if (valid && s == 0) agg_store(g, c, sk);
}

template <int K, typename VT>
__global__ void __launch_bounds__(kBlock, (K >= 16 || sizeof(VT) == 8) ? 2 : 4) k_agg_mg(const AggArgs g) {
    __shared__ BlockSmem<K, VT> sm;
    const int64_t blk = (int64_t)gridDim.x - 1 - (int64_t)blockIdx.x;
    int b = 0;
#pragma unroll
    for (int q = 1; q < CD_MAX_BUCKETS; ++q)
        if (q < g.a.bt.nb && blk >= g.a.bt.bbegin[q]) b = q;
    const int L = g.a.bt.lanes[b];
    const int64_t lb = blk - g.a.bt.bbegin[b];
    const int vpb = L >= kBlock ? 1 : kBlock / L;
    const int64_t vi = g.a.bt.vbegin[b] + lb * vpb + threadIdx.x / L;
    const bool valid = vi < g.a.bt.vbegin[b + 1];
    switch (L) {
        case 1: agg_group<1, K, VT>(g, vi, valid); break;
        case 2: agg_group<2, K, VT>(g, vi, valid); break;
        case 4: agg_group<4, K, VT>(g, vi, valid); break;
        case 8: agg_group<8, K, VT>(g, vi, valid); break;
        case 16: agg_group<16, K, VT>(g, vi, valid); break;
        case 32: agg_group<32, K, VT>(g, vi, valid); break;
        case 64: agg_block<64, K, VT>(g, vi, valid, sm); break;
        case 128: agg_block<128, K, VT>(g, vi, valid, sm); break;
        default: agg_block<256, K, VT>(g, vi, valid, sm); break;
    }
}

template <int K>
cudaError_t launch_agg_k(const AggArgs& g, bool wide, int64_t nblocks, cudaStream_t s) {
    if (nblocks == 0) return cudaSuccess;
    note_launch();  // one of the two branches launches
    if (wide) k_agg_mg<K, unsigned long long><<<(unsigned)nblocks, kBlock, 0, s>>>(g);
    else k_agg_mg<K, uint32_t><<<(unsigned)nblocks, kBlock, 0, s>>>(g);
    return cudaGetLastError();
}

template <int K, typename VT, typename U>
cudaError_t launch_k_mode(const SweepArgs& a, int64_t nblocks, cudaStream_t s) {
    note_launch();
    k_sweep_mg<K, VT, U><<<(unsigned)nblocks, kBlock, 0, s>>>(a);
    return cudaGetLastError();
}

// subtract = 2 (the textbook summary) is compiled for k <= 8 only
template <int K, typename VT>
cudaError_t launch_k_vt(const SweepArgs& a, int64_t nblocks, cudaStream_t s) {
    if (a.uncond == 2) {
        if constexpr (K <= 8) return launch_k_mode<K, VT, TextbookMG>(a, nblocks, s);
        else return cudaErrorInvalidValue;
    }
    return launch_k_mode<K, VT, int>(a, nblocks, s);
}

template <int K>
cudaError_t launch_k(const SweepArgs& a, bool wide, int64_t nblocks, cudaStream_t s) {
    if (wide) return launch_k_vt<K, unsigned long long>(a, nblocks, s);
    return launch_k_vt<K, uint32_t>(a, nblocks, s);
}

}  // namespace cdk
