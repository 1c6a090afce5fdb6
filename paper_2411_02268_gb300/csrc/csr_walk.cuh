// Warp-cooperative walk over a range of CSR entries with the row of every
// entry: lane l takes entries e0 + l, e0 + l + 32, ... (coalesced), and the
// rows come from 32 consecutive row ends held one per lane and searched with
// shuffles, instead of a binary search over all rows per entry or per chunk.
#pragma once

#include <cstdint>

#include "cd_internal.cuh"

namespace cdk {

// Largest r in [0, n) with off[r] <= e (the row holding entry e, skipping
// empty rows); e must be < off[n].
__device__ __forceinline__ int64_t row_of_entry(const int64_t* __restrict__ off, int64_t n, int64_t e) {
    int64_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (off[mid] <= e) lo = mid; else hi = mid;
    }
    return lo;
}

// Calls f(e, row) for every entry e in [e0, e1), lane by lane in steps of
// 32; every lane of the warp must call it with the same range.  Returns false
// (on every lane) when the offsets do not cover the entries (off[n] <= some
// e, or offsets out of order): the walk then stops without reading past the
// arrays.
// With kAllLanes, f(e, row, valid) is called on every lane at every step (for
// warp collectives inside f; row is meaningful only where valid).
template <bool kAllLanes = false, typename F>
__device__ __forceinline__ bool warp_walk(const int64_t* __restrict__ off, int64_t n, int64_t e0, int64_t e1,
                                          F&& f) {
    if (e0 >= e1) return true;
    const int lane = threadIdx.x & 31;
    int64_t base = 0;
    if (lane == 0) base = row_of_entry(off, n, e0);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (int64_t eb = e0; eb < e1; eb += 32) {
        const int64_t e = eb + lane;
        const bool valid = e < e1;
        int64_t row = -1;
        for (int64_t rb = base; rb < n; rb += 32) {  // off[rb] <= every entry of this step
            // ends of rows rb .. rb + 31
            const int64_t q = rb + 1 + lane;
            const int64_t bnd = q <= n ? off[q] : INT64_MAX;
            // number of those ends <= e, by a search over the lanes' values
            int pos = 0;
#pragma unroll
            for (int st = 16; st >= 1; st >>= 1) {
                const int64_t v = __shfl_sync(0xffffffffu, bnd, pos + st - 1);
                if (v <= e) pos += st;
            }
            const int64_t last = __shfl_sync(0xffffffffu, bnd, pos);
            if (last <= e) ++pos;
            if (valid && row < 0 && pos < 32) row = rb + pos;
            if (__all_sync(0xffffffffu, !valid || row >= 0)) break;
        }
        const bool bad = valid && (row < 0 || row >= n);
        if (__any_sync(0xffffffffu, bad)) return false;
        if constexpr (kAllLanes) f(e, row, valid);
        else if (valid) f(e, row);
        const int tail = (int)((e1 - eb) < 32 ? (e1 - eb) - 1 : 31);
        base = __shfl_sync(0xffffffffu, row, tail);
    }
    return true;
}

}  // namespace cdk
