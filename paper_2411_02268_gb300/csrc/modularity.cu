// Modularity (Eq. 1, Section 3.2) in exact integers:
//   Q = (2m * sum_c sigma_c - sum_c Sigma_c^2) / (2m)^2,
// sum_c sigma_c = sum of w over CSR entries (i, j) with C_i = C_j, and
// Sigma_c = sum of K_i over the members of c.
#include "cd_internal.cuh"
#include "csr_walk.cuh"

namespace cdk {

constexpr int64_t kQTile = 4096;  // CSR entries per warp

// sum_c sigma_c: one warp per 4096-entry tile walks the entries with their
// rows (csr_walk.cuh), coalesced.
__global__ void k_sigma_in(const int64_t* __restrict__ off, const int32_t* __restrict__ cols,
                           const uint32_t* __restrict__ w, const uint32_t* __restrict__ labels, int64_t n,
                           int64_t nnz, Globals* glob) {
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t e0 = warp * kQTile;
    if (e0 >= nnz) return;  // the whole warp
    const int64_t e1 = e0 + kQTile < nnz ? e0 + kQTile : nnz;
    unsigned long long sum = 0;
    bool badcol = false;
    const bool ok = warp_walk(off, n, e0, e1, [&](int64_t e, int64_t r) {
        const uint32_t j = (uint32_t)cols[e];
        if (j >= (uint32_t)n) { badcol = true; return; }
        if (__ldg(labels + j) == labels[r]) sum += w[e];
    });
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
    const int lane = threadIdx.x & 31;
    if (lane == 0 && sum) atomicAdd(&glob->sigma_in, sum);
    if (lane == 0 && !ok) atomicOr(&glob->err, kErrBadOffsets);
    if (badcol) atomicOr(&glob->err, kErrBadCol);
}

// sum_c Sigma_c^2 as a 128-bit integer (two 64-bit halves with carry).
__global__ void k_sum_sq(const unsigned long long* __restrict__ Sigma, int64_t n, Globals* glob) {
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    u128 sq = 0;
    if (c < n) {
        unsigned long long s = Sigma[c];
        sq = (u128)s * (u128)s;
    }
    unsigned long long lo = (unsigned long long)sq, hi = (unsigned long long)(sq >> 64);
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        unsigned long long l2 = __shfl_down_sync(0xffffffffu, lo, o);
        unsigned long long h2 = __shfl_down_sync(0xffffffffu, hi, o);
        unsigned long long nl = lo + l2;
        hi = hi + h2 + (nl < lo ? 1ull : 0ull);
        lo = nl;
    }
    if ((threadIdx.x & 31) == 0 && (lo | hi)) {
        unsigned long long old = atomicAdd(&glob->sq_lo, lo);
        unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
        if (hi + carry) atomicAdd(&glob->sq_hi, hi + carry);
    }
}

// Sigma_scratch: n entries; sizes_scratch: n entries.  glob->two_m, sigma_in,
// sq_lo and sq_hi must be zero on entry.
cudaError_t launch_modularity(const int64_t* off, const int32_t* cols, const uint32_t* w,
                              const uint32_t* labels, int64_t n, int64_t nnz, const uint64_t* K,
                              uint64_t* Sigma_scratch, uint32_t* sizes_scratch, Globals* glob,
                              cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    cudaError_t e = launch_totals(labels, K, n, Sigma_scratch, sizes_scratch, glob, s);
    if (e != cudaSuccess) return e;
    if (nnz > 0) {
        const int64_t warps = (nnz + kQTile - 1) / kQTile;
        note_launch();
        k_sigma_in<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(off, cols, w, labels, n, nnz, glob);
    }
    note_launch();
    k_sum_sq<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((const unsigned long long*)Sigma_scratch, n, glob);
    return cudaGetLastError();
}

}  // namespace cdk
