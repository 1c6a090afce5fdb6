// Exclusive prefix sums over device arrays (three phases: tile sums, a scan
// of the tile sums in one block, tile scans offset by their prefix).  Used by
// community renumbering and the super-vertex graph construction.
#include "cd_internal.cuh"

namespace cdk {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;  // 4096

int64_t scan_tiles(int64_t n) { return (n + kScanTile - 1) / kScanTile; }

template <typename T>
__device__ __forceinline__ T block_exclusive(T v, T* sh, T* total) {
    // sh: kScanThreads entries
    const int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int o = 1; o < kScanThreads; o <<= 1) {
        T x = t >= o ? sh[t - o] : (T)0;
        __syncthreads();
        sh[t] += x;
        __syncthreads();
    }
    T incl = sh[t];
    if (total) *total = sh[kScanThreads - 1];
    __syncthreads();
    return incl - v;
}

template <typename T, typename S>
__global__ void k_tile_sums(const T* __restrict__ in, int64_t n, S* __restrict__ sums) {
    __shared__ S sh[kScanThreads];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    S s = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q)
        if (base + q < n) s += (S)in[base + q];
    S tot;
    block_exclusive<S>(s, sh, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// One block scans the tile sums in place (exclusive) and stores the total.
template <typename S>
__global__ void k_scan_sums(S* __restrict__ sums, int64_t m, S* __restrict__ total) {
    __shared__ S sh[kScanThreads];
    S carry = 0;
    for (int64_t base = 0; base < m; base += kScanThreads) {
        int64_t i = base + threadIdx.x;
        S v = i < m ? sums[i] : (S)0;
        S tot;
        S ex = block_exclusive<S>(v, sh, &tot);
        if (i < m) sums[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *total = carry;
}

template <typename T, typename S, typename O>
__global__ void k_tile_scan(const T* __restrict__ in, int64_t n, const S* __restrict__ sums, O* __restrict__ out) {
    __shared__ S sh[kScanThreads];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    T v[kScanItems];
    S s = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        v[q] = base + q < n ? in[base + q] : (T)0;
        s += (S)v[q];
    }
    S run = block_exclusive<S>(s, sh, nullptr) + sums[blockIdx.x];
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        if (base + q < n) out[base + q] = (O)run;
        run += (S)v[q];
    }
}

// out[i] = sum of in[0..i); *total_dev = sum of all.  tile_scratch needs
// scan_tiles(n) entries.  in and out may alias.
cudaError_t launch_exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n,
                                      unsigned long long* tile_scratch, unsigned long long* total_dev,
                                      cudaStream_t s) {
    if (n == 0) return cudaMemsetAsync(total_dev, 0, sizeof(unsigned long long), s);
    int64_t nt = scan_tiles(n);
    note_launch();
    k_tile_sums<uint32_t, unsigned long long><<<(unsigned)nt, kScanThreads, 0, s>>>(in, n, tile_scratch);
    note_launch();
    k_scan_sums<unsigned long long><<<1, kScanThreads, 0, s>>>(tile_scratch, nt, total_dev);
    note_launch();
    k_tile_scan<uint32_t, unsigned long long, uint32_t><<<(unsigned)nt, kScanThreads, 0, s>>>(in, n, tile_scratch,
                                                                                           out);
    return cudaGetLastError();
}

cudaError_t launch_exclusive_scan_u32_to_i64(const uint32_t* in, int64_t* out, int64_t n,
                                             unsigned long long* tile_scratch, unsigned long long* total_dev,
                                             cudaStream_t s) {
    if (n == 0) return cudaMemsetAsync(total_dev, 0, sizeof(unsigned long long), s);
    int64_t nt = scan_tiles(n);
    note_launch();
    k_tile_sums<uint32_t, unsigned long long><<<(unsigned)nt, kScanThreads, 0, s>>>(in, n, tile_scratch);
    note_launch();
    k_scan_sums<unsigned long long><<<1, kScanThreads, 0, s>>>(tile_scratch, nt, total_dev);
    note_launch();
    k_tile_scan<uint32_t, unsigned long long, int64_t><<<(unsigned)nt, kScanThreads, 0, s>>>(in, n, tile_scratch,
                                                                                          out);
    return cudaGetLastError();
}

}  // namespace cdk
