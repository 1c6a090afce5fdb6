// cd_modularity_noalloc: the modularity computation of cd_modularity with its
// device scratch (weighted degrees, community totals, community sizes and the
// call's scalars) in one fixed array of this file instead of cudaMallocAsync.
//
// Every GPU that loads the library holds the array until the process exits.
// Host code cannot use the array's name as a device address, so the address is
// looked up once per device with cudaGetSymbolAddress and cached.
#include <mutex>

#include "cd_internal.cuh"

namespace cdk {
void record_cuda_error(cudaError_t e);
void begin_call_stats();
void record_modularity(double q);
}

using namespace cdk;

namespace {

constexpr int64_t kNoAllocMaxN = int64_t(1) << 20;  // vertices
constexpr size_t kHeadBytes = 256;                  // Globals, padded
constexpr size_t kNoAllocBytes =
    kHeadBytes + (size_t)kNoAllocMaxN * (sizeof(uint64_t) + sizeof(uint64_t) + sizeof(uint32_t));

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

static_assert(sizeof(Globals) <= kHeadBytes, "Globals must fit the head of the scratch array");

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {};

// Device address of the array on the current device (looked up on first use).
int scratch_address(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        record_cuda_error(e);
        return CD_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return CD_EINVAL;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            record_cuda_error(e);
            return CD_ECUDA;
        }
        g_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_addr[dev];
    return CD_OK;
}

int fail(cudaError_t e) {
    record_cuda_error(e);
    return CD_ECUDA;
}

}  // namespace

extern "C" int cd_modularity_noalloc(const cd_csr* g, const uint32_t* labels, void* stream, double* q_out,
                                     cd_modularity_parts* parts) {
    begin_call_stats();
    if (!g || !labels) return CD_EINVAL;
    if (g->memory != CD_MEM_DEVICE) return CD_EINVAL;
    if (g->n < 0 || g->nnz < 0 || !g->offsets || (g->nnz > 0 && (!g->cols || !g->weights))) return CD_EINVAL;
    if (g->n > kNoAllocMaxN) return CD_ESIZE;
    unsigned char* base = nullptr;
    int rc = scratch_address(&base);
    if (rc != CD_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    Globals* glob = reinterpret_cast<Globals*>(base);
    uint64_t* K = reinterpret_cast<uint64_t*>(base + kHeadBytes);
    uint64_t* Sigma = K + kNoAllocMaxN;
    uint32_t* sizes = reinterpret_cast<uint32_t*>(Sigma + kNoAllocMaxN);
    // the array keeps the previous call's contents: clear the scalars; K,
    // Sigma and sizes are cleared by the launches that fill them
    cudaError_t e = cudaMemsetAsync(glob, 0, sizeof(Globals), s);
    if (e != cudaSuccess) return fail(e);
    if (g->n > 0) {
        e = launch_degrees(g->offsets, g->weights, g->n, g->nnz, K, glob, s);
        if (e != cudaSuccess) return fail(e);
        e = launch_modularity(g->offsets, g->cols, g->weights, labels, g->n, g->nnz, K, Sigma, sizes, glob, s);
        if (e != cudaSuccess) return fail(e);
    }
    Globals h;
    e = cudaMemcpyAsync(&h, glob, sizeof(Globals), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(e);
    if (h.err) return CD_EINVAL;
    u128 sq = ((u128)h.sq_hi << 64) | (u128)h.sq_lo;
    u128 tm = h.two_m;
    double q = 0.0;
    if (tm > 0) {
        i128 num = (i128)(tm * (u128)h.sigma_in) - (i128)sq;
        q = (double)((long double)num / ((long double)tm * (long double)tm));
    }
    if (parts) {
        parts->sigma_in = h.sigma_in;
        parts->sum_sq_lo = h.sq_lo;
        parts->sum_sq_hi = h.sq_hi;
        parts->two_m = h.two_m;
    }
    record_modularity(q);
    if (q_out) *q_out = q;
    return CD_OK;
}
