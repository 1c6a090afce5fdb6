// Host side of the C ABI (include/cd.h): argument checks, stream-ordered
// scratch, the launch sequence of one sweep, modularity, and host-memory
// staging.  Every entry point returns a status code and never aborts.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "cd_internal.cuh"

using namespace cdk;

namespace {

thread_local cd_stats g_stats;

void reset_stats() {
    std::memset(&g_stats, 0, sizeof(g_stats));
}

int cuda_fail(cudaError_t e) {
    std::snprintf(g_stats.cuda_error, sizeof(g_stats.cuda_error), "%s", cudaGetErrorString(e));
    cudaGetLastError();  // clear a sticky launch error of this thread
    return e == cudaErrorMemoryAllocation ? CD_ENOMEM : CD_ECUDA;
}

#define CD_CUDA(x)                                   \
    do {                                             \
        cudaError_t _e = (x);                        \
        if (_e != cudaSuccess) return cuda_fail(_e); \
    } while (0)

#define CD_TRY(x)                   \
    do {                            \
        int _rc = (x);              \
        if (_rc != CD_OK) return _rc; \
    } while (0)

// Stream-ordered device scratch of one call; everything is released (in stream
// order) when the object goes out of scope.
struct Scratch {
    cudaStream_t s;
    std::vector<void*> ptrs;
    int64_t bytes = 0;
    explicit Scratch(cudaStream_t st) : s(st) {}
    ~Scratch() {
        for (void* p : ptrs) cudaFreeAsync(p, s);
        if (bytes > g_stats.scratch_bytes) g_stats.scratch_bytes = bytes;
    }
    template <typename T>
    int get(T** p, int64_t count) {
        size_t nb = sizeof(T) * (size_t)(count > 0 ? count : 1);
        nb = (nb + 255) & ~(size_t)255;
        void* q = nullptr;
        cudaError_t e = cudaMallocAsync(&q, nb, s);
        if (e != cudaSuccess) return cuda_fail(e);
        ptrs.push_back(q);
        bytes += (int64_t)nb;
        *p = static_cast<T*>(q);
        return CD_OK;
    }
};

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int check_csr(const cd_csr* g) {
    if (!g) return CD_EINVAL;
    if (g->n < 0 || g->n >= 0x7FFFFFFFLL || g->nnz < 0) return CD_EINVAL;
    if (g->memory != CD_MEM_DEVICE && g->memory != CD_MEM_HOST) return CD_EINVAL;
    if (!g->offsets) return CD_EINVAL;
    if (g->nnz > 0 && (!g->cols || !g->weights)) return CD_EINVAL;
    if (g->memory == CD_MEM_DEVICE && g->nnz > 0 && (!aligned16(g->cols) || !aligned16(g->weights)))
        return CD_EINVAL;
    if (g->memory == CD_MEM_HOST) {
        // full structural check on the host
        const int64_t* off = g->offsets;
        if (off[0] != 0 || off[g->n] != g->nnz) return CD_EINVAL;
        for (int64_t i = 0; i < g->n; ++i)
            if (off[i + 1] < off[i]) return CD_EINVAL;
        for (int64_t e = 0; e < g->nnz; ++e)
            if (g->cols[e] < 0 || g->cols[e] >= g->n || g->weights[e] == 0) return CD_EINVAL;
    }
    return CD_OK;
}

void default_schedule(cd_schedule* s) {
    // Streams per row by row length: one stream up to 32 entries, then about
    // 16-128 entries per stream so that the merge tree stays cheaper than the
    // scan; narrow length bands keep the groups of one warp balanced.
    static const int64_t dm[] = {2, 4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048, 4096, 8192, 32768,
                                 INT64_MAX};
    static const int32_t ln[] = {1, 1, 1, 1, 1, 2, 2, 4, 4, 8, 8, 16, 32, 128, 256};
    std::memset(s, 0, sizeof(*s));
    s->nbuckets = 15;
    s->vec = 4;
    for (int b = 0; b < 15; ++b) { s->deg_max[b] = dm[b]; s->lanes[b] = ln[b]; }
}

int check_schedule(const cd_schedule* s) {
    if (s->nbuckets < 1 || s->nbuckets > CD_MAX_BUCKETS || s->vec != 4) return CD_EINVAL;
    for (int b = 0; b < s->nbuckets; ++b) {
        int L = s->lanes[b];
        if (L < 1 || L > 256 || (L & (L - 1))) return CD_EINVAL;
        if (s->deg_max[b] < 1) return CD_EINVAL;
        if (b > 0 && s->deg_max[b] <= s->deg_max[b - 1]) return CD_EINVAL;
    }
    return CD_OK;
}

int check_params(const cd_params* p) {
    if (!p) return CD_EINVAL;
    if (!(p->k == 0 || p->k == 1 || p->k == 2 || p->k == 4 || p->k == 8 || p->k == 16)) return CD_EINVAL;
    if (p->subtract != 0 && p->subtract != 1) return CD_EINVAL;
    if (p->sched) CD_TRY(check_schedule(p->sched));
    return CD_OK;
}

// The exact-hashtable sweep splits rows by the size of their table: groups of
// G lanes share a shared-memory table of 2*deg_max slots (48 KB per block), a
// block takes one row with a shared table up to 2048 entries, and longer rows
// use tables in device scratch.
struct ExactBucket { int64_t deg_max; int G; uint32_t T; int global; };
const ExactBucket kExact[] = {
    {8, 1, 16, 0},    {16, 2, 32, 0},    {32, 4, 64, 0},      {64, 8, 128, 0},
    {128, 16, 256, 0}, {256, 32, 512, 0}, {2048, 256, 4096, 0}, {INT64_MAX, 256, 0, 1},
};
constexpr int kExactBuckets = 8;

BucketTable table_from(const cd_schedule& s) {
    BucketTable bt;
    std::memset(&bt, 0, sizeof(bt));
    bt.nb = s.nbuckets;
    for (int b = 0; b < s.nbuckets; ++b) { bt.deg_max[b] = s.deg_max[b]; bt.lanes[b] = s.lanes[b]; }
    return bt;
}

BucketTable exact_table() {
    BucketTable bt;
    std::memset(&bt, 0, sizeof(bt));
    bt.nb = kExactBuckets;
    for (int b = 0; b < kExactBuckets; ++b) { bt.deg_max[b] = kExact[b].deg_max; bt.lanes[b] = kExact[b].G; }
    return bt;
}

// Device state of one graph during a pass.
struct Level {
    int64_t n = 0, nnz = 0;
    const int64_t* off = nullptr;
    const int32_t* cols = nullptr;
    const uint32_t* w = nullptr;
    uint64_t* K = nullptr;
    uint64_t* Sigma = nullptr;
    uint32_t* size = nullptr;
    uint32_t* verts = nullptr;
    uint32_t* movers = nullptr;
    BucketTable bt;
    bool wide = false;  // sketch values need 64 bits
    unsigned long long two_m = 0;
};

struct HostGlobals {
    Globals g;
    int64_t starts[CD_MAX_BUCKETS + 1];
};

int read_globals(Globals* dglob, int64_t* dstarts, int nb, HostGlobals* out, cudaStream_t s) {
    CD_CUDA(cudaMemcpyAsync(&out->g, dglob, sizeof(Globals), cudaMemcpyDeviceToHost, s));
    if (dstarts) CD_CUDA(cudaMemcpyAsync(out->starts, dstarts, sizeof(int64_t) * (nb + 1),
                                         cudaMemcpyDeviceToHost, s));
    CD_CUDA(cudaStreamSynchronize(s));
    unsigned err = out->g.err;
    if (err) return CD_EINVAL;
    return CD_OK;
}

// K, totals from `labels`, buckets; reads back 2m, max K and bucket sizes.
int prepare_level(Level& L, const uint32_t* labels, uint32_t* labels_out_copy, bool exact,
                  const cd_schedule& sched, Scratch& sc, Globals* dglob, cudaStream_t s) {
    CD_TRY(sc.get(&L.K, L.n));
    CD_TRY(sc.get(&L.Sigma, L.n));
    CD_TRY(sc.get(&L.size, L.n));
    CD_TRY(sc.get(&L.verts, L.n));
    L.bt = exact ? exact_table() : table_from(sched);
    int64_t ntiles = bucket_tiles(L.n);
    uint32_t *tc, *to;
    int64_t* starts;
    CD_TRY(sc.get(&tc, ntiles * L.bt.nb));
    CD_TRY(sc.get(&to, ntiles * L.bt.nb));
    CD_TRY(sc.get(&starts, CD_MAX_BUCKETS + 1));
    CD_CUDA(cudaMemsetAsync(dglob, 0, sizeof(Globals), s));
    CD_CUDA(launch_degrees(L.off, L.w, L.n, L.nnz, L.K, dglob, s));
    CD_CUDA(launch_totals(labels, L.K, L.n, L.Sigma, L.size, dglob, s));
    CD_CUDA(launch_bucket(L.off, L.n, L.nnz, L.bt, tc, to, starts, L.verts, labels, labels_out_copy,
                          dglob, s));
    HostGlobals hg;
    CD_TRY(read_globals(dglob, starts, L.bt.nb, &hg, s));
    L.two_m = hg.g.two_m;
    if (L.two_m >= (1ull << 62)) return CD_EOVERFLOW;
    L.wide = hg.g.max_k >= (1ull << 32);
    int64_t blk = 0;
    for (int b = 0; b < L.bt.nb; ++b) {
        L.bt.vbegin[b] = hg.starts[b];
        L.bt.bbegin[b] = blk;
        int64_t nv = (b + 1 < L.bt.nb ? hg.starts[b + 1] : hg.starts[L.bt.nb]) - hg.starts[b];
        int Lb = L.bt.lanes[b];
        int vpb = Lb >= kBlock ? 1 : kBlock / Lb;
        blk += (nv + vpb - 1) / vpb;
    }
    L.bt.vbegin[L.bt.nb] = hg.starts[L.bt.nb];
    L.bt.bbegin[L.bt.nb] = blk;
    return CD_OK;
}

SweepArgs make_args(const Level& L, const uint32_t* labels_in, uint32_t* labels_out, const uint8_t* active,
                    const uint32_t* bound, Globals* dglob, int mode, int uncond) {
    SweepArgs a;
    std::memset(&a, 0, sizeof(a));
    a.off = L.off; a.cols = L.cols; a.w = L.w;
    a.labels = labels_in; a.K = L.K; a.Sigma = L.Sigma; a.size = L.size;
    a.active = active; a.bound = bound; a.labels_out = labels_out; a.movers = L.movers;
    a.glob = dglob; a.verts = L.verts; a.n = L.n; a.nnz = L.nnz; a.mode = mode; a.uncond = uncond;
    a.bt = L.bt;
    return a;
}

// Launches one sweep (all buckets) on stream s.
int launch_sweep(const Level& L, const SweepArgs& a, int k, Scratch& sc, cudaStream_t s) {
    if (k > 0) {
        CD_CUDA(launch_sweep_mg(a, k, L.wide, L.bt.bbegin[L.bt.nb], s));
        return CD_OK;
    }
    for (int b = 0; b < kExactBuckets; ++b) {
        const ExactBucket& eb = kExact[b];
        int64_t nv = L.bt.vbegin[b + 1] - L.bt.vbegin[b];
        if (nv == 0) continue;
        if (!eb.global) {
            if (eb.G <= 32) CD_CUDA(launch_exact_group(a, b, eb.G, eb.T, s));
            else CD_CUDA(launch_exact_block(a, b, eb.T, nullptr, nullptr, nullptr, s));
            continue;
        }
        // rows too long for shared memory: per-row tables in device scratch
        int64_t* sizes;
        CD_TRY(sc.get(&sizes, nv));
        CD_CUDA(launch_exact_table_sizes(a, b, sizes, s));
        std::vector<int64_t> hs((size_t)nv), hoff((size_t)nv + 1);
        CD_CUDA(cudaMemcpyAsync(hs.data(), sizes, sizeof(int64_t) * nv, cudaMemcpyDeviceToHost, s));
        CD_CUDA(cudaStreamSynchronize(s));
        hoff[0] = 0;
        for (int64_t q = 0; q < nv; ++q) hoff[q + 1] = hoff[q] + hs[q];
        int64_t* doff;
        uint32_t* gk;
        unsigned long long* gv;
        CD_TRY(sc.get(&doff, nv + 1));
        CD_TRY(sc.get(&gk, hoff[nv]));
        CD_TRY(sc.get(&gv, hoff[nv]));
        CD_CUDA(cudaMemcpyAsync(doff, hoff.data(), sizeof(int64_t) * (nv + 1), cudaMemcpyHostToDevice, s));
        CD_CUDA(launch_exact_block(a, b, 0, gk, gv, doff, s));
        CD_CUDA(cudaStreamSynchronize(s));  // hoff must outlive the copy
    }
    return CD_OK;
}

// Copies a host array into stream-ordered scratch.
template <typename T>
int stage_in(const T* host, int64_t count, T** dev, Scratch& sc) {
    CD_TRY(sc.get(dev, count));
    if (count > 0) CD_CUDA(cudaMemcpyAsync(*dev, host, sizeof(T) * count, cudaMemcpyHostToDevice, sc.s));
    return CD_OK;
}

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    bool on = false;
    int init(bool enable) {
        on = enable;
        if (!on) return CD_OK;
        CD_CUDA(cudaEventCreate(&a));
        CD_CUDA(cudaEventCreate(&b));
        return CD_OK;
    }
    ~Timer() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

}  // namespace

extern "C" {

const char* cd_strerror(int code) {
    switch (code) {
        case CD_OK: return "ok";
        case CD_EINVAL: return "invalid argument";
        case CD_ENOMEM: return "out of memory";
        case CD_ECUDA: return "CUDA error";
        case CD_ETIMEOUT: return "device wait timed out";
        case CD_EOVERFLOW: return "integer overflow";
        case CD_ENOTIMPL: return "not implemented";
        default: return "unknown status";
    }
}

int cd_last_stats(cd_stats* out) {
    if (!out) return CD_EINVAL;
    *out = g_stats;
    return CD_OK;
}

int cd_default_schedule(int k, cd_schedule* out) {
    if (!out || k < 0) return CD_EINVAL;
    default_schedule(out);
    return CD_OK;
}

int cd_sweep(const cd_csr* g, const cd_params* p, int mode, const uint32_t* labels_in,
             const uint8_t* active, const uint32_t* bound, uint32_t* labels_out, int64_t* moved_out,
             uint64_t* gain_out) {
    reset_stats();
    CD_TRY(check_csr(g));
    CD_TRY(check_params(p));
    if (mode != CD_MODE_LOUVAIN && mode != CD_MODE_LPA) return mode == CD_MODE_REFINE ? CD_ENOTIMPL : CD_EINVAL;
    if (!labels_in || !labels_out || labels_in == labels_out) return CD_EINVAL;
    cudaStream_t s = (cudaStream_t)p->stream;
    cd_schedule sched;
    if (p->sched) sched = *p->sched; else default_schedule(&sched);
    const bool host = g->memory == CD_MEM_HOST;
    if (host) {
        for (int64_t i = 0; i < g->n; ++i)
            if ((int64_t)labels_in[i] >= g->n) return CD_EINVAL;
    }
    Scratch sc(s);
    Level L;
    L.n = g->n;
    L.nnz = g->nnz;
    const uint32_t* lin = labels_in;
    uint32_t* lout = labels_out;
    const uint8_t* act = active;
    if (host) {
        int64_t *off; int32_t* cols; uint32_t* w; uint32_t* li;
        CD_TRY(stage_in(g->offsets, g->n + 1, &off, sc));
        CD_TRY(stage_in(g->cols, g->nnz, &cols, sc));
        CD_TRY(stage_in(g->weights, g->nnz, &w, sc));
        CD_TRY(stage_in(labels_in, g->n, &li, sc));
        CD_TRY(sc.get(&lout, g->n));
        if (active) { uint8_t* da; CD_TRY(stage_in(active, g->n, &da, sc)); act = da; }
        L.off = off; L.cols = cols; L.w = w; lin = li;
    } else {
        L.off = g->offsets; L.cols = g->cols; L.w = g->weights;
    }
    Globals* dglob;
    CD_TRY(sc.get(&dglob, 1));
    if (L.n == 0) {
        if (moved_out) *moved_out = 0;
        if (gain_out) { gain_out[0] = 0; gain_out[1] = 0; }
        return CD_OK;
    }
    CD_TRY(prepare_level(L, lin, lout, p->k == 0, sched, sc, dglob, s));
    SweepArgs a = make_args(L, lin, lout, act, bound, dglob, mode, p->subtract);
    Timer tm;
    CD_TRY(tm.init(p->timing != 0));
    if (tm.on) CD_CUDA(cudaEventRecord(tm.a, s));
    CD_TRY(launch_sweep(L, a, p->k, sc, s));
    if (tm.on) CD_CUDA(cudaEventRecord(tm.b, s));
    if (host) CD_CUDA(cudaMemcpyAsync(labels_out, lout, sizeof(uint32_t) * g->n, cudaMemcpyDeviceToHost, s));
    HostGlobals hg;
    CD_TRY(read_globals(dglob, nullptr, 0, &hg, s));
    if (tm.on) {
        float ms = 0;
        CD_CUDA(cudaEventElapsedTime(&ms, tm.a, tm.b));
        g_stats.sweep_kernel_ms += ms;
        g_stats.sweep_kernel_launches += 1;
    }
    g_stats.sweeps = 1;
    g_stats.moved = (int64_t)hg.g.moved;
    g_stats.gain_lo = hg.g.gain_lo;
    g_stats.gain_hi = hg.g.gain_hi;
    if (moved_out) *moved_out = (int64_t)hg.g.moved;
    if (gain_out) { gain_out[0] = hg.g.gain_lo; gain_out[1] = hg.g.gain_hi; }
    return CD_OK;
}

int cd_modularity(const cd_csr* g, const uint32_t* labels, void* stream, double* q_out,
                  cd_modularity_parts* parts) {
    reset_stats();
    CD_TRY(check_csr(g));
    if (!labels) return CD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    Scratch sc(s);
    const int64_t* off = g->offsets;
    const int32_t* cols = g->cols;
    const uint32_t* w = g->weights;
    const uint32_t* lab = labels;
    if (g->memory == CD_MEM_HOST) {
        for (int64_t i = 0; i < g->n; ++i)
            if ((int64_t)labels[i] >= g->n) return CD_EINVAL;
        int64_t* doff; int32_t* dc; uint32_t* dw; uint32_t* dl;
        CD_TRY(stage_in(g->offsets, g->n + 1, &doff, sc));
        CD_TRY(stage_in(g->cols, g->nnz, &dc, sc));
        CD_TRY(stage_in(g->weights, g->nnz, &dw, sc));
        CD_TRY(stage_in(labels, g->n, &dl, sc));
        off = doff; cols = dc; w = dw; lab = dl;
    }
    Globals* dglob;
    uint64_t *K, *Sig;
    uint32_t* sz;
    CD_TRY(sc.get(&dglob, 1));
    CD_TRY(sc.get(&K, g->n));
    CD_TRY(sc.get(&Sig, g->n));
    CD_TRY(sc.get(&sz, g->n));
    CD_CUDA(cudaMemsetAsync(dglob, 0, sizeof(Globals), s));
    if (g->n > 0) {
        CD_CUDA(launch_degrees(off, w, g->n, g->nnz, K, dglob, s));
        CD_CUDA(launch_modularity(off, cols, w, lab, g->n, g->nnz, K, Sig, sz, dglob, s));
    }
    HostGlobals hg;
    CD_TRY(read_globals(dglob, nullptr, 0, &hg, s));
    u128 sq = ((u128)hg.g.sq_hi << 64) | (u128)hg.g.sq_lo;
    u128 tm = hg.g.two_m;
    double q = 0.0;
    if (tm > 0) {
        i128 num = (i128)(tm * (u128)hg.g.sigma_in) - (i128)sq;
        long double qq = (long double)num / ((long double)tm * (long double)tm);
        q = (double)qq;
    }
    if (parts) {
        parts->sigma_in = hg.g.sigma_in;
        parts->sum_sq_lo = hg.g.sq_lo;
        parts->sum_sq_hi = hg.g.sq_hi;
        parts->two_m = hg.g.two_m;
    }
    g_stats.modularity = q;
    if (q_out) *q_out = q;
    return CD_OK;
}

int cd_louvain(const cd_csr*, const cd_params*, uint32_t*, double*) { return CD_ENOTIMPL; }
int cd_lpa(const cd_csr*, const cd_params*, uint32_t*, double*) { return CD_ENOTIMPL; }
int cd_leiden(const cd_csr*, const cd_params*, uint32_t*, double*) { return CD_ENOTIMPL; }
int cd_aggregate(const cd_csr*, const uint32_t*, void*, uint32_t*, int64_t*, int32_t*, uint32_t*, int64_t*,
                 int64_t*) {
    return CD_ENOTIMPL;
}

}  // extern "C"
