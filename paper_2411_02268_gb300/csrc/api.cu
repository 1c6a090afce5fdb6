// Host side of the C ABI (include/cd.h): argument checks, stream-ordered
// scratch, the launch sequence of one sweep, modularity, and host-memory
// staging.  Every entry point returns a status code and never aborts.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <vector>

#include "batch.cuh"
#include "cd_internal.cuh"

using namespace cdk;

namespace cdk {
thread_local int64_t g_kernel_launches = 0;
}  // namespace cdk

namespace {

thread_local cd_stats g_stats;

void reset_stats() {
    std::memset(&g_stats, 0, sizeof(g_stats));
    g_kernel_launches = 0;
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

// The device's default memory pool (which cudaMallocAsync draws from) keeps
// freed scratch between calls instead of returning it to the driver at every
// synchronisation: calls that allocate the same scratch again (every sweep of
// a benchmark, every host-memory call) then reuse mapped memory instead of
// mapping it anew (mapping several GB costs tens of milliseconds).  The pool
// keeps at least kPoolKeep bytes, and twice the largest scratch of one call
// seen so far on the device (a pool holding little more than one call's
// scratch fragments and maps again every few calls), at most a quarter of
// the device's memory.  Per device, for this process only.
constexpr uint64_t kPoolKeep = 16ull << 30;
constexpr int kMaxDevices = 64;
std::atomic<uint64_t> g_pool_keep[kMaxDevices];

void set_pool_keep(int dev, uint64_t want) {
    uint64_t cur = g_pool_keep[dev].load();
    while (want > cur && !g_pool_keep[dev].compare_exchange_weak(cur, want)) {
    }
    if (want <= cur) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) return;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &want);
}

void keep_pool_memory() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return;
    if (g_pool_keep[dev].load() == 0) set_pool_keep(dev, kPoolKeep);
}

// After a call: let the pool keep twice this call's scratch (see above).
void grow_pool_keep(int64_t bytes) {
    int dev = 0;
    if (bytes <= 0 || cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return;
    const uint64_t want = 2ull * (uint64_t)bytes;
    if (want <= g_pool_keep[dev].load()) return;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return;
    set_pool_keep(dev, std::min<uint64_t>(want, (uint64_t)total_b / 4));
}

// Fault injection for tests: with CD_FAIL_ALLOC=n (n >= 1) in the
// environment, the n-th scratch allocation of every call fails as out of
// memory on the host, before the device is asked for anything.
int64_t injected_alloc_failure() {
    const char* e = std::getenv("CD_FAIL_ALLOC");
    if (!e || !*e) return 0;
    char* end = nullptr;
    const long long v = std::strtoll(e, &end, 10);
    return (end && *end == 0 && v > 0) ? (int64_t)v : 0;
}

// Stream-ordered device scratch of one call; everything is released (in stream
// order) when the object goes out of scope.
struct Scratch {
    cudaStream_t s;
    std::vector<void*> ptrs;
    int64_t bytes = 0;
    int64_t fail_at = 0, count = 0;
    explicit Scratch(cudaStream_t st) : s(st), fail_at(injected_alloc_failure()) { keep_pool_memory(); }
    ~Scratch() {
        for (void* p : ptrs) cudaFreeAsync(p, s);
        if (bytes > g_stats.scratch_bytes) g_stats.scratch_bytes = bytes;
        grow_pool_keep(bytes);
    }
    template <typename T>
    int get(T** p, int64_t count_) {
        if (fail_at > 0 && ++count == fail_at) {
            std::snprintf(g_stats.cuda_error, sizeof(g_stats.cuda_error), "injected allocation failure");
            return CD_ENOMEM;
        }
        size_t nb = sizeof(T) * (size_t)(count_ > 0 ? count_ : 1);
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

int check_csr(const cd_csr* g, bool scan_host = true) {
    if (!g) return CD_EINVAL;
    if (g->n < 0 || g->n >= 0x7FFFFFFFLL || g->nnz < 0) return CD_EINVAL;
    if (g->memory != CD_MEM_DEVICE && g->memory != CD_MEM_HOST) return CD_EINVAL;
    if (!g->offsets) return CD_EINVAL;
    if (g->nnz > 0 && (!g->cols || !g->weights)) return CD_EINVAL;
    if (g->memory == CD_MEM_DEVICE && g->nnz > 0 && (!aligned16(g->cols) || !aligned16(g->weights)))
        return CD_EINVAL;
    if (g->memory == CD_MEM_HOST) {
        // offsets are checked here; columns and weights are checked by the
        // kernels that read them (device-side error flags)
        const int64_t* off = g->offsets;
        if (off[0] != 0 || off[g->n] != g->nnz) return CD_EINVAL;
        if (scan_host)
            for (int64_t i = 0; i < g->n; ++i)
                if (off[i + 1] < off[i]) return CD_EINVAL;
    }
    return CD_OK;
}

// The O(n) checks of host inputs (offsets in order, labels below n), run on
// a host thread while the call stages the inputs on the device.
struct HostCheck {
    std::thread t;
    int rc = CD_OK;
    void start(const cd_csr* g, const uint32_t* labels) {
        if (g->memory != CD_MEM_HOST) return;
        t = std::thread([this, g, labels]() {
            const int64_t* off = g->offsets;
            for (int64_t i = 0; i < g->n; ++i)
                if (off[i + 1] < off[i]) { rc = CD_EINVAL; return; }
            if (labels)
                for (int64_t i = 0; i < g->n; ++i)
                    if ((int64_t)labels[i] >= g->n) { rc = CD_EINVAL; return; }
        });
    }
    int join() {
        if (t.joinable()) t.join();
        return rc;
    }
    ~HostCheck() { join(); }
};

void default_schedule(int k, cd_schedule* s) {
    // Streams per row by row length: one stream up to 128 entries, then about
    // 64-256 entries per stream (the merge tree costs about k updates per
    // stream), 256 streams for the hubs; narrow length bands keep the rows
    // of one warp balanced.  Tuned on R-MAT scale 22 (1.34 -> 1.27 ms against
    // the previous bands; coarser bands cost 30%).
    static const int64_t dm[] = {2, 4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048, 4096, 16384, INT64_MAX};
    static const int32_t ln[] = {1, 1, 1, 1, 1, 1, 1, 2, 4, 4, 8, 8, 32, 256};
    const int nb = 14;
    std::memset(s, 0, sizeof(*s));
    s->nbuckets = nb;
    s->vec = 4;
    // sketches of 32 or 64 slots merge inside one warp: at most 32 streams
    const int cap = k >= 32 ? 32 : 256;
    for (int b = 0; b < nb; ++b) { s->deg_max[b] = dm[b]; s->lanes[b] = ln[b] < cap ? ln[b] : cap; }
}

int check_schedule(const cd_schedule* s) {
    if (s->nbuckets < 1 || s->nbuckets > CD_MAX_BUCKETS || s->vec != 4) return CD_EINVAL;
    if (s->blocks_per_sm < 0 || s->blocks_per_sm > 8) return CD_EINVAL;
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
    if (!(p->k == 0 || p->k == 1 || p->k == 2 || p->k == 4 || p->k == 8 || p->k == 16 || p->k == 32 ||
          p->k == 64))
        return CD_EINVAL;
    if (p->subtract < 0 || p->subtract > 2) return CD_EINVAL;
    // the textbook summary is compiled for sketches of up to 8 slots, sweeps only
    if (p->subtract == 2 && (p->k > 8 || p->agg_k != 0)) return CD_EINVAL;
    if (p->one_scan != 0 && p->one_scan != 1) return CD_EINVAL;
    if (p->one_scan && p->k == 0) return CD_EINVAL;
    if (!(p->agg_k == 0 || p->agg_k == 1 || p->agg_k == 2 || p->agg_k == 4 || p->agg_k == 8 || p->agg_k == 16))
        return CD_EINVAL;
    if (p->skip_rule < 0 || p->skip_rule > 2 || (p->skip_rule == 1 && !p->skip_model)) return CD_EINVAL;
    if (p->sched) {
        CD_TRY(check_schedule(p->sched));
        if (p->k >= 32)
            for (int b = 0; b < p->sched->nbuckets; ++b)
                if (p->sched->lanes[b] > 32) return CD_EINVAL;
    }
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
    bt.resident = s.blocks_per_sm;
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
    uint32_t* elab = nullptr;       // MG sweeps with k <= 16: per-entry labels of the first scan
    const uint32_t* cid = nullptr;  // colour id of every vertex (null: the vertex id)
    bool reuse = false;   // prepare_level keeps the buffers of an earlier call (schedule trials)
    uint32_t *tc = nullptr, *to = nullptr;  // bucketing scratch
    int64_t* dstarts = nullptr;
    unsigned long long* btiles = nullptr;   // scan scratch of the bucketing
    BucketTable bt;     // bucket layout; ranges of colour class 0
    int colors = 1;
    std::vector<int64_t> starts;  // (colour, bucket) range starts, colors * nb + 1
    bool wide = false;  // sketch values need 64 bits
    unsigned long long two_m = 0;

    // Bucket table of colour class p (vertex ranges and grid blocks).
    BucketTable table_for(int p) const {
        BucketTable t = bt;
        int64_t blk = 0;
        for (int b = 0; b < bt.nb; ++b) {
            t.vbegin[b] = starts[(size_t)p * bt.nb + b];
            t.bbegin[b] = blk;
            int64_t nv = starts[(size_t)p * bt.nb + b + 1] - t.vbegin[b];
            int Lb = threads_per_row(bt, b);
            int vpb = Lb >= kBlock ? 1 : kBlock / Lb;
            blk += (nv + vpb - 1) / vpb;
        }
        t.vbegin[bt.nb] = starts[(size_t)p * bt.nb + bt.nb];
        t.bbegin[bt.nb] = blk;
        return t;
    }
};

constexpr int kMaxColors = 16;

struct HostGlobals {
    Globals g;
    int64_t starts[kMaxColors * CD_MAX_BUCKETS + 1];
};

int read_globals(Globals* dglob, int64_t* dstarts, int nb, HostGlobals* out, cudaStream_t s) {
    CD_CUDA(cudaMemcpyAsync(&out->g, dglob, sizeof(Globals), cudaMemcpyDeviceToHost, s));
    if (dstarts) CD_CUDA(cudaMemcpyAsync(out->starts, dstarts, sizeof(int64_t) * (nb + 1),
                                         cudaMemcpyDeviceToHost, s));
    CD_CUDA(cudaStreamSynchronize(s));
    unsigned err = out->g.err;
    if (err & kErrWeightOverflow) return CD_EOVERFLOW;
    if (err) return CD_EINVAL;
    return CD_OK;
}

// K, totals from `labels`, buckets by (colour class, row length); reads back
// 2m, max K and the bucket ranges.
int prepare_level(Level& L, const uint32_t* labels, uint32_t* labels_out_copy, int k,
                  const cd_schedule& sched, int colors, Scratch& sc, Globals* dglob, cudaStream_t s,
                  bool singletons = false, cudaEvent_t weights_ready = nullptr) {
    const bool exact = k == 0;
    const bool fresh = !L.reuse || !L.K;
    if (fresh) {
        CD_TRY(sc.get(&L.K, L.n));
        CD_TRY(sc.get(&L.Sigma, L.n));
        CD_TRY(sc.get(&L.size, L.n));
        CD_TRY(sc.get(&L.verts, L.n));
        if (k > 0 && k <= 16) CD_TRY(sc.get(&L.elab, L.nnz));
    }
    L.bt = exact ? exact_table() : table_from(sched);
    L.bt.qmul = slot_lanes(k);
    L.colors = colors;
    const int nkeys = colors * L.bt.nb;
    int64_t ntiles = bucket_tiles(L.n);
    if (fresh) {
        const int64_t cap = L.reuse ? (int64_t)kMaxColors * CD_MAX_BUCKETS : nkeys;
        CD_TRY(sc.get(&L.tc, ntiles * cap));
        CD_TRY(sc.get(&L.to, ntiles * cap));
        CD_TRY(sc.get(&L.dstarts, cap + 1));
        CD_TRY(sc.get(&L.btiles, scan_tiles(ntiles * cap) + 1));
    }
    uint32_t *tc = L.tc, *to = L.to;
    int64_t* starts = L.dstarts;
    CD_CUDA(cudaMemsetAsync(dglob, 0, sizeof(Globals), s));
    CD_CUDA(launch_bucket(L.off, L.n, L.nnz, L.bt, colors, L.cid, tc, to, starts, L.verts, labels, labels_out_copy,
                          dglob, s, L.btiles));
    HostGlobals hg;
    CD_TRY(read_globals(dglob, starts, nkeys, &hg, s));
    L.starts.assign(hg.starts, hg.starts + nkeys + 1);
    // weighted degrees row by row over the buckets (one launch per colour
    // class), then community totals
    CD_CUDA(cudaMemsetAsync(L.K, 0, sizeof(uint64_t) * (size_t)(L.n > 0 ? L.n : 1), s));
    if (weights_ready) CD_CUDA(cudaStreamWaitEvent(s, weights_ready, 0));
    for (int c = 0; c < colors; ++c)
        CD_CUDA(launch_row_sums(L.off, L.w, L.n, L.nnz, L.verts, L.table_for(c), L.K, dglob, s));
    // singletons: known to the caller, or found by the bucketing (no label
    // differs from its vertex id: glob->pad stayed 0)
    const bool single = singletons || (labels && hg.g.pad == 0);
    CD_CUDA(launch_totals(single ? nullptr : labels, L.K, L.n, L.Sigma, L.size, dglob, s));
    CD_TRY(read_globals(dglob, nullptr, 0, &hg, s));
    L.two_m = hg.g.two_m;
    if (L.two_m >= (1ull << 62)) return CD_EOVERFLOW;
    L.wide = hg.g.max_k >= (1ull << 32);
    L.bt = L.table_for(0);
    return CD_OK;
}

SweepArgs make_args(const Level& L, const uint32_t* labels_in, uint32_t* labels_out, const uint8_t* active,
                    const uint32_t* bound, Globals* dglob, int mode, int uncond, int colors = 1, int sub_color = 0) {
    SweepArgs a;
    std::memset(&a, 0, sizeof(a));
    a.off = L.off; a.cols = L.cols; a.w = L.w;
    a.labels = labels_in; a.K = L.K; a.Sigma = L.Sigma; a.size = L.size;
    a.active = active; a.bound = bound; a.labels_out = labels_out; a.movers = L.movers;
    a.elab = L.elab;
    a.glob = dglob; a.verts = L.verts; a.n = L.n; a.nnz = L.nnz; a.mode = mode; a.uncond = uncond;
    a.colors = colors; a.sub_color = sub_color;
    a.one_scan = 0;
    a.out_all = 1;
    a.bt = L.bt;
    return a;
}

// Launches one sweep (all buckets) on stream s.
int launch_sweep(const Level& L, const SweepArgs& a, int k, Scratch& sc, cudaStream_t s) {
    if (k > 0) {
        int64_t nblocks = L.bt.bbegin[L.bt.nb];
        if (L.bt.resident > 0) {
            // a resident grid striding over the virtual blocks
            int dev = 0, sms = 0;
            CD_CUDA(cudaGetDevice(&dev));
            CD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            nblocks = std::min<int64_t>(nblocks, (int64_t)sms * L.bt.resident);
        }
        CD_CUDA(launch_sweep_mg(a, k, L.wide, nblocks, s));
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

// Host inputs copied on a side stream in the order the call needs them
// (offsets and labels, then weights, then columns), with an event after each
// group, so that degree bucketing and row sums run while the columns still
// copy.
struct SideCopies {
    cudaStream_t cs = nullptr;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    int init() {
        CD_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        for (auto& e : ev) CD_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        return CD_OK;
    }
    ~SideCopies() {
        // the copies finish before the scratch they fill is released (a call
        // that fails part-way has not made its stream wait for them)
        if (cs) cudaStreamSynchronize(cs);
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
        if (cs) cudaStreamDestroy(cs);
    }
};

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


// Renumbers `labels` of level L densely (dense, n entries) and reads back the
// number of communities.
int renumber_level(const Level& L, const uint32_t* labels, uint32_t* dense, Scratch& sc, Globals* dglob,
                   int64_t* nc, cudaStream_t s) {
    uint32_t* tmp;
    unsigned long long* tiles;
    CD_TRY(sc.get(&tmp, L.n));
    CD_TRY(sc.get(&tiles, scan_tiles(L.n) + 1));
    CD_CUDA(cudaMemsetAsync(dglob, 0, sizeof(Globals), s));
    CD_CUDA(launch_renumber(labels, L.n, dense, tmp, tiles, &dglob->count, dglob, s));
    HostGlobals hg;
    CD_TRY(read_globals(dglob, nullptr, 0, &hg, s));
    *nc = (int64_t)hg.g.count;
    return CD_OK;
}

// Super-vertex graph of level L under dense labels (nc communities).  Output
// arrays are taken from the caller (off_out n+1 >= nc+1, cols/w >= nnz) or,
// when null, from scratch.
int aggregate_level(const Level& L, const uint32_t* dense, int64_t nc, Scratch& sc, Globals* dglob,
                    cudaStream_t s, int64_t* off_out, int32_t* cols_out, uint32_t* w_out, Level* next) {
    const int64_t m = L.nnz;
    AggScratch a;
    CD_TRY(sc.get(&a.src, m));
    CD_TRY(sc.get(&a.dst, m));
    CD_TRY(sc.get(&a.w, m));
    CD_TRY(sc.get(&a.src2, m));
    CD_TRY(sc.get(&a.dst2, m));
    CD_TRY(sc.get(&a.w2, m));
    CD_TRY(sc.get(&a.heads, m));
    CD_TRY(sc.get(&a.hist, radix_tiles(m) * 256));
    int64_t tiles = scan_tiles(radix_tiles(m) * 256);
    if (scan_tiles(m) > tiles) tiles = scan_tiles(m);
    if (scan_tiles(nc + 1) > tiles) tiles = scan_tiles(nc + 1);
    CD_TRY(sc.get(&a.tiles, tiles + 1));
    CD_CUDA(cudaMemsetAsync(dglob, 0, sizeof(Globals), s));
    CD_CUDA(launch_expand(L.off, L.cols, L.n, m, dense, a.src, a.dst, dglob, s));
    if (m > 0) CD_CUDA(cudaMemcpyAsync(a.w, L.w, sizeof(uint32_t) * m, cudaMemcpyDeviceToDevice, s));
    CD_CUDA(radix_sort_pairs(a, m, nc, dglob, s));
    CD_CUDA(launch_heads(a, m, s));
    uint32_t* uidx;
    CD_TRY(sc.get(&uidx, m));
    CD_CUDA(launch_exclusive_scan_u32(a.heads, uidx, m, a.tiles, &dglob->count, s));
    HostGlobals hg;
    CD_TRY(read_globals(dglob, nullptr, 0, &hg, s));
    const int64_t m2 = (int64_t)hg.g.count;
    CD_TRY(sc.get(&a.wsum, m2));
    uint32_t* rowcnt;
    CD_TRY(sc.get(&rowcnt, nc + 1));
    if (!off_out) {
        CD_TRY(sc.get(&off_out, nc + 1));
        CD_TRY(sc.get(&cols_out, m2));
        CD_TRY(sc.get(&w_out, m2));
    }
    CD_CUDA(cudaMemsetAsync(a.wsum, 0, sizeof(unsigned long long) * (m2 > 0 ? m2 : 1), s));
    CD_CUDA(cudaMemsetAsync(rowcnt, 0, sizeof(uint32_t) * (nc + 1), s));
    CD_CUDA(launch_segsum(a, uidx, m, cols_out, rowcnt, s));
    CD_CUDA(launch_narrow(a.wsum, m2, w_out, dglob, s));
    CD_CUDA(launch_exclusive_scan_u32_to_i64(rowcnt, off_out, nc + 1, a.tiles, &dglob->count, s));
    CD_TRY(read_globals(dglob, nullptr, 0, &hg, s));
    if (next) {
        *next = Level();
        next->n = nc;
        next->nnz = m2;
        next->off = off_out;
        next->cols = cols_out;
        next->w = w_out;
    }
    return CD_OK;
}

// MG aggregation (Section 4.1 "aggregation phase", Fig. 3; Leiden's symmetric
// form, Section 4.2): one k-slot sketch per community over its members' edges,
// emitted without a second pass.  Output arrays as in aggregate_level.
int aggregate_mg_level(const Level& L, const uint32_t* dense, int64_t nc, int k, bool symmetric, int uncond,
                       const cd_schedule& sched, Scratch& sc, Globals* dglob, cudaStream_t s, int64_t* off_out,
                       int32_t* cols_out, uint32_t* w_out, Level* next, int64_t cap = -1) {
    const int64_t n = L.n, m = L.nnz;
    // members grouped by community, ascending vertex id (stable radix sort)
    AggScratch a;
    CD_TRY(sc.get(&a.src, n));
    CD_TRY(sc.get(&a.dst, n));
    CD_TRY(sc.get(&a.w, n));
    CD_TRY(sc.get(&a.src2, n));
    CD_TRY(sc.get(&a.dst2, n));
    CD_TRY(sc.get(&a.w2, n));
    CD_TRY(sc.get(&a.hist, radix_tiles(n) * 256));
    int64_t tiles = scan_tiles(radix_tiles(n) * 256);
    if (scan_tiles(nc + 1) > tiles) tiles = scan_tiles(nc + 1);
    if (scan_tiles(2 * nc * k + 1) > tiles) tiles = scan_tiles(2 * nc * k + 1);
    CD_TRY(sc.get(&a.tiles, tiles + 1));
    CD_CUDA(cudaMemsetAsync(dglob, 0, sizeof(Globals), s));
    CD_CUDA(cudaMemcpyAsync(a.src, dense, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
    CD_CUDA(launch_iota(a.dst, n, s));
    CD_CUDA(launch_iota(a.w, n, s));
    CD_CUDA(radix_sort_keys(a, n, bits_for(nc), 0, dglob, s));
    const uint32_t* members = a.dst;
    // member ranges and entry counts per community
    uint32_t *cnt, *ecnt;
    int64_t *moff, *coff;
    CD_TRY(sc.get(&cnt, nc + 1));
    CD_TRY(sc.get(&ecnt, nc + 1));
    CD_TRY(sc.get(&moff, nc + 1));
    CD_TRY(sc.get(&coff, nc + 1));
    CD_CUDA(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * (nc + 1), s));
    CD_CUDA(cudaMemsetAsync(ecnt, 0, sizeof(uint32_t) * (nc + 1), s));
    CD_CUDA(launch_community_counts(L.off, dense, n, cnt, ecnt, s));
    CD_CUDA(launch_exclusive_scan_u32_to_i64(cnt, moff, nc + 1, a.tiles, &dglob->count, s));
    CD_CUDA(launch_exclusive_scan_u32_to_i64(ecnt, coff, nc + 1, a.tiles, &dglob->count, s));
    // communities bucketed by their entry count
    Level C;
    C.n = nc;
    C.nnz = m;
    C.off = coff;
    C.bt = table_from(sched);
    C.colors = 1;
    const int nkeys = C.bt.nb;
    int64_t ntiles = bucket_tiles(nc);
    uint32_t *tc, *to;
    int64_t* starts;
    CD_TRY(sc.get(&C.verts, nc));
    CD_TRY(sc.get(&tc, ntiles * nkeys));
    CD_TRY(sc.get(&to, ntiles * nkeys));
    CD_TRY(sc.get(&starts, nkeys + 1));
    CD_CUDA(launch_bucket(coff, nc, m, C.bt, 1, nullptr, tc, to, starts, C.verts, nullptr, nullptr, dglob, s));
    HostGlobals hg;
    CD_TRY(read_globals(dglob, starts, nkeys, &hg, s));
    C.starts.assign(hg.starts, hg.starts + nkeys + 1);
    C.bt = C.table_for(0);
    // one sketch per community
    uint32_t* keys;
    unsigned long long* vals;
    CD_TRY(sc.get(&keys, nc * k));
    CD_TRY(sc.get(&vals, nc * k));
    CD_CUDA(cudaMemsetAsync(keys, 0xFF, sizeof(uint32_t) * nc * k, s));
    CD_CUDA(cudaMemsetAsync(vals, 0, sizeof(unsigned long long) * nc * k, s));
    AggArgs g;
    std::memset(&g, 0, sizeof(g));
    g.a.off = L.off; g.a.cols = L.cols; g.a.w = L.w; g.a.labels = dense;
    g.a.glob = dglob; g.a.verts = C.verts; g.a.n = n; g.a.nnz = m; g.a.uncond = uncond; g.a.bt = C.bt;
    g.moff = moff; g.members = members; g.out_keys = keys; g.out_vals = vals;
    CD_CUDA(launch_agg_mg(g, k, L.two_m >= (1ull << 32), C.bt.bbegin[C.bt.nb], s));
    // rows
    uint32_t *count, *self_less;
    CD_TRY(sc.get(&count, nc + 1));
    CD_TRY(sc.get(&self_less, nc + 1));
    CD_CUDA(cudaMemsetAsync(count, 0, sizeof(uint32_t) * (nc + 1), s));
    CD_CUDA(cudaMemsetAsync(self_less, 0, sizeof(uint32_t) * (nc + 1), s));
    CD_CUDA(launch_mg_sort_rows(keys, vals, nc, k, count, symmetric ? self_less : nullptr, s));
    int64_t m2 = 0;
    if (!symmetric) {
        int64_t* roff;
        CD_TRY(sc.get(&roff, nc + 1));
        CD_CUDA(launch_exclusive_scan_u32_to_i64(count, roff, nc + 1, a.tiles, &dglob->count, s));
        CD_TRY(read_globals(dglob, nullptr, 0, &hg, s));
        m2 = (int64_t)hg.g.count;
        if (cap >= 0 && m2 > cap) return CD_EINVAL;
        if (!off_out) {
            CD_TRY(sc.get(&off_out, nc + 1));
            CD_TRY(sc.get(&cols_out, m2));
            CD_TRY(sc.get(&w_out, m2));
        }
        CD_CUDA(launch_mg_write_rows(keys, vals, nc, k, roff, cols_out, w_out, dglob, s));
        CD_CUDA(cudaMemcpyAsync(off_out, roff, sizeof(int64_t) * (nc + 1), cudaMemcpyDeviceToDevice, s));
    } else {
        int64_t *fpos, *rpos;
        CD_TRY(sc.get(&fpos, nc + 1));
        CD_TRY(sc.get(&rpos, nc + 1));
        CD_CUDA(launch_exclusive_scan_u32_to_i64(count, fpos, nc + 1, a.tiles, &dglob->count, s));
        CD_TRY(read_globals(dglob, nullptr, 0, &hg, s));
        const int64_t F = (int64_t)hg.g.count;
        CD_CUDA(launch_exclusive_scan_u32_to_i64(self_less, rpos, nc + 1, a.tiles, &dglob->count, s));
        CD_TRY(read_globals(dglob, nullptr, 0, &hg, s));
        const int64_t M = F + (int64_t)hg.g.count;
        AggScratch b;
        CD_TRY(sc.get(&b.src, M));
        CD_TRY(sc.get(&b.dst, M));
        CD_TRY(sc.get(&b.w, M));
        CD_TRY(sc.get(&b.src2, M));
        CD_TRY(sc.get(&b.dst2, M));
        CD_TRY(sc.get(&b.w2, M));
        CD_TRY(sc.get(&b.hist, radix_tiles(M) * 256));
        int64_t bt = scan_tiles(radix_tiles(M) * 256);
        if (scan_tiles(M + 1) > bt) bt = scan_tiles(M + 1);
        if (scan_tiles(nc + 1) > bt) bt = scan_tiles(nc + 1);
        CD_TRY(sc.get(&b.tiles, bt + 1));
        CD_CUDA(launch_mg_candidates(keys, vals, nc, k, fpos, rpos, F, b, dglob, s));
        CD_CUDA(radix_sort_pairs(b, M, nc, dglob, s));
        uint32_t *keep, *pos, *rowcnt;
        CD_TRY(sc.get(&keep, M));
        CD_TRY(sc.get(&pos, M));
        CD_TRY(sc.get(&rowcnt, nc + 1));
        CD_CUDA(launch_mg_select(b, M, keep, s));
        CD_CUDA(launch_exclusive_scan_u32(keep, pos, M, b.tiles, &dglob->count, s));
        CD_TRY(read_globals(dglob, nullptr, 0, &hg, s));
        m2 = (int64_t)hg.g.count;
        if (cap >= 0 && m2 > cap) return CD_EINVAL;
        if (!off_out) {
            CD_TRY(sc.get(&off_out, nc + 1));
            CD_TRY(sc.get(&cols_out, m2));
            CD_TRY(sc.get(&w_out, m2));
        }
        CD_CUDA(cudaMemsetAsync(rowcnt, 0, sizeof(uint32_t) * (nc + 1), s));
        CD_CUDA(launch_mg_compact(b, keep, pos, M, cols_out, w_out, rowcnt, s));
        CD_CUDA(launch_exclusive_scan_u32_to_i64(rowcnt, off_out, nc + 1, b.tiles, &dglob->count, s));
    }
    CD_TRY(read_globals(dglob, nullptr, 0, &hg, s));
    if (next) {
        *next = Level();
        next->n = nc;
        next->nnz = m2;
        next->off = off_out;
        next->cols = cols_out;
        next->w = w_out;
    }
    return CD_OK;
}

double gain_as_double(unsigned long long lo, unsigned long long hi) {
    return (double)hi * 18446744073709551616.0 + (double)lo;
}

// Local-moving phase on level L from singleton labels: sweeps (each followed
// by the commit into Sigma and sizes) until nobody moves, the sweep's summed
// delta-Q is at most tol (Louvain), at most tol * n labels change (LPA), or
// max_sweeps.  Returns the final labels in *labels (one of two scratch buffers).
int resolve_colors(const cd_params* p) { return p->colors == 0 ? 8 : p->colors; }

// Local-moving phase on level L from `init` labels (singletons when null):
// every sweep is `colors` sub-sweeps (sub-sweep c decides the vertices of
// colour class c from the state left by the previous ones), each followed by
// the commit into Sigma and sizes, until nobody moves, the sweep's summed
// delta-Q is at most tol (Louvain), at most tol * n labels change (LPA), or
// max_sweeps.  Returns the final labels in *labels (a scratch buffer).
// Move traces recorded by local_move (cd_trace).
struct Trace {
    double rate = 0.0;
    void* x = nullptr;   // capacity x 8 float16
    uint8_t* y = nullptr;
    int64_t cap = 0;
    int64_t count = 0;
};

// Model parameters in device scratch (float32, the cd_mlp layout).
int stage_model(const cd_mlp* m, Scratch& sc, float** dparam, cudaStream_t s) {
    CD_TRY(sc.get(dparam, mlp_param_count()));
    CD_CUDA(cudaMemcpyAsync(*dparam, m, sizeof(float) * mlp_param_count(), cudaMemcpyHostToDevice, s));
    return CD_OK;
}

// Per-graph state of the batched form during one level (a disjoint union of
// graphs, see batch.cu).  Device arrays have G + 1 entries (the last one is
// the sentinel graph of the padding vertices, which never decides).
struct BatchLevel {
    int G = 0;
    const uint32_t* gid = nullptr;   // graph of every vertex of the level
    const int64_t* vb = nullptr;     // first vertex of every graph (device, G)
    const int64_t* nv = nullptr;     // vertices of every graph (device, G)
    unsigned long long* two_m_g = nullptr;
    uint8_t* gdone = nullptr;
    uint32_t* gsweeps = nullptr;
    unsigned long long* gstat = nullptr;  // moved, gain_lo, gain_hi (3 x (G + 1))
    std::vector<uint8_t> finished;   // host: graphs whose passes have ended
};

// One sweep replayed from a CUDA graph (see local_move).
struct Replay {
    cudaStream_t cs = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;  // kernel launches recorded in the graph
    ~Replay() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cs) cudaStreamDestroy(cs);
    }
};

// True when launch_sweep on level L enqueues kernels only (no host sync).
bool sweep_is_async(const Level& L, int k) {
    if (k > 0) return true;
    for (int b = 0; b < kExactBuckets; ++b)
        if (kExact[b].global && L.starts.size() > 0) {
            for (int c = 0; c < L.colors; ++c)
                if (L.starts[(size_t)c * L.bt.nb + b + 1] > L.starts[(size_t)c * L.bt.nb + b]) return false;
        }
    return true;
}

// Local-moving phase on level L from `init` labels (singletons when null):
// every sweep is `colors` sub-sweeps (sub-sweep c decides the vertices of
// colour class c from the state left by the previous ones), each followed by
// the commit into Sigma and sizes, until nobody moves, the sweep's summed
// delta-Q is at most tol (Louvain), at most tol * n labels change (LPA), or
// max_sweeps.  With a skip rule, sweeps after the first decide only the
// proposed vertices; a proposal sweep that moves nobody or gains at most tol
// is followed by a full sweep, which decides convergence.  In the batched
// form (B) the stopping rule is applied per graph on the device and the
// phase ends when every graph has stopped.  With p->capture the launches of
// one sweep are recorded once as a CUDA graph and replayed every sweep.
// Returns the final labels in *labels (a scratch buffer).
int local_move(Level& L, const cd_params* p, int mode, double tol, const cd_schedule& sched, Scratch& sc,
               Globals* dglob, cudaStream_t s, const uint32_t* init, uint32_t** labels, int64_t* sweeps_out,
               Trace* trace = nullptr, BatchLevel* B = nullptr) {
    uint32_t *la, *lb;
    CD_TRY(sc.get(&la, L.n));
    CD_TRY(sc.get(&lb, L.n));
    CD_TRY(sc.get(&L.movers, L.n));
    if (init) CD_CUDA(cudaMemcpyAsync(la, init, sizeof(uint32_t) * L.n, cudaMemcpyDeviceToDevice, s));
    else CD_CUDA(launch_iota(la, L.n, s));
    const int colors = resolve_colors(p);
    CD_TRY(prepare_level(L, la, lb, p->k, sched, colors, sc, dglob, s, init == nullptr));
    const int rule = trace ? 0 : p->skip_rule;
    const bool track = rule != 0 || trace;
    uint8_t *active = nullptr, *moved_last = nullptr, *since_move = nullptr;
    uint32_t* before = nullptr;
    void* x = nullptr;
    float* param = nullptr;
    if (track) {
        CD_TRY(sc.get(&active, L.n));
        CD_TRY(sc.get(&moved_last, L.n));
        CD_TRY(sc.get(&since_move, L.n));
        CD_TRY(sc.get(&before, L.n));
        CD_CUDA(cudaMemsetAsync(moved_last, 1, L.n, s));
        CD_CUDA(cudaMemsetAsync(since_move, 0, L.n, s));
    }
    float* attach = nullptr;
    uint32_t *tflags = nullptr, *tpos = nullptr;
    unsigned long long* ttiles = nullptr;
    if (rule == 1 || trace) {
        CD_TRY(sc.get(&attach, L.n));
        CD_CUDA(cudaMemsetAsync(attach, 0, sizeof(float) * L.n, s));
    }
    if (trace) {
        uint16_t* xh;  // feature rows of the traced sweeps
        CD_TRY(sc.get(&xh, L.n * 8));
        x = xh;
        CD_TRY(sc.get(&tflags, L.n));
        CD_TRY(sc.get(&tpos, L.n));
        CD_TRY(sc.get(&ttiles, scan_tiles(L.n) + 1));
    }
    if (rule == 1) CD_TRY(stage_model(p->skip_model, sc, &param, s));
    // skip sweeps of the MG kernels run over the compacted list of deciding
    // vertices (device-side ranges), so the skipped ones cost no blocks
    const bool compact = rule != 0 && p->k > 0;
    const int64_t n_listed = L.starts.empty() ? 0 : L.starts.back();
    uint32_t *cflags = nullptr, *cpos = nullptr, *cverts = nullptr;
    unsigned long long *ctiles = nullptr, *ctotal = nullptr;
    DevRanges* cdr = nullptr;
    if (compact) {
        CD_TRY(sc.get(&cflags, n_listed));
        CD_TRY(sc.get(&cpos, n_listed));
        CD_TRY(sc.get(&cverts, n_listed));
        CD_TRY(sc.get(&ctiles, scan_tiles(n_listed) + 1));
        CD_TRY(sc.get(&ctotal, 1));
        CD_TRY(sc.get(&cdr, colors));
    }
    const int G = B ? B->G : 0;
    if (B) {
        CD_CUDA(launch_graph_two_m(L.K, B->vb, B->nv, G, B->two_m_g, s));
        std::vector<uint8_t> d0(B->finished);
        d0.push_back(1);  // sentinel graph
        if (p->max_sweeps == 0) std::fill(d0.begin(), d0.end(), (uint8_t)1);
        CD_CUDA(cudaMemcpyAsync(B->gdone, d0.data(), (size_t)G + 1, cudaMemcpyHostToDevice, s));
        CD_CUDA(cudaMemsetAsync(B->gsweeps, 0, sizeof(uint32_t) * ((size_t)G + 1), s));
        CD_CUDA(cudaStreamSynchronize(s));  // d0 must outlive the copy
    }
    std::vector<Timer> tms((size_t)colors);
    for (auto& t : tms) CD_TRY(t.init(p->timing != 0));
    const size_t stat_off = offsetof(Globals, moved);
    const size_t stat_len = offsetof(Globals, sigma_in) - stat_off;
    // the launches of one sweep on stream st
    auto enqueue = [&](cudaStream_t st, bool use_mask) -> int {
        CD_CUDA(cudaMemsetAsync(reinterpret_cast<char*>(dglob) + stat_off, 0, stat_len, st));
        if (B) {
            CD_CUDA(cudaMemsetAsync(B->gstat, 0, sizeof(unsigned long long) * 3 * ((size_t)G + 1), st));
            CD_CUDA(cudaMemsetAsync(&dglob->count, 0, sizeof(unsigned long long), st));
        }
        for (int c = 0; c < colors; ++c) {
            // sub-sweep c: vertices of colour c decide from la and write lb; the
            // movers' new labels are then copied into la for sub-sweep c+1
            CD_CUDA(cudaMemcpyAsync(&dglob->mark, &dglob->moved, sizeof(unsigned long long),
                                    cudaMemcpyDeviceToDevice, st));
            Level Lc = L;
            Lc.bt = L.table_for(c);
            SweepArgs a = make_args(Lc, la, lb, use_mask ? active : nullptr, nullptr, dglob, mode, p->subtract,
                                    colors, c);
            a.cid = L.cid;
            a.one_scan = p->one_scan;
            a.attach = attach;
            a.out_all = 0;  // k_commit reads the movers' entries of lb only
            if (use_mask && compact) {
                a.verts = cverts;
                a.dr = cdr + c;
            }
            if (B) {
                a.gid = B->gid;
                a.two_m_g = B->two_m_g;
                a.gdone = B->gdone;
                a.g_moved = B->gstat;
                a.g_gain_lo = B->gstat + (G + 1);
                a.g_gain_hi = B->gstat + 2 * (G + 1);
            }
            if (tms[c].on) CD_CUDA(cudaEventRecord(tms[c].a, st));
            CD_TRY(launch_sweep(Lc, a, p->k, sc, st));
            if (tms[c].on) CD_CUDA(cudaEventRecord(tms[c].b, st));
            CD_CUDA(launch_commit(L.movers, la, lb, L.K, L.n, L.Sigma, L.size, dglob, st));
        }
        if (B)
            CD_CUDA(launch_batch_converge(G, B->two_m_g, B->gstat, B->gstat + (G + 1), B->gstat + 2 * (G + 1), tol,
                                          p->max_sweeps, B->gsweeps, B->gdone, dglob, st));
        return CD_OK;
    };
    // one sweep: the skip proposal (masked sweeps), the sub-sweeps, the move state
    auto sweep_seq = [&](cudaStream_t st, bool use_mask) -> int {
        if (use_mask && rule == 2) {
            // movers of the previous sweep and their neighbours
            CD_CUDA(cudaMemsetAsync(active, 0, L.n, st));
            CD_CUDA(launch_mark_neighbours(L.off, L.cols, L.movers, dglob, active, st));
        }
        if (use_mask && rule == 1)
            CD_CUDA(launch_propose(L.off, L.K, la, L.Sigma, L.size, L.two_m, moved_last, since_move, attach, L.n,
                                   param, p->skip_threshold, active, st));
        if (use_mask && compact)
            CD_CUDA(launch_compact(L.verts, n_listed, active, L.dstarts, L.bt, colors, cflags, cpos, ctiles, ctotal,
                                   cverts, cdr, st));
        if (track) CD_CUDA(cudaMemcpyAsync(before, la, sizeof(uint32_t) * L.n, cudaMemcpyDeviceToDevice, st));
        CD_TRY(enqueue(st, use_mask));
        if (track) CD_CUDA(launch_move_state(before, la, L.n, moved_last, since_move, st));
        return CD_OK;
    };
    // full and masked sweeps recorded once each as CUDA graphs (replayed on s)
    Replay rp[2];
    if (p->capture && !trace && !p->timing && sweep_is_async(L, p->k)) {
        for (int m = 0; m < (rule != 0 ? 2 : 1); ++m) {
            CD_CUDA(cudaStreamCreateWithFlags(&rp[m].cs, cudaStreamNonBlocking));
            CD_CUDA(cudaStreamBeginCapture(rp[m].cs, cudaStreamCaptureModeThreadLocal));
            const int64_t before = g_kernel_launches;
            const int rc = sweep_seq(rp[m].cs, m == 1);
            // recorded, not run: counted at every replay instead
            rp[m].kernels = g_kernel_launches - before;
            g_kernel_launches = before;
            cudaGraph_t gr = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(rp[m].cs, &gr);
            rp[m].graph = gr;
            CD_TRY(rc);
            CD_CUDA(ec);
            CD_CUDA(cudaGraphInstantiate(&rp[m].exec, rp[m].graph, 0));
        }
    }
    int64_t sw = 0;
    bool force_full = false;
    for (; sw < p->max_sweeps;) {
        const bool use_mask = rule != 0 && sw > 0 && !force_full;
        if (trace && sw > 0)
            CD_CUDA(launch_features(L.off, L.K, la, L.Sigma, L.size, L.two_m, moved_last, since_move, attach, true,
                                    L.n, x, s));
        if (rp[use_mask ? 1 : 0].exec) {
            CD_CUDA(cudaGraphLaunch(rp[use_mask ? 1 : 0].exec, s));
            note_launch(rp[use_mask ? 1 : 0].kernels);
        } else {
            CD_TRY(sweep_seq(s, use_mask));
        }
        HostGlobals hg;
        if (trace && sw > 0) {
            const double r = trace->rate < 0 ? 0 : (trace->rate > 1 ? 1 : trace->rate);
            const uint32_t thr32 = r >= 1.0 ? 0xFFFFFFFFu : (uint32_t)(r * 4294967296.0);
            CD_CUDA(launch_trace_flags(L.off, L.n, (int)sw, thr32, tflags, s));
            CD_CUDA(launch_exclusive_scan_u32(tflags, tpos, L.n, ttiles, &dglob->count, s));
            CD_CUDA(launch_trace_write(x, moved_last, tflags, tpos, L.n, trace->count, trace->x, trace->y,
                                       trace->cap, s));
        }
        CD_TRY(read_globals(dglob, nullptr, 0, &hg, s));
        if (trace && sw > 0) trace->count = std::min<int64_t>(trace->count + (int64_t)hg.g.count, trace->cap);
        for (auto& t : tms) {
            if (!t.on) continue;
            float ms = 0;
            CD_CUDA(cudaEventElapsedTime(&ms, t.a, t.b));
            g_stats.sweep_kernel_ms += ms;
            g_stats.sweep_kernel_launches += 1;
        }
        ++sw;
        g_stats.moved = (int64_t)hg.g.moved;
        g_stats.gain_lo = hg.g.gain_lo;
        g_stats.gain_hi = hg.g.gain_hi;
        g_stats.entries_scanned += (int64_t)hg.g.scanned;
        g_stats.candidates += (int64_t)hg.g.cands;
        if (!use_mask) g_stats.full_sweeps += 1;
        if (B) {
            if (hg.g.count == 0) break;  // every graph has stopped
            continue;
        }
        bool done = hg.g.moved == 0;
        if (!done) {
            if (mode == CD_MODE_LPA) {
                done = (double)hg.g.moved <= tol * (double)L.n;
            } else {
                double dq = gain_as_double(hg.g.gain_lo, hg.g.gain_hi) /
                            ((double)L.two_m * (double)L.two_m / 2.0);
                done = dq <= tol;
            }
        }
        if (done && use_mask) {
            force_full = true;  // a proposal sweep stalled: the next sweep is a full one
            continue;
        }
        force_full = false;
        if (done) break;
    }
    *labels = la;
    *sweeps_out = sw;
    return CD_OK;
}

// Leiden refinement (Section 3.4, 4.2) of level L within the communities
// `bound`: sub-communities start as singletons; one sweep of `colors`
// sub-sweeps in refine mode (only singletons move, only inside their bound,
// never into a same-colour singleton).  Returns the sub-community labels.
int refine_level(Level& L, const cd_params* p, const uint32_t* bound, const cd_schedule& sched, Scratch& sc,
                 Globals* dglob, cudaStream_t s, uint32_t** labels) {
    uint32_t *la, *lb;
    CD_TRY(sc.get(&la, L.n));
    CD_TRY(sc.get(&lb, L.n));
    CD_TRY(sc.get(&L.movers, L.n));
    CD_CUDA(launch_iota(la, L.n, s));
    const int colors = resolve_colors(p);
    CD_TRY(prepare_level(L, la, lb, p->k, sched, colors, sc, dglob, s, true));
    const size_t stat_off = offsetof(Globals, moved);
    const size_t stat_len = offsetof(Globals, sigma_in) - stat_off;
    CD_CUDA(cudaMemsetAsync(reinterpret_cast<char*>(dglob) + stat_off, 0, stat_len, s));
    for (int c = 0; c < colors; ++c) {
        CD_CUDA(cudaMemcpyAsync(&dglob->mark, &dglob->moved, sizeof(unsigned long long),
                                cudaMemcpyDeviceToDevice, s));
        Level Lc = L;
        Lc.bt = L.table_for(c);
        SweepArgs a = make_args(Lc, la, lb, nullptr, bound, dglob, CD_MODE_REFINE, p->subtract, colors, c);
        a.out_all = 0;
        CD_TRY(launch_sweep(Lc, a, p->k, sc, s));
        CD_CUDA(launch_commit(L.movers, la, lb, L.K, L.n, L.Sigma, L.size, dglob, s));
    }
    HostGlobals hg;
    CD_TRY(read_globals(dglob, nullptr, 0, &hg, s));
    g_stats.sweeps += 1;
    *labels = la;
    return CD_OK;
}

// Stages a host graph into scratch (or passes a device graph through).
int input_level(const cd_csr* g, Scratch& sc, Level* L) {
    L->n = g->n;
    L->nnz = g->nnz;
    if (g->memory == CD_MEM_HOST) {
        int64_t* off; int32_t* cols; uint32_t* w;
        CD_TRY(stage_in(g->offsets, g->n + 1, &off, sc));
        CD_TRY(stage_in(g->cols, g->nnz, &cols, sc));
        CD_TRY(stage_in(g->weights, g->nnz, &w, sc));
        L->off = off; L->cols = cols; L->w = w;
    } else {
        L->off = g->offsets; L->cols = g->cols; L->w = g->weights;
    }
    return CD_OK;
}

// Q of labels on the level's graph.  The weighted degrees are the level's
// own (L.K, left by a local-moving phase on it) when it has them, else they
// are computed here.
int modularity_of(const Level& L, const uint32_t* labels, Scratch& sc, Globals* dglob, cudaStream_t s,
                  double* q) {
    uint64_t *K = L.K, *Sig;
    uint32_t* sz;
    if (!K) CD_TRY(sc.get(&K, L.n));
    CD_TRY(sc.get(&Sig, L.n));
    CD_TRY(sc.get(&sz, L.n));
    CD_CUDA(cudaMemsetAsync(dglob, 0, sizeof(Globals), s));
    if (L.n > 0) {
        if (!L.K) CD_CUDA(launch_degrees(L.off, L.w, L.n, L.nnz, K, dglob, s));
        CD_CUDA(launch_modularity(L.off, L.cols, L.w, labels, L.n, L.nnz, K, Sig, sz, dglob, s));
    }
    HostGlobals hg;
    CD_TRY(read_globals(dglob, nullptr, 0, &hg, s));
    u128 sq = ((u128)hg.g.sq_hi << 64) | (u128)hg.g.sq_lo;
    u128 tm = hg.g.two_m;
    *q = 0.0;
    if (tm > 0) {
        i128 num = (i128)(tm * (u128)hg.g.sigma_in) - (i128)sq;
        *q = (double)((long double)num / ((long double)tm * (long double)tm));
    }
    g_stats.modularity = *q;
    return CD_OK;
}

int check_driver_params(const cd_params* p) {
    CD_TRY(check_params(p));
    if (p->max_sweeps < 0 || p->max_passes < 0) return CD_EINVAL;
    if (!(p->tolerance >= 0.0) || !(p->tolerance_drop >= 1.0) || !(p->aggregation_tolerance > 0.0))
        return CD_EINVAL;
    return CD_OK;
}

// Writes dense labels (device) to the caller's buffer (device or host).
int emit_labels(const cd_csr* g, const uint32_t* dense, uint32_t* labels_out, cudaStream_t s) {
    if (g->n == 0) return CD_OK;
    cudaMemcpyKind kind = g->memory == CD_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    CD_CUDA(cudaMemcpyAsync(labels_out, dense, sizeof(uint32_t) * g->n, kind, s));
    CD_CUDA(cudaStreamSynchronize(s));
    return CD_OK;
}

// Packs `G` input graphs (all in one memory space) into one disjoint union
// (batch.cu): graph g at vertices [vb0_g, vb0_g + n_g] (the last one its
// padding vertex), entries from a multiple of kPackAlign.  Fills the level
// `in` (with colour ids = ids inside each graph), the graph of every vertex
// (*gid0) and the per-graph layout vectors.
int pack_union(const cd_csr* graphs, int G, Scratch& sc, Globals* dglob, cudaStream_t s, std::vector<PackGraph>& pg,
               std::vector<int64_t>& vb0, std::vector<int64_t>& n0, std::vector<int64_t>& tstart, Level* in,
               uint32_t** gid0, uint32_t** lid0) {
    pg.assign((size_t)G, PackGraph());
    vb0.assign((size_t)G, 0);
    n0.assign((size_t)G, 0);
    tstart.assign((size_t)G + 1, 0);
    int64_t V = 0, E = 0;
    for (int g = 0; g < G; ++g) {
        const cd_csr& c = graphs[g];
        PackGraph& q = pg[(size_t)g];
        std::memset(&q, 0, sizeof(q));
        if (c.memory == CD_MEM_HOST) {
            int64_t* off; int32_t* cols; uint32_t* w;
            CD_TRY(stage_in(c.offsets, c.n + 1, &off, sc));
            CD_TRY(stage_in(c.cols, c.nnz, &cols, sc));
            CD_TRY(stage_in(c.weights, c.nnz, &w, sc));
            q.off = off; q.cols = cols; q.w = w;
        } else {
            q.off = c.offsets; q.cols = c.cols; q.w = c.weights;
        }
        q.vsrc0 = 0; q.n = c.n; q.nnz = c.nnz;
        q.vbase = V; q.ebase = E;
        q.pad = (E + c.nnz + kPackAlign - 1) / kPackAlign * kPackAlign - (E + c.nnz);
        q.col_shift = V; q.check_first = 1;
        vb0[(size_t)g] = V;
        n0[(size_t)g] = c.n;
        V += c.n + 1;
        E += c.nnz + q.pad;
        tstart[(size_t)g + 1] = tstart[(size_t)g] + pack_tiles(q);
        if (V >= 0x7FFFFFFFLL) return CD_EINVAL;  // union ids must fit int32 columns
    }
    int64_t* uoff; int32_t* ucols; uint32_t* uw;
    PackGraph* dpg; int64_t* dts;
    CD_TRY(sc.get(&uoff, V + 1));
    CD_TRY(sc.get(&ucols, E));
    CD_TRY(sc.get(&uw, E));
    CD_TRY(sc.get(gid0, V));
    CD_TRY(sc.get(lid0, V));
    CD_TRY(stage_in(pg.data(), G, &dpg, sc));
    CD_TRY(stage_in(tstart.data(), G + 1, &dts, sc));
    CD_CUDA(cudaMemsetAsync(dglob, 0, sizeof(Globals), s));
    CD_CUDA(launch_pack(dpg, dts, G, tstart[(size_t)G], uoff, ucols, uw, *gid0, *lid0, V, E, dglob, s));
    HostGlobals hg;
    CD_TRY(read_globals(dglob, nullptr, 0, &hg, s));
    *in = Level();
    in->n = V; in->nnz = E; in->off = uoff; in->cols = ucols; in->w = uw; in->cid = *lid0;
    return CD_OK;
}

}  // namespace

namespace cdk {
// Records a CUDA error string in the calling thread's statistics.
void record_cuda_error(cudaError_t e) {
    reset_stats();
    std::snprintf(g_stats.cuda_error, sizeof(g_stats.cuda_error), "%s", cudaGetErrorString(e));
    cudaGetLastError();
}
// For entry points defined in other files: start a call's statistics, and
// record the modularity it computed.
void begin_call_stats() { reset_stats(); }
void record_modularity(double q) { g_stats.modularity = q; }
}  // namespace cdk

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
        case CD_ESIZE: return "input exceeds the fixed scratch of this entry point";
        default: return "unknown status";
    }
}

int cd_last_stats(cd_stats* out) {
    if (!out) return CD_EINVAL;
    *out = g_stats;
    out->kernel_launches = g_kernel_launches;
    return CD_OK;
}

int cd_default_schedule(int k, cd_schedule* out) {
    if (!out || k < 0) return CD_EINVAL;
    default_schedule(k, out);
    return CD_OK;
}

int cd_sweep(const cd_csr* g, const cd_params* p, int mode, const uint32_t* labels_in,
             const uint8_t* active, const uint32_t* bound, uint32_t* labels_out, int64_t* moved_out,
             uint64_t* gain_out) {
    reset_stats();
    CD_TRY(check_csr(g, false));  // the O(n) host checks run beside the staging (HostCheck)
    CD_TRY(check_params(p));
    if (mode != CD_MODE_LOUVAIN && mode != CD_MODE_LPA && mode != CD_MODE_REFINE) return CD_EINVAL;
    if ((mode == CD_MODE_REFINE) != (bound != nullptr)) return CD_EINVAL;
    if (p->one_scan && mode != CD_MODE_LPA) return CD_EINVAL;
    // colour classes of this sweep: refine mode defaults to 8, the others to 1
    const int ncol = mode == CD_MODE_REFINE ? resolve_colors(p) : (p->colors == 0 ? 1 : p->colors);
    if (p->colors < 0 || p->colors > 16 || p->sub_color < 0 || p->sub_color >= ncol) return CD_EINVAL;
    if (!labels_in || !labels_out || labels_in == labels_out) return CD_EINVAL;
    cudaStream_t s = (cudaStream_t)p->stream;
    cd_schedule sched;
    if (p->sched) sched = *p->sched; else default_schedule(p->k, &sched);
    const bool host = g->memory == CD_MEM_HOST;
    const auto t_start = std::chrono::steady_clock::now();
    auto since_ms = [&](std::chrono::steady_clock::time_point t) {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t).count();
    };
    HostCheck hc;
    hc.start(g, labels_in);
    Scratch sc(s);
    Level L;
    L.n = g->n;
    L.nnz = g->nnz;
    const uint32_t* lin = labels_in;
    uint32_t* lout = labels_out;
    const uint8_t* act = active;
    SideCopies side;
    auto stage = [&]() -> int {
        // allocations are ordered on s; the copies run on the side stream
        int64_t *off; int32_t* cols; uint32_t* w; uint32_t* li;
        CD_TRY(sc.get(&off, g->n + 1));
        CD_TRY(sc.get(&li, g->n));
        CD_TRY(sc.get(&w, g->nnz));
        CD_TRY(sc.get(&cols, g->nnz));
        CD_TRY(sc.get(&lout, g->n));
        uint8_t* da = nullptr;
        uint32_t* db = nullptr;
        if (active) CD_TRY(sc.get(&da, g->n));
        if (bound) CD_TRY(sc.get(&db, g->n));
        CD_TRY(side.init());
        CD_CUDA(cudaEventRecord(side.ev[0], s));
        CD_CUDA(cudaStreamWaitEvent(side.cs, side.ev[0], 0));  // the allocations precede the copies
        CD_CUDA(cudaMemcpyAsync(off, g->offsets, sizeof(int64_t) * (g->n + 1), cudaMemcpyHostToDevice, side.cs));
        if (g->n > 0) {
            CD_CUDA(cudaMemcpyAsync(li, labels_in, sizeof(uint32_t) * g->n, cudaMemcpyHostToDevice, side.cs));
            if (da) CD_CUDA(cudaMemcpyAsync(da, active, g->n, cudaMemcpyHostToDevice, side.cs));
            if (db) CD_CUDA(cudaMemcpyAsync(db, bound, sizeof(uint32_t) * g->n, cudaMemcpyHostToDevice, side.cs));
        }
        if (da) act = da;
        if (db) bound = db;
        CD_CUDA(cudaEventRecord(side.ev[0], side.cs));
        if (g->nnz > 0) CD_CUDA(cudaMemcpyAsync(w, g->weights, sizeof(uint32_t) * g->nnz, cudaMemcpyHostToDevice,
                                                side.cs));
        CD_CUDA(cudaEventRecord(side.ev[1], side.cs));
        if (g->nnz > 0) CD_CUDA(cudaMemcpyAsync(cols, g->cols, sizeof(int32_t) * g->nnz, cudaMemcpyHostToDevice,
                                                side.cs));
        CD_CUDA(cudaEventRecord(side.ev[2], side.cs));
        CD_CUDA(cudaStreamWaitEvent(s, side.ev[0], 0));  // offsets and labels before the bucketing
        L.off = off; L.cols = cols; L.w = w; lin = li;
        return CD_OK;
    };
    if (host) {
        const int st = stage();
        g_stats.phase_ms[0] = since_ms(t_start);
        CD_TRY(hc.join());  // bad host inputs are reported as such, staged or not
        g_stats.phase_ms[1] = since_ms(t_start);
        CD_TRY(st);
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
    CD_TRY(prepare_level(L, lin, lout, p->k, sched, 1, sc, dglob, s, false, host ? side.ev[1] : nullptr));
    g_stats.phase_ms[2] = since_ms(t_start);
    if (host) CD_CUDA(cudaStreamWaitEvent(s, side.ev[2], 0));  // the columns before the sweep
    // refine: the driver's colour classes (0 = 8); Louvain: the singleton
    // rule's classes (0 = one class, every vertex decides together)
    SweepArgs a = make_args(L, lin, lout, act, bound, dglob, mode, p->subtract, ncol, p->sub_color);
    a.one_scan = p->one_scan;
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
    g_stats.full_sweeps = active ? 0 : 1;
    g_stats.entries_scanned = (int64_t)hg.g.scanned;
    g_stats.candidates = (int64_t)hg.g.cands;
    g_stats.moved = (int64_t)hg.g.moved;
    g_stats.gain_lo = hg.g.gain_lo;
    g_stats.gain_hi = hg.g.gain_hi;
    if (moved_out) *moved_out = (int64_t)hg.g.moved;
    if (gain_out) { gain_out[0] = hg.g.gain_lo; gain_out[1] = hg.g.gain_hi; }
    g_stats.phase_ms[3] = since_ms(t_start);
    return CD_OK;
}

int cd_modularity(const cd_csr* g, const uint32_t* labels, void* stream, double* q_out,
                  cd_modularity_parts* parts) {
    reset_stats();
    CD_TRY(check_csr(g, false));
    if (!labels) return CD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    Scratch sc(s);
    const int64_t* off = g->offsets;
    const int32_t* cols = g->cols;
    const uint32_t* w = g->weights;
    const uint32_t* lab = labels;
    if (g->memory == CD_MEM_HOST) {
        HostCheck hc;
        hc.start(g, labels);
        auto stage = [&]() -> int {
            int64_t* doff; int32_t* dc; uint32_t* dw; uint32_t* dl;
            CD_TRY(stage_in(g->offsets, g->n + 1, &doff, sc));
            CD_TRY(stage_in(g->cols, g->nnz, &dc, sc));
            CD_TRY(stage_in(g->weights, g->nnz, &dw, sc));
            CD_TRY(stage_in(labels, g->n, &dl, sc));
            off = doff; cols = dc; w = dw; lab = dl;
            return CD_OK;
        };
        const int st = stage();
        CD_TRY(hc.join());
        CD_TRY(st);
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

int cd_louvain(const cd_csr* g, const cd_params* p, uint32_t* labels_out, double* q_out) {
    reset_stats();
    CD_TRY(check_csr(g));
    CD_TRY(check_driver_params(p));
    if (p->one_scan) return CD_EINVAL;
    if (!labels_out) return CD_EINVAL;
    cudaStream_t s = (cudaStream_t)p->stream;
    cd_schedule sched;
    if (p->sched) sched = *p->sched; else default_schedule(p->k, &sched);
    Scratch sc(s);
    Globals* dglob;
    CD_TRY(sc.get(&dglob, 1));
    Level in;
    CD_TRY(input_level(g, sc, &in));
    uint32_t* top;
    CD_TRY(sc.get(&top, in.n));
    CD_CUDA(launch_iota(top, in.n, s));
    Level cur = in;
    double tol = p->tolerance;
    int64_t ncom = in.n;
    for (int pass = 0; pass < p->max_passes && cur.n > 0; ++pass) {
        uint32_t* lab;
        int64_t sw = 0;
        CD_TRY(local_move(cur, p, CD_MODE_LOUVAIN, tol, sched, sc, dglob, s, nullptr, &lab, &sw));
        if (pass == 0) in.K = cur.K;  // the input's weighted degrees, for the final Q
        g_stats.sweeps += sw;
        g_stats.passes += 1;
        uint32_t* dense;
        CD_TRY(sc.get(&dense, cur.n));
        int64_t nc = 0;
        CD_TRY(renumber_level(cur, lab, dense, sc, dglob, &nc, s));
        CD_CUDA(launch_compose(top, in.n, dense, s));
        ncom = nc;
        if (nc == cur.n || (double)nc > p->aggregation_tolerance * (double)cur.n) break;
        if (pass + 1 >= p->max_passes) break;
        Level next;
        if (p->agg_k > 0)
            CD_TRY(aggregate_mg_level(cur, dense, nc, p->agg_k, false, p->subtract, sched, sc, dglob, s, nullptr,
                                      nullptr, nullptr, &next));
        else
            CD_TRY(aggregate_level(cur, dense, nc, sc, dglob, s, nullptr, nullptr, nullptr, &next));
        cur = next;
        tol /= p->tolerance_drop;
    }
    g_stats.communities = ncom;
    double q = 0.0;
    CD_TRY(modularity_of(in, top, sc, dglob, s, &q));
    CD_TRY(emit_labels(g, top, labels_out, s));
    if (q_out) *q_out = q;
    return CD_OK;
}

int cd_louvain_batched(const cd_csr* graphs, int ngraphs, const cd_params* p, uint32_t* const* labels_out,
                       double* q_out, int64_t* sweeps_out) {
    reset_stats();
    if (!graphs || ngraphs < 1 || !labels_out) return CD_EINVAL;
    CD_TRY(check_driver_params(p));
    if (p->one_scan || p->skip_rule) return CD_EINVAL;
    const int G = ngraphs;
    const int mem = graphs[0].memory;
    for (int g = 0; g < G; ++g) {
        CD_TRY(check_csr(&graphs[g]));
        if (graphs[g].memory != mem) return CD_EINVAL;
        if (graphs[g].n > 0 && !labels_out[g]) return CD_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)p->stream;
    cd_schedule sched;
    if (p->sched) sched = *p->sched; else default_schedule(p->k, &sched);
    Scratch sc(s);
    Globals* dglob;
    CD_TRY(sc.get(&dglob, 1));
    std::vector<PackGraph> pg;
    std::vector<int64_t> vb0, n0, tstart;
    Level in;
    uint32_t *gid0, *lid0;
    CD_TRY(pack_union(graphs, G, sc, dglob, s, pg, vb0, n0, tstart, &in, &gid0, &lid0));
    const int64_t V = in.n;
    // ---- per-graph state
    BatchLevel bl;
    bl.G = G;
    int64_t *dvb, *dnv, *ddummy;
    uint32_t* ddense_dummy;
    CD_TRY(sc.get(&bl.two_m_g, G + 1));
    CD_TRY(sc.get(&bl.gdone, G + 1));
    CD_TRY(sc.get(&bl.gsweeps, G + 1));
    CD_TRY(sc.get(&bl.gstat, 3 * (G + 1)));
    CD_TRY(sc.get(&dvb, G));
    CD_TRY(sc.get(&dnv, G));
    CD_TRY(sc.get(&ddummy, G));
    CD_TRY(sc.get(&ddense_dummy, G));
    bl.vb = dvb;
    bl.nv = dnv;
    std::vector<int64_t> vb(vb0), nv(n0), dummy((size_t)G), gsw((size_t)G, 0);
    for (int g = 0; g < G; ++g) dummy[(size_t)g] = vb0[(size_t)g] + n0[(size_t)g];
    std::vector<uint8_t> finished((size_t)G);
    for (int g = 0; g < G; ++g) finished[(size_t)g] = n0[(size_t)g] == 0;
    uint32_t* top;
    CD_TRY(sc.get(&top, V));
    CD_CUDA(launch_iota(top, V, s));
    Level cur = in;
    const uint32_t* gid = gid0;
    double tol = p->tolerance;
    auto all_finished = [&]() {
        for (uint8_t f : finished) if (!f) return false;
        return true;
    };
    for (int pass = 0; pass < p->max_passes && !all_finished(); ++pass) {
        bl.gid = gid;
        bl.finished = finished;
        CD_CUDA(cudaMemcpyAsync(dvb, vb.data(), sizeof(int64_t) * G, cudaMemcpyHostToDevice, s));
        CD_CUDA(cudaMemcpyAsync(dnv, nv.data(), sizeof(int64_t) * G, cudaMemcpyHostToDevice, s));
        uint32_t* lab;
        int64_t sw = 0;
        CD_TRY(local_move(cur, p, CD_MODE_LOUVAIN, tol, sched, sc, dglob, s, nullptr, &lab, &sw, nullptr, &bl));
        g_stats.sweeps += sw;
        g_stats.passes += 1;
        std::vector<uint32_t> gs((size_t)G);
        CD_CUDA(cudaMemcpyAsync(gs.data(), bl.gsweeps, sizeof(uint32_t) * G, cudaMemcpyDeviceToHost, s));
        uint32_t* dense;
        CD_TRY(sc.get(&dense, cur.n));
        int64_t nc = 0;
        CD_TRY(renumber_level(cur, lab, dense, sc, dglob, &nc, s));  // synchronises s
        for (int g = 0; g < G; ++g)
            if (!finished[(size_t)g]) gsw[(size_t)g] += gs[(size_t)g];
        CD_CUDA(launch_compose(top, in.n, dense, s));
        // every graph's communities: a contiguous dense range ending at its
        // padding vertex
        std::vector<uint32_t> dd((size_t)G);
        CD_CUDA(cudaMemcpyAsync(ddummy, dummy.data(), sizeof(int64_t) * G, cudaMemcpyHostToDevice, s));
        CD_CUDA(launch_gather_u32(dense, ddummy, G, ddense_dummy, s));
        CD_CUDA(cudaMemcpyAsync(dd.data(), ddense_dummy, sizeof(uint32_t) * G, cudaMemcpyDeviceToHost, s));
        CD_CUDA(cudaStreamSynchronize(s));
        for (int g = 0; g < G; ++g) {
            const int64_t cb = g == 0 ? 0 : (int64_t)dd[(size_t)g - 1] + 1;
            const int64_t ncg = (int64_t)dd[(size_t)g] - cb;
            const size_t u = (size_t)g;
            if (!finished[u] && (ncg == nv[u] || (double)ncg > p->aggregation_tolerance * (double)nv[u]))
                finished[u] = 1;
            vb[u] = cb;
            nv[u] = ncg;
            dummy[u] = (int64_t)dd[u];
        }
        if (pass + 1 >= p->max_passes || all_finished()) break;
        Level next;
        if (p->agg_k > 0)
            CD_TRY(aggregate_mg_level(cur, dense, nc, p->agg_k, false, p->subtract, sched, sc, dglob, s, nullptr,
                                      nullptr, nullptr, &next));
        else
            CD_TRY(aggregate_level(cur, dense, nc, sc, dglob, s, nullptr, nullptr, nullptr, &next));
        // re-pack the super-vertex graph with aligned entry bases
        std::vector<int64_t> idx((size_t)2 * G), ob((size_t)2 * G);
        for (int g = 0; g < G; ++g) {
            idx[(size_t)2 * g] = vb[(size_t)g];
            idx[(size_t)2 * g + 1] = vb[(size_t)g] + nv[(size_t)g];
        }
        int64_t *didx, *dob;
        CD_TRY(stage_in(idx.data(), 2 * G, &didx, sc));
        CD_TRY(sc.get(&dob, 2 * G));
        CD_CUDA(launch_gather_i64(next.off, didx, 2 * G, dob, s));
        CD_CUDA(cudaMemcpyAsync(ob.data(), dob, sizeof(int64_t) * 2 * G, cudaMemcpyDeviceToHost, s));
        CD_CUDA(cudaStreamSynchronize(s));
        int64_t E2 = 0;
        tstart[0] = 0;
        for (int g = 0; g < G; ++g) {
            PackGraph& q = pg[(size_t)g];
            std::memset(&q, 0, sizeof(q));
            q.off = next.off; q.cols = next.cols; q.w = next.w;
            q.vsrc0 = vb[(size_t)g]; q.n = nv[(size_t)g];
            q.nnz = ob[(size_t)2 * g + 1] - ob[(size_t)2 * g];
            q.vbase = vb[(size_t)g]; q.ebase = E2;
            q.pad = (E2 + q.nnz + kPackAlign - 1) / kPackAlign * kPackAlign - (E2 + q.nnz);
            q.col_shift = 0; q.check_first = 0;
            E2 += q.nnz + q.pad;
            tstart[(size_t)g + 1] = tstart[(size_t)g] + pack_tiles(q);
        }
        Level packed;
        int64_t* uoff; int32_t* ucols; uint32_t* uw;
        uint32_t *gidn, *lidn;
        PackGraph* dpg; int64_t* dts;
        CD_TRY(sc.get(&uoff, nc + 1));
        CD_TRY(sc.get(&ucols, E2));
        CD_TRY(sc.get(&uw, E2));
        CD_TRY(sc.get(&gidn, nc));
        CD_TRY(sc.get(&lidn, nc));
        CD_TRY(stage_in(pg.data(), G, &dpg, sc));
        CD_TRY(stage_in(tstart.data(), G + 1, &dts, sc));
        CD_CUDA(cudaMemsetAsync(dglob, 0, sizeof(Globals), s));
        CD_CUDA(launch_pack(dpg, dts, G, tstart[(size_t)G], uoff, ucols, uw, gidn, lidn, nc, E2, dglob, s));
        HostGlobals hg;
        CD_TRY(read_globals(dglob, nullptr, 0, &hg, s));
        packed.n = nc; packed.nnz = E2; packed.off = uoff; packed.cols = ucols; packed.w = uw; packed.cid = lidn;
        cur = packed;
        gid = gidn;
        tol /= p->tolerance_drop;
    }
    // ---- outputs: labels inside every graph, modularity on every input
    int64_t* dcb;
    uint32_t *loc, *qlab;
    CD_TRY(stage_in(vb.data(), G, &dcb, sc));
    int64_t *dvb0, *dn0;
    CD_TRY(stage_in(vb0.data(), G, &dvb0, sc));
    CD_TRY(stage_in(n0.data(), G, &dn0, sc));
    CD_TRY(sc.get(&loc, V));
    CD_TRY(sc.get(&qlab, V));
    CD_CUDA(launch_batch_labels(top, gid0, V, G, dvb0, dcb, loc, qlab, s));
    uint64_t *K, *Sig;
    uint32_t* sz;
    unsigned long long* acc;
    CD_TRY(sc.get(&K, V));
    CD_TRY(sc.get(&Sig, V));
    CD_TRY(sc.get(&sz, V));
    CD_TRY(sc.get(&acc, 3 * G));
    CD_CUDA(cudaMemsetAsync(dglob, 0, sizeof(Globals), s));
    CD_CUDA(cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * 3 * G, s));
    CD_CUDA(launch_degrees(in.off, in.w, V, in.nnz, K, dglob, s));
    CD_CUDA(launch_totals(qlab, K, V, Sig, sz, dglob, s));
    CD_CUDA(launch_graph_two_m(K, dvb0, dn0, G, bl.two_m_g, s));
    CD_CUDA(launch_batch_modularity(in.off, in.cols, in.w, qlab, Sig, dvb0, dn0, G, acc, s));
    std::vector<unsigned long long> hacc((size_t)3 * G), htm((size_t)G);
    CD_CUDA(cudaMemcpyAsync(hacc.data(), acc, sizeof(unsigned long long) * 3 * G, cudaMemcpyDeviceToHost, s));
    CD_CUDA(cudaMemcpyAsync(htm.data(), bl.two_m_g, sizeof(unsigned long long) * G, cudaMemcpyDeviceToHost, s));
    const cudaMemcpyKind kind = mem == CD_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    for (int g = 0; g < G; ++g)
        if (n0[(size_t)g] > 0)
            CD_CUDA(cudaMemcpyAsync(labels_out[g], loc + vb0[(size_t)g], sizeof(uint32_t) * n0[(size_t)g], kind, s));
    HostGlobals hg;
    CD_TRY(read_globals(dglob, nullptr, 0, &hg, s));
    int64_t ncom = 0;
    for (int g = 0; g < G; ++g) {
        ncom += nv[(size_t)g];
        const u128 sq = ((u128)hacc[(size_t)3 * g + 2] << 64) | (u128)hacc[(size_t)3 * g + 1];
        const u128 tm = htm[(size_t)g];
        double q = 0.0;
        if (tm > 0) {
            const i128 num = (i128)(tm * (u128)hacc[(size_t)3 * g]) - (i128)sq;
            q = (double)((long double)num / ((long double)tm * (long double)tm));
        }
        if (q_out) q_out[g] = q;
        if (sweeps_out) sweeps_out[g] = gsw[(size_t)g];
    }
    g_stats.communities = ncom;
    return CD_OK;
}

int cd_autotune(const cd_csr* graphs, int ngraphs, const cd_params* p, const int* ks, int nks, double q_tol,
                cd_schedule* sched_out, int* k_out, cd_tune_report* report) {
    reset_stats();
    if (!graphs || ngraphs < 1 || !ks || nks < 1 || nks > CD_TUNE_MAX_K || !sched_out || !k_out) return CD_EINVAL;
    if (!(q_tol >= 0.0)) return CD_EINVAL;
    CD_TRY(check_driver_params(p));
    for (int i = 0; i < nks; ++i) {
        cd_params pk = *p;
        pk.k = ks[i];
        CD_TRY(check_params(&pk));
    }
    const int G = ngraphs;
    const int mem = graphs[0].memory;
    for (int g = 0; g < G; ++g) {
        CD_TRY(check_csr(&graphs[g]));
        if (graphs[g].memory != mem) return CD_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)p->stream;
    cd_schedule base;
    if (p->sched) base = *p->sched; else default_schedule(p->k, &base);
    cd_tune_report rep;
    std::memset(&rep, 0, sizeof(rep));
    std::vector<cd_schedule> tuned((size_t)nks, base);
    int64_t V = 0;
    {
        Scratch sc(s);
        Globals* dglob;
        CD_TRY(sc.get(&dglob, 1));
        std::vector<PackGraph> pg;
        std::vector<int64_t> vb0, n0, tstart;
        Level L;
        uint32_t *gid0, *lid0;
        CD_TRY(pack_union(graphs, G, sc, dglob, s, pg, vb0, n0, tstart, &L, &gid0, &lid0));
        V = L.n;
        L.reuse = true;
        uint32_t *la, *lb;
        CD_TRY(sc.get(&la, V));
        CD_TRY(sc.get(&lb, V));
        CD_TRY(sc.get(&L.movers, V));
        CD_CUDA(launch_iota(la, V, s));
        int64_t *dvb, *dnv;
        CD_TRY(stage_in(vb0.data(), G, &dvb, sc));
        CD_TRY(stage_in(n0.data(), G, &dnv, sc));
        unsigned long long *two_m_g, *gstat;
        uint8_t* gdone;
        CD_TRY(sc.get(&two_m_g, G + 1));
        CD_TRY(sc.get(&gstat, 3 * (G + 1)));
        CD_TRY(sc.get(&gdone, G + 1));
        CD_CUDA(cudaMemsetAsync(gdone, 0, (size_t)G + 1, s));
        CD_CUDA(cudaMemsetAsync(gdone + G, 1, 1, s));
        Timer tm;
        CD_TRY(tm.init(true));
        const size_t stat_off = offsetof(Globals, moved);
        const size_t stat_len = offsetof(Globals, sigma_in) - stat_off;
        // median time of one full sweep of the batch with schedule sc_try and k
        auto time_sweep = [&](const cd_schedule& st, int k, double* ms_out) -> int {
            CD_TRY(prepare_level(L, la, lb, k, st, 1, sc, dglob, s, true));
            CD_CUDA(launch_graph_two_m(L.K, dvb, dnv, G, two_m_g, s));
            SweepArgs a = make_args(L, la, lb, nullptr, nullptr, dglob, CD_MODE_LOUVAIN, p->subtract);
            a.gid = gid0;
            a.two_m_g = two_m_g;
            a.gdone = gdone;
            a.g_moved = gstat;
            a.g_gain_lo = gstat + (G + 1);
            a.g_gain_hi = gstat + 2 * (G + 1);
            float t[3];
            for (int r = 0; r < 3; ++r) {
                CD_CUDA(cudaMemsetAsync(reinterpret_cast<char*>(dglob) + stat_off, 0, stat_len, s));
                CD_CUDA(cudaEventRecord(tm.a, s));
                CD_TRY(launch_sweep(L, a, k, sc, s));
                CD_CUDA(cudaEventRecord(tm.b, s));
                CD_CUDA(cudaEventSynchronize(tm.b));
                CD_CUDA(cudaEventElapsedTime(&t[r], tm.a, tm.b));
                rep.trials += 1;
            }
            std::sort(t, t + 3);
            *ms_out = t[1];
            HostGlobals hg;
            return read_globals(dglob, nullptr, 0, &hg, s);
        };
        {
            cd_schedule b0 = base;
            if (ks[0] >= 32)
                for (int b = 0; b < b0.nbuckets; ++b) b0.lanes[b] = std::min(b0.lanes[b], 32);
            CD_TRY(time_sweep(b0, ks[0], &rep.default_ms));
        }
        for (int i = 0; i < nks; ++i) {
            const int k = ks[i];
            cd_schedule cur = base;
            const int cap = k >= 32 ? 32 : 256;
            for (int b = 0; b < cur.nbuckets; ++b) cur.lanes[b] = std::min(cur.lanes[b], cap);
            double best = 0.0;
            CD_TRY(time_sweep(cur, k, &best));
            if (k > 0) {
                // bands with rows, longest first
                for (int b = cur.nbuckets - 1; b >= 0; --b) {
                    bool any = false;
                    for (size_t q = (size_t)b; q + 1 < L.starts.size(); q += (size_t)L.bt.nb)
                        if (L.starts[q + 1] > L.starts[q]) any = true;
                    if (!any) continue;
                    const int l0 = cur.lanes[b];
                    for (int cand : {l0 / 2, l0 * 2}) {
                        if (cand < 1 || cand > cap) continue;
                        cd_schedule t = cur;
                        t.lanes[b] = cand;
                        double ms = 0.0;
                        CD_TRY(time_sweep(t, k, &ms));
                        if (ms < 0.98 * best) {
                            best = ms;
                            cur = t;
                        }
                    }
                }
                // band thresholds: each finite deg_max moves to 3/4 or 3/2 of
                // its value when the order of the bands allows it
                for (int b = 0; b + 1 < cur.nbuckets; ++b) {
                    const int64_t d0 = cur.deg_max[b];
                    for (int64_t cand : {d0 * 3 / 4, d0 * 3 / 2}) {
                        const int64_t lo = b > 0 ? cur.deg_max[b - 1] : 0;
                        if (cand <= lo || cand >= cur.deg_max[b + 1] || cand == d0) continue;
                        cd_schedule t = cur;
                        t.deg_max[b] = cand;
                        double ms = 0.0;
                        CD_TRY(time_sweep(t, k, &ms));
                        if (ms < 0.98 * best) {
                            best = ms;
                            cur = t;
                        }
                    }
                }
                // launch shape: one block per virtual block, or a resident grid
                for (int r : {4, 2}) {
                    cd_schedule t = cur;
                    t.blocks_per_sm = r;
                    double ms = 0.0;
                    CD_TRY(time_sweep(t, k, &ms));
                    if (ms < 0.98 * best) {
                        best = ms;
                        cur = t;
                    }
                }
            }
            tuned[(size_t)i] = cur;
            rep.sweep_ms[i] = best;
        }
    }
    // whole runs with each candidate
    std::vector<uint32_t*> outs((size_t)G, nullptr);
    std::vector<std::vector<uint32_t>> hbuf;
    uint32_t* dbuf = nullptr;
    if (mem == CD_MEM_HOST) {
        hbuf.resize((size_t)G);
        for (int g = 0; g < G; ++g) {
            hbuf[(size_t)g].resize((size_t)std::max<int64_t>(graphs[g].n, 1));
            outs[(size_t)g] = hbuf[(size_t)g].data();
        }
    } else {
        CD_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&dbuf), sizeof(uint32_t) * (size_t)std::max<int64_t>(V, 1), s));
        int64_t o = 0;
        for (int g = 0; g < G; ++g) {
            outs[(size_t)g] = dbuf + o;
            o += graphs[g].n + 1;
        }
    }
    std::vector<double> q((size_t)G);
    int rc = CD_OK;
    for (int i = 0; i < nks && rc == CD_OK; ++i) {
        cd_params pk = *p;
        pk.k = ks[i];
        pk.sched = &tuned[(size_t)i];
        cudaEvent_t e0, e1;
        if (cudaEventCreate(&e0) != cudaSuccess) { rc = CD_ECUDA; break; }
        if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); rc = CD_ECUDA; break; }
        cudaEventRecord(e0, s);
        rc = cd_louvain_batched(graphs, G, &pk, outs.data(), q.data(), nullptr);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        double qs = 0.0;
        for (double x : q) qs += x;
        rep.run_ms[i] = ms;
        rep.q_mean[i] = qs / G;
    }
    const int trials = rep.trials;
    if (dbuf) cudaFreeAsync(dbuf, s);
    cudaStreamSynchronize(s);
    if (rc != CD_OK) return rc;
    double qbest = rep.q_mean[0];
    for (int i = 1; i < nks; ++i) qbest = std::max(qbest, rep.q_mean[i]);
    int pick = -1;
    for (int i = 0; i < nks; ++i) {
        if (rep.q_mean[i] < qbest - q_tol * std::fabs(qbest)) continue;
        if (pick < 0 || rep.run_ms[i] < rep.run_ms[pick]) pick = i;
    }
    rep.chosen = pick;
    rep.trials = trials;
    *sched_out = tuned[(size_t)pick];
    *k_out = ks[pick];
    if (report) *report = rep;
    return CD_OK;
}

int cd_lpa(const cd_csr* g, const cd_params* p, uint32_t* labels_out, double* q_out) {
    reset_stats();
    CD_TRY(check_csr(g));
    CD_TRY(check_driver_params(p));
    if (!labels_out) return CD_EINVAL;
    cudaStream_t s = (cudaStream_t)p->stream;
    cd_schedule sched;
    if (p->sched) sched = *p->sched; else default_schedule(p->k, &sched);
    Scratch sc(s);
    Globals* dglob;
    CD_TRY(sc.get(&dglob, 1));
    Level in;
    CD_TRY(input_level(g, sc, &in));
    uint32_t* dense;
    CD_TRY(sc.get(&dense, in.n));
    if (in.n > 0) {
        uint32_t* lab;
        int64_t sw = 0;
        CD_TRY(local_move(in, p, CD_MODE_LPA, p->tolerance, sched, sc, dglob, s, nullptr, &lab, &sw));
        g_stats.sweeps = sw;
        g_stats.passes = 1;
        int64_t nc = 0;
        CD_TRY(renumber_level(in, lab, dense, sc, dglob, &nc, s));
        g_stats.communities = nc;
    }
    double q = 0.0;
    CD_TRY(modularity_of(in, dense, sc, dglob, s, &q));
    CD_TRY(emit_labels(g, dense, labels_out, s));
    if (q_out) *q_out = q;
    return CD_OK;
}

int cd_leiden(const cd_csr* g, const cd_params* p, uint32_t* labels_out, double* q_out) {
    reset_stats();
    CD_TRY(check_csr(g));
    CD_TRY(check_driver_params(p));
    if (p->one_scan) return CD_EINVAL;
    if (!labels_out) return CD_EINVAL;
    if (resolve_colors(p) < 2) return CD_EINVAL;  // refinement needs two colour classes or more
    cudaStream_t s = (cudaStream_t)p->stream;
    cd_schedule sched;
    if (p->sched) sched = *p->sched; else default_schedule(p->k, &sched);
    Scratch sc(s);
    Globals* dglob;
    CD_TRY(sc.get(&dglob, 1));
    Level in;
    CD_TRY(input_level(g, sc, &in));
    uint32_t *top, *result;
    CD_TRY(sc.get(&top, in.n));
    CD_TRY(sc.get(&result, in.n));
    CD_CUDA(launch_iota(top, in.n, s));
    CD_CUDA(launch_iota(result, in.n, s));
    Level cur = in;
    const uint32_t* init = nullptr;
    double tol = p->tolerance;
    int64_t ncom = in.n;
    for (int pass = 0; pass < p->max_passes && cur.n > 0; ++pass) {
        uint32_t* lab;
        int64_t sw = 0;
        CD_TRY(local_move(cur, p, CD_MODE_LOUVAIN, tol, sched, sc, dglob, s, init, &lab, &sw));
        if (pass == 0) in.K = cur.K;  // the input's weighted degrees, for the final Q
        g_stats.sweeps += sw;
        g_stats.passes += 1;
        uint32_t* dc;
        CD_TRY(sc.get(&dc, cur.n));
        int64_t nc = 0;
        CD_TRY(renumber_level(cur, lab, dc, sc, dglob, &nc, s));
        // result = community (bound) of every input vertex at this level
        CD_CUDA(cudaMemcpyAsync(result, top, sizeof(uint32_t) * in.n, cudaMemcpyDeviceToDevice, s));
        CD_CUDA(launch_compose(result, in.n, dc, s));
        ncom = nc;
        if (nc == cur.n || pass + 1 >= p->max_passes) break;
        Level rl = cur;
        uint32_t* rlab;
        CD_TRY(refine_level(rl, p, dc, sched, sc, dglob, s, &rlab));
        uint32_t* dr;
        CD_TRY(sc.get(&dr, cur.n));
        int64_t nr = 0;
        CD_TRY(renumber_level(cur, rlab, dr, sc, dglob, &nr, s));
        if (nr == cur.n || (double)nr > p->aggregation_tolerance * (double)cur.n) break;
        // next level: one vertex per sub-community, starting in its bound
        uint32_t* next_init;
        CD_TRY(sc.get(&next_init, nr));
        CD_CUDA(launch_scatter_bound(dr, dc, cur.n, next_init, s));
        CD_CUDA(launch_compose(top, in.n, dr, s));
        Level next;
        if (p->agg_k > 0)
            CD_TRY(aggregate_mg_level(cur, dr, nr, p->agg_k, true, p->subtract, sched, sc, dglob, s, nullptr,
                                      nullptr, nullptr, &next));
        else
            CD_TRY(aggregate_level(cur, dr, nr, sc, dglob, s, nullptr, nullptr, nullptr, &next));
        cur = next;
        init = next_init;
        tol /= p->tolerance_drop;
    }
    g_stats.communities = ncom;
    double q = 0.0;
    CD_TRY(modularity_of(in, result, sc, dglob, s, &q));
    CD_TRY(emit_labels(g, result, labels_out, s));
    if (q_out) *q_out = q;
    return CD_OK;
}

int cd_features(const cd_csr* g, const uint32_t* labels, const uint8_t* moved_last, const uint8_t* since_move,
                const float* attach, uint16_t* x_out, void* stream) {
    reset_stats();
    CD_TRY(check_csr(g));
    if (g->memory != CD_MEM_DEVICE || !labels || !x_out) return CD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    Scratch sc(s);
    Globals* dglob;
    CD_TRY(sc.get(&dglob, 1));
    Level L;
    CD_TRY(input_level(g, sc, &L));
    CD_TRY(sc.get(&L.K, L.n));
    CD_TRY(sc.get(&L.Sigma, L.n));
    CD_TRY(sc.get(&L.size, L.n));
    CD_CUDA(cudaMemsetAsync(dglob, 0, sizeof(Globals), s));
    if (L.n > 0) {
        CD_CUDA(launch_degrees(L.off, L.w, L.n, L.nnz, L.K, dglob, s));
        CD_CUDA(launch_totals(labels, L.K, L.n, L.Sigma, L.size, dglob, s));
    }
    HostGlobals hg;
    CD_TRY(read_globals(dglob, nullptr, 0, &hg, s));
    CD_CUDA(launch_features(L.off, L.K, labels, L.Sigma, L.size, hg.g.two_m, moved_last, since_move, attach, false,
                            L.n, x_out, s));
    CD_CUDA(cudaStreamSynchronize(s));
    return CD_OK;
}

int cd_mlp_forward(const uint16_t* x, int64_t n, const cd_mlp* model, float* p_out, void* stream) {
    reset_stats();
    if (!x || !model || !p_out || n < 0) return CD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    Scratch sc(s);
    float* param;
    CD_TRY(stage_model(model, sc, &param, s));
    CD_CUDA(launch_mlp_forward(x, n, param, p_out, nullptr, 0.0f, s));
    CD_CUDA(cudaStreamSynchronize(s));
    return CD_OK;
}

int cd_mlp_gradient(const uint16_t* x, const uint8_t* y, int64_t n, const cd_mlp* model, cd_mlp* grad_out,
                    double* loss_out, void* stream) {
    reset_stats();
    if (!x || !y || !model || !grad_out || n <= 0) return CD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    Scratch sc(s);
    float *param, *partial, *lpart, *grad, *loss;
    CD_TRY(stage_model(model, sc, &param, s));
    CD_TRY(sc.get(&partial, mlp_grad_blocks(n) * mlp_param_count()));
    CD_TRY(sc.get(&lpart, mlp_grad_blocks(n)));
    CD_TRY(sc.get(&grad, mlp_param_count()));
    CD_TRY(sc.get(&loss, 1));
    CD_CUDA(launch_mlp_grad(x, y, n, param, partial, lpart, grad, loss, s));
    float hl = 0;
    CD_CUDA(cudaMemcpyAsync(grad_out, grad, sizeof(float) * mlp_param_count(), cudaMemcpyDeviceToHost, s));
    CD_CUDA(cudaMemcpyAsync(&hl, loss, sizeof(float), cudaMemcpyDeviceToHost, s));
    CD_CUDA(cudaStreamSynchronize(s));
    if (loss_out) *loss_out = hl;
    return CD_OK;
}

int cd_mlp_train(const uint16_t* x, const uint8_t* y, int64_t n, int steps, double lr, cd_mlp* model,
                 double* loss_out, void* stream) {
    reset_stats();
    if (!x || !y || !model || n <= 0 || steps < 0 || !(lr > 0)) return CD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    Scratch sc(s);
    float *param, *partial, *lpart, *grad, *loss, *m1, *m2;
    const int P = mlp_param_count();
    CD_TRY(stage_model(model, sc, &param, s));
    CD_TRY(sc.get(&partial, mlp_grad_blocks(n) * P));
    CD_TRY(sc.get(&lpart, mlp_grad_blocks(n)));
    CD_TRY(sc.get(&grad, P));
    CD_TRY(sc.get(&loss, 1));
    CD_TRY(sc.get(&m1, P));
    CD_TRY(sc.get(&m2, P));
    CD_CUDA(cudaMemsetAsync(m1, 0, sizeof(float) * P, s));
    CD_CUDA(cudaMemsetAsync(m2, 0, sizeof(float) * P, s));
    for (int t = 1; t <= steps; ++t) {
        CD_CUDA(launch_mlp_grad(x, y, n, param, partial, lpart, grad, loss, s));
        CD_CUDA(launch_adam(param, grad, m1, m2, t, (float)lr, s));
    }
    float hl = 0;
    CD_CUDA(cudaMemcpyAsync(model, param, sizeof(float) * P, cudaMemcpyDeviceToHost, s));
    CD_CUDA(cudaMemcpyAsync(&hl, loss, sizeof(float), cudaMemcpyDeviceToHost, s));
    CD_CUDA(cudaStreamSynchronize(s));
    if (loss_out) *loss_out = hl;
    return CD_OK;
}

int cd_trace(const cd_csr* g, const cd_params* p, double sample_rate, uint16_t* x_out, uint8_t* y_out,
             int64_t capacity, int64_t* count_out) {
    reset_stats();
    CD_TRY(check_csr(g));
    CD_TRY(check_driver_params(p));
    if (g->memory != CD_MEM_DEVICE || !x_out || !y_out || capacity < 0 || !count_out) return CD_EINVAL;
    cudaStream_t s = (cudaStream_t)p->stream;
    cd_schedule sched;
    if (p->sched) sched = *p->sched; else default_schedule(p->k, &sched);
    Scratch sc(s);
    Globals* dglob;
    CD_TRY(sc.get(&dglob, 1));
    Level in;
    CD_TRY(input_level(g, sc, &in));
    Trace tr;
    tr.rate = sample_rate;
    tr.x = x_out;
    tr.y = y_out;
    tr.cap = capacity;
    if (in.n > 0) {
        uint32_t* lab;
        int64_t sw = 0;
        CD_TRY(local_move(in, p, CD_MODE_LOUVAIN, p->tolerance, sched, sc, dglob, s, nullptr, &lab, &sw, &tr));
        g_stats.sweeps = sw;
    }
    *count_out = tr.count;
    return CD_OK;
}

int cd_aggregate_mg(const cd_csr* g, const uint32_t* labels, int k, int subtract, int symmetric,
                    const cd_schedule* schedp, void* stream, uint32_t* dense_out, int64_t* offsets_out,
                    int32_t* cols_out, uint32_t* weights_out, int64_t* n_out, int64_t* nnz_out) {
    reset_stats();
    CD_TRY(check_csr(g));
    if (g->memory != CD_MEM_DEVICE) return CD_EINVAL;
    if (!(k == 1 || k == 2 || k == 4 || k == 8 || k == 16) || (subtract != 0 && subtract != 1)) return CD_EINVAL;
    if (!labels || !dense_out || !offsets_out || !n_out || !nnz_out) return CD_EINVAL;
    if (g->n > 0 && (!cols_out || !weights_out)) return CD_EINVAL;
    cd_schedule sched;
    if (schedp) { CD_TRY(check_schedule(schedp)); sched = *schedp; } else default_schedule(k, &sched);
    cudaStream_t s = (cudaStream_t)stream;
    Scratch sc(s);
    Globals* dglob;
    CD_TRY(sc.get(&dglob, 1));
    Level L;
    CD_TRY(input_level(g, sc, &L));
    // 2m for the sketch width
    uint64_t* K;
    CD_TRY(sc.get(&K, L.n));
    CD_CUDA(cudaMemsetAsync(dglob, 0, sizeof(Globals), s));
    CD_CUDA(launch_degrees(L.off, L.w, L.n, L.nnz, K, dglob, s));
    uint64_t* Sig;
    uint32_t* sz;
    CD_TRY(sc.get(&Sig, L.n));
    CD_TRY(sc.get(&sz, L.n));
    CD_CUDA(launch_totals(labels, K, L.n, Sig, sz, dglob, s));
    HostGlobals hg;
    CD_TRY(read_globals(dglob, nullptr, 0, &hg, s));
    L.two_m = hg.g.two_m;
    int64_t nc = 0;
    CD_TRY(renumber_level(L, labels, dense_out, sc, dglob, &nc, s));
    Level next;
    CD_TRY(aggregate_mg_level(L, dense_out, nc, k, symmetric != 0, subtract, sched, sc, dglob, s, offsets_out,
                              cols_out, weights_out, &next, g->nnz));
    CD_CUDA(cudaStreamSynchronize(s));
    *n_out = next.n;
    *nnz_out = next.nnz;
    g_stats.communities = nc;
    return CD_OK;
}

int cd_aggregate(const cd_csr* g, const uint32_t* labels, void* stream, uint32_t* dense_out,
                 int64_t* offsets_out, int32_t* cols_out, uint32_t* weights_out, int64_t* n_out,
                 int64_t* nnz_out) {
    reset_stats();
    CD_TRY(check_csr(g));
    if (g->memory != CD_MEM_DEVICE) return CD_EINVAL;
    if (!labels || !dense_out || !offsets_out || (g->nnz > 0 && (!cols_out || !weights_out)) || !n_out ||
        !nnz_out)
        return CD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    Scratch sc(s);
    Globals* dglob;
    CD_TRY(sc.get(&dglob, 1));
    Level L;
    CD_TRY(input_level(g, sc, &L));
    int64_t nc = 0;
    CD_TRY(renumber_level(L, labels, dense_out, sc, dglob, &nc, s));
    Level next;
    CD_TRY(aggregate_level(L, dense_out, nc, sc, dglob, s, offsets_out, cols_out, weights_out, &next));
    CD_CUDA(cudaStreamSynchronize(s));
    *n_out = next.n;
    *nnz_out = next.nnz;
    g_stats.communities = nc;
    return CD_OK;
}

}  // extern "C"
