// bc_api.cu -- the C ABI (include/bc_gb300.h): graph upload and checks,
// work-item plan, device memory plan, and the batch scheduler that drives the
// level loop of the multi-source path.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <string>
#include <mutex>
#include <thread>
#include <vector>

#include "bc_internal.cuh"
#include "plain.cuh"
#include "sched.cuh"
#include "weighted.cuh"
#include "many.cuh"
#include "dense.cuh"
#include "minplus.cuh"
#include "pairs.cuh"

namespace {

thread_local std::string g_err;

// BC_LOG=1 in the environment: bc_result writes one JSON line per run to stderr.
bool log_enabled() {
    static const bool on = [] {
        const char *v = std::getenv("BC_LOG");
        return v && *v && std::strcmp(v, "0") != 0;
    }();
    return on;
}

int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(e_ == cudaErrorMemoryAllocation ? BC_ERR_OOM : BC_ERR_CUDA,           \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                  \
    } while (0)

// Device blocks of closed graph handles, kept for the next handles (per
// device, best fit within twice the request): creating and closing handles
// then pays neither cudaMalloc nor cudaFree's wait for the whole device. A
// block enters the cache only from bc_destroy_graph, after the device has
// finished all work; an allocation that fails empties the cache and retries.
namespace devcache {
std::mutex mu;
struct Block {
    int dev;
    void *p;
    size_t bytes;
};
std::vector<Block> blocks;
size_t cached = 0;
constexpr size_t kMaxBytes = 24ull << 30;
thread_local bool t_recycle = false;  // set while bc_destroy_graph frees a handle

void trim(int dev) {  // dev < 0: every device
    std::lock_guard<std::mutex> lk(mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (size_t i = 0; i < blocks.size();) {
        if (dev < 0 || blocks[i].dev == dev) {
            cudaSetDevice(blocks[i].dev);
            cudaFree(blocks[i].p);
            cached -= blocks[i].bytes;
            blocks.erase(blocks.begin() + (long)i);
        } else {
            ++i;
        }
    }
    cudaSetDevice(cur);
}
cudaError_t alloc(void **p, size_t bytes, size_t *got) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> lk(mu);
        size_t best = SIZE_MAX;
        for (size_t i = 0; i < blocks.size(); ++i)
            if (blocks[i].dev == dev && blocks[i].bytes >= bytes && blocks[i].bytes / 2 <= bytes &&
                (best == SIZE_MAX || blocks[i].bytes < blocks[best].bytes))
                best = i;
        if (best != SIZE_MAX) {
            *p = blocks[best].p;
            *got = blocks[best].bytes;
            cached -= blocks[best].bytes;
            blocks.erase(blocks.begin() + (long)best);
            return cudaSuccess;
        }
    }
    e = cudaMalloc(p, bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        trim(dev);
        e = cudaMalloc(p, bytes);
    }
    if (e == cudaSuccess) *got = bytes;
    return e;
}
void release(void *p, size_t bytes) {
    if (!p) return;
    if (t_recycle) {
        int dev = 0;
        cudaGetDevice(&dev);
        std::lock_guard<std::mutex> lk(mu);
        if (cached + bytes <= kMaxBytes) {
            blocks.push_back({dev, p, bytes});
            cached += bytes;
            return;
        }
    }
    cudaFree(p);
}
}  // namespace devcache

template <class T>
struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
    size_t bytes = 0;
    void release() {
        devcache::release(p, bytes);
        p = nullptr;
        n = 0;
        bytes = 0;
    }
    cudaError_t ensure(size_t count) {
        if (count <= n && p) return cudaSuccess;
        release();
        size_t c = count ? count : 1;
        void *q = nullptr;
        size_t got = 0;
        cudaError_t e = devcache::alloc(&q, c * sizeof(T), &got);
        if (e == cudaSuccess) {
            p = static_cast<T *>(q);
            n = got / sizeof(T);
            bytes = got;
        }
        return e;
    }
};

// A DevBuf owned by one scope (cudaFree waits for the device's work first).
template <class T>
struct ScopedBuf : DevBuf<T> {
    ScopedBuf() = default;
    ScopedBuf(const ScopedBuf &) = delete;
    ScopedBuf &operator=(const ScopedBuf &) = delete;
    ~ScopedBuf() { this->release(); }
};

// Copy `count` elements from a host-or-device pointer into a host vector.
template <class T>
cudaError_t fetch(std::vector<T> &dst, const T *src, size_t count) {
    dst.resize(count);
    if (count == 0) return cudaSuccess;
    return cudaMemcpy(dst.data(), src, count * sizeof(T), cudaMemcpyDefault);
}

}  // namespace

// Work items of one level sweep: one per vertex, except vertices with more
// than `chunk` arcs, which are split into chunks combining through slots.
struct ItemPlan {
    int32_t chunk = 0, nitems = 0, nslots = 0;
    DevBuf<int32_t> blob;  // item_v, item_beg, item_end, item_slot [nitems], slot_first, slot_nch [nslots]
    const int32_t *item_v = nullptr, *item_beg = nullptr, *item_end = nullptr, *item_slot = nullptr;
    const int32_t *slot_first = nullptr, *slot_nch = nullptr;
    void release() {
        blob.release();
        item_v = item_beg = item_end = item_slot = slot_first = slot_nch = nullptr;
        chunk = nitems = nslots = 0;
    }
};

constexpr int kSweepLanes = 8;                    // concurrent batches of the unweighted sweep
constexpr int kSideStreams = 4;                   // side streams of the dense path's per-batch summaries
constexpr double kLaneBudgetBytes = 8.0 * (1 << 30);  // batch state of the extra lanes

// An extra lane of the batched sweep: its own stream, batch state, control
// blocks and BC accumulator, so that batches run concurrently (one lane's
// latency-bound levels overlap another lane's wide ones).
struct SweepLane {
    int dev = -1;  // device of the stream and buffers
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    int32_t W = 0, Lcap = 0, n = 0, s_levels = 2;
    size_t slots = 0;
    DevBuf<uint64_t> sigma, part;
    DevBuf<float> cval;
    DevBuf<uint16_t> Smask;
    DevBuf<uint32_t> wideflags, F, ufr, V, pmask, cnt;
    DevBuf<double> bc;
    bcgb::DevCtl *ctl = nullptr;
    bcgb::HostCtl *hctl = nullptr, *hctl_d = nullptr;
    void release() {
        sigma.release();
        part.release();
        cval.release();
        Smask.release();
        for (auto *b : {&wideflags, &F, &ufr, &V, &pmask, &cnt}) b->release();
        bc.release();
        if (ctl) cudaFree(ctl);
        if (hctl) cudaFreeHost(hctl);
        if (ev) cudaEventDestroy(ev);
        if (st) cudaStreamDestroy(st);
        ctl = nullptr;
        hctl = hctl_d = nullptr;
        ev = nullptr;
        st = nullptr;
        W = Lcap = n = 0;
        slots = 0;
        dev = -1;
    }
};

// Lanes of destroyed graphs are kept for the next graph on the same device
// (stream, control blocks and buffers, which grow when a graph needs more):
// a program that builds many graphs in turn allocates them once.
namespace lane_pool {
std::mutex mu;
std::vector<SweepLane> idle;
constexpr size_t kMax = 16;

// Move lane `from` into `to` (the fields are plain handles and pointers).
void move_lane(SweepLane &to, SweepLane &from) {
    to = from;
    from = SweepLane{};
}
bool take(SweepLane &ln, int dev) {
    std::lock_guard<std::mutex> lk(mu);
    for (size_t i = 0; i < idle.size(); ++i)
        if (idle[i].dev == dev) {
            move_lane(ln, idle[i]);
            idle.erase(idle.begin() + (long)i);
            // the progress block carries the previous owner's batch numbers
            std::memset(ln.hctl, 0, sizeof(bcgb::HostCtl));
            return true;
        }
    return false;
}
void give(SweepLane &ln) {
    if (!ln.st) return;
    cudaStreamSynchronize(ln.st);  // nothing of the previous owner may still run on it
    std::lock_guard<std::mutex> lk(mu);
    if (idle.size() < kMax) {
        idle.emplace_back();
        move_lane(idle.back(), ln);
    } else {
        ln.release();
    }
}
}  // namespace lane_pool

struct bc_graph {
    int32_t n = 0;
    int64_t narcs = 0;
    bool weighted = false;
    bool directed = false;
    std::vector<int32_t> h_row_ptr;     // host copy (work-item plans)
    std::vector<int32_t> h_row_ptr_in;  // directed: in-arc CSR rows (forward plan)
    std::vector<int32_t> rank;       // landmark-order position of every vertex (built on first use)
    DevBuf<int32_t> row_ptr, col, w;
    DevBuf<int32_t> row_ptr_in, col_in, w_in;  // directed: the transpose

    // work items of the forward and backward sweeps (each for its chunk size)
    ItemPlan fplan, bplan;

    // multi-source batch state for (W, Lcap)
    int32_t W = 0, Lcap = 0;
    int32_t s_levels = 2;  // masked-row buffers: Lcap (one per level) or 2 (by parity)
    DevBuf<uint64_t> sigma, part;
    DevBuf<float> cval;
    DevBuf<uint16_t> Smask;
    DevBuf<uint32_t> wideflags, F, ufr, V, pmask, cnt;
    // direction of level 0 -> 1 (top-down while the batch's source arcs are
    // fewer than 2m / alpha) and the look-ahead's tail threshold (one level
    // ahead once a shrinking frontier holds at most beta x n vertices)
    float alpha = 1.0f, beta = 1.0f / 64.0f;
    uint64_t dev_wait_ns = 0;  // bound on each device wait (0: the kernels' default)
    uint32_t test_hold = 0;    // BC_TEST_WAIT_EXPIRY
    bool bottom_up0 = false;   // BC_FORCE_BOTTOMUP: level 0 -> 1 pulled too
    // options bc_run uses when given NULL (bc_autotune / bc_set_default_options)
    bool has_defaults = false;
    bc_options defaults{};
    bc_options last_opt{};  // what the last bc_run was given (after the NULL substitution)
    std::chrono::steady_clock::time_point run_t0;  // host clock at the last bc_run's start (BC_LOG)

    // results
    DevBuf<double> bc;
    DevBuf<int32_t> sources;
    DevBuf<int32_t> src_index;  // caller's index of each staged source (reordered runs)
    bool reordered = false;
    DevBuf<uint64_t> h_sigma, h_dist;
    DevBuf<int64_t> dist_sum, reach;
    int32_t last_nsrc = 0;
    bool has_run = false, has_hash = false;
    cudaStream_t last_stream = nullptr;

    bcgb::DevCtl *ctl = nullptr;
    bcgb::HostCtl *hctl = nullptr;    // host view
    bcgb::HostCtl *hctl_d = nullptr;  // device view
    uint32_t seq = 0;
    SweepLane lanes[kSweepLanes - 1];  // lanes 1.. of the concurrent sweep (lane 0 is the state above)
    cudaEvent_t ev0 = nullptr;        // lane 0's join / fork event
    cudaStream_t side[kSideStreams] = {};     // independent per-batch launches of the dense path
    cudaEvent_t side_ev[kSideStreams] = {};
    cudaEvent_t side_fork = nullptr;

    // timing
    struct Ev {
        cudaEvent_t a, b;
        int kind;
        int level;  // sweep level of the launch (-1: none)
    };
    std::vector<Ev> evpool;
    size_t evused = 0;
    bool timing = false;
    int64_t launches = 0;

    bcgb::PlainState plain;

    // dense (tensor-core) levels: bf16 adjacency, per-batch limb rows, TMA
    // maps, and the state of a group of batches run in lockstep
    int32_t npad = 0;
    DevBuf<__nv_bfloat16> dA, dX;
    DevBuf<uint8_t> dA8;  // the adjacency in e4m3 (forward levels with 4-bit limbs)
    DevBuf<bcgb::DenseCtl> dctl;
    bcgb::DenseMaps maps{};
    double dense_flops = 0.0, dense_flops_f8 = 0.0;  // tensor-core work: bf16 and e4m3 products
    int32_t gNB = 0, gLcap = 0;  // group capacity (batches) and its level capacity
    DevBuf<uint64_t> gsigma;
    DevBuf<uint32_t> gF, gV, gufr;
    DevBuf<double> gbcpart;
    DevBuf<int32_t> gmeta;  // [3][gNB]: active list, valid sources, depth

    // weighted algebraic forward (BC_DENSE on a weighted graph): dense weights
    DevBuf<int32_t> mpW;

    // weighted path: per-wave state
    int32_t maxw = 1;
    int32_t wG = 0, wK = 0, wC = 0;
    DevBuf<int32_t> wdist, worder, wgrp, wslots, wpos, wsrc;
    DevBuf<uint64_t> wds;     // packed per-vertex state of the packed kernel
    DevBuf<uint8_t> wredo;    // sources whose counts need 64 bits
    std::vector<int32_t> h_sources;  // host copy of the staged source list
    DevBuf<uint64_t> wsigma;
    DevBuf<float> wcval, wrows;
    // the weighted sweep's relabelled copy of the graph (built on first
    // use): the CSR (and a directed graph's in-arc CSR) in a numbering with
    // locality, old -> new ids (wperm, also on the host) and new -> old
    // (wvid), and a run's sources in the new numbering
    bool relabel_ok = false;
    std::vector<int32_t> h_wperm;
    DevBuf<int32_t> prow_ptr, pcol, pw, prow_ptr_in, pcol_in, pw_in, wperm, wvid, wpsrc;
    // lanes 1..3 of the weighted waves: stream, packed state, rows, BC accumulator
    struct WLane {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        DevBuf<int32_t> order, grp, slots;
        DevBuf<uint64_t> ds;
        DevBuf<float> rows;
        DevBuf<double> bc;
    };
    WLane wl[3];
    cudaEvent_t wev = nullptr;
};

namespace {

void free_graph(bc_graph *g) {
    for (auto *b : {&g->row_ptr, &g->col, &g->w, &g->row_ptr_in, &g->col_in, &g->w_in, &g->sources, &g->src_index})
        b->release();
    g->fplan.release();
    g->bplan.release();
    g->sigma.release();
    g->Smask.release();
    g->wideflags.release();
    g->part.release();
    g->cval.release();
    for (auto *b : {&g->F, &g->ufr, &g->V, &g->pmask, &g->cnt}) b->release();
    g->mpW.release();
    g->gsigma.release();
    for (auto *b : {&g->gF, &g->gV, &g->gufr}) b->release();
    g->gbcpart.release();
    g->gmeta.release();
    for (auto *b : {&g->wpos, &g->wsrc}) b->release();
    for (auto &l : g->wl) {
        for (auto *b : {&l.order, &l.grp, &l.slots}) b->release();
        l.ds.release();
        l.rows.release();
        l.bc.release();
        if (l.ev) cudaEventDestroy(l.ev);
        if (l.st) cudaStreamDestroy(l.st);
    }
    if (g->wev) cudaEventDestroy(g->wev);
    for (int i = 0; i < kSideStreams; ++i) {
        if (g->side_ev[i]) cudaEventDestroy(g->side_ev[i]);
        if (g->side[i]) cudaStreamDestroy(g->side[i]);
    }
    if (g->side_fork) cudaEventDestroy(g->side_fork);
    g->wds.release();
    g->wredo.release();
    g->bc.release();
    g->h_sigma.release();
    g->h_dist.release();
    g->dist_sum.release();
    g->reach.release();
    if (g->ctl) cudaFree(g->ctl);
    if (g->hctl) cudaFreeHost(g->hctl);
    for (auto &ln : g->lanes) lane_pool::give(ln);
    if (g->ev0) cudaEventDestroy(g->ev0);
    for (auto &e : g->evpool) {
        cudaEventDestroy(e.a);
        cudaEventDestroy(e.b);
    }
    bcgb::plain_free(g->plain);
    g->dA.release();
    g->dA8.release();
    g->dX.release();
    g->dctl.release();
    for (auto *b : {&g->wdist, &g->worder, &g->wgrp, &g->wslots}) b->release();
    for (auto *b : {&g->prow_ptr, &g->pcol, &g->pw, &g->prow_ptr_in, &g->pcol_in, &g->pw_in, &g->wperm, &g->wvid,
                    &g->wpsrc})
        b->release();
    g->wsigma.release();
    g->wcval.release();
    g->wrows.release();
    delete g;
}

// Host check of the paper's graph model: every arc has its reverse with the
// same weight, no self-loops, no duplicate arcs, positive weights.
int check_graph(int32_t n, const std::vector<int32_t> &rp, const std::vector<int32_t> &col,
                const std::vector<int32_t> *w, bool directed) {
    if (rp[0] != 0) return fail(BC_ERR_ARG, "row_ptr[0] != 0");
    for (int32_t v = 0; v < n; ++v)
        if (rp[v + 1] < rp[v]) return fail(BC_ERR_ARG, "row_ptr not non-decreasing");
    const int64_t m = rp[n];
    int64_t maxw = 1;
    for (int64_t e = 0; e < m; ++e) {
        if (col[e] < 0 || col[e] >= n) return fail(BC_ERR_ARG, "col id out of range");
        if (w) {
            if ((*w)[e] <= 0) return fail(BC_ERR_WEIGHT, "non-positive weight");
            maxw = std::max<int64_t>(maxw, (*w)[e]);
        }
    }
    if (w && (int64_t)n * maxw >= (int64_t(1) << 31))
        return fail(BC_ERR_WEIGHT, "n * max weight >= 2^31 (distances would not fit int32)");
    // sorted copy of every row (with weights) for reverse-arc lookups
    std::vector<std::pair<int32_t, int32_t>> arcs(m);
    for (int32_t v = 0; v < n; ++v) {
        for (int64_t e = rp[v]; e < rp[v + 1]; ++e) arcs[e] = {col[e], w ? (*w)[e] : 1};
        std::sort(arcs.begin() + rp[v], arcs.begin() + rp[v + 1]);
        for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
            if (arcs[e].first == v) return fail(BC_ERR_NOT_SYMMETRIC, "self-loop at vertex " + std::to_string(v));
            if (e > rp[v] && arcs[e].first == arcs[e - 1].first)
                return fail(BC_ERR_NOT_SYMMETRIC, "duplicate arc at vertex " + std::to_string(v));
        }
    }
    if (directed) return BC_OK;
    for (int32_t v = 0; v < n; ++v) {
        for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
            const int32_t u = arcs[e].first;
            auto lo = arcs.begin() + rp[u], hi = arcs.begin() + rp[u + 1];
            auto it = std::lower_bound(lo, hi, std::make_pair(v, INT32_MIN));
            if (it == hi || it->first != v) return fail(BC_ERR_NOT_SYMMETRIC, "missing reverse arc");
            if (it->second != arcs[e].second) return fail(BC_ERR_NOT_SYMMETRIC, "asymmetric weight");
        }
    }
    return BC_OK;
}

// Work items: one per vertex, except vertices with more than `chunk` arcs,
// which are split into chunks that combine through partial slots. Heavy
// chunks come first, then vertices by descending degree.
int build_items(bc_graph *g, ItemPlan &pl, int32_t chunk, const std::vector<int32_t> &rp) {
    if (pl.chunk == chunk && pl.item_v) return BC_OK;
    const int32_t n = g->n;
    // items: the chunks of the split vertices (in vertex order), then the
    // other vertices by decreasing degree (a stable counting sort: degree <= chunk)
    int64_t nitems = 0, nslots = 0;
    std::vector<int32_t> cnt((size_t)chunk + 2, 0);
    for (int32_t v = 0; v < n; ++v) {
        const int64_t deg = rp[v + 1] - rp[v];
        if (deg > chunk) {
            const int64_t nch = (deg + chunk - 1) / chunk;
            nitems += nch;
            nslots += nch;
        } else {
            ++cnt[(size_t)(chunk - deg) + 1];
            ++nitems;
        }
    }
    for (size_t x = 1; x < cnt.size(); ++x) cnt[x] += cnt[x - 1];
    // one host block, one device allocation and one copy for the six arrays
    std::vector<int32_t> h((size_t)(4 * nitems + 2 * nslots));
    int32_t *iv = h.data(), *ib = iv + nitems, *ie = ib + nitems, *is = ie + nitems;
    int32_t *sf = is + nitems, *sn = sf + nslots;
    int64_t k = 0;
    for (int32_t v = 0; v < n; ++v) {
        const int64_t deg = rp[v + 1] - rp[v];
        if (deg <= chunk) continue;
        const int64_t nch = (deg + chunk - 1) / chunk;
        const int32_t first = (int32_t)k;
        for (int64_t c = 0; c < nch; ++c, ++k) {
            iv[k] = v;
            ib[k] = (int32_t)(rp[v] + c * chunk);
            ie[k] = (int32_t)std::min<int64_t>(rp[v + 1], rp[v] + (c + 1) * chunk);
            is[k] = (int32_t)k;
            sf[k] = first;
            sn[k] = (int32_t)nch;
        }
    }
    for (int32_t v = 0; v < n; ++v) {
        const int64_t deg = rp[v + 1] - rp[v];
        if (deg > chunk) continue;
        const int64_t t = nslots + cnt[(size_t)(chunk - deg)]++;
        iv[t] = v;
        ib[t] = rp[v];
        ie[t] = rp[v + 1];
        is[t] = -1;
    }
    pl.nitems = (int32_t)nitems;
    pl.nslots = (int32_t)nslots;
    CK(pl.blob.ensure(h.size()));
    if (!h.empty()) CK(cudaMemcpy(pl.blob.p, h.data(), h.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    pl.item_v = pl.blob.p;
    pl.item_beg = pl.item_v + nitems;
    pl.item_end = pl.item_beg + nitems;
    pl.item_slot = pl.item_end + nitems;
    pl.slot_first = pl.item_slot + nitems;
    pl.slot_nch = pl.slot_first + nslots;
    pl.chunk = chunk;
    // partial slots depend on the plans: force the state to be re-sized
    g->W = 0;
    return BC_OK;
}

// The sweeps' plans (measured on R-MAT with eight concurrent lanes: 256 arcs
// per chunk in both sweeps; one lane alone prefers 128 in the backward, but
// with lanes fewer, larger items win). An explicit chunk size applies to both.
// Two plans are kept because the forward pulls over in-arcs and the backward
// over out-arcs (different on directed graphs).
int build_plans(bc_graph *g, const bc_options *opt) {
    const int32_t fc = (opt && opt->chunk > 0) ? opt->chunk : 256;
    const int32_t bch = (opt && opt->chunk > 0) ? opt->chunk : 256;
    // the forward sweep pulls over in-arcs, the backward over out-arcs
    int r = build_items(g, g->fplan, fc, g->directed ? g->h_row_ptr_in : g->h_row_ptr);
    if (!r) r = build_items(g, g->bplan, bch, g->h_row_ptr);
    return r;
}

void use_plan(bcgb::MsParams &p, const ItemPlan &pl) {
    p.nitems = pl.nitems;
    p.item_v = pl.item_v;
    p.item_beg = pl.item_beg;
    p.item_end = pl.item_end;
    p.item_slot = pl.item_slot;
    p.slot_first = pl.slot_first;
    p.slot_nch = pl.slot_nch;
}

// One masked-row buffer per level lets the backward read each pair's count
// as 2 bytes (instead of the 8-byte sigma); it costs Lcap rows per vertex, so
// deep graphs (a large level capacity) keep the two parity buffers instead.
constexpr double kSLevelsBudget = 1.5 * (1 << 30);
int s_levels_for(size_t n, size_t B, int Lcap) {
    return (double)Lcap * (double)n * (double)B * 2.0 <= kSLevelsBudget ? Lcap : 2;
}

int ensure_state(bc_graph *g, int W, int Lcap) {
    if (g->W == W && g->Lcap >= Lcap && g->sigma.p) return BC_OK;
    const size_t n = (size_t)std::max(g->n, 1);
    const size_t B = 32 * (size_t)W;
    const size_t nw32 = (n + 31) / 32;
    CK(g->sigma.ensure(n * B));
    g->s_levels = s_levels_for(n, B, Lcap);
    CK(g->Smask.ensure((size_t)g->s_levels * n * B));
    CK(g->wideflags.ensure((size_t)2 * Lcap));  // per-level flags, then the frontier sizes
    CK(g->cval.ensure(2 * n * B));
    CK(g->F.ensure((size_t)Lcap * n * W));
    CK(g->ufr.ensure((size_t)Lcap * nw32));
    CK(g->V.ensure(2 * n * W));
    const size_t slots = (size_t)std::max({g->fplan.nslots, g->bplan.nslots, 1});
    CK(g->part.ensure(slots * B));
    CK(g->pmask.ensure(slots * W));
    CK(g->cnt.ensure(slots));
    CK(cudaMemset(g->cnt.p, 0, g->cnt.n * sizeof(uint32_t)));
    g->W = W;
    g->Lcap = Lcap;
    return BC_OK;
}

size_t timer_begin(bc_graph *g, cudaStream_t st, int kind, int level = -1) {
    g->launches++;
    if (!g->timing) return SIZE_MAX;
    if (g->evused == g->evpool.size()) {
        bc_graph::Ev e{};
        cudaEventCreate(&e.a);
        cudaEventCreate(&e.b);
        g->evpool.push_back(e);
    }
    const size_t idx = g->evused++;
    g->evpool[idx].kind = kind;
    g->evpool[idx].level = level;
    cudaEventRecord(g->evpool[idx].a, st);
    return idx;
}

void timer_end(bc_graph *g, cudaStream_t st, size_t idx) {
    if (idx != SIZE_MAX) cudaEventRecord(g->evpool[idx].b, st);
}

// Scoped launch accounting: counts the launch and, with BC_TIMING, brackets
// it with CUDA events on the launching stream.
struct Timer {
    bc_graph *g;
    cudaStream_t st;
    size_t idx;
    Timer(bc_graph *g_, cudaStream_t s, int k, int level = -1) : g(g_), st(s), idx(timer_begin(g_, s, k, level)) {}
    ~Timer() { timer_end(g, st, idx); }
    Timer(const Timer &) = delete;
    Timer &operator=(const Timer &) = delete;
};

size_t hook_begin(void *ctx, int kind) {
    auto *c = static_cast<std::pair<bc_graph *, cudaStream_t> *>(ctx);
    return timer_begin(c->first, c->second, kind);
}
void hook_end(void *ctx, size_t idx) {
    auto *c = static_cast<std::pair<bc_graph *, cudaStream_t> *>(ctx);
    timer_end(c->first, c->second, idx);
}

bcgb::MsParams make_params(bc_graph *g) {
    bcgb::MsParams p{};
    p.n = g->n;
    p.nw32 = (std::max(g->n, 1) + 31) / 32;
    p.Lcap = g->Lcap;
    p.row_ptr = g->row_ptr.p;
    p.col = g->col.p;
    p.col_f = g->directed ? g->col_in.p : g->col.p;
    use_plan(p, g->fplan);
    p.sigma = g->sigma.p;
    p.S = g->Smask.p;
    p.s_levels = g->s_levels;
    p.wide = g->wideflags.p;
    p.lsize = g->wideflags.p + g->Lcap;
    p.cval = g->cval.p;
    p.F = g->F.p;
    p.ufr = g->ufr.p;
    p.V = g->V.p;
    p.part = g->part.p;
    p.pmask = g->pmask.p;
    p.cnt = g->cnt.p;
    p.wait_ns = g->dev_wait_ns;
    p.test_hold = g->test_hold;
    p.bc = g->bc.p;
    p.ctl = g->ctl;
    p.hctl = g->hctl_d;
    return p;
}

// Batch state of sweep lane k >= 1 (same shapes as ensure_state's), plus its
// stream, control blocks and BC accumulator, created on first use.
int ensure_lane(bc_graph *g, SweepLane &ln, int W, int Lcap) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    bool fresh = false;
    if (!ln.st) fresh = lane_pool::take(ln, dev);
    if (!ln.st) {
        fresh = true;
        ln.dev = dev;
        CK(cudaStreamCreateWithFlags(&ln.st, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&ln.ev, cudaEventDisableTiming));
        CK(cudaMalloc((void **)&ln.ctl, sizeof(bcgb::DevCtl)));
        CK(cudaMemset(ln.ctl, 0, sizeof(bcgb::DevCtl)));
        CK(cudaHostAlloc((void **)&ln.hctl, sizeof(bcgb::HostCtl), cudaHostAllocMapped | cudaHostAllocPortable));
        std::memset(ln.hctl, 0, sizeof(bcgb::HostCtl));
        CK(cudaHostGetDevicePointer((void **)&ln.hctl_d, ln.hctl, 0));
    }
    const size_t slots = (size_t)std::max({g->fplan.nslots, g->bplan.nslots, 1});
    if (!fresh && ln.W == W && ln.Lcap >= Lcap && ln.n >= g->n && ln.slots >= slots && ln.sigma.p) return BC_OK;
    const size_t n = (size_t)std::max(g->n, 1);
    const size_t B = 32 * (size_t)W;
    const size_t nw32 = (n + 31) / 32;
    CK(ln.sigma.ensure(n * B));
    ln.s_levels = s_levels_for(n, B, Lcap);
    CK(ln.Smask.ensure((size_t)ln.s_levels * n * B));
    CK(ln.wideflags.ensure((size_t)2 * Lcap));  // per-level flags, then the frontier sizes
    CK(ln.cval.ensure(2 * n * B));
    CK(ln.F.ensure((size_t)Lcap * n * W));
    CK(ln.ufr.ensure((size_t)Lcap * nw32));
    CK(ln.V.ensure(2 * n * W));
    CK(ln.part.ensure(slots * B));
    CK(ln.pmask.ensure(slots * W));
    CK(ln.cnt.ensure(slots));
    CK(cudaMemset(ln.cnt.p, 0, ln.cnt.n * sizeof(uint32_t)));
    CK(ln.bc.ensure(n));
    ln.W = W;
    ln.Lcap = Lcap;
    ln.n = (int32_t)n;
    ln.slots = slots;
    return BC_OK;
}

// Kernel parameters of sweep lane k (0: the graph's own state).
bcgb::MsParams lane_params(bc_graph *g, int k) {
    bcgb::MsParams p = make_params(g);
    if (k == 0) return p;
    SweepLane &ln = g->lanes[k - 1];
    p.Lcap = ln.Lcap;
    p.sigma = ln.sigma.p;
    p.S = ln.Smask.p;
    p.s_levels = ln.s_levels;
    p.wide = ln.wideflags.p;
    p.lsize = ln.wideflags.p + ln.Lcap;
    p.cval = ln.cval.p;
    p.F = ln.F.p;
    p.ufr = ln.ufr.p;
    p.V = ln.V.p;
    p.part = ln.part.p;
    p.pmask = ln.pmask.p;
    p.cnt = ln.cnt.p;
    p.bc = ln.bc.p;
    p.ctl = ln.ctl;
    p.hctl = ln.hctl_d;
    return p;
}

// Per-run settings of the level sweeps taken from the options (NULL: defaults).
void set_run_options(bc_graph *g, const bc_options *opt) {
    g->alpha = (opt && opt->alpha > 0.0f) ? opt->alpha : 1.0f;
    g->beta = (opt && opt->beta > 0.0f) ? std::min(opt->beta, 1.0f) : 1.0f / 64.0f;
    g->dev_wait_ns = (opt && opt->device_wait_us > 0) ? (uint64_t)opt->device_wait_us * 1000ull : 0ull;
    g->test_hold = (opt && (opt->flags & BC_TEST_WAIT_EXPIRY)) ? 16u : 0u;
    g->bottom_up0 = opt && (opt->flags & BC_FORCE_BOTTOMUP);
}

int resolve_batch(const bc_options *opt, int *W) {
    int b = (opt && opt->batch) ? opt->batch : 256;
    if (b % 32 != 0 || !bcgb::ms_supported_width(b / 32)) return fail(BC_ERR_ARG, "batch must be 32, 64, 128 or 256");
    *W = b / 32;
    return BC_OK;
}

// Upload (or copy) a source list; returns its length.
// Landmark order of the vertices. The batches of the level sweep run best
// when the sources of one 32-source word have nearly the same distances to
// every vertex: their masked rows are then either useful for most of the
// word or not needed at all. Vertices are ordered lexicographically by their
// BFS distances to K landmarks (the K highest-degree vertices, ties by id),
// then by id; rank[v] is v's position. The distances come from one batched
// forward pass on the device (ensure_rank); here, stable counting sorts,
// last key first.
// A barrier for the few host threads of rank_from_dist.
struct SpinBarrier {
    std::atomic<int> count{0}, gen{0};
    int n;
    explicit SpinBarrier(int n_) : n(n_) {}
    void wait() {
        const int g = gen.load(std::memory_order_acquire);
        if (count.fetch_add(1, std::memory_order_acq_rel) == n - 1) {
            count.store(0, std::memory_order_relaxed);
            gen.fetch_add(1, std::memory_order_release);
        } else {
            while (gen.load(std::memory_order_acquire) == g) std::this_thread::yield();
        }
    }
};

void rank_from_dist(bc_graph *g, std::vector<int32_t> &dist, int k) {
    const int32_t n = g->n;
    // Each vertex's key: its distances to landmarks 0, 1, ... (unreachable
    // after every reachable distance) packed most significant first into 128
    // bits, each field just wide enough for its landmark's largest value;
    // landmarks that no longer fit are left out. A stable LSD radix sort on
    // the key (8-bit digits, digits every key shares skipped) orders the
    // vertices lexicographically by their distance profiles, ties by id. The
    // host threads take contiguous ranges; the counts of a pass are laid out
    // thread by thread within each digit value, which keeps the sort stable.
    const int T = n < 16384 ? 1 : std::max(1, std::min<int>(8, (int)std::thread::hardware_concurrency()));
    std::vector<uint64_t> key[2][2];  // [buffer][hi, lo]
    for (auto &b : key)
        for (auto &x : b) x.assign((size_t)n, 0);
    std::vector<int32_t> ord[2];
    ord[0].resize(n);
    ord[1].resize(n);
    std::vector<int32_t> dm((size_t)T * k, 0);
    std::vector<size_t> cnt((size_t)T * 256);
    int final_cur = 0;
    bool skip = false;
    SpinBarrier bar(T);
    auto work = [&](int t) {
        int cur = 0;  // which buffer holds the current order (the same in every thread)
        const int32_t v0 = (int32_t)((int64_t)n * t / T), v1 = (int32_t)((int64_t)n * (t + 1) / T);
        for (int i = 0; i < k; ++i) {
            const int32_t *d = dist.data() + (size_t)i * n;
            int32_t m = 0;
            for (int32_t v = v0; v < v1; ++v) m = std::max(m, d[v]);
            dm[(size_t)t * k + i] = m;
        }
        bar.wait();
        uint64_t *hi = key[0][0].data(), *lo = key[0][1].data();
        int used = 0;
        for (int i = 0; i < k; ++i) {
            int32_t dmax = 0;
            for (int q = 0; q < T; ++q) dmax = std::max(dmax, dm[(size_t)q * k + i]);
            const uint64_t unreached = (uint64_t)dmax + 1;
            int b = 1;
            while ((uint64_t{1} << b) <= unreached) ++b;
            if (used + b > 128) break;
            used += b;
            const int32_t *d = dist.data() + (size_t)i * n;
            for (int32_t v = v0; v < v1; ++v) {
                const uint64_t x = d[v] < 0 ? unreached : (uint64_t)d[v];
                hi[v] = (hi[v] << b) | (lo[v] >> (64 - b));
                lo[v] = (lo[v] << b) | x;
            }
        }
        for (int32_t v = v0; v < v1; ++v) ord[0][v] = v;
        bar.wait();
        for (int digit = 0; digit < 16; ++digit) {
            const int sh = 8 * (digit & 7);
            const int part = digit < 8 ? 1 : 0;
            const uint64_t *kk = key[cur][part].data();
            size_t *c = cnt.data() + (size_t)t * 256;
            std::fill(c, c + 256, 0);
            for (int32_t x = v0; x < v1; ++x) ++c[(kk[x] >> sh) & 0xFF];
            bar.wait();
            if (t == 0) {  // offsets: digit value major, thread minor
                size_t run = 0, top = 0;
                for (int dv = 0; dv < 256; ++dv) {
                    size_t tot = 0;
                    for (int q = 0; q < T; ++q) {
                        const size_t x = cnt[(size_t)q * 256 + dv];
                        cnt[(size_t)q * 256 + dv] = run;
                        run += x;
                        tot += x;
                    }
                    top = std::max(top, tot);
                }
                skip = top == (size_t)n;  // every key has this digit: the pass changes nothing
            }
            bar.wait();
            if (!skip) {
                const int nx = cur ^ 1;
                for (int32_t x = v0; x < v1; ++x) {
                    const size_t at = c[(kk[x] >> sh) & 0xFF]++;
                    ord[nx][at] = ord[cur][x];
                    key[nx][0][at] = key[cur][0][x];
                    key[nx][1][at] = key[cur][1][x];
                }
            }
            const bool flipped = !skip;
            bar.wait();  // skip is rewritten by the next pass only after every thread read it
            if (flipped) cur ^= 1;
        }
        if (t == 0) final_cur = cur;
    };
    std::vector<std::thread> th;
    if (T == 1) {
        work(0);
    } else {
        for (int t = 1; t < T; ++t) th.emplace_back(work, t);
        work(0);
        for (auto &x : th) x.join();
    }
    g->rank.assign(n, 0);
    for (int32_t t = 0; t < n; ++t) g->rank[ord[final_cur][t]] = t;
}

// Validate and upload the source list. With `order`, the sources are staged
// in landmark order (stable, so duplicates keep their relative order) and
// src_index maps each staged position back to the caller's index.
int stage_sources(bc_graph *g, const int32_t *sources, int32_t num, int32_t *count, bool order = false) {
    std::vector<int32_t> hs;
    if (!sources) {
        hs.resize(g->n);
        for (int32_t i = 0; i < g->n; ++i) hs[i] = i;
    } else {
        if (num < 0) return fail(BC_ERR_ARG, "num_sources < 0");
        CK(fetch(hs, sources, (size_t)num));
        for (int32_t s : hs)
            if (s < 0 || s >= g->n) return fail(BC_ERR_ARG, "source id out of range");
    }
    g->reordered = false;
    if (order && hs.size() > 32 && (int32_t)g->rank.size() == g->n) {
        const int32_t n = g->n;
        std::vector<int32_t> cnt((size_t)n + 1, 0), idx(hs.size()), hs2(hs.size());
        for (int32_t s : hs) ++cnt[g->rank[s] + 1];
        for (int32_t x = 1; x <= n; ++x) cnt[x] += cnt[x - 1];
        for (size_t i = 0; i < hs.size(); ++i) idx[cnt[g->rank[hs[i]]]++] = (int32_t)i;
        for (size_t t = 0; t < hs.size(); ++t) hs2[t] = hs[idx[t]];
        CK(g->src_index.ensure(idx.size()));
        CK(cudaMemcpy(g->src_index.p, idx.data(), idx.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
        hs.swap(hs2);
        g->reordered = true;
    }
    CK(g->sources.ensure(hs.size()));
    if (!hs.empty()) CK(cudaMemcpy(g->sources.p, hs.data(), hs.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    *count = (int32_t)hs.size();
    g->h_sources.swap(hs);
    return BC_OK;
}

int ensure_dense(bc_graph *g, cudaStream_t st) {
    if (g->dA.p) return BC_OK;
    if (g->weighted) return fail(BC_ERR_UNSUPPORTED, "BC_DENSE needs an unweighted graph");
    if (g->directed) return fail(BC_ERR_UNSUPPORTED, "BC_DENSE needs an undirected graph");
    if (g->n > bcgb::kDenseMaxN) return fail(BC_ERR_UNSUPPORTED, "BC_DENSE supports n <= 65536");
    const int32_t npad = std::max(128, (g->n + 127) / 128 * 128);  // whole 128-vertex tiles
    CK(g->dA.ensure((size_t)npad * npad));
    if (bcgb::dense_build_adjacency(g->row_ptr.p, g->col.p, g->n, npad, g->dA.p, st))
        return fail(BC_ERR_CUDA, "dense adjacency build failed");
    CK(g->dA8.ensure((size_t)npad * npad));
    if (bcgb::dense_build_adjacency8(g->row_ptr.p, g->col.p, g->n, npad, g->dA8.p, st))
        return fail(BC_ERR_CUDA, "dense adjacency build failed");
    g->npad = npad;
    return BC_OK;
}

// State of a group of nb batches (B = 128) with level capacity Lcap; the X
// map covers the group's limb rows.
int ensure_dense_group(bc_graph *g, int nb, int Lcap, cudaStream_t st) {
    if (g->gNB >= nb && g->gLcap == Lcap && g->gsigma.p) return BC_OK;
    const size_t n = (size_t)std::max(g->n, 1), nw32 = (n + 31) / 32;
    CK(g->gsigma.ensure((size_t)nb * n * 128));
    CK(g->gF.ensure((size_t)nb * Lcap * n * 4));
    CK(g->gV.ensure((size_t)nb * 2 * n * 4));
    CK(g->gufr.ensure((size_t)nb * Lcap * nw32));
    CK(g->gbcpart.ensure((size_t)nb * n));
    CK(g->gmeta.ensure((size_t)3 * nb));
    CK(g->dctl.ensure((size_t)nb));
    CK(g->dX.ensure((size_t)nb * bcgb::kDenseXRows * g->npad));
    CK(cudaMemsetAsync(g->dX.p, 0, g->dX.n * sizeof(__nv_bfloat16), st));
    if (bcgb::dense_make_maps(&g->maps, g->dX.p, (uint64_t)nb * bcgb::kDenseXRows, g->dA.p, g->dA8.p, g->npad))
        return fail(BC_ERR_CUDA, "cuTensorMapEncodeTiled failed for the dense operands");
    g->gNB = nb;
    g->gLcap = Lcap;
    return BC_OK;
}

// BC_DENSE on an unweighted graph: batches of 128 sources in groups run level
// by level in lockstep, one tensor-core launch per level for the whole group
// (every batch's state stays resident). Forward: level 0 -> 1 by the sparse
// first-level kernel per batch, then limb products until every batch's
// frontier is empty; each level's outcome fixes the next limb count.
// Backward: from the deepest level of the group down, the split c rows times
// A per level (or, with BC_SPARSE_BACKWARD, the sparse backward per batch);
// BC partials of the group are added in batch order.
// Side streams start after the work queued on st (fork) and st waits for
// everything queued on them (join).
int fork_side(bc_graph *g, cudaStream_t st) {
    if (!g->side_fork) CK(cudaEventCreateWithFlags(&g->side_fork, cudaEventDisableTiming));
    CK(cudaEventRecord(g->side_fork, st));
    for (int i = 0; i < kSideStreams; ++i) {
        if (!g->side[i]) {
            CK(cudaStreamCreateWithFlags(&g->side[i], cudaStreamNonBlocking));
            CK(cudaEventCreateWithFlags(&g->side_ev[i], cudaEventDisableTiming));
        }
        CK(cudaStreamWaitEvent(g->side[i], g->side_fork, 0));
    }
    return BC_OK;
}
int join_side(bc_graph *g, cudaStream_t st) {
    for (int i = 0; i < kSideStreams; ++i) {
        CK(cudaEventRecord(g->side_ev[i], g->side[i]));
        CK(cudaStreamWaitEvent(st, g->side_ev[i], 0));
    }
    return BC_OK;
}

constexpr size_t kDenseGroupBudget = 24ull << 30;
constexpr int kDenseL2Group = 8;  // batches that share each adjacency tile in turn

int run_dense_group(bc_graph *g, int32_t nsrc, const bc_options *opt, cudaStream_t st, bool backward, bool hash,
                    uint64_t *rows_sig, int32_t *rows_dist) {
    constexpr int W = 4, B = 128;
    const int32_t n = g->n;
    const size_t nn = (size_t)std::max(n, 1), nw32 = (nn + 31) / 32;
    const bool sparse_bwd = opt && (opt->flags & BC_SPARSE_BACKWARD);
    int r = build_plans(g, opt);
    if (r) return r;
    r = ensure_state(g, W, std::max(g->Lcap, 32));
    if (r) return r;
    const int nbat = (nsrc + B - 1) / B;
    for (int gb0 = 0; gb0 < nbat;) {
        const int Lcap = g->Lcap;
        const size_t per = nn * B * 10 + (size_t)Lcap * nn * 16 + 2 * nn * 16 + (size_t)Lcap * nw32 * 4 +
                           (size_t)bcgb::kDenseXRows * g->npad * 2 + nn * 8;
        const int NB = (int)std::max<size_t>(1, std::min<size_t>((size_t)(nbat - gb0), kDenseGroupBudget / per));
        r = ensure_dense_group(g, NB, Lcap, st);
        if (r) return r;
        const size_t sstr = nn * B, fstr = (size_t)Lcap * nn * W, vstr = 2 * nn * W, ustr = (size_t)Lcap * nw32;
        std::vector<int32_t> nbs(NB), depth(NB, 0);
        std::vector<bcgb::MsParams> ps(NB);
        for (int b = 0; b < NB; ++b) {
            const int32_t b0 = (gb0 + b) * B;
            nbs[b] = std::min<int32_t>(B, nsrc - b0);
            bcgb::MsParams p = make_params(g);
            p.nb = nbs[b];
            p.first = 1;
            // no frontier sizes from the tensor-core forward: the sparse
            // backward keeps the union filter on every level (it also hides
            // the frontier row below the deepest, which a group whose pairs
            // were all reached a level early never writes)
            p.lsize = nullptr;
            p.seq = ++g->seq;
            p.sources = g->sources.p + b0;
            p.sigma = g->gsigma.p + b * sstr;
            p.s_levels = 2;  // the dense levels write sigma only: the backward reads it there
            p.F = g->gF.p + b * fstr;
            p.V = g->gV.p + b * vstr;
            p.ufr = g->gufr.p + b * ustr;
            p.Lcap = Lcap;
            if (hash) {
                p.h_sigma = g->h_sigma.p + b0;
                p.h_dist = g->h_dist.p + b0;
                p.dist_sum = g->dist_sum.p + b0;
                p.reach = g->reach.p + b0;
            }
            ps[b] = p;
        }
        int32_t *d_blist = g->gmeta.p, *d_nbs = g->gmeta.p + NB, *d_depth = g->gmeta.p + 2 * NB;
        CK(cudaMemcpyAsync(d_nbs, nbs.data(), NB * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        bcgb::DenseParams d{};
        d.n = n;
        d.npad = g->npad;
        d.nw32 = (int32_t)nw32;
        d.Lcap = Lcap;
        d.group = kDenseL2Group;
        d.blist = d_blist;
        d.nbs = d_nbs;
        d.depth = d_depth;
        d.sig_stride = sstr;
        d.f_stride = fstr;
        d.v_stride = vstr;
        d.u_stride = ustr;
        d.xrows = bcgb::kDenseXRows;
        d.sigma = g->gsigma.p;
        d.F = g->gF.p;
        d.V = g->gV.p;
        d.ufr = g->gufr.p;
        d.X = g->dX.p;
        d.bcpart = g->gbcpart.p;
        d.ctl = g->ctl;
        d.dctl = g->dctl.p;
        // with the tensor-core backward the summaries come from its levels
        // (and the deepest level's split) instead of a pass over the batch state
        const bool dense_hash = hash && backward && !sparse_bwd;
        d.sources = g->sources.p + (size_t)gb0 * B;
        d.src_base = gb0 * B;
        d.h_sigma = dense_hash ? g->h_sigma.p : nullptr;
        d.h_dist = dense_hash ? g->h_dist.p : nullptr;
        d.dist_sum = dense_hash ? g->dist_sum.p : nullptr;
        d.reach = dense_hash ? g->reach.p : nullptr;
        {
            // levels 0 and 1 of the whole group in one launch
            Timer t(g, st, BC_KERNEL_FORWARD);
            if (bcgb::dense_launch_first(d, NB, g->sources.p + (size_t)gb0 * B, g->row_ptr.p, g->col.p, st))
                return fail(BC_ERR_CUDA, std::string("dense first level: ") + cudaGetErrorString(cudaGetLastError()));
        }
        // ---- forward, all batches in lockstep
        std::vector<int32_t> active(NB);
        std::iota(active.begin(), active.end(), 0);
        std::vector<bcgb::DenseCtl> res(NB);
        int nl = 1, nq = 1;  // level-1 counts are all 1 (one 8-bit or one 4-bit limb)
        bool capped = false;
        for (int l = 1; !active.empty(); ++l) {
            if (l + 2 >= Lcap) {
                capped = true;
                break;
            }
            CK(cudaMemcpyAsync(d_blist, active.data(), active.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
            CK(cudaMemsetAsync(g->dctl.p, 0, NB * sizeof(bcgb::DenseCtl), st));
            d.nactive = (int32_t)active.size();
            if (bcgb::dense_level_f8(g->maps, nq))
                g->dense_flops_f8 += 2.0 * B * nq * (double)g->npad * (double)g->npad * (double)active.size();
            else
                g->dense_flops += 2.0 * B * nl * (double)g->npad * (double)g->npad * (double)active.size();
            {
                Timer t(g, st, BC_KERNEL_DENSE);
                if (bcgb::dense_launch_level(g->maps, d, l, nl, nq, st))
                    return fail(BC_ERR_CUDA, std::string("dense level launch: ") + cudaGetErrorString(cudaGetLastError()));
            }
            uint32_t status = 0;
            CK(cudaMemcpyAsync(res.data(), g->dctl.p, NB * sizeof(bcgb::DenseCtl), cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(&status, &g->ctl->status, 4, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            if (status & BC_STATUS_DENSE_TIMEOUT) return fail(BC_ERR_TIMEOUT, "tensor-core pipeline wait timed out");
            std::vector<int32_t> still;
            unsigned long long maxsig = 0;
            for (int b : active) {
                if (!res[b].produced) {
                    depth[b] = l;
                } else if (res[b].remaining == 0) {  // every pair reached: the next frontier is empty
                    depth[b] = l + 1;
                } else {
                    still.push_back(b);
                    maxsig = std::max(maxsig, res[b].maxsig);
                }
            }
            active.swap(still);
            nl = 1;
            while (nl < bcgb::kDenseMaxLimbs && (maxsig >> (8 * nl)) != 0ull) ++nl;
            nq = 1;
            while (nq < 2 * bcgb::kDenseMaxLimbs && (maxsig >> (4 * nq)) != 0ull) ++nq;
            if (status & BC_STATUS_SIGMA_OVERFLOW) {
                nl = bcgb::kDenseMaxLimbs;
                nq = 2 * bcgb::kDenseMaxLimbs;
            }
        }
        if (capped) {  // deeper than the level capacity: grow it and redo this group
            CK(cudaStreamSynchronize(st));
            r = ensure_state(g, W, g->Lcap * 2);
            if (r) return r;
            continue;
        }
        CK(cudaMemcpyAsync(d_depth, depth.data(), NB * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        // ---- backward
        if (backward && sparse_bwd) {
            for (int b = 0; b < NB; ++b) {
                bcgb::MsParams pb = ps[b];
                use_plan(pb, g->bplan);
                for (int l = depth[b]; l >= 1; --l) {
                    Timer t(g, st, BC_KERNEL_BACKWARD);
                    bcgb::ms_launch_backward(W, pb, l, st);
                }
            }
        } else if (backward) {
            CK(cudaMemsetAsync(g->gbcpart.p, 0, (size_t)NB * nn * sizeof(double), st));
            Timer t(g, st, BC_KERNEL_DENSE);
            if (bcgb::dense_launch_bwd_last(d, NB, st)) return fail(BC_ERR_CUDA, "dense backward launch");
            const int Lmax = *std::max_element(depth.begin(), depth.end());
            for (int l = Lmax - 1; l >= 1; --l) {
                active.clear();
                for (int b = 0; b < NB; ++b)
                    if (depth[b] - 1 >= l) active.push_back(b);
                CK(cudaMemcpyAsync(d_blist, active.data(), active.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                                   st));
                d.nactive = (int32_t)active.size();
                g->dense_flops += 2.0 * B * 3.0 * (double)g->npad * (double)g->npad * (double)active.size();
                if (bcgb::dense_launch_bwd_level(g->maps, d, l, st))
                    return fail(BC_ERR_CUDA, std::string("dense backward launch: ") +
                                                 cudaGetErrorString(cudaGetLastError()));
            }
            if (bcgb::dense_reduce_bc(g->gbcpart.p, NB, n, g->bc.p, st)) return fail(BC_ERR_CUDA, "BC reduction");
        }
        if (hash && !dense_hash) {
            // the batches' summaries are independent: spread over side streams
            Timer t(g, st, BC_KERNEL_HASH);
            r = fork_side(g, st);
            if (r) return r;
            for (int b = 0; b < NB; ++b) bcgb::ms_launch_hash(W, ps[b], depth[b], g->side[b % kSideStreams]);
            r = join_side(g, st);
            if (r) return r;
        }
        for (int b = 0; b < NB; ++b) {
            const int32_t b0 = (gb0 + b) * B;
            if (rows_sig || rows_dist) {
                Timer t(g, st, BC_KERNEL_HASH);
                bcgb::ms_launch_rows(W, ps[b], depth[b], rows_sig ? rows_sig + (size_t)b0 * n : nullptr,
                                     rows_dist ? rows_dist + (size_t)b0 * n : nullptr, st);
            }
        }
        CK(cudaGetLastError());
        gb0 += NB;
    }
    return BC_OK;
}

// A shrinking frontier of at most this many vertices is taken as the tail of the
// BFS: the host then launches one level at a time instead of kLookahead ahead
// (a launch past the last level still costs a grid's start-up).
int32_t small_frontier_items(const bc_graph *g) { return std::max<int32_t>(32, (int32_t)(g->beta * (float)g->n)); }

// Beamer's direction rule for level 0 -> 1, the one level whose frontier (the
// batch's sources) is known on the host: top-down (k_first, a push over the
// sources' arcs) while those arcs are fewer than the 2m arcs a bottom-up pull
// reads divided by alpha, else bottom-up. BC_FORCE_BOTTOMUP always pulls.
// *arcs receives the count (0 when not counted).
int first_level_top_down(const bc_graph *g, const int32_t *src_host, int32_t nb, int64_t *arcs_out) {
    *arcs_out = 0;
    if (!src_host) return g->bottom_up0 ? 0 : 1;
    int64_t arcs = 0;
    for (int32_t b = 0; b < nb; ++b) arcs += g->h_row_ptr[src_host[b] + 1] - g->h_row_ptr[src_host[b]];
    *arcs_out = arcs;
    if (g->bottom_up0) return 0;
    if (g->directed) return 1;  // (directed graphs: the pull runs over in-arcs)
    return (double)arcs * (double)g->alpha < (double)g->narcs ? 1 : 0;
}

// The multi-source driver shared by bc_run and bc_forward_rows.
// Concurrent sweep over K lanes (K >= 2). Batch i runs on lane i % K, each
// lane on its own stream with its own batch state and BC accumulator, so the
// narrow, latency-bound levels of one batch overlap the wide levels of
// another. The host drives every lane's level loop without blocking on any
// of them (the same look-ahead as drive_forward). The lanes start after the
// work already queued on st; at the end st waits for them and adds lanes
// 1..K-1 into the graph's BC in lane order, so the result is the same on
// every run. A batch deeper than the level capacity stops every lane: the
// capacity is doubled and each lane's unfinished batch starts over.
int run_lanes(bc_graph *g, int32_t nsrc, int W, int K, cudaStream_t st, bool backward, bool hash,
              uint64_t *rows_sig, int32_t *rows_dist, int64_t wait_ms) {
    const int B = 32 * W;
    const int32_t nbat = (nsrc + B - 1) / B;
    int Lcap = g->Lcap;
    for (int k = 1; k < K; ++k) {
        const int r = ensure_lane(g, g->lanes[k - 1], W, Lcap);
        if (r) return r;
    }
    if (!g->ev0) CK(cudaEventCreateWithFlags(&g->ev0, cudaEventDisableTiming));
    CK(cudaEventRecord(g->ev0, st));
    for (int k = 1; k < K; ++k) {
        SweepLane &ln = g->lanes[k - 1];
        CK(cudaStreamWaitEvent(ln.st, g->ev0, 0));
        CK(cudaMemsetAsync(ln.bc.p, 0, (size_t)g->n * sizeof(double), ln.st));
        CK(cudaMemsetAsync(ln.ctl, 0, sizeof(bcgb::DevCtl), ln.st));
    }
    auto lane_stream = [&](int k) { return k == 0 ? st : g->lanes[k - 1].st; };
    auto lane_hctl = [&](int k) -> const bcgb::HostCtl * { return k == 0 ? g->hctl : g->lanes[k - 1].hctl; };
    struct Job {
        int32_t bi = -1;
        int phase = 0;  // 0: no batch in flight, 1: forward levels in flight
        int launched = 0;
        bcgb::MsParams p{};
        std::chrono::steady_clock::time_point t0;
    };
    Job jobs[kSweepLanes];
    int32_t next[kSweepLanes];
    const int32_t small_frontier = small_frontier_items(g);
    for (int k = 0; k < K; ++k) next[k] = k;
    using clock = std::chrono::steady_clock;
    for (long spins = 0;; ++spins) {
        bool moved = false, busy = false;
        for (int k = 0; k < K; ++k) {
            Job &j = jobs[k];
            const cudaStream_t ls = lane_stream(k);
            if (j.phase == 0 && next[k] < nbat) {
                j.bi = next[k];
                next[k] += K;
                const int32_t b0 = j.bi * B;
                j.p = lane_params(g, k);
                j.p.nb = std::min<int32_t>(B, nsrc - b0);
                j.p.first = first_level_top_down(g, g->h_sources.data() + b0, j.p.nb, &j.p.first_arcs);
                j.p.seq = ++g->seq;
                j.p.sources = g->sources.p + b0;
                if (hash) {
                    const int32_t o = g->reordered ? 0 : b0;
                    j.p.h_sigma = g->h_sigma.p + o;
                    j.p.h_dist = g->h_dist.p + o;
                    j.p.dist_sum = g->dist_sum.p + o;
                    j.p.reach = g->reach.p + o;
                    j.p.out_index = g->reordered ? g->src_index.p + b0 : nullptr;
                }
                {
                    Timer t(g, ls, BC_KERNEL_INIT);
                    bcgb::ms_launch_init(W, j.p, ls);
                }
                j.phase = 1;
                j.launched = 0;
                j.t0 = clock::now();
                moved = true;
            }
            if (j.phase != 1) continue;
            busy = true;
            const bcgb::HostCtl *h = lane_hctl(k);
            int done_lv = 0, ahead = bcgb::kLookahead;
            if (bcgb::word_for(&h->progress, j.p.seq, &done_lv)) ahead = bcgb::lookahead(h, small_frontier);
            while (j.launched <= j.p.Lcap - 2 && j.launched < done_lv + ahead) {
                Timer t(g, ls, BC_KERNEL_FORWARD, j.launched);
                if (j.launched == 0 && j.p.first)
                    bcgb::ms_launch_first(W, j.p, ls);
                else
                    bcgb::ms_launch_forward(W, j.p, j.launched, ls);
                ++j.launched;
                moved = true;
            }
            int L = 0;
            if (!bcgb::word_for(&h->done, j.p.seq, &L)) continue;
            moved = true;
            if (L < 0) {
                // deeper than the level capacity: grow it on every lane and
                // start each lane's unfinished batch again
                for (int q = 0; q < K; ++q) CK(cudaStreamSynchronize(lane_stream(q)));
                Lcap *= 2;
                int r = ensure_state(g, W, Lcap);
                for (int q = 1; q < K && !r; ++q) r = ensure_lane(g, g->lanes[q - 1], W, Lcap);
                if (r) return r;
                for (int q = 0; q < K; ++q)
                    if (jobs[q].phase == 1) {
                        jobs[q].phase = 0;
                        next[q] = jobs[q].bi;
                    }
                break;
            }
            if (backward) {
                bcgb::MsParams pb = j.p;
                use_plan(pb, g->bplan);
                for (int l = L; l >= 1; --l) {
                    Timer t(g, ls, BC_KERNEL_BACKWARD, l);
                    bcgb::ms_launch_backward(W, pb, l, ls);
                }
            }
            if (hash) {
                Timer t(g, ls, BC_KERNEL_HASH);
                bcgb::ms_launch_hash(W, j.p, L, ls);
            }
            if (rows_sig || rows_dist) {
                Timer t(g, ls, BC_KERNEL_HASH);
                const size_t off = (size_t)j.bi * B * g->n;
                bcgb::ms_launch_rows(W, j.p, L, rows_sig ? rows_sig + off : nullptr, rows_dist ? rows_dist + off : nullptr,
                                     ls);
            }
            CK(cudaGetLastError());
            j.phase = 0;
        }
        if (!busy && !moved) {
            bool left = false;
            for (int k = 0; k < K; ++k) left |= next[k] < nbat;
            if (!left) break;
        }
        if (moved) continue;
        if (spins % 64 == 63) {
            CK(cudaGetLastError());
            for (int k = 0; k < K; ++k) {
                if (jobs[k].phase != 1) continue;
                const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(clock::now() - jobs[k].t0).count();
                if (ms > wait_ms)
                    return fail(BC_ERR_TIMEOUT, "the device did not report the end of a forward pass within the wait limit");
                const cudaError_t e = cudaStreamQuery(lane_stream(k));
                if (e != cudaSuccess && e != cudaErrorNotReady)
                    return fail(BC_ERR_CUDA, std::string("device error during a forward pass: ") + cudaGetErrorString(e));
                int dummy = 0;
                if (e == cudaSuccess && !bcgb::word_for(&lane_hctl(k)->done, jobs[k].p.seq, &dummy) &&
                    jobs[k].launched > jobs[k].p.Lcap - 2)
                    return fail(BC_ERR_STATE, "forward pass ended without reporting its depth");
            }
            if (spins % 4096 == 4095) std::this_thread::yield();
        }
    }
    // join: st waits for every lane, then adds their BC and counters in lane order
    for (int k = 1; k < K; ++k) {
        SweepLane &ln = g->lanes[k - 1];
        CK(cudaEventRecord(ln.ev, ln.st));
        CK(cudaStreamWaitEvent(st, ln.ev, 0));
    }
    for (int k = 1; k < K; ++k) {
        SweepLane &ln = g->lanes[k - 1];
        bcgb::ms_launch_merge(ln.bc.p, g->bc.p, g->n, ln.ctl, g->ctl, st);
    }
    CK(cudaGetLastError());
    return BC_OK;
}

int run_batches(bc_graph *g, int32_t nsrc, int W, const bc_options *opt, cudaStream_t st, bool backward,
                bool hash, uint64_t *rows_sig, int32_t *rows_dist) {
    const int64_t wait_ms = (opt && opt->wait_limit_ms > 0) ? opt->wait_limit_ms : 600000;
    if (opt && (opt->flags & BC_DENSE)) {
        int rd = ensure_dense(g, st);
        if (rd) return rd;
        return run_dense_group(g, nsrc, opt, st, backward, hash, rows_sig, rows_dist);
    }
    int r = build_plans(g, opt);
    if (r) return r;
    r = ensure_state(g, W, std::max(g->Lcap, 32));
    if (r) return r;
    const int B = 32 * W;
    {
        // lanes: as many as there are batches, up to kSweepLanes, within a
        // memory budget for the extra lanes' batch state. With BC_TIMING one
        // lane, so that every launch's event time is its own.
        const int32_t nbat = (nsrc + B - 1) / B;
        const double lane_bytes = (double)std::max(g->n, 1) * ((double)B * 24.0 + (double)g->Lcap * W * 4.0 + 16.0) +
                                  (double)g->s_levels * std::max(g->n, 1) * B * 2.0;
        int K = g->timing ? 1 : std::min<int32_t>(kSweepLanes, nbat);
        while (K > 1 && (K - 1) * lane_bytes > kLaneBudgetBytes) --K;
        if (K > 1) return run_lanes(g, nsrc, W, K, st, backward, hash, rows_sig, rows_dist, wait_ms);
    }
    for (int32_t b0 = 0; b0 < nsrc;) {
        const int32_t nb = std::min<int32_t>(B, nsrc - b0);
        bcgb::MsParams p = make_params(g);
        p.nb = nb;
        p.first = first_level_top_down(g, g->h_sources.data() + b0, nb, &p.first_arcs);
        p.seq = ++g->seq;
        p.sources = g->sources.p + b0;
        if (hash) {
            const int32_t o = g->reordered ? 0 : b0;  // reordered: summaries go through src_index
            p.h_sigma = g->h_sigma.p + o;
            p.h_dist = g->h_dist.p + o;
            p.dist_sum = g->dist_sum.p + o;
            p.reach = g->reach.p + o;
            p.out_index = g->reordered ? g->src_index.p + b0 : nullptr;
        }
        {
            Timer t(g, st, BC_KERNEL_INIT);
            bcgb::ms_launch_init(W, p, st);
        }
        int L = 0;
        {
            auto launch = [&](int level) {
                Timer t(g, st, BC_KERNEL_FORWARD, level);
                if (level == 0 && p.first)
                    bcgb::ms_launch_first(W, p, st);
                else
                    bcgb::ms_launch_forward(W, p, level, st);
            };
            r = bcgb::drive_forward(g->hctl, p.seq, g->Lcap - 2, launch, wait_ms, st, &g_err, &L,
                                    small_frontier_items(g));
        }
        if (r) return r;
        if (L < 0) {  // deeper than the level capacity: grow it and redo this batch
            CK(cudaStreamSynchronize(st));
            r = ensure_state(g, W, g->Lcap * 2);
            if (r) return r;
            continue;
        }
        if (backward) {
            bcgb::MsParams pb = p;
            use_plan(pb, g->bplan);
            for (int l = L; l >= 1; --l) {
                Timer t(g, st, BC_KERNEL_BACKWARD, l);
                bcgb::ms_launch_backward(W, pb, l, st);
            }
        }
        if (hash) {
            Timer t(g, st, BC_KERNEL_HASH);
            bcgb::ms_launch_hash(W, p, L, st);
        }
        if (rows_sig || rows_dist) {
            Timer t(g, st, BC_KERNEL_HASH);
            bcgb::ms_launch_rows(W, p, L, rows_sig ? rows_sig + (size_t)b0 * g->n : nullptr,
                                 rows_dist ? rows_dist + (size_t)b0 * g->n : nullptr, st);
        }
        CK(cudaGetLastError());
        b0 += nb;
    }
    return BC_OK;
}

// Distances from the landmarks (one W = 1 batch of the forward sweep, rows
// copied back), then the counting sorts; once per graph.
int ensure_rank(bc_graph *g, cudaStream_t st) {
    constexpr int kLandmarks = 32;  // one full 32-source batch of the forward sweep
    if ((int32_t)g->rank.size() == g->n || g->n <= 32) return BC_OK;
    const int32_t n = g->n;
    const auto &rp = g->h_row_ptr;
    const int k = std::min<int32_t>(kLandmarks, n);
    std::vector<int32_t> vs(n);
    std::iota(vs.begin(), vs.end(), 0);
    auto deg = [&](int32_t v) { return rp[v + 1] - rp[v]; };
    std::partial_sort(vs.begin(), vs.begin() + k, vs.end(),
                      [&](int32_t a, int32_t b) { return deg(a) > deg(b) || (deg(a) == deg(b) && a < b); });
    int32_t cnt = 0;
    int r = stage_sources(g, vs.data(), k, &cnt, false);
    if (r) return r;
    ScopedBuf<int32_t> dd;
    CK(dd.ensure((size_t)k * n));
    bc_options o{};
    o.batch = 32;
    r = run_batches(g, k, 1, &o, st, false, false, nullptr, dd.p);
    if (r) return r;
    std::vector<int32_t> dist((size_t)k * n);
    CK(cudaMemcpyAsync(dist.data(), dd.p, dist.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    rank_from_dist(g, dist, k);
    return BC_OK;
}

int sm_count_host() {
    static int c = 0;
    if (c == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
        if (c <= 0) c = 1;
    }
    return c;
}

// The relabelled copy of a weighted graph (relabel.cu's numbering of the
// out-arc CSR): vertex v becomes wperm[v]; each row keeps its arcs' weights,
// with the heads renumbered and sorted; a directed graph's in-arc CSR is
// renumbered the same way. Built once per handle; host code plus uploads.
int ensure_relabel(bc_graph *g) {
    if (g->relabel_ok) return BC_OK;
    const int32_t n = g->n;
    const int64_t m2 = g->narcs;
    std::vector<int32_t> cl, ww;
    CK(fetch(cl, (const int32_t *)g->col.p, (size_t)m2));
    CK(fetch(ww, (const int32_t *)g->w.p, (size_t)m2));
    std::vector<int32_t> perm((size_t)n), vid((size_t)n);
    bcgb::locality_order(n, g->h_row_ptr.data(), cl.data(), perm.data());
    for (int32_t v = 0; v < n; ++v) vid[(size_t)perm[v]] = v;
    // row x of the result holds row vid[x] of (rp, col, w), heads renumbered
    auto permute = [&](const std::vector<int32_t> &rp, const std::vector<int32_t> &col,
                       const std::vector<int32_t> &w, std::vector<int32_t> &prp, std::vector<int32_t> &pcl,
                       std::vector<int32_t> &pww) {
        prp.assign((size_t)n + 1, 0);
        pcl.resize(col.size());
        pww.resize(col.size());
        std::vector<std::pair<int32_t, int32_t>> row;
        for (int32_t x = 0; x < n; ++x) {
            const int32_t v = vid[(size_t)x];
            row.clear();
            for (int64_t e = rp[(size_t)v]; e < rp[(size_t)v + 1]; ++e)
                row.emplace_back(perm[(size_t)col[(size_t)e]], w[(size_t)e]);
            std::sort(row.begin(), row.end());
            const int32_t at = prp[(size_t)x];
            for (size_t i = 0; i < row.size(); ++i) {
                pcl[(size_t)at + i] = row[i].first;
                pww[(size_t)at + i] = row[i].second;
            }
            prp[(size_t)x + 1] = at + (int32_t)row.size();
        }
    };
    auto up = [&](DevBuf<int32_t> &d, const std::vector<int32_t> &h) -> int {
        CK(d.ensure(h.size()));
        if (!h.empty()) CK(cudaMemcpy(d.p, h.data(), h.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
        return BC_OK;
    };
    std::vector<int32_t> prp, pcl, pww;
    permute(g->h_row_ptr, cl, ww, prp, pcl, pww);
    int r = up(g->prow_ptr, prp);
    if (!r) r = up(g->pcol, pcl);
    if (!r) r = up(g->pw, pww);
    if (!r && g->directed) {
        CK(fetch(cl, (const int32_t *)g->col_in.p, (size_t)m2));
        CK(fetch(ww, (const int32_t *)g->w_in.p, (size_t)m2));
        permute(g->h_row_ptr_in, cl, ww, prp, pcl, pww);
        r = up(g->prow_ptr_in, prp);
        if (!r) r = up(g->pcol_in, pcl);
        if (!r) r = up(g->pw_in, pww);
    }
    if (!r) r = up(g->wperm, perm);
    if (!r) r = up(g->wvid, vid);
    if (r) return r;
    g->h_wperm.swap(perm);
    g->relabel_ok = true;
    return BC_OK;
}

// Weighted sweep (csrc/sssp_packed.cu; csrc/sssp_weighted.cu for 64-bit
// counts): waves of G sources, one CTA each. G is opt->batch if set, else
// kWSmallPerSm sources per SM for the 128-thread CTAs of small graphs, else
// three per SM, two of them resident (512-thread CTAs: on the relabelled
// 512x512 grid 1 / 2 / 3 / 4 per SM measured 258 / 257 / 241 / 252 ms, with
// 256-thread CTAs 274 / 255 / 253 / 256; on the caller's row-major numbering
// more sources in flight only added random DRAM sectors), capped so the wave
// state stays within 8 GiB. Waves run on
// kWeightedLanes lanes: wave k runs on lane k % lanes, each with its own stream,
// state, delta rows and BC accumulator, so one wave's slowest sources overlap
// the next waves. The delta rows of a wave are added to its lane's BC in
// source order right after the wave; lanes 1.. are added into the graph's BC
// in lane order at the end, so the result does not change from run to run.
// Sources whose path counts reach 2^32 write nothing in the packed kernel;
// they are flagged and computed again at the end by the 64-bit kernel, whose
// delta rows are added in the order of the flagged sources.
constexpr int kWeightedLanes = 2;  // measured: 3 or 4 lanes no faster on the 512x512 grid
constexpr int kWSmallPerSm = 8;    // wave of the 128-thread CTAs (small graphs), per SM: all resident

constexpr double kWeightedLaneBudget = 24.0 * (1 << 30);  // packed wave state of all lanes

int run_weighted(bc_graph *g, int32_t nsrc, const bc_options *opt, cudaStream_t st, bool backward, bool hash,
                 uint64_t *rows_sig, int32_t *rows_dist) {
    const int32_t n = g->n;
    const int K = g->maxw + 1;
    if (K > bcgb::kMaxRing)
        return fail(BC_ERR_UNSUPPORTED, "weighted path: maximum weight must be below " +
                                            std::to_string(bcgb::kMaxRing));
    int C = (int)std::min<int64_t>(std::max<int64_t>(1024, (4ll << 20) / K / 4), (int64_t)n + 1);
    C = std::max(C, 64);
    const size_t per_src = (size_t)n * (4 + 8 + 4 + 4 + 4 + 4 + 8) + 4 + (size_t)K * C * 4;
    const int per_sm = bcgb::w_packed_threads(n) == 128 ? kWSmallPerSm : 3;
    int G = (opt && opt->batch > 0) ? opt->batch : per_sm * sm_count_host();
    G = (int)std::min<size_t>((size_t)G, std::max<size_t>(1, (8ull << 30) / per_src));
    G = std::max(1, std::min(G, std::max(nsrc, 1)));
    const int32_t nwaves = (nsrc + G - 1) / G;
    // lanes: up to kWeightedLanes within the memory budget; BC_TIMING: one
    // lane, so that every launch's event time is its own
    const double lane_bytes = (double)G * ((double)n * 20.0 + (double)K * C * 4.0);
    int lanes = g->timing ? 1 : std::min<int32_t>(kWeightedLanes, nwaves);
    while (lanes > 1 && lanes * lane_bytes > kWeightedLaneBudget) --lanes;
    if (g->wG < G || g->wK != K || g->wC != C) {
        CK(g->wdist.ensure((size_t)G * n));
        CK(g->wsigma.ensure((size_t)G * n));
        CK(g->wcval.ensure((size_t)G * n));
        CK(g->worder.ensure((size_t)G * n));
        CK(g->wgrp.ensure((size_t)G * (n + 1)));
        CK(g->wslots.ensure((size_t)G * K * C));
        CK(g->wrows.ensure((size_t)G * n));
        CK(g->wds.ensure((size_t)G * n));
        CK(g->wpos.ensure((size_t)G));
        CK(g->wsrc.ensure((size_t)G));
        g->wG = G;
        g->wK = K;
        g->wC = C;
    }
    CK(g->wredo.ensure((size_t)std::max(nsrc, 1)));
    CK(cudaMemsetAsync(g->wredo.p, 0, (size_t)std::max(nsrc, 1), st));
    // the sweep runs on the relabelled copy (BC_KEEP_ORDER: on the caller's
    // numbering): sources mapped in, summaries, rows and BC mapped back to
    // the caller's ids by the kernels
    const bool relabel = n > 1 && !(opt && (opt->flags & BC_KEEP_ORDER));
    if (relabel) {
        int r = ensure_relabel(g);
        if (r) return r;
        CK(g->wpsrc.ensure((size_t)std::max(nsrc, 1)));
        Timer t(g, st, BC_KERNEL_INIT);
        bcgb::launch_map_ids(g->wperm.p, g->sources.p, g->wpsrc.p, nsrc, st);
    }
    const int32_t *vid = relabel ? g->wvid.p : nullptr;
    const int32_t *srcs = relabel ? g->wpsrc.p : g->sources.p;
    if (lanes > 1 && !g->wev) CK(cudaEventCreateWithFlags(&g->wev, cudaEventDisableTiming));
    if (lanes > 1) CK(cudaEventRecord(g->wev, st));
    for (int k = 1; k < lanes; ++k) {
        auto &l = g->wl[k - 1];
        if (!l.st) {
            CK(cudaStreamCreateWithFlags(&l.st, cudaStreamNonBlocking));
            CK(cudaEventCreateWithFlags(&l.ev, cudaEventDisableTiming));
        }
        CK(l.order.ensure((size_t)G * n));
        CK(l.grp.ensure((size_t)G * (n + 1)));
        CK(l.slots.ensure((size_t)G * K * C));
        CK(l.rows.ensure((size_t)G * n));
        CK(l.ds.ensure((size_t)G * n));
        CK(l.bc.ensure((size_t)std::max(n, 1)));
        CK(cudaStreamWaitEvent(l.st, g->wev, 0));
        CK(cudaMemsetAsync(l.bc.p, 0, (size_t)std::max(n, 1) * sizeof(double), l.st));
    }
    bcgb::WParams base{};
    base.n = n;
    base.K = K;
    base.C = C;
    base.dmax = (int32_t)std::min<int64_t>((int64_t)n * g->maxw, INT32_MAX - 1);
    base.row_ptr = relabel ? g->prow_ptr.p : g->row_ptr.p;
    base.col = relabel ? g->pcol.p : g->col.p;
    base.w = relabel ? g->pw.p : g->w.p;
    base.vid = vid;
    if (g->directed) {
        base.row_ptr_in = relabel ? g->prow_ptr_in.p : g->row_ptr_in.p;
        base.col_in = relabel ? g->pcol_in.p : g->col_in.p;
        base.w_in = relabel ? g->pw_in.p : g->w_in.p;
    }
    base.ctl = g->ctl;
    for (int32_t k = 0; k < nwaves; ++k) {
        const int32_t w0 = k * G;
        const int nw = std::min<int32_t>(G, nsrc - w0);
        const int ln = k % lanes;
        bc_graph::WLane *l = ln == 0 ? nullptr : &g->wl[ln - 1];
        const cudaStream_t ls = l ? l->st : st;
        bcgb::WParams p = base;
        p.sources = srcs + w0;
        p.order = l ? l->order.p : g->worder.p;
        p.grp = l ? l->grp.p : g->wgrp.p;
        p.slots = l ? l->slots.p : g->wslots.p;
        p.ds = l ? l->ds.p : g->wds.p;
        float *rows = l ? l->rows.p : g->wrows.p;
        p.delta_rows = backward ? rows : nullptr;
        if (hash) {
            p.h_sigma = g->h_sigma.p + w0;
            p.h_dist = g->h_dist.p + w0;
            p.dist_sum = g->dist_sum.p + w0;
            p.reach = g->reach.p + w0;
        }
        p.rows_sigma = rows_sig ? rows_sig + (size_t)w0 * n : nullptr;
        p.rows_dist = rows_dist ? rows_dist + (size_t)w0 * n : nullptr;
        p.redo = g->wredo.p + w0;
        {
            Timer t(g, ls, BC_KERNEL_FORWARD);
            bcgb::w_launch_wave_packed(p, nw, ls);
        }
        if (backward) {
            Timer t(g, ls, BC_KERNEL_BACKWARD);
            bcgb::w_launch_reduce(rows, nw, n, vid, l ? l->bc.p : g->bc.p, sm_count_host(), ls);
        }
        CK(cudaGetLastError());
    }
    for (int k = 1; k < lanes; ++k) {
        auto &l = g->wl[k - 1];
        CK(cudaEventRecord(l.ev, l.st));
        CK(cudaStreamWaitEvent(st, l.ev, 0));
    }
    for (int k = 1; k < lanes && backward; ++k) bcgb::ms_launch_merge(g->wl[k - 1].bc.p, g->bc.p, n, nullptr, nullptr, st);
    // sources whose path counts need 64 bits: again with the 64-bit kernel
    std::vector<uint8_t> redo((size_t)std::max(nsrc, 1));
    CK(cudaMemcpyAsync(redo.data(), g->wredo.p, redo.size(), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    std::vector<int32_t> rpos, rsrc;
    for (int32_t i = 0; i < nsrc; ++i)
        if (redo[i]) {
            rpos.push_back(i);
            rsrc.push_back(relabel ? g->h_wperm[(size_t)g->h_sources[(size_t)i]] : g->h_sources[(size_t)i]);
        }
    for (size_t r0 = 0; r0 < rpos.size(); r0 += (size_t)G) {
        const int nr = (int)std::min<size_t>((size_t)G, rpos.size() - r0);
        CK(cudaMemcpyAsync(g->wpos.p, rpos.data() + r0, (size_t)nr * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(g->wsrc.p, rsrc.data() + r0, (size_t)nr * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        bcgb::WParams p = base;
        p.sources = g->wsrc.p;
        p.pos = g->wpos.p;
        p.dist = g->wdist.p;
        p.sigma = g->wsigma.p;
        p.cval = g->wcval.p;
        p.order = g->worder.p;
        p.grp = g->wgrp.p;
        p.slots = g->wslots.p;
        p.delta_rows = backward ? g->wrows.p : nullptr;
        if (hash) {
            p.h_sigma = g->h_sigma.p;
            p.h_dist = g->h_dist.p;
            p.dist_sum = g->dist_sum.p;
            p.reach = g->reach.p;
        }
        p.rows_sigma = rows_sig;
        p.rows_dist = rows_dist;
        {
            Timer t(g, st, BC_KERNEL_FORWARD);
            bcgb::w_launch_wave(p, nr, st);
        }
        if (backward) {
            Timer t(g, st, BC_KERNEL_BACKWARD);
            bcgb::w_launch_reduce(g->wrows.p, nr, n, vid, g->bc.p, sm_count_host(), st);
        }
        CK(cudaGetLastError());
    }
    return BC_OK;
}

// Algorithm 2 (Section 4.2.1): forward rows of every source (distances and
// path counts, n x n), then BC from the pair formula (pairs.cu).
constexpr int32_t kPairsMaxN = 16384;

int run_pairs(bc_graph *g, int32_t nsrc, int W, const bc_options *opt, cudaStream_t st, bool hash) {
    const int32_t n = g->n;
    if (nsrc != n) return fail(BC_ERR_ARG, "BC_PAIRS needs every vertex as a source");
    if (n == 0) return BC_OK;
    const size_t cells = (size_t)n * n;
    ScopedBuf<int32_t> D;
    ScopedBuf<uint64_t> L;
    ScopedBuf<unsigned char> scratch;
    CK(D.ensure(cells));
    CK(L.ensure(cells));
    CK(scratch.ensure(bcgb::pair_scratch_bytes(n)));
    int r = g->weighted ? run_weighted(g, n, opt, st, false, hash, L.p, D.p)
                        : run_batches(g, n, W, opt, st, false, hash, L.p, D.p);
    if (r) return r;
    {
        Timer t(g, st, BC_KERNEL_BACKWARD);
        if (bcgb::pair_launch(D.p, L.p, n, scratch.p, g->bc.p, sm_count_host(), st))
            return fail(BC_ERR_CUDA, std::string("pair formula launch: ") + cudaGetErrorString(cudaGetLastError()));
    }
    CK(cudaStreamSynchronize(st));
    return BC_OK;
}

// Weighted algebraic forward (Section 3.2; BC_DENSE on a weighted graph):
// per batch of sources, distance products with path counts on the dense
// weight matrix until a step changes nothing (minplus.cu). Rows of the
// staged sources [b0, b0 + nsrc) go to rows_sig / rows_dist in that order.
constexpr int32_t kMpMaxN = 32768;
constexpr int kMpBatch = 512;

int run_minplus(bc_graph *g, int32_t nsrc, cudaStream_t st, bool hash, uint64_t *rows_sig, int32_t *rows_dist) {
    const int32_t n = g->n;
    if (n > kMpMaxN) return fail(BC_ERR_UNSUPPORTED, "BC_DENSE on a weighted graph supports n <= 32768");
    if ((int64_t)n * g->maxw >= (int64_t)bcgb::kMpInf)
        return fail(BC_ERR_UNSUPPORTED, "BC_DENSE on a weighted graph needs n * max weight < 2^30 - 1");
    if (!rows_sig || !rows_dist) return fail(BC_ERR_ARG, "weighted dense forward writes full rows");
    const int sms = sm_count_host();
    if (!g->mpW.p) {
        CK(g->mpW.ensure((size_t)n * n));
        if (bcgb::mp_build_weights(g->row_ptr.p, g->col.p, g->w.p, n, g->mpW.p, sms, st))
            return fail(BC_ERR_CUDA, "weight matrix build");
    }
    const int B = std::min<int32_t>(kMpBatch, std::max<int32_t>(nsrc, 1));
    ScopedBuf<int32_t> xd;
    ScopedBuf<uint64_t> xc;
    ScopedBuf<uint32_t> flag;
    CK(xd.ensure(2 * (size_t)B * n));
    CK(xc.ensure(2 * (size_t)B * n));
    CK(flag.ensure(1));
    for (int32_t b0 = 0; b0 < nsrc; b0 += B) {
        const int nb = std::min<int32_t>(B, nsrc - b0);
        const size_t half = (size_t)B * n;
        int cur = 0;
        if (bcgb::mp_init(xd.p, xc.p, g->sources.p + b0, nb, n, sms, st)) return fail(BC_ERR_CUDA, "min-plus init");
        for (int step = 0;; ++step) {
            if (step > n) return fail(BC_ERR_BOUNDS, "distance products did not settle within n steps");
            CK(cudaMemsetAsync(flag.p, 0, sizeof(uint32_t), st));
            {
                Timer t(g, st, BC_KERNEL_DENSE);
                if (bcgb::mp_step(xd.p + cur * half, xc.p + cur * half, xd.p + (1 - cur) * half, xc.p + (1 - cur) * half,
                                  g->mpW.p, g->sources.p + b0, nb, n, flag.p, &g->ctl->status, st))
                    return fail(BC_ERR_CUDA, "min-plus step launch");
            }
            uint32_t f = 0;
            CK(cudaMemcpyAsync(&f, flag.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            cur ^= 1;
            if (!(f & 1u)) break;
        }
        int32_t *dr = rows_dist + (size_t)b0 * n;
        uint64_t *sr = rows_sig + (size_t)b0 * n;
        if (bcgb::mp_rows(xd.p + cur * half, xc.p + cur * half, nb, n, dr, sr, sms, st))
            return fail(BC_ERR_CUDA, "min-plus rows");
        if (hash && bcgb::mp_row_hashes(dr, sr, nb, n, g->h_sigma.p + b0, g->h_dist.p + b0, g->dist_sum.p + b0,
                                        g->reach.p + b0, sms, st))
            return fail(BC_ERR_CUDA, "row summaries");
    }
    CK(cudaStreamSynchronize(st));
    return BC_OK;
}

// BC_DENSE on a weighted graph: every source's rows by distance products,
// then Algorithm 2's pair formula.
int run_dense_weighted(bc_graph *g, int32_t nsrc, cudaStream_t st, bool hash) {
    const int32_t n = g->n;
    if (nsrc != n) return fail(BC_ERR_ARG, "BC_DENSE on a weighted graph takes every vertex as a source");
    if (n > kPairsMaxN) return fail(BC_ERR_UNSUPPORTED, "BC_DENSE on a weighted graph computes BC for n <= 16384");
    if (n == 0) return BC_OK;
    const size_t cells = (size_t)n * n;
    ScopedBuf<int32_t> D;
    ScopedBuf<uint64_t> L;
    ScopedBuf<unsigned char> scratch;
    CK(D.ensure(cells));
    CK(L.ensure(cells));
    CK(scratch.ensure(bcgb::pair_scratch_bytes(n)));
    int r = run_minplus(g, n, st, hash, L.p, D.p);
    if (r) return r;
    {
        Timer t(g, st, BC_KERNEL_BACKWARD);
        if (bcgb::pair_launch(D.p, L.p, n, scratch.p, g->bc.p, sm_count_host(), st))
            return fail(BC_ERR_CUDA, std::string("pair formula launch: ") + cudaGetErrorString(cudaGetLastError()));
    }
    CK(cudaStreamSynchronize(st));
    return BC_OK;
}

}  // namespace

extern "C" {

int bc_create_graph(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *weights,
                    uint32_t flags, bc_graph **out) {
    g_err.clear();
    if (!out) return fail(BC_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n < 0) return fail(BC_ERR_ARG, "n < 0");
    if (!row_ptr) return fail(BC_ERR_ARG, "row_ptr is NULL");
    std::vector<int32_t> rp, cl, ww;
    CK(fetch(rp, row_ptr, (size_t)n + 1));
    const int64_t m2 = rp[n];
    if (m2 < 0) return fail(BC_ERR_ARG, "row_ptr[n] < 0");
    if (m2 > 0 && !col) return fail(BC_ERR_ARG, "col is NULL");
    CK(fetch(cl, col, (size_t)m2));
    if (weights) CK(fetch(ww, weights, (size_t)m2));
    const bool directed = (flags & BC_GRAPH_DIRECTED) != 0;
    if (!(flags & BC_GRAPH_TRUST_INPUT)) {
        int r = check_graph(n, rp, cl, weights ? &ww : nullptr, directed);
        if (r) return r;
    }
    // directed: the in-arc CSR (transpose), rows by head, tails in arc order
    std::vector<int32_t> rpi, cli, wwi;
    if (directed) {
        rpi.assign((size_t)n + 1, 0);
        for (int64_t e = 0; e < m2; ++e) ++rpi[(size_t)cl[e] + 1];
        for (int32_t v = 0; v < n; ++v) rpi[v + 1] += rpi[v];
        std::vector<int32_t> pos(rpi.begin(), rpi.end() - 1);
        cli.resize(m2);
        if (weights) wwi.resize(m2);
        for (int32_t u = 0; u < n; ++u)
            for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
                const int32_t at = pos[cl[e]]++;
                cli[at] = u;
                if (weights) wwi[at] = ww[e];
            }
    }
    bc_graph *g = new (std::nothrow) bc_graph();
    if (!g) return fail(BC_ERR_OOM, "host allocation failed");
    g->n = n;
    g->narcs = m2;
    g->weighted = weights != nullptr;
    g->h_row_ptr = rp;
    g->directed = directed;
    if (directed) g->h_row_ptr_in = rpi;
    for (int32_t x : ww) g->maxw = std::max(g->maxw, x);
    auto up = [&](DevBuf<int32_t> &d, const std::vector<int32_t> &h) -> int {
        CK(d.ensure(h.size()));
        if (!h.empty()) CK(cudaMemcpy(d.p, h.data(), h.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
        return BC_OK;
    };
    int r = up(g->row_ptr, rp);
    if (!r) r = up(g->col, cl);
    if (!r && weights) r = up(g->w, ww);
    if (!r && directed) r = up(g->row_ptr_in, rpi);
    if (!r && directed) r = up(g->col_in, cli);
    if (!r && directed && weights) r = up(g->w_in, wwi);
    if (!r) {
        cudaError_t e = g->bc.ensure((size_t)std::max(n, 1));
        if (e == cudaSuccess) e = cudaMalloc((void **)&g->ctl, sizeof(bcgb::DevCtl));
        if (e == cudaSuccess) e = cudaMemset(g->ctl, 0, sizeof(bcgb::DevCtl));
        if (e == cudaSuccess) e = cudaMemset(g->bc.p, 0, g->bc.n * sizeof(double));
        if (e == cudaSuccess)
            e = cudaHostAlloc((void **)&g->hctl, sizeof(bcgb::HostCtl), cudaHostAllocMapped | cudaHostAllocPortable);
        if (e == cudaSuccess) {
            std::memset(g->hctl, 0, sizeof(bcgb::HostCtl));
            e = cudaHostGetDevicePointer((void **)&g->hctl_d, g->hctl, 0);
        }
        if (e != cudaSuccess)
            r = fail(e == cudaErrorMemoryAllocation ? BC_ERR_OOM : BC_ERR_CUDA,
                     std::string("graph allocation: ") + cudaGetErrorString(e));
    }
    if (r) {
        free_graph(g);
        return r;
    }
    *out = g;
    return BC_OK;
}

int bc_run(bc_graph *g, const int32_t *sources, int32_t num_sources, const bc_options *opt, void *cuda_stream) {
    g_err.clear();
    if (!g) return fail(BC_ERR_ARG, "graph is NULL");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    g->run_t0 = std::chrono::steady_clock::now();
    if (!opt && g->has_defaults) opt = &g->defaults;  // the tuned (or installed) choice
    g->last_opt = opt ? *opt : bc_options{};
    const uint32_t flags = opt ? opt->flags : 0u;
    int W = 0;
    int r = g->weighted ? BC_OK : resolve_batch(opt, &W);
    if (r) return r;
    if (opt && opt->delta != 0 && opt->delta != 1)
        return fail(BC_ERR_UNSUPPORTED, "delta: only bucket width 1 (one distance value per bucket) is supported");
    set_run_options(g, opt);
    if (g->weighted && (flags & BC_PLAIN)) return fail(BC_ERR_UNSUPPORTED, "the one-source path is unweighted only");
    int32_t nsrc = 0;
    if (g->weighted && (flags & BC_DENSE) && sources)
        return fail(BC_ERR_ARG, "BC_DENSE on a weighted graph takes every vertex as a source (sources = NULL)");
    if ((flags & BC_PAIRS) && (sources || (flags & (BC_PLAIN | BC_DENSE))))
        return fail(BC_ERR_ARG, "BC_PAIRS takes every vertex as a source (sources = NULL), without BC_PLAIN / BC_DENSE");
    if ((flags & BC_PAIRS) && g->n > kPairsMaxN)
        return fail(BC_ERR_UNSUPPORTED, "BC_PAIRS supports n <= " + std::to_string(kPairsMaxN));
    const bool order = !g->weighted && !(flags & (BC_PLAIN | BC_KEEP_ORDER | BC_DENSE | BC_PAIRS)) &&
                       (sources ? num_sources : g->n) > 32;
    if (order) {
        // size the sweep state for this run's width first, so the landmark
        // pass (32 sources) runs in it instead of allocating its own
        r = build_plans(g, opt);
        if (!r) r = ensure_state(g, W, std::max(g->Lcap, 32));
        if (!r) r = ensure_rank(g, st);
        if (r) return r;
    }
    r = stage_sources(g, sources, num_sources, &nsrc, order);
    if (r) return r;
    g->timing = (flags & BC_TIMING) != 0;
    g->evused = 0;
    g->launches = 0;
    g->dense_flops = 0.0;
    g->dense_flops_f8 = 0.0;
    g->has_run = false;
    const bool hash = !(flags & BC_NO_HASH);
    if (!(flags & BC_ACCUMULATE)) CK(cudaMemsetAsync(g->bc.p, 0, g->bc.n * sizeof(double), st));
    CK(cudaMemsetAsync(&g->ctl->status, 0, sizeof(uint32_t), st));
    CK(cudaMemsetAsync(&g->ctl->dag_arcs, 0, 2 * sizeof(unsigned long long), st));
    if (hash) {
        CK(g->h_sigma.ensure(nsrc));
        CK(g->h_dist.ensure(nsrc));
        CK(g->dist_sum.ensure(nsrc));
        CK(g->reach.ensure(nsrc));
        if (nsrc) {
            CK(cudaMemsetAsync(g->h_sigma.p, 0, nsrc * sizeof(uint64_t), st));
            CK(cudaMemsetAsync(g->h_dist.p, 0, nsrc * sizeof(uint64_t), st));
            CK(cudaMemsetAsync(g->dist_sum.p, 0, nsrc * sizeof(int64_t), st));
            CK(cudaMemsetAsync(g->reach.p, 0, nsrc * sizeof(int64_t), st));
        }
    }
    if (flags & BC_PAIRS) {
        r = run_pairs(g, nsrc, W, opt, st, hash);
        if (r) return r;
    } else if (flags & BC_PLAIN) {
        std::pair<bc_graph *, cudaStream_t> ctx{g, st};
        bcgb::LaunchHook hook{&ctx, hook_begin, hook_end};
        const int64_t wait_ms = (opt && opt->wait_limit_ms > 0) ? opt->wait_limit_ms : 600000;
        r = bcgb::plain_run(g->plain, g->n, g->row_ptr.p, g->col.p, g->sources.p, nsrc, g->bc.p,
                            hash ? g->h_sigma.p : nullptr, hash ? g->h_dist.p : nullptr,
                            hash ? g->dist_sum.p : nullptr, hash ? g->reach.p : nullptr, g->ctl, g->hctl,
                            g->hctl_d, &g->seq, st, hook, wait_ms, &g_err);
        if (r) return r;
    } else if (g->weighted && (flags & BC_DENSE)) {
        r = run_dense_weighted(g, nsrc, st, hash);
        if (r) return r;
    } else if (g->weighted) {
        r = run_weighted(g, nsrc, opt, st, true, hash, nullptr, nullptr);
        if (r) return r;
    } else {
        r = run_batches(g, nsrc, W, opt, st, true, hash, nullptr, nullptr);
        if (r) return r;
    }
    if (flags & BC_HALVE) {
        Timer t(g, st, BC_KERNEL_HASH);
        bcgb::launch_scale(g->bc.p, g->n, 0.5, st);
    }
    CK(cudaGetLastError());
    g->last_nsrc = nsrc;
    g->has_run = true;
    g->has_hash = hash;
    g->last_stream = st;
    return BC_OK;
}

int bc_result(bc_graph *g, double *bc, uint32_t *status_flags) {
    g_err.clear();
    if (!g) return fail(BC_ERR_ARG, "graph is NULL");
    if (!g->has_run) return fail(BC_ERR_STATE, "no completed bc_run");
    uint32_t status = 0;
    if (bc && g->n) CK(cudaMemcpyAsync(bc, g->bc.p, (size_t)g->n * sizeof(double), cudaMemcpyDefault, g->last_stream));
    CK(cudaMemcpyAsync(&status, &g->ctl->status, sizeof(uint32_t), cudaMemcpyDefault, g->last_stream));
    CK(cudaStreamSynchronize(g->last_stream));
    if (status_flags) *status_flags = status;
    if (log_enabled()) {
        // one JSON line per completed run on stderr (environment variable BC_LOG=1)
        const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - g->run_t0).count();
        const bc_options &o = g->last_opt;
        std::fprintf(stderr,
                     "{\"bc_log\": \"run\", \"n\": %d, \"m\": %lld, \"weighted\": %d, \"directed\": %d, "
                     "\"sources\": %d, \"batch\": %d, \"flags\": %u, \"chunk\": %d, \"alpha\": %g, \"beta\": %g, "
                     "\"launches\": %lld, \"wall_ms\": %.3f, \"edges_per_s\": %.6g, \"status\": %u}\n",
                     g->n, (long long)(g->directed ? g->narcs : g->narcs / 2), (int)g->weighted, (int)g->directed,
                     g->last_nsrc, o.batch, o.flags, o.chunk, (double)o.alpha, (double)o.beta, (long long)g->launches,
                     ms, ms > 0.0 ? (double)g->last_nsrc * (double)(g->directed ? g->narcs : g->narcs / 2) / (ms / 1e3) : 0.0,
                     status);
    }
    if (status & BC_STATUS_BOUNDS) return fail(BC_ERR_BOUNDS, "device bounds check fired");
    if (status & BC_STATUS_DENSE_TIMEOUT) return fail(BC_ERR_TIMEOUT, "tensor-core pipeline wait timed out");
    if (status & BC_STATUS_COPY_TIMEOUT) return fail(BC_ERR_TIMEOUT, "staged row copy wait timed out");
    if (status & BC_STATUS_SIGMA_OVERFLOW) return BC_WARN_SIGMA_OVERFLOW;
    return BC_OK;
}

int bc_source_hashes(bc_graph *g, uint64_t *h_sigma, uint64_t *h_dist, int64_t *dist_sum, int64_t *reach) {
    g_err.clear();
    if (!g) return fail(BC_ERR_ARG, "graph is NULL");
    if (!g->has_run || !g->has_hash) return fail(BC_ERR_STATE, "no bc_run with per-source summaries");
    const size_t k = (size_t)g->last_nsrc;
    cudaStream_t st = g->last_stream;
    if (k) {
        if (h_sigma) CK(cudaMemcpyAsync(h_sigma, g->h_sigma.p, k * 8, cudaMemcpyDefault, st));
        if (h_dist) CK(cudaMemcpyAsync(h_dist, g->h_dist.p, k * 8, cudaMemcpyDefault, st));
        if (dist_sum) CK(cudaMemcpyAsync(dist_sum, g->dist_sum.p, k * 8, cudaMemcpyDefault, st));
        if (reach) CK(cudaMemcpyAsync(reach, g->reach.p, k * 8, cudaMemcpyDefault, st));
    }
    CK(cudaStreamSynchronize(st));
    return BC_OK;
}

int bc_forward_rows(bc_graph *g, const int32_t *sources, int32_t k, uint64_t *sigma, int32_t *dist,
                    const bc_options *opt, void *cuda_stream) {
    g_err.clear();
    if (!g) return fail(BC_ERR_ARG, "graph is NULL");
    if (k < 0 || (k > 0 && !sources)) return fail(BC_ERR_ARG, "bad source list");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int W = 0;
    int r = g->weighted ? BC_OK : resolve_batch(opt, &W);
    if (!r) set_run_options(g, opt);
    if (r) return r;
    int32_t nsrc = 0;
    r = stage_sources(g, sources, k, &nsrc);
    if (r) return r;
    if (nsrc == 0) return BC_OK;
    const size_t cells = (size_t)nsrc * g->n;
    DevBuf<uint64_t> ds;
    DevBuf<int32_t> dd;
    if (sigma) CK(ds.ensure(cells));
    if (dist) CK(dd.ensure(cells));
    CK(cudaMemsetAsync(&g->ctl->status, 0, sizeof(uint32_t), st));
    g->timing = false;
    if (g->weighted && opt && (opt->flags & BC_DENSE)) {
        if (!sigma || !dist) return fail(BC_ERR_ARG, "BC_DENSE rows of a weighted graph need both outputs");
        r = run_minplus(g, nsrc, st, false, ds.p, dd.p);
    } else if (g->weighted)
        r = run_weighted(g, nsrc, opt, st, false, false, sigma ? ds.p : nullptr, dist ? dd.p : nullptr);
    else
        r = run_batches(g, nsrc, W, opt, st, false, false, sigma ? ds.p : nullptr, dist ? dd.p : nullptr);
    uint32_t status = 0;
    if (!r) {
        cudaError_t e = cudaSuccess;
        if (sigma) e = cudaMemcpyAsync(sigma, ds.p, cells * 8, cudaMemcpyDefault, st);
        if (e == cudaSuccess && dist) e = cudaMemcpyAsync(dist, dd.p, cells * 4, cudaMemcpyDefault, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&status, &g->ctl->status, 4, cudaMemcpyDefault, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) r = fail(BC_ERR_CUDA, std::string("forward rows: ") + cudaGetErrorString(e));
    }
    cudaStreamSynchronize(st);
    ds.release();
    dd.release();
    if (r) return r;
    if (status & (BC_STATUS_DENSE_TIMEOUT | BC_STATUS_COPY_TIMEOUT))
        return fail(BC_ERR_TIMEOUT, "a device wait timed out");
    return (status & BC_STATUS_SIGMA_OVERFLOW) ? BC_WARN_SIGMA_OVERFLOW : BC_OK;
}

int bc_kernel_time(bc_graph *g, int32_t kind, int64_t *launches, double *total_ms) {
    g_err.clear();
    if (!g || kind < 0 || kind >= BC_KERNEL_KINDS) return fail(BC_ERR_ARG, "bad graph or kernel kind");
    if (!g->has_run) return fail(BC_ERR_STATE, "no completed bc_run");
    CK(cudaStreamSynchronize(g->last_stream));
    int64_t cnt = 0;
    double tot = 0.0;
    for (size_t i = 0; i < g->evused; ++i) {
        if (g->evpool[i].kind != kind) continue;
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, g->evpool[i].a, g->evpool[i].b));
        tot += ms;
        ++cnt;
    }
    if (launches) *launches = cnt;
    if (total_ms) *total_ms = tot;
    return BC_OK;
}

int bc_kernel_trace(bc_graph *g, int64_t cap, int32_t *kind, int32_t *level, float *ms, int64_t *count) {
    g_err.clear();
    if (!g || cap < 0 || (cap > 0 && (!kind || !level || !ms))) return fail(BC_ERR_ARG, "bad arguments");
    if (!g->has_run) return fail(BC_ERR_STATE, "no completed bc_run");
    CK(cudaStreamSynchronize(g->last_stream));
    const int64_t k = std::min<int64_t>(cap, (int64_t)g->evused);
    for (int64_t i = 0; i < k; ++i) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, g->evpool[i].a, g->evpool[i].b));
        kind[i] = g->evpool[i].kind;
        level[i] = g->evpool[i].level;
        ms[i] = t;
    }
    if (count) *count = (int64_t)g->evused;
    return BC_OK;
}

int64_t bc_launch_count(const bc_graph *g) { return g ? g->launches : 0; }

int bc_run_stats(bc_graph *g, int64_t *dag_arcs, int64_t *depth_sum, double *tensor_flops,
                 double *tensor_flops_f8) {
    g_err.clear();
    if (!g) return fail(BC_ERR_ARG, "graph is NULL");
    if (!g->has_run) return fail(BC_ERR_STATE, "no completed bc_run");
    unsigned long long v[2] = {0, 0};
    CK(cudaMemcpyAsync(v, &g->ctl->dag_arcs, sizeof(v), cudaMemcpyDeviceToHost, g->last_stream));
    CK(cudaStreamSynchronize(g->last_stream));
    if (dag_arcs) *dag_arcs = (int64_t)v[0];
    if (depth_sum) *depth_sum = (int64_t)v[1];
    if (tensor_flops) *tensor_flops = g->dense_flops;
    if (tensor_flops_f8) *tensor_flops_f8 = g->dense_flops_f8;
    return BC_OK;
}

int bc_set_default_options(bc_graph *g, const bc_options *opt) {
    g_err.clear();
    if (!g) return fail(BC_ERR_ARG, "graph is NULL");
    g->has_defaults = opt != nullptr;
    g->defaults = opt ? *opt : bc_options{};
    return BC_OK;
}

int bc_last_options(const bc_graph *g, bc_options *out) {
    g_err.clear();
    if (!g || !out) return fail(BC_ERR_ARG, "bad arguments");
    *out = g->last_opt;
    return BC_OK;
}

int bc_autotune(bc_graph *g, int32_t sample, bc_options *out, void *cuda_stream) {
    g_err.clear();
    if (!g) return fail(BC_ERR_ARG, "graph is NULL");
    if (sample < 0) return fail(BC_ERR_ARG, "sample < 0");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int32_t n = g->n;
    if (n == 0) {
        g->has_defaults = false;
        if (out) *out = bc_options{};
        return BC_OK;
    }
    const int32_t k = std::min<int32_t>(n, sample > 0 ? sample : 2048);
    std::vector<int32_t> src(k);
    for (int32_t i = 0; i < k; ++i) src[i] = (int32_t)(((int64_t)i * n) / k);  // spread over the ids
    ScopedBuf<int32_t> d_src;
    CK(d_src.ensure(k));
    CK(cudaMemcpy(d_src.p, src.data(), (size_t)k * sizeof(int32_t), cudaMemcpyHostToDevice));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    int err = BC_OK;
    // the shorter of two timed runs after one warm-up
    auto time_ms = [&](const bc_options &o, float *ms) -> int {
        float best = 0.0f;
        for (int rep = 0; rep < 3; ++rep) {
            if (cudaEventRecord(e0, st) != cudaSuccess) return fail(BC_ERR_CUDA, "event record");
            int r = bc_run(g, d_src.p, k, &o, st);
            if (r < 0) return r;
            r = bc_result(g, nullptr, nullptr);
            if (r < 0) return r;
            if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
                return fail(BC_ERR_CUDA, "event wait");
            float t = 0.0f;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep == 1 || (rep == 2 && t < best)) best = t;
        }
        *ms = best;
        return BC_OK;
    };
    bc_options best{};
    float best_ms = 0.0f;
    auto consider = [&](const bc_options &o) -> int {
        float ms = 0.0f;
        const int r = time_ms(o, &ms);
        if (r < 0) return r;
        if (best_ms == 0.0f || ms < best_ms) {
            best_ms = ms;
            best = o;
        }
        return BC_OK;
    };
    if (g->weighted) {
        // sources per wave of the bucket kernel: 1 to 4 or 8 per SM
        for (int per : {1, 2, 3, 4, 8}) {
            bc_options o{};
            o.flags = BC_NO_HASH;
            o.batch = per * sm_count_host();
            if ((err = consider(o)) < 0) break;
        }
    } else {
        // batch width x work-item chunk, then the set thresholds of the sweeps
        for (int b : {64, 128, 256})
            for (int c : {128, 256, 512}) {
                bc_options o{};
                o.flags = BC_NO_HASH;
                o.batch = b;
                o.chunk = c;
                if (err >= 0 && (err = consider(o)) < 0) break;
            }
        // then the look-ahead's tail threshold (the base's 1/64 is already timed)
        const bc_options base = best;
        for (float bt : {1.0f / 256.0f, 1.0f / 16.0f}) {
            bc_options o = base;
            o.beta = bt;
            if (err >= 0 && (err = consider(o)) < 0) break;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err < 0) return err;
    best.flags = 0;
    g->has_defaults = true;
    g->defaults = best;
    if (out) *out = best;
    return BC_OK;
}

int bc_graph_size(const bc_graph *g, int32_t *n, int64_t *m, int32_t *weighted) {
    if (!g) return fail(BC_ERR_ARG, "graph is NULL");
    if (n) *n = g->n;
    if (m) *m = g->narcs / 2;
    if (weighted) *weighted = g->weighted ? 1 : 0;
    return BC_OK;
}

void bc_destroy_graph(bc_graph *g) {
    if (!g) return;
    cudaDeviceSynchronize();
    devcache::t_recycle = true;  // the device is idle: the handle's blocks may serve the next handles
    free_graph(g);
    devcache::t_recycle = false;
}

void bc_release_cached_memory(void) { devcache::trim(-1); }

int bc_vertex_order(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t *perm) {
    g_err.clear();
    if (n < 0) return fail(BC_ERR_ARG, "n < 0");
    if (!row_ptr || !perm) return fail(BC_ERR_ARG, "row_ptr or perm is NULL");
    if (row_ptr[0] != 0) return fail(BC_ERR_ARG, "row_ptr[0] != 0");
    for (int32_t v = 0; v < n; ++v)
        if (row_ptr[v + 1] < row_ptr[v]) return fail(BC_ERR_ARG, "row_ptr decreases");
    if (row_ptr[n] > 0 && !col) return fail(BC_ERR_ARG, "col is NULL");
    for (int64_t e = 0; e < row_ptr[n]; ++e)
        if (col[e] < 0 || col[e] >= n) return fail(BC_ERR_ARG, "arc head out of range");
    bcgb::locality_order(n, row_ptr, col, perm);
    return BC_OK;
}

const char *bc_status_string(int status) {
    switch (status) {
        case BC_OK: return "ok";
        case BC_WARN_SIGMA_OVERFLOW: return "warning: a shortest-path count reached 2^64 (sigma wrapped)";
        case BC_ERR_ARG: return "invalid argument";
        case BC_ERR_NOT_SYMMETRIC: return "graph is not undirected (missing reverse arc, self-loop or duplicate)";
        case BC_ERR_WEIGHT: return "invalid weight";
        case BC_ERR_OOM: return "out of memory";
        case BC_ERR_CUDA: return "CUDA error";
        case BC_ERR_TIMEOUT: return "timed out waiting for the device";
        case BC_ERR_BOUNDS: return "device bounds check failed";
        case BC_ERR_UNSUPPORTED: return "unsupported option for this graph";
        case BC_ERR_STATE: return "call out of order";
        default: return "unknown status";
    }
}

const char *bc_last_error(void) { return g_err.c_str(); }

}  // extern "C"

struct bc_many {
    std::vector<bc_graph *> graphs;
    int W = 1, grid = 0, Lcap = 64;
    bool hash = true;  // per-source summaries into each graph's handle
    int32_t nitems = 0;
    DevBuf<bcgb::ManyGraph> d_graphs;
    DevBuf<bcgb::ManyItem> d_items;
    DevBuf<unsigned> queue, arrive, capped;
    DevBuf<double> partial;
    DevBuf<uint64_t> sigma;
    DevBuf<uint16_t> Smask;
    DevBuf<float> cval;
    DevBuf<uint32_t> F, V, ufr;
    bcgb::DevCtl *ctl = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t last_stream = nullptr;
    bool ran = false;
    int64_t arcs = 0;  // DAG arcs counted by the last persistent launch
};

namespace {

void free_many(bc_many *m) {
    if (m->exec) cudaGraphExecDestroy(m->exec);
    if (m->graph) cudaGraphDestroy(m->graph);
    m->d_graphs.release();
    m->d_items.release();
    m->queue.release();
    m->arrive.release();
    m->capped.release();
    m->partial.release();
    m->sigma.release();
    m->Smask.release();
    m->cval.release();
    m->F.release();
    m->V.release();
    m->ufr.release();
    if (m->ctl) cudaFree(m->ctl);
    delete m;
}

// Work items of the many-graph launch: each graph's source batches, split
// into several items when one graph alone is more than half a CTA's fair
// share of the total, then sorted by decreasing cost (LPT).
int build_many(bc_many *m) {
    const int B = 32 * m->W;
    struct GInfo {
        int nb;
        double cost;
    };
    std::vector<GInfo> info(m->graphs.size());
    double total = 0.0;
    int nmax = 1;
    for (size_t i = 0; i < m->graphs.size(); ++i) {
        const bc_graph *g = m->graphs[i];
        info[i].nb = (g->n + B - 1) / B;
        info[i].cost = (double)info[i].nb * (double)(g->n + g->narcs + 1);
        total += info[i].cost;
        nmax = std::max(nmax, g->n);
    }
    m->grid = bcgb::many_blocks_per_sm(m->W) * sm_count_host();
    const double share = std::max(1.0, total / (2.0 * m->grid));
    struct Item {
        bcgb::ManyItem it;
        double cost;
    };
    std::vector<Item> items;
    std::vector<bcgb::ManyGraph> gd(m->graphs.size());
    int64_t part_off = 0;
    for (size_t i = 0; i < m->graphs.size(); ++i) {
        const bc_graph *g = m->graphs[i];
        const int nb = info[i].nb;
        int q = (int)std::min<double>(nb, std::max(1.0, std::ceil(info[i].cost / share)));
        if (nb == 0) q = 0;
        gd[i].n = g->n;
        gd[i].nitems = std::max(q, 1);
        gd[i].part_off = q > 1 ? part_off : 0;
        gd[i].row_ptr = g->row_ptr.p;
        gd[i].col = g->col.p;
        gd[i].bc = g->bc.p;
        gd[i].h_sigma = gd[i].h_dist = nullptr;
        gd[i].dist_sum = gd[i].reach = nullptr;
        if (m->hash && g->n > 0) {
            bc_graph *gw = m->graphs[i];
            CK(gw->h_sigma.ensure(g->n));
            CK(gw->h_dist.ensure(g->n));
            CK(gw->dist_sum.ensure(g->n));
            CK(gw->reach.ensure(g->n));
            gd[i].h_sigma = gw->h_sigma.p;
            gd[i].h_dist = gw->h_dist.p;
            gd[i].dist_sum = gw->dist_sum.p;
            gd[i].reach = gw->reach.p;
        }
        if (q > 1) part_off += (int64_t)q * g->n;
        for (int k = 0; k < q; ++k) {
            Item x;
            x.it.graph = (int32_t)i;
            x.it.batch_lo = (int32_t)((int64_t)nb * k / q);
            x.it.batch_hi = (int32_t)((int64_t)nb * (k + 1) / q);
            x.it.part = k;
            x.cost = info[i].cost * (x.it.batch_hi - x.it.batch_lo) / nb;
            items.push_back(x);
        }
    }
    std::stable_sort(items.begin(), items.end(), [](const Item &a, const Item &b) { return a.cost > b.cost; });
    std::vector<bcgb::ManyItem> hit(items.size());
    for (size_t i = 0; i < items.size(); ++i) hit[i] = items[i].it;
    m->nitems = (int32_t)hit.size();
    m->Lcap = 64;
    const size_t nw32 = ((size_t)nmax + 31) / 32;
    const size_t G = (size_t)m->grid;
    CK(m->d_graphs.ensure(gd.size()));
    CK(cudaMemcpy(m->d_graphs.p, gd.data(), gd.size() * sizeof(gd[0]), cudaMemcpyHostToDevice));
    CK(m->d_items.ensure(hit.size()));
    if (!hit.empty()) CK(cudaMemcpy(m->d_items.p, hit.data(), hit.size() * sizeof(hit[0]), cudaMemcpyHostToDevice));
    CK(m->queue.ensure(1));
    CK(m->arrive.ensure(gd.size()));
    CK(m->capped.ensure(gd.size()));
    CK(cudaMemset(m->arrive.p, 0, gd.size() * sizeof(unsigned)));
    CK(m->partial.ensure((size_t)std::max<int64_t>(part_off, 1)));
    CK(m->sigma.ensure(G * nmax * B));
    CK(m->Smask.ensure(G * 2 * nmax * B));
    CK(m->cval.ensure(G * 2 * nmax * B));
    CK(m->F.ensure(G * m->Lcap * nmax * m->W));
    CK(m->V.ensure(G * 2 * nmax * m->W));
    CK(m->ufr.ensure(G * m->Lcap * nw32));
    CK(cudaMalloc((void **)&m->ctl, sizeof(bcgb::DevCtl)));

    bcgb::ManyParams p{};
    p.ngraphs = (int32_t)gd.size();
    p.nitems = m->nitems;
    p.nmax = nmax;
    p.nw32max = (int32_t)nw32;
    p.Lcap = m->Lcap;
    p.graphs = m->d_graphs.p;
    p.items = m->d_items.p;
    p.queue = m->queue.p;
    p.arrive = m->arrive.p;
    p.capped = m->capped.p;
    p.partial = m->partial.p;
    p.sigma = m->sigma.p;
    p.S = m->Smask.p;
    p.cval = m->cval.p;
    p.F = m->F.p;
    p.V = m->V.p;
    p.ufr = m->ufr.p;
    p.ctl = m->ctl;
    // capture the reset + persistent launch once; every run replays it
    cudaStream_t cap = nullptr;
    CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->queue.p, 0, sizeof(unsigned), cap);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->capped.p, 0, gd.size() * sizeof(unsigned), cap);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->ctl, 0, sizeof(bcgb::DevCtl), cap);
    if (e == cudaSuccess && m->nitems > 0) {
        bcgb::many_launch(m->W, p, m->grid, cap);
        e = cudaGetLastError();
    }
    cudaGraph_t gr = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cap, &gr);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&m->exec, gr, 0);
    m->graph = gr;
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) return fail(BC_ERR_CUDA, std::string("many-graph capture: ") + cudaGetErrorString(e));
    return BC_OK;
}

}  // namespace

extern "C" {

int bc_many_create(bc_graph *const *graphs, int32_t k, const bc_options *opt, bc_many **out) {
    g_err.clear();
    if (!out || (k > 0 && !graphs) || k < 0) return fail(BC_ERR_ARG, "bad arguments");
    *out = nullptr;
    const int b = (opt && opt->batch) ? opt->batch : 32;
    if (b != 32 && b != 64 && b != 128 && b != 256) return fail(BC_ERR_ARG, "many-graph batch must be 32, 64, 128 or 256");
    bc_many *m = new (std::nothrow) bc_many();
    if (!m) return fail(BC_ERR_OOM, "host allocation failed");
    m->W = b / 32;
    m->hash = !(opt && (opt->flags & BC_NO_HASH));
    for (int32_t i = 0; i < k; ++i) {
        if (!graphs[i] || graphs[i]->weighted || graphs[i]->directed) {
            free_many(m);
            return fail(BC_ERR_UNSUPPORTED, "bc_many takes unweighted undirected graph handles");
        }
        m->graphs.push_back(graphs[i]);
    }
    const int r = build_many(m);
    if (r) {
        free_many(m);
        return r;
    }
    *out = m;
    return BC_OK;
}

int bc_many_run(bc_many *m, void *cuda_stream) {
    g_err.clear();
    if (!m) return fail(BC_ERR_ARG, "plan is NULL");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (m->exec) CK(cudaGraphLaunch(m->exec, st));
    for (bc_graph *g : m->graphs) {
        g->has_run = true;
        g->has_hash = m->hash;
        g->reordered = false;
        g->last_stream = st;
        g->last_nsrc = g->n;
        g->launches = 0;
    }
    m->last_stream = st;
    m->ran = true;
    return BC_OK;
}

int bc_many_result(bc_many *m, uint32_t *status_flags, int32_t *rerun) {
    g_err.clear();
    if (!m) return fail(BC_ERR_ARG, "plan is NULL");
    if (!m->ran) return fail(BC_ERR_STATE, "no bc_many_run");
    uint32_t status = 0;
    unsigned long long arcs = 0;
    std::vector<unsigned> capped(m->graphs.size());
    CK(cudaMemcpyAsync(&status, &m->ctl->status, 4, cudaMemcpyDeviceToHost, m->last_stream));
    CK(cudaMemcpyAsync(&arcs, &m->ctl->dag_arcs, 8, cudaMemcpyDeviceToHost, m->last_stream));
    if (!capped.empty())
        CK(cudaMemcpyAsync(capped.data(), m->capped.p, capped.size() * 4, cudaMemcpyDeviceToHost, m->last_stream));
    CK(cudaStreamSynchronize(m->last_stream));
    m->arcs = (int64_t)arcs;
    int32_t nre = 0;
    for (size_t i = 0; i < capped.size(); ++i) {
        if (!capped[i]) continue;
        bc_options o{};
        o.batch = 32;
        const int r = bc_run(m->graphs[i], nullptr, 0, &o, m->last_stream);
        if (r < 0) return r;
        uint32_t st2 = 0;
        const int r2 = bc_result(m->graphs[i], nullptr, &st2);
        if (r2 < 0) return r2;
        status |= st2;
        ++nre;
    }
    if (rerun) *rerun = nre;
    if (status_flags) *status_flags = status;
    return (status & BC_STATUS_SIGMA_OVERFLOW) ? BC_WARN_SIGMA_OVERFLOW : BC_OK;
}

int bc_many_stats(const bc_many *m, int64_t *dag_arcs) {
    g_err.clear();
    if (!m) return fail(BC_ERR_ARG, "plan is NULL");
    if (!m->ran) return fail(BC_ERR_STATE, "no bc_many_run");
    if (dag_arcs) *dag_arcs = m->arcs;
    return BC_OK;
}

void bc_many_destroy(bc_many *m) {
    if (!m) return;
    cudaDeviceSynchronize();
    free_many(m);
}

int bc_run_many(bc_graph *const *graphs, int32_t k, const bc_options *opt, void *cuda_stream) {
    bc_many *m = nullptr;
    int r = bc_many_create(graphs, k, opt, &m);
    if (r) return r;
    r = bc_many_run(m, cuda_stream);
    if (!r) r = bc_many_result(m, nullptr, nullptr);
    bc_many_destroy(m);
    return r;
}

}  // extern "C"
