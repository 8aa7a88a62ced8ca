// msbfs.cu -- batched multi-source Brandes for unweighted graphs.
//
// One batch runs B = 32*W sources in lockstep, level by level (Section 4's
// "nodes are visited level by level", applied to many sources at once):
//
//   forward, level l -> l+1 (pull):  for every vertex v still unvisited by
//     some source, sigma_s(v) = sum over neighbours u with d(s,u) = l of
//     sigma_s(u), i.e. the sum over P_s(v) of Section 1.1; v joins frontier
//     l+1 for every source whose sum is non-zero.
//   backward, level l (pull over successors, Theorem 1.1): with
//     c_s(w) = (1 + delta_s*(w)) / sigma_s(w) stored for level l+1,
//     delta_s*(v) = sigma_s(v) * sum_{w adjacent, d(s,w) = l+1} c_s(w),
//     which is Lemma 3.5's ((D_l + Delta_l) div Lambda) . A masked to level
//     l-1 and multiplied by Lambda, one row per source.
//   BC(v) += sum over the batch of delta_s*(v) (FP64, fixed order), fused
//     into the backward step; the source itself (level 0) is never summed.
//
// Thread mapping: one warp per work item (a vertex, or a chunk of a
// high-degree vertex's arcs); the per-vertex steps (probe, bit-transposed
// walk, stores) are in msbfs_body.cuh. Warps are persistent and stride over
// the items, which are sorted by decreasing degree. Chunks of one vertex
// combine through partial buffers: the last chunk to arrive (atomic counter)
// sums them in chunk order, so every result is deterministic and no wait is
// needed.
#include <cuda_runtime.h>

#include <atomic>

#include "bc_internal.cuh"
#include "msbfs_body.cuh"
#include "pdl.cuh"

namespace bcgb {
namespace {

constexpr int kBlock = 256;
constexpr int kWarps = kBlock / 32;
constexpr unsigned kFull = 0xffffffffu;
using body::load_row;
using body::valid_word;
using body::transpose32;

// A level's union-frontier filter pays when its frontier is narrow: a wide
// one lets most neighbours through, and the filter's bit load is one more
// dependent load per arc. Wide: at least n / kFilterRatio vertices (the size
// the forward recorded; no record, always filter).
constexpr uint32_t kFilterRatio = 32;
__device__ __forceinline__ bool filter_level(const MsParams &p, int l) {
    return p.lsize == nullptr || (uint64_t)p.lsize[l] * kFilterRatio < (uint64_t)p.n;
}

template <int W>
__global__ void __launch_bounds__(kBlock) k_init(const MsParams p) {
    constexpr int B = 32 * W;
    pdl::enter();
    const size_t nW = (size_t)p.n * W;
    const size_t stride = (size_t)gridDim.x * kBlock;
    const size_t tid = (size_t)blockIdx.x * kBlock + threadIdx.x;
    for (size_t i = tid; i < 2 * nW; i += stride) {
        p.F[i] = 0u;  // frontiers of levels 0 and 1
        p.V[i] = 0u;  // visited through levels -1 and 0
    }
    const size_t nu = (size_t)p.Lcap * p.nw32;
    for (size_t i = tid; i < nu; i += stride) p.ufr[i] = 0u;
    // masked level-0 rows of the sources start at zero
    for (size_t i = tid; i < (size_t)p.nb * B; i += stride) p.S[(size_t)p.sources[i / B] * B + i % B] = 0;
    for (size_t i = tid; i < (size_t)p.Lcap; i += stride) p.wide[i] = 0u;
    __shared__ bool s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&p.ctl->blocks_done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // d(s,s) = 0 and sigma_s(s) = 1 (Section 1.1); the sources are the
    // vertices visited through level 0
    for (int b = threadIdx.x; b < p.nb; b += kBlock) {
        const int s = p.sources[b];
        atomicOr(p.F + (size_t)s * W + (b >> 5), 1u << (b & 31));
        atomicOr(p.V + nW + (size_t)s * W + (b >> 5), 1u << (b & 31));
        atomicOr(p.ufr + (s >> 5), 1u << (s & 31));
        p.sigma[(size_t)s * B + b] = 1ull;
        p.S[(size_t)s * B + b] = 1;
    }
    if (threadIdx.x == 0) {
        if (p.lsize) p.lsize[0] = (uint32_t)p.nb;
        p.ctl->fwd_done = 0u;
        p.ctl->nonempty = 0u;
        p.ctl->nlevels = 0;
        p.ctl->batch_arcs = 0ull;
        p.ctl->front_new = 0u;
        p.ctl->front_last = 0xffffffffu;  // level 0 (the sources) is not counted
        p.ctl->seq = p.seq;
        atomicExch(&p.ctl->blocks_done, 0u);
    }
}

// Level 0 -> 1 straight from the sources' rows: the vertices at distance 1
// from s are its neighbours, each with exactly one shortest path (through
// the arc from s). The batch's arcs out of its sources are dealt over the
// whole grid (block scan of the source degrees), so a high-degree source is
// shared out. No masked rows are written: the next level sees that every
// count is 1 and counts predecessors instead (fwd_sum, `ones`).
template <int W>
__global__ void __launch_bounds__(kBlock) k_first(const MsParams p) {
    constexpr int B = 32 * W;
    pdl::enter();
    __shared__ int s_off[kBlock + 1];
    __shared__ int s_wsum[kWarps];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    {
        int deg = 0;
        if (t < p.nb) deg = p.row_ptr[p.sources[t] + 1] - p.row_ptr[p.sources[t]];
        int x = deg;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(kFull, x, off);
            if (lane >= off) x += y;
        }
        if (lane == 31) s_wsum[wid] = x;
        __syncthreads();
        int base = 0;
        for (int k = 0; k < wid; ++k) base += s_wsum[k];
        s_off[t] = base + x - deg;
        if (t == kBlock - 1) s_off[kBlock] = base + x;
        __syncthreads();
    }
    const size_t nW = (size_t)p.n * W;
    uint32_t *F1 = p.F + nW;
    uint32_t *uf1 = p.ufr + p.nw32;
    const int total = s_off[p.nb];
    for (int a = blockIdx.x * kBlock + t; a < total; a += gridDim.x * kBlock) {
        int lo = 0, hi = p.nb - 1;  // the source b whose arcs hold position a: s_off[b] <= a < s_off[b + 1]
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_off[mid] <= a) lo = mid; else hi = mid - 1;
        }
        const int b = lo;
        const int s = p.sources[b];
        const int v = p.col[p.row_ptr[s] + (a - s_off[b])];
        atomicOr(F1 + (size_t)v * W + (b >> 5), 1u << (b & 31));
        atomicOr(uf1 + (v >> 5), 1u << (v & 31));
        p.sigma[(size_t)v * B + b] = 1ull;
    }
    __syncthreads();
    if (t != 0) return;
    __threadfence();
    if (atomicAdd(&p.ctl->blocks_done, 1u) != gridDim.x - 1) return;
    __threadfence();
    atomicExch(&p.ctl->blocks_done, 0u);
    atomicAdd(&p.ctl->batch_arcs, (unsigned long long)total);
    if (total == 0) {  // every source isolated: depth 0
        p.ctl->fwd_done = 1u;
        p.ctl->nlevels = 0;
        host_word(&p.hctl->done, p.seq, 0u);
    }
    // level 1 has at most `total` vertices (the arcs out of the sources)
    p.ctl->front_last = (uint32_t)total;
    if (p.lsize) p.lsize[1] = (uint32_t)total;
    host_word(&p.hctl->counts, (uint32_t)total, 0xffffffffu);
    host_word(&p.hctl->progress, p.seq, 1u);
}

template <int W, bool HOOK>
__global__ void __launch_bounds__(kBlock, 3) k_forward(const MsParams p, const int l) {
    constexpr int B = 32 * W;
    pdl::enter();
    __shared__ uint32_t s_U[kWarps][32][W];  // unvisited words of the group's items
    __shared__ uint64_t s_bar[kWarps];
    __shared__ uint32_t s_qz[kWarps][32];
    extern __shared__ __align__(128) uint8_t s_stage[];
    __shared__ uint32_t s_flags;
    __shared__ unsigned long long s_arcs;
    __shared__ uint32_t s_front;  // vertices this block put into frontier l+1
    __shared__ int32_t s_u[kWarps][32];
    __shared__ uint32_t s_nz[kWarps][32];
    if (threadIdx.x == 0) {
        s_flags = 0u;
        s_arcs = 0ull;
        s_front = 0u;
    }
    __syncthreads();
    // speculative launches past the last level, and the level-capacity guard
    if (*(volatile uint32_t *)&p.ctl->fwd_done != 0u || l + 1 >= p.Lcap) return;

    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const size_t nW = (size_t)p.n * W;
    const uint32_t *Fl = p.F + (size_t)l * nW;
    uint32_t *Fn = p.F + (size_t)(l + 1) * nW;
    const uint32_t *ufl = p.ufr + (size_t)l * p.nw32;
    uint32_t *ufn = p.ufr + (size_t)(l + 1) * p.nw32;
    const uint32_t *Vin = p.V + (size_t)(l & 1) * nW;
    uint32_t *Vout = p.V + (size_t)((l + 1) & 1) * nW;
    const uint16_t *Sl = p.S_rd;  // masked rows of level l and l+1 (set by the launcher)
    uint16_t *Sn = p.S_wr;
    const bool wide = *(volatile uint32_t *)(p.wide + l) != 0u;
    const bool ones = l == 1 && p.first;  // level 1 written by k_first: all counts 1, no masked rows
    const uint32_t *ufl_f = filter_level(p, l) ? ufl : nullptr;  // the union filter, on narrow frontiers only
    bool produced = false, ovf = false, wide_next = false;
    uint32_t arcs = 0;  // predecessor relations counted by this lane
    body::WarpStage ws{s_stage + wib * stage::kFwdStageBytes, s_bar + wib, s_qz[wib], 0u, false,
                       body::stage_wctl(p.wait_ns, p.test_hold)};
    if (lane == 0) stage::bar_init(ws.bar);
    __syncwarp();

    // Persistent warps stride over the items (sorted by decreasing degree, so
    // every warp gets a similar mix; the chunks of one heavy vertex land on
    // different warps). A warp takes its next 32 items at once: lane k checks
    // item k's vertex (visited words; the new frontier row cleared when
    // nothing is left to find), then the warp works through the active ones.
    const int G = gridDim.x * kWarps;
    for (int g0 = blockIdx.x * kWarps + wib; g0 < p.nitems; g0 += 32 * G) {
        bool act = false;
        __syncwarp();  // the previous group's reads of s_U are done
        const int ik = g0 + lane * G;
        if (ik < p.nitems) {
            const int vk = p.item_v[ik];
            const int sk = p.item_slot[ik];
            uint32_t a[W], f[W];
            load_row<W>(Vin + (size_t)vk * W, a);
            load_row<W>(Fl + (size_t)vk * W, f);
            uint32_t any = 0;
#pragma unroll
            for (int j = 0; j < W; ++j) {
                const uint32_t vis = a[j] | f[j];
                Vout[(size_t)vk * W + j] = vis;  // chunks of one vertex write the same words
                const uint32_t u = ~vis & valid_word(p.nb, j);
                s_U[wib][lane][j] = u;
                any |= u;
            }
            act = any != 0u;
            if (!act && (sk < 0 || p.slot_first[sk] == sk))
#pragma unroll
                for (int j = 0; j < W; ++j) Fn[(size_t)vk * W + j] = 0u;
        }
        unsigned todo = __ballot_sync(kFull, act);
        __syncwarp();
        while (todo) {
            const int kk = __ffs(todo) - 1;
            todo &= todo - 1;
            const int it = g0 + kk * G;
            const int v = p.item_v[it];
            const int beg = p.item_beg[it];
            const int end = p.item_end[it];
            const int slot = p.item_slot[it];
            uint32_t U[W];
#pragma unroll
            for (int j = 0; j < W; ++j) U[j] = s_U[wib][kk][j];
            uint64_t acc[W];  // lane owns source 32j + lane
            uint32_t nf[W];
#pragma unroll
            for (int j = 0; j < W; ++j) {
                acc[j] = 0ull;
                nf[j] = 0u;
            }
            body::fwd_sum<W, true, true, HOOK>(p.col_f, beg, end, ufl_f, Fl, Sl, p.sigma, wide, ones, U, s_u[wib], s_nz[wib], lane,
                                         acc, nf, ovf, arcs, &ws);
            if (slot < 0) {
                const bool joined = body::store_next<W>(p.sigma, Sn, Fn, ufn, v, acc, nf, lane, wide_next);
                produced |= joined;
                if (joined && lane == 0) atomicAdd(&s_front, 1u);
                continue;
            }
            uint64_t *pp = p.part + (size_t)slot * B + lane;
#pragma unroll
            for (int j = 0; j < W; ++j) pp[32 * j] = acc[j];
#pragma unroll
            for (int j = 0; j < W; ++j)
                if (lane == j) p.pmask[(size_t)slot * W + j] = nf[j];
            __threadfence();
            __syncwarp();
            const int first = p.slot_first[slot];
            const int nch = p.slot_nch[slot];
            unsigned old = 0;
            if (lane == 0) old = atomicAdd(p.cnt + first, 1u);
            old = __shfl_sync(kFull, old, 0);
            if (old != (unsigned)(nch - 1)) continue;
            __threadfence();
#pragma unroll
            for (int j = 0; j < W; ++j) {
                acc[j] = 0ull;
                nf[j] = 0u;
            }
            for (int c = 0; c < nch; ++c) {
                const uint64_t *q = p.part + (size_t)(first + c) * B + lane;
                const uint32_t *qm = p.pmask + (size_t)(first + c) * W;
#pragma unroll
                for (int j = 0; j < W; ++j) {
                    const uint64_t x = __ldcg(q + 32 * j);
                    const uint64_t y = acc[j] + x;
                    ovf |= y < x;
                    acc[j] = y;
                    nf[j] |= __ldcg(qm + j);
                }
            }
            const bool joined = body::store_next<W>(p.sigma, Sn, Fn, ufn, v, acc, nf, lane, wide_next);
            produced |= joined;
            if (joined && lane == 0) atomicAdd(&s_front, 1u);
            if (lane == 0) p.cnt[first] = 0u;
        }
    }
    const unsigned wovf = __ballot_sync(kFull, ovf);
    const unsigned wwide = __ballot_sync(kFull, wide_next);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) arcs += __shfl_xor_sync(kFull, arcs, off);
    if (lane == 0) {
        if (produced) atomicOr(&s_flags, 1u);
        if (wovf) atomicOr(&s_flags, 2u);
        if (wwide) atomicOr(&s_flags, 4u);
        if (ws.fail) atomicOr(&s_flags, 8u);
        if (arcs) atomicAdd(&s_arcs, (unsigned long long)arcs);
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    if (s_arcs) atomicAdd(&p.ctl->batch_arcs, s_arcs);
    if (s_front) atomicAdd(&p.ctl->front_new, s_front);
    if (s_flags & 1u) atomicOr(&p.ctl->nonempty, 1u);
    if (s_flags & 2u) atomicOr(&p.ctl->status, BC_STATUS_SIGMA_OVERFLOW);
    if (s_flags & 8u) atomicOr(&p.ctl->status, BC_STATUS_COPY_TIMEOUT);
    if (s_flags & 4u) atomicOr(p.wide + l + 1, 1u);
    __threadfence();
    if (atomicAdd(&p.ctl->blocks_done, 1u) != gridDim.x - 1) return;
    // last block of this level: decide whether the forward pass ended
    __threadfence();
    const unsigned ne = atomicExch(&p.ctl->nonempty, 0u);
    atomicExch(&p.ctl->blocks_done, 0u);
    if (ne == 0u) {
        p.ctl->fwd_done = 1u;
        p.ctl->nlevels = l;
        p.ctl->depth_sum += (unsigned long long)l;
        p.ctl->dag_arcs += atomicExch(&p.ctl->batch_arcs, 0ull);
        host_word(&p.hctl->done, p.seq, (uint32_t)l);
    } else if (l + 2 >= p.Lcap) {
        p.ctl->fwd_done = 1u;
        p.ctl->nlevels = -1;
        host_word(&p.hctl->done, p.seq, 0xffffffffu);
    }
    // the sizes of frontiers l+1 and l (vertices), a hint for the host's look-ahead
    const uint32_t nxt = atomicExch(&p.ctl->front_new, 0u);
    const uint32_t cur = p.ctl->front_last;
    p.ctl->front_last = nxt;
    if (p.lsize) p.lsize[l + 1] = nxt;
    host_word(&p.hctl->counts, nxt, cur);
    host_word(&p.hctl->progress, p.seq, (uint32_t)(l + 1));
}

template <int W, bool HOOK>
__global__ void __launch_bounds__(kBlock, 4) k_backward(const MsParams p, const int l) {
    constexpr int B = 32 * W;
    pdl::enter();
    __shared__ uint32_t s_f[kWarps][32][W];  // level-l words of the group's items
    __shared__ int32_t s_v[kWarps][32];      // and their vertices
    __shared__ uint64_t s_bar[kWarps];
    __shared__ uint32_t s_qz[kWarps][32];
    extern __shared__ __align__(128) uint8_t s_stage[];
    __shared__ int32_t s_u[kWarps][32];
    __shared__ uint32_t s_nz[kWarps][32];
    __shared__ __align__(16) uint16_t s_sig[kWarps][W][32];  // the counts of the item being finalized
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const size_t nW = (size_t)p.n * W;
    const uint32_t *Fl = p.F + (size_t)l * nW;
    const uint32_t *Fs = p.F + (size_t)(l + 1) * nW;
    const uint32_t *ufs = p.ufr + (size_t)(l + 1) * p.nw32;
    const size_t nB = (size_t)p.n * B;
    // level 1 is the last level the backward computes (the sources' own
    // dependencies are not part of BC), so its c values have no reader
    float *Cl = l > 1 ? p.cval + (size_t)(l & 1) * nB : nullptr;
    const float *Cs = p.cval + (size_t)((l + 1) & 1) * nB;
    const uint32_t *ufs_f = filter_level(p, l + 1) ? ufs : nullptr;  // the union filter, on narrow frontiers only
    body::WarpStage ws{s_stage + wib * stage::kBwdStageBytes, s_bar + wib, s_qz[wib], 0u, false,
                       body::stage_wctl(p.wait_ns, p.test_hold)};
    if (lane == 0) stage::bar_init(ws.bar);
    __syncwarp();
    // where the finalize reads sigma_s(v) for the pairs at level l: none at
    // level 1 from k_first (every count is 1), the level's masked uint16 row
    // when each level has its own buffer and the level is narrow, else the
    // uint64 array
    const bool sig_ones = l == 1 && p.first;
    const uint16_t *Sl = (!sig_ones && p.s_levels > 2 && *(volatile const uint32_t *)(p.wide + l) == 0u)
                             ? p.S + (size_t)l * nB
                             : nullptr;
    // sigma row span of item k of the group (its words at level l), brought
    // into L2 two items ahead of the step that reads it
    auto prefetch_sigma = [&](int k) {
        if (sig_ones) return;
        uint32_t any = 0;
        int lo = W, hi = -1;
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const uint32_t x = s_f[wib][k][j];
            any |= x;
            if (x != 0u) {
                lo = j < lo ? j : lo;
                hi = j;
            }
        }
        if (any != 0u) {
            if (Sl)
                stage::prefetch_l2(Sl + (size_t)s_v[wib][k] * B + 32 * lo, 64u * (uint32_t)(hi - lo + 1));
            else
                stage::prefetch_l2(p.sigma + (size_t)s_v[wib][k] * B + 32 * lo, 256u * (uint32_t)(hi - lo + 1));
        }
    };
    // the forward pass's item striding; lane k of a warp checks whether its
    // k-th next item's vertex is at level l for any source (the same for all
    // chunks of v), then the warp works through the active items
    const int G = gridDim.x * kWarps;
    for (int g0 = blockIdx.x * kWarps + wib; g0 < p.nitems; g0 += 32 * G) {
        bool act = false;
        __syncwarp();  // the previous group's reads of s_f are done
        const int ik = g0 + lane * G;
        if (ik < p.nitems) {
            const int vk = p.item_v[ik];
            uint32_t f[W];
            load_row<W>(Fl + (size_t)vk * W, f);
            uint32_t any = 0;
#pragma unroll
            for (int j = 0; j < W; ++j) {
                s_f[wib][lane][j] = f[j];
                any |= f[j];
            }
            s_v[wib][lane] = vk;
            act = any != 0u;
        }
        unsigned todo = __ballot_sync(kFull, act);
        __syncwarp();
        if (act && __popc(todo & ((1u << lane) - 1u)) < 2) prefetch_sigma(lane);
        while (todo) {
            const int kk = __ffs(todo) - 1;
            todo &= todo - 1;
            if (lane == 0) {
                const unsigned k2 = __fns(todo, 0, 2);  // two active items ahead
                if (k2 < 32u) prefetch_sigma((int)k2);
            }
            const int it = g0 + kk * G;
            const int v = p.item_v[it];
            const int beg = p.item_beg[it];
            const int end = p.item_end[it];
            const int slot = p.item_slot[it];
            uint32_t f[W];
#pragma unroll
            for (int j = 0; j < W; ++j) f[j] = s_f[wib][kk][j];

            // an unsplit vertex finalizes right after its scan: its counts
            // (the words with a level-l source) are copied to shared memory
            // while the neighbours are scanned (even lanes, 4 bytes each)
            const bool early = slot < 0 && Sl != nullptr;
            if (early) {
#pragma unroll
                for (int j = 0; j < W; ++j)
                    if (f[j] != 0u && (lane & 1) == 0) {
                        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&s_sig[wib][j][lane]);
                        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst),
                                     "l"(Sl + (size_t)v * B + 32 * j + lane)
                                     : "memory");
                    }
                asm volatile("cp.async.commit_group;" ::: "memory");
            }
            float S[W];  // lane owns source 32j + lane
#pragma unroll
            for (int j = 0; j < W; ++j) S[j] = 0.0f;
            body::bwd_sum<W, true, true, HOOK>(p.col, beg, end, ufs_f, Fs, Cs, f, s_u[wib], s_nz[wib], lane, S, &ws);
            if (slot < 0) {
                if (early) {
                    asm volatile("cp.async.wait_group 0;" ::: "memory");
                    __syncwarp();
                }
                body::finalize_dep<W>(p.sigma, Sl, sig_ones, Cl, p.bc, v, f, S, lane,
                                      early ? &s_sig[wib][0][0] : nullptr);
                __syncwarp();  // the next item's copies overwrite s_sig
                continue;
            }
            float *pp = reinterpret_cast<float *>(p.part) + (size_t)slot * B + lane;
#pragma unroll
            for (int j = 0; j < W; ++j) pp[32 * j] = S[j];
            __threadfence();
            __syncwarp();
            const int first = p.slot_first[slot];
            const int nch = p.slot_nch[slot];
            unsigned old = 0;
            if (lane == 0) old = atomicAdd(p.cnt + first, 1u);
            old = __shfl_sync(kFull, old, 0);
            if (old != (unsigned)(nch - 1)) continue;
            __threadfence();
#pragma unroll
            for (int j = 0; j < W; ++j) S[j] = 0.0f;
#pragma unroll 4
            for (int c = 0; c < nch; ++c) {  // chunk order; the unrolled loads are independent
                const float *q = reinterpret_cast<const float *>(p.part) + (size_t)(first + c) * B + lane;
#pragma unroll
                for (int j = 0; j < W; ++j) S[j] += __ldcg(q + 32 * j);
            }
            body::finalize_dep<W>(p.sigma, Sl, sig_ones, Cl, p.bc, v, f, S, lane);
            if (lane == 0) p.cnt[first] = 0u;
        }
    }
    if (lane == 0 && ws.fail) atomicOr(&p.ctl->status, BC_STATUS_COPY_TIMEOUT);
}

// Per-source summaries over tiles of 32 vertices x 32 sources: a warp keeps
// one frontier word j (sources 32j .. 32j+31) and strides over the vertex
// tiles. Lane k loads word j of vertex v0+k for the reached set (visited
// through level L-1 or in frontier L) and for every frontier F[l], l <= L;
// a 32x32 bit transpose gives lane s the 32-vertex mask of its own source.
// Per level, the count of set bits and the sum of (v+1) over them (a popcount
// of the mask and five popcounts weighted by the bits of the in-tile index)
// give the distance terms; the path-count term adds sigma_s(v) (v+1) over the
// reached vertices, one coalesced 8-byte load per vertex. All loads of a
// tile are issued before any is used. Every sum is an integer mod 2^64, so
// the block totals go straight into the outputs with atomic adds (the run
// zeroes them first) and the result does not depend on the order of adds.
template <int W>
__global__ void __launch_bounds__(kBlock, 2) k_hash(const MsParams p, const int L) {
    constexpr int B = 32 * W;
    constexpr int kHL = 12;  // frontier levels loaded up front; deeper ones in a loop
    pdl::enter();
    __shared__ unsigned long long sh[4][B];
    for (int i = threadIdx.x; i < 4 * B; i += kBlock) (&sh[0][0])[i] = 0ull;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int j = gw % W;                        // this warp's frontier word
    const int tstride = gridDim.x * kWarps / W;  // warps per word
    const int ntiles = (p.n + 31) / 32;
    const size_t nW = (size_t)p.n * W;
    const uint32_t *Vl = p.V + (size_t)(L & 1) * nW;
    const uint32_t *FL = p.F + (size_t)L * nW;
    uint64_t hs = 0, hd = 0, ds = 0, rc = 0;
    auto level_terms = [&](uint32_t word, int l, int v0) {
        const uint32_t T = transpose32(word, lane);
        const uint32_t c = (uint32_t)__popc(T);
        // the sum of the in-tile indices k of the set bits, bit by bit of k
        const uint32_t ks = (uint32_t)__popc(T & 0xAAAAAAAAu) + 2u * (uint32_t)__popc(T & 0xCCCCCCCCu) +
                            4u * (uint32_t)__popc(T & 0xF0F0F0F0u) + 8u * (uint32_t)__popc(T & 0xFF00FF00u) +
                            16u * (uint32_t)__popc(T & 0xFFFF0000u);
        const uint64_t vsum = (uint64_t)c * (uint64_t)(v0 + 1) + (uint64_t)ks;  // sum of (v+1)
        hd += (uint64_t)(l + 1) * vsum;
        ds += (uint64_t)l * (uint64_t)c;
    };
    for (int t = gw / W; t < ntiles; t += tstride) {
        const int v0 = 32 * t;
        const int vk = v0 + lane;
        const bool in = vk < p.n;
        const size_t wk = (size_t)(in ? vk : 0) * W + j;
        uint32_t fw[kHL];
#pragma unroll
        for (int l = 0; l < kHL; ++l) fw[l] = (in && l <= L) ? __ldg(p.F + (size_t)l * nW + wk) : 0u;
        const uint32_t rv = in ? (__ldg(Vl + wk) | __ldg(FL + wk)) : 0u;
        const int nk = p.n - v0 < 32 ? p.n - v0 : 32;  // vertices in this tile
        const uint64_t *sg = p.sigma + (size_t)v0 * B + 32 * j + lane;
        uint64_t x[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) x[k] = k < nk ? __ldg(sg + (size_t)k * B) : 0ull;
        const uint32_t R = transpose32(rv, lane);
        rc += (uint64_t)__popc(R);
#pragma unroll
        for (int l = 0; l < kHL; ++l)
            if (l <= L) level_terms(fw[l], l, v0);
        for (int l = kHL; l <= L; ++l) level_terms(in ? __ldg(p.F + (size_t)l * nW + wk) : 0u, l, v0);
#pragma unroll
        for (int k = 0; k < 16; ++k)
            if ((R >> k) & 1u) hs += x[k] * (uint64_t)(v0 + k + 1);
#pragma unroll
        for (int k = 0; k < 16; ++k) x[k] = 16 + k < nk ? __ldg(sg + (size_t)(16 + k) * B) : 0ull;
#pragma unroll
        for (int k = 0; k < 16; ++k)
            if ((R >> (16 + k)) & 1u) hs += x[k] * (uint64_t)(v0 + 16 + k + 1);
    }
    atomicAdd(&sh[0][32 * j + lane], (unsigned long long)hs);
    atomicAdd(&sh[1][32 * j + lane], (unsigned long long)hd);
    atomicAdd(&sh[2][32 * j + lane], (unsigned long long)ds);
    atomicAdd(&sh[3][32 * j + lane], (unsigned long long)rc);
    __syncthreads();
    for (int b = threadIdx.x; b < p.nb; b += kBlock) {
        const int o = p.out_index ? p.out_index[b] : b;
        atomicAdd(reinterpret_cast<unsigned long long *>(p.h_sigma + o), sh[0][b]);
        atomicAdd(reinterpret_cast<unsigned long long *>(p.h_dist + o), sh[1][b]);
        atomicAdd(reinterpret_cast<unsigned long long *>(p.dist_sum + o), sh[2][b]);
        atomicAdd(reinterpret_cast<unsigned long long *>(p.reach + o), sh[3][b]);
    }
}

// Rows of the forward pass for bc_forward_rows: out[b][v] for this batch.
template <int W>
__global__ void __launch_bounds__(kBlock) k_rows(const MsParams p, const int L, uint64_t *sig_out,
                                                 int32_t *dist_out) {
    pdl::enter();
    constexpr int B = 32 * W;
    const size_t nW = (size_t)p.n * W;
    const size_t total = (size_t)p.n * B;
    for (size_t i = (size_t)blockIdx.x * kBlock + threadIdx.x; i < total; i += (size_t)gridDim.x * kBlock) {
        const int v = (int)(i / B);
        const int b = (int)(i % B);
        if (b >= p.nb) continue;
        int lev = -1;
        for (int l = 0; l <= L; ++l)
            if ((p.F[(size_t)l * nW + (size_t)v * W + (b >> 5)] >> (b & 31)) & 1u) lev = l;
        const size_t o = (size_t)b * p.n + v;
        if (dist_out) dist_out[o] = lev;
        if (sig_out) sig_out[o] = lev >= 0 ? p.sigma[(size_t)v * B + b] : 0ull;
    }
}

__global__ void k_merge(const double *__restrict__ src, double *__restrict__ dst, int32_t n, const DevCtl *from,
                        DevCtl *to) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] += src[i];
    if (from && blockIdx.x == 0 && threadIdx.x == 0) {
        atomicOr(&to->status, from->status);
        atomicAdd(&to->dag_arcs, from->dag_arcs);
        atomicAdd(&to->depth_sum, from->depth_sum);
    }
}

__global__ void k_scale(double *x, int32_t n, double f) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] *= f;
}

int sm_count() {
    static int c = 0;
    if (c == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
        if (c <= 0) c = 1;
    }
    return c;
}

// dynamic shared memory of the level kernels: one row stage per warp
constexpr size_t kFwdSmem = (size_t)kWarps * stage::kFwdStageBytes;
constexpr size_t kBwdSmem = (size_t)kWarps * stage::kBwdStageBytes;

// Raise the kernel's dynamic shared memory limit once per device.
template <class K>
void stage_attr(K kernel, size_t bytes, std::atomic<uint32_t> &done) {
    int dev = 0;
    cudaGetDevice(&dev);
    const uint32_t bit = 1u << (dev & 31);
    if (done.load(std::memory_order_acquire) & bit) return;
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    done.fetch_or(bit, std::memory_order_acq_rel);
}
template <int W, bool HOOK>
void fwd_attr() {
    static std::atomic<uint32_t> done{0};
    stage_attr(k_forward<W, HOOK>, kFwdSmem, done);
}
template <int W, bool HOOK>
void bwd_attr() {
    static std::atomic<uint32_t> done{0};
    stage_attr(k_backward<W, HOOK>, kBwdSmem, done);
}

template <class K>
int item_blocks(const MsParams &p, K kernel, size_t dyn_smem = 0) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, dyn_smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const int need = (p.nitems + kWarps - 1) / kWarps;
    const int cap = per_sm * sm_count();
    return need < cap ? need : cap;
}

// The level kernels with the wait bound / test hook read (HOOK), for runs
// that set either; the others carry neither in their staging loop.
bool uses_hook(const MsParams &p) { return p.wait_ns != 0 || p.test_hold != 0; }

template <int W, bool HOOK>
void launch_forward_t(const MsParams &p, int level, cudaStream_t st) {
    fwd_attr<W, HOOK>();
    pdl::launch(k_forward<W, HOOK>, item_blocks(p, k_forward<W, HOOK>, kFwdSmem), kBlock, kFwdSmem, st, p, level);
}
template <int W, bool HOOK>
void launch_backward_t(const MsParams &p, int level, cudaStream_t st) {
    bwd_attr<W, HOOK>();
    pdl::launch(k_backward<W, HOOK>, item_blocks(p, k_backward<W, HOOK>, kBwdSmem), kBlock, kBwdSmem, st, p,
                level);
}

// Persistent grid: as many blocks as fit on the GPU at once (occupancy of
// the kernel instance), never more than the items need.
template <int W>
void launch_init_t(const MsParams &p, cudaStream_t st) {
    const size_t work = (size_t)p.n * W;
    int g = (int)((work + kBlock - 1) / kBlock);
    g = g < 1 ? 1 : (g > 8 * sm_count() ? 8 * sm_count() : g);
    pdl::launch(k_init<W>, g, kBlock, 0, st, p);
}

}  // namespace

bool ms_supported_width(int W) { return W == 1 || W == 2 || W == 4 || W == 8; }

#define BCGB_DISPATCH_W(W, CALL)                  \
    switch (W) {                                  \
        case 1: { constexpr int kW = 1; CALL; } break; \
        case 2: { constexpr int kW = 2; CALL; } break; \
        case 4: { constexpr int kW = 4; CALL; } break; \
        case 8: { constexpr int kW = 8; CALL; } break; \
        default: break;                           \
    }

void ms_launch_init(int W, const MsParams &p, cudaStream_t st) {
    BCGB_DISPATCH_W(W, launch_init_t<kW>(p, st));
}

void ms_launch_first(int W, const MsParams &p, cudaStream_t st) {
    if (p.nb == 0) return;
    // one thread per arc out of the batch's sources when the host counted them
    int g = 2 * sm_count();
    if (p.first_arcs > 0) {
        const int64_t need = (p.first_arcs + kBlock - 1) / kBlock;
        g = need < g ? (int)need : g;
    }
    BCGB_DISPATCH_W(W, pdl::launch(k_first<kW>, g, kBlock, 0, st, p));
}

void ms_launch_forward(int W, const MsParams &p0, int level, cudaStream_t st) {
    if (p0.nitems == 0) return;
    MsParams p = p0;
    const size_t nB = (size_t)p.n * 32 * W;
    p.S_rd = p.S + (size_t)(level % p.s_levels) * nB;  // one buffer per level, or two by parity
    p.S_wr = p.S + (size_t)((level + 1) % p.s_levels) * nB;
    if (uses_hook(p)) {
        BCGB_DISPATCH_W(W, (launch_forward_t<kW, true>(p, level, st)));
    } else {
        BCGB_DISPATCH_W(W, (launch_forward_t<kW, false>(p, level, st)));
    }
}

void ms_launch_backward(int W, const MsParams &p, int level, cudaStream_t st) {
    if (p.nitems == 0) return;
    if (uses_hook(p)) {
        BCGB_DISPATCH_W(W, (launch_backward_t<kW, true>(p, level, st)));
    } else {
        BCGB_DISPATCH_W(W, (launch_backward_t<kW, false>(p, level, st)));
    }
}

void ms_launch_hash(int W, const MsParams &p, int nlevels, cudaStream_t st) {
    const int units = ((p.n + 31) / 32) * W;  // (tile, word) pairs
    const int need = (units + kWarps - 1) / kWarps;
    const int cap = 2 * sm_count();            // one wave at the kernel's occupancy
    const int g = need < 1 ? 1 : (need < cap ? need : cap);
    BCGB_DISPATCH_W(W, pdl::launch(k_hash<kW>, g, kBlock, 0, st, p, nlevels));
}

void ms_launch_rows(int W, const MsParams &p, int nlevels, uint64_t *sig_out, int32_t *dist_out,
                    cudaStream_t st) {
    const int g = 4 * sm_count();
    BCGB_DISPATCH_W(W, pdl::launch(k_rows<kW>, g, kBlock, 0, st, p, nlevels, sig_out, dist_out));
}

void ms_launch_merge(const double *src, double *dst, int32_t n, const DevCtl *from, DevCtl *to, cudaStream_t st) {
    int g = (n + kBlock - 1) / kBlock;
    g = g < 1 ? 1 : (g > 4 * sm_count() ? 4 * sm_count() : g);
    k_merge<<<g, kBlock, 0, st>>>(src, dst, n, from, to);
}

void launch_scale(double *x, int32_t n, double f, cudaStream_t st) {
    if (n <= 0) return;
    int g = (n + kBlock - 1) / kBlock;
    g = g > 4 * sm_count() ? 4 * sm_count() : g;
    k_scale<<<g, kBlock, 0, st>>>(x, n, f);
}

}  // namespace bcgb
