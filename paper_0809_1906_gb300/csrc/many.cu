// many.cu -- exact all-sources betweenness of many small graphs in one
// persistent launch (bc_many_* / bc_run_many).
//
// Work item = (graph, range of source batches). Items are ordered by
// decreasing cost (longest-processing-time first) and CTAs take them from an
// atomic queue. A CTA runs its item's batches alone: the same per-vertex
// forward and backward steps as the one-graph path (msbfs_body.cuh), with the
// CTA's warps striding over vertices and __syncthreads between levels, so
// no level ever waits on another CTA. Sources are the vertices in order,
// B = 32*W per batch.
//
// BC of a graph handled by one item is written by that CTA alone. A large
// graph is split into several items; each writes its own partial vector and
// the last item to finish (atomic arrival counter) adds the partials in item
// order into the graph's BC. Every result is deterministic.
//
// A graph deeper than the level capacity is flagged and left to the caller
// (bc_many_status reports it; the host re-runs it with bc_run).
#include <cuda_runtime.h>

#include <algorithm>
#include <numeric>
#include <string>
#include <vector>

#include "bc_internal.cuh"
#include "many.cuh"
#include "msbfs_body.cuh"

namespace bcgb {
namespace {

constexpr int kMBlock = 256;
constexpr int kMWarps = kMBlock / 32;
constexpr unsigned kFull = 0xffffffffu;

template <int W>
__global__ void __launch_bounds__(kMBlock, W >= 4 ? 3 : 4) k_many(const ManyParams p) {
    constexpr int B = 32 * W;
    __shared__ int s_item;
    __shared__ int s_last;
    __shared__ int32_t s_u[kMWarps][32];
    __shared__ uint32_t s_nz[kMWarps][32];
    __shared__ uint32_t s_w[kMWarps][32][W];  // per-lane words of a warp's 32 vertices
    __shared__ unsigned long long s_sum[4][B];  // per-source summaries of the running batch
    __shared__ __align__(16) uint64_t s_sig[kMWarps][W][32];  // counts of the vertex being finalized
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    uint64_t *sigma = p.sigma + (size_t)blockIdx.x * p.nmax * B;
    uint16_t *Sbuf = p.S + (size_t)blockIdx.x * 2 * p.nmax * B;
    float *cval = p.cval + (size_t)blockIdx.x * 2 * p.nmax * B;
    uint32_t *F = p.F + (size_t)blockIdx.x * p.Lcap * p.nmax * W;
    uint32_t *V = p.V + (size_t)blockIdx.x * 2 * p.nmax * W;
    uint32_t *ufr = p.ufr + (size_t)blockIdx.x * p.Lcap * p.nw32max;
    bool ovf = false;
    uint32_t arcs = 0;

    for (;;) {
        __syncthreads();
        if (tid == 0) s_item = (int)atomicAdd(p.queue, 1u);
        __syncthreads();
        const int it = s_item;
        if (it >= p.nitems) break;
        const ManyItem item = p.items[it];
        const ManyGraph gd = p.graphs[item.graph];
        const int n = gd.n;
        const size_t nW = (size_t)n * W;
        const int nw32 = (n + 31) / 32;
        const bool split = gd.nitems > 1;
        double *target = split ? p.partial + gd.part_off + (size_t)item.part * n : gd.bc;
        for (int v = tid; v < n; v += kMBlock) target[v] = 0.0;
        bool capped = false;

        for (int bt = item.batch_lo; bt < item.batch_hi && !capped; ++bt) {
            const int s0 = bt * B;
            const int nb = min(B, n - s0);
            for (size_t i = tid; i < nW; i += kMBlock) {
                F[i] = 0u;
                V[i] = 0u;
            }
            for (int i = tid; i < p.Lcap * nw32; i += kMBlock) ufr[i] = 0u;
            __syncthreads();
            const size_t nB = (size_t)n * B;
            for (int b = tid; b < nb; b += kMBlock) {  // d(s,s) = 0, sigma_s(s) = 1
                const int s = s0 + b;
                F[(size_t)s * W + (b >> 5)] |= 1u << (b & 31);  // one source per (s, b): no race
                atomicOr(ufr + (s >> 5), 1u << (s & 31));
                sigma[(size_t)s * B + b] = 1ull;
                // masked level-0 row: the word holding b (the only word read)
                for (int k = 32 * (b >> 5); k < 32 * (b >> 5) + 32; ++k) Sbuf[(size_t)s * B + k] = k == b ? 1 : 0;
            }
            __syncthreads();
            // forward levels
            int L = 0;
            bool wide = false;  // the current level has a count >= 2^16
            for (int l = 0;; ++l) {
                if (l + 1 >= p.Lcap) {
                    capped = true;
                    break;
                }
                const uint32_t *Fl = F + (size_t)l * nW;
                uint32_t *Fn = F + (size_t)(l + 1) * nW;
                const uint32_t *ufl = ufr + (size_t)l * nw32;
                uint32_t *ufn = ufr + (size_t)(l + 1) * nw32;
                const uint32_t *Vin = V + (size_t)(l & 1) * nW;
                uint32_t *Vout = V + (size_t)((l + 1) & 1) * nW;
                const uint16_t *Sl = Sbuf + (size_t)(l & 1) * nB;
                uint16_t *Sn = Sbuf + (size_t)((l + 1) & 1) * nB;
                bool produced = false, wide_next = false;
                // a warp checks its next 32 vertices at once (lane k: vertex
                // v0 + k * kMWarps), then works through the active ones
                for (int v0 = wib; v0 < n; v0 += 32 * kMWarps) {
                    const int vk = v0 + lane * kMWarps;
                    bool act = false;
                    __syncwarp();  // the previous group's reads of s_w are done
                    if (vk < n) {
                        uint32_t a[W], f[W];
                        body::load_row<W, false>(Vin + (size_t)vk * W, a);
                        body::load_row<W, false>(Fl + (size_t)vk * W, f);
                        uint32_t any = 0;
#pragma unroll
                        for (int j = 0; j < W; ++j) {
                            const uint32_t vis = a[j] | f[j];
                            Vout[(size_t)vk * W + j] = vis;
                            const uint32_t u = ~vis & body::valid_word(nb, j);
                            s_w[wib][lane][j] = u;
                            any |= u;
                        }
                        act = any != 0u;
                        if (!act)
#pragma unroll
                            for (int j = 0; j < W; ++j) Fn[(size_t)vk * W + j] = 0u;
                    }
                    unsigned todo = __ballot_sync(kFull, act);
                    __syncwarp();
                    while (todo) {
                        const int v = v0 + (__ffs(todo) - 1) * kMWarps;
                        uint32_t U[W];
#pragma unroll
                        for (int j = 0; j < W; ++j) U[j] = s_w[wib][__ffs(todo) - 1][j];
                        todo &= todo - 1;
                        uint64_t acc[W];
                        uint32_t nf[W];
#pragma unroll
                        for (int j = 0; j < W; ++j) {
                            acc[j] = 0ull;
                            nf[j] = 0u;
                        }
                        body::fwd_sum<W, false>(gd.col, gd.row_ptr[v], gd.row_ptr[v + 1], ufl, Fl, Sl, sigma, wide, false, U,
                                                s_u[wib], s_nz[wib], lane, acc, nf, ovf, arcs);
                        produced |= body::store_next<W, false>(sigma, Sn, Fn, ufn, v, acc, nf, lane, wide_next);
                    }
                }
                wide = __syncthreads_or(wide_next);
                if (!__syncthreads_or(produced)) {
                    L = l;
                    break;
                }
            }
            if (capped) break;
            if (gd.h_sigma) {
                // per-source summaries over tiles of 32 vertices x 32 sources:
                // lane k loads word j of vertex v0+k (reached set, frontier of
                // every level), a 32x32 bit transpose gives lane s the tile mask
                // of source 32j+s; popcounts give the distance terms, and
                // sigma_s(v) (v+1) is added over the reached vertices
                for (int i = tid; i < 4 * B; i += kMBlock) (&s_sum[0][0])[i] = 0ull;
                __syncthreads();
                const uint32_t *Vr = V + (size_t)((L + 1) & 1) * nW;  // visited through level L
                const int ntiles = (n + 31) / 32;
                for (int u = wib; u < ntiles * W; u += kMWarps) {
                    const int t = u / W, j = u % W;
                    const int v0 = 32 * t, vk = v0 + lane;
                    const bool in = vk < n;
                    const size_t wk = (size_t)(in ? vk : 0) * W + j;
                    unsigned long long hs = 0, hd = 0, ds = 0;
                    const uint32_t R = body::transpose32(in ? Vr[wk] : 0u, lane);
                    for (int l = 0; l <= L; ++l) {
                        const uint32_t T = body::transpose32(in ? F[(size_t)l * nW + wk] : 0u, lane);
                        const uint32_t c = (uint32_t)__popc(T);
                        const uint32_t ks = (uint32_t)__popc(T & 0xAAAAAAAAu) + 2u * (uint32_t)__popc(T & 0xCCCCCCCCu) +
                                            4u * (uint32_t)__popc(T & 0xF0F0F0F0u) +
                                            8u * (uint32_t)__popc(T & 0xFF00FF00u) +
                                            16u * (uint32_t)__popc(T & 0xFFFF0000u);
                        const unsigned long long vsum = (unsigned long long)c * (unsigned long long)(v0 + 1) + ks;
                        hd += (unsigned long long)(l + 1) * vsum;
                        ds += (unsigned long long)l * c;
                    }
                    const uint64_t *sg = sigma + (size_t)v0 * B + 32 * j + lane;
                    for (int k = 0; k < 32 && v0 + k < n; ++k)
                        if ((R >> k) & 1u) hs += sg[(size_t)k * B] * (unsigned long long)(v0 + k + 1);
                    atomicAdd(&s_sum[0][32 * j + lane], hs);
                    atomicAdd(&s_sum[1][32 * j + lane], hd);
                    atomicAdd(&s_sum[2][32 * j + lane], ds);
                    atomicAdd(&s_sum[3][32 * j + lane], (unsigned long long)__popc(R));
                }
                __syncthreads();
                for (int b = tid; b < nb; b += kMBlock) {  // one batch per source: plain stores
                    gd.h_sigma[s0 + b] = s_sum[0][b];
                    gd.h_dist[s0 + b] = s_sum[1][b];
                    gd.dist_sum[s0 + b] = (int64_t)s_sum[2][b];
                    gd.reach[s0 + b] = (int64_t)s_sum[3][b];
                }
            }
            // backward levels (Theorem 1.1), BC into this item's target
            for (int l = L; l >= 1; --l) {
                const uint32_t *Fl = F + (size_t)l * nW;
                const uint32_t *Fs = F + (size_t)(l + 1) * nW;
                const uint32_t *ufs = ufr + (size_t)(l + 1) * nw32;
                float *Cl = l > 1 ? cval + (size_t)(l & 1) * nB : nullptr;  // level-1 c values have no reader
                const float *Cs = cval + (size_t)((l + 1) & 1) * nB;
                for (int v0 = wib; v0 < n; v0 += 32 * kMWarps) {
                    const int vk = v0 + lane * kMWarps;
                    bool act = false;
                    __syncwarp();  // the previous group's reads of s_w are done
                    if (vk < n) {
                        uint32_t f[W];
                        body::load_row<W, false>(Fl + (size_t)vk * W, f);
                        uint32_t any = 0;
#pragma unroll
                        for (int j = 0; j < W; ++j) {
                            s_w[wib][lane][j] = f[j];
                            any |= f[j];
                        }
                        act = any != 0u;
                    }
                    unsigned todo = __ballot_sync(kFull, act);
                    __syncwarp();
                    while (todo) {
                        const int v = v0 + (__ffs(todo) - 1) * kMWarps;
                        uint32_t f[W];
#pragma unroll
                        for (int j = 0; j < W; ++j) f[j] = s_w[wib][__ffs(todo) - 1][j];
                        todo &= todo - 1;
                        // v's counts (the words with a level-l source) go to
                        // shared memory while its neighbours are scanned
#pragma unroll
                        for (int j = 0; j < W; ++j)
                            if (f[j] != 0u) {
                                const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&s_sig[wib][j][lane]);
                                asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst),
                                             "l"(sigma + (size_t)v * B + 32 * j + lane)
                                             : "memory");
                            }
                        asm volatile("cp.async.commit_group;" ::: "memory");
                        float S[W];
#pragma unroll
                        for (int j = 0; j < W; ++j) S[j] = 0.0f;
                        body::bwd_sum<W, false>(gd.col, gd.row_ptr[v], gd.row_ptr[v + 1], ufs, Fs, Cs, f, s_u[wib], s_nz[wib], lane, S);
                        asm volatile("cp.async.wait_group 0;" ::: "memory");
                        __syncwarp();
                        body::finalize_dep<W, false>(sigma, Cl, target, v, f, S, lane, &s_sig[wib][0][0]);
                        __syncwarp();  // the next vertex's copies overwrite s_sig
                    }
                }
                __syncthreads();
            }
        }
        if (capped && tid == 0) p.capped[item.graph] = 1u;
        if (!split) continue;
        // last item of a split graph adds the partials in item order
        __threadfence();
        __syncthreads();
        if (tid == 0) s_last = atomicAdd(p.arrive + item.graph, 1u) == (unsigned)(gd.nitems - 1);
        __syncthreads();
        if (!s_last) continue;
        __threadfence();
        const double *part = p.partial + gd.part_off;
        for (int v = tid; v < n; v += kMBlock) {
            double acc = 0.0;
            for (int q = 0; q < gd.nitems; ++q) acc += __ldcg(part + (size_t)q * n + v);
            gd.bc[v] = acc;
        }
        if (tid == 0) p.arrive[item.graph] = 0u;
    }
    const bool wovf = __any_sync(kFull, ovf);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) arcs += __shfl_xor_sync(kFull, arcs, off);
    if (lane == 0) {
        if (wovf) atomicOr(&p.ctl->status, BC_STATUS_SIGMA_OVERFLOW);
        if (arcs) atomicAdd(&p.ctl->dag_arcs, (unsigned long long)arcs);
    }
}

}  // namespace

int many_blocks_per_sm(int W) {
    int nb = 0;
    switch (W) {
        case 1: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_many<1>, kMBlock, 0); break;
        case 2: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_many<2>, kMBlock, 0); break;
        case 4: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_many<4>, kMBlock, 0); break;
        default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_many<8>, kMBlock, 0); break;
    }
    return nb < 1 ? 1 : nb;
}

void many_launch(int W, const ManyParams &p, int grid, cudaStream_t st) {
    switch (W) {
        case 1: k_many<1><<<grid, kMBlock, 0, st>>>(p); break;
        case 2: k_many<2><<<grid, kMBlock, 0, st>>>(p); break;
        case 4: k_many<4><<<grid, kMBlock, 0, st>>>(p); break;
        default: k_many<8><<<grid, kMBlock, 0, st>>>(p); break;
    }
}

}  // namespace bcgb
