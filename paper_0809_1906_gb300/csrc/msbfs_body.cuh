// msbfs_body.cuh -- per-vertex steps of the multi-source level sweep, shared
// by the one-graph kernels (msbfs.cu) and the many-graph persistent kernel
// (many.cu).
//
// A batch holds B = 32*W sources; every per-vertex row (sigma, c, frontier
// words) is contiguous. A warp owns a vertex v (or a chunk of its arcs) and
// walks v's arcs 32 at a time:
//   probe    lane k takes arc k of the chunk: neighbour u_k, one bit of the
//            union-frontier bitmap (is u_k in any source's frontier?), then
//            u_k's W frontier words ANDed with the sources v still wants;
//   walk     per source word j, a 5-step shuffle transposes the 32 x 32 bit
//            block (candidate k, source 32j+i) so that lane i holds the
//            candidates that matter to its own source; each lane then reads
//            only those neighbours' entries and keeps its sums in registers.
// Every lane does useful work for its own source, whatever the density of
// the masks, and no atomics touch the per-source sums.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace bcgb {
namespace body {

constexpr unsigned kFull = 0xffffffffu;

// Mask of valid sources in word j of a batch with nb sources.
__device__ __forceinline__ uint32_t valid_word(int nb, int j) {
    const int lo = 32 * j;
    if (nb >= lo + 32) return 0xffffffffu;
    if (nb <= lo) return 0u;
    return (1u << (nb - lo)) - 1u;
}

template <int W>
__device__ __forceinline__ void load_row(const uint32_t *__restrict__ p, uint32_t (&w)[W]) {
    if constexpr (W % 4 == 0) {
        const uint4 *q = reinterpret_cast<const uint4 *>(p);
#pragma unroll
        for (int i = 0; i < W / 4; ++i) {
            const uint4 t = __ldg(q + i);
            w[4 * i] = t.x;
            w[4 * i + 1] = t.y;
            w[4 * i + 2] = t.z;
            w[4 * i + 3] = t.w;
        }
    } else if constexpr (W % 2 == 0) {
        const uint2 *q = reinterpret_cast<const uint2 *>(p);
#pragma unroll
        for (int i = 0; i < W / 2; ++i) {
            const uint2 t = __ldg(q + i);
            w[2 * i] = t.x;
            w[2 * i + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < W; ++i) w[i] = __ldg(p + i);
    }
}

// Warp-wide 32x32 bit transpose: lane k holds row k; returns column `lane`
// (bit k of the result = bit `lane` of lane k's input). Five exchange steps,
// each swapping the off-diagonal s x s blocks of every 2s x 2s block.
__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane) {
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const uint32_t M = s == 16 ? 0x0000FFFFu : s == 8 ? 0x00FF00FFu : s == 4 ? 0x0F0F0F0Fu
                         : s == 2 ? 0x33333333u : 0x55555555u;
        const uint32_t y = __shfl_xor_sync(kFull, x, s);
        x = (lane & s) ? ((x & ~M) | ((y >> s) & M)) : ((x & M) | ((y & M) << s));
    }
    return x;
}

// One 32-arc chunk: lane k gets arc e (if e < end), its neighbour u_k (stored
// in s_u[k]) and masks m_k[j] = frontier words of u_k AND want[j] (zero for
// arcs that cannot contribute). Returns the ballot of contributing lanes.
template <int W>
__device__ __forceinline__ unsigned probe_chunk(const int32_t *__restrict__ col, int e, int end,
                                                const uint32_t *__restrict__ ufr, const uint32_t *__restrict__ Fx,
                                                const uint32_t (&want)[W], uint32_t (&m)[W], int32_t *s_u,
                                                int lane) {
    int u = 0;
    bool cand = false;
#pragma unroll
    for (int j = 0; j < W; ++j) m[j] = 0u;
    if (e < end) {
        u = __ldg(col + e);
        if ((__ldg(ufr + (u >> 5)) >> (u & 31)) & 1u) {
            uint32_t fu[W];
            load_row<W>(Fx + (size_t)u * W, fu);
            uint32_t any = 0;
#pragma unroll
            for (int j = 0; j < W; ++j) {
                m[j] = fu[j] & want[j];
                any |= m[j];
            }
            cand = any != 0u;
        }
    }
    s_u[lane] = u;
    __syncwarp();
    return __ballot_sync(kFull, cand);
}

// Forward sums over arcs [beg, end) of v for level l -> l+1: for source
// s = 32j + lane, acc[j] += sigma_s(u) over neighbours u with d(s,u) = l and
// v unvisited by s (U); nf[j] collects the sources that reach v. Exact
// uint64 adds; ovf records a carry out of bit 63. arcs counts predecessor
// relations (lane-local).
template <int W>
__device__ __forceinline__ void fwd_sum(const int32_t *__restrict__ col, int beg, int end,
                                        const uint32_t *__restrict__ ufl, const uint32_t *__restrict__ Fl,
                                        const uint64_t *__restrict__ sigma, const uint32_t (&U)[W],
                                        int32_t *s_u, int lane, uint64_t (&acc)[W], uint32_t (&nf)[W],
                                        bool &ovf, uint32_t &arcs) {
    constexpr int B = 32 * W;
    for (int e0 = beg; e0 < end; e0 += 32) {
        uint32_t m[W];
        const unsigned bal = probe_chunk<W>(col, e0 + lane, end, ufl, Fl, U, m, s_u, lane);
        if (bal) {
            // t[j]: the chunk's neighbours that are predecessors for source 32j + lane
            uint32_t t[W];
#pragma unroll
            for (int j = 0; j < W; ++j) {
                t[j] = __ballot_sync(kFull, m[j] != 0u) ? transpose32(m[j], lane) : 0u;
                nf[j] |= __ballot_sync(kFull, t[j] != 0u);
                arcs += __popc(t[j]);
            }
            // drain one candidate of every word per step: up to W independent loads in flight
            for (;;) {
                uint32_t left = 0;
                uint64_t x[W];
#pragma unroll
                for (int j = 0; j < W; ++j) {
                    x[j] = 0ull;
                    if (t[j]) {
                        const int k = __ffs(t[j]) - 1;
                        t[j] &= t[j] - 1;
                        x[j] = __ldg(sigma + (size_t)s_u[k] * B + 32 * j + lane);
                    }
                    left |= t[j];
                }
#pragma unroll
                for (int j = 0; j < W; ++j) {
                    const uint64_t y = acc[j] + x[j];
                    ovf |= y < x[j];
                    acc[j] = y;
                }
                if (!left) break;
            }
        }
        __syncwarp();
    }
}

// Backward sums over arcs [beg, end) of v at level l: for source s = 32j +
// lane with d(s,v) = l (f), S[j] += c_s(w) over neighbours w with
// d(s,w) = l+1, i.e. over the w with v in P_s(w).
template <int W>
__device__ __forceinline__ void bwd_sum(const int32_t *__restrict__ col, int beg, int end,
                                        const uint32_t *__restrict__ ufs, const uint32_t *__restrict__ Fs,
                                        const float *__restrict__ cval, const uint32_t (&f)[W], int32_t *s_u,
                                        int lane, float (&S)[W]) {
    constexpr int B = 32 * W;
    for (int e0 = beg; e0 < end; e0 += 32) {
        uint32_t m[W];
        const unsigned bal = probe_chunk<W>(col, e0 + lane, end, ufs, Fs, f, m, s_u, lane);
        if (bal) {
            uint32_t t[W];
#pragma unroll
            for (int j = 0; j < W; ++j) t[j] = __ballot_sync(kFull, m[j] != 0u) ? transpose32(m[j], lane) : 0u;
            for (;;) {
                uint32_t left = 0;
                float x[W];
#pragma unroll
                for (int j = 0; j < W; ++j) {
                    x[j] = 0.0f;
                    if (t[j]) {
                        const int k = __ffs(t[j]) - 1;
                        t[j] &= t[j] - 1;
                        x[j] = __ldg(cval + (size_t)s_u[k] * B + 32 * j + lane);
                    }
                    left |= t[j];
                }
#pragma unroll
                for (int j = 0; j < W; ++j) S[j] += x[j];
                if (!left) break;
            }
        }
        __syncwarp();
    }
}

// Store sigma and the new frontier words of v (its level-(l+1) sums are final).
template <int W>
__device__ __forceinline__ bool store_next(uint64_t *sigma, uint32_t *Fn, uint32_t *ufn, int v,
                                           const uint64_t (&acc)[W], const uint32_t (&nf)[W], int lane) {
    constexpr int B = 32 * W;
    uint32_t any = 0;
#pragma unroll
    for (int j = 0; j < W; ++j) {
        any |= nf[j];
        if (lane == j) Fn[(size_t)v * W + j] = nf[j];
        if ((nf[j] >> lane) & 1u) sigma[(size_t)v * B + 32 * j + lane] = acc[j];
    }
    if (any != 0 && lane == 0) atomicOr(ufn + (v >> 5), 1u << (v & 31));
    return any != 0;
}

// Theorem 1.1 at v for the sources in f: delta = sigma * S,
// c = (1 + delta) / sigma (FP32), and the FP64 sum of delta over the batch
// (fixed butterfly order) added to bc[v]. v at level >= 1, so never a source.
template <int W>
__device__ __forceinline__ void finalize_dep(const uint64_t *sigma, float *cval, double *bc, int v,
                                             const uint32_t (&f)[W], const float (&S)[W], int lane) {
    constexpr int B = 32 * W;
    double sum = 0.0;
#pragma unroll
    for (int j = 0; j < W; ++j) {
        if ((f[j] >> lane) & 1u) {
            const size_t idx = (size_t)v * B + 32 * j + lane;
            const float sg = __ull2float_rn(sigma[idx]);
            const float d = sg * S[j];    // delta_s*(v) = sigma_s(v) * sum_w c_s(w)
            cval[idx] = (1.0f + d) / sg;  // c_s(v) for the level above
            sum += (double)d;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(kFull, sum, off);
    if (lane == 0) bc[v] += sum;
}

}  // namespace body
}  // namespace bcgb
