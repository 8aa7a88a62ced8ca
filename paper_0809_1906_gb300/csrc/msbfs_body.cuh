// msbfs_body.cuh -- per-vertex steps of the multi-source level sweep, shared
// by the one-graph kernels (msbfs.cu) and the many-graph persistent kernel
// (many.cu).
//
// A batch holds B = 32*W sources; every per-vertex row (sigma, c, frontier
// words) is contiguous, lane i of a warp owns sources 32j + i (j < W). Beside
// the permanent uint64 sigma array, each level keeps *masked rows*: row v of
// level l holds sigma_s(v) (forward, as uint16) or c_s(v) (backward, FP32)
// for the sources s with d(s,v) = l and 0 for every other source: c rows in
// two buffers alternating by level parity, sigma rows in one buffer per level
// (or two by parity when that would take too much memory; the many-graph
// kernel). A level whose counts do not all fit in 16 bits is marked "wide";
// the next level then reads the permanent uint64 sigma under per-source masks
// instead (exact either way). A warp owns a vertex v (or a chunk of its arcs)
// and walks v's arcs 32 at a time:
//   probe  lane k takes arc k of the chunk: neighbour u_k, one bit of the
//          union-frontier bitmap (is u_k in any source's frontier?), then
//          u_k's W frontier words ANDed with the sources v cares about; arcs
//          whose AND is empty are dropped;
//   add    for each remaining neighbour the warp adds the words of its
//          masked row that can contribute to its W per-lane sums, with no
//          per-source test: within such a word the masked row is zero
//          wherever u_k does not contribute.
// The frontier words of v come from an OR-reduction of the probe masks.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "rowstage.cuh"

namespace bcgb {
namespace body {

// A warp's row stage (rowstage.cuh): buffer (stage::kFwdStageBytes forward,
// stage::kBwdStageBytes backward), its
// mbarrier and phase, per-slot word masks (backward), and the failure flag
// set when a wait gave up (the warp then stops adding rows).
struct WarpStage {
    uint8_t *buf;
    uint64_t *bar;
    uint32_t *qz;
    uint32_t phase;
    bool fail;
    // read only by the sweeps instantiated with HOOK (a run that sets a wait
    // bound or the timeout test hook): bits 7..0, bytes each round expects
    // beyond its copies, which no copy delivers (the test hook; 0 otherwise);
    // bits 31..8, the bound on each wait in microseconds (0: stage::kWaitNs)
    uint32_t wctl;
};

// wctl of a warp stage from a wait bound (ns, 0 = default) and held bytes.
__host__ __device__ __forceinline__ uint32_t stage_wctl(uint64_t wait_ns, uint32_t hold) {
    uint64_t us = wait_ns / 1000ull;
    if (wait_ns && us == 0) us = 1;
    if (us > 0xffffffull) us = 0xffffffull;
    return (uint32_t)(us << 8) | (hold & 0xffu);
}
__device__ __forceinline__ uint32_t stage_hold(const WarpStage *ws) { return ws->wctl & 0xffu; }
__device__ __forceinline__ uint32_t stage_limit_us(const WarpStage *ws) { return ws->wctl >> 8; }

// A staged round's wait gave up: release the held bytes, then wait (bounded)
// for the copies this warp already issued, so that no copy lands in the stage
// after the warp stops using it; the warp stages nothing more.
__device__ __forceinline__ void give_up(WarpStage *ws, uint32_t parity, int lane, uint32_t hold) {
    if (lane == 0 && hold) stage::complete_tx(ws->bar, hold);
    __syncwarp();
    stage::wait(ws->bar, parity);
    __syncwarp();
    ws->fail = true;
}

constexpr unsigned kFull = 0xffffffffu;

// Loads of data written by an earlier kernel launch may take the read-only
// (non-coherent) path; data written earlier in the same launch (the
// many-graph kernel runs every level in one launch) must use coherent loads.
template <bool NC, class T>
__device__ __forceinline__ T ldx(const T *p) {
    if constexpr (NC)
        return __ldg(p);
    else
        return *p;
}

// Mask of valid sources in word j of a batch with nb sources.
__device__ __forceinline__ uint32_t valid_word(int nb, int j) {
    const int lo = 32 * j;
    if (nb >= lo + 32) return 0xffffffffu;
    if (nb <= lo) return 0u;
    return (1u << (nb - lo)) - 1u;
}

template <int W, bool NC = true>
__device__ __forceinline__ void load_row(const uint32_t *__restrict__ p, uint32_t (&w)[W]) {
    if constexpr (W % 4 == 0) {
        const uint4 *q = reinterpret_cast<const uint4 *>(p);
#pragma unroll
        for (int i = 0; i < W / 4; ++i) {
            const uint4 t = ldx<NC>(q + i);
            w[4 * i] = t.x;
            w[4 * i + 1] = t.y;
            w[4 * i + 2] = t.z;
            w[4 * i + 3] = t.w;
        }
    } else if constexpr (W % 2 == 0) {
        const uint2 *q = reinterpret_cast<const uint2 *>(p);
#pragma unroll
        for (int i = 0; i < W / 2; ++i) {
            const uint2 t = ldx<NC>(q + i);
            w[2 * i] = t.x;
            w[2 * i + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < W; ++i) w[i] = ldx<NC>(p + i);
    }
}

// Warp-wide 32x32 bit transpose: lane k holds row k; returns column `lane`
// (bit k of the result = bit `lane` of lane k's input). Five exchange steps,
// each swapping the off-diagonal s x s blocks of every 2s x 2s block with
// partner lane ^ s: the partner's word rotated by s (towards the high bits
// for lanes with bit s clear, the low bits otherwise) supplies exactly the
// bits outside this lane's kept mask, so a step is a shuffle, a rotate and a
// bitwise select.
__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane) {
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const uint32_t M = s == 16 ? 0x0000FFFFu : s == 8 ? 0x00FF00FFu : s == 4 ? 0x0F0F0F0Fu
                         : s == 2 ? 0x33333333u : 0x55555555u;
        const bool hi = (lane & s) != 0;
        const uint32_t keep = hi ? ~M : M;
        const uint32_t y = __shfl_xor_sync(kFull, x, s);
        const uint32_t a = __funnelshift_l(y, y, hi ? 32 - s : s);
        x = (x & keep) | (a & ~keep);
    }
    return x;
}

// Packed view of a staged row: lane l reads the W consecutive entries of
// sources W*l .. W*l+W-1 with one vector load (its sources all lie in word
// (W*l)/32 of the row). The adders sum in this view and hand the sums back
// in the lane-owns-32j+lane view through shared memory.
template <int W>
__device__ __forceinline__ void lds_packed(const uint16_t *p, uint32_t (&x)[(W + 1) / 2]) {
    if constexpr (W == 8) {
        const uint4 t = *reinterpret_cast<const uint4 *>(p);
        x[0] = t.x;
        x[1] = t.y;
        x[2] = t.z;
        x[3] = t.w;
    } else if constexpr (W == 4) {
        const uint2 t = *reinterpret_cast<const uint2 *>(p);
        x[0] = t.x;
        x[1] = t.y;
    } else if constexpr (W == 2) {
        x[0] = *reinterpret_cast<const uint32_t *>(p);
    } else {
        x[0] = *p;
    }
}
template <int W>
__device__ __forceinline__ void lds_packed(const float *p, float (&x)[W]) {
    if constexpr (W >= 4) {
#pragma unroll
        for (int i = 0; i < W / 4; ++i) {
            const float4 t = reinterpret_cast<const float4 *>(p)[i];
            x[4 * i] = t.x;
            x[4 * i + 1] = t.y;
            x[4 * i + 2] = t.z;
            x[4 * i + 3] = t.w;
        }
    } else if constexpr (W == 2) {
        const float2 t = *reinterpret_cast<const float2 *>(p);
        x[0] = t.x;
        x[1] = t.y;
    } else {
        x[0] = *p;
    }
}
__device__ __forceinline__ uint32_t as_bits(uint32_t x) { return x; }
__device__ __forceinline__ uint32_t as_bits(float x) { return __float_as_uint(x); }

// Lane l stores its W packed values at p[W*l ..]; after the warp synchronises,
// lane l reads entries 32j + l.
template <int W, class T>
__device__ __forceinline__ void unpack_lanes(T *p, const T (&x)[W], T (&out)[W], int lane) {
    T *q = p + W * lane;
    if constexpr (W >= 4) {
#pragma unroll
        for (int i = 0; i < W / 4; ++i) {
            uint4 t;
            t.x = as_bits(x[4 * i]);
            t.y = as_bits(x[4 * i + 1]);
            t.z = as_bits(x[4 * i + 2]);
            t.w = as_bits(x[4 * i + 3]);
            reinterpret_cast<uint4 *>(q)[i] = t;
        }
    } else {
#pragma unroll
        for (int i = 0; i < W; ++i) q[i] = x[i];
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < W; ++j) out[j] = p[32 * j + lane];
    __syncwarp();
    // the stage is written by bulk copies next: order these generic accesses first
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One 32-arc chunk: lane k gets arc e (if e < end), its neighbour u_k (stored
// in s_u[k]) and masks m_k[j] = frontier words of u_k AND want[j] (zero for
// arcs that cannot contribute); s_nz[k] gets the W-bit set of non-zero words
// of m_k, so the adders load only the words that can contribute.
// Returns the ballot of contributing lanes; u and nz are lane k's own
// neighbour and word set. ufr (the union of the level's frontiers, one bit
// per vertex) skips the row loads of neighbours in no frontier; null when the
// level's frontier is wide enough that most neighbours pass.
template <int W, bool NC>
__device__ __forceinline__ unsigned probe_chunk(const int32_t *__restrict__ col, int e, int end,
                                                const uint32_t *__restrict__ ufr, const uint32_t *__restrict__ Fx,
                                                const uint32_t (&want)[W], uint32_t (&m)[W], int32_t *s_u,
                                                uint32_t *s_nz, int lane, int &u, uint32_t &nz) {
    u = 0;
    nz = 0;
#pragma unroll
    for (int j = 0; j < W; ++j) m[j] = 0u;
    if (e < end) {
        u = __ldg(col + e);
        if (ufr == nullptr || ((ldx<NC>(ufr + (u >> 5)) >> (u & 31)) & 1u)) {
            uint32_t fu[W];
            load_row<W, NC>(Fx + (size_t)u * W, fu);
#pragma unroll
            for (int j = 0; j < W; ++j) {
                m[j] = fu[j] & want[j];
                nz |= (m[j] != 0u ? 1u : 0u) << j;
            }
        }
    }
    s_u[lane] = u;
    s_nz[lane] = nz;
    __syncwarp();
    return __ballot_sync(kFull, nz != 0u);
}

// Forward sums over arcs [beg, end) of v for level l -> l+1: for source
// s = 32j + lane, acc[j] += sigma_s(u) over the neighbours u in P_s(v), for
// every s still unvisited at v (U); other entries of acc are discarded by the
// caller. Narrow levels add the masked uint16 rows Sl (zero wherever u is not
// a predecessor); a wide level reads sigma under the per-source masks; a level
// whose counts are all 1 (ones) just counts predecessors. nf[j]
// gets the sources reaching v; exact uint64 sums, ovf flags a carry out of
// bit 63; arcs counts predecessor relations (lane-local).
template <int W, bool NC = true, bool STAGED = false, bool HOOK = false>
__device__ __forceinline__ void fwd_sum(const int32_t *__restrict__ col, int beg, int end,
                                        const uint32_t *__restrict__ ufl, const uint32_t *__restrict__ Fl,
                                        const uint16_t *__restrict__ Sl, const uint64_t *__restrict__ sigma,
                                        bool wide, bool ones, const uint32_t (&U)[W], int32_t *s_u, uint32_t *s_nz,
                                        int lane, uint64_t (&acc)[W], uint32_t (&nf)[W], bool &ovf, uint32_t &arcs,
                                        WarpStage *ws = nullptr) {
    constexpr int B = 32 * W;
    for (int e0 = beg; e0 < end; e0 += 32) {
        uint32_t m[W];
        int u;
        uint32_t nz;
        unsigned bal = probe_chunk<W, NC>(col, e0 + lane, end, ufl, Fl, U, m, s_u, s_nz, lane, u, nz);
        if (!bal) continue;
#pragma unroll
        for (int j = 0; j < W; ++j) {
            nf[j] |= __reduce_or_sync(kFull, m[j]);
            arcs += __popc(m[j]);
        }
        if (ones) {
            // every count of this level is 1 (level 1: one shortest path from
            // s to each neighbour of s), so the sum is the number of
            // predecessors: per source, a column count of the chunk's masks
#pragma unroll
            for (int j = 0; j < W; ++j)
                if (__any_sync(kFull, m[j] != 0u)) acc[j] += (uint64_t)__popc(transpose32(m[j], lane));
        } else if (STAGED && !wide) {
            // rounds of up to R rows: each contributing lane copies the span of
            // its neighbour's masked row from the first to the last word that
            // can contribute into slot `rank` of the stage; the warp waits
            // once and adds the contributing words of the slots (at most 32
            // values below 2^16 per chunk: 32-bit sums are exact)
            constexpr int RB = 2 * B;
            constexpr int R = (int)stage::kFwdStageBytes / RB < 32 ? (int)stage::kFwdStageBytes / RB : 32;
            constexpr int P = (W + 1) / 2;  // packed 32-bit words per lane
            const uint16_t *st = reinterpret_cast<const uint16_t *>(ws->buf);
            const int jl = (W * lane) >> 5;  // the row word holding this lane's sources
            // X: wrapping sums of the packed words; H: sums of their high
            // halves. The low-half sums are X - (H << 16), exact while below 2^32.
            uint32_t X[P], H[P];
#pragma unroll
            for (int i = 0; i < P; ++i) X[i] = H[i] = 0u;
            while (bal && !ws->fail) {
                const int rank = __popc(bal & ((1u << lane) - 1u));
                const bool go = ((bal >> lane) & 1u) && rank < R;
                const unsigned take = __ballot_sync(kFull, go);
                const int nq = __popc(take);
                const int lo = __ffs(nz) - 1, hi = 31 - __clz(nz);
                const uint32_t bytes = go ? 64u * (uint32_t)(hi - lo + 1) : 0u;
                const uint32_t tot = __reduce_add_sync(kFull, bytes);
                if (go) ws->qz[rank] = nz;
                if (lane == 0) stage::expect_tx(ws->bar, tot + (HOOK ? stage_hold(ws) : 0u));
                __syncwarp();
                if (go) stage::copy(ws->buf + rank * RB + 64 * lo, Sl + (size_t)u * B + 32 * lo, bytes, ws->bar);
                const uint32_t ph = ws->phase;
                const bool ok = stage::wait(ws->bar, ph, HOOK ? stage_limit_us(ws) : 0u);
                ws->phase ^= 1u;
                if (!__all_sync(kFull, ok)) {
                    give_up(ws, ph, lane, HOOK ? stage_hold(ws) : 0u);
                    break;
                }
#pragma unroll 4
                for (int q = 0; q < nq; ++q) {
                    if ((ws->qz[q] >> jl) & 1u) {
                        uint32_t x[P];
                        lds_packed<W>(st + q * B + W * lane, x);
#pragma unroll
                        for (int i = 0; i < P; ++i) {
                            X[i] += x[i];
                            H[i] += x[i] >> 16;
                        }
                    }
                }
                __syncwarp();
                bal &= ~take;
            }
            uint32_t sums[W], a32[W];
#pragma unroll
            for (int i = 0; i < P; ++i) {
                sums[2 * i] = X[i] - (H[i] << 16);
                if (2 * i + 1 < W) sums[2 * i + 1] = H[i];
            }
            unpack_lanes<W>(reinterpret_cast<uint32_t *>(ws->buf), sums, a32, lane);
#pragma unroll
            for (int j = 0; j < W; ++j) {
                const uint64_t y = acc[j] + (uint64_t)a32[j];
                ovf |= y < acc[j];
                acc[j] = y;
            }
        } else if (!wide) {
            // two neighbours per step: up to 2W independent coalesced loads in
            // flight, only the words that can contribute (the many-graph kernel:
            // its batch state does not fit L2, so every word skipped is DRAM
            // traffic saved; 411 -> 382 ms on the 2000-graph set). At most 32
            // values below 2^16 per chunk: 32-bit sums are exact and are folded
            // into the 64-bit ones once per chunk.
            const uint16_t *base = Sl + lane;
            uint32_t a32[W];
#pragma unroll
            for (int j = 0; j < W; ++j) a32[j] = 0u;
            while (bal) {
                const int k0 = __ffs(bal) - 1;
                bal &= bal - 1;
                const int k1 = bal ? __ffs(bal) - 1 : -1;
                if (k1 >= 0) bal &= bal - 1;
                const uint16_t *r0 = base + (size_t)s_u[k0] * B;
                const uint16_t *r1 = base + (size_t)s_u[k1 >= 0 ? k1 : k0] * B;
                const uint32_t z0 = s_nz[k0], z1 = k1 >= 0 ? s_nz[k1] : 0u;
                uint32_t x0[W], x1[W];
#pragma unroll
                for (int j = 0; j < W; ++j) {
                    x0[j] = ((z0 >> j) & 1u) ? (uint32_t)ldx<NC>(r0 + 32 * j) : 0u;
                    x1[j] = ((z1 >> j) & 1u) ? (uint32_t)ldx<NC>(r1 + 32 * j) : 0u;
                }
#pragma unroll
                for (int j = 0; j < W; ++j) a32[j] += x0[j] + x1[j];
            }
#pragma unroll
            for (int j = 0; j < W; ++j) {
                const uint64_t y = acc[j] + (uint64_t)a32[j];
                ovf |= y < acc[j];
                acc[j] = y;
            }
        } else {
            const uint64_t *base = sigma + lane;
            while (bal) {
                const int k = __ffs(bal) - 1;
                bal &= bal - 1;
                const uint64_t *row = base + (size_t)s_u[k] * B;
#pragma unroll
                for (int j = 0; j < W; ++j) {
                    const uint32_t mk = __shfl_sync(kFull, m[j], k);
                    if ((mk >> lane) & 1u) {
                        const uint64_t x = ldx<NC>(row + 32 * j);
                        const uint64_t y = acc[j] + x;
                        ovf |= y < x;
                        acc[j] = y;
                    }
                }
            }
        }
        __syncwarp();
    }
}

// Backward sums over arcs [beg, end) of v at level l: for source s = 32j +
// lane with d(s,v) = l (f), S[j] += Cs[w][s] over the neighbours w whose
// level-(l+1) frontier meets f. Cs is the masked level-(l+1) c buffer, so
// for s in f this is the sum of c_s(w) over the w with v in P_s(w).
// Sources of a vertex at most which the backward takes the sparse-source
// form (below).
constexpr int kSparseSrc = 8;

// Sparse-source form of the backward sums, for a vertex v at level l for at
// most kSparseSrc sources (their positions in pos[], ascending): lane k adds
// c_s(w_k) of its own arc's neighbour for each listed source s with w_k in
// P_s's next level (one 4-byte load each), and each source's partial sums
// are added across the warp once at the end. For such vertices this reads a
// few values per arc instead of whole row words.
template <int W, bool NC>
__device__ __forceinline__ void bwd_sum_sparse(const int32_t *__restrict__ col, int beg, int end,
                                               const uint32_t *__restrict__ ufs, const uint32_t *__restrict__ Fs,
                                               const float *__restrict__ Cs, const uint32_t (&f)[W], int32_t *s_u,
                                               uint32_t *s_nz, int lane, float (&S)[W], const uint32_t *pos,
                                               int nsrc) {
    constexpr int B = 32 * W;
    float P[kSparseSrc];
#pragma unroll
    for (int i = 0; i < kSparseSrc; ++i) P[i] = 0.0f;
    for (int e0 = beg; e0 < end; e0 += 32) {
        uint32_t m[W];
        int u;
        uint32_t nz;
        const unsigned bal = probe_chunk<W, NC>(col, e0 + lane, end, ufs, Fs, f, m, s_u, s_nz, lane, u, nz);
        if (bal) {
            // bit i of cm: the arc contributes to listed source i (f's set
            // bits in order, word by word)
            uint32_t cm = 0;
            int i = 0;
#pragma unroll
            for (int j = 0; j < W; ++j) {
                uint32_t x = f[j];
                const uint32_t mw = m[j];
                while (x) {
                    const int b = __ffs(x) - 1;
                    x &= x - 1;
                    cm |= ((mw >> b) & 1u) << i;
                    ++i;
                }
            }
            const float *row = Cs + (size_t)u * B;
#pragma unroll
            for (int k = 0; k < kSparseSrc; ++k)
                if ((cm >> k) & 1u) P[k] += ldx<NC>(row + pos[k]);
        }
        __syncwarp();
    }
#pragma unroll
    for (int i = 0; i < kSparseSrc; ++i) {
        if (i < nsrc) {
            float t = P[i];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(kFull, t, off);
            const uint32_t p = pos[i];
#pragma unroll
            for (int j = 0; j < W; ++j)
                if (p == 32u * j + (uint32_t)lane) S[j] += t;
        }
    }
}

template <int W, bool NC = true, bool STAGED = false, bool HOOK = false>
__device__ __forceinline__ void bwd_sum(const int32_t *__restrict__ col, int beg, int end,
                                        const uint32_t *__restrict__ ufs, const uint32_t *__restrict__ Fs,
                                        const float *__restrict__ Cs, const uint32_t (&f)[W], int32_t *s_u,
                                        uint32_t *s_nz, int lane, float (&S)[W], WarpStage *ws = nullptr) {
    constexpr int B = 32 * W;
    if constexpr (STAGED) {
        int nsrc = 0;
#pragma unroll
        for (int j = 0; j < W; ++j) nsrc += __popc(f[j]);
        if (nsrc <= kSparseSrc) {
            // list the sources in the stage's slot-mask array (free in this form)
            if (lane == 0) {
                int k = 0;
#pragma unroll
                for (int j = 0; j < W; ++j) {
                    uint32_t x = f[j];
                    while (x) {
                        ws->qz[k++] = 32u * j + (uint32_t)(__ffs(x) - 1);
                        x &= x - 1;
                    }
                }
            }
            __syncwarp();
            bwd_sum_sparse<W, NC>(col, beg, end, ufs, Fs, Cs, f, s_u, s_nz, lane, S, ws->qz, nsrc);
            __syncwarp();
            return;
        }
    }
    float Sp[W];  // staged sums, packed view (lane owns sources W*lane + t)
#pragma unroll
    for (int t = 0; t < W; ++t) Sp[t] = 0.0f;
    bool staged = false;
    for (int e0 = beg; e0 < end; e0 += 32) {
        uint32_t m[W];
        int u;
        uint32_t nz;
        unsigned bal = probe_chunk<W, NC>(col, e0 + lane, end, ufs, Fs, f, m, s_u, s_nz, lane, u, nz);
        if constexpr (STAGED) {
            // rounds of up to R rows; a lane copies the span of its
            // neighbour's c row from the first to the last word that can
            // contribute, and the adder takes only the contributing words
            constexpr int RB = 4 * B;
            constexpr int R = (int)stage::kBwdStageBytes / RB < 32 ? (int)stage::kBwdStageBytes / RB : 32;
            const float *st = reinterpret_cast<const float *>(ws->buf);
            const int jl = (W * lane) >> 5;  // the row word holding this lane's sources
            while (bal && !ws->fail) {
                const int rank = __popc(bal & ((1u << lane) - 1u));
                const bool go = ((bal >> lane) & 1u) && rank < R;
                const unsigned take = __ballot_sync(kFull, go);
                const int nq = __popc(take);
                const int lo = __ffs(nz) - 1, hi = 31 - __clz(nz);
                const uint32_t bytes = go ? 128u * (uint32_t)(hi - lo + 1) : 0u;
                const uint32_t tot = __reduce_add_sync(kFull, bytes);
                if (go) ws->qz[rank] = nz;
                if (lane == 0) stage::expect_tx(ws->bar, tot + (HOOK ? stage_hold(ws) : 0u));
                __syncwarp();
                if (go) stage::copy(ws->buf + rank * RB + 128 * lo, Cs + (size_t)u * B + 32 * lo, bytes, ws->bar);
                const uint32_t ph = ws->phase;
                const bool ok = stage::wait(ws->bar, ph, HOOK ? stage_limit_us(ws) : 0u);
                ws->phase ^= 1u;
                if (!__all_sync(kFull, ok)) {
                    give_up(ws, ph, lane, HOOK ? stage_hold(ws) : 0u);
                    break;
                }
#pragma unroll 2
                for (int q = 0; q < nq; ++q) {
                    if ((ws->qz[q] >> jl) & 1u) {
                        float x[W];
                        lds_packed<W>(st + q * B + W * lane, x);
#pragma unroll
                        for (int t = 0; t < W; ++t) Sp[t] += x[t];
                    }
                }
                __syncwarp();
                bal &= ~take;
                staged = true;
            }
            __syncwarp();
            continue;
        }
        const float *base = Cs + lane;
        // two neighbours per step: 2W independent coalesced loads in flight
        while (bal) {
            const int k0 = __ffs(bal) - 1;
            bal &= bal - 1;
            const int k1 = bal ? __ffs(bal) - 1 : -1;
            if (k1 >= 0) bal &= bal - 1;
            const float *r0 = base + (size_t)s_u[k0] * B;
            const float *r1 = base + (size_t)s_u[k1 >= 0 ? k1 : k0] * B;
            const uint32_t z0 = s_nz[k0], z1 = k1 >= 0 ? s_nz[k1] : 0u;
            float x0[W], x1[W];
#pragma unroll
            for (int j = 0; j < W; ++j) {
                x0[j] = ((z0 >> j) & 1u) ? ldx<NC>(r0 + 32 * j) : 0.0f;
                x1[j] = ((z1 >> j) & 1u) ? ldx<NC>(r1 + 32 * j) : 0.0f;
            }
#pragma unroll
            for (int j = 0; j < W; ++j) S[j] += x0[j] + x1[j];
        }
        __syncwarp();
    }
    if constexpr (STAGED) {
        if (staged) {
            float Sj[W];
            unpack_lanes<W>(reinterpret_cast<float *>(ws->buf), Sp, Sj, lane);
#pragma unroll
            for (int j = 0; j < W; ++j) S[j] += Sj[j];
        }
    }
}

// Store sigma and the new frontier words of v (its level-(l+1) sums are final).
// Sn: the masked level-(l+1) uint16 row buffer (zeros for the sources v is
// not new for), written in full when v joins some frontier, or with
// ALL_WORDS = false only in the words that hold a new source of v: every
// adder reads word j of v's row only when v is in frontier l+1 for a source
// of word j. Returns whether v joined; wide is set when one of its new counts
// needs more than 16 bits.
template <int W, bool ALL_WORDS = true>
__device__ __forceinline__ bool store_next(uint64_t *sigma, uint16_t *Sn, uint32_t *Fn, uint32_t *ufn, int v,
                                           const uint64_t (&acc)[W], const uint32_t (&nf)[W], int lane,
                                           bool &wide) {
    constexpr int B = 32 * W;
    uint32_t any = 0;
#pragma unroll
    for (int j = 0; j < W; ++j) {
        any |= nf[j];
        if (lane == j) Fn[(size_t)v * W + j] = nf[j];
        if ((nf[j] >> lane) & 1u) sigma[(size_t)v * B + 32 * j + lane] = acc[j];
    }
    if (any != 0u) {
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const bool mine = (nf[j] >> lane) & 1u;
            wide |= mine && (acc[j] >> 16) != 0ull;
            if (ALL_WORDS || nf[j] != 0u) Sn[(size_t)v * B + 32 * j + lane] = mine ? (uint16_t)acc[j] : (uint16_t)0;
        }
    }
    if (any != 0 && lane == 0) atomicOr(ufn + (v >> 5), 1u << (v & 31));
    return any != 0;
}

// sigma as FP32, correctly rounded; the 32-bit conversion when it fits.
__device__ __forceinline__ float sigma_f32(uint64_t x) {
    return (x >> 32) ? __ull2float_rn(x) : __uint2float_rn((uint32_t)x);
}

// Cl: the masked level-l c buffer (zeros for the sources v is not at level l
// for; null at level 1, whose c values no level reads), written in full, or
// with ALL_WORDS = false only in the words that
// hold a level-l source of v (every backward adder reads word j of v's row
// only when v is at level l for a source of word j). For s with d(s,v) = l: delta_s(v) = sigma_s(v) * S
// and c_s(v) = (1 + delta_s(v)) / sigma_s(v) = 1/sigma_s(v) + S (1/sigma_s(v)
// by the fast reciprocal, within 2 ulp; the correctly rounded one measured
// 1.2 ms slower per R-MAT step). The batch's FP32 delta values of v are summed as an
// unevaluated pair of FP32 words (two_sum_add: W per lane in order, then a
// 5-step tree across the warp, a fixed order) and the total goes into bc[v]
// in FP64.
// sigma_s(v) comes from the level's masked uint16 row Sl when given (a
// narrow level: every count below 2^16), is 1 when `ones` (level 1, reached
// from the sources directly), else from the uint64 array. Ssh: when not null,
// v's words of Sl already copied to shared memory ([W][32], the words with a
// level-l source), read there instead.
template <int W, bool ALL_WORDS = true>
__device__ __forceinline__ void finalize_dep(const uint64_t *sigma, const uint16_t *Sl, bool ones, float *Cl,
                                             double *bc, int v, const uint32_t (&f)[W], const float (&S)[W],
                                             int lane, const uint16_t *Ssh = nullptr,
                                             const uint64_t *Ssig = nullptr) {
    constexpr int B = 32 * W;
    float hi = 0.0f, lo = 0.0f;  // the running sum hi + lo, carried without rounding loss
#pragma unroll
    for (int j = 0; j < W; ++j) {
        const size_t idx = (size_t)v * B + 32 * j + lane;
        float c = 0.0f;
        if ((f[j] >> lane) & 1u) {
            const float sg = ones ? 1.0f
                                  : (Ssh ? __uint2float_rn((uint32_t)Ssh[32 * j + lane])
                                         : (Ssig ? sigma_f32(Ssig[32 * j + lane])
                                                 : (Sl ? __uint2float_rn((uint32_t)Sl[idx]) : sigma_f32(sigma[idx]))));
            const float d = sg * S[j];        // delta_s(v) = sigma_s(v) * sum_w c_s(w)
            c = __fdividef(1.0f, sg) + S[j];  // c_s(v) for the level above (1/sigma within 2 ulp)
            two_sum_add(hi, lo, d);
        }
        if (Cl && (ALL_WORDS || f[j] != 0u)) Cl[idx] = c;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float h2 = __shfl_xor_sync(kFull, hi, off);
        const float l2 = __shfl_xor_sync(kFull, lo, off);
        two_sum_add(hi, lo, h2);
        lo += l2;
    }
    if (lane == 0) bc[v] += (double)hi + (double)lo;
}

template <int W, bool ALL_WORDS = true>
__device__ __forceinline__ void finalize_dep(const uint64_t *sigma, float *Cl, double *bc, int v,
                                             const uint32_t (&f)[W], const float (&S)[W], int lane,
                                             const uint64_t *Ssig = nullptr) {
    finalize_dep<W, ALL_WORDS>(sigma, nullptr, false, Cl, bc, v, f, S, lane, nullptr, Ssig);
}

}  // namespace body
}  // namespace bcgb
