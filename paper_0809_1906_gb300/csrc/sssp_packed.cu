// sssp_packed.cu -- the weighted per-source sweep (one CTA per source,
// Dial's buckets; see sssp_weighted.cu for the algorithm) with each vertex's
// state packed in one 64-bit word:
//   forward:   bits 63..32 = tentative / final distance, bits 31..0 = sigma
//              (0 until the vertex is settled),
//   backward:  bits 31..0 = the FP32 c value once the vertex is finished.
// A relaxation is one 64-bit atomicMin(word, nd << 32): it lowers the
// distance (and leaves sigma 0) and returns the neighbour's word, whose
// distance and sigma decide whether it is a predecessor (Section 1.1's
// P_s(v)). A settled vertex's word never changes again: every later
// relaxation into it carries a larger distance. Settling ORs sigma into the
// low half. In the backward pass the successors of v (larger distance) are
// finished first, so one 8-byte load gives a successor's distance and c.
// One random sector per arc instead of two or three.
//
// sigma is 32-bit here: a source whose count reaches 2^32 writes no output,
// sets redo[its position] and is recomputed by the 64-bit kernel.
#include <cuda_runtime.h>

#include "bc_internal.cuh"
#include "weighted.cuh"

namespace bcgb {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint32_t kDInf = 0x7fffffffu;

struct PSmem {
    int32_t cnt[kMaxRing];
    uint32_t ovf[kMaxRing / 32];
    int32_t nset[2];  // vertices settled in the current step, by step parity
    int32_t pending;
    int32_t ngroups;
    uint32_t flags;  // 1: sigma overflowed 32 bits
    unsigned long long red[4][32];  // one slot per warp (up to 1024 threads)
};

__device__ __forceinline__ uint32_t pd(uint64_t x) { return (uint32_t)(x >> 32); }
__device__ __forceinline__ uint32_t pl(uint64_t x) { return (uint32_t)x; }

__device__ __forceinline__ void push(const WParams &p, PSmem &sm, int32_t *slots, int32_t u, int32_t nd) {
    const int b = nd % p.K;
    const int at = atomicAdd(&sm.cnt[b], 1);
    atomicAdd(&sm.pending, 1);
    if (at < p.C)
        slots[(size_t)b * p.C + at] = u;
    else
        atomicOr(&sm.ovf[b >> 5], 1u << (b & 31));
}

// kPBlk threads per source (w_packed_threads)
template <int kPBlk>
__global__ void __launch_bounds__(kPBlk, 1024 / kPBlk) k_wsssp_packed(const WParams p) {
    __shared__ PSmem sm;
    const int i = blockIdx.x;
    const int o = p.pos ? p.pos[i] : i;  // output position
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int32_t src = p.sources[i];
    const int n = p.n;
    unsigned long long *ds = reinterpret_cast<unsigned long long *>(p.ds + (size_t)i * n);
    int32_t *order = p.order + (size_t)i * n;
    int32_t *grp = p.grp + (size_t)i * (n + 1);
    int32_t *slots = p.slots + (size_t)i * p.K * p.C;
    float *drow = p.delta_rows ? p.delta_rows + (size_t)i * n : nullptr;  // reduced after the wave

    for (int v = tid; v < n; v += kPBlk) {
        ds[v] = (unsigned long long)kDInf << 32;
        if (drow) drow[v] = 0.0f;
    }
    for (int b = tid; b < p.K; b += kPBlk) sm.cnt[b] = 0;
    for (int b = tid; b < kMaxRing / 32; b += kPBlk) sm.ovf[b] = 0u;
    if (tid == 0) {
        sm.nset[0] = sm.nset[1] = 0;
        sm.pending = 0;
        sm.ngroups = 0;
        sm.flags = 0u;
    }
    __syncthreads();
    if (tid == 0) {
        ds[src] = 0ull;
        push(p, sm, slots, src, 0);
    }
    __syncthreads();

    unsigned long long arcs = 0;
    bool big = false;  // a count reached 2^32
    int32_t done = 0;
    int32_t d = 0;
    int par = 0;  // parity of the non-empty steps (which settled counter is live)
    while (sm.pending > 0) {
        const int b = d % p.K;
        const int cnt = sm.cnt[b];
        const bool spill = (sm.ovf[b >> 5] >> (b & 31)) & 1u;
        if (d > p.dmax) {
            if (tid == 0) atomicOr(&p.ctl->status, BC_STATUS_BOUNDS);
            break;
        }
        if (cnt == 0 && !spill) {
            ++d;
            continue;
        }
        // every settled vertex (tentative distance d is final) is relaxed by
        // the thread that found it: the push only fires on a strict decrease,
        // so a vertex sits once in its final bucket; its predecessors were all
        // settled at smaller distances; pushes go to other buckets (w >= 1,
        // the ring is wider than the largest weight)
        auto settle = [&](const int v) {
            uint32_t s = v == src ? 1u : 0u;
            if (p.col_in) {
                // directed: sigma over v's in-arcs (their tails below d are final)
                if (v != src)
                    for (int e = p.row_ptr_in[v]; e < p.row_ptr_in[v + 1]; ++e) {
                        const unsigned long long x = __ldcg(ds + p.col_in[e]);
                        if (pd(x) < (uint32_t)d && pd(x) + (uint32_t)p.w_in[e] == (uint32_t)d) {
                            const uint32_t y = s + pl(x);
                            big |= y < s;
                            s = y;
                            ++arcs;
                        }
                    }
                for (int e = p.row_ptr[v]; e < p.row_ptr[v + 1]; ++e) {
                    const int u = p.col[e];
                    const int nd = d + p.w[e];
                    const unsigned long long old = atomicMin(ds + u, (unsigned long long)nd << 32);
                    if ((uint32_t)nd < pd(old)) push(p, sm, slots, u, nd);
                }
            } else {
                // undirected: one atomicMin per arc relaxes it and returns the
                // neighbour's word; it is a predecessor when its (final)
                // distance plus the arc weight is d
                const int e1 = p.row_ptr[v + 1];
                for (int e = p.row_ptr[v]; e < e1; e += 4) {
                    int u[4], nd[4];
                    uint32_t w[4];
                    unsigned long long old[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        u[q] = -1;
                        w[q] = 0u;
                        if (e + q < e1) {
                            u[q] = p.col[e + q];
                            w[q] = (uint32_t)p.w[e + q];
                            nd[q] = d + (int)w[q];  // <= n * max weight < 2^31
                        }
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        old[q] = u[q] >= 0 ? atomicMin(ds + u[q], (unsigned long long)nd[q] << 32)
                                           : ((unsigned long long)kDInf << 32);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const uint32_t du = pd(old[q]);
                        // u before v (du < d, final) with du + w(u,v) = d
                        const bool pred = u[q] >= 0 && v != src && du < (uint32_t)d && du + w[q] == (uint32_t)d;
                        if (pred) {
                            const uint32_t y = s + pl(old[q]);
                            big |= y < s;
                            s = y;
                            ++arcs;
                        }
                        if (u[q] >= 0 && (uint32_t)nd[q] < du) push(p, sm, slots, u[q], nd[q]);
                    }
                }
            }
            atomicOr(ds + v, (unsigned long long)s);  // settled: sigma into the low half
        };
        if (!spill) {
            for (int k = tid; k < cnt; k += kPBlk) {
                const int v = __ldcg(slots + (size_t)b * p.C + k);
                if (pd(__ldcg(ds + v)) == (uint32_t)d) {
                    order[done + atomicAdd(&sm.nset[par], 1)] = v;
                    settle(v);
                }
            }
        } else {
            for (int v = tid; v < n; v += kPBlk)
                if (pd(__ldcg(ds + v)) == (uint32_t)d) {
                    order[done + atomicAdd(&sm.nset[par], 1)] = v;
                    settle(v);
                }
        }
        __syncthreads();
        const int k = sm.nset[par];
        if (tid == 0) {
            sm.cnt[b] = 0;
            atomicAnd(&sm.ovf[b >> 5], ~(1u << (b & 31)));
            atomicSub(&sm.pending, cnt);
            if (k > 0) grp[sm.ngroups++] = done;
            sm.nset[par ^ 1] = 0;  // the next step's counter (nobody reads it in this one)
        }
        done += k;
        par ^= 1;
        ++d;
        __syncthreads();
    }
    const int ng = sm.ngroups;
    if (tid == 0) grp[ng] = done;
    if (__syncthreads_or(big)) {  // leave this source to the 64-bit kernel
        if (tid == 0) p.redo[o] = 1u;
        return;
    }

    // ---- per-source summaries and optional rows
    unsigned long long hs = 0, hd = 0, dsum = 0, rc = 0;
    for (int t = tid; t < done; t += kPBlk) {
        const int v = order[t];
        const unsigned long long x = ds[v];
        const unsigned long long id1 = (unsigned long long)(p.vid ? p.vid[v] : v) + 1ull;  // the caller's id + 1
        hs += (unsigned long long)pl(x) * id1;
        hd += (unsigned long long)(pd(x) + 1) * id1;
        dsum += pd(x);
        rc += 1ull;
    }
    if (p.rows_dist || p.rows_sigma) {
        for (int v = tid; v < n; v += kPBlk) {
            const unsigned long long x = ds[v];
            const bool r = pd(x) != kDInf;
            const size_t at = (size_t)o * n + (size_t)(p.vid ? p.vid[v] : v);
            if (p.rows_dist) p.rows_dist[at] = r ? (int32_t)pd(x) : -1;
            if (p.rows_sigma) p.rows_sigma[at] = r ? (unsigned long long)pl(x) : 0ull;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        hs += __shfl_xor_sync(kFull, hs, off);
        hd += __shfl_xor_sync(kFull, hd, off);
        dsum += __shfl_xor_sync(kFull, dsum, off);
        rc += __shfl_xor_sync(kFull, rc, off);
        arcs += __shfl_xor_sync(kFull, arcs, off);
    }
    if (lane == 0) {
        sm.red[0][wid] = hs;
        sm.red[1][wid] = hd;
        sm.red[2][wid] = dsum;
        sm.red[3][wid] = rc;
        if (arcs) atomicAdd(&p.ctl->dag_arcs, arcs);
    }
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < kPBlk / 32; ++w)
            for (int q = 0; q < 4; ++q) sm.red[q][0] += sm.red[q][w];
        if (p.h_sigma) {
            p.h_sigma[o] = sm.red[0][0];
            p.h_dist[o] = sm.red[1][0];
            p.dist_sum[o] = (int64_t)sm.red[2][0];
            p.reach[o] = (int64_t)sm.red[3][0];
        }
        atomicAdd(&p.ctl->depth_sum, (unsigned long long)(ng > 0 ? ng - 1 : 0));
    }
    if (!drow) return;
    __syncthreads();  // the summaries read sigma before the backward overwrites it

    // ---- backward: distance groups in decreasing order (Theorem 1.1)
    for (int g = ng - 1; g >= 0; --g) {
        const int a = grp[g], z = grp[g + 1];
        for (int t = a + tid; t < z; t += kPBlk) {
            const int v = order[t];
            const unsigned long long xv = ds[v];
            const uint32_t dv = pd(xv);
            const int e1 = p.row_ptr[v + 1];
            float S = 0.0f;
            for (int e = p.row_ptr[v]; e < e1; e += 4) {
                unsigned long long x[4];
                uint32_t want[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    want[q] = kDInf;
                    x[q] = 0ull;
                    if (e + q < e1) {
                        want[q] = dv + (uint32_t)p.w[e + q];
                        x[q] = __ldcg(ds + p.col[e + q]);
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (pd(x[q]) == want[q] && pd(x[q]) != kDInf) S += __uint_as_float(pl(x[q]));  // v in P_s(x)
            }
            const float sg = __uint2float_rn(pl(xv));
            const float dl = sg * S;
            if (v != src) drow[v] = dl;
            ds[v] = ((unsigned long long)dv << 32) | __float_as_uint(__fdividef(1.0f, sg) + S);  // c_s(v)
        }
        __syncthreads();
    }
}

}  // namespace

int w_packed_threads(int32_t n) { return n < kWSmallN ? 128 : 512; }

void w_launch_wave_packed(const WParams &p, int nsrc, cudaStream_t st) {
    if (w_packed_threads(p.n) == 128)
        k_wsssp_packed<128><<<nsrc, 128, 0, st>>>(p);
    else
        k_wsssp_packed<512><<<nsrc, 512, 0, st>>>(p);
}

}  // namespace bcgb
