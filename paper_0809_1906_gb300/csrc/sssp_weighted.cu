// sssp_weighted.cu -- exact betweenness for positive integer weights.
//
// One CTA per source; a launch runs a whole wave of sources (one per resident
// CTA), so the batch is the set of CTAs in flight and no level loop needs the
// host. Inside a CTA the single-source problem is solved with integer
// buckets of width one (delta-stepping with delta = 1, i.e. Dial's bucket
// queue): a ring of K > max weight buckets indexed by distance mod K. At step
// d the CTA
//   1. settles every vertex whose tentative distance is d (bucket entries
//      whose distance is still d; entries left behind by a later improvement
//      are stale and skipped),
//   2. counts its shortest paths over the predecessor set of Section 1.1,
//        sigma_s(v) = sum_{u : (u,v) in E, d(s,u) + w(u,v) = d} sigma_s(u),
//      which is final because every predecessor has a smaller distance and
//      was settled at an earlier step (ties of any length are all counted),
//   3. relaxes v's arcs (atomicMin on the tentative distance, push on a strict
//      improvement).
// The settle order is kept with one group per distinct distance. The backward
// pass walks the groups in reverse (Theorem 1.1, decreasing distance):
//   delta_s*(v) = sigma_s(v) * sum_{w : v in P_s(w)} c_s(w),
//   c_s(v) = (1 + delta_s*(v)) / sigma_s(v)   (FP32),
// and writes delta_s*(v) to the wave's row; a second kernel adds the rows to
// BC in FP64 in source order (deterministic).
//
// A bucket whose entry list fills up sets a flag and is settled by scanning
// every vertex's distance instead (correct, slower); nothing waits on another
// CTA.
#include <cuda_runtime.h>

#include "bc_internal.cuh"
#include "weighted.cuh"

namespace bcgb {
namespace {

constexpr int kWBlock = 256;
constexpr unsigned kFull = 0xffffffffu;
constexpr int32_t kInf = 0x7fffffff;

struct WSmem {
    int32_t cnt[kMaxRing];       // entries pushed into each bucket
    uint32_t ovf[kMaxRing / 32]; // bucket overflowed its entry list
    int32_t nset;                // vertices settled at the current step
    int32_t pending;             // entries not yet consumed
    int32_t ngroups;
    uint32_t flags;
    unsigned long long red[4][kWBlock / 32];
};

__device__ __forceinline__ void push_entry(const WParams &p, WSmem &sm, int32_t *slots, int32_t u, int32_t nd) {
    const int b = nd % p.K;
    const int pos = atomicAdd(&sm.cnt[b], 1);
    atomicAdd(&sm.pending, 1);
    if (pos < p.C)
        slots[(size_t)b * p.C + pos] = u;
    else
        atomicOr(&sm.ovf[b >> 5], 1u << (b & 31));
}

__global__ void __launch_bounds__(kWBlock, 4) k_wsssp(const WParams p) {
    __shared__ WSmem sm;
    const int i = blockIdx.x;  // source index within the wave
    const int o = p.pos ? p.pos[i] : i;  // output position
    const int tid = threadIdx.x;
    const int lane = tid & 31, wid = tid >> 5;
    const int32_t src = p.sources[i];
    const int n = p.n;
    int32_t *dist = p.dist + (size_t)i * n;
    uint64_t *sigma = p.sigma + (size_t)i * n;
    float *cval = p.cval + (size_t)i * n;
    int32_t *order = p.order + (size_t)i * n;
    int32_t *grp = p.grp + (size_t)i * (n + 1);
    int32_t *slots = p.slots + (size_t)i * p.K * p.C;
    float *drow = p.delta_rows ? p.delta_rows + (size_t)i * n : nullptr;  // reduced after the wave

    for (int v = tid; v < n; v += kWBlock) {
        dist[v] = kInf;
        if (drow) drow[v] = 0.0f;
    }
    for (int b = tid; b < p.K; b += kWBlock) sm.cnt[b] = 0;
    for (int b = tid; b < kMaxRing / 32; b += kWBlock) sm.ovf[b] = 0u;
    if (tid == 0) {
        sm.nset = 0;
        sm.pending = 0;
        sm.ngroups = 0;
        sm.flags = 0u;
    }
    __syncthreads();
    if (tid == 0) {
        dist[src] = 0;
        push_entry(p, sm, slots, src, 0);
    }
    __syncthreads();

    unsigned long long arcs = 0;
    bool ovf64 = false;
    int32_t done = 0;  // vertices settled so far = next position in order[]
    int32_t d = 0;
    // ---- forward: Dial's buckets, one distance value per step
    while (sm.pending > 0) {
        const int b = d % p.K;
        const int cnt = sm.cnt[b];
        const bool spill = (sm.ovf[b >> 5] >> (b & 31)) & 1u;
        if (d > p.dmax) {  // cannot happen for valid input: a guard against looping forever
            if (tid == 0) atomicOr(&p.ctl->status, BC_STATUS_BOUNDS);
            break;
        }
        if (cnt == 0 && !spill) {
            ++d;
            continue;
        }
        __syncthreads();  // everyone has read cnt / spill / pending for this step
        // 1. settle: entries whose distance is still d
        if (!spill) {
            for (int k = tid; k < cnt; k += kWBlock) {
                const int v = __ldcg(slots + (size_t)b * p.C + k);
                if (__ldcg(dist + v) == d) order[done + atomicAdd(&sm.nset, 1)] = v;
            }
        } else {
            for (int v = tid; v < n; v += kWBlock)
                if (__ldcg(dist + v) == d) order[done + atomicAdd(&sm.nset, 1)] = v;
        }
        __syncthreads();
        const int k = sm.nset;
        if (tid == 0) {
            // other threads may push into other buckets meanwhile: atomics only
            sm.cnt[b] = 0;
            atomicAnd(&sm.ovf[b >> 5], ~(1u << (b & 31)));
            atomicSub(&sm.pending, cnt);
            if (k > 0) grp[sm.ngroups++] = done;
        }
        // 2 + 3. path counts over P_s(v) and relaxation, four arcs at a time.
        // One atomicMin per arc does both: the value it returns is u's
        // distance before the call, which is final whenever it is below d
        // (this step only produces distances above d), so u is in P_s(v)
        // exactly when that value equals d - w(u,v); and the call itself
        // relaxes the arc.
        for (int t = tid; p.col_in && t < k; t += kWBlock) {
            // directed graphs: P_s(v) over v's in-arcs, whose tails below d are
            // final; the out-arcs are relaxed below
            const int v = order[done + t];
            uint64_t s = v == src ? 1ull : 0ull;
            if (v != src) {
                for (int e = p.row_ptr_in[v]; e < p.row_ptr_in[v + 1]; ++e) {
                    const int u = p.col_in[e];
                    const int du = __ldcg(dist + u);
                    if (du < d && du + p.w_in[e] == d) {
                        const uint64_t x = __ldcg(sigma + u);
                        const uint64_t y = s + x;
                        ovf64 |= y < x;
                        s = y;
                        ++arcs;
                    }
                }
            }
            sigma[v] = s;
            for (int e = p.row_ptr[v]; e < p.row_ptr[v + 1]; ++e) {
                const int u = p.col[e];
                const int nd = d + p.w[e];
                const int old = atomicMin(dist + u, nd);
                if (nd < old) push_entry(p, sm, slots, u, nd);
            }
        }
        for (int t = tid; t < k && !p.col_in; t += kWBlock) {
            const int v = order[done + t];
            const int e0 = p.row_ptr[v], e1 = p.row_ptr[v + 1];
            uint64_t s = v == src ? 1ull : 0ull;
            for (int e = e0; e < e1; e += 4) {
                int u[4], nd[4], old[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    u[i] = -1;
                    if (e + i < e1) {
                        u[i] = p.col[e + i];
                        nd[i] = d + p.w[e + i];
                    }
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) old[i] = u[i] >= 0 ? atomicMin(dist + u[i], nd[i]) : kInf;
                uint64_t x[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    // u before v (old < d, final) with old + w(u,v) = d; nd - d = w
                    const bool pred = u[i] >= 0 && v != src && old[i] < d && old[i] + (nd[i] - d) == d;
                    x[i] = pred ? __ldcg(sigma + u[i]) : 0ull;
                    arcs += pred ? 1ull : 0ull;
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const uint64_t y = s + x[i];
                    ovf64 |= y < x[i];
                    s = y;
                    if (u[i] >= 0 && nd[i] < old[i]) push_entry(p, sm, slots, u[i], nd[i]);
                }
            }
            sigma[v] = s;
        }
        __syncthreads();
        done += k;
        if (tid == 0) sm.nset = 0;
        ++d;
        __syncthreads();
    }
    const int ng = sm.ngroups;
    if (tid == 0) grp[ng] = done;
    __syncthreads();

    // ---- per-source summaries and optional rows
    unsigned long long hs = 0, hd = 0, ds = 0, rc = 0;
    for (int t = tid; t < done; t += kWBlock) {
        const int v = order[t];
        const int dv = dist[v];
        const uint64_t sg = sigma[v];
        const unsigned long long id1 = (unsigned long long)(p.vid ? p.vid[v] : v) + 1ull;  // the caller's id + 1
        hs += sg * id1;
        hd += (unsigned long long)(dv + 1) * id1;
        ds += (unsigned long long)dv;
        rc += 1ull;
    }
    if (p.rows_dist || p.rows_sigma) {
        for (int v = tid; v < n; v += kWBlock) {
            const int dv = dist[v];
            const size_t at = (size_t)o * n + (size_t)(p.vid ? p.vid[v] : v);
            if (p.rows_dist) p.rows_dist[at] = dv == kInf ? -1 : dv;
            if (p.rows_sigma) p.rows_sigma[at] = dv == kInf ? 0ull : sigma[v];
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        hs += __shfl_xor_sync(kFull, hs, off);
        hd += __shfl_xor_sync(kFull, hd, off);
        ds += __shfl_xor_sync(kFull, ds, off);
        rc += __shfl_xor_sync(kFull, rc, off);
        arcs += __shfl_xor_sync(kFull, arcs, off);
    }
    const bool wovf = __any_sync(kFull, ovf64);
    if (lane == 0) {
        sm.red[0][wid] = hs;
        sm.red[1][wid] = hd;
        sm.red[2][wid] = ds;
        sm.red[3][wid] = rc;
        if (arcs) atomicAdd(&p.ctl->dag_arcs, arcs);
        if (wovf) atomicOr(&sm.flags, 1u);
    }
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < kWBlock / 32; ++w)
            for (int q = 0; q < 4; ++q) sm.red[q][0] += sm.red[q][w];
        if (p.h_sigma) {
            p.h_sigma[o] = sm.red[0][0];
            p.h_dist[o] = sm.red[1][0];
            p.dist_sum[o] = (int64_t)sm.red[2][0];
            p.reach[o] = (int64_t)sm.red[3][0];
        }
        if (sm.flags & 1u) atomicOr(&p.ctl->status, BC_STATUS_SIGMA_OVERFLOW);
        atomicAdd(&p.ctl->depth_sum, (unsigned long long)(ng > 0 ? ng - 1 : 0));
    }
    if (!drow) return;

    // ---- backward: distance groups in decreasing order (Theorem 1.1)
    for (int g = ng - 1; g >= 0; --g) {
        const int a = grp[g], z = grp[g + 1];
        for (int t = a + tid; t < z; t += kWBlock) {
            const int v = order[t];
            const int dv = dist[v];
            const int e0 = p.row_ptr[v], e1 = p.row_ptr[v + 1];
            float S = 0.0f;
            for (int e = e0; e < e1; e += 4) {
                int x[4], dx[4], want[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    x[i] = -1;
                    if (e + i < e1) {
                        x[i] = p.col[e + i];
                        want[i] = dv + p.w[e + i];
                    }
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) dx[i] = x[i] >= 0 ? dist[x[i]] : kInf;
                float c[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) c[i] = (x[i] >= 0 && dx[i] == want[i]) ? __ldcg(cval + x[i]) : 0.0f;  // v in P_s(x)
#pragma unroll
                for (int i = 0; i < 4; ++i) S += c[i];
            }
            const float sg = __ull2float_rn(sigma[v]);
            const float dl = sg * S;
            cval[v] = (1.0f + dl) / sg;
            if (v != src) drow[v] = dl;
        }
        __syncthreads();
    }
}

// BC(v) += sum over the wave's rows in row order (FP64).
__global__ void __launch_bounds__(256) k_wreduce(const float *__restrict__ rows, int32_t nrows, int32_t n,
                                                 const int32_t *__restrict__ vid, double *__restrict__ bc) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int r = 0; r < nrows; ++r) acc += (double)rows[(size_t)r * n + v];
        bc[vid ? vid[v] : v] += acc;
    }
}

}  // namespace

void w_launch_wave(const WParams &p, int nsrc, cudaStream_t st) {
    k_wsssp<<<nsrc, kWBlock, 0, st>>>(p);
}

void w_launch_reduce(const float *rows, int nrows, int n, const int32_t *vid, double *bc, int sms,
                     cudaStream_t st) {
    int g = (n + 255) / 256;
    g = g > 4 * sms ? 4 * sms : (g < 1 ? 1 : g);
    k_wreduce<<<g, 256, 0, st>>>(rows, nrows, n, vid, bc);
}

}  // namespace bcgb
