// plain.cu -- one source per launch sequence: the classic level-synchronous
// GPU Brandes (top-down BFS with a vertex queue, atomic path-count updates,
// then a pull over successors level by level). It is the unbatched
// comparator of the multi-source path and computes the same quantities:
//   forward: d(s,v) and sigma_s(v) = sum_{u in P_s(v)} sigma_s(u)  (Section 1.1),
//   backward: delta_s*(v) by Theorem 1.1 in the form
//             delta_s*(v) = sigma_s(v) * sum_{w : v in P_s(w)} c_s(w),
//             c_s(w) = (1 + delta_s*(w)) / sigma_s(w),
//   BC(v) += delta_s*(v) for v != s, in FP64.
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "plain.cuh"
#include "sched.cuh"

namespace bcgb {
namespace {

constexpr int kBlock = 256;
constexpr int kWarps = kBlock / 32;
constexpr unsigned kFull = 0xffffffffu;

struct PlainParams {
    int32_t n;
    int32_t src;
    uint32_t seq;
    const int32_t *row_ptr;
    const int32_t *col;
    int32_t *dist;
    uint64_t *sigma;
    float *cval;
    int32_t *queue;
    int32_t *level_off;
    uint32_t *tail;
    double *bc;
    uint64_t *h_sigma;  // this source's summary slots (or null)
    uint64_t *h_dist;
    int64_t *dist_sum;
    int64_t *reach;
    DevCtl *ctl;
    HostCtl *hctl;
};

__global__ void __launch_bounds__(kBlock) p_init(const PlainParams p) {
    const int stride = gridDim.x * kBlock;
    for (int v = blockIdx.x * kBlock + threadIdx.x; v < p.n; v += stride) {
        p.dist[v] = -1;
        p.sigma[v] = 0ull;
    }
    __shared__ bool s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&p.ctl->blocks_done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last || threadIdx.x != 0) return;
    __threadfence();
    p.dist[p.src] = 0;
    p.sigma[p.src] = 1ull;
    p.queue[0] = p.src;
    p.level_off[0] = 0;
    p.level_off[1] = 1;
    *p.tail = 1u;
    p.ctl->fwd_done = 0u;
    p.ctl->nonempty = 0u;
    p.ctl->seq = p.seq;
    atomicExch(&p.ctl->blocks_done, 0u);
}

__global__ void __launch_bounds__(kBlock) p_forward(const PlainParams p, const int l) {
    __shared__ uint32_t s_ovf;
    __shared__ unsigned long long s_arcs;
    if (threadIdx.x == 0) {
        s_ovf = 0u;
        s_arcs = 0ull;
    }
    __syncthreads();
    if (*(volatile uint32_t *)&p.ctl->fwd_done != 0u || l + 2 > p.n + 1) return;
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * kBlock + threadIdx.x) >> 5;
    const int nwarps = gridDim.x * kWarps;
    const int qb = p.level_off[l], qe = p.level_off[l + 1];
    bool ovf = false;
    uint32_t arcs = 0;
    for (int i = qb + warp; i < qe; i += nwarps) {
        const int u = p.queue[i];
        const uint64_t su = p.sigma[u];
        for (int e = p.row_ptr[u] + lane; e < p.row_ptr[u + 1]; e += 32) {
            const int v = p.col[e];
            int d = __ldcg(p.dist + v);
            if (d < 0) {
                const int old = atomicCAS(p.dist + v, -1, l + 1);
                if (old == -1) {
                    const unsigned pos = atomicAdd(p.tail, 1u);
                    p.queue[pos] = v;
                    d = l + 1;
                } else {
                    d = old;
                }
            }
            if (d == l + 1) {  // u in P_s(v)
                const uint64_t old = atomicAdd(reinterpret_cast<unsigned long long *>(p.sigma + v), su);
                ovf |= old + su < old;
                ++arcs;
            }
        }
    }
    if (__any_sync(kFull, ovf) && lane == 0) atomicOr(&s_ovf, 1u);
    if (arcs) atomicAdd(&s_arcs, (unsigned long long)arcs);
    __syncthreads();
    if (threadIdx.x != 0) return;
    if (s_ovf) atomicOr(&p.ctl->status, BC_STATUS_SIGMA_OVERFLOW);
    if (s_arcs) atomicAdd(&p.ctl->dag_arcs, s_arcs);
    __threadfence();
    if (atomicAdd(&p.ctl->blocks_done, 1u) != gridDim.x - 1) return;
    __threadfence();
    atomicExch(&p.ctl->blocks_done, 0u);
    const int nt = (int)atomicAdd(p.tail, 0u);
    p.level_off[l + 2] = nt;
    if (nt == qe) {
        p.ctl->fwd_done = 1u;
        p.ctl->nlevels = l;
        p.ctl->depth_sum += (unsigned long long)l;
        host_word(&p.hctl->done, p.seq, (uint32_t)l);
    }
    host_word(&p.hctl->progress, p.seq, (uint32_t)(l + 1));
}

__global__ void __launch_bounds__(kBlock) p_backward(const PlainParams p, const int l) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * kBlock + threadIdx.x) >> 5;
    const int nwarps = gridDim.x * kWarps;
    const int qb = p.level_off[l], qe = p.level_off[l + 1];
    for (int i = qb + warp; i < qe; i += nwarps) {
        const int v = p.queue[i];
        float s = 0.0f;
        for (int e = p.row_ptr[v] + lane; e < p.row_ptr[v + 1]; e += 32) {
            const int w = p.col[e];
            if (p.dist[w] == l + 1) s += p.cval[w];  // v in P_s(w)
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(kFull, s, off);
        if (lane == 0) {
            const float sg = __ull2float_rn(p.sigma[v]);
            const float d = sg * s;
            p.cval[v] = (1.0f + d) / sg;
            p.bc[v] += (double)d;
        }
    }
}

__global__ void __launch_bounds__(kBlock) p_hash(const PlainParams p) {
    uint64_t hs = 0, hd = 0, ds = 0, rc = 0;
    const int total = (int)*p.tail;
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < total; i += gridDim.x * kBlock) {
        const int v = p.queue[i];
        const int d = p.dist[v];
        hs += p.sigma[v] * (uint64_t)(v + 1);
        hd += (uint64_t)(d + 1) * (uint64_t)(v + 1);
        ds += (uint64_t)d;
        rc += 1ull;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        hs += __shfl_xor_sync(kFull, hs, off);
        hd += __shfl_xor_sync(kFull, hd, off);
        ds += __shfl_xor_sync(kFull, ds, off);
        rc += __shfl_xor_sync(kFull, rc, off);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(reinterpret_cast<unsigned long long *>(p.h_sigma), hs);
        atomicAdd(reinterpret_cast<unsigned long long *>(p.h_dist), hd);
        atomicAdd(reinterpret_cast<unsigned long long *>(p.dist_sum), ds);
        atomicAdd(reinterpret_cast<unsigned long long *>(p.reach), rc);
    }
}

int grid_for(int n) {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    int g = (n + kBlock - 1) / kBlock;
    return g < 1 ? 1 : (g > 2 * sms ? 2 * sms : g);
}

}  // namespace

void plain_free(PlainState &s) {
    if (s.dist) cudaFree(s.dist);
    if (s.sigma) cudaFree(s.sigma);
    if (s.cval) cudaFree(s.cval);
    if (s.queue) cudaFree(s.queue);
    if (s.level_off) cudaFree(s.level_off);
    if (s.tail) cudaFree(s.tail);
    s = PlainState{};
}

int plain_run(PlainState &s, int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *sources,
              int32_t nsrc, double *bc, uint64_t *h_sigma, uint64_t *h_dist, int64_t *dist_sum, int64_t *reach,
              DevCtl *ctl, HostCtl *hctl_host, HostCtl *hctl_dev, uint32_t *seq, cudaStream_t st,
              const LaunchHook &hook, int64_t wait_ms, std::string *err) {
    if (n == 0 || nsrc == 0) return BC_OK;
    if (s.n != n) {
        plain_free(s);
        cudaError_t e = cudaMalloc((void **)&s.dist, (size_t)n * sizeof(int32_t));
        if (e == cudaSuccess) e = cudaMalloc((void **)&s.sigma, (size_t)n * sizeof(uint64_t));
        if (e == cudaSuccess) e = cudaMalloc((void **)&s.cval, (size_t)n * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc((void **)&s.queue, (size_t)n * sizeof(int32_t));
        if (e == cudaSuccess) e = cudaMalloc((void **)&s.level_off, (size_t)(n + 2) * sizeof(int32_t));
        if (e == cudaSuccess) e = cudaMalloc((void **)&s.tail, sizeof(uint32_t));
        if (e != cudaSuccess) {
            plain_free(s);
            *err = std::string("plain path allocation: ") + cudaGetErrorString(e);
            return e == cudaErrorMemoryAllocation ? BC_ERR_OOM : BC_ERR_CUDA;
        }
        s.n = n;
    }
    // source ids live on the device; the host needs them to fill kernel arguments
    std::vector<int32_t> hsrc(nsrc);
    cudaError_t e = cudaMemcpy(hsrc.data(), sources, (size_t)nsrc * sizeof(int32_t), cudaMemcpyDefault);
    if (e != cudaSuccess) {
        *err = std::string("plain path: ") + cudaGetErrorString(e);
        return BC_ERR_CUDA;
    }
    const int g = grid_for(n);
    for (int32_t i = 0; i < nsrc; ++i) {
        PlainParams p{};
        p.n = n;
        p.src = hsrc[i];
        p.seq = ++*seq;
        p.row_ptr = row_ptr;
        p.col = col;
        p.dist = s.dist;
        p.sigma = s.sigma;
        p.cval = s.cval;
        p.queue = s.queue;
        p.level_off = s.level_off;
        p.tail = s.tail;
        p.bc = bc;
        p.ctl = ctl;
        p.hctl = hctl_dev;
        {
            const size_t t = hook.begin(hook.ctx, BC_KERNEL_INIT);
            p_init<<<g, kBlock, 0, st>>>(p);
            hook.end(hook.ctx, t);
        }
        int L = 0;
        auto launch = [&](int level) {
            const size_t t = hook.begin(hook.ctx, BC_KERNEL_PLAIN);
            p_forward<<<g, kBlock, 0, st>>>(p, level);
            hook.end(hook.ctx, t);
        };
        int r = drive_forward(hctl_host, p.seq, n - 1, launch, wait_ms, st, err, &L);
        if (r) return r;
        for (int l = L; l >= 1; --l) {
            const size_t t = hook.begin(hook.ctx, BC_KERNEL_PLAIN);
            p_backward<<<g, kBlock, 0, st>>>(p, l);
            hook.end(hook.ctx, t);
        }
        if (h_sigma) {
            p.h_sigma = h_sigma + i;
            p.h_dist = h_dist + i;
            p.dist_sum = dist_sum + i;
            p.reach = reach + i;
            const size_t t = hook.begin(hook.ctx, BC_KERNEL_HASH);
            p_hash<<<g, kBlock, 0, st>>>(p);
            hook.end(hook.ctx, t);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) {
            *err = std::string("plain path launch: ") + cudaGetErrorString(e);
            return BC_ERR_CUDA;
        }
    }
    return BC_OK;
}

}  // namespace bcgb
