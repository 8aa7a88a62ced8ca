// minplus.cu -- the weighted algebraic forward pass (Section 3.2): distance
// products with path counts on a dense weight matrix.
//
// For a batch of sources s the state is X[s][v] = (d, c). One step computes
//   Y[s][v] = (+)_u  X[s][u] (x) (w(u,v), 1)   (+)   [v = s] (0, 1)
// with (d, c) (x) (w, 1) = (d + w, c) and (d, c) (+) (d', c') = (min(d, d'),
// sum of the counts that reach the min). By induction on k, after k steps
// X[s][v] holds the least weight of an s-v walk of at most k arcs and the
// number of such walks of that weight; with positive weights those walks
// are simple paths, so once k reaches the largest arc count of any shortest
// path from the batch's sources, X = (d(s,v), lambda_sv) and a further step
// changes nothing. The host repeats steps until one reports no change.
//
// k_mp_step is a GEMM-shaped kernel on CUDA cores (there is no tensor-core
// min-plus): a block owns 64 sources x 64 targets, stages 32 intermediate
// vertices u at a time (distances, counts, weight rows) in shared memory, and
// each thread keeps a 4 x 4 tile of (d, c) in registers, in two passes over u
// (least weights, then the counts that reach them). Counts are uint64
// (mod 2^64, a carry sets the overflow status bit); distances int32 with
// kMpInf for "no walk yet" (the caller guarantees every distance < 2^30).
#include <cuda_runtime.h>

#include <cstdint>

#include "bc_internal.cuh"
#include "minplus.cuh"

namespace bcgb {
namespace {

constexpr int kMS = 64;       // sources per block
constexpr int kMV = 64;       // targets per block
constexpr int kMU = 32;       // intermediate vertices per stage
constexpr int kMBlk = 256;    // 16 x 16 threads, 4 x 4 outputs each

__global__ void __launch_bounds__(256) k_mp_init(int32_t *__restrict__ xd, uint64_t *__restrict__ xc,
                                                 const int32_t *__restrict__ src, int nb, int n) {
    const size_t cells = (size_t)nb * n;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < cells; i += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(i / n), v = (int)(i % n);
        const bool self = v == src[b];
        xd[i] = self ? 0 : kMpInf;
        xc[i] = self ? 1ull : 0ull;
    }
}

// wm: [n][n] weight of arc (u, v), kMpInf when there is none.
// Two passes over the intermediate vertices u: the first finds the least
// walk weight of every (s, v) of the tile (an add and a min per element), the
// second adds the counts of the walks that reach it (a compare and a
// predicated 64-bit add whose carry is kept, per element). That is about
// half the instructions of one pass that tracks both together.
__device__ __forceinline__ void add_if_equal(int32_t t, int32_t b, uint32_t alo, uint32_t ahi, uint32_t &lo,
                                             uint32_t &hi, uint32_t &ov) {
    asm("{\n\t.reg .pred p;\n\t"
        "setp.eq.s32 p, %3, %4;\n\t"
        "@p add.cc.u32 %0, %0, %5;\n\t"
        "@p addc.cc.u32 %1, %1, %6;\n\t"
        "@p addc.u32 %2, %2, 0;\n\t}"
        : "+r"(lo), "+r"(hi), "+r"(ov)
        : "r"(t), "r"(b), "r"(alo), "r"(ahi));
}

__global__ void __launch_bounds__(kMBlk) k_mp_step(const int32_t *__restrict__ xd, const uint64_t *__restrict__ xc,
                                                   int32_t *__restrict__ yd, uint64_t *__restrict__ yc,
                                                   const int32_t *__restrict__ wm, const int32_t *__restrict__ src,
                                                   int nb, int n, uint32_t *__restrict__ flags,
                                                   uint32_t *__restrict__ status) {
    __shared__ int32_t s_d[kMU][kMS + 1];  // transposed: [u][s], padded against bank conflicts
    __shared__ uint32_t s_lo[kMU][kMS + 1];
    __shared__ uint32_t s_hi[kMU][kMS + 1];
    __shared__ int32_t s_w[kMU][kMV];
    const int s0 = blockIdx.y * kMS, v0 = blockIdx.x * kMV;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // target group, source group
    auto load_w = [&](int u0) {
        for (int i = threadIdx.x; i < kMU * kMV; i += kMBlk) {
            const int r = i / kMV, c = i % kMV;
            const int u = u0 + r, v = v0 + c;
            s_w[r][c] = (u < n && v < n) ? wm[(size_t)u * n + v] : kMpInf;
        }
    };
    int32_t best[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) best[i][j] = kMpInf;
    // pass 1: least walk weights
    for (int u0 = 0; u0 < n; u0 += kMU) {
        __syncthreads();
        for (int i = threadIdx.x; i < kMU * kMS; i += kMBlk) {
            const int r = i / kMU, c = i % kMU;  // source r, vertex u0 + c (coalesced along u)
            const int s = s0 + r, u = u0 + c;
            s_d[c][r] = (s < nb && u < n) ? xd[(size_t)s * n + u] : kMpInf;
        }
        load_w(u0);
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < kMU; ++k) {
            int32_t ad[4], wv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                ad[i] = s_d[k][ty + 16 * i];
                wv[i] = s_w[k][tx + 16 * i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) best[i][j] = min(best[i][j], ad[i] + wv[j]);  // both below 2^30
        }
    }
    // pass 2: counts of the walks of least weight
    uint32_t lo[4][4], hi[4][4], ov[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        ov[i] = 0u;
#pragma unroll
        for (int j = 0; j < 4; ++j) lo[i][j] = hi[i][j] = 0u;
    }
    for (int u0 = 0; u0 < n; u0 += kMU) {
        __syncthreads();
        for (int i = threadIdx.x; i < kMU * kMS; i += kMBlk) {
            const int r = i / kMU, c = i % kMU;
            const int s = s0 + r, u = u0 + c;
            const bool in = s < nb && u < n;
            const uint64_t x = in ? xc[(size_t)s * n + u] : 0ull;
            s_d[c][r] = in ? xd[(size_t)s * n + u] : kMpInf;
            s_lo[c][r] = (uint32_t)x;
            s_hi[c][r] = (uint32_t)(x >> 32);
        }
        load_w(u0);
        __syncthreads();
#pragma unroll 2
        for (int k = 0; k < kMU; ++k) {
            int32_t ad[4], wv[4];
            uint32_t alo[4], ahi[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                ad[i] = s_d[k][ty + 16 * i];
                alo[i] = s_lo[k][ty + 16 * i];
                ahi[i] = s_hi[k][ty + 16 * i];
                wv[i] = s_w[k][tx + 16 * i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) add_if_equal(ad[i] + wv[j], best[i][j], alo[i], ahi[i], lo[i][j], hi[i][j], ov[i]);
        }
    }
    bool changed = false;
    bool carry = false;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int s = s0 + ty + 16 * i;
        if (s >= nb) continue;
        const int self = src[s];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int v = v0 + tx + 16 * j;
            if (v >= n) continue;
            int32_t d = best[i][j] >= kMpInf ? kMpInf : best[i][j];
            uint64_t c = d >= kMpInf ? 0ull : (((uint64_t)hi[i][j] << 32) | lo[i][j]);
            if (d < kMpInf) carry |= ov[i] != 0u;
            if (v == self) {  // the empty walk; every other walk back to s is longer
                d = 0;
                c = 1ull;
            }
            const size_t at = (size_t)s * n + v;
            changed |= d != xd[at] || c != xc[at];
            yd[at] = d;
            yc[at] = c;
        }
    }
    if (__syncthreads_or(changed) && threadIdx.x == 0) atomicOr(flags, 1u);
    if (__syncthreads_or(carry) && threadIdx.x == 0) atomicOr(status, BC_STATUS_SIGMA_OVERFLOW);
}

// Rows for the caller: distance -1 where unreachable, counts 0 there.
__global__ void __launch_bounds__(256) k_mp_rows(const int32_t *__restrict__ xd, const uint64_t *__restrict__ xc,
                                                 int nb, int n, int32_t *__restrict__ dist, uint64_t *__restrict__ sig) {
    const size_t cells = (size_t)nb * n;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < cells; i += (size_t)gridDim.x * blockDim.x) {
        const int32_t d = xd[i];
        if (dist) dist[i] = d >= kMpInf ? -1 : d;
        if (sig) sig[i] = d >= kMpInf ? 0ull : xc[i];
    }
}

// Per-source summaries from full rows (one block per row, fixed reduction order).
__global__ void __launch_bounds__(256) k_mp_row_hash(const int32_t *__restrict__ dist, const uint64_t *__restrict__ sig,
                                                     int nb, int n, uint64_t *__restrict__ h_sigma,
                                                     uint64_t *__restrict__ h_dist, int64_t *__restrict__ dist_sum,
                                                     int64_t *__restrict__ reach) {
    __shared__ uint64_t sh[4][256];
    for (int b = blockIdx.x; b < nb; b += gridDim.x) {
        uint64_t hs = 0, hd = 0, ds = 0, rc = 0;
        for (int v = threadIdx.x; v < n; v += 256) {
            const int32_t d = dist[(size_t)b * n + v];
            if (d < 0) continue;
            const uint64_t vv = (uint64_t)(v + 1);
            hs += sig[(size_t)b * n + v] * vv;
            hd += (uint64_t)(d + 1) * vv;
            ds += (uint64_t)d;
            rc += 1ull;
        }
        __syncthreads();
        sh[0][threadIdx.x] = hs;
        sh[1][threadIdx.x] = hd;
        sh[2][threadIdx.x] = ds;
        sh[3][threadIdx.x] = rc;
        __syncthreads();
        for (int off = 128; off > 0; off >>= 1) {
            if (threadIdx.x < off)
                for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + off];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            h_sigma[b] = sh[0][0];
            h_dist[b] = sh[1][0];
            dist_sum[b] = (int64_t)sh[2][0];
            reach[b] = (int64_t)sh[3][0];
        }
    }
}

__global__ void k_mp_weights(const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                             const int32_t *__restrict__ w, int n, int32_t *__restrict__ wm) {
    for (int u = blockIdx.x; u < n; u += gridDim.x)
        for (int e = rp[u] + threadIdx.x; e < rp[u + 1]; e += blockDim.x) wm[(size_t)u * n + col[e]] = w[e];
}

__global__ void __launch_bounds__(256) k_mp_fill(int32_t *__restrict__ a, size_t cells, int32_t value) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < cells; i += (size_t)gridDim.x * blockDim.x)
        a[i] = value;
}

int grid_for(size_t cells, int sms) {
    size_t g = (cells + 255) / 256;
    const size_t cap = (size_t)8 * sms;
    return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

int mp_build_weights(const int32_t *rp, const int32_t *col, const int32_t *w, int n, int32_t *wm, int sms,
                     cudaStream_t st) {
    k_mp_fill<<<grid_for((size_t)n * n, sms), 256, 0, st>>>(wm, (size_t)n * n, kMpInf);
    int g = n < 8 * sms ? (n < 1 ? 1 : n) : 8 * sms;
    k_mp_weights<<<g, 128, 0, st>>>(rp, col, w, n, wm);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int mp_init(int32_t *xd, uint64_t *xc, const int32_t *src, int nb, int n, int sms, cudaStream_t st) {
    k_mp_init<<<grid_for((size_t)nb * n, sms), 256, 0, st>>>(xd, xc, src, nb, n);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int mp_step(const int32_t *xd, const uint64_t *xc, int32_t *yd, uint64_t *yc, const int32_t *wm, const int32_t *src,
            int nb, int n, uint32_t *flags, uint32_t *status, cudaStream_t st) {
    const dim3 grid((n + kMV - 1) / kMV, (nb + kMS - 1) / kMS);
    k_mp_step<<<grid, kMBlk, 0, st>>>(xd, xc, yd, yc, wm, src, nb, n, flags, status);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int mp_row_hashes(const int32_t *dist, const uint64_t *sig, int nb, int n, uint64_t *h_sigma, uint64_t *h_dist,
                  int64_t *dist_sum, int64_t *reach, int sms, cudaStream_t st) {
    const int g = nb < 4 * sms ? (nb < 1 ? 1 : nb) : 4 * sms;
    k_mp_row_hash<<<g, 256, 0, st>>>(dist, sig, nb, n, h_sigma, h_dist, dist_sum, reach);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int mp_rows(const int32_t *xd, const uint64_t *xc, int nb, int n, int32_t *dist, uint64_t *sig, int sms,
            cudaStream_t st) {
    k_mp_rows<<<grid_for((size_t)nb * n, sms), 256, 0, st>>>(xd, xc, nb, n, dist, sig);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace bcgb
