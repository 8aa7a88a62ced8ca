// pairs.cu -- betweenness from all-pairs distances and path counts with the
// pair formula of Algorithm 2 (Section 4.2.1):
//
//   BC(v) = sum over ordered pairs (s, t), s != v != t, with
//           d(s,v) + d(v,t) = d(s,t), of  lambda_sv * lambda_vt / lambda_st
//
// (lambda = number of shortest paths). The inputs are the forward rows of
// every source: D [n][n] int32 (-1 = unreachable) and Lambda [n][n] uint64.
// With positive weights d = 0 only on the diagonal, so "s != v, t != v"
// is d(s,v) > 0 and d(v,t) > 0, which also excludes unreachable pairs.
//
// k_pair_prep turns Lambda into FP32 lambda and 1/lambda. k_pair_bc: a block
// owns 32 vertices v x 64 targets t and streams the source rows s through
// shared memory 32 at a time; thread (v, t-group) keeps d(v,t) and lambda_vt
// of its 8 targets in registers and adds lambda_sv * lambda_vt / lambda_st
// for every s where the distances add up. Terms are positive; each thread
// adds them in FP32 over one 32-row stage (8 accumulators), then in FP64.
// Block partials go to part[t-block][v]; k_pair_reduce adds them in t-block
// order (deterministic).
#include <cuda_runtime.h>

#include <cstdint>

#include "pairs.cuh"

namespace bcgb {
namespace {

constexpr int kTV = 32;      // vertices per block
constexpr int kTT = 64;      // targets per block
constexpr int kTS = 32;      // source rows per shared-memory stage
constexpr int kTG = 8;       // targets per thread
constexpr int kPBlock = 256; // 8 warps: warp w owns vertices 4w..4w+3, lane = 8 * (v % 4) + t-group

__global__ void __launch_bounds__(256) k_pair_prep(const uint64_t *__restrict__ lam, float *__restrict__ lamf,
                                                   float *__restrict__ rlam, size_t cells) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < cells; i += (size_t)gridDim.x * blockDim.x) {
        const uint64_t x = lam[i];
        const float f = (x >> 32) ? __ull2float_rn(x) : __uint2float_rn((uint32_t)x);
        lamf[i] = f;
        rlam[i] = x ? __frcp_rn(f) : 0.0f;
    }
}

__global__ void __launch_bounds__(kPBlock) k_pair_bc(const int32_t *__restrict__ D, const float *__restrict__ lamf,
                                                     const float *__restrict__ rlam, int n,
                                                     double *__restrict__ part) {
    __shared__ __align__(16) int32_t s_dst[kTS][kTT];
    __shared__ __align__(16) float s_rst[kTS][kTT];
    __shared__ int32_t s_dsv[kTS][kTV];
    __shared__ float s_lsv[kTS][kTV];
    const int v0 = blockIdx.x * kTV, t0 = blockIdx.y * kTT;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int vl = 4 * wid + (lane >> 3);   // local vertex
    const int tg = lane & 7;                // target group: targets t0 + 8 tg .. + 7
    const int v = v0 + vl;
    int32_t dvt[kTG];
    float lvt[kTG];
#pragma unroll
    for (int k = 0; k < kTG; ++k) {
        const int t = t0 + kTG * tg + k;
        const bool in = v < n && t < n;
        dvt[k] = in ? D[(size_t)v * n + t] : -1;
        lvt[k] = in ? lamf[(size_t)v * n + t] : 0.0f;
    }
    double total = 0.0;
    for (int s0 = 0; s0 < n; s0 += kTS) {
        __syncthreads();  // the previous stage's reads are done
        for (int i = tid; i < kTS * kTT; i += kPBlock) {
            const int r = i / kTT, c = i % kTT;
            const int s = s0 + r, t = t0 + c;
            const bool in = s < n && t < n;
            s_dst[r][c] = in ? D[(size_t)s * n + t] : -1;
            s_rst[r][c] = in ? rlam[(size_t)s * n + t] : 0.0f;
        }
        for (int i = tid; i < kTS * kTV; i += kPBlock) {
            const int r = i / kTV, c = i % kTV;
            const int s = s0 + r, vv = v0 + c;
            const bool in = s < n && vv < n;
            s_dsv[r][c] = in ? D[(size_t)s * n + vv] : -1;
            s_lsv[r][c] = in ? lamf[(size_t)s * n + vv] : 0.0f;
        }
        __syncthreads();
        float acc[kTG];
#pragma unroll
        for (int k = 0; k < kTG; ++k) acc[k] = 0.0f;
#pragma unroll 4
        for (int r = 0; r < kTS; ++r) {
            const int32_t dsv = s_dsv[r][vl];
            if (dsv <= 0) continue;  // s = v, or v unreachable from s
            const float lsv = s_lsv[r][vl];
            const int4 *dq = reinterpret_cast<const int4 *>(&s_dst[r][kTG * tg]);
            const float4 *rq = reinterpret_cast<const float4 *>(&s_rst[r][kTG * tg]);
#pragma unroll
            for (int h = 0; h < kTG / 4; ++h) {
                const int4 d4 = dq[h];
                const float4 r4 = rq[h];
                const int32_t dd[4] = {d4.x, d4.y, d4.z, d4.w};
                const float rr[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int k = 4 * h + q;
                    // unsigned: two distances below 2^31 add up below 2^32 - 1,
                    // so the sum never equals an unreachable (-1) d(s,t)
                    if (dvt[k] > 0 && (uint32_t)dsv + (uint32_t)dvt[k] == (uint32_t)dd[q])
                        acc[k] += lsv * (lvt[k] * rr[q]);  // lambda_vt / lambda_st <= 1 / lambda_sv
                }
            }
        }
        float a = 0.0f;
#pragma unroll
        for (int k = 0; k < kTG; ++k) a += acc[k];
        total += (double)a;
    }
    // the 8 target groups of one vertex are lanes 8i..8i+7 of one warp
#pragma unroll
    for (int off = 4; off > 0; off >>= 1) total += __shfl_xor_sync(0xffffffffu, total, off);
    if (tg == 0 && v < n) part[(size_t)blockIdx.y * n + v] = total;
}

__global__ void __launch_bounds__(256) k_pair_reduce(const double *__restrict__ part, int tblocks, int n,
                                                     double *__restrict__ bc) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int b = 0; b < tblocks; ++b) acc += part[(size_t)b * n + v];
        bc[v] += acc;
    }
}

}  // namespace

size_t pair_scratch_bytes(int n) {
    const size_t cells = (size_t)n * n;
    const size_t tb = (size_t)(n + kTT - 1) / kTT;
    return cells * 8 + tb * (size_t)n * 8;  // lamf + rlam, block partials
}

int pair_launch(const int32_t *D, const uint64_t *lam, int n, void *scratch, double *bc, int sms, cudaStream_t st) {
    if (n <= 0) return 0;
    const size_t cells = (size_t)n * n;
    float *lamf = reinterpret_cast<float *>(scratch);
    float *rlam = lamf + cells;
    double *part = reinterpret_cast<double *>(rlam + cells);
    int g = (int)((cells + 255) / 256);
    g = g > 8 * sms ? 8 * sms : g;
    k_pair_prep<<<g, 256, 0, st>>>(lam, lamf, rlam, cells);
    const int tb = (n + kTT - 1) / kTT;
    const dim3 grid((n + kTV - 1) / kTV, tb);
    k_pair_bc<<<grid, kPBlock, 0, st>>>(D, lamf, rlam, n, part);
    int gr = (n + 255) / 256;
    gr = gr > 4 * sms ? 4 * sms : gr;
    k_pair_reduce<<<gr, 256, 0, st>>>(part, tb, n, bc);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace bcgb
