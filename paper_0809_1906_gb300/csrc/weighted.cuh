// weighted.cuh -- parameters of the weighted (integer delta-stepping) path.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "bc_internal.cuh"

namespace bcgb {

constexpr int kMaxRing = 4096;  // bucket ring size limit: max weight < kMaxRing

struct WParams {
    int32_t n;
    int32_t K;     // ring size (> max weight)
    int32_t C;     // entry capacity of one bucket
    int32_t dmax;  // bound on any distance (n * max weight), a loop guard
    const int32_t *row_ptr;
    const int32_t *col;
    const int32_t *row_ptr_in;  // directed graphs: in-arc CSR for P_s(v) (null when undirected)
    const int32_t *col_in;
    const int32_t *w_in;
    const int32_t *w;
    const int32_t *sources;  // this wave's sources
    const int32_t *vid;      // the caller's id of each vertex when the graph was relabelled (null: the same);
                             // summaries and rows use the caller's ids
    const int32_t *pos;      // position of each CTA's source in the summaries and rows (null: its index);
                             // delta rows are always at the CTA's index
    uint64_t *ds;            // [wave][n] packed state (distance << 32 | sigma or c bits)
    uint8_t *redo;           // [wave] set where a count reached 2^32 (packed kernel; that source writes nothing)
    int32_t *dist;           // [wave][n]
    uint64_t *sigma;         // [wave][n]
    float *cval;             // [wave][n]
    int32_t *order;          // [wave][n] settle order
    int32_t *grp;            // [wave][n+1] start of each distinct-distance group in order
    int32_t *slots;          // [wave][K][C] bucket entries
    float *delta_rows;       // [wave][n] delta_s*(v) per source (null: forward only)
    uint64_t *h_sigma;       // per-source summaries, indexed by wave position (or null)
    uint64_t *h_dist;
    int64_t *dist_sum;
    int64_t *reach;
    uint64_t *rows_sigma;    // optional rows [wave][n]
    int32_t *rows_dist;
    DevCtl *ctl;
};

// relabel.cu: perm[v] = v's id in a numbering with locality (multilevel
// heavy-edge matching over the CSR; host code), and out[i] = perm[in[i]]
// for i < k on the device.
void locality_order(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t *perm);
void launch_map_ids(const int32_t *perm, const int32_t *in, int32_t *out, int32_t k, cudaStream_t st);

void w_launch_wave(const WParams &p, int nsrc, cudaStream_t st);         // 64-bit counts
void w_launch_wave_packed(const WParams &p, int nsrc, cudaStream_t st);  // packed state, 32-bit counts
// Threads per source of the packed kernel: a distance step settles about n /
// (distinct distances) vertices, so small graphs leave wide CTAs idle at every
// barrier while large ones need the threads. Square grids with 5% long-range
// edges, best wave of each (ms): n = 4096 (all sources) 128 threads 18.1, 512
// threads 58.2; n = 16384 (2048 sources) 11.8 / 35.0; n = 65536 30.5 / 41.0;
// n = 262144 146.4 / 123.4. The switch sits between the last two sizes.
constexpr int32_t kWSmallN = 131072;
int w_packed_threads(int32_t n);
// bc[vid[v]] += the FP64 sum over r < nrows of rows[r][v], rows in order (vid null: bc[v])
void w_launch_reduce(const float *rows, int nrows, int n, const int32_t *vid, double *bc, int sms,
                     cudaStream_t st);

}  // namespace bcgb
