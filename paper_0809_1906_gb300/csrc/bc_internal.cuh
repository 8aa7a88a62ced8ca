// bc_internal.cuh -- structures shared by the library's translation units.
//
// Layout of the multi-source state in HBM (B = 32*W sources per batch, n
// vertices; every per-vertex row is contiguous so a warp reads a neighbour's
// row in one coalesced access):
//   sigma  uint64 [n][B]        exact path counts sigma_s(v)        (Section 1.1)
//   S      uint16 [s_levels][n][B]  masked rows: sigma_s(v) where d(s,v) = l,
//                               0 for the other sources; one buffer per level
//                               (s_levels = Lcap), or two by level parity
//                               (s_levels = 2)
//   wide   uint32 [Lcap]        level l has a count >= 2^16 (S unusable there)
//   cval   float  [2][n][B]     masked rows by level parity of
//                               c_s(v) = (1 + delta_s*(v)) / sigma_s(v)
//   F      uint32 [Lcap][n][W]  frontier bit of source b at level l (d(s_b, v) = l)
//   ufr    uint32 [Lcap][n/32]  bit v set iff F[l][v] has any bit (union frontier)
//   V      uint32 [2][n][W]     visited bits through level l-1 / l (ping-pong)
//   part   uint64 [slots][B]    partial sums of high-degree vertices split in chunks
//   pmask  uint32 [slots][W]    partial next-frontier words of those chunks
//   cnt    uint32 [slots]       arrival counters (indexed by a vertex's first slot)
#pragma once

#include <cstddef>
#include <cstdint>

#include "../../include/bc_gb300.h"

namespace bcgb {

// Device-side control block of a graph (device memory).
struct DevCtl {
    uint32_t status;       // BC_STATUS_* bits, sticky for one bc_run
    uint32_t fwd_done;     // 1 once the running batch's forward pass ended
    int32_t nlevels;       // deepest non-empty level of the running batch
    uint32_t nonempty;     // OR over blocks: next frontier not empty
    uint32_t blocks_done;  // arrival counter for last-block detection
    uint32_t seq;          // batch sequence number
    uint32_t pad[2];
    unsigned long long dag_arcs;  // sum over the run's sources of |{(u,v): u in P_s(v)}|
    unsigned long long depth_sum; // sum over batches (or sources) of the BFS depth
    unsigned long long batch_arcs; // the running batch's arcs, added to dag_arcs when its forward
                                   // pass ends (a batch restarted with more levels counts once)
    uint32_t front_new;   // vertices put into the next frontier so far (summed over blocks)
    uint32_t front_last;  // vertices in the newest complete frontier
};

// Host-mapped block the host polls while the level loop runs (pinned). Each
// word is written with one 64-bit relaxed store at system scope, the batch
// sequence number in its high half and the value in its low half, so the host
// learns both from one read: nothing has to be ordered, and the last block of
// a level does not wait for its writes to reach host memory.
struct HostCtl {
    unsigned long long done;      // (seq << 32) | depth L once the forward pass ended (-1: level capacity hit)
    unsigned long long progress;  // (seq << 32) | number of forward levels completed
    unsigned long long counts;    // (vertices in the newest frontier << 32) | (in the one before), each
                                  // -1 when not counted; a hint for the host's look-ahead only
    unsigned long long pad;
};

#ifdef __CUDACC__
__device__ __forceinline__ void host_word(unsigned long long *w, uint32_t hi, uint32_t lo) {
    const unsigned long long x = ((unsigned long long)hi << 32) | lo;
    asm volatile("st.relaxed.sys.global.u64 [%0], %1;" ::"l"(w), "l"(x) : "memory");
}

// hi + lo += x with Knuth's two-sum: the rounding error of hi + x, which is
// exact in FP32, goes into lo. For k terms, all >= 0, the sum's error stays
// below about k^2 2^-48 of the sum (2^-32 for a 256-source batch; a plain FP32
// sum's bound is k 2^-24), in FP32 arithmetic only: GB300's FP64 rate is a
// small fraction of its FP32 rate, so the FP64 units take just the one add
// into BC(v) per vertex and level.
__device__ __forceinline__ void two_sum_add(float &hi, float &lo, float x) {
    const float s = hi + x;
    const float bp = s - hi;
    const float err = (hi - (s - bp)) + (x - bp);
    hi = s;
    lo += err;
}
#endif

struct MsParams {
    int32_t n;
    int32_t nitems;
    int32_t nw32;  // words of one union-frontier bitmap
    int32_t Lcap;  // level slots in F / ufr
    int32_t nb;    // sources in this batch (<= B)
    int32_t first; // level 1 was produced by k_first (all its counts are 1)
    int64_t first_arcs;  // arcs out of this batch's sources (0: not counted; sizes k_first's grid)
    uint32_t seq;
    const int32_t *row_ptr;  // out-arcs: level 0->1 and the backward sweep
    const int32_t *col;
    const int32_t *col_f;    // arcs the forward sweep pulls over: in-arcs (= col when undirected)
    const int32_t *item_v;
    const int32_t *item_beg;
    const int32_t *item_end;
    const int32_t *item_slot;   // -1: whole vertex; else partial slot of a chunk
    const int32_t *slot_first;  // first slot of the chunk's vertex
    const int32_t *slot_nch;    // number of chunks of that vertex
    const int32_t *sources;     // this batch's source ids [nb]
    uint64_t *sigma;
    uint16_t *S;   // [s_levels][n][B]
    int32_t s_levels;  // Lcap: level l in buffer l, which the backward reads for sigma; 2: by parity
    const uint16_t *S_rd;  // set per forward launch: the buffer of level l (read)
    uint16_t *S_wr;        // and of level l+1 (written)
    uint32_t *wide;  // [Lcap]
    uint32_t *lsize;  // [Lcap] or null: vertices in frontier l (written as the forward reaches it)
    float *cval;   // [2][n][B]
    uint32_t *F;
    uint32_t *ufr;
    uint32_t *V;
    uint64_t *part;
    uint32_t *pmask;
    uint32_t *cnt;
    uint64_t wait_ns;         // bound on each device wait for staged rows (0: 2 s)
    uint32_t test_hold;       // bytes every staged round expects beyond its copies (timeout test hook)
    double *bc;
    uint64_t *h_sigma;  // per-source summaries, indexed from this batch's first source
    uint64_t *h_dist;
    int64_t *dist_sum;
    int64_t *reach;
    const int32_t *out_index;  // may be null: summary of batch source b goes to index out_index[b]
    DevCtl *ctl;
    HostCtl *hctl;  // device pointer of the host-mapped block
};

// Launchers (msbfs.cu). W = words per vertex row (B = 32 W).
bool ms_supported_width(int W);
void ms_launch_init(int W, const MsParams &p, cudaStream_t st);
void ms_launch_first(int W, const MsParams &p, cudaStream_t st);  // level 0 -> 1
void ms_launch_forward(int W, const MsParams &p, int level, cudaStream_t st);
void ms_launch_backward(int W, const MsParams &p, int level, cudaStream_t st);
void ms_launch_hash(int W, const MsParams &p, int nlevels, cudaStream_t st);
void ms_launch_rows(int W, const MsParams &p, int nlevels, uint64_t *sig_out, int32_t *dist_out,
                    cudaStream_t st);
void launch_scale(double *x, int32_t n, double f, cudaStream_t st);
// dst[i] += src[i] for i < n; unless from is null, to's status |= from's and
// its arc and depth sums += from's
void ms_launch_merge(const double *src, double *dst, int32_t n, const DevCtl *from, DevCtl *to, cudaStream_t st);

}  // namespace bcgb
