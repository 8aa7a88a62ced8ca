// dense.cuh -- parameters of the tensor-core level expansion (dense.cu).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "bc_internal.cuh"

namespace bcgb {

constexpr int kDenseMaxLimbs = 8;     // 8-bit limbs of a uint64 path count
constexpr int kDenseMaxN = 65536;     // 255 * n < 2^24 keeps FP32 sums exact

struct DenseCtl {
    unsigned produced;             // some (source, vertex) reached at this level
    unsigned pad;
    unsigned long long maxsig;     // largest new path count (fixes the next limb count)
    unsigned long long remaining;  // (source, vertex) pairs still unreached
};

// A group of batches processed level by level in lockstep: every batch keeps
// its own state slice (batch b at offset b * stride), one launch per level
// covers (active batch, 64-vertex tile) pairs.
struct DenseParams {
    int32_t n, npad, nw32, Lcap;
    int32_t nactive;        // batches in this launch (blist[0 .. nactive))
    int32_t group;          // batches that share each adjacency tile in turn (L2 reuse)
    const int32_t *blist;   // active batch ids
    const int32_t *nbs;     // valid sources of each batch (<= 128)
    const int32_t *depth;   // backward: depth L of each batch
    size_t sig_stride;      // sigma: n * 128
    size_t f_stride;        // F: Lcap * n * 4
    size_t v_stride;        // V: 2 * n * 4
    size_t u_stride;        // ufr: Lcap * nw32
    int32_t xrows;          // X rows per batch
    uint64_t *sigma;        // [batch][n][128]
    uint32_t *F, *V, *ufr;
    __nv_bfloat16 *X;       // [batch][xrows][npad]: limb rows (forward) or two blocks of 3 x 128 split rows
    double *bcpart;         // [batch][n] BC contributions of each batch (added in batch order later)
    DevCtl *ctl;
    DenseCtl *dctl;         // [batch]
    // per-source summaries (may be null): the backward levels and the deepest
    // level's split add the terms of the pairs they visit, the split also the
    // sources' own (level 0); batch b's source j goes to index src_base + 128 b + j
    const int32_t *sources;  // the group's sources, 128 per batch
    int32_t src_base;
    uint64_t *h_sigma, *h_dist;
    int64_t *dist_sum, *reach;
};

struct DenseMaps {
    CUtensorMap x, a, a_wide;  // K = 64 boxes (128-byte swizzle); adjacency boxes of 64 and 128 rows
    CUtensorMap x32, a_wide32; // K = 32 boxes (64-byte swizzle)
    CUtensorMap a_x, a_x32;    // adjacency boxes of 256 rows, K = 64 and 32 (when npad is a multiple of 256)
    CUtensorMap x8, a8;        // e4m3 operands: 128-byte rows, X (4-bit limbs) and adjacency boxes of 128 rows
    bool has_f8;
};

constexpr int kDenseXRows = kDenseMaxLimbs * 128;  // X rows per batch (>= 2 x 3 x 128 for the backward)

int dense_build_adjacency(const int32_t *row_ptr, const int32_t *col, int32_t n, int32_t npad, __nv_bfloat16 *A,
                          cudaStream_t st);
// The adjacency in e4m3 (A8 [npad][npad] bytes, 1.0 where an arc is).
int dense_build_adjacency8(const int32_t *row_ptr, const int32_t *col, int32_t n, int32_t npad, uint8_t *A8,
                           cudaStream_t st);
// Maps for X ([xrows_total][npad]), A ([npad][npad]) and, when A8 is not null,
// the e4m3 views of X and A8.
int dense_make_maps(DenseMaps *maps, __nv_bfloat16 *X, uint64_t xrows_total, __nv_bfloat16 *A, uint8_t *A8,
                    int32_t npad);
// Forward level l -> l+1 for the p.nactive batches of p.blist (limbs, then
// the product): nl 8-bit limbs of the level's counts, or nq <= 4 4-bit ones
// in e4m3 when the maps have that form.
int dense_launch_level(const DenseMaps &maps, const DenseParams &p, int l, int nl, int nq, cudaStream_t st);
// Whether dense_launch_level takes the e4m3 form for nq 4-bit limbs.
bool dense_level_f8(const DenseMaps &maps, int nq);
// Levels 0 and 1 of batches 0 .. nbatch (sources: 128 per batch, in batch
// order): zeroes the group's frontier, visited and union-frontier words, then
// sets the sources and their neighbours.
int dense_launch_first(const DenseParams &p, int nbatch, const int32_t *sources, const int32_t *row_ptr,
                       const int32_t *col, cudaStream_t st);
// Split c rows of each batch's deepest level (batches 0 .. nbatch).
int dense_launch_bwd_last(const DenseParams &p, int nbatch, cudaStream_t st);
// Backward level l for the p.nactive batches with depth > l (BC into p.bcpart).
int dense_launch_bwd_level(const DenseMaps &maps, const DenseParams &p, int l, cudaStream_t st);
// bc[v] += sum over batches 0 .. nbatch of bcpart[b][v], in batch order.
int dense_reduce_bc(const double *bcpart, int nbatch, int n, double *bc, cudaStream_t st);

}  // namespace bcgb
