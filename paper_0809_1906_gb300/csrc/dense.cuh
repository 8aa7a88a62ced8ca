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

struct DenseParams {
    int32_t n, npad, nb, nw32;
    uint64_t *sigma;  // [n][128]
    uint16_t *lvl;    // [n][128]
    uint32_t *F, *V, *ufr;
    __nv_bfloat16 *X;  // [8 * 128][npad] limb matrix (backward: two blocks of 3 * 128 split rows)
    double *bc;
    DevCtl *ctl;
    DenseCtl *dctl;
};

struct DenseMaps {
    CUtensorMap x, a;
};

int dense_build_adjacency(const int32_t *row_ptr, const int32_t *col, int32_t n, int32_t npad, __nv_bfloat16 *A,
                          cudaStream_t st);
int dense_make_maps(DenseMaps *maps, __nv_bfloat16 *X, __nv_bfloat16 *A, int32_t npad);
int dense_launch_level(const DenseMaps &maps, const DenseParams &p, int l, int nl, cudaStream_t st);
// Backward levels L-1 .. 1 on the tensor cores (BC accumulated into p.bc).
int dense_launch_backward(const DenseMaps &maps, const DenseParams &p, int L, cudaStream_t st);

}  // namespace bcgb
