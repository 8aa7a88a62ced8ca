// pairs.cuh -- Algorithm 2's pair formula on all-pairs rows (pairs.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace bcgb {

// Scratch for pair_launch on n vertices (bytes).
size_t pair_scratch_bytes(int n);

// BC[v] += sum_{s != v != t, d(s,v)+d(v,t)=d(s,t)} lambda_sv lambda_vt / lambda_st
// over every ordered pair, from D [n][n] (-1 unreachable) and lambda [n][n].
// Returns 0, or -1 when a launch failed.
int pair_launch(const int32_t *D, const uint64_t *lam, int n, void *scratch, double *bc, int sms,
                cudaStream_t st);

}  // namespace bcgb
