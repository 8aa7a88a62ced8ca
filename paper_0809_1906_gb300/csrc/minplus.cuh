// minplus.cuh -- distance products with path counts (minplus.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace bcgb {

constexpr int32_t kMpInf = 0x3FFFFFFF;  // "no walk": every distance must stay below it

// wm [n][n] = weight of arc (u, v), kMpInf where there is none.
int mp_build_weights(const int32_t *rp, const int32_t *col, const int32_t *w, int n, int32_t *wm, int sms,
                     cudaStream_t st);
// X[b][v] = (0, 1) at v = src[b], (inf, 0) elsewhere.
int mp_init(int32_t *xd, uint64_t *xc, const int32_t *src, int nb, int n, int sms, cudaStream_t st);
// One product step X -> Y; flags |= 1 when Y != X; a count carry out of bit 63
// sets BC_STATUS_SIGMA_OVERFLOW in status.
int mp_step(const int32_t *xd, const uint64_t *xc, int32_t *yd, uint64_t *yc, const int32_t *wm, const int32_t *src,
            int nb, int n, uint32_t *flags, uint32_t *status, cudaStream_t st);
// Per-source summaries (hash of sigma and of distances, distance sum, reach)
// of nb full rows.
int mp_row_hashes(const int32_t *dist, const uint64_t *sig, int nb, int n, uint64_t *h_sigma, uint64_t *h_dist,
                  int64_t *dist_sum, int64_t *reach, int sms, cudaStream_t st);
// Rows: dist -1 and count 0 where unreachable (either output may be null).
int mp_rows(const int32_t *xd, const uint64_t *xc, int nb, int n, int32_t *dist, uint64_t *sig, int sms,
            cudaStream_t st);

}  // namespace bcgb
