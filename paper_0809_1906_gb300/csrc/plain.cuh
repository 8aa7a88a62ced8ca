// plain.cuh -- the one-source-at-a-time GPU Brandes (flag BC_PLAIN): the
// unbatched comparator for the multi-source path.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "bc_internal.cuh"

namespace bcgb {

// Launch accounting callback: begin(ctx, kind) before a launch returns a
// token that end(ctx, token) receives after it.
struct LaunchHook {
    void *ctx;
    size_t (*begin)(void *ctx, int kind);
    void (*end)(void *ctx, size_t token);
};

struct PlainState {
    int32_t n = 0;
    int32_t *dist = nullptr;
    uint64_t *sigma = nullptr;
    float *cval = nullptr;
    int32_t *queue = nullptr;
    int32_t *level_off = nullptr;  // [n + 2]: level l occupies queue[level_off[l], level_off[l+1])
    uint32_t *tail = nullptr;
};

void plain_free(PlainState &s);

int plain_run(PlainState &s, int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *sources,
              int32_t nsrc, double *bc, uint64_t *h_sigma, uint64_t *h_dist, int64_t *dist_sum, int64_t *reach,
              DevCtl *ctl, HostCtl *hctl_host, HostCtl *hctl_dev, uint32_t *seq, cudaStream_t st,
              const LaunchHook &hook, int64_t wait_ms, std::string *err);

}  // namespace bcgb
