// sched.cuh -- host side of the level loop shared by the batched and the
// one-source paths.
//
// The depth of a BFS is known only when a level comes out empty. Rather than
// synchronising after every level, the host launches level kernels a few
// levels ahead of the device (a launch past the end exits at once on a device
// flag) and polls a pinned, host-mapped block that the last block of every
// level kernel updates with system-scope fences. Every wait is bounded by a
// wall-clock limit and also stops on a device error.
#pragma once

#include <cuda_runtime.h>

#include <chrono>
#include <string>
#include <thread>

#include "bc_internal.cuh"

namespace bcgb {

constexpr int kLookahead = 3;

inline uint32_t load_acquire_u(const uint32_t *p) { return __atomic_load_n(p, __ATOMIC_ACQUIRE); }
inline int32_t load_acquire_i(const int32_t *p) { return __atomic_load_n(p, __ATOMIC_ACQUIRE); }

// launch(level) enqueues the kernel of forward level `level`; levels
// 0..max_level may be launched. On BC_OK, *depth is the depth reported by the
// device (-1: the level capacity was too small).
template <class Launch>
int drive_forward(const HostCtl *hctl, uint32_t seq, int max_level, Launch &&launch, int64_t wait_ms,
                  cudaStream_t st, std::string *err, int *depth) {
    int launched = 0;
    const auto t0 = std::chrono::steady_clock::now();
    for (long spins = 0;; ++spins) {
        int done_lv = 0;
        if (load_acquire_u(&hctl->progress_seq) == seq) done_lv = load_acquire_i(&hctl->progress);
        bool issued = false;
        while (launched <= max_level && launched < done_lv + kLookahead) {
            launch(launched++);
            issued = true;
        }
        if (issued) {
            const cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) {
                *err = std::string("level kernel launch: ") + cudaGetErrorString(e);
                return BC_ERR_CUDA;
            }
        }
        if (load_acquire_u(&hctl->done_seq) == seq) {
            *depth = load_acquire_i(&hctl->nlevels);
            return BC_OK;
        }
        if (spins % 64 == 63) {
            const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(
                                std::chrono::steady_clock::now() - t0)
                                .count();
            if (ms > wait_ms) {
                *err = "the device did not report the end of a forward pass within the wait limit";
                return BC_ERR_TIMEOUT;
            }
            const cudaError_t e = cudaStreamQuery(st);
            if (e != cudaSuccess && e != cudaErrorNotReady) {
                *err = std::string("device error during a forward pass: ") + cudaGetErrorString(e);
                return BC_ERR_CUDA;
            }
            if (e == cudaSuccess && load_acquire_u(&hctl->done_seq) != seq && launched > max_level) {
                *err = "forward pass ended without reporting its depth";
                return BC_ERR_STATE;
            }
            if (spins % 4096 == 4095) std::this_thread::yield();
        }
    }
}

}  // namespace bcgb
