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

inline unsigned long long load_word(const unsigned long long *p) { return __atomic_load_n(p, __ATOMIC_ACQUIRE); }

// The value of a HostCtl word written for batch `seq`, or false when the word
// still belongs to an earlier batch.
inline bool word_for(const unsigned long long *p, uint32_t seq, int32_t *value) {
    const unsigned long long w = load_word(p);
    if ((uint32_t)(w >> 32) != seq) return false;
    *value = (int32_t)(uint32_t)w;
    return true;
}

// Levels to launch ahead of the last completed one: kLookahead, or one once
// the newest frontier is small (at most `small` vertices; the level
// kernels publish the counts) and under half the one before it: the pass is
// then about to end, and a launch past its end still costs a grid's start-up.
// A frontier that stays small without shrinking (a long path, a grid) keeps
// the full look-ahead.
inline int lookahead(const HostCtl *h, int32_t small) {
    const unsigned long long w = load_word(&h->counts);
    const int32_t c = (int32_t)(uint32_t)(w >> 32), c0 = (int32_t)(uint32_t)w;
    return (c >= 0 && c <= small && c0 >= 0 && 2 * (int64_t)c < (int64_t)c0) ? 1 : kLookahead;
}

// launch(level) enqueues the kernel of forward level `level`; levels
// 0..max_level may be launched. On BC_OK, *depth is the depth reported by the
// device (-1: the level capacity was too small).
template <class Launch>
int drive_forward(const HostCtl *hctl, uint32_t seq, int max_level, Launch &&launch, int64_t wait_ms,
                  cudaStream_t st, std::string *err, int *depth, int32_t small = -1) {
    int launched = 0;
    const auto t0 = std::chrono::steady_clock::now();
    for (long spins = 0;; ++spins) {
        int done_lv = 0, ahead = kLookahead;
        if (word_for(&hctl->progress, seq, &done_lv)) ahead = lookahead(hctl, small);
        bool issued = false;
        while (launched <= max_level && launched < done_lv + ahead) {
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
        if (word_for(&hctl->done, seq, depth)) return BC_OK;
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
            int dummy = 0;
            if (e == cudaSuccess && !word_for(&hctl->done, seq, &dummy) && launched > max_level) {
                *err = "forward pass ended without reporting its depth";
                return BC_ERR_STATE;
            }
            if (spins % 4096 == 4095) std::this_thread::yield();
        }
    }
}

}  // namespace bcgb
