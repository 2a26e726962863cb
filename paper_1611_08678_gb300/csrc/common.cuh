// Shared definitions of the CUDA library: status word, launch helpers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/abm.h"

namespace abm {

constexpr int kMaxD = 3;        // largest state dimension of a built-in system
constexpr int kMaxParams = 9;   // largest parameter count of a built-in system
constexpr int kTrajPerTile = 32;  // trajectories per column tile (one warp of the near kernel)

// Device status word: code in bits 60..63, trajectory in 32..59, step in 0..31.
// The first error of a call wins (atomicCAS from zero).
__device__ __forceinline__ void report_status(unsigned long long* status, int code, long long traj,
                                              long long step) {
  unsigned long long w = ((unsigned long long)code << 60) |
                         (((unsigned long long)traj & 0x0FFFFFFFull) << 32) |
                         ((unsigned long long)step & 0xFFFFFFFFull);
  atomicCAS(status, 0ull, w);
}

// Parameters of one trajectory passed by value (single-trajectory path).
struct TrajParams {
  double p[kMaxParams];
  double y0[kMaxD];
};

}  // namespace abm
