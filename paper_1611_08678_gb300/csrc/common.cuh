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

// Sites of a bounded wait that ran out (bits 56..59 of an ABM_ERR_TIMEOUT
// status word; bits 32..55 hold the index of the unit that waited, bits 0..31
// a position inside it).
enum TimeoutSite : int {
  kSiteSingleNear = 1,    // single trajectory: stepping CTA waiting for tile `index`'s far sums
  kSiteSingleFar = 2,     // single trajectory: far CTA waiting for the rows before tile `index`
  kSiteFarProducer = 3,   // tensor-core far kernel, column tile `index`: loader after `pos` loads
  kSiteFarAccum = 4,      // ... MMA issuer waiting for accumulator chunk `pos` to drain
  kSiteFarLoad = 5        // ... MMA issuer waiting for the operands of K block `pos`
};

__device__ __forceinline__ void report_timeout(unsigned long long* status, int site, long long index,
                                               long long pos) {
  unsigned long long w = ((unsigned long long)ABM_ERR_TIMEOUT << 60) | ((unsigned long long)(site & 0xF) << 56) |
                         (((unsigned long long)index & 0xFFFFFFull) << 32) | ((unsigned long long)pos & 0xFFFFFFFFull);
  atomicCAS(status, 0ull, w);
}

// ---- checked build (compiled with ABM_CHECKED) ----
// Every index a kernel derives from the host's layout (tile offsets, leading
// dimensions, lags, tensor-map coordinates, partial-sum slots) is compared
// with the extent of the buffer it addresses; an index outside is not
// accessed, and the first one is reported as ABM_ERR_BOUNDS with the site in
// bits 52..59 and the index in bits 0..51 of the status word.  Without
// ABM_CHECKED in_bounds() is the constant true and costs nothing.
#ifdef ABM_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

enum CheckSite : int {
  kChkSetup = 1, kChkNear = 2, kChkNearSplit = 3, kChkFarFp64 = 4, kChkFarFp32 = 5, kChkFarPerComp = 6,
  kChkFarTc = 7, kChkSingle = 8, kChkImport = 9, kChkExport = 10, kChkAdjoint = 11, kChkWeights = 12
};

__device__ __forceinline__ bool in_bounds(unsigned long long* status, int site, long long idx, long long extent) {
  if constexpr (!kChecked) {
    return true;
  } else {
    if (idx >= 0 && idx < extent) return true;
    unsigned long long w = ((unsigned long long)ABM_ERR_BOUNDS << 60) | ((unsigned long long)(site & 0xFF) << 52) |
                           ((unsigned long long)idx & 0xFFFFFFFFFFFFFull);
    atomicCAS(status, 0ull, w);
    return false;
  }
}

// x is neither infinite nor NaN: an exponent-bit test on the integer pipe
// (GB300's FP64 pipe is the bottleneck of the sequential steps).
__device__ __forceinline__ bool finite_bits(double x) {
  return (__double2hiint(x) & 0x7ff00000) != 0x7ff00000;
}

// Sum of ks FP64 partials p[0], p[stride], ...: starts from the first one (an
// explicit 0.0 + p[0] would cost an FP64 add).
__device__ __forceinline__ double sum_parts(const double* p, int ks, size_t stride) {
  double v = p[0];
  for (int q = 1; q < ks; ++q) v += p[q * stride];
  return v;
}

// Parameters of one trajectory passed by value (single-trajectory path).
struct TrajParams {
  double p[kMaxParams];
  double y0[kMaxD];
  double y0d[kMaxD];  // initial derivatives y'(0), used by components of order above one
};

}  // namespace abm
