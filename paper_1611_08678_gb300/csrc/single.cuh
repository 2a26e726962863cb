// Argument blocks and launchers of the single-trajectory kernels (single.cu).
#pragma once
#include "common.cuh"

namespace abm {

struct FarSingleArgs {
  const double* F;      // rows x D
  const double* b;      // FP64 weights
  const double* a;
  long long s;          // first target step of the tile
  long long k_lo, k_hi; // history rows
  long long chunk;      // rows per CTA
  double* partial;      // [gridDim.x][B][2D]
  double* out;          // [B][2D]: P then C per row
  unsigned int* ticket; // zero before the launch, reset to zero by the last CTA
};

// Persistent single-trajectory kernel (single_persistent.cu).
constexpr int kPersistB = 32;  // time-tile length
constexpr int kPersistRing = 4;

struct PersistArgs {
  double* F;                   // (N+1) x D history, FP64
  double* Y;                   // (N+1) x D
  double* YP;                  // (N+1) x D or null
  // weights per state component (all equal for a commensurate order): b_m,
  // a_m, c_m over lags 0..N+2B+1 and g = 1/Gamma(alpha+2)
  const double* b[kMaxD];
  const double* a[kMaxD];
  const double* c[kMaxD];
  const double* g[kMaxD];
  double* partial;             // [kPersistRing][grid-1][kPersistB][2D]
  unsigned long long* flags;   // [0] rows_done, [1..kPersistRing] far counts; zero at launch
  unsigned long long* status;
  TrajParams tp;
  double alpha[kMaxD];         // order per component (alpha[0] also enters the manufactured f)
  double h;
  int taylor_mask;             // bit c: component c has order above one (y'(0) t in its Taylor sum)
  int N;
  long long spin_budget;       // clock64 cycles per wait
  int withhold_tile;           // testing: far CTAs never count this tile (-1 = off)
  int passes;                  // corrector passes per step (1 = PECE)
  int start_tile;              // resume: first time tile stepped; F rows 0..start_tile*B hold
                               // the history of an earlier solve (0 = a fresh solve)
  long long f_elems, w_elems, partial_elems;  // extents of F, each weight vector, partial (checked build)
};

cudaError_t launch_far_single(int d, const FarSingleArgs& A, int B, int grid, cudaStream_t st);
// nc = 1: one weight set for every component; nc = d: one per component.
cudaError_t launch_persistent(int sys, int nc, const PersistArgs& A, int grid, cudaStream_t st);
int persistent_max_grid(int sys);
size_t persistent_smem_bytes();

}  // namespace abm
