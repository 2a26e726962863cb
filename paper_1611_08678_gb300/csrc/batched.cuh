// Device-side descriptors of the batched path (built on the host by the
// scheduler in api.cu, read by the kernels in batched.cu / far_tc.cu).
#pragma once
#include "common.cuh"

namespace abm {

// One column tile: up to 32 trajectories of one alpha group.
struct TileDesc {
  int traj[kTrajPerTile];  // trajectory index per lane, -1 = padding
  int bucket;              // alpha group
  int n_tile;              // largest N in the tile
  long long f_off;         // element offset of the tile's history in F / F32
};

struct BatchArgs {
  const TileDesc* tiles;   // sorted by n_tile, descending
  int n_tiles;
  int B;                   // time-tile length
  int ksplit;              // history split of the far kernel
  // per alpha group
  const double* bucket_alpha;
  const double* const* bucket_b;
  const double* const* bucket_a;
  const double* const* bucket_c;
  const float* const* bucket_b32;
  const float* const* bucket_a32;
  const double* bucket_g;
  // per trajectory (device)
  const double* h;
  const int* N;
  const double* params;
  const double* y0;
  double* hhat;
  // histories
  double* F;               // FP64, per tile [rows][32*D]
  float* F32;              // FP32 shadow or null
  double* far;             // [ksplit][n_tiles][2][B][32*D]
  // outputs
  double* Y;
  double* YP;
  long long ldY;
  unsigned long long* status;
};

}  // namespace abm
