// Device-side descriptors of the batched path (built on the host by the
// scheduler in api.cu, read by the kernels in batched.cu / far_tc.cu).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>

#include "common.cuh"

namespace abm {

// One column tile: up to 32 trajectories of one alpha group.
struct TileDesc {
  int traj[kTrajPerTile];  // trajectory index per lane, -1 = padding
  int bucket;              // alpha group
  int n_tile;              // largest N in the tile
  int slot;                // the tile's place in the split history pieces (Fsh / Xsh): its
                           // index in the N-sorted tile table (2t + hist for adjoint tiles)
  long long f_off;         // element offset of the tile's history in F / F32
};

struct BatchArgs {
  const TileDesc* tiles;   // sorted by n_tile, descending
  int n_tiles;
  int B;                   // time-tile length
  int ksplit;              // history split of the far kernel
  int far_k0;              // first history row of the far sums: 1 forward (row 0 = the
                           // j = 0 term, kept in FP64), 0 adjoint
  int per_comp;            // 1: some group's orders differ per component (the SIMT far
                           // kernels then take one weight set per component)
  // per order group (trajectories with the same orders) and state component:
  // entry [group * kMaxD + component]
  const double* bucket_alpha;
  const double* const* bucket_b;
  const double* const* bucket_a;
  const double* const* bucket_c;
  const float* const* bucket_b32;
  const float* const* bucket_a32;
  const double* bucket_g;
  const int* bucket_taylor;  // per group: bit c = component c has order above one
  // per trajectory (device)
  const double* h;
  const int* N;
  const double* params;
  const double* y0;
  const double* y0d;       // initial derivatives [M][D] (orders above one) or null
  double* hhat;            // h^alpha per trajectory and component, [M][kMaxD]
  // histories
  double* F;               // FP64, per tile [rows][32*D]
  float* F32;              // FP32 shadow or null
  __nv_bfloat16* Fsh;      // BF16 split history or null, K-block tiled: piece p, column tile t,
                           // K block kb = k / 64 is the contiguous [96 columns][64 rows] block
                           // at ((t * fsh_ld / 64 + kb) * 96 + col) * 64 + k % 64
  long long fsh_ld;        // history rows per column of Fsh (a multiple of 64)
  long long fsh_plane;     // elements per split piece
  double* far;             // [ksplit][n_tiles][2][B][32*D]
  unsigned int* far_ticket;  // per tile, zero between launches: the SIMT far kernels' last
                           // CTA of a tile adds the ksplit partials into slot 0
  // outputs
  double* Y;
  double* YP;
  long long ldY;
  unsigned long long* status;
  int passes;              // corrector passes per step (1 = PECE)
  long long resume_row;    // resume: history rows 0..resume_row were imported and Y rows up
                           // to it are the caller's (0 = a fresh solve)
  // extents of the buffers above, in elements (checked build)
  long long f_elems, w_elems, far_elems, y_elems, fsh_plane_elems;
  int bad_traj;            // testing (checked build): trajectory whose output row is offset, -1 = off
};

// Arguments of the tensor-core far kernel (far_tc.cu).
struct FarTcArgs {
  const TileDesc* tiles;
  const CUtensorMap* tmapW;  // [bucket][3]: pre-expanded Toeplitz pieces hi, mid, lo
  const CUtensorMap* tmapF;  // [3]: BF16 split history pieces
  double* far;               // [n_tiles][2][64][96] sums; ksplit > 1: zeroed before the
                             // launch, the CTAs of a tile add their parts with FP64 atomics
  unsigned long long* status;
  long long s;               // time tile start (multiple of 64)
  long long Lbase;           // x offset base of the pre-expanded Toeplitz
  long long budget;          // clock cycles per bounded wait
  int n_tiles;
  int ksplit;
  int f_kblocks;             // 64-row K blocks per column tile in the history pieces
  // extents (checked build): rows of the history and Toeplitz tensor maps,
  // elements of far
  long long f_map_rows, w_map_rows, far_elems;
};

// Arguments of the adjoint kernels (adjoint.cu).
struct AdjArgs {
  const TileDesc* tiles;   // forward column tiles (sorted by n_tile descending)
  const TileDesc* atiles;  // adjoint tiles: 2t = mu~ history, 2t+1 = lambda~ history
  int B;
  // tables as in BatchArgs ([group * kMaxD + component]); the adjoint takes
  // commensurate orders and reads component 0
  const double* bucket_alpha;
  const double* const* bucket_b;
  const double* const* bucket_a;
  const double* const* bucket_c;
  const double* bucket_g;
  const double* h;
  const int* N;
  const double* params;
  const double* y0;
  double* hhat;            // [M][kMaxD], component 0 used
  const double* Y;
  const double* YP;
  const double* G;
  long long ldY;
  double* X;               // FP64 adjoint histories, tile t at atiles[t].f_off, [rows][32*D]
  __nv_bfloat16* Xsh;      // BF16 split planes of the adjoint histories (tensor paths) or null
  long long xsh_ld, xsh_plane;
  const double* far;       // far sums: [ksplit][far_tiles][2][B][32*D]
  int far_ksplit, far_tiles;
  double* acc_dp;          // [M][D][NP]
  double* acc_dy0;         // [M][D]
  double* phi0c;           // [M][D] running sum_n c_{n-1} lambda_n
  double* dparams;         // [M][NP] (written by the finish kernel)
  double* dy0;             // [M][D]
  unsigned long long* status;
};

}  // namespace abm
