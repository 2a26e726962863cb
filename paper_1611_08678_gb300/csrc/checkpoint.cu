// History checkpoint and resume of the batched path (abm_history_batched,
// abm_solve_batched_resume).  The state of the scheme at step n is y(0),
// y'(0) and the f history f_0..f_n (Sec. 2: every later step reads the whole
// history); these kernels move f rows between the per-trajectory layout the
// caller keeps, [M][ldF][D], and the plan's column-tile layout (time-major
// rows of 32 trajectories x D columns), including the shadows the far kernels
// stream: the FP32 copy and the BF16 split pieces (K-block tiled, row 0 zero:
// the j = 0 terms stay FP64).
#include "batched.cuh"
#include "bf16split.cuh"
#include "common.cuh"

namespace abm {

// Rows 0..s0 of every trajectory into its tile (padding lanes take lane 0's
// trajectory, as the stepping kernels do).  One thread per (tile, row, column).
template <int D>
__global__ void import_history_kernel(BatchArgs A, int n_tiles, long long s0, const double* __restrict__ Fin,
                                      long long ldF, long long fin_elems) {
  constexpr int ld = kTrajPerTile * D;
  const long long rows = s0 + 1;
  const long long total = (long long)n_tiles * rows * ld;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int col = (int)(idx % ld);
    const long long k = (idx / ld) % rows;
    const int t = (int)(idx / ((long long)ld * rows));
    const TileDesc& T = A.tiles[t];
    const int lane = col / D, c = col % D;
    const int src = T.traj[lane] >= 0 ? T.traj[lane] : T.traj[0];
    if (!in_bounds(A.status, kChkImport, ((long long)src * ldF + k) * D + c, fin_elems) ||
        !in_bounds(A.status, kChkImport, T.f_off + k * ld + col, A.f_elems))
      continue;
    const double v = Fin[((size_t)src * ldF + k) * D + c];
    A.F[T.f_off + k * ld + col] = v;
    if (A.F32) A.F32[T.f_off + k * ld + col] = (float)v;
  }
}

// BF16 split pieces of rows [0, s0) of every tile, from the FP64 rows just
// imported: a unit is 8 rows of one column, stored as one 16-byte chunk per
// piece, in the layout the near kernel writes.
template <int D>
__global__ void import_pieces_kernel(BatchArgs A, int n_tiles, long long s0) {
  constexpr int ld = kTrajPerTile * D;
  const long long kblocks = s0 / 64;
  const long long total = (long long)n_tiles * kblocks * ld * 8;
  for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < total;
       u += (long long)gridDim.x * blockDim.x) {
    const int part = (int)(u % 8);
    const int col = (int)((u / 8) % ld);
    const long long kb = (u / (8 * ld)) % kblocks;
    const int t = (int)(u / (8 * ld * kblocks));
    const TileDesc& T = A.tiles[t];
    __align__(16) __nv_bfloat16 v[3][8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const long long row = kb * 64 + part * 8 + r;
      __nv_bfloat16 pcs[3];
      const bool ok = in_bounds(A.status, kChkImport, T.f_off + row * ld + col, A.f_elems);
      split3_bf16(row == 0 || !ok ? 0.0 : A.F[T.f_off + row * ld + col], pcs);
      v[0][r] = pcs[0];
      v[1][r] = pcs[1];
      v[2][r] = pcs[2];
    }
    const size_t off = (((size_t)T.slot * (A.fsh_ld / 64) + kb) * ld + col) * 64 + part * 8;
    if (!in_bounds(A.status, kChkImport, (long long)off + 7, A.fsh_plane_elems)) continue;
#pragma unroll
    for (int pc = 0; pc < 3; ++pc)
      *reinterpret_cast<uint4*>(A.Fsh + (size_t)pc * A.fsh_plane + off) = *reinterpret_cast<const uint4*>(v[pc]);
  }
}

// f_0 .. f_{min(rows, N_i + 1) - 1} of every trajectory out of its tile.
template <int D>
__global__ void export_history_kernel(BatchArgs A, int n_tiles, long long rows, double* __restrict__ Fout,
                                      long long ldF, long long fout_elems) {
  constexpr int ld = kTrajPerTile * D;
  const long long total = (long long)n_tiles * rows * ld;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int col = (int)(idx % ld);
    const long long k = (idx / ld) % rows;
    const int t = (int)(idx / ((long long)ld * rows));
    const TileDesc& T = A.tiles[t];
    const int lane = col / D, c = col % D;
    const int traj = T.traj[lane];
    if (traj < 0 || k > A.N[traj]) continue;
    if (!in_bounds(A.status, kChkExport, ((long long)traj * ldF + k) * D + c, fout_elems) ||
        !in_bounds(A.status, kChkExport, T.f_off + k * ld + col, A.f_elems))
      continue;
    Fout[((size_t)traj * ldF + k) * D + c] = A.F[T.f_off + k * ld + col];
  }
}

namespace {
int grid_for(long long total) {
  const long long g = (total + 255) / 256;
  return (int)(g < 152 * 32 ? (g > 0 ? g : 1) : 152 * 32);
}
}  // namespace

cudaError_t launch_import_history(int d, const BatchArgs& A, int n_tiles, long long s0, const double* Fin,
                                  long long ldF, long long fin_elems, cudaStream_t st) {
  const long long total = (long long)n_tiles * (s0 + 1) * kTrajPerTile * d;
  if (d == 3) import_history_kernel<3><<<grid_for(total), 256, 0, st>>>(A, n_tiles, s0, Fin, ldF, fin_elems);
  else import_history_kernel<1><<<grid_for(total), 256, 0, st>>>(A, n_tiles, s0, Fin, ldF, fin_elems);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !A.Fsh || s0 < 64) return e;
  const long long units = (long long)n_tiles * (s0 / 64) * kTrajPerTile * d * 8;
  if (d == 3) import_pieces_kernel<3><<<grid_for(units), 256, 0, st>>>(A, n_tiles, s0);
  else return cudaErrorInvalidValue;  // the tensor-core paths take d = 3 only
  return cudaGetLastError();
}

cudaError_t launch_export_history(int d, const BatchArgs& A, int n_tiles, long long rows, double* Fout, long long ldF,
                                  long long fout_elems, cudaStream_t st) {
  const long long total = (long long)n_tiles * rows * kTrajPerTile * d;
  if (d == 3) export_history_kernel<3><<<grid_for(total), 256, 0, st>>>(A, n_tiles, rows, Fout, ldF, fout_elems);
  else export_history_kernel<1><<<grid_for(total), 256, 0, st>>>(A, n_tiles, rows, Fout, ldF, fout_elems);
  return cudaGetLastError();
}

}  // namespace abm
