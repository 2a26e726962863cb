// Batched path (abm_solve_batched): many independent trajectories.
//
// Trajectories are grouped on the host by alpha (one weight vector per
// group) and, inside a group, ordered by N and cut into column tiles of 32
// trajectories.  Each column tile keeps its own f history F[k][32*D] in
// time-major order, so one history row of a tile is contiguous.  For the time
// tile of targets n in [s, s+nb):
//   far  (rows k in [1, s))   : a Toeplitz-tile x F-tile contraction,
//                               W[2B x s] * F[s x 32D], W rows = b and a lags
//   near (rows k in [s, n])   : sequential PECE steps, one thread per
//                               trajectory, FP64
//   k = 0 terms b_n f_0, c_n f_0 : near kernel, FP64
// (Sec. 2 formulas; the split is the per-tile form of the partial sums the
// paper gathers across processes, Sec. 3 Fig. 2.)
#include "common.cuh"
#include "systems.cuh"
#include "batched.cuh"

namespace abm {

// ---------------------------------------------------------------------------
// Setup: h^alpha per trajectory, y_0 and f_0 into Y/YP/F.
// ---------------------------------------------------------------------------
template <int SYS>
__global__ void batched_setup_kernel(BatchArgs A) {
  using S = Sys<SYS>;
  constexpr int D = S::D;
  int tile = blockIdx.x, lane = threadIdx.x;
  const TileDesc& T = A.tiles[tile];
  int traj = T.traj[lane];
  int src = traj >= 0 ? traj : T.traj[0];
  double alpha = A.bucket_alpha[T.bucket];
  double p[kMaxParams], y0[D], f0[D];
#pragma unroll
  for (int q = 0; q < S::NP; ++q) p[q] = A.params[(size_t)src * S::NP + q];
#pragma unroll
  for (int c = 0; c < D; ++c) y0[c] = A.y0[(size_t)src * D + c];
  S::f(p, alpha, 0.0, y0, f0);
  double* F = A.F + T.f_off;
#pragma unroll
  for (int c = 0; c < D; ++c) F[lane * D + c] = f0[c];
  if (A.F32) {
    float* F32 = A.F32 + T.f_off;
#pragma unroll
    for (int c = 0; c < D; ++c) F32[lane * D + c] = (float)f0[c];
  }
  if (traj >= 0) {
    A.hhat[traj] = pow(A.h[traj], alpha);
#pragma unroll
    for (int c = 0; c < D; ++c) {
      A.Y[(size_t)traj * A.ldY * D + c] = y0[c];
      if (A.YP) A.YP[(size_t)traj * A.ldY * D + c] = y0[c];
    }
  }
}

// ---------------------------------------------------------------------------
// Near kernel: one CTA per column tile, one warp per state component, one
// lane per trajectory, nb sequential PECE steps.  Warp c forms the predictor
// and corrector sums of component c; the components meet through shared
// memory before each evaluation of f, so the FP64 work of a step is spread
// over D sub-partitions of the SM.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void split3_bf16(double x, __nv_bfloat16* out) {
  out[0] = __double2bfloat16(x);
  double r = x - (double)__bfloat162float(out[0]);
  out[1] = __double2bfloat16(r);
  r -= (double)__bfloat162float(out[1]);
  out[2] = __double2bfloat16(r);
}

template <int SYS>
__global__ void __launch_bounds__(32 * Sys<SYS>::D) batched_near_kernel(BatchArgs A, long long s, int nb) {
  using S = Sys<SYS>;
  constexpr int D = S::D;
  constexpr int NT = 32 * D;
  // BF16 split rows s..s+63 of this tile's history, [piece][column][row - s],
  // written out K-major (128 contiguous bytes per column) at the end
  __shared__ __align__(16) __nv_bfloat16 stg[3][kTrajPerTile * D][64];
  __shared__ double ysh[2][D][32], ysh2[2][D][32];  // predictor / corrector exchange
  const int tile = blockIdx.x, c = threadIdx.x >> 5, lane = threadIdx.x & 31;  // warp c = component c
  const TileDesc& T = A.tiles[tile];
  const int traj = T.traj[lane];
  const int src = traj >= 0 ? traj : T.traj[0];
  const double alpha = A.bucket_alpha[T.bucket];
  const double* __restrict__ wb = A.bucket_b[T.bucket];
  const double* __restrict__ wa = A.bucket_a[T.bucket];
  const double* __restrict__ wc = A.bucket_c[T.bucket];
  const double g = A.bucket_g[T.bucket];
  const long long Ntraj = traj >= 0 ? (long long)A.N[traj] : 0;
  const double h = A.h[src];
  const double hh = traj >= 0 ? A.hhat[traj] : pow(h, alpha);
  double p[kMaxParams];
#pragma unroll
  for (int q = 0; q < S::NP; ++q) p[q] = A.params[(size_t)src * S::NP + q];
  const double y0c = A.y0[(size_t)src * D + c];
  double* __restrict__ F = A.F + T.f_off;
  float* __restrict__ F32 = A.F32 ? A.F32 + T.f_off : nullptr;
  constexpr int ld = kTrajPerTile * D;  // row stride of the tile history
  const int col = lane * D + c;         // this thread's history column
  const double F0c = F[col];
  const long long e = s > 1 ? s : 1;  // first near row
  if (A.Fsh) {  // row s: zero for s = 0 (the j = 0 term stays in FP64), else f_s
    __nv_bfloat16 pc[3];
    split3_bf16(s == 0 ? 0.0 : F[s * ld + col], pc);
#pragma unroll
    for (int q = 0; q < 3; ++q) stg[q][col][0] = pc[q];
  }
  bool reported = false;
  for (int i = 0; i < nb; ++i) {
    const long long n = s + i;
    const int par = i & 1;
    // far part: sum of the K-split partials, then the k = 0 terms
    double sp = 0.0, sc = 0.0;
    if (s > 1) {
      for (int q = 0; q < A.ksplit; ++q) {
        const size_t base = (((size_t)q * A.n_tiles + tile) * 2) * A.B;
        sp += A.far[(base + i) * ld + col];
        sc += A.far[(base + A.B + i) * ld + col];
      }
    }
    sp = fma(wb[n], F0c, sp);
    sc = fma(wc[n], F0c, sc);
    // near rows k in [e, n], FP64
    for (long long k = e; k <= n; ++k) {
      const double fv = F[k * ld + col];
      sp = fma(wb[n - k], fv, sp);
      sc = fma(wa[n - k], fv, sc);
    }
    const double t1 = (double)(n + 1) * h;
    const double yp = fma(hh, sp, y0c);
    ysh[par][c][lane] = yp;
    asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
    double ypv[D];
#pragma unroll
    for (int q = 0; q < D; ++q) ypv[q] = ysh[par][q][lane];
    const double fp = S::fc(c, p, alpha, t1, ypv);
    const double y = fma(hh, fma(g, fp, sc), y0c);
    ysh2[par][c][lane] = y;
    asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
    double yv[D];
#pragma unroll
    for (int q = 0; q < D; ++q) yv[q] = ysh2[par][q][lane];
    const double fy = S::fc(c, p, alpha, t1, yv);
    F[(n + 1) * ld + col] = fy;
    if (F32) F32[(n + 1) * ld + col] = (float)fy;
    if (A.Fsh && i + 1 < 64) {
      __nv_bfloat16 pc[3];
      split3_bf16(fy, pc);
#pragma unroll
      for (int q = 0; q < 3; ++q) stg[q][col][i + 1] = pc[q];
    }
    if (n + 1 <= Ntraj) {
      A.Y[((size_t)traj * A.ldY + (n + 1)) * D + c] = y;
      if (A.YP) A.YP[((size_t)traj * A.ldY + (n + 1)) * D + c] = yp;
      if (!reported && !(isfinite(y) && isfinite(fy))) {
        report_status(A.status, ABM_ERR_NONFINITE, traj, n + 1);
        reported = true;
      }
    }
  }
  if (A.Fsh) {
    __syncthreads();
    // 3 pieces x 32*D columns x 8 chunks of 16 bytes
    constexpr int CHUNKS = 3 * kTrajPerTile * D * 8;
    for (int q = threadIdx.x; q < CHUNKS; q += NT) {
      const int pc = q / (kTrajPerTile * D * 8), rem = q % (kTrajPerTile * D * 8);
      const int cc = rem / 8, part = rem % 8;
      const uint4 v = *reinterpret_cast<const uint4*>(&stg[pc][cc][part * 8]);
      __nv_bfloat16* dst = A.Fsh + (size_t)pc * A.fsh_plane +
                           ((size_t)blockIdx.x * kTrajPerTile * D + cc) * A.fsh_ld + s + part * 8;
      *reinterpret_cast<uint4*>(dst) = v;
    }
  }
}

// ---------------------------------------------------------------------------
// Far kernel, FP64 (plain comparator path).  Grid (active tiles, ksplit).
// 256 threads = 8 warps; warp w owns target rows [w*B/8, (w+1)*B/8), lane =
// trajectory.  Every lane of a warp uses the same Toeplitz lag, so the weight
// window is warp-uniform; F rows are read coalesced (32*D doubles per row).
// ---------------------------------------------------------------------------
template <int D, int B>
__global__ void __launch_bounds__(256) batched_far_fp64_kernel(BatchArgs A, long long s) {
  constexpr int R = B / 8;  // rows per warp
  constexpr int ld = kTrajPerTile * D;
  const int tile = blockIdx.x, q = blockIdx.y, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const TileDesc& T = A.tiles[tile];
  const double* __restrict__ wb = A.bucket_b[T.bucket];
  const double* __restrict__ wa = A.bucket_a[T.bucket];
  const double* __restrict__ F = A.F + T.f_off;
  // history rows [1, s) split into ksplit chunks
  const long long K = s - 1;
  const long long chunk = (K + A.ksplit - 1) / A.ksplit;
  const long long kb = 1 + (long long)q * chunk, ke = min(s, kb + chunk);
  const int i0 = warp * R;
  double accP[R][D], accC[R][D];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) accP[r][c] = accC[r][c] = 0.0;
  if (kb < ke) {
    double wbv[R], wav[R];
#pragma unroll
    for (int r = 0; r < R; ++r) { wbv[r] = wb[s + i0 + r - kb]; wav[r] = wa[s + i0 + r - kb]; }
    for (long long k = kb; k < ke; ++k) {
      double f[D];
#pragma unroll
      for (int c = 0; c < D; ++c) f[c] = F[k * ld + lane * D + c];
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) {
          accP[r][c] = fma(wbv[r], f[c], accP[r][c]);
          accC[r][c] = fma(wav[r], f[c], accC[r][c]);
        }
#pragma unroll
      for (int r = R - 1; r > 0; --r) { wbv[r] = wbv[r - 1]; wav[r] = wav[r - 1]; }
      if (k + 1 < ke) { wbv[0] = wb[s + i0 - (k + 1)]; wav[0] = wa[s + i0 - (k + 1)]; }
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    double* P = A.far + ((((size_t)q * A.n_tiles + tile) * 2 + 0) * B + i0 + r) * ld + lane * D;
    double* C = A.far + ((((size_t)q * A.n_tiles + tile) * 2 + 1) * B + i0 + r) * ld + lane * D;
#pragma unroll
    for (int c = 0; c < D; ++c) { P[c] = accP[r][c]; C[c] = accC[r][c]; }
  }
}

// ---------------------------------------------------------------------------
// Far kernel, FP32 operands (SIMT): FP32 products and accumulation inside a
// lag block of KB rows, blocks combined in FP64.  Same layout as the FP64
// kernel; 512 threads = 16 warps, warp w owns B/16 rows.
// ---------------------------------------------------------------------------
template <int D, int B, int KB>
__global__ void __launch_bounds__(512) batched_far_fp32_kernel(BatchArgs A, long long s) {
  constexpr int R = B / 16;
  constexpr int ld = kTrajPerTile * D;
  const int tile = blockIdx.x, q = blockIdx.y, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const TileDesc& T = A.tiles[tile];
  const float* __restrict__ wb = A.bucket_b32[T.bucket];
  const float* __restrict__ wa = A.bucket_a32[T.bucket];
  const float* __restrict__ F = A.F32 + T.f_off;
  const long long K = s - 1;
  const long long chunk = (K + A.ksplit - 1) / A.ksplit;
  const long long kb = 1 + (long long)q * chunk, ke = min(s, kb + chunk);
  const int i0 = warp * R;
  double dP[R][D], dC[R][D];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) dP[r][c] = dC[r][c] = 0.0;
  for (long long k0 = kb; k0 < ke; k0 += KB) {
    const long long k1 = min(ke, k0 + KB);
    float accP[R][D], accC[R][D];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) accP[r][c] = accC[r][c] = 0.0f;
    float wbv[R], wav[R];
#pragma unroll
    for (int r = 0; r < R; ++r) { wbv[r] = wb[s + i0 + r - k0]; wav[r] = wa[s + i0 + r - k0]; }
    for (long long k = k0; k < k1; ++k) {
      float f[D];
#pragma unroll
      for (int c = 0; c < D; ++c) f[c] = F[k * ld + lane * D + c];
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) {
          accP[r][c] = fmaf(wbv[r], f[c], accP[r][c]);
          accC[r][c] = fmaf(wav[r], f[c], accC[r][c]);
        }
#pragma unroll
      for (int r = R - 1; r > 0; --r) { wbv[r] = wbv[r - 1]; wav[r] = wav[r - 1]; }
      if (k + 1 < k1) { wbv[0] = wb[s + i0 - (k + 1)]; wav[0] = wa[s + i0 - (k + 1)]; }
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) { dP[r][c] += (double)accP[r][c]; dC[r][c] += (double)accC[r][c]; }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    double* P = A.far + ((((size_t)q * A.n_tiles + tile) * 2 + 0) * B + i0 + r) * ld + lane * D;
    double* C = A.far + ((((size_t)q * A.n_tiles + tile) * 2 + 1) * B + i0 + r) * ld + lane * D;
#pragma unroll
    for (int c = 0; c < D; ++c) { P[c] = dP[r][c]; C[c] = dC[r][c]; }
  }
}

// ---------------------------------------------------------------------------
cudaError_t launch_batched_setup(int sys, const BatchArgs& A, int n_tiles, cudaStream_t st) {
  ABM_DISPATCH_SYSTEM(sys, (batched_setup_kernel<SYS><<<n_tiles, kTrajPerTile, 0, st>>>(A)));
  return cudaGetLastError();
}

cudaError_t launch_batched_near(int sys, const BatchArgs& A, int n_active, long long s, int nb,
                                cudaStream_t st) {
  ABM_DISPATCH_SYSTEM(sys, (batched_near_kernel<SYS><<<n_active, kTrajPerTile * Sys<SYS>::D, 0, st>>>(A, s, nb)));
  return cudaGetLastError();
}

cudaError_t launch_batched_far(int d, abm_precision prec, const BatchArgs& A, int n_active, long long s,
                               cudaStream_t st) {
  dim3 grid(n_active, A.ksplit);
  if (prec == ABM_PREC_FP64) {
    if (A.B != 64) return cudaErrorInvalidValue;
    if (d == 3) batched_far_fp64_kernel<3, 64><<<grid, 256, 0, st>>>(A, s);
    else batched_far_fp64_kernel<1, 64><<<grid, 256, 0, st>>>(A, s);
  } else {
    if (A.B != 64) return cudaErrorInvalidValue;
    if (d == 3) batched_far_fp32_kernel<3, 64, 512><<<grid, 512, 0, st>>>(A, s);
    else batched_far_fp32_kernel<1, 64, 512><<<grid, 512, 0, st>>>(A, s);
  }
  return cudaGetLastError();
}

}  // namespace abm
