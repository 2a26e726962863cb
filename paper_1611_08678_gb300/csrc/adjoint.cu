// A6 - discrete adjoint of the batched ABM solve (the paper has no adjoint;
// this differentiates exactly the scheme of Sec. 2).
//
// Forward (per trajectory): y^P_{n+1} = y0 + h^a sum_{k<=n} b_{n-k} f_k,
// y_{n+1} = y0 + h^a (c_n f_0 + sum_{1<=k<=n} a_{n-k} f_k + g f(t_{n+1}, y^P_{n+1})),
// f_k = f(t_k, y_k), loss L(y_0..y_N) with partials G_n = dL/dy_n (given).
// Reverse sweep over k = N..0 with lambda_k = dL/dy_k, mu_k = dL/dy^P_k,
// phi_k = dL/df_k (all total derivatives):
//   phi_k    = h^a sum_{n>k} (b_{n-1-k} mu_n + a_{n-1-k} lambda_n)   (k >= 1; phi_N = 0)
//   phi_0    = h^a sum_{n>=1} (b_{n-1} mu_n + c_{n-1} lambda_n)
//   lambda_k = G_k + J(t_k, y_k)^T phi_k
//   mu_k     = h^a g J(t_k, y^P_k)^T lambda_k                         (k >= 1)
//   dL/dp    = sum_k Q(t_k, y_k)^T phi_k + h^a g sum_{k>=1} Q(t_k, y^P_k)^T lambda_k
//   dL/dy0   = G_0 + J(0, y_0)^T phi_0 + sum_{k>=1} (lambda_k + mu_k)
// (J = df/dy, Q = df/dp, recomputed from the stored y_k and y^P_k; no
// Jacobian is stored.)  In reversed time r = N - k the phi sum is the same
// Toeplitz contraction as the forward history sums: for target t = r - 1,
//   phi = h^a (sum_{r' <= t} b_{t-r'} mu~_{r'} + sum_{r' <= t} a_{t-r'} lambda~_{r'}),
// so the batched machinery is reused: each forward column tile becomes two
// adjoint tiles (mu~ and lambda~ histories), the far kernels (tensor-core or
// FP64) produce the far sums, and the near kernel below runs the reverse
// steps with the window lags in FP64.
#include "batched.cuh"
#include "bf16split.cuh"
#include "common.cuh"
#include "systems.cuh"

namespace abm {


namespace {
template <int D>
__device__ __forceinline__ void bar_components() {
  asm volatile("bar.sync 1, %0;" ::"n"(32 * D) : "memory");
}
}  // namespace

// k = N_i: lambda_N = G_N, mu_N = h^a g JP^T lambda_N; row 0 of both histories.
template <int SYS>
__global__ void __launch_bounds__(32 * Sys<SYS>::D) adjoint_setup_kernel(AdjArgs A) {
  using S = Sys<SYS>;
  constexpr int D = S::D, NP = S::NP, ld = kTrajPerTile * D;
  __shared__ double lsh[D][32];
  const int tile = blockIdx.x, c = threadIdx.x >> 5, lane = threadIdx.x & 31, col = lane * D + c;
  const TileDesc& T = A.tiles[tile];
  const int traj = T.traj[lane];
  const int src = traj >= 0 ? traj : T.traj[0];
  const double alpha = A.bucket_alpha[T.bucket * kMaxD];
  const double g = A.bucket_g[T.bucket * kMaxD];
  const double* wc = A.bucket_c[T.bucket * kMaxD];
  const long long N = A.N[src];
  const double h = A.h[src];
  const double hh = pow(h, alpha);
  double p[kMaxParams];
#pragma unroll
  for (int q = 0; q < NP; ++q) p[q] = A.params[(size_t)src * NP + q];
  const double* yPN = A.YP + ((size_t)src * A.ldY + N) * D;
  double yp[D];
#pragma unroll
  for (int q = 0; q < D; ++q) yp[q] = yPN[q];
  const double lam = A.G[((size_t)src * A.ldY + N) * D + c];
  lsh[c][lane] = lam;
  bar_components<D>();
  double J[D * D], Q[D * NP];
  S::jac(p, alpha, (double)N * h, yp, J, Q);
  double jl = 0.0;
#pragma unroll
  for (int j = 0; j < D; ++j) jl = fma(J[j * D + c], lsh[j][lane], jl);
  const double mu = hh * g * jl;
  const bool act = traj >= 0;
  if (act) {
    if (c == 0) A.hhat[(size_t)traj * kMaxD] = hh;
#pragma unroll
    for (int q = 0; q < NP; ++q) A.acc_dp[((size_t)traj * D + c) * NP + q] = hh * g * Q[c * NP + q] * lam;
    A.acc_dy0[(size_t)traj * D + c] = lam + mu;
    A.phi0c[(size_t)traj * D + c] = wc[N - 1] * lam;
  }
  A.X[A.atiles[2 * tile].f_off + col] = act ? mu : 0.0;
  A.X[A.atiles[2 * tile + 1].f_off + col] = act ? lam : 0.0;
}

// Reverse steps for targets t = s..s+nb-1 (row t+1 of the histories),
// forward index k = N_i - 1 - t.  Chain warps (one per state component, one
// lane per trajectory) run the reverse step; the components meet through
// shared memory for J^T phi and J^T lambda.  As in the forward near kernel,
// HS helper warps per component sum step i+1's window over the rows already
// known while step i's chain runs, and the chain adds the newest row; HS = 0
// leaves the whole window to the chain warps.
template <int SYS, int HS>
__global__ void __launch_bounds__(32 * (HS + 1) * Sys<SYS>::D) adjoint_near_kernel(AdjArgs A, long long s, int nb) {
  using S = Sys<SYS>;
  constexpr int D = S::D, NP = S::NP, ld = kTrajPerTile * D;
  constexpr int NT = 32 * (HS + 1) * D, HSX = HS > 0 ? HS : 1;
  extern __shared__ double adj_dyn[];
  double (*Wm)[ld] = reinterpret_cast<double (*)[ld]>(adj_dyn);            // mu~ rows s..s+64
  double (*Wl)[ld] = reinterpret_cast<double (*)[ld]>(adj_dyn + 65 * ld);  // lambda~ rows s..s+64
  // helpers' partial window sums, [step parity][slice][column]
  double (*Rm)[HSX][ld] = reinterpret_cast<double (*)[HSX][ld]>(adj_dyn + 130 * ld);
  double (*Rl)[HSX][ld] = reinterpret_cast<double (*)[HSX][ld]>(adj_dyn + (130 + 2 * HS) * ld);
  __shared__ double wsb[65], wsa[65];
  __shared__ double xsh[D][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool chain = warp < D;
  const int c = chain ? warp : (warp - D) % D;  // component (column group)
  const int q = chain ? 0 : (warp - D) / D;     // helper slice
  const int tile = blockIdx.x, col = lane * D + c;
  const TileDesc& T = A.tiles[tile];
  const int traj = T.traj[lane];
  const int src = traj >= 0 ? traj : T.traj[0];
  const double* wb = A.bucket_b[T.bucket * kMaxD];
  const double* wa = A.bucket_a[T.bucket * kMaxD];
  double* Xm = A.X + A.atiles[2 * tile].f_off;
  double* Xl = A.X + A.atiles[2 * tile + 1].f_off;
  for (int m = threadIdx.x; m < 65; m += NT) { wsb[m] = wb[m]; wsa[m] = wa[m]; }
  for (int m = threadIdx.x; m < ld; m += NT) {
    Wm[0][m] = Xm[s * ld + m];
    Wl[0][m] = Xl[s * ld + m];
  }
  for (int m = threadIdx.x; m < HS * ld; m += NT) {  // step 0 has no earlier window rows
    Rm[0][m / ld][m % ld] = 0.0;
    Rl[0][m / ld][m % ld] = 0.0;
  }

  if (chain) {
    const double alpha = A.bucket_alpha[T.bucket * kMaxD];
    const double* wc = A.bucket_c[T.bucket * kMaxD];
    const double g = A.bucket_g[T.bucket * kMaxD];
    const long long Ni = traj >= 0 ? (long long)A.N[traj] : -1;
    const double h = A.h[src];
    const double hh = traj >= 0 ? A.hhat[(size_t)traj * kMaxD] : 0.0;
    double p[kMaxParams];
#pragma unroll
    for (int k = 0; k < NP; ++k) p[k] = A.params[(size_t)src * NP + k];
    double adp[NP], ady0 = 0.0, phc = 0.0;
#pragma unroll
    for (int k = 0; k < NP; ++k) adp[k] = 0.0;
    if (traj >= 0) {
#pragma unroll
      for (int k = 0; k < NP; ++k) adp[k] = A.acc_dp[((size_t)traj * D + c) * NP + k];
      ady0 = A.acc_dy0[(size_t)traj * D + c];
      phc = A.phi0c[(size_t)traj * D + c];
    }
    __syncthreads();
    const size_t fstride = (size_t)A.far_tiles * 2 * A.B * ld;
    for (int i = 0; i < nb; ++i) {
      const long long t = s + i;
      const long long k = Ni - 1 - t;  // forward index of this reverse step
      const bool act = k >= 0;
      const long long kk = act ? k : 0;
      const int par = i & 1;
      // inputs at k: y_k, y^P_k, G_k
      double yk[D], ypk[D];
#pragma unroll
      for (int j = 0; j < D; ++j) {
        yk[j] = A.Y[((size_t)src * A.ldY + kk) * D + j];
        ypk[j] = A.YP[((size_t)src * A.ldY + kk) * D + j];
      }
      const double Gk = A.G[((size_t)src * A.ldY + kk) * D + c];
      // far sums (mu~ rows through b, lambda~ rows through a)
      double Sm = 0.0, Sl = 0.0;
      if (s > 0) {
        for (int kq = 0; kq < A.far_ksplit; ++kq) {
          Sm += A.far[kq * fstride + ((((size_t)2 * tile) * 2 + 0) * A.B + i) * ld + col];
          Sl += A.far[kq * fstride + ((((size_t)2 * tile + 1) * 2 + 1) * A.B + i) * ld + col];
        }
      }
      if constexpr (HS > 0) {
#pragma unroll
        for (int j = 0; j < HS; ++j) { Sm += Rm[par][j][col]; Sl += Rl[par][j][col]; }
        Sm = fma(wsb[0], Wm[i][col], Sm);  // the newest window row
        Sl = fma(wsa[0], Wl[i][col], Sl);
      } else {  // the whole window, rows [0, i], two chains per sum
        double Sm1 = 0.0, Sl1 = 0.0;
        int r = 0;
        for (; r + 1 <= i; r += 2) {
          Sm = fma(wsb[i - r], Wm[r][col], Sm);
          Sl = fma(wsa[i - r], Wl[r][col], Sl);
          Sm1 = fma(wsb[i - r - 1], Wm[r + 1][col], Sm1);
          Sl1 = fma(wsa[i - r - 1], Wl[r + 1][col], Sl1);
        }
        if (r <= i) {
          Sm = fma(wsb[i - r], Wm[r][col], Sm);
          Sl = fma(wsa[i - r], Wl[r][col], Sl);
        }
        Sm += Sm1;
        Sl += Sl1;
      }
      const double phi = hh * (Sm + (k >= 1 ? Sl : phc));
      xsh[c][lane] = phi;
      bar_components<D>();
      // Jacobians recomputed from the stored states: at y_k and at y^P_k; this
      // warp uses column c of J and row c of Q (selected with compile-time
      // indices so that the arrays stay in registers)
      double Jy[D * D], Qy[D * NP], Jp[D * D], Qp[D * NP];
      S::jac(p, alpha, (double)kk * h, yk, Jy, Qy);
      S::jac(p, alpha, (double)kk * h, ypk, Jp, Qp);
      double Jyc[D], Jpc[D], Qyc[NP], Qpc[NP];
#pragma unroll
      for (int j = 0; j < D; ++j) { Jyc[j] = Jy[j * D]; Jpc[j] = Jp[j * D]; }
#pragma unroll
      for (int j = 0; j < NP; ++j) { Qyc[j] = Qy[j]; Qpc[j] = Qp[j]; }
#pragma unroll
      for (int cc = 1; cc < D; ++cc) {
        if (c == cc) {
#pragma unroll
          for (int j = 0; j < D; ++j) { Jyc[j] = Jy[j * D + cc]; Jpc[j] = Jp[j * D + cc]; }
#pragma unroll
          for (int j = 0; j < NP; ++j) { Qyc[j] = Qy[cc * NP + j]; Qpc[j] = Qp[cc * NP + j]; }
        }
      }
      double lam = Gk;
#pragma unroll
      for (int j = 0; j < D; ++j) lam = fma(Jyc[j], xsh[j][lane], lam);
      bar_components<D>();
      xsh[c][lane] = lam;
      bar_components<D>();
      double jl = 0.0;
#pragma unroll
      for (int j = 0; j < D; ++j) jl = fma(Jpc[j], xsh[j][lane], jl);
      bar_components<D>();
      const double mu = hh * g * jl;
      if (act) {
#pragma unroll
        for (int j = 0; j < NP; ++j) adp[j] = fma(Qyc[j], phi, adp[j]);
        if (k >= 1) {
#pragma unroll
          for (int j = 0; j < NP; ++j) adp[j] = fma(hh * g * Qpc[j], lam, adp[j]);
          ady0 += lam + mu;
          phc = fma(wc[k - 1], lam, phc);
        } else {  // k = 0: lambda here is G_0 + J_0^T phi_0
          A.dy0[(size_t)traj * D + c] = ady0 + lam;
        }
        if (!(finite_bits(lam) && finite_bits(phi))) report_status(A.status, ABM_ERR_NONFINITE, traj, k);
      }
      const bool row = act && k >= 1;
      Wm[i + 1][col] = row ? mu : 0.0;
      Wl[i + 1][col] = row ? lam : 0.0;
      Xm[(t + 1) * ld + col] = row ? mu : 0.0;
      Xl[(t + 1) * ld + col] = row ? lam : 0.0;
      __syncthreads();
    }
    if (traj >= 0) {
#pragma unroll
      for (int j = 0; j < NP; ++j) A.acc_dp[((size_t)traj * D + c) * NP + j] = adp[j];
      A.acc_dy0[(size_t)traj * D + c] = ady0;
      A.phi0c[(size_t)traj * D + c] = phc;
    }
  } else {
    __syncthreads();
    for (int i = 0; i < nb; ++i) {
      if (i + 1 < nb) {
        // partial window sums of step i+1 over rows r in [0, i], r = q mod HS
        const int nxt = (i + 1) & 1;
        double sm0 = 0.0, sl0 = 0.0, sm1 = 0.0, sl1 = 0.0;
        int r = q;
#pragma unroll 1
        for (; r + HSX <= i; r += 2 * HSX) {
          sm0 = fma(wsb[i + 1 - r], Wm[r][col], sm0);
          sl0 = fma(wsa[i + 1 - r], Wl[r][col], sl0);
          sm1 = fma(wsb[i + 1 - r - HSX], Wm[r + HSX][col], sm1);
          sl1 = fma(wsa[i + 1 - r - HSX], Wl[r + HSX][col], sl1);
        }
        if (r <= i) {
          sm0 = fma(wsb[i + 1 - r], Wm[r][col], sm0);
          sl0 = fma(wsa[i + 1 - r], Wl[r][col], sl0);
        }
        Rm[nxt][q][col] = sm0 + sm1;
        Rl[nxt][q][col] = sl0 + sl1;
      }
      __syncthreads();
    }
  }
  if (A.Xsh) {
    __syncthreads();
    // BF16 split rows s..s+63 of both histories: K block s / 64 of adjoint
    // tiles 2 tile + hist (K-block tiled like the forward history pieces)
    constexpr int UNITS = 2 * ld * 8;  // (history, column, 8 rows), split once, 3 stores
    for (int u = threadIdx.x; u < UNITS; u += NT) {
      const int hist = u / (ld * 8), rem = u % (ld * 8);
      const int cc = rem / 8, part = rem % 8;
      __align__(16) __nv_bfloat16 v[3][8];
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        __nv_bfloat16 pcs[3];
        split3_bf16(hist == 0 ? Wm[part * 8 + r][cc] : Wl[part * 8 + r][cc], pcs);
        v[0][r] = pcs[0];
        v[1][r] = pcs[1];
        v[2][r] = pcs[2];
      }
      const size_t off = (((size_t)(2 * tile + hist) * (A.xsh_ld / 64) + s / 64) * ld + cc) * 64 + part * 8;
#pragma unroll
      for (int pc = 0; pc < 3; ++pc)
        *reinterpret_cast<uint4*>(A.Xsh + (size_t)pc * A.xsh_plane + off) = *reinterpret_cast<const uint4*>(v[pc]);
    }
  }
}

// The reverse steps with each forward column tile spread over L CTAs (as the
// forward split near kernel): CTA b serves tile b / L, trajectories
// (b % L) * T .. + T - 1 of it (T = 32 / L); one warp per state component,
// lane = j * L + l serves trajectory j and lag slice l of the two windows,
// the slices added with shuffles.  All lanes of a trajectory run the same
// reverse step (identical values); lane l = 0 stores.  Used when few tiles
// are active, so that the FP64 window work runs on more SMs.
template <int SYS, int L>
__global__ void __launch_bounds__(32 * Sys<SYS>::D) adjoint_near_split_kernel(AdjArgs A, long long s, int nb) {
  using S = Sys<SYS>;
  constexpr int D = S::D, NP = S::NP, ld = kTrajPerTile * D;
  constexpr int T = kTrajPerTile / L, ldc = T * D, NT = 32 * D;
  __shared__ double Wm[65][ldc], Wl[65][ldc];  // mu~ / lambda~ rows s..s+64 of this CTA's columns
  __shared__ double wsb[65], wsa[65];
  __shared__ double xsh[D][T];
  const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = lane / L, l = lane % L;
  const int tile = blockIdx.x / L, part = blockIdx.x % L;
  const int tl = part * T + j, col = tl * D + c, cloc = j * D + c;
  const TileDesc& Td = A.tiles[tile];
  const int traj = Td.traj[tl];
  const int src = traj >= 0 ? traj : Td.traj[0];
  const double* wb = A.bucket_b[Td.bucket * kMaxD];
  const double* wa = A.bucket_a[Td.bucket * kMaxD];
  double* Xm = A.X + A.atiles[2 * tile].f_off;
  double* Xl = A.X + A.atiles[2 * tile + 1].f_off;
  for (int m = threadIdx.x; m < 65; m += NT) { wsb[m] = wb[m]; wsa[m] = wa[m]; }
  for (int m = threadIdx.x; m < ldc; m += NT) {
    Wm[0][m] = Xm[s * ld + part * ldc + m];
    Wl[0][m] = Xl[s * ld + part * ldc + m];
  }
  const double alpha = A.bucket_alpha[Td.bucket * kMaxD];
  const double* wc = A.bucket_c[Td.bucket * kMaxD];
  const double g = A.bucket_g[Td.bucket * kMaxD];
  const long long Ni = traj >= 0 ? (long long)A.N[traj] : -1;
  const double h = A.h[src];
  const double hh = traj >= 0 ? A.hhat[(size_t)traj * kMaxD] : 0.0;
  double p[kMaxParams];
#pragma unroll
  for (int k = 0; k < NP; ++k) p[k] = A.params[(size_t)src * NP + k];
  double adp[NP], ady0 = 0.0, phc = 0.0;
#pragma unroll
  for (int k = 0; k < NP; ++k) adp[k] = 0.0;
  if (traj >= 0) {
#pragma unroll
    for (int k = 0; k < NP; ++k) adp[k] = A.acc_dp[((size_t)traj * D + c) * NP + k];
    ady0 = A.acc_dy0[(size_t)traj * D + c];
    phc = A.phi0c[(size_t)traj * D + c];
  }
  __syncthreads();
  const size_t fstride = (size_t)A.far_tiles * 2 * A.B * ld;
  for (int i = 0; i < nb; ++i) {
    const long long t = s + i;
    const long long k = Ni - 1 - t;  // forward index of this reverse step
    const bool act = k >= 0;
    const long long kk = act ? k : 0;
    double yk[D], ypk[D];
#pragma unroll
    for (int q = 0; q < D; ++q) {
      yk[q] = A.Y[((size_t)src * A.ldY + kk) * D + q];
      ypk[q] = A.YP[((size_t)src * A.ldY + kk) * D + q];
    }
    const double Gk = A.G[((size_t)src * A.ldY + kk) * D + c];
    // lane slice l of the two windows, rows r = l mod L in [0, i]
    double Sm = 0.0, Sl = 0.0, Sm1 = 0.0, Sl1 = 0.0;
    int r = l;
    for (; r + L <= i; r += 2 * L) {
      Sm = fma(wsb[i - r], Wm[r][cloc], Sm);
      Sl = fma(wsa[i - r], Wl[r][cloc], Sl);
      Sm1 = fma(wsb[i - r - L], Wm[r + L][cloc], Sm1);
      Sl1 = fma(wsa[i - r - L], Wl[r + L][cloc], Sl1);
    }
    if (r <= i) {
      Sm = fma(wsb[i - r], Wm[r][cloc], Sm);
      Sl = fma(wsa[i - r], Wl[r][cloc], Sl);
    }
    Sm += Sm1;
    Sl += Sl1;
#pragma unroll
    for (int o = 1; o < L; o <<= 1) {
      Sm += __shfl_xor_sync(0xffffffffu, Sm, o);
      Sl += __shfl_xor_sync(0xffffffffu, Sl, o);
    }
    if (s > 0) {  // far sums (mu~ rows through b, lambda~ rows through a)
      for (int kq = 0; kq < A.far_ksplit; ++kq) {
        Sm += A.far[kq * fstride + ((((size_t)2 * tile) * 2 + 0) * A.B + i) * ld + col];
        Sl += A.far[kq * fstride + ((((size_t)2 * tile + 1) * 2 + 1) * A.B + i) * ld + col];
      }
    }
    const double phi = hh * (Sm + (k >= 1 ? Sl : phc));
    if (l == 0) xsh[c][j] = phi;
    bar_components<D>();
    double Jy[D * D], Qy[D * NP], Jp[D * D], Qp[D * NP];
    S::jac(p, alpha, (double)kk * h, yk, Jy, Qy);
    S::jac(p, alpha, (double)kk * h, ypk, Jp, Qp);
    double Jyc[D], Jpc[D], Qyc[NP], Qpc[NP];
#pragma unroll
    for (int q = 0; q < D; ++q) { Jyc[q] = Jy[q * D]; Jpc[q] = Jp[q * D]; }
#pragma unroll
    for (int q = 0; q < NP; ++q) { Qyc[q] = Qy[q]; Qpc[q] = Qp[q]; }
#pragma unroll
    for (int cc = 1; cc < D; ++cc) {
      if (c == cc) {
#pragma unroll
        for (int q = 0; q < D; ++q) { Jyc[q] = Jy[q * D + cc]; Jpc[q] = Jp[q * D + cc]; }
#pragma unroll
        for (int q = 0; q < NP; ++q) { Qyc[q] = Qy[cc * NP + q]; Qpc[q] = Qp[cc * NP + q]; }
      }
    }
    double lam = Gk;
#pragma unroll
    for (int q = 0; q < D; ++q) lam = fma(Jyc[q], xsh[q][j], lam);
    bar_components<D>();
    if (l == 0) xsh[c][j] = lam;
    bar_components<D>();
    double jl = 0.0;
#pragma unroll
    for (int q = 0; q < D; ++q) jl = fma(Jpc[q], xsh[q][j], jl);
    bar_components<D>();
    const double mu = hh * g * jl;
    if (act) {
#pragma unroll
      for (int q = 0; q < NP; ++q) adp[q] = fma(Qyc[q], phi, adp[q]);
      if (k >= 1) {
#pragma unroll
        for (int q = 0; q < NP; ++q) adp[q] = fma(hh * g * Qpc[q], lam, adp[q]);
        ady0 += lam + mu;
        phc = fma(wc[k - 1], lam, phc);
      } else if (l == 0) {  // k = 0: lambda here is G_0 + J_0^T phi_0
        A.dy0[(size_t)traj * D + c] = ady0 + lam;
      }
      if (l == 0 && !(finite_bits(lam) && finite_bits(phi))) report_status(A.status, ABM_ERR_NONFINITE, traj, k);
    }
    const bool row = act && k >= 1;
    if (l == 0) {
      Wm[i + 1][cloc] = row ? mu : 0.0;
      Wl[i + 1][cloc] = row ? lam : 0.0;
      Xm[(t + 1) * ld + col] = row ? mu : 0.0;
      Xl[(t + 1) * ld + col] = row ? lam : 0.0;
    }
    bar_components<D>();
  }
  if (traj >= 0 && l == 0) {
#pragma unroll
    for (int q = 0; q < NP; ++q) A.acc_dp[((size_t)traj * D + c) * NP + q] = adp[q];
    A.acc_dy0[(size_t)traj * D + c] = ady0;
    A.phi0c[(size_t)traj * D + c] = phc;
  }
  if (A.Xsh) {
    // BF16 split of rows s..s+63 of both histories, this CTA's columns
    constexpr int UNITS = 2 * ldc * 8;  // (history, column, 8 rows), split once, 3 stores
    for (int u = threadIdx.x; u < UNITS; u += NT) {
      const int hist = u / (ldc * 8), rem = u % (ldc * 8);
      const int cc = rem / 8, prt = rem % 8;
      __align__(16) __nv_bfloat16 v[3][8];
#pragma unroll
      for (int rr = 0; rr < 8; ++rr) {
        __nv_bfloat16 pcs[3];
        split3_bf16(hist == 0 ? Wm[prt * 8 + rr][cc] : Wl[prt * 8 + rr][cc], pcs);
        v[0][rr] = pcs[0];
        v[1][rr] = pcs[1];
        v[2][rr] = pcs[2];
      }
      const size_t off =
          (((size_t)(2 * tile + hist) * (A.xsh_ld / 64) + s / 64) * ld + part * ldc + cc) * 64 + prt * 8;
#pragma unroll
      for (int pc = 0; pc < 3; ++pc)
        *reinterpret_cast<uint4*>(A.Xsh + (size_t)pc * A.xsh_plane + off) = *reinterpret_cast<const uint4*>(v[pc]);
    }
  }
}

template <int SYS>
__global__ void adjoint_finish_kernel(AdjArgs A, int M) {
  using S = Sys<SYS>;
  constexpr int D = S::D, NP = S::NP;
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * NP) return;
  const int traj = idx / NP, q = idx % NP;
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < D; ++c) s += A.acc_dp[((size_t)traj * D + c) * NP + q];
  A.dparams[(size_t)traj * NP + q] = s;
}

cudaError_t launch_adjoint_setup(int sys, const AdjArgs& A, int n_tiles, cudaStream_t st) {
  ABM_DISPATCH_SYSTEM(sys, (adjoint_setup_kernel<SYS><<<n_tiles, 32 * Sys<SYS>::D, 0, st>>>(A)));
  return cudaGetLastError();
}

// static: internal linkage, so the flag below belongs to this build of the
// library (a function-local static of an external template is one object for
// the whole process, shared by every loaded build)
template <int SYS, int HS>
static cudaError_t launch_adjoint_near_t(const AdjArgs& A, int n_active, long long s, int nb, cudaStream_t st) {
  constexpr int D = Sys<SYS>::D;
  const size_t smem = (size_t)(130 + 4 * HS) * kTrajPerTile * D * sizeof(double);
  static bool attr_set = false;  // per instantiation
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(adjoint_near_kernel<SYS, HS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    // the far kernels between these launches need the largest shared-memory
    // carveout; asking for it here too saves a reconfiguration per switch
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(adjoint_near_kernel<SYS, HS>, cudaFuncAttributePreferredSharedMemoryCarveout,
                               cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  adjoint_near_kernel<SYS, HS><<<n_active, 32 * (HS + 1) * D, smem, st>>>(A, s, nb);
  return cudaGetLastError();
}

template <int SYS, int L>
cudaError_t launch_adjoint_near_split_t(const AdjArgs& A, int n_active, long long s, int nb, cudaStream_t st) {
  adjoint_near_split_kernel<SYS, L><<<n_active * L, 32 * Sys<SYS>::D, 0, st>>>(A, s, nb);
  return cudaGetLastError();
}

// wpc: warps per state component, 1 (chain only), 2 or 3 (chain + helpers);
// split 4 or 8: the split kernel with each forward tile spread over split CTAs
cudaError_t launch_adjoint_near(int sys, const AdjArgs& A, int n_active, long long s, int nb, int wpc,
                                int split, cudaStream_t st) {
  cudaError_t err = cudaErrorInvalidValue;
  if (split == 4) {
    ABM_DISPATCH_SYSTEM(sys, err = (launch_adjoint_near_split_t<SYS, 4>(A, n_active, s, nb, st)));
    return err;
  }
  if (split == 8) {
    ABM_DISPATCH_SYSTEM(sys, err = (launch_adjoint_near_split_t<SYS, 8>(A, n_active, s, nb, st)));
    return err;
  }
  if (wpc == 3) {
    ABM_DISPATCH_SYSTEM(sys, err = (launch_adjoint_near_t<SYS, 2>(A, n_active, s, nb, st)));
  } else if (wpc == 2) {
    ABM_DISPATCH_SYSTEM(sys, err = (launch_adjoint_near_t<SYS, 1>(A, n_active, s, nb, st)));
  } else if (wpc == 1) {
    ABM_DISPATCH_SYSTEM(sys, err = (launch_adjoint_near_t<SYS, 0>(A, n_active, s, nb, st)));
  }
  return err;
}

cudaError_t launch_adjoint_finish(int sys, const AdjArgs& A, int M, cudaStream_t st) {
  ABM_DISPATCH_SYSTEM(sys, (adjoint_finish_kernel<SYS><<<(M * Sys<SYS>::NP + 255) / 256, 256, 0, st>>>(A, M)));
  return cudaGetLastError();
}

}  // namespace abm
