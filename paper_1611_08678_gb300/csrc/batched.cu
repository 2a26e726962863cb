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
#include <type_traits>

#include "bf16split.cuh"
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
  const int bk = T.bucket * kMaxD;
  double alpha = A.bucket_alpha[bk];
  double p[kMaxParams], y0[D], f0[D];
#pragma unroll
  for (int q = 0; q < S::NP; ++q) p[q] = A.params[(size_t)src * S::NP + q];
#pragma unroll
  for (int c = 0; c < D; ++c) y0[c] = A.y0[(size_t)src * D + c];
  if (traj >= 0) {
#pragma unroll
    for (int c = 0; c < D; ++c) A.hhat[(size_t)traj * kMaxD + c] = pow(A.h[traj], A.bucket_alpha[bk + c]);
  }
  if (A.resume_row > 0) return;  // f_0 was imported with the history; Y row 0 is the caller's
  S::f(p, alpha, 0.0, y0, f0);
  double* F = A.F + T.f_off;
  if (!in_bounds(A.status, kChkSetup, T.f_off + lane * D + D - 1, A.f_elems)) return;
#pragma unroll
  for (int c = 0; c < D; ++c) F[lane * D + c] = f0[c];
  if (A.F32) {
    float* F32 = A.F32 + T.f_off;
#pragma unroll
    for (int c = 0; c < D; ++c) F32[lane * D + c] = (float)f0[c];
  }
  if (traj >= 0 && in_bounds(A.status, kChkSetup, (long long)traj * A.ldY * D + D - 1, A.y_elems)) {
#pragma unroll
    for (int c = 0; c < D; ++c) {
      A.Y[(size_t)traj * A.ldY * D + c] = y0[c];
      if (A.YP) A.YP[(size_t)traj * A.ldY * D + c] = y0[c];
    }
  }
}

// ---------------------------------------------------------------------------
// Near kernel: one CTA per column tile, nb sequential PECE steps in FP64, one
// lane per trajectory.  The window sums of step i+1 over rows already known
// (all but the newest, f_{s+i+1}) do not depend on step i, so they run one
// step ahead of the chain:
//   chain warps  (D, warp c = component c): add the far sums, the j = 0
//     terms, the helpers' partial window sums and the newest row term, then
//     y^P, f(y^P), y, f(y); the components meet through shared memory before
//     each evaluation of f (named barrier 1)
//   helper warps (HS per component): while step i's chain runs, helper
//     (c, q) sums rows r = q mod HS of step i+1's window over rows already in
//     shared memory, into a double-buffered partial-sum slot
// so the window (the FP64-throughput part) overlaps the chain (the FP64-
// latency part) instead of following it.  One barrier per step.  HS = 0: no
// helpers, each chain warp sums its whole window itself (fewer instructions;
// best when several tiles share an SM and hide each other's latency).
// ---------------------------------------------------------------------------
template <int SYS, int HS, int NC>
__global__ void __launch_bounds__(32 * (HS + 1) * Sys<SYS>::D) batched_near_kernel(BatchArgs A, long long s, int nb) {
  using S = Sys<SYS>;
  constexpr int D = S::D;
  constexpr int NT = 32 * (HS + 1) * D;
  constexpr int ld = kTrajPerTile * D;  // columns of the tile history
  // dynamic shared memory: f rows s..s+64 of this tile (FP64, the window every
  // sum reads) and the helpers' partial sums, [step parity][slice][column]
  extern __shared__ double near_dyn[];
  double (*Fw)[ld] = reinterpret_cast<double (*)[ld]>(near_dyn);
  constexpr int HSX = HS > 0 ? HS : 1;
  double (*Rp)[HSX][ld] = reinterpret_cast<double (*)[HSX][ld]>(near_dyn + 65 * ld);
  double (*Rc)[HSX][ld] = reinterpret_cast<double (*)[HSX][ld]>(near_dyn + (65 + 2 * HS) * ld);
  __shared__ double ysh[2][D][32], ysh2[2][D][32];  // predictor / corrector exchange
  // per weight set (NC = 1: every component; NC = D: one per component, for
  // orders that differ per component): lags 0..64, b_n and c_n of this tile's
  // targets.  NC is a template parameter so that equal orders keep the small
  // static footprint (four CTAs of the chain-only kernel per SM).
  __shared__ double wsb_[NC][65], wsa_[NC][65], bns_[NC][64], cns_[NC][64];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool chain = warp < D;
  const int c = chain ? warp : (warp - D) % D;  // component (column group)
  const int q = chain ? 0 : (warp - D) / D;     // helper slice
  const int tile = blockIdx.x;
  const TileDesc& T = A.tiles[tile];
  const int traj = T.traj[lane];
  const int src = traj >= 0 ? traj : T.traj[0];
  const int bk = T.bucket * kMaxD;
  const double alpha = A.bucket_alpha[bk];  // the system's own use of alpha
  const int col = lane * D + c;  // this thread's history column
  double* __restrict__ F = A.F + T.f_off;
  for (int m = threadIdx.x; m < NC * 65; m += NT) {
    wsb_[m / 65][m % 65] = A.bucket_b[bk + m / 65][m % 65];
    wsa_[m / 65][m % 65] = A.bucket_a[bk + m / 65][m % 65];
  }
  const bool w_ok = in_bounds(A.status, kChkNear, s + 63, A.w_elems);
  for (int m = threadIdx.x; m < NC * 64; m += NT) {
    bns_[m / 64][m % 64] = w_ok ? A.bucket_b[bk + m / 64][s + m % 64] : 0.0;
    cns_[m / 64][m % 64] = w_ok ? A.bucket_c[bk + m / 64][s + m % 64] : 0.0;
  }
  const int wset = NC == 1 ? 0 : c;  // this warp's component's weight set
  const double* wsb = wsb_[wset];
  const double* wsa = wsa_[wset];
  const double* bns = bns_[wset];
  const double* cns = cns_[wset];
  // the tile's rows s .. s + nb are read or written below
  const bool f_ok = in_bounds(A.status, kChkNear, T.f_off + (s + nb + 1) * ld - 1, A.f_elems);
  for (int m = threadIdx.x; m < ld; m += NT) Fw[0][m] = f_ok ? F[s * ld + m] : 0.0;
  for (int m = threadIdx.x; m < HS * ld; m += NT) {  // step 0 has no earlier window rows (helpers)
    Rp[0][m / ld][m % ld] = 0.0;
    Rc[0][m / ld][m % ld] = 0.0;
  }
  const int kfirst = s > 1 ? 0 : 1;  // window rows relative to s (row 0 is f_0 when s = 0)

  if (chain) {
    const double g = A.bucket_g[bk + c];
    const long long Ntraj = traj >= 0 ? (long long)A.N[traj] : 0;
    const double h = A.h[src];
    const double hh = traj >= 0 ? A.hhat[(size_t)traj * kMaxD + c] : pow(h, A.bucket_alpha[bk + c]);
    double p[kMaxParams];
#pragma unroll
    for (int k = 0; k < S::NP; ++k) p[k] = A.params[(size_t)src * S::NP + k];
    const double y0c0 = A.y0[(size_t)src * D + c];
    // Taylor sum of the initial values (eq. 2): y0, plus t y'(0) for an order above one
    const bool taylor2 = (A.bucket_taylor[T.bucket] >> c) & 1;
    const double y0dc = taylor2 && A.y0d ? A.y0d[(size_t)src * D + c] : 0.0;
    float* __restrict__ F32 = A.F32 ? A.F32 + T.f_off : nullptr;
    const double F0c = F[col];
    const double* __restrict__ farP = A.far + (((size_t)tile * 2) * A.B) * ld + col;
    const size_t far_q_stride = (size_t)A.n_tiles * 2 * A.B * ld;
    const size_t far_c_off = (size_t)A.B * ld;
    const bool far_ok = s <= 1 || in_bounds(A.status, kChkNear,
                                            (long long)((A.ksplit - 1) * far_q_stride + far_c_off +
                                                        (size_t)(((size_t)tile * 2) * A.B) * ld + (A.B - 1) * ld + col),
                                            A.far_elems);
    // far partial sums of the next target, loaded a step ahead
    double nxp = 0.0, nxc = 0.0;
    if (s > 1 && far_ok) {
      nxp = sum_parts(farP, A.ksplit, far_q_stride);
      nxc = sum_parts(farP + far_c_off, A.ksplit, far_q_stride);
    }
    bool reported = false;
    __syncthreads();
    for (int i = 0; i < nb; ++i) {
      const long long n = s + i;
      const int par = i & 1;
      double sp = fma(bns[i], F0c, nxp), sc = fma(cns[i], F0c, nxc);
      nxp = nxc = 0.0;
      if (s > 1 && i + 1 < nb && far_ok) {
        nxp = sum_parts(farP + (size_t)(i + 1) * ld, A.ksplit, far_q_stride);
        nxc = sum_parts(farP + far_c_off + (size_t)(i + 1) * ld, A.ksplit, far_q_stride);
      }
      if constexpr (HS > 0) {
#pragma unroll
        for (int k = 0; k < HS; ++k) { sp += Rp[par][k][col]; sc += Rc[par][k][col]; }
        if (i >= kfirst) {  // the newest window row, f_{s+i}
          const double fi = Fw[i][col];
          sp = fma(wsb[0], fi, sp);
          sc = fma(wsa[0], fi, sc);
        }
      } else {  // the whole window, rows [kfirst, i], two chains per sum
        double sp1 = 0.0, sc1 = 0.0;
        int r = kfirst;
        for (; r + 1 <= i; r += 2) {
          const double f0 = Fw[r][col], f1 = Fw[r + 1][col];
          sp = fma(wsb[i - r], f0, sp);
          sc = fma(wsa[i - r], f0, sc);
          sp1 = fma(wsb[i - r - 1], f1, sp1);
          sc1 = fma(wsa[i - r - 1], f1, sc1);
        }
        if (r <= i) {
          const double f0 = Fw[r][col];
          sp = fma(wsb[i - r], f0, sp);
          sc = fma(wsa[i - r], f0, sc);
        }
        sp += sp1;
        sc += sc1;
      }
      const double t1 = (double)(n + 1) * h;
      const double y0c = taylor2 ? fma(t1, y0dc, y0c0) : y0c0;
      const double yp = fma(hh, sp, y0c);
      ysh[par][c][lane] = yp;
      asm volatile("bar.sync 1, %0;" ::"n"(32 * D) : "memory");
      double ypv[D];
#pragma unroll
      for (int k = 0; k < D; ++k) ypv[k] = ysh[par][k][lane];
      const double fp = S::fc(c, p, alpha, t1, ypv);
      double y = fma(hh, fma(g, fp, sc), y0c);
      ysh2[par][c][lane] = y;
      asm volatile("bar.sync 1, %0;" ::"n"(32 * D) : "memory");
      double yv[D];
#pragma unroll
      for (int k = 0; k < D; ++k) yv[k] = ysh2[par][k][lane];
      // P(EC)^m E: further corrector passes evaluate f at the previous pass's
      // state; the exchange alternates between ysh and ysh2 (every chain warp
      // read the other one before the barrier it just passed)
      for (int it = 1; it < A.passes; ++it) {
        const double fq = S::fc(c, p, alpha, t1, yv);
        y = fma(hh, fma(g, fq, sc), y0c);
        double(*xb)[32] = (it & 1) ? ysh[par] : ysh2[par];
        xb[c][lane] = y;
        asm volatile("bar.sync 1, %0;" ::"n"(32 * D) : "memory");
#pragma unroll
        for (int k = 0; k < D; ++k) yv[k] = xb[k][lane];
      }
      const double fy = S::fc(c, p, alpha, t1, yv);
      Fw[i + 1][col] = fy;
      if (f_ok) {
        F[(n + 1) * ld + col] = fy;
        if (F32) F32[(n + 1) * ld + col] = (float)fy;
      }
      // the output row; a testing option of the checked build moves one
      // trajectory's row past the end of Y
      const long long yrow = (n + 1) + ((kChecked && traj == A.bad_traj) ? A.ldY * (long long)(1 << 20) : 0);
      if (n + 1 <= Ntraj && in_bounds(A.status, kChkNear, ((long long)traj * A.ldY + yrow) * D + c, A.y_elems)) {
        A.Y[((size_t)traj * A.ldY + yrow) * D + c] = y;
        if (A.YP) A.YP[((size_t)traj * A.ldY + yrow) * D + c] = yp;
        if (!reported && !(finite_bits(y) && finite_bits(fy))) {
          report_status(A.status, ABM_ERR_NONFINITE, traj, n + 1);
          reported = true;
        }
      }
      __syncthreads();
    }
  } else {
    __syncthreads();
    for (int i = 0; i < nb; ++i) {
      if (i + 1 < nb) {
        // partial window sums of step i+1 over rows r in [kfirst, i], r = q mod HS
        // (weights of lag i+1-r); two accumulator chains per sum
        const int nxt = (i + 1) & 1;
        double sp0 = 0.0, sc0 = 0.0, sp1 = 0.0, sc1 = 0.0;
        int r = kfirst + ((q - kfirst) % HS + HS) % HS;
#pragma unroll 1
        for (; r + HS <= i; r += 2 * HS) {
          const double f0 = Fw[r][col], f1 = Fw[r + HS][col];
          sp0 = fma(wsb[i + 1 - r], f0, sp0);
          sc0 = fma(wsa[i + 1 - r], f0, sc0);
          sp1 = fma(wsb[i + 1 - r - HS], f1, sp1);
          sc1 = fma(wsa[i + 1 - r - HS], f1, sc1);
        }
        if (r <= i) {
          const double f0 = Fw[r][col];
          sp0 = fma(wsb[i + 1 - r], f0, sp0);
          sc0 = fma(wsa[i + 1 - r], f0, sc0);
        }
        Rp[nxt][q][col] = sp0 + sp1;
        Rc[nxt][q][col] = sc0 + sc1;
      }
      __syncthreads();
    }
  }
  __syncthreads();
  if (A.Fsh) {
    // BF16 split of rows s..s+63 = K block s / 64 of this column tile (K-block
    // tiled, K-major inside): a unit is 8 rows of one column, split once and
    // stored as one 16-byte chunk per piece (row s of the first tile stays
    // zero: the j = 0 term is FP64)
    constexpr int UNITS = ld * 8;
    for (int u = threadIdx.x; u < UNITS; u += NT) {
      const int cc = u / 8, part = u % 8;
      __align__(16) __nv_bfloat16 v[3][8];
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int row = part * 8 + r;
        __nv_bfloat16 pcs[3];
        split3_bf16((s == 0 && row == 0) ? 0.0 : Fw[row][cc], pcs);
        v[0][r] = pcs[0];
        v[1][r] = pcs[1];
        v[2][r] = pcs[2];
      }
      const size_t off = (((size_t)T.slot * (A.fsh_ld / 64) + s / 64) * ld + cc) * 64 + part * 8;
      if (!in_bounds(A.status, kChkNear, (long long)off + 7, A.fsh_plane_elems)) continue;
#pragma unroll
      for (int pc = 0; pc < 3; ++pc)
        *reinterpret_cast<uint4*>(A.Fsh + (size_t)pc * A.fsh_plane + off) = *reinterpret_cast<const uint4*>(v[pc]);
    }
  }
}

// ---------------------------------------------------------------------------
// Split near kernel, for time tiles with few active column tiles: column tile
// t is spread over L CTAs (CTA b: tile b / L, part b % L), each holding
// T = 32 / L of its trajectories, so that the FP64 window work of a tile
// runs on L SMs.  One warp per state component; lane = j * L + l serves
// trajectory j of the part and lag slice l: the window sums of a step run
// over rows r = l mod L, and the L lanes of a trajectory add their slices
// with shuffles.  Every lane of a trajectory then runs the same PECE chain
// (identical values), lane l = 0 stores.  Same inputs, outputs and history
// layout as batched_near_kernel (the parts of a tile write disjoint columns).
// ---------------------------------------------------------------------------
template <int SYS, int L, int NC>
__global__ void __launch_bounds__(32 * Sys<SYS>::D) batched_near_split_kernel(BatchArgs A, long long s, int nb) {
  using S = Sys<SYS>;
  constexpr int D = S::D;
  constexpr int T = kTrajPerTile / L;       // trajectories of this CTA
  constexpr int ldt = kTrajPerTile * D;     // columns of the tile history
  constexpr int ldc = T * D;                // columns of this CTA
  __shared__ double Fw[65][ldc];            // f rows s..s+64 of this CTA's columns
  __shared__ double ysh[2][D][T], ysh2[2][D][T];
  __shared__ double wsb_[NC][65], wsa_[NC][65], bns_[NC][64], cns_[NC][64];  // per weight set
  const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;  // component, lane
  const int j = lane / L, l = lane % L;                      // trajectory of the part, lag slice
  const int tile = blockIdx.x / L, part = blockIdx.x % L;
  const TileDesc& Td = A.tiles[tile];
  const int tl = part * T + j;               // trajectory lane in the tile
  const int traj = Td.traj[tl];
  const int src = traj >= 0 ? traj : Td.traj[0];
  const int bk = Td.bucket * kMaxD;
  const double alpha = A.bucket_alpha[bk];  // the system's own use of alpha
  const int col = tl * D + c;                // column in the tile history
  const int cloc = j * D + c;                // column in this CTA's window
  double* __restrict__ F = A.F + Td.f_off;
  constexpr int NT = 32 * D;
  for (int m = threadIdx.x; m < NC * 65; m += NT) {
    wsb_[m / 65][m % 65] = A.bucket_b[bk + m / 65][m % 65];
    wsa_[m / 65][m % 65] = A.bucket_a[bk + m / 65][m % 65];
  }
  const bool w_ok = in_bounds(A.status, kChkNearSplit, s + 63, A.w_elems);
  for (int m = threadIdx.x; m < NC * 64; m += NT) {
    bns_[m / 64][m % 64] = w_ok ? A.bucket_b[bk + m / 64][s + m % 64] : 0.0;
    cns_[m / 64][m % 64] = w_ok ? A.bucket_c[bk + m / 64][s + m % 64] : 0.0;
  }
  const int wset = NC == 1 ? 0 : c;  // this warp's component's weight set
  const double* wsb = wsb_[wset];
  const double* wsa = wsa_[wset];
  const double* bns = bns_[wset];
  const double* cns = cns_[wset];
  const bool f_ok = in_bounds(A.status, kChkNearSplit, Td.f_off + (s + nb + 1) * ldt - 1, A.f_elems);
  for (int m = threadIdx.x; m < ldc; m += NT) Fw[0][m] = f_ok ? F[s * ldt + part * ldc + m] : 0.0;
  const int kfirst = s > 1 ? 0 : 1;  // window rows relative to s (row 0 is f_0 when s = 0)
  const double g = A.bucket_g[bk + c];
  const long long Ntraj = traj >= 0 ? (long long)A.N[traj] : 0;
  const double h = A.h[src];
  const double hh = traj >= 0 ? A.hhat[(size_t)traj * kMaxD + c] : pow(h, A.bucket_alpha[bk + c]);
  double p[kMaxParams];
#pragma unroll
  for (int k = 0; k < S::NP; ++k) p[k] = A.params[(size_t)src * S::NP + k];
  const double y0c0 = A.y0[(size_t)src * D + c];
  // Taylor sum of the initial values (eq. 2): y0, plus t y'(0) for an order above one
  const bool taylor2 = (A.bucket_taylor[Td.bucket] >> c) & 1;
  const double y0dc = taylor2 && A.y0d ? A.y0d[(size_t)src * D + c] : 0.0;
  float* __restrict__ F32 = A.F32 ? A.F32 + Td.f_off : nullptr;
  const double F0c = F[col];
  const double* __restrict__ farP = A.far + (((size_t)tile * 2) * A.B) * ldt + col;
  const size_t far_q_stride = (size_t)A.n_tiles * 2 * A.B * ldt;
  const size_t far_c_off = (size_t)A.B * ldt;
  const bool far_ok = s <= 1 || in_bounds(A.status, kChkNearSplit,
                                          (long long)((A.ksplit - 1) * far_q_stride + far_c_off +
                                                      (size_t)(((size_t)tile * 2) * A.B) * ldt + (A.B - 1) * ldt + col),
                                          A.far_elems);
  double nxp = 0.0, nxc = 0.0;  // far sums of the next target, loaded a step ahead
  if (s > 1 && l == 0 && far_ok) {
    nxp = sum_parts(farP, A.ksplit, far_q_stride);
    nxc = sum_parts(farP + far_c_off, A.ksplit, far_q_stride);
  }
  bool reported = false;
  __syncthreads();
  for (int i = 0; i < nb; ++i) {
    const long long n = s + i;
    const int par = i & 1;
    // lane slice of the window sums over rows [kfirst, i], two chains per sum
    double sp = 0.0, sc = 0.0, sp1 = 0.0, sc1 = 0.0;
    int r = kfirst + ((l - kfirst) % L + L) % L;
    for (; r + L <= i; r += 2 * L) {
      const double f0 = Fw[r][cloc], f1 = Fw[r + L][cloc];
      sp = fma(wsb[i - r], f0, sp);
      sc = fma(wsa[i - r], f0, sc);
      sp1 = fma(wsb[i - r - L], f1, sp1);
      sc1 = fma(wsa[i - r - L], f1, sc1);
    }
    if (r <= i) {
      const double f0 = Fw[r][cloc];
      sp = fma(wsb[i - r], f0, sp);
      sc = fma(wsa[i - r], f0, sc);
    }
    sp += sp1;
    sc += sc1;
#pragma unroll
    for (int o = 1; o < L; o <<= 1) {  // add the L slices of this trajectory
      sp += __shfl_xor_sync(0xffffffffu, sp, o);
      sc += __shfl_xor_sync(0xffffffffu, sc, o);
    }
    // far sums and the j = 0 term (lane 0 of the trajectory holds the far sums)
    sp += __shfl_sync(0xffffffffu, nxp, lane - l);
    sc += __shfl_sync(0xffffffffu, nxc, lane - l);
    sp = fma(bns[i], F0c, sp);
    sc = fma(cns[i], F0c, sc);
    nxp = nxc = 0.0;
    if (s > 1 && i + 1 < nb && l == 0 && far_ok) {
      nxp = sum_parts(farP + (size_t)(i + 1) * ldt, A.ksplit, far_q_stride);
      nxc = sum_parts(farP + far_c_off + (size_t)(i + 1) * ldt, A.ksplit, far_q_stride);
    }
    const double t1 = (double)(n + 1) * h;
    const double y0c = taylor2 ? fma(t1, y0dc, y0c0) : y0c0;
    const double yp = fma(hh, sp, y0c);
    if (l == 0) ysh[par][c][j] = yp;
    asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
    double ypv[D];
#pragma unroll
    for (int k = 0; k < D; ++k) ypv[k] = ysh[par][k][j];
    const double fp = S::fc(c, p, alpha, t1, ypv);
    double y = fma(hh, fma(g, fp, sc), y0c);
    if (l == 0) ysh2[par][c][j] = y;
    asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
    double yv[D];
#pragma unroll
    for (int k = 0; k < D; ++k) yv[k] = ysh2[par][k][j];
    // P(EC)^m E passes, exchanged through ysh / ysh2 alternately as in
    // batched_near_kernel
    for (int it = 1; it < A.passes; ++it) {
      const double fq = S::fc(c, p, alpha, t1, yv);
      y = fma(hh, fma(g, fq, sc), y0c);
      double(*xb)[T] = (it & 1) ? ysh[par] : ysh2[par];
      if (l == 0) xb[c][j] = y;
      asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
#pragma unroll
      for (int k = 0; k < D; ++k) yv[k] = xb[k][j];
    }
    const double fy = S::fc(c, p, alpha, t1, yv);
    if (l == 0) {
      Fw[i + 1][cloc] = fy;
      if (f_ok) {
        F[(n + 1) * ldt + col] = fy;
        if (F32) F32[(n + 1) * ldt + col] = (float)fy;
      }
      const long long yrow = (n + 1) + ((kChecked && traj == A.bad_traj) ? A.ldY * (long long)(1 << 20) : 0);
      if (n + 1 <= Ntraj && in_bounds(A.status, kChkNearSplit, ((long long)traj * A.ldY + yrow) * D + c, A.y_elems)) {
        A.Y[((size_t)traj * A.ldY + yrow) * D + c] = y;
        if (A.YP) A.YP[((size_t)traj * A.ldY + yrow) * D + c] = yp;
        if (!reported && !(finite_bits(y) && finite_bits(fy))) {
          report_status(A.status, ABM_ERR_NONFINITE, traj, n + 1);
          reported = true;
        }
      }
    }
    asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
  }
  if (A.Fsh) {
    // BF16 split of rows s..s+63 of this CTA's columns (layout as in
    // batched_near_kernel: K-block tiled, a unit is 8 rows of one column split
    // once, one 16-byte store per piece; row s of the first tile stays zero)
    constexpr int UNITS = ldc * 8;
    for (int u = threadIdx.x; u < UNITS; u += NT) {
      const int cc = u / 8, prt = u % 8;
      __align__(16) __nv_bfloat16 v[3][8];
#pragma unroll
      for (int rr = 0; rr < 8; ++rr) {
        const int row = prt * 8 + rr;
        __nv_bfloat16 pcs[3];
        split3_bf16((s == 0 && row == 0) ? 0.0 : Fw[row][cc], pcs);
        v[0][rr] = pcs[0];
        v[1][rr] = pcs[1];
        v[2][rr] = pcs[2];
      }
      const size_t off = (((size_t)Td.slot * (A.fsh_ld / 64) + s / 64) * ldt + part * ldc + cc) * 64 + prt * 8;
      if (!in_bounds(A.status, kChkNearSplit, (long long)off + 7, A.fsh_plane_elems)) continue;
#pragma unroll
      for (int pc = 0; pc < 3; ++pc)
        *reinterpret_cast<uint4*>(A.Fsh + (size_t)pc * A.fsh_plane + off) = *reinterpret_cast<const uint4*>(v[pc]);
    }
  }
}

// ---------------------------------------------------------------------------
// K-split reduction of the SIMT far kernels: once every CTA of a tile has
// stored its partial sums, the last one to finish (an atomic ticket per tile)
// adds the ksplit partials in split order into slot 0, so the sums are
// deterministic and the near kernel reads one value per target.  Thread
// layout of the callers: rows i0 .. i0+R-1, columns lane*D .. lane*D+D-1.
// ---------------------------------------------------------------------------
template <int D, int B, int R>
__device__ void reduce_split_partials(const BatchArgs& A, int tile, int i0, int lane, bool stored = true) {
  if (A.ksplit <= 1) return;
  constexpr int ld = kTrajPerTile * D;
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(A.far_ticket + tile, 1u) == (unsigned)(A.ksplit - 1);
  __syncthreads();
  if (!last) return;
  if (!stored) {  // (checked build) a CTA skipped its stores: only the ticket is reset
    if (threadIdx.x == 0) A.far_ticket[tile] = 0u;
    return;
  }
  __threadfence();
  const size_t qstride = (size_t)A.n_tiles * 2 * B * ld;
#pragma unroll
  for (int half = 0; half < 2; ++half)
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        double* out = A.far + (((size_t)tile * 2 + half) * B + i0 + r) * ld + lane * D + c;
        double v = __ldcg(out);
        for (int q = 1; q < A.ksplit; ++q) v += __ldcg(out + q * qstride);
        *out = v;
      }
  if (threadIdx.x == 0) A.far_ticket[tile] = 0u;  // ready for the next launch
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
  const double* __restrict__ wb = A.bucket_b[T.bucket * kMaxD];
  const double* __restrict__ wa = A.bucket_a[T.bucket * kMaxD];
  const double* __restrict__ F = A.F + T.f_off;
  // history rows [1, s) split into ksplit chunks
  const long long K = s - A.far_k0;
  const long long chunk = (K + A.ksplit - 1) / A.ksplit;
  const long long kb = A.far_k0 + (long long)q * chunk, ke = min(s, kb + chunk);
  const int i0 = warp * R;
  double accP[R][D], accC[R][D];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) accP[r][c] = accC[r][c] = 0.0;
  // rows [kb, ke) of the tile and lags up to s + B - 1 - kb are read; the
  // partial sums of this split are written below
  const bool ok = kb >= ke || (in_bounds(A.status, kChkFarFp64, T.f_off + ke * ld - 1, A.f_elems) &&
                               in_bounds(A.status, kChkFarFp64, s + B - 1 - kb, A.w_elems));
  const bool out_ok =
      in_bounds(A.status, kChkFarFp64, ((((long long)q * A.n_tiles + tile) * 2 + 1) * B + B - 1) * ld + ld - 1,
                A.far_elems);
  if (!out_ok) {
    reduce_split_partials<D, B, R>(A, tile, i0, lane, false);
    return;
  }
  if (kb < ke && ok) {
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
  reduce_split_partials<D, B, R>(A, tile, i0, lane);
}

// ---------------------------------------------------------------------------
// Far kernel, FP32 operands (SIMT): the far sums of Sec. 2 with F and the
// weights rounded to FP32, FP32 products and sums within 64-row history
// blocks, and the block sums added into a compensated FP32 pair (TwoSum) per
// output, widened to FP64 at the end.  Grid (active tiles, history splits),
// 256 threads: warp w owns target rows 8w .. 8w+7, lane = trajectory (its D
// columns), so a thread holds an 8 x D tile of predictor and corrector sums.
// Each 64-row block of the tile's FP32 history (24 KB for D = 3) is staged in
// shared memory by cp.async, double-buffered, with the 127 lags of b and a
// that block needs; a thread walks the block in chunks of 8 rows with the
// 15 weights those rows and targets need in registers (the Toeplitz
// structure: w_{i-k} for i - k in a 15-wide band).
// ---------------------------------------------------------------------------
namespace {
constexpr int kF32Block = 64;  // history rows per staged block and per FP32 partial sum
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
// (hi, lo) += x, compensated (TwoSum)
__device__ __forceinline__ void two_sum_f32(float& hi, float& lo, float x) {
  const float sum = __fadd_rn(hi, x);
  const float bp = __fsub_rn(sum, hi);
  lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(sum, bp)), __fsub_rn(x, bp)));
  hi = sum;
}
}  // namespace

template <int D, int B>
__global__ void __launch_bounds__(256, 1) batched_far_fp32_kernel(BatchArgs A, long long s) {
  static_assert(B == 64, "one warp per 8 of the 64 target rows");
  constexpr int R = 8, KS = kF32Block, WL = KS + B - 1;  // lags per block: 127
  constexpr int ld = kTrajPerTile * D;
  extern __shared__ __align__(16) float f32_dyn[];
  float (*Fs)[KS][ld] = reinterpret_cast<float (*)[KS][ld]>(f32_dyn);  // [2][KS][ld]
  float (*Wbs)[WL + 1] = reinterpret_cast<float (*)[WL + 1]>(f32_dyn + 2 * KS * ld);
  float (*Was)[WL + 1] = Wbs + 2;
  const int tile = blockIdx.x, q = blockIdx.y, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const TileDesc& T = A.tiles[tile];
  const float* __restrict__ wb = A.bucket_b32[T.bucket * kMaxD];
  const float* __restrict__ wa = A.bucket_a32[T.bucket * kMaxD];
  const float* __restrict__ F = A.F32 + T.f_off;
  const long long K = s - A.far_k0;
  const long long chunk = (K + A.ksplit - 1) / A.ksplit;
  const long long kb = A.far_k0 + (long long)q * chunk, ke = min(s, kb + chunk);
  const int i0 = warp * R;
  const bool ok = kb >= ke || (in_bounds(A.status, kChkFarFp32, T.f_off + ke * ld - 1, A.f_elems) &&
                               in_bounds(A.status, kChkFarFp32, s + B - 1 - kb, A.w_elems));
  if (!in_bounds(A.status, kChkFarFp32, ((((long long)q * A.n_tiles + tile) * 2 + 1) * B + B - 1) * ld + ld - 1,
                 A.far_elems)) {
    reduce_split_partials<D, B, R>(A, tile, i0, lane, false);
    return;
  }
  float hiP[R][D], loP[R][D], hiC[R][D], loC[R][D];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) hiP[r][c] = loP[r][c] = hiC[r][c] = loC[r][c] = 0.0f;
  const int nblk = ok && kb < ke ? (int)((ke - kb + KS - 1) / KS) : 0;
  // stage block t: rows kb + t KS ... (whole 16-byte chunks; rows at or past
  // ke are zero-filled so they add nothing) and lags s - k0 - 63 .. s + 63 - k0
  auto stage = [&](int t) {
    const long long k0 = kb + (long long)t * KS;
    const int rows = (int)min((long long)KS, ke - k0);
    float* dst = &Fs[t & 1][0][0];
    const float* src = F + k0 * ld;
    for (int v = threadIdx.x; v < KS * ld / 4; v += blockDim.x) {
      if (v * 4 < rows * ld) cp_async16(dst + v * 4, src + v * 4);
      else *reinterpret_cast<float4*>(dst + v * 4) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int j = threadIdx.x; j < WL; j += blockDim.x) {
      const long long lag = s - k0 - (KS - 1) + j;
      const bool in = lag >= 0 && lag < A.w_elems;
      Wbs[t & 1][j] = in ? wb[lag] : 0.0f;
      Was[t & 1][j] = in ? wa[lag] : 0.0f;
    }
    cp_async_commit();
  };
  if (nblk > 0) stage(0);
  for (int t = 0; t < nblk; ++t) {
    if (t + 1 < nblk) {
      stage(t + 1);
      cp_async_wait_one();
    } else {
      cp_async_wait_all();
    }
    __syncthreads();
    const int buf = t & 1;
    float accP[R][D], accC[R][D];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) accP[r][c] = accC[r][c] = 0.0f;
#pragma unroll 1
    for (int k8 = 0; k8 < KS; k8 += 8) {
      // w_{lag} for lag = s + i - k, i = i0 + r, k = k0 + k8 + kk: staged index
      // i - (k - k0) + 63 = i0 - k8 + 56 + (r - kk + 7)
      float b15[15], a15[15];
#pragma unroll
      for (int u = 0; u < 15; ++u) {
        b15[u] = Wbs[buf][i0 - k8 + 56 + u];
        a15[u] = Was[buf][i0 - k8 + 56 + u];
      }
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        float f[D];
#pragma unroll
        for (int c = 0; c < D; ++c) f[c] = Fs[buf][k8 + kk][lane * D + c];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
          for (int c = 0; c < D; ++c) {
            accP[r][c] = fmaf(b15[r - kk + 7], f[c], accP[r][c]);
            accC[r][c] = fmaf(a15[r - kk + 7], f[c], accC[r][c]);
          }
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        two_sum_f32(hiP[r][c], loP[r][c], accP[r][c]);
        two_sum_f32(hiC[r][c], loC[r][c], accC[r][c]);
      }
    __syncthreads();  // this buffer is staged again two blocks on
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    double* P = A.far + ((((size_t)q * A.n_tiles + tile) * 2 + 0) * B + i0 + r) * ld + lane * D;
    double* C = A.far + ((((size_t)q * A.n_tiles + tile) * 2 + 1) * B + i0 + r) * ld + lane * D;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      P[c] = (double)hiP[r][c] + (double)loP[r][c];
      C[c] = (double)hiC[r][c] + (double)loC[r][c];
    }
  }
  reduce_split_partials<D, B, R>(A, tile, i0, lane);
}

size_t far_fp32_smem_bytes(int d) {
  return (2 * (size_t)kF32Block * kTrajPerTile * d + 4 * (size_t)(kF32Block + 64)) * sizeof(float);
}

// ---------------------------------------------------------------------------
// Far kernels for order groups whose components have different orders
// (non-commensurate systems): the same sums with component c's weights on
// column lane * D + c, one component after another (lane = trajectory).
// FP64, or FP32 operands with FP32 sums within KB-row blocks (KB = 0: FP64).
// ---------------------------------------------------------------------------
template <int D, int B, int KB>
__global__ void __launch_bounds__(256) batched_far_percomp_kernel(BatchArgs A, long long s) {
  constexpr int R = B / 8;
  constexpr int ld = kTrajPerTile * D;
  using real = typename std::conditional<KB == 0, double, float>::type;
  const int tile = blockIdx.x, q = blockIdx.y, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const TileDesc& T = A.tiles[tile];
  const long long K = s - A.far_k0;
  const long long chunk = (K + A.ksplit - 1) / A.ksplit;
  const long long kb = A.far_k0 + (long long)q * chunk, ke = min(s, kb + chunk);
  const long long blk = KB == 0 ? (ke > kb ? ke - kb : 1) : KB;
  const int i0 = warp * R;
  const bool ok = kb >= ke || (in_bounds(A.status, kChkFarPerComp, T.f_off + ke * ld - 1, A.f_elems) &&
                               in_bounds(A.status, kChkFarPerComp, s + B - 1 - kb, A.w_elems));
  if (!ok || !in_bounds(A.status, kChkFarPerComp, ((((long long)q * A.n_tiles + tile) * 2 + 1) * B + B - 1) * ld + ld - 1,
                        A.far_elems)) {
    reduce_split_partials<D, B, R>(A, tile, i0, lane, false);
    return;
  }
  for (int c = 0; c < D; ++c) {
    const real* __restrict__ wb;
    const real* __restrict__ wa;
    const real* __restrict__ F;
    if constexpr (KB == 0) {
      wb = A.bucket_b[T.bucket * kMaxD + c];
      wa = A.bucket_a[T.bucket * kMaxD + c];
      F = A.F + T.f_off;
    } else {
      wb = A.bucket_b32[T.bucket * kMaxD + c];
      wa = A.bucket_a32[T.bucket * kMaxD + c];
      F = A.F32 + T.f_off;
    }
    double dP[R], dC[R];
#pragma unroll
    for (int r = 0; r < R; ++r) dP[r] = dC[r] = 0.0;
    for (long long k0 = kb; k0 < ke; k0 += blk) {
      const long long k1 = min(ke, k0 + blk);
      real accP[R], accC[R], wbv[R], wav[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        accP[r] = accC[r] = (real)0;
        wbv[r] = wb[s + i0 + r - k0];
        wav[r] = wa[s + i0 + r - k0];
      }
      for (long long k = k0; k < k1; ++k) {
        const real f = F[k * ld + lane * D + c];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          accP[r] = fma(wbv[r], f, accP[r]);
          accC[r] = fma(wav[r], f, accC[r]);
        }
#pragma unroll
        for (int r = R - 1; r > 0; --r) { wbv[r] = wbv[r - 1]; wav[r] = wav[r - 1]; }
        if (k + 1 < k1) { wbv[0] = wb[s + i0 - (k + 1)]; wav[0] = wa[s + i0 - (k + 1)]; }
      }
#pragma unroll
      for (int r = 0; r < R; ++r) { dP[r] += (double)accP[r]; dC[r] += (double)accC[r]; }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      A.far[((((size_t)q * A.n_tiles + tile) * 2 + 0) * B + i0 + r) * ld + lane * D + c] = dP[r];
      A.far[((((size_t)q * A.n_tiles + tile) * 2 + 1) * B + i0 + r) * ld + lane * D + c] = dC[r];
    }
  }
  reduce_split_partials<D, B, R>(A, tile, i0, lane);
}

// ---------------------------------------------------------------------------
cudaError_t launch_batched_setup(int sys, const BatchArgs& A, int n_tiles, cudaStream_t st) {
  ABM_DISPATCH_SYSTEM(sys, (batched_setup_kernel<SYS><<<n_tiles, kTrajPerTile, 0, st>>>(A)));
  return cudaGetLastError();
}

// static: internal linkage, so the flag below belongs to this build of the
// library (a function-local static of an external template is one object for
// the whole process, shared by every loaded build)
template <int SYS, int HS, int NC>
static cudaError_t launch_near_nc(const BatchArgs& A, int n_active, long long s, int nb, cudaStream_t st) {
  constexpr int D = Sys<SYS>::D;
  const size_t smem = (size_t)(65 + 4 * HS) * kTrajPerTile * D * sizeof(double);
  static bool attr_set = false;  // per instantiation; a plan is used from one thread
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(batched_near_kernel<SYS, HS, NC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    // the far kernels between these launches need the largest shared-memory
    // carveout; asking for it here too saves a reconfiguration per switch
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(batched_near_kernel<SYS, HS, NC>, cudaFuncAttributePreferredSharedMemoryCarveout,
                               cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  batched_near_kernel<SYS, HS, NC><<<n_active, 32 * (HS + 1) * D, smem, st>>>(A, s, nb);
  return cudaGetLastError();
}

template <int SYS, int HS>
static cudaError_t launch_near_t(const BatchArgs& A, int n_active, long long s, int nb, cudaStream_t st) {
  if (A.per_comp) return launch_near_nc<SYS, HS, Sys<SYS>::D>(A, n_active, s, nb, st);
  return launch_near_nc<SYS, HS, 1>(A, n_active, s, nb, st);
}

template <int SYS, int L>
cudaError_t launch_near_split_t(const BatchArgs& A, int n_active, long long s, int nb, cudaStream_t st) {
  if (A.per_comp)
    batched_near_split_kernel<SYS, L, Sys<SYS>::D><<<n_active * L, 32 * Sys<SYS>::D, 0, st>>>(A, s, nb);
  else
    batched_near_split_kernel<SYS, L, 1><<<n_active * L, 32 * Sys<SYS>::D, 0, st>>>(A, s, nb);
  return cudaGetLastError();
}

// wpc: warps per state component, 1 (chain only), 2, 3 or 5 (chain + helpers);
// split > 1: the split kernel with each column tile spread over split CTAs
cudaError_t launch_batched_near(int sys, const BatchArgs& A, int n_active, long long s, int nb, int wpc,
                                int split, cudaStream_t st) {
  cudaError_t err = cudaErrorInvalidValue;
  if (split == 2) {
    ABM_DISPATCH_SYSTEM(sys, err = (launch_near_split_t<SYS, 2>(A, n_active, s, nb, st)));
    return err;
  }
  if (split == 4) {
    ABM_DISPATCH_SYSTEM(sys, err = (launch_near_split_t<SYS, 4>(A, n_active, s, nb, st)));
    return err;
  }
  if (split == 8) {
    ABM_DISPATCH_SYSTEM(sys, err = (launch_near_split_t<SYS, 8>(A, n_active, s, nb, st)));
    return err;
  }
  if (split == 16) {
    ABM_DISPATCH_SYSTEM(sys, err = (launch_near_split_t<SYS, 16>(A, n_active, s, nb, st)));
    return err;
  }
  if (wpc == 5) {
    ABM_DISPATCH_SYSTEM(sys, err = (launch_near_t<SYS, 4>(A, n_active, s, nb, st)));
  } else if (wpc == 3) {
    ABM_DISPATCH_SYSTEM(sys, err = (launch_near_t<SYS, 2>(A, n_active, s, nb, st)));
  } else if (wpc == 2) {
    ABM_DISPATCH_SYSTEM(sys, err = (launch_near_t<SYS, 1>(A, n_active, s, nb, st)));
  } else if (wpc == 1) {
    ABM_DISPATCH_SYSTEM(sys, err = (launch_near_t<SYS, 0>(A, n_active, s, nb, st)));
  }
  return err;
}

// static: internal linkage, so the flag belongs to this build of the library
template <int D>
static cudaError_t set_far_fp32_smem() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(batched_far_fp32_kernel<D, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)far_fp32_smem_bytes(D));
  if (e == cudaSuccess) done = true;
  return e;
}

cudaError_t launch_batched_far(int d, abm_precision prec, const BatchArgs& A, int n_active, long long s,
                               cudaStream_t st) {
  dim3 grid(n_active, A.ksplit);
  if (A.per_comp) {
    if (A.B != 64) return cudaErrorInvalidValue;
    if (prec == ABM_PREC_FP64) {
      if (d == 3) batched_far_percomp_kernel<3, 64, 0><<<grid, 256, 0, st>>>(A, s);
      else batched_far_percomp_kernel<1, 64, 0><<<grid, 256, 0, st>>>(A, s);
    } else {
      if (d == 3) batched_far_percomp_kernel<3, 64, 128><<<grid, 256, 0, st>>>(A, s);
      else batched_far_percomp_kernel<1, 64, 128><<<grid, 256, 0, st>>>(A, s);
    }
    return cudaGetLastError();
  }
  if (prec == ABM_PREC_FP64) {
    if (A.B != 64) return cudaErrorInvalidValue;
    if (d == 3) batched_far_fp64_kernel<3, 64><<<grid, 256, 0, st>>>(A, s);
    else batched_far_fp64_kernel<1, 64><<<grid, 256, 0, st>>>(A, s);
  } else {
    if (A.B != 64) return cudaErrorInvalidValue;
    if (d == 3) {
      cudaError_t e = set_far_fp32_smem<3>();
      if (e != cudaSuccess) return e;
      batched_far_fp32_kernel<3, 64><<<grid, 256, far_fp32_smem_bytes(3), st>>>(A, s);
    } else {
      cudaError_t e = set_far_fp32_smem<1>();
      if (e != cudaSuccess) return e;
      batched_far_fp32_kernel<1, 64><<<grid, 256, far_fp32_smem_bytes(1), st>>>(A, s);
    }
  }
  return cudaGetLastError();
}

}  // namespace abm
