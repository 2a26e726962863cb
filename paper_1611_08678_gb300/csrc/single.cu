// Stand-alone FP64 far-history kernel (abm_far_history): the history sums of
// Sec. 2 (eq. (2) predictor, corrector) for one tile of B targets over a
// range of history rows, split over many CTAs.  The single-trajectory solve
// itself runs in single_persistent.cu.
#include "common.cuh"
#include "systems.cuh"
#include "single.cuh"

namespace abm {

// ----------------------------------------------------------------------------
// Far kernel: P[i][c] = sum_{k in [k_lo,k_hi)} b_{s+i-k} F[k][c],
//             C[i][c] = sum_{k in [k_lo,k_hi)} a_{s+i-k} F[k][c],  i in [0, B).
// Each CTA takes a contiguous chunk of k, each thread R consecutive target rows
// over a contiguous sub-chunk, with the Toeplitz weights kept as a sliding
// register window (one new b and one new a per k).  Partials of all CTAs are
// combined in a fixed order by the last CTA to finish (ticket counter), so the
// result does not depend on scheduling.
// ----------------------------------------------------------------------------


template <int D, int B, int R>
__global__ void __launch_bounds__(128) far_single_kernel(FarSingleArgs A) {
  constexpr int RG = B / R;          // row groups
  constexpr int KL = 128 / RG;       // k lanes per row group
  static_assert(RG * KL == 128, "thread layout");
  constexpr int V = 2 * D;           // values per target row
  __shared__ double red[KL][B * V];
  __shared__ bool am_last;

  const int tid = threadIdx.x;
  const int rg = tid % RG, kl = tid / RG;
  const int i0 = rg * R;
  const long long c0 = A.k_lo + (long long)blockIdx.x * A.chunk;
  const long long c1 = min(A.k_hi, c0 + A.chunk);
  const long long sub = (c1 - c0 + KL - 1) / KL;
  const long long kb = c0 + kl * sub, ke = min(c1, kb + sub);

  double accP[R][D], accC[R][D];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) accP[r][c] = accC[r][c] = 0.0;

  if (kb < ke) {
    double wb[R], wa[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      long long lag = A.s + i0 + r - kb;  // >= 1 because kb < k_hi <= s
      wb[r] = A.b[lag];
      wa[r] = A.a[lag];
    }
    for (long long k = kb; k < ke; ++k) {
      double f[D];
#pragma unroll
      for (int c = 0; c < D; ++c) f[c] = A.F[k * D + c];
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) {
          accP[r][c] = fma(wb[r], f[c], accP[r][c]);
          accC[r][c] = fma(wa[r], f[c], accC[r][c]);
        }
      // slide the window: lag of row r at k+1 is the lag of row r-1 at k
#pragma unroll
      for (int r = R - 1; r > 0; --r) { wb[r] = wb[r - 1]; wa[r] = wa[r - 1]; }
      long long lag0 = A.s + i0 - (k + 1);
      if (k + 1 < ke) { wb[0] = A.b[lag0]; wa[0] = A.a[lag0]; }
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      red[kl][(i0 + r) * V + c] = accP[r][c];
      red[kl][(i0 + r) * V + D + c] = accC[r][c];
    }
  __syncthreads();
  double* mine = A.partial + (size_t)blockIdx.x * B * V;
  for (int idx = tid; idx < B * V; idx += 128) {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < KL; ++q) s += red[q][idx];
    mine[idx] = s;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    unsigned int t = atomicAdd(A.ticket, 1u);
    am_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (am_last) {
    __threadfence();
    for (int idx = tid; idx < B * V; idx += 128) {
      double s = 0.0;
      for (unsigned int g = 0; g < gridDim.x; ++g) s += __ldcg(A.partial + (size_t)g * B * V + idx);
      A.out[idx] = s;
    }
    if (tid == 0) *A.ticket = 0u;
  }
}

cudaError_t launch_far_single(int d, const FarSingleArgs& A, int B, int grid, cudaStream_t st) {
  if (d == 3 && B == 64) far_single_kernel<3, 64, 4><<<grid, 128, 0, st>>>(A);
  else if (d == 1 && B == 64) far_single_kernel<1, 64, 4><<<grid, 128, 0, st>>>(A);
  else if (d == 3 && B == 32) far_single_kernel<3, 32, 2><<<grid, 128, 0, st>>>(A);
  else if (d == 1 && B == 32) far_single_kernel<1, 32, 2><<<grid, 128, 0, st>>>(A);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace abm
