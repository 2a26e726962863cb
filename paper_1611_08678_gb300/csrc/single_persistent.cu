// Single-trajectory path (abm_solve) as one cooperative persistent kernel,
// FP64 throughout.  Time tiles of PB = 32 target steps.
//
// CTA 0 (near role) runs the sequential PECE steps of Sec. 2:
//   warps 0..D-1 : the chain, one state component per warp (component c on
//                  warp c, so the components of f evaluate on different
//                  SM sub-partitions): y^P_{n+1}, f(t_{n+1}, y^P), y_{n+1},
//                  f(t_{n+1}, y_{n+1}) (eq. (2) predictor and the corrector)
//   warp 3       : the scatter - when f_n is final it adds its contribution
//                  w_{m-n} f_n to every later target m of this tile and of
//                  the next tile (lane = target), so no per-step reduction is
//                  needed; the chain only adds the lag-0 term itself
// CTAs 1..G-1 (far role) compute, for tile j (targets [jB, jB+B)), the sums
// over history rows [1, (j-1)B) - rows that were final before tile j-1
// started, so far(j) overlaps the near steps of tile j-1.  CTA 0 adds the G-1
// partials in a fixed order (deterministic), plus the k = 0 terms
// b_n f_0, c_n f_0.  Rows [(j-1)B, jB) reach tile j through the scatter.
// This is the per-tile form of the paper's partial sums over earlier blocks
// gathered by the block owner (Sec. 3, Fig. 2).
//
// Synchronisation: CTA 0 publishes rows_done after each tile; far CTAs
// publish one count per tile slot.  Every wait is a bounded spin (clock64
// budget) that also gives up when another CTA has reported an error, so the
// kernel always terminates; a wait that runs out sets ABM_ERR_TIMEOUT.
#include <cuda/atomic>

#include <algorithm>
#include <cmath>
#include <cstdio>

#include "common.cuh"
#include "single.cuh"
#include "status_text.h"
#include "systems.cuh"

namespace abm {

namespace {

constexpr int PB = kPersistB;  // time-tile length
constexpr int PR = 4;          // ring of far slots
constexpr int PT = 256;        // threads per CTA

using dev_atomic = cuda::atomic_ref<unsigned long long, cuda::thread_scope_device>;

__device__ bool spin_geq(unsigned long long* flag, unsigned long long target, unsigned long long* status,
                         long long budget, int site, long long tile) {
  dev_atomic f(*flag), st(*status);
  const long long t0 = clock64();
  while (f.load(cuda::memory_order_acquire) < target) {
    if (st.load(cuda::memory_order_relaxed) != 0ull) return false;
    if (clock64() - t0 > budget) {
      report_timeout(status, site, tile, 0);
      return false;
    }
    __nanosleep(64);
  }
  return true;
}

__device__ __forceinline__ void named_bar(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

}  // namespace

// Sums over history rows [c0, c1) for targets s..s+B-1 of
//   b_{s+i-k} F[k][c] and a_{s+i-k} F[k][c];  writes B x 2D values to out.
// NT threads: each owns R consecutive targets over a contiguous sub-range of
// rows, the Toeplitz weights kept as a sliding register window.  NC = 1: one
// weight vector for every component; NC = D: component c uses b[c], a[c]
// (orders that differ per component).  F is read through L2
// (ld.global.cg): rows next to the ones read may be written by another SM
// later in the same launch.
template <int D, int B, int R, int NT, int NC>
__device__ void far_chunk(const double* __restrict__ F, const double* const* bv, const double* const* av,
                          long long s, long long c0, long long c1, double* red, double* out) {
  constexpr int RG = B / R, KL = NT / RG, V = 2 * D;
  static_assert(RG * KL == NT, "thread layout");
  static_assert(NC == 1 || NC == D, "weight sets");
  const int tid = threadIdx.x, rg = tid % RG, kl = tid / RG, i0 = rg * R;
  const long long len = c1 > c0 ? c1 - c0 : 0;
  const long long sub = (len + KL - 1) / KL;
  const long long kb = c0 + kl * sub, ke = min(c1, kb + sub);
  double accP[R][D], accC[R][D];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) accP[r][c] = accC[r][c] = 0.0;
  if (kb < ke) {
    const double* b[NC];
    const double* a[NC];
#pragma unroll
    for (int w = 0; w < NC; ++w) { b[w] = bv[w]; a[w] = av[w]; }
    double wb[R][NC], wa[R][NC];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int w = 0; w < NC; ++w) {
        wb[r][w] = __ldg(b[w] + (s + i0 + r - kb));
        wa[r][w] = __ldg(a[w] + (s + i0 + r - kb));
      }
    for (long long k = kb; k < ke; ++k) {
      double f[D];
#pragma unroll
      for (int c = 0; c < D; ++c) f[c] = __ldcg(F + k * D + c);
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) {
          accP[r][c] = fma(wb[r][NC == 1 ? 0 : c], f[c], accP[r][c]);
          accC[r][c] = fma(wa[r][NC == 1 ? 0 : c], f[c], accC[r][c]);
        }
#pragma unroll
      for (int r = R - 1; r > 0; --r)
#pragma unroll
        for (int w = 0; w < NC; ++w) { wb[r][w] = wb[r - 1][w]; wa[r][w] = wa[r - 1][w]; }
      if (k + 1 < ke) {
#pragma unroll
        for (int w = 0; w < NC; ++w) {
          wb[0][w] = __ldg(b[w] + (s + i0 - (k + 1)));
          wa[0][w] = __ldg(a[w] + (s + i0 - (k + 1)));
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      red[kl * (B * V) + (i0 + r) * V + c] = accP[r][c];
      red[kl * (B * V) + (i0 + r) * V + D + c] = accC[r][c];
    }
  __syncthreads();
  for (int idx = tid; idx < B * V; idx += NT) {
    double sum = 0.0;
#pragma unroll 8
    for (int q = 0; q < KL; ++q) sum += red[q * (B * V) + idx];
    out[idx] = sum;
  }
  __syncthreads();
}

template <int SYS, int NC>
__global__ void __launch_bounds__(PT, 1) single_persistent_kernel(PersistArgs A) {
  using S = Sys<SYS>;
  constexpr int D = S::D, V = 2 * D;
  constexpr int WL = 2 * PB + 1;  // near lags kept in shared memory per weight set
  extern __shared__ __align__(16) double dyn[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int W = gridDim.x - 1;  // far CTAs
  const int N = A.N;
  const int ntiles = (N + PB - 1) / PB;
  unsigned long long* rows_done = A.flags;
  unsigned long long* far_count = A.flags + 1;  // [PR]
  __shared__ int ok_s;

  const int j0 = A.start_tile;          // first tile stepped (resume)
  const int jfar = j0 > 2 ? j0 : 2;      // first tile with far sums computed here
  if (blockIdx.x > 0) {
    // ------------------------------ far role ------------------------------
    const int w = blockIdx.x - 1;
    for (int j = jfar; j < ntiles; ++j) {
      const long long s = (long long)j * PB, e = (long long)(j - 1) * PB;
      if (tid == 0) ok_s = spin_geq(rows_done, (unsigned long long)e, A.status, A.spin_budget, kSiteSingleFar, j);
      __syncthreads();
      if (!ok_s) return;
      const long long K = e - 1, chunk = (K + W - 1) / W;
      long long c0 = 1 + (long long)w * chunk, c1 = min(e, c0 + chunk);
      const size_t pofs = ((size_t)(j % PR) * W + w) * (PB * V);
      if (!in_bounds(A.status, kChkSingle, (long long)pofs + PB * V - 1, A.partial_elems)) return;
      if (c0 < c1 && !(in_bounds(A.status, kChkSingle, c1 * D - 1, A.f_elems) &&
                       in_bounds(A.status, kChkSingle, s + PB - 1 - c0, A.w_elems)))
        c1 = c0;  // reads nothing: zero sums
      far_chunk<D, PB, 4, PT, NC>(A.F, A.b, A.a, s, c0, c1, dyn, A.partial + pofs);
      __threadfence();
      __syncthreads();
      if (tid == 0 && j != A.withhold_tile) atomicAdd(far_count + (j % PR), 1ull);
    }
    return;
  }

  // -------------------------------- near role --------------------------------
  double* farv = dyn;                    // [PB * V]
  double* wsb = farv + PB * V;           // [NC][lags 0..2PB]
  double* wsa = wsb + NC * WL;
  __shared__ double Fs[4][kMaxD];        // ring of the last f rows
  __shared__ double accn[2][8];          // sums handed from the scatter warp to the chain
  __shared__ double ysh[kMaxD], ysh2[kMaxD], F0s[kMaxD], hhs[kMaxD], gs[kMaxD];

  const double* p = A.tp.p;
  for (int m = tid; m < NC * WL; m += PT) {
    wsb[m] = A.b[m / WL][m % WL];
    wsa[m] = A.a[m / WL][m % WL];
  }
  if (tid < NC) {
    hhs[tid] = pow(A.h, A.alpha[tid]);
    gs[tid] = *A.g[tid];
  }
  if (j0 == 0) {
    if (warp < D && lane == 0) {
      const int c = warp;
      double y0v[D];
#pragma unroll
      for (int q = 0; q < D; ++q) y0v[q] = A.tp.y0[q];
      const double f0 = S::fc(c, p, A.alpha[0], 0.0, y0v);
      F0s[c] = f0;
      Fs[0][c] = f0;
      A.F[c] = f0;
      A.Y[c] = A.tp.y0[c];
      if (A.YP) A.YP[c] = A.tp.y0[c];
    }
  } else {
    // resume at row s0 = j0 B: f_0 and the ring of the last rows from the
    // imported history; rows s0 + 1 and beyond are stepped below
    const long long s0 = (long long)j0 * PB;
    if (tid < D) {
      F0s[tid] = A.F[tid];
      for (long long n = s0 - 3 > 0 ? s0 - 3 : 0; n <= s0; ++n) Fs[n & 3][tid] = A.F[n * D + tid];
    }
    if (tid == 0) {  // rows 0..s0 are final: the far CTAs may start
      dev_atomic rd(*rows_done);
      rd.store((unsigned long long)(s0 + 1), cuda::memory_order_release);
    }
  }
  __syncthreads();
  const double h = A.h;

  // scatter-warp registers: sums for targets of this tile (cur) and the next
  double sPc[D], sCc[D], sPn[D], sCn[D];
#pragma unroll
  for (int q = 0; q < D; ++q) sPc[q] = sCc[q] = sPn[q] = sCn[q] = 0.0;
  if (j0 > 0 && warp == 3) {
    // resume: the next-tile sums tile j0 - 1 would have handed over - rows of
    // tile j0 - 1 weighted for the targets of tile j0, added in row order with
    // the same operations as in the stepping loop below
    const long long sp = (long long)(j0 - 1) * PB;
    for (long long n = sp > 1 ? sp : 1; n < sp + PB; ++n) {
      const long long lagn = sp + PB + lane - n;
#pragma unroll
      for (int q = 0; q < D; ++q) {
        const int w = (NC == 1 ? 0 : q) * WL;
        const double fq = A.F[n * D + q];
        sPn[q] = fma(wsb[w + lagn], fq, sPn[q]);
        sCn[q] = fma(wsa[w + lagn], fq, sCn[q]);
      }
    }
  }

  for (int j = j0; j < ntiles; ++j) {
    const long long s = (long long)j * PB;
    const int nb = (int)min((long long)PB, (long long)N - s);
    if (kChecked && tid == 0)  // rows written and lags read in this tile
      ok_s = in_bounds(A.status, kChkSingle, (s + nb + 1) * D - 1, A.f_elems) &&
             in_bounds(A.status, kChkSingle, s + PB - 1, A.w_elems);
    if (kChecked) {
      __syncthreads();
      if (!ok_s) return;
    }
    // ---- far sums of this tile: fixed-order sum of the W partials ----
    if (j >= 2) {
      if (tid == 0) {
        // far CTAs have counted every tile from jfar on in its slot j % PR
        const unsigned long long target = (unsigned long long)W * (unsigned long long)((j - jfar) / PR + 1);
        ok_s = spin_geq(far_count + (j % PR), target, A.status, A.spin_budget, kSiteSingleNear, j);
      }
      __syncthreads();
      if (!ok_s) return;
      const double* base = A.partial + (size_t)(j % PR) * W * (PB * V);
      for (int idx = tid; idx < PB * V; idx += PT) {
        double sum = 0.0;
        for (int q = 0; q < W; ++q) sum += __ldcg(base + (size_t)q * (PB * V) + idx);
        farv[idx] = sum;
      }
    } else {
      for (int idx = tid; idx < PB * V; idx += PT) farv[idx] = 0.0;
    }
    __syncthreads();
    // ---- scatter prologue: hand over the next-tile sums, add far and k = 0 terms ----
    if (warp == 3) {
      const long long m = s + lane;
#pragma unroll
      for (int q = 0; q < D; ++q) {
        sPc[q] = sPn[q]; sCc[q] = sCn[q];
        sPn[q] = 0.0; sCn[q] = 0.0;
      }
      if (lane < nb) {
#pragma unroll
        for (int q = 0; q < D; ++q) {
          const int w = NC == 1 ? 0 : q;
          sPc[q] += fma(A.b[w][m], F0s[q], farv[lane * V + q]);
          sCc[q] += fma(A.c[w][m], F0s[q], farv[lane * V + D + q]);
        }
      }
      if (lane == 0) {
#pragma unroll
        for (int q = 0; q < D; ++q) { accn[0][q] = sPc[q]; accn[0][D + q] = sCc[q]; }
      }
    }
    __syncthreads();
    // ---- the nb sequential steps ----
    if (warp < 4) {
      for (int i = 0; i < nb; ++i) {
        const long long n = s + i;
        const int par = i & 1;
        if (warp < D) {
          const int c = warp;
          const int wc = NC == 1 ? 0 : c;
          const double hh = hhs[wc], g = gs[wc];
          const double t1 = (double)(n + 1) * h;
          double y0c = A.tp.y0[0], y0dc = A.tp.y0d[0];
#pragma unroll
          for (int q = 1; q < D; ++q) {
            y0c = (c == q) ? A.tp.y0[q] : y0c;
            y0dc = (c == q) ? A.tp.y0d[q] : y0dc;
          }
          // Taylor sum of the initial values (eq. 2): y0, plus t y'(0) for an
          // order above one
          if ((A.taylor_mask >> c) & 1) y0c = fma(t1, y0dc, y0c);
          double v = 0.0;
          if (lane < 2) {
            v = accn[par][lane == 0 ? c : D + c];
            if (n >= 1) v = fma(lane == 0 ? wsb[wc * WL] : wsa[wc * WL], Fs[n & 3][c], v);
          }
          const double vc = __shfl_sync(0xffffffffu, v, 1);
          const double yp = fma(hh, v, y0c);
          if (lane == 0) ysh[c] = yp;
          named_bar(2, 32 * D);
          double ypv[D];
#pragma unroll
          for (int q = 0; q < D; ++q) ypv[q] = ysh[q];
          const double fp = S::fc(c, p, A.alpha[0], t1, ypv);
          double y = fma(hh, fma(g, fp, vc), y0c);
          if (lane == 0) ysh2[c] = y;
          named_bar(2, 32 * D);
          double yv[D];
#pragma unroll
          for (int q = 0; q < D; ++q) yv[q] = ysh2[q];
          // P(EC)^m E: further corrector passes evaluate f at the previous
          // pass's state; the exchange alternates between ysh and ysh2 (every
          // warp read the other one before the barrier it just passed)
          for (int it = 1; it < A.passes; ++it) {
            const double fq = S::fc(c, p, A.alpha[0], t1, yv);
            y = fma(hh, fma(g, fq, vc), y0c);
            double* xb = (it & 1) ? ysh : ysh2;
            if (lane == 0) xb[c] = y;
            named_bar(2, 32 * D);
#pragma unroll
            for (int q = 0; q < D; ++q) yv[q] = xb[q];
          }
          const double fy = S::fc(c, p, A.alpha[0], t1, yv);
          if (lane == 0) {
            Fs[(n + 1) & 3][c] = fy;
            A.F[(n + 1) * D + c] = fy;
            A.Y[(n + 1) * D + c] = y;
            if (A.YP) A.YP[(n + 1) * D + c] = yp;  // lane 0 of warp c holds component c
            if (!finite_bits(y) || !finite_bits(fy)) report_status(A.status, ABM_ERR_NONFINITE, 0, n + 1);
          }
        } else if (warp == 3) {
          if (n >= 1) {
            double fn[D];
#pragma unroll
            for (int q = 0; q < D; ++q) fn[q] = Fs[n & 3][q];
            const long long lagc = s + lane - n;       // target s+lane of this tile
            if (lagc > 0) {
#pragma unroll
              for (int q = 0; q < D; ++q) {
                const int w = (NC == 1 ? 0 : q) * WL;
                sPc[q] = fma(wsb[w + lagc], fn[q], sPc[q]);
                sCc[q] = fma(wsa[w + lagc], fn[q], sCc[q]);
              }
            }
            const long long lagn = s + PB + lane - n;  // target s+PB+lane of the next tile, >= 1
#pragma unroll
            for (int q = 0; q < D; ++q) {
              const int w = (NC == 1 ? 0 : q) * WL;
              sPn[q] = fma(wsb[w + lagn], fn[q], sPn[q]);
              sCn[q] = fma(wsa[w + lagn], fn[q], sCn[q]);
            }
          }
          if (i + 1 < nb && lane == i + 1) {
#pragma unroll
            for (int q = 0; q < D; ++q) { accn[par ^ 1][q] = sPc[q]; accn[par ^ 1][D + q] = sCc[q]; }
          }
        }
        named_bar(1, 128);
      }
    }
    // ---- publish: rows 0..s+nb are final ----
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      dev_atomic rd(*rows_done);
      rd.store((unsigned long long)(s + nb + 1), cuda::memory_order_release);
    }
    if (tid == 0) {
      dev_atomic st(*A.status);
      ok_s = st.load(cuda::memory_order_relaxed) == 0ull;  // any reported error ends the solve
    }
    __syncthreads();
    if (!ok_s) return;
  }
}

size_t persistent_smem_bytes() { return 116 * 1024; }

template <int SYS, int NC>
cudaError_t launch_persistent_t(const PersistArgs& A, int grid, cudaStream_t st) {
  auto fn = single_persistent_kernel<SYS, NC>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)persistent_smem_bytes());
  if (e != cudaSuccess) return e;
  PersistArgs a = A;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel((void*)fn, dim3(grid), dim3(PT), args, persistent_smem_bytes(), st);
}

cudaError_t launch_persistent(int sys, int nc, const PersistArgs& A, int grid, cudaStream_t st) {
  cudaError_t err = cudaErrorInvalidValue;
  if (nc == 1) {
    ABM_DISPATCH_SYSTEM(sys, err = (launch_persistent_t<SYS, 1>(A, grid, st)));
  } else {
    ABM_DISPATCH_SYSTEM(sys, {
      if (nc == Sys<SYS>::D) err = (launch_persistent_t<SYS, Sys<SYS>::D>(A, grid, st));
    });
  }
  return err;
}

int persistent_max_grid(int sys) {
  int blocks = 0, sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  ABM_DISPATCH_SYSTEM(sys, {
    cudaFuncSetAttribute(single_persistent_kernel<SYS, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)persistent_smem_bytes());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, single_persistent_kernel<SYS, 1>, PT,
                                                  persistent_smem_bytes());
    if (Sys<SYS>::D > 1) {  // the per-component kernel must fit as many CTAs
      int b2 = 0;
      cudaFuncSetAttribute(single_persistent_kernel<SYS, Sys<SYS>::D>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)persistent_smem_bytes());
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, single_persistent_kernel<SYS, Sys<SYS>::D>, PT,
                                                    persistent_smem_bytes());
      blocks = b2 < blocks ? b2 : blocks;
    }
  });
  return blocks * sms;
}

}  // namespace abm

// ============================================================================
// abm_solve_noalloc: the single-trajectory solve above for callers that may
// not allocate device memory.  Its scratch (f history, weights, far partials,
// flags, status) lives in one file-scope device array of fixed size that every
// GPU loading this library keeps until the process exits.
// ============================================================================
namespace abm {
cudaError_t launch_weights(double alpha, int M, double* b, double* a, double* c, double* g, cudaStream_t st);
namespace {

constexpr int kNoallocMaxN = 32768;  // largest N accepted
constexpr int kNoallocMaxW = 255;    // largest number of far CTAs (grid - 1)
constexpr size_t kAlignD = 32;       // 256-byte alignment, in doubles

constexpr size_t align_d(size_t n) { return (n + kAlignD - 1) / kAlignD * kAlignD; }
constexpr size_t kOffF = 0;
constexpr size_t kOffB = kOffF + align_d((size_t)(kNoallocMaxN + 1) * kMaxD);
constexpr size_t kWeightLen = (size_t)kNoallocMaxN + 2 * kPersistB + 2;  // lags 0..N+2B+1
constexpr size_t kOffA = kOffB + align_d(kWeightLen);
constexpr size_t kOffC = kOffA + align_d(kWeightLen);
constexpr size_t kOffG = kOffC + align_d(kWeightLen);
constexpr size_t kOffPart = kOffG + kAlignD;
constexpr size_t kOffFlags = kOffPart + align_d((size_t)kPersistRing * kNoallocMaxW * kPersistB * 2 * kMaxD);
constexpr size_t kScratchDoubles = kOffFlags + kAlignD;  // flags [0..4], status [8]

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

void set_msg(char* buf, size_t len, const char* msg) {
  if (buf && len) std::snprintf(buf, len, "%s", msg);
}

}  // namespace
}  // namespace abm

extern "C" abm_status abm_solve_noalloc(abm_system sys, double alpha, double h, int N, const double* params,
                                        const double* y0, double* Y, double* YP, void* stream, char* errbuf,
                                        size_t errbuf_len) {
  using namespace abm;
  int d = -1, np = -1;
  switch (sys) {
    case ABM_SYS_LINEAR: d = 1; np = 3; break;
    case ABM_SYS_MANUFACTURED: d = 1; np = 9; break;
    case ABM_SYS_LORENZ: case ABM_SYS_CHEN: case ABM_SYS_ROSSLER: case ABM_SYS_FINANCIAL: d = 3; np = 3; break;
    case ABM_SYS_HINDMARSH_ROSE: d = 3; np = 8; break;
  }
  if (d < 0) { set_msg(errbuf, errbuf_len, "abm_solve_noalloc: unknown system"); return ABM_ERR_INVALID_ARG; }
  if (N < 1 || N > kNoallocMaxN) {
    char m[160];
    std::snprintf(m, sizeof m, "abm_solve_noalloc: N = %d outside [1, %d], the size of its static scratch", N,
                  kNoallocMaxN);
    set_msg(errbuf, errbuf_len, m);
    return ABM_ERR_INVALID_ARG;
  }
  if (!(std::isfinite(alpha) && alpha > 0.0 && alpha <= 1.0) || !(std::isfinite(h) && h > 0.0) || !params ||
      !y0 || !Y) {
    set_msg(errbuf, errbuf_len, "abm_solve_noalloc: need alpha in (0,1], finite h > 0, non-null params/y0/Y");
    return ABM_ERR_INVALID_ARG;
  }
  TrajParams tp{};
  for (int i = 0; i < np; ++i) {
    if (!std::isfinite(params[i])) { set_msg(errbuf, errbuf_len, "abm_solve_noalloc: non-finite parameter"); return ABM_ERR_INVALID_ARG; }
    tp.p[i] = params[i];
  }
  for (int i = 0; i < d; ++i) {
    if (!std::isfinite(y0[i])) { set_msg(errbuf, errbuf_len, "abm_solve_noalloc: non-finite y0"); return ABM_ERR_INVALID_ARG; }
    tp.y0[i] = y0[i];
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) {
    set_msg(errbuf, errbuf_len, "abm_solve_noalloc: no usable current device");
    return ABM_ERR_CUDA;
  }
  // the array's device address on the current device, looked up on every call
  // (this allocates nothing once the library's module is loaded; the first
  // call on a device may load it); never cached, so it cannot go stale after
  // a device reset
  double* base = nullptr;
  {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) {
      char m[160];
      std::snprintf(m, sizeof m, "abm_solve_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      set_msg(errbuf, errbuf_len, m);
      return ABM_ERR_CUDA;
    }
    base = (double*)ptr;
  }
  int grid = persistent_max_grid(sys);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  grid = std::min(std::min(grid, sms), kNoallocMaxW + 1);
  if (grid < 2) { set_msg(errbuf, errbuf_len, "abm_solve_noalloc: fewer than 2 co-resident CTAs"); return ABM_ERR_UNSUPPORTED; }
  cudaStream_t st = (cudaStream_t)stream;
  auto cuda_err = [&](cudaError_t e, const char* what) {
    char m[200];
    std::snprintf(m, sizeof m, "abm_solve_noalloc: %s: %s", what, cudaGetErrorString(e));
    set_msg(errbuf, errbuf_len, m);
    return ABM_ERR_CUDA;
  };
  cudaError_t e;
  double* flags_d = base + kOffFlags;  // [0..4] wait flags, [8] status word
  // flags and status must start at zero: the array keeps the last call's contents
  if ((e = cudaMemsetAsync(flags_d, 0, kAlignD * sizeof(double), st)) != cudaSuccess) return cuda_err(e, "memset");
  // lags 0..N+2B+1: the largest lag the kernel reads is below N + 2B
  if ((e = launch_weights(alpha, N + 2 * kPersistB + 1, base + kOffB, base + kOffA, base + kOffC, base + kOffG, st)) !=
      cudaSuccess)
    return cuda_err(e, "weights kernel");
  PersistArgs A{};
  A.F = base + kOffF;
  A.Y = Y;
  A.YP = YP;
  for (int c = 0; c < kMaxD; ++c) {
    A.b[c] = base + kOffB;
    A.a[c] = base + kOffA;
    A.c[c] = base + kOffC;
    A.g[c] = base + kOffG;
    A.alpha[c] = alpha;
  }
  A.partial = base + kOffPart;
  A.flags = reinterpret_cast<unsigned long long*>(flags_d);
  A.status = reinterpret_cast<unsigned long long*>(flags_d + 8);
  A.tp = tp;
  A.h = h;
  A.taylor_mask = 0;
  A.N = N;
  A.spin_budget = 4000000000LL;
  A.withhold_tile = -1;
  A.passes = 1;
  A.start_tile = 0;
  if ((e = launch_persistent(sys, 1, A, grid, st)) != cudaSuccess) return cuda_err(e, "persistent kernel");
  unsigned long long w = 0;
  if ((e = cudaMemcpyAsync(&w, A.status, sizeof(w), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_err(e, "status read");
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_err(e, "stream synchronize");
  const int code = (int)(w >> 60);
  if (code) {
    char t[200], m[240];
    status_text(w, t, sizeof t);
    std::snprintf(m, sizeof m, "abm_solve_noalloc: device reported %s", t);
    set_msg(errbuf, errbuf_len, m);
    return (abm_status)code;
  }
  set_msg(errbuf, errbuf_len, "");
  return ABM_OK;
}
