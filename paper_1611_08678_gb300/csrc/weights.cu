// A1 - weight generation.  One thread per lag m, as in the paper's CUDA
// variant (Sec. 4, "CUDA simulations": each thread computes the weight of its
// index).  The definitions (Sec. 2; the '+' printed inside b_n read as '-'):
//   b_m = ((m+1)^a - m^a) / Gamma(a+1)
//   a_m = ((m+2)^(a+1) - 2(m+1)^(a+1) + m^(a+1)) / Gamma(a+2)
//   c_m = (m^(a+1) - (m-a)(m+1)^a) / Gamma(a+2)
// Evaluated without the catastrophic cancellation of the plain differences:
//   b_m (m >= 1): m^a * expm1(a * log1p(1/m)) / Gamma(a+1)
//   a_m (m >= 16): centred expansion at m+1, z = 1/(m+1), p = a+1,
//          (m+1)^p * 2 * sum_{j>=1} C(p, 2j) z^(2j) / Gamma(a+2)  (terms > 0 for
//          a <= 1; for a in (1, 2] the later terms alternate, each below
//          z^2 / 12 of the one before)
//   c_m (m >= 16): x = 1/m,
//          m^p * sum_{k>=2} C(a, k-1) (k-1)(a+1)/k x^k / Gamma(a+2)
//   a_m, c_m (1 <= m < 16): 16-point Gauss-Legendre quadrature of the
//          product-integration kernels (u^(a-1) times the hat functions of the
//          piecewise-linear interpolant), smooth on each cell for m >= 1:
//          a_m = [int_m^{m+1} u^(a-1)(u-m) du + int_{m+1}^{m+2} u^(a-1)(m+2-u) du] / Gamma(a)
//          c_m = int_m^{m+1} u^(a-1)(u-m) du / Gamma(a)
//   m = 0: b_0 = 1/Gamma(a+1), a_0 = 2 expm1(a ln 2)/Gamma(a+2), c_0 = a/Gamma(a+2).
// Gamma: the host C library's tgammal in extended precision (called, not
// reimplemented), rounded once to FP64.
#include <cmath>

#include "common.cuh"

namespace abm {

// Gauss-Legendre nodes/weights on [-1, 1], 16 points (8 symmetric pairs).
__constant__ double kGLx[8] = {
    9.50125098376374405e-02, 2.81603550779258915e-01, 4.58016777657227370e-01,
    6.17876244402643771e-01, 7.55404408355002999e-01, 8.65631202387831755e-01,
    9.44575023073232600e-01, 9.89400934991649939e-01};
__constant__ double kGLw[8] = {
    1.89450610455068641e-01, 1.82603415044923639e-01, 1.69156519395002647e-01,
    1.49595988816576708e-01, 1.24628971255534071e-01, 9.51585116824926053e-02,
    6.22535239386474565e-02, 2.71524594117541762e-02};

constexpr int kQuadBelow = 16;

// int_lo^{lo+1} u^(a-1) * (u - lo) du      (rising half-hat)
__device__ double quad_rise(double alpha, double lo) {
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    double u1 = lo + 0.5 + 0.5 * kGLx[q], u2 = lo + 0.5 - 0.5 * kGLx[q];
    s += kGLw[q] * (pow(u1, alpha - 1.0) * (u1 - lo) + pow(u2, alpha - 1.0) * (u2 - lo));
  }
  return 0.5 * s;
}

// int_lo^{lo+1} u^(a-1) * (lo + 1 - u) du  (falling half-hat)
__device__ double quad_fall(double alpha, double lo) {
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    double u1 = lo + 0.5 + 0.5 * kGLx[q], u2 = lo + 0.5 - 0.5 * kGLx[q];
    s += kGLw[q] * (pow(u1, alpha - 1.0) * (lo + 1.0 - u1) + pow(u2, alpha - 1.0) * (lo + 1.0 - u2));
  }
  return 0.5 * s;
}

// g0, g1, g2: Gamma(alpha), Gamma(alpha + 1), Gamma(alpha + 2), evaluated once
// on the host in extended precision and rounded to FP64 (the weights inherit
// their relative error).
__global__ void weights_kernel(double alpha, int M, double* __restrict__ b, double* __restrict__ a,
                               double* __restrict__ c, double* __restrict__ g_out, double g0, double g1, double g2) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m > M) return;
  const double p = alpha + 1.0;
  if (m == 0) {
    if (g_out) *g_out = 1.0 / g2;  // weight of the j = n+1 term of the corrector
    b[0] = 1.0 / g1;
    a[0] = 2.0 * expm1(alpha * 0.69314718055994530942) / g2;
    c[0] = alpha / g2;
    return;
  }
  const double dm = (double)m;
  b[m] = pow(dm, alpha) * expm1(alpha * log1p(1.0 / dm)) / g1;
  if (m < kQuadBelow) {
    const double ga = g0;
    double rise = quad_rise(alpha, dm);
    a[m] = (rise + quad_fall(alpha, dm + 1.0)) / ga;
    c[m] = rise / ga;
    return;
  }
  // a_m: (m+1)^p * 2 * sum_j C(p,2j) z^(2j), terms falling like z^2.
  {
    const double z = 1.0 / (dm + 1.0), z2 = z * z;
    double coef = p * (p - 1.0) * 0.5;  // C(p, 2)
    double zp = z2, sum = coef * zp;
    for (int k = 2; k < 64; k += 2) {
      coef *= (p - k) * (p - k - 1.0) / ((k + 1.0) * (k + 2.0));  // C(p, k+2)
      zp *= z2;
      double term = coef * zp;
      sum += term;
      if (fabs(term) <= 1e-18 * fabs(sum)) break;
    }
    a[m] = pow(dm + 1.0, p) * 2.0 * sum / g2;
  }
  // c_m: m^p * sum_{k>=2} C(a,k-1)(k-1)(a+1)/k x^k, alternating, |x| <= 1/16.
  {
    const double x = 1.0 / dm;
    double cm1 = alpha;  // C(alpha, k-1) at k = 2
    double xk = x * x, sum = 0.0;
    for (int k = 2; k < 64; ++k) {
      double term = cm1 * (k - 1.0) * p / k * xk;
      sum += term;
      if (fabs(term) <= 1e-18 * fabs(sum)) break;
      cm1 *= (alpha - (k - 1.0)) / k;  // C(alpha, k)
      xk *= x;
    }
    c[m] = pow(dm, p) * sum / g2;
  }
}

// Shadow copies for the reduced-precision far history.
__global__ void weights_to_f32_kernel(int M, const double* __restrict__ b, const double* __restrict__ a,
                                      float* __restrict__ b32, float* __restrict__ a32) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m > M) return;
  b32[m] = (float)b[m];
  a32[m] = (float)a[m];
}

cudaError_t launch_weights(double alpha, int M, double* b, double* a, double* c, double* g,
                           cudaStream_t st) {
  int threads = 256, blocks = (M + 1 + threads - 1) / threads;
  const long double al = alpha;
  const double g0 = (double)std::tgamma(al), g1 = (double)std::tgamma(al + 1.0L),
               g2 = (double)std::tgamma(al + 2.0L);
  weights_kernel<<<blocks, threads, 0, st>>>(alpha, M, b, a, c, g, g0, g1, g2);
  return cudaGetLastError();
}

cudaError_t launch_weights_f32(int M, const double* b, const double* a, float* b32, float* a32,
                               cudaStream_t st) {
  int threads = 256, blocks = (M + 1 + threads - 1) / threads;
  weights_to_f32_kernel<<<blocks, threads, 0, st>>>(M, b, a, b32, a32);
  return cudaGetLastError();
}

}  // namespace abm
