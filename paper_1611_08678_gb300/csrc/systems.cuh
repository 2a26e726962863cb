// Device-side catalogue of right-hand sides f(t, y) (eq. (1)) with their
// Jacobians J = df/dy and parameter derivatives Q = df/dp, used by the PECE
// kernels and the adjoint.  Parameter layouts are declared in include/abm.h.
#pragma once
#include "common.cuh"

namespace abm {

template <int SYS>
struct Sys;

template <>
struct Sys<ABM_SYS_LINEAR> {
  static constexpr int D = 1, NP = 3;
  // component c of f (the same arithmetic as f, one component)
  __device__ __forceinline__ static double fc(int, const double* p, double, double t, const double* y) {
    return fma(p[0], y[0], fma(p[2], t, p[1]));
  }
  __device__ __forceinline__ static void f(const double* p, double, double t, const double* y,
                                           double* out) {
    out[0] = fma(p[0], y[0], fma(p[2], t, p[1]));
  }
  __device__ __forceinline__ static void jac(const double* p, double, double t, const double* y,
                                             double* J, double* Q) {
    J[0] = p[0];
    Q[0] = y[0]; Q[1] = 1.0; Q[2] = t;
  }
};

template <>
struct Sys<ABM_SYS_MANUFACTURED> {
  static constexpr int D = 1, NP = 9;
  // component c of f (the same arithmetic as f, one component)
  __device__ __forceinline__ static double fc(int, const double* p, double alpha, double t, const double* y) {
    double o;
    f(p, alpha, t, y, &o);
    return o;
  }
  __device__ __forceinline__ static double curve(const double* p, double alpha, double t, double& ta) {
    ta = (t > 0.0) ? pow(t, alpha) : 0.0;
    return p[5] + ta * (p[6] + t * (p[7] + t * p[8]));
  }
  __device__ __forceinline__ static void f(const double* p, double alpha, double t, const double* y,
                                           double* out) {
    double ta;
    double r = y[0] - curve(p, alpha, t, ta);
    out[0] = p[0] + t * (p[1] + t * p[2]) + r * (p[3] + p[4] * r * r);
  }
  __device__ __forceinline__ static void jac(const double* p, double alpha, double t, const double* y,
                                             double* J, double* Q) {
    double ta;
    double r = y[0] - curve(p, alpha, t, ta);
    double dfdr = p[3] + 3.0 * p[4] * r * r;
    J[0] = dfdr;
    Q[0] = 1.0; Q[1] = t; Q[2] = t * t; Q[3] = r; Q[4] = r * r * r;
    Q[5] = -dfdr; Q[6] = -dfdr * ta; Q[7] = -dfdr * ta * t; Q[8] = -dfdr * ta * t * t;
  }
};

template <>
struct Sys<ABM_SYS_LORENZ> {
  static constexpr int D = 3, NP = 3;
  // component c of f (the same arithmetic as f, one component)
  __device__ __forceinline__ static double fc(int c, const double* p, double, double, const double* y) {
    if (c == 0) return p[0] * (y[1] - y[0]);
    if (c == 1) return fma(y[0], p[1] - y[2], -y[1]);
    return fma(y[0], y[1], -p[2] * y[2]);
  }
  __device__ __forceinline__ static void f(const double* p, double, double, const double* y,
                                           double* out) {
    out[0] = p[0] * (y[1] - y[0]);
    out[1] = fma(y[0], p[1] - y[2], -y[1]);
    out[2] = fma(y[0], y[1], -p[2] * y[2]);
  }
  __device__ __forceinline__ static void jac(const double* p, double, double, const double* y,
                                             double* J, double* Q) {
    J[0] = -p[0];        J[1] = p[0];  J[2] = 0.0;
    J[3] = p[1] - y[2];  J[4] = -1.0;  J[5] = -y[0];
    J[6] = y[1];         J[7] = y[0];  J[8] = -p[2];
    Q[0] = y[1] - y[0];  Q[1] = 0.0;   Q[2] = 0.0;
    Q[3] = 0.0;          Q[4] = y[0];  Q[5] = 0.0;
    Q[6] = 0.0;          Q[7] = 0.0;   Q[8] = -y[2];
  }
};

template <>
struct Sys<ABM_SYS_CHEN> {
  static constexpr int D = 3, NP = 3;
  // component c of f (the same arithmetic as f, one component)
  __device__ __forceinline__ static double fc(int c, const double* p, double, double, const double* y) {
    if (c == 0) return p[0] * (y[1] - y[0]);
    if (c == 1) return fma(p[2] - p[0], y[0], fma(-y[0], y[2], p[2] * y[1]));
    return fma(y[0], y[1], -p[1] * y[2]);
  }
  __device__ __forceinline__ static void f(const double* p, double, double, const double* y,
                                           double* out) {
    out[0] = p[0] * (y[1] - y[0]);
    out[1] = fma(p[2] - p[0], y[0], fma(-y[0], y[2], p[2] * y[1]));
    out[2] = fma(y[0], y[1], -p[1] * y[2]);
  }
  __device__ __forceinline__ static void jac(const double* p, double, double, const double* y,
                                             double* J, double* Q) {
    J[0] = -p[0];               J[1] = p[0];  J[2] = 0.0;
    J[3] = p[2] - p[0] - y[2];  J[4] = p[2];  J[5] = -y[0];
    J[6] = y[1];                J[7] = y[0];  J[8] = -p[1];
    Q[0] = y[1] - y[0];  Q[1] = 0.0;    Q[2] = 0.0;
    Q[3] = -y[0];        Q[4] = 0.0;    Q[5] = y[0] + y[1];
    Q[6] = 0.0;          Q[7] = -y[2];  Q[8] = 0.0;
  }
};

template <>
struct Sys<ABM_SYS_ROSSLER> {
  static constexpr int D = 3, NP = 3;
  // component c of f (the same arithmetic as f, one component)
  __device__ __forceinline__ static double fc(int c, const double* p, double, double, const double* y) {
    if (c == 0) return -y[1] - y[2];
    if (c == 1) return fma(p[0], y[1], y[0]);
    return fma(y[2], y[0] - p[2], p[1]);
  }
  __device__ __forceinline__ static void f(const double* p, double, double, const double* y,
                                           double* out) {
    out[0] = -y[1] - y[2];
    out[1] = fma(p[0], y[1], y[0]);
    out[2] = fma(y[2], y[0] - p[2], p[1]);
  }
  __device__ __forceinline__ static void jac(const double* p, double, double, const double* y,
                                             double* J, double* Q) {
    J[0] = 0.0;   J[1] = -1.0;  J[2] = -1.0;
    J[3] = 1.0;   J[4] = p[0];  J[5] = 0.0;
    J[6] = y[2];  J[7] = 0.0;   J[8] = y[0] - p[2];
    Q[0] = 0.0;   Q[1] = 0.0;   Q[2] = 0.0;
    Q[3] = y[1];  Q[4] = 0.0;   Q[5] = 0.0;
    Q[6] = 0.0;   Q[7] = 1.0;   Q[8] = -y[2];
  }
};

template <>
struct Sys<ABM_SYS_FINANCIAL> {
  static constexpr int D = 3, NP = 3;
  // component c of f (the same arithmetic as f, one component)
  __device__ __forceinline__ static double fc(int c, const double* p, double, double, const double* y) {
    if (c == 0) return fma(y[1] - p[0], y[0], y[2]);
    if (c == 1) return fma(-y[0], y[0], fma(-p[1], y[1], 1.0));
    return fma(-p[2], y[2], -y[0]);
  }
  __device__ __forceinline__ static void f(const double* p, double, double, const double* y,
                                           double* out) {
    out[0] = fma(y[1] - p[0], y[0], y[2]);
    out[1] = fma(-y[0], y[0], fma(-p[1], y[1], 1.0));
    out[2] = fma(-p[2], y[2], -y[0]);
  }
  __device__ __forceinline__ static void jac(const double* p, double, double, const double* y,
                                             double* J, double* Q) {
    J[0] = y[1] - p[0];  J[1] = y[0];   J[2] = 1.0;
    J[3] = -2.0 * y[0];  J[4] = -p[1];  J[5] = 0.0;
    J[6] = -1.0;         J[7] = 0.0;    J[8] = -p[2];
    Q[0] = -y[0];  Q[1] = 0.0;    Q[2] = 0.0;
    Q[3] = 0.0;    Q[4] = -y[1];  Q[5] = 0.0;
    Q[6] = 0.0;    Q[7] = 0.0;    Q[8] = -y[2];
  }
};

// The 3-D Hindmarsh-Rose neuron model (the system the paper simulates in
// Sec. 4, CUDA simulations), parameters (a, b, c, d, r, s, xR, I).
template <>
struct Sys<ABM_SYS_HINDMARSH_ROSE> {
  static constexpr int D = 3, NP = 8;
  // component c of f (the same arithmetic as f, one component)
  __device__ __forceinline__ static double fc(int c, const double* p, double, double, const double* y) {
    if (c == 0) return fma(fma(-p[0], y[0], p[1]), y[0] * y[0], y[1] - y[2] + p[7]);
    if (c == 1) return fma(-p[3], y[0] * y[0], p[2] - y[1]);
    return p[4] * fma(p[5], y[0] - p[6], -y[2]);
  }
  __device__ __forceinline__ static void f(const double* p, double, double, const double* y,
                                           double* out) {
    out[0] = fma(fma(-p[0], y[0], p[1]), y[0] * y[0], y[1] - y[2] + p[7]);
    out[1] = fma(-p[3], y[0] * y[0], p[2] - y[1]);
    out[2] = p[4] * fma(p[5], y[0] - p[6], -y[2]);
  }
  __device__ __forceinline__ static void jac(const double* p, double, double, const double* y,
                                             double* J, double* Q) {
    const double x = y[0];
    J[0] = x * fma(-3.0 * p[0], x, 2.0 * p[1]);  J[1] = 1.0;   J[2] = -1.0;
    J[3] = -2.0 * p[3] * x;                     J[4] = -1.0;  J[5] = 0.0;
    J[6] = p[4] * p[5];                         J[7] = 0.0;   J[8] = -p[4];
#pragma unroll
    for (int k = 0; k < 3 * NP; ++k) Q[k] = 0.0;
    Q[0] = -x * x * x;  Q[1] = x * x;  Q[7] = 1.0;      // row 0: a, b, I
    Q[NP + 2] = 1.0;    Q[NP + 3] = -x * x;             // row 1: c, d
    Q[2 * NP + 4] = fma(p[5], x - p[6], -y[2]);         // row 2: r, s, xR
    Q[2 * NP + 5] = p[4] * (x - p[6]);
    Q[2 * NP + 6] = -p[4] * p[5];
  }
};

// Runtime system id -> template instantiation.
#define ABM_DISPATCH_SYSTEM(sys, BODY)                                   \
  switch (sys) {                                                         \
    case ABM_SYS_LINEAR: { constexpr int SYS = ABM_SYS_LINEAR; BODY; } break;             \
    case ABM_SYS_MANUFACTURED: { constexpr int SYS = ABM_SYS_MANUFACTURED; BODY; } break; \
    case ABM_SYS_LORENZ: { constexpr int SYS = ABM_SYS_LORENZ; BODY; } break;             \
    case ABM_SYS_CHEN: { constexpr int SYS = ABM_SYS_CHEN; BODY; } break;                 \
    case ABM_SYS_ROSSLER: { constexpr int SYS = ABM_SYS_ROSSLER; BODY; } break;           \
    case ABM_SYS_FINANCIAL: { constexpr int SYS = ABM_SYS_FINANCIAL; BODY; } break;       \
    case ABM_SYS_HINDMARSH_ROSE: { constexpr int SYS = ABM_SYS_HINDMARSH_ROSE; BODY; } break; \
    default: break;                                                      \
  }

}  // namespace abm
