// Forward-mode dual numbers (value + N tangents) for the gradient kernels: the chain
// from parameters to per-sub-pixel intensities (FP32) and to per-sample MGE, deprojection,
// table and delay quantities (FP64) is propagated exactly, term by term.
#pragma once
#include <math.h>

template <int N, class F>
struct Dual {
  F v;
  F d[N];
  __host__ __device__ Dual() {}
  __host__ __device__ Dual(F x) : v(x) {
#pragma unroll
    for (int i = 0; i < N; ++i) d[i] = F(0);
  }
  __host__ __device__ static Dual var(F x, int i) {
    Dual r(x);
    r.d[i] = F(1);
    return r;
  }
};

#define DUAL_T template <int N, class F>
#define DL Dual<N, F>

DUAL_T __host__ __device__ inline DL operator+(const DL &a, const DL &b) {
  DL r;
  r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
DUAL_T __host__ __device__ inline DL operator-(const DL &a, const DL &b) {
  DL r;
  r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
DUAL_T __host__ __device__ inline DL operator-(const DL &a) {
  DL r;
  r.v = -a.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
  return r;
}
DUAL_T __host__ __device__ inline DL operator*(const DL &a, const DL &b) {
  DL r;
  r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
DUAL_T __host__ __device__ inline DL operator/(const DL &a, const DL &b) {
  DL r;
  const F ib = F(1) / b.v;
  r.v = a.v * ib;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
  return r;
}
// mixed with plain scalars
DUAL_T __host__ __device__ inline DL operator+(const DL &a, F b) {
  DL r = a;
  r.v += b;
  return r;
}
DUAL_T __host__ __device__ inline DL operator+(F b, const DL &a) { return a + b; }
DUAL_T __host__ __device__ inline DL operator-(const DL &a, F b) {
  DL r = a;
  r.v -= b;
  return r;
}
DUAL_T __host__ __device__ inline DL operator-(F b, const DL &a) { return (-a) + b; }
DUAL_T __host__ __device__ inline DL operator*(const DL &a, F b) {
  DL r;
  r.v = a.v * b;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b;
  return r;
}
DUAL_T __host__ __device__ inline DL operator*(F b, const DL &a) { return a * b; }
DUAL_T __host__ __device__ inline DL operator/(const DL &a, F b) { return a * (F(1) / b); }
DUAL_T __host__ __device__ inline DL operator/(F a, const DL &b) {
  DL r;
  const F ib = F(1) / b.v;
  r.v = a * ib;
  const F s = -r.v * ib;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = s * b.d[i];
  return r;
}

// apply f with derivative fp at a.v
DUAL_T __host__ __device__ inline DL dual_apply(const DL &a, F f, F fp) {
  DL r;
  r.v = f;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = fp * a.d[i];
  return r;
}

// elementary functions: FP64 versions use the double overloads, FP32 the float ones
template <int N>
__device__ inline Dual<N, double> dsqrt(const Dual<N, double> &a) {
  const double s = sqrt(a.v);
  return dual_apply(a, s, 0.5 / s);
}
template <int N>
__device__ inline Dual<N, double> dexp(const Dual<N, double> &a) {
  const double e = exp(a.v);
  return dual_apply(a, e, e);
}
template <int N>
__device__ inline Dual<N, double> dlog(const Dual<N, double> &a) {
  return dual_apply(a, log(a.v), 1.0 / a.v);
}
template <int N>
__device__ inline Dual<N, double> dlog1p(const Dual<N, double> &a) {
  return dual_apply(a, log1p(a.v), 1.0 / (1.0 + a.v));
}
template <int N>
__device__ inline Dual<N, double> datan(const Dual<N, double> &a) {
  return dual_apply(a, atan(a.v), 1.0 / (1.0 + a.v * a.v));
}
template <int N>
__device__ inline Dual<N, double> datanh(const Dual<N, double> &a) {
  return dual_apply(a, atanh(a.v), 1.0 / (1.0 - a.v * a.v));
}
template <int N>
__device__ inline Dual<N, double> dpow(const Dual<N, double> &a, const Dual<N, double> &b) {
  return dexp(b * dlog(a));
}
template <int N>
__device__ inline Dual<N, double> dsin(const Dual<N, double> &a) {
  return dual_apply(a, sin(a.v), cos(a.v));
}
template <int N>
__device__ inline Dual<N, double> dcos(const Dual<N, double> &a) {
  return dual_apply(a, cos(a.v), -sin(a.v));
}
template <int N>
__device__ inline Dual<N, double> dfabs(const Dual<N, double> &a) {
  return a.v < 0 ? -a : a;
}
template <int N>
__device__ inline Dual<N, float> dsqrt(const Dual<N, float> &a) {
  const float s = sqrtf(a.v);
  return dual_apply(a, s, 0.5f / s);
}
template <int N>
__device__ inline Dual<N, float> datan(const Dual<N, float> &a) {
  return dual_apply(a, atanf(a.v), 1.0f / (1.0f + a.v * a.v));
}
template <int N>
__device__ inline Dual<N, float> datanh(const Dual<N, float> &a) {
  return dual_apply(a, atanhf(a.v), 1.0f / (1.0f - a.v * a.v));
}
template <int N>
__device__ inline Dual<N, float> dexp2(const Dual<N, float> &a) {
  const float e = exp2f(a.v);
  return dual_apply(a, e, e * 0.6931471805599453f);
}
template <int N>
__device__ inline Dual<N, float> dlog2(const Dual<N, float> &a) {
  return dual_apply(a, log2f(a.v), 1.4426950408889634f / a.v);
}

// plain-scalar versions so templated code works for T = double
__device__ inline double dsqrt(double a) { return sqrt(a); }
__device__ inline double dexp(double a) { return exp(a); }
__device__ inline double dlog(double a) { return log(a); }
__device__ inline double dlog1p(double a) { return log1p(a); }
__device__ inline double datan(double a) { return atan(a); }
__device__ inline double datanh(double a) { return atanh(a); }
__device__ inline double dpow(double a, double b) { return pow(a, b); }
__device__ inline double dsin(double a) { return sin(a); }
__device__ inline double dcos(double a) { return cos(a); }
__device__ inline double dfabs(double a) { return fabs(a); }

template <class T>
__device__ inline double dval(const T &a) { return a.v; }
__device__ inline double dval(double a) { return a; }

#undef DUAL_T
#undef DL
