// Complex arithmetic (FP64) for the 1-D MGE's Euler inversion (Sect. 3.2), which evaluates the
// radial profiles at complex radii: products, quotients, principal exp, log and powers, the
// Chameleon profile (Eq. Chameleon) and the projected NFW shape (Eq. kappa_enfw).
#pragma once
#include <math.h>

struct cplx {
  double r, i;
};
__device__ inline cplx cmul(cplx a, cplx b) { return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }
__device__ inline cplx cexp_(cplx a) {
  double s, c;
  sincos(a.i, &s, &c);
  const double e = exp(a.r);
  return {e * c, e * s};
}
__device__ inline cplx clog_(cplx a) { return {log(hypot(a.r, a.i)), atan2(a.i, a.r)}; }
__device__ inline cplx cdiv(cplx a, cplx b) {
  const double d = b.r * b.r + b.i * b.i;
  return {(a.r * b.r + a.i * b.i) / d, (a.i * b.r - a.r * b.i) / d};
}
__device__ inline cplx cpow_(cplx a, double e) {  // principal a^e
  const cplx l = clog_(a);
  return cexp_({e * l.r, e * l.i});
}

// Chameleon profile (Eq. Chameleon) at complex radius z: A [(z^2 + sc^2)^-1/2 - (z^2 + st^2)^-1/2]
__device__ inline cplx chameleon_c(cplx z, double A, double sc, double st) {
  const cplx z2 = cmul(z, z);
  const cplx a = cpow_({z2.r + sc * sc, z2.i}, -0.5), b = cpow_({z2.r + st * st, z2.i}, -0.5);
  return {A * (a.r - b.r), A * (a.i - b.i)};
}

// projected NFW shape k(u) at complex u (Re u > 0): with w^2 = 1 - u^2, k = 2 (1 - arctanh(w)/w)
// / (u^2 - 1), even in w, arctanh(w) = (ln(1 + w) - ln(1 - w))/2 (principal branches: no cut is
// crossed for Re u > 0); near u = 1 (|w| < 0.1) the series 2 sum_n w^(2n)/(2n + 3).  With
// duk = 1 also u dk/du: (-2 (1 - u^2 F)/w^2 + 2 u^2 k)/w^2, or -4 u^2 sum_n n w^(2n-2)/(2n + 3)
__device__ inline cplx nfw_k_c(cplx u, cplx *udk) {
  const cplx u2 = cmul(u, u);
  const cplx w2 = {1.0 - u2.r, -u2.i};
  cplx k;
  if (w2.r * w2.r + w2.i * w2.i < 1e-2 * 1e-2) {
    cplx sk = {0.0, 0.0}, sd = {0.0, 0.0}, p = {1.0, 0.0}, pm = {0.0, 0.0};
    for (int n = 0; n < 12; ++n) {
      sk.r += 2.0 * p.r / (2 * n + 3);
      sk.i += 2.0 * p.i / (2 * n + 3);
      if (n >= 1) {
        sd.r += n * pm.r / (2 * n + 3);
        sd.i += n * pm.i / (2 * n + 3);
      }
      pm = p;
      p = cmul(p, w2);
    }
    k = sk;
    if (udk) {
      const cplx t = cmul(u2, sd);
      *udk = {-4.0 * t.r, -4.0 * t.i};
    }
    return k;
  }
  const cplx w = cpow_(w2, 0.5);
  const cplx l1 = clog_({1.0 + w.r, w.i}), l2 = clog_({1.0 - w.r, -w.i});
  const cplx F = cdiv({0.5 * (l1.r - l2.r), 0.5 * (l1.i - l2.i)}, w);
  k = cdiv({2.0 * (1.0 - F.r), -2.0 * F.i}, {u2.r - 1.0, u2.i});
  if (udk) {
    const cplx u2F = cmul(u2, F), u2k = cmul(u2, k);
    const cplx a = cdiv({-2.0 * (1.0 - u2F.r), 2.0 * u2F.i}, w2);
    *udk = cdiv({a.r + 2.0 * u2k.r, a.i + 2.0 * u2k.i}, w2);
  }
  return k;
}

