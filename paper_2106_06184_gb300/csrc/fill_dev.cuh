// Device helpers shared by the fill translation units: the 6-point rule,
// precision traits of the destination, FP64 closed-form potentials of a flat
// triangle, and the smooth remainders of G and grad G used on touching pairs.
#pragma once
#include <cmath>

#include "internal.h"

namespace sldm {

// ---------------------------------------------------------------- Dunavant rule
// Six-point degree-4 rule (Dunavant 1985): barycentric points and weights
// (weights sum to 1).
static __constant__ double c_bary[6][3] = {
    {0.108103018168070, 0.445948490915965, 0.445948490915965},
    {0.445948490915965, 0.108103018168070, 0.445948490915965},
    {0.445948490915965, 0.445948490915965, 0.108103018168070},
    {0.816847572980459, 0.091576213509771, 0.091576213509771},
    {0.091576213509771, 0.816847572980459, 0.091576213509771},
    {0.091576213509771, 0.091576213509771, 0.816847572980459}};
static __constant__ double c_w[6] = {0.223381589678011, 0.223381589678011, 0.223381589678011,
                              0.109951743655322, 0.109951743655322, 0.109951743655322};

constexpr double PI = 3.14159265358979323846;
constexpr double INV4PI = 0.25 / PI;

// ---------------------------------------------------------------- precision traits
template <class R>
struct M;
template <>
struct M<float> {
  // sin and cos of the FP32 phase k R: the argument is first reduced to
  // [-pi, pi] with 2 pi split into two floats (6.2831855 + (-1.7484555e-7), a
  // Cody-Waite reduction whose error stays below that of the FP32 argument
  // itself for |x| < 2^12), then the special-function unit evaluates sin and cos
  // (absolute error ~4e-7 on that interval).  Two SFU operations and five FMA-pipe
  // operations, against a long branchy sequence for sincosf: the bulk fill
  // inlines 36 of these per triangle pair.
  static __device__ __forceinline__ void sincos_(float x, float* s, float* c) {
    const float n = rintf(x * 0.15915494309189535f);
    const float r = __fmaf_rn(-n, -1.7484555e-7f, __fmaf_rn(-n, 6.2831855f, x));
    *s = __sinf(r);
    *c = __cosf(r);
  }
  static __device__ __forceinline__ float exp_(float x) { return __expf(x); }
  static __device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
  static __device__ __forceinline__ void add(void* base, int64_t idx, float re, float im) {
    atomicAdd(reinterpret_cast<float2*>(base) + idx, make_float2(re, im));
  }
  static __device__ __forceinline__ void store(void* base, int64_t idx, double re, double im) {
    reinterpret_cast<float2*>(base)[idx] = make_float2(float(re), float(im));
  }
  static __device__ __forceinline__ void store_r(void* base, int64_t idx, float re, float im) {
    reinterpret_cast<float2*>(base)[idx] = make_float2(re, im);
  }
};
template <>
struct M<double> {
  static __device__ __forceinline__ void sincos_(double x, double* s, double* c) { sincos(x, s, c); }
  static __device__ __forceinline__ double exp_(double x) { return exp(x); }
  static __device__ __forceinline__ double rsqrt_(double x) { return rsqrt(x); }
  static __device__ __forceinline__ void add(void* base, int64_t idx, double re, double im) {
    double* p = reinterpret_cast<double*>(base) + 2 * idx;
    atomicAdd(p, re);
    atomicAdd(p + 1, im);
  }
  static __device__ __forceinline__ void store(void* base, int64_t idx, double re, double im) {
    reinterpret_cast<double2*>(base)[idx] = make_double2(re, im);
  }
  static __device__ __forceinline__ void store_r(void* base, int64_t idx, double re, double im) { store(base, idx, re, im); }
};
// atomic add of a double result into a destination of precision R
template <class R>
__device__ __forceinline__ void add_d(void* base, int64_t idx, double re, double im) {
  M<R>::add(base, idx, R(re), R(im));
}

// ---------------------------------------------------------------- FP64 closed forms
// Integrals over the flat triangle (p1, p2, p3) seen from r: each surface
// integral is reduced to a sum over the three edges with the surface divergence
// theorem in the plane of the triangle (Wilton, Rao, Glisson, Schaubert, Al-Bundak
// and Butler, IEEE Trans. AP-32, 1984; Graglia, IEEE Trans. AP-41, 1993).
struct Pot {
  double inv_r, r;            // int 1/R, int R
  double por[3], pr[3];       // int (rho' - rho)/R, int (rho' - rho) R
  double grad[3];             // int grad_r (1/R)
  double rho[3];              // projection of r on the plane
};

static __device__ void potentials(const double* r, const double* p1, const double* p2, const double* p3, Pot& o) {
  double u[3], w[3], n[3];
  for (int d = 0; d < 3; ++d) {
    u[d] = p2[d] - p1[d];
    w[d] = p3[d] - p1[d];
  }
  n[0] = u[1] * w[2] - u[2] * w[1];
  n[1] = u[2] * w[0] - u[0] * w[2];
  n[2] = u[0] * w[1] - u[1] * w[0];
  double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  for (int d = 0; d < 3; ++d) n[d] /= nn;
  double h = n[0] * (r[0] - p1[0]) + n[1] * (r[1] - p1[1]) + n[2] * (r[2] - p1[2]);
  for (int d = 0; d < 3; ++d) o.rho[d] = r[d] - h * n[d];
  double ah = fabs(h);
  double sum_tf = 0, omega = 0, sum_r = 0;
  double por[3] = {0, 0, 0}, pr[3] = {0, 0, 0}, gm[3] = {0, 0, 0};
  const double* P[4] = {p1, p2, p3, p1};
  for (int e = 0; e < 3; ++e) {
    const double* a = P[e];
    const double* b = P[e + 1];
    double s[3], m[3];
    double L = sqrt((b[0] - a[0]) * (b[0] - a[0]) + (b[1] - a[1]) * (b[1] - a[1]) + (b[2] - a[2]) * (b[2] - a[2]));
    for (int d = 0; d < 3; ++d) s[d] = (b[d] - a[d]) / L;
    m[0] = s[1] * n[2] - s[2] * n[1];
    m[1] = s[2] * n[0] - s[0] * n[2];
    m[2] = s[0] * n[1] - s[1] * n[0];
    double sm = 0, sp = 0, t0 = 0;
    for (int d = 0; d < 3; ++d) {
      sm += (a[d] - o.rho[d]) * s[d];
      sp += (b[d] - o.rho[d]) * s[d];
      t0 += (a[d] - o.rho[d]) * m[d];
    }
    double R02 = t0 * t0 + h * h;
    double Rm = sqrt(sm * sm + R02), Rp = sqrt(sp * sp + R02);
    double f;
    if (sp <= 0 && sm <= 0) {
      f = log((Rm - sm) / (Rp - sp));
    } else {
      double num = sp > 0 ? Rp + sp : R02 / (Rp - sp);
      double den = sm > 0 ? Rm + sm : R02 / (Rm - sm);
      f = log(num / den);
    }
    double q1 = R02 + ah * Rp, q2 = R02 + ah * Rm;
    double beta = (q1 > 0 ? atan(t0 * sp / q1) : 0.0) - (q2 > 0 ? atan(t0 * sm / q2) : 0.0);
    omega += beta;
    sum_tf += t0 * f;
    double line1 = sp * Rp - sm * Rm + R02 * f;  // 2 int_edge R dl
    sum_r += t0 * line1;
    double line3 = (sp * Rp * Rp * Rp - sm * Rm * Rm * Rm) / 4.0 + 3.0 * R02 * (sp * Rp - sm * Rm) / 8.0 +
                   3.0 * R02 * R02 * f / 8.0;   // int_edge R^3 dl
    for (int d = 0; d < 3; ++d) {
      por[d] += m[d] * 0.5 * line1;
      pr[d] += m[d] * line3 / 3.0;
      gm[d] -= m[d] * f;
    }
  }
  o.inv_r = sum_tf - ah * omega;
  o.r = sum_r / 6.0 + h * h / 3.0 * o.inv_r;
  double sg = h > 0 ? 1.0 : (h < 0 ? -1.0 : 0.0);
  for (int d = 0; d < 3; ++d) {
    o.por[d] = por[d];
    o.pr[d] = pr[d];
    o.grad[d] = gm[d] - sg * omega * n[d];
  }
}

// complex helpers (double)
struct cd {
  double r, i;
};
__device__ __forceinline__ cd cmul(cd a, cd b) { return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }

// G - 1/(4 pi R) + k^2 R/(8 pi) (Taylor series for |kR| < 0.05)
static __device__ cd green_smooth(cd k, double R) {
  cd x = {k.r * R, k.i * R};
  double ax = sqrt(x.r * x.r + x.i * x.i);
  if (ax < 0.05) {
    // sum_{n>=1, n!=2} (-j k)^n R^(n-1) / n!
    cd mjk = {k.i, -k.r};  // -j k
    cd p = mjk;            // (-jk)^1
    cd acc = p;            // n = 1 term (R^0)
    double Rp = 1.0, fact = 1.0;
    for (int n = 2; n <= 11; ++n) {
      p = cmul(p, mjk);
      Rp *= R;
      fact *= n;
      if (n == 2) continue;
      acc.r += p.r * Rp / fact;
      acc.i += p.i * Rp / fact;
    }
    return {acc.r * INV4PI, acc.i * INV4PI};
  }
  double sn, cn;
  sincos(x.r, &sn, &cn);
  double ex = exp(x.i);  // exp(-j k R) = exp(ki R) (cos - j sin)
  cd e = {ex * cn - 1.0, -ex * sn};
  cd k2 = cmul(k, k);
  return {e.r * INV4PI / R + k2.r * R * 0.5 * INV4PI, e.i * INV4PI / R + k2.i * R * 0.5 * INV4PI};
}

// g1 of grad(G - 1/(4 pi R)) = (r - r') g1: (1 - (1 + jkR) exp(-jkR)) / (4 pi R^3)
static __device__ cd grad_smooth(cd k, double R) {
  cd x = {-k.i * R, k.r * R};  // j k R
  double ax = sqrt(x.r * x.r + x.i * x.i);
  double iR3 = INV4PI / (R * R * R);
  if (ax < 0.05) {
    // sum_{n>=2} (-1)^n (n-1) x^n / n!
    cd p = x, acc = {0, 0};
    double fact = 1.0;
    for (int n = 2; n <= 13; ++n) {
      p = cmul(p, x);
      fact *= n;
      double c = ((n & 1) ? -1.0 : 1.0) * (n - 1) / fact;
      acc.r += c * p.r;
      acc.i += c * p.i;
    }
    return {acc.r * iR3, acc.i * iR3};
  }
  double sn, cn;
  sincos(k.r * R, &sn, &cn);
  double ex = exp(k.i * R);
  cd e = {ex * cn, -ex * sn};              // exp(-jkR)
  cd one_x = {1.0 + x.r, x.i};             // 1 + jkR
  cd pr = cmul(one_x, e);
  return {(1.0 - pr.r) * iR3, -pr.i * iR3};
}

// sum over the 8 lanes of a group
__device__ __forceinline__ double grp_sum8(double v) {
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  return v;
}

}  // namespace sldm
