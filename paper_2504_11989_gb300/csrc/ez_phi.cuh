// Device library for Phi_a(t) = t^{-a} Gamma(a, t) = int_1^inf s^{a-1} e^{-t s} ds,
// a in Z/2: the upper incomplete gamma function of the splitting of Z (orders
// a = nu/2 in real space and a = (d - nu)/2 in reciprocal space).
//
// Two paths:
//  * phi_accurate(a, t): used only while building tables.  Closed form for
//    integer a >= 1; for a <= 0 and t > 1 the even part of Legendre's continued
//    fraction for Gamma(a, t) (DLMF 8.9.2) by the modified Lentz method; for
//    t <= 1 the E_1 power series (A&S 5.1.11) or sqrt(pi/t) erfc(sqrt t),
//    then the recurrence t Phi_{a+1} = a Phi_a + e^{-t}.
//  * phi_eval(PhiInfo, t): the hot path.  Piecewise polynomial on [kT0, t_hi],
//    entire-part series plus singular term below kT0, asymptotic series above.
#pragma once

#include <math_constants.h>

#include <cmath>

#include "ez_ff.cuh"
#include "ez_internal.h"

namespace ez {

__host__ __device__ inline double e1_series(double t) {
  // E_1(t) = -gamma - log t - sum_{k>=1} (-t)^k / (k k!)
  double sum = 0.0, term = 1.0;
  for (int k = 1; k < 60; ++k) {
    term *= -t / k;
    double add = term / k;
    sum += add;
    if (fabs(add) < 1e-19 * fabs(sum)) break;
  }
  return -0.57721566490153286060651209 - log(t) - sum;
}

__host__ __device__ inline double phi_cf(double a, double t) {
  // Phi_a(t) = e^{-t} / (t + 1 - a - 1(1-a)/(t + 3 - a - 2(2-a)/(t + 5 - a - ...)))
  const double tiny = 1e-300;
  double b = t + 1.0 - a;
  double c = 1.0 / tiny;
  double dd = 1.0 / b;
  double h = dd;
  for (int i = 1; i < 20000; ++i) {
    double an = -(double)i * ((double)i - a);
    b += 2.0;
    dd = fma(an, dd, b);
    if (fabs(dd) < tiny) dd = tiny;
    c = b + an / c;
    if (fabs(c) < tiny) c = tiny;
    dd = 1.0 / dd;
    double del = dd * c;
    h *= del;
    if (fabs(del - 1.0) < 2e-17) break;
  }
  return exp(-t) * h;
}

// t e^{t} Phi_a(t) for large t (t > a + 1): t times the Legendre continued fraction, so
// that nothing underflows (used to fit the binary32 tail of the mixed form).
__host__ __device__ inline double phi_scaled_large(double a, double t) {
  const double tiny = 1e-300;
  double b = t + 1.0 - a, c = 1.0 / tiny, dd = 1.0 / b, h = dd;
  for (int i = 1; i < 20000; ++i) {
    double an = -(double)i * ((double)i - a);
    b += 2.0;
    dd = fma(an, dd, b);
    if (fabs(dd) < tiny) dd = tiny;
    c = b + an / c;
    if (fabs(c) < tiny) c = tiny;
    dd = 1.0 / dd;
    double del = dd * c;
    h *= del;
    if (fabs(del - 1.0) < 2e-17) break;
  }
  return t * h;
}

// Legendre's continued fraction for Phi_a(t) evaluated backward from depth n (no forward
// accumulation of rounding; converges for t > 0, fast where t is not far below a).
__host__ __device__ inline double phi_cf_backward(double a, double t, int n) {
  double h = t + 2.0 * n + 1.0 - a;
  for (int i = n; i > 0; --i) h = (t + 2.0 * i - 1.0 - a) - (double)i * (i - a) / h;
  return exp(-t) / h;
}

// Real a that is not a multiple of 1/2 (non-integer exponents).  a > 1, t < a:
// Phi_a = Gamma(a) t^{-a} - e^{-t} sum_n t^n / (a (a+1) ... (a+n)), the lower incomplete gamma
// by its series of positive terms (Gamma(a, t) is a sizeable part of Gamma(a) there); else for
// t >= 1/2 the continued fraction evaluated backward, at depths 200, 400, ... until two agree;
// for t < 1/2, Gamma(a) t^{-a} minus the entire series sum_n (-t)^n / (n! (a + n)) (a is then
// not a pole of Gamma).
__host__ __device__ inline double phi_general(double a, double t) {
  if (a > 1.0 && t < a) {
    double s = 0.0, term = 1.0 / a;
    for (int n = 0; n < 400; ++n) {
      if (n > 0) term *= t / (a + n);
      s += term;
      if (term < 1e-18 * s) break;
    }
    return tgamma(a) * exp(-a * log(t)) - exp(-t) * s;
  }
  if (t >= 0.5) {
    double prev = phi_cf_backward(a, t, 200);
    for (int n = 400; n <= 6400; n *= 2) {
      const double cur = phi_cf_backward(a, t, n);
      if (fabs(cur - prev) <= 1e-17 * fabs(cur)) return cur;
      prev = cur;
    }
    return prev;
  }
  double s = 0.0, term = 1.0;  // (-t)^n / n!
  for (int n = 0; n < 80; ++n) {
    if (n > 0) term *= -t / n;
    const double add = term / (a + n);
    s += add;
    if (n > 4 && fabs(add) < 1e-18 * fabs(s)) break;
  }
  return tgamma(a) * exp(-a * log(t)) - s;
}

__host__ __device__ inline double phi_accurate(double a, double t) {
  int two_a = (int)lrint(2.0 * a);
  if (!(t > 0.0)) return a < 0.0 ? -1.0 / a : (double)INFINITY;
  if (fabs(2.0 * a - two_a) > 1e-12) return phi_general(a, t);
  bool integer = (two_a & 1) == 0;
  if (integer && a >= 1.0) {
    int n = two_a / 2;
    double s = 0.0, term = 1.0, fact = 1.0;
    for (int k = 0; k < n; ++k) {
      s += term;
      term *= t / (k + 1);
    }
    for (int k = 2; k < n; ++k) fact *= k;  // (n-1)!
    double tp = 1.0;
    for (int k = 0; k < n; ++k) tp *= t;
    return fact * exp(-t) * s / tp;
  }
  if (a <= 0.0 && t > 1.0) return phi_cf(a, t);
  double et = exp(-t);
  if (integer) {  // a <= 0, t <= 1: from Phi_0 = E_1 downward
    double p = e1_series(t);
    for (int c = 0; c > two_a / 2; --c) p = (t * p - et) / (double)(c - 1);
    return p;
  }
  double p = sqrt(kPi / t) * erfc(sqrt(t));  // Phi_{1/2}
  double cur = 0.5;
  while (cur < a - 0.25) {
    p = (cur * p + et) / t;
    cur += 1.0;
  }
  while (cur > a + 0.25) {
    p = (t * p - et) / (cur - 1.0);
    cur -= 1.0;
  }
  return p;
}

// t^{-two_a/2} for t > 0 using sqrt and integer powers only.
__device__ __forceinline__ double pow_half(double t, int two_a) {
  int e = -two_a;  // power of sqrt(t)
  double base = (e & 1) ? sqrt(t) : 1.0;
  int k = e >> 1;  // floor(e/2)
  double r = base;
  double tt = t;
  if (k < 0) {
    tt = 1.0 / t;
    k = -k;
  }
  while (k) {
    if (k & 1) r *= tt;
    tt *= tt;
    k >>= 1;
  }
  return r;
}

// Interval index of t in a table (t >= kT0), computed in binary32.
__device__ __forceinline__ int phi_interval(float tf, float t_geo_end_f) {
  int i;
  if (tf < t_geo_end_f) {
    // log_{1.4}(t / kT0) = log2(2 t) / log2(1.4)
    i = (int)(__log2f(2.0f * tf) * 2.06008f);
    i = max(0, min(i, kNGeo - 1));
  } else {
    const float u = 2.0f * (tf - t_geo_end_f);  // half-width intervals, then unit width
    i = u < (float)kNHalf ? kNGeo + (int)u : kNGeo + kNHalf + (int)(0.5f * (u - (float)kNHalf));
  }
  return i;
}

// Horner over the kept coefficients in blocks of four (a real loop: the length
// varies by interval and must not be if-converted into always-issued predicated
// DFMAs).  Returns the value and the number of coefficients used.
__device__ __forceinline__ double phi_poly(const double* r, double x, int& n_used) {
  const int n = __ldg(reinterpret_cast<const int*>(r));
  n_used = n;
  if (n == 1) return __ldg(r + 4);  // constant on the interval (below the tolerance)
  const double2* c2 = reinterpret_cast<const double2*>(r + 4);
  int blk = (n >> 2) - 1;
  double2 hi = __ldg(c2 + 2 * blk + 1), lo = __ldg(c2 + 2 * blk);
  double p = fma(hi.y, x, hi.x);
  p = fma(p, x, lo.y);
  p = fma(p, x, lo.x);
#pragma unroll 1
  for (--blk; blk >= 0; --blk) {
    hi = __ldg(c2 + 2 * blk + 1);
    lo = __ldg(c2 + 2 * blk);
    p = fma(p, x, hi.y);
    p = fma(p, x, hi.x);
    p = fma(p, x, lo.y);
    p = fma(p, x, lo.x);
  }
  return p;
}

static __device__ __noinline__ double phi_small(const PhiInfo& P, double t) {
  const float tf = (float)t;
  int N = 4;
#pragma unroll
  for (int i = 0; i < 6; ++i) N += tf >= P.ser_brk[i] ? 2 : 0;
  double s = P.ser[N - 1];
#pragma unroll 1
  for (int k = N - 2; k >= 0; --k) s = fma(s, t, P.ser[k]);
  if (t == 0.0) return P.log_m >= 0 ? (P.log_m == 0 ? CUDART_INF : s) : (P.a < 0.0 ? s : CUDART_INF);
  if (P.log_m >= 0) {
    double tm = 1.0;
    for (int k = 0; k < P.log_m; ++k) tm *= t;
    return s - P.gam * tm * log(t);
  }
  return s + P.gam * (P.half ? pow_half(t, P.two_a) : exp(-P.a * log(t)));
}

// t < kT0, binary64, with log t (log-case and non-half-integer orders), 1/t and sqrt t
// supplied by the caller, who shares them between the orders of one reciprocal term: the
// entire series cut at the breakpoints brk plus the singular part.  n_used: series terms.
__device__ __forceinline__ double phi_small_shared(const PhiInfo& P, double t, double lt, double it, double st,
                                                   int& n_used, const float* brk) {
  const float tf = (float)t;
  int N = 4;
#pragma unroll
  for (int i = 0; i < 6; ++i) N += tf >= brk[i] ? 2 : 0;
  n_used = N;
  double s = P.ser[N - 1];
#pragma unroll 1
  for (int k = N - 2; k >= 0; --k) s = fma(s, t, P.ser[k]);
  if (P.log_m >= 0) {
    double tm = 1.0;
    for (int k = 0; k < P.log_m; ++k) tm *= t;
    return s - P.gam * tm * lt;
  }
  if (!P.half) return s + P.gam * exp(-P.a * lt);  // non-half-integer order (lt = log t)
  const int e = -P.two_a;  // t^{-a} = sqrt(t)^e
  double r = (e & 1) ? st : 1.0;
  const int k = e >> 1;  // floor(e / 2)
  const double b = k < 0 ? it : t;
  for (int q = 0; q < (k < 0 ? -k : k); ++q) r *= b;
  return s + P.gam * r;
}

static __device__ __noinline__ double phi_large(const PhiInfo& P, double t) {
  double inv = 1.0 / t;
  double s = 1.0, term = 1.0;
  for (int k = 1; k <= 8; ++k) {
    term *= (P.a - k) * inv;
    s += term;
  }
  return exp(-t) * inv * s;
}

// Phi_a(c |q|^2) from qq = |q|^2 (binary64) and tf ~ c |q|^2 (binary32, used only to
// pick the branch and the interval).  n_used: coefficients evaluated (work count).
__device__ __forceinline__ double phi_eval_qq(const PhiInfo& P, double qq, float tf, int& n_used) {
  if (tf < (float)kT0) {
    n_used = kNSer;
    return phi_small(P, P.c_lam * qq);
  }
  if (tf > P.t_hi_f) {
    n_used = kNC;
    return phi_large(P, P.c_lam * qq);
  }
  const int i = min(phi_interval(tf, P.t_geo_end_f), P.n_int - 1);
  const double* r = P.tab + (size_t)i * kRec;
  const double2 so = __ldg(reinterpret_cast<const double2*>(r) + 0);  // (n|pad, s) -- s in .y
  if (__double2loint(so.x) == 1) {  // constant record: no argument, no Horner scheme
    n_used = 0;
    return __ldg(r + 4);
  }
  const double o = __ldg(r + 2);
  return phi_poly(r, fma(qq, so.y, o), n_used);
}

// mixed form, tail (t >= t_mix): e^{-t} t^{-1} P(t_mix / t), no tables and no branches
__device__ __forceinline__ float phi_tail_poly(const PhiInfo& P, float sv) {
  float p = P.tail_p[7];
#pragma unroll
  for (int k = 6; k >= 0; --k) p = fmaf(p, sv, P.tail_p[k]);
  return p;
}

// mixed form, middle range: binary32 Horner scheme on the binary32 record r at x
__device__ __forceinline__ float phi_poly_f(const float* r, float xf) {
  const int n = __ldg(reinterpret_cast<const int*>(r));
  const float4* c4 = reinterpret_cast<const float4*>(r + 4);
  int blk = (n >> 2) - 1;
  float4 c = __ldg(c4 + blk);
  float p = fmaf(c.w, xf, c.z);
  p = fmaf(p, xf, c.y);
  p = fmaf(p, xf, c.x);
#pragma unroll 1
  for (--blk; blk >= 0; --blk) {
    c = __ldg(c4 + blk);
    p = fmaf(p, xf, c.w);
    p = fmaf(p, xf, c.z);
    p = fmaf(p, xf, c.y);
    p = fmaf(p, xf, c.x);
  }
  return p;
}

// mixed form, heads: Horner scheme in float-float on the float-float record r (coefficient
// pairs (hi, lo), two per 16-byte load); n_used: coefficients evaluated
// The coefficients j >= J (J even, from the record) are small enough for binary32 with x.hi;
// the scheme continues in float-float below J.
__device__ __forceinline__ ff phi_poly_ff(const float* r, ff x, int& n_used) {
  const int2 nj = __ldg(reinterpret_cast<const int2*>(r));  // (n, J)
  n_used = nj.x;
  const float4* c4 = reinterpret_cast<const float4*>(r + 8);
  int blk = (nj.x >> 1) - 1;
  const int blk_ff = (nj.y >> 1) - 1;
  float pf = 0.0f;
#pragma unroll 1
  for (; blk > blk_ff; --blk) {
    const float4 c = __ldg(c4 + blk);  // (b_{2 blk}, b_{2 blk + 1})
    pf = fmaf(fmaf(pf, x.hi, c.z), x.hi, c.x);
  }
  float4 c = __ldg(c4 + blk);
  ff p = ff_add(ff_mul(ff{pf, 0.0f}, x), ff{c.z, c.w});
  p = ff_add(ff_mul(p, x), ff{c.x, c.y});
#pragma unroll 1
  for (--blk; blk >= 0; --blk) {
    c = __ldg(c4 + blk);
    p = ff_add(ff_mul(p, x), ff{c.z, c.w});
    p = ff_add(ff_mul(p, x), ff{c.x, c.y});
  }
  return p;
}

__device__ __forceinline__ double phi_eval(const PhiInfo& P, double t) {
  int n;
  return phi_eval_qq(P, t / P.c_lam, (float)t, n);
}

__device__ __forceinline__ G4 ldg_g4(const G4* p) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p));
  const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  return G4{a.x, a.y, b.x, b.y};
}

}  // namespace ez
