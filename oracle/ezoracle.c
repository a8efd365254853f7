/*
 * ezoracle.c -- plain, slow FP64 CPU oracle for the Epstein zeta method
 * ("Epstein zeta method for many-body lattice sums", Buchheit & Busse).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py; never by the product path.  It
 * shares no code with the CUDA library.  Every function follows the paper's
 * definitions in their order, with no blocking or fusion:
 *
 *   Def. "Epstein zeta function"      Z_{Lambda,nu}(x,k) = sum'_z e^{-2 pi i z.k} |z-x|^{-nu}
 *   (cited, not printed) incomplete-gamma splitting of Z.  Written out here from
 *       the Mellin integral |z|^{-nu} = pi^{nu/2}/Gamma(nu/2) int t^{nu/2-1} e^{-pi t |z|^2} dt
 *       split at t = 1/lam^2 with Poisson summation on the lower part:
 *       Z = P_nu [ sum_{z != x} Phi_{nu/2}(pi|z-x|^2/lam^2) e^{-2 pi i y.z}
 *                + lam^d/V sum_{g in Lambda*} Phi_{(d-nu)/2}(pi lam^2 |g+y|^2) e^{-2 pi i x.(g+y)}
 *                - [x in Lambda] (2/nu) e^{-2 pi i x.y} ],   P_nu = pi^{nu/2}/(Gamma(nu/2) lam^nu),
 *       Phi_a(t) = t^{-a} Gamma(a,t).
 *   Sec. 3, singular split  Z = Z^reg + s_hat_nu / |det A| (power or log form).
 *   Thm "Epstein representation" + Cor. "Duffy transformation": sectors (j, p),
 *       k~ = u sigma^j(p v, 1), k = A^{-T} k~, weight 2 u^{d-1} w_u prod w_v.
 *   Sec. 3, meromorphic continuation: eps-split, Taylor series of Z^reg of order
 *       2 ell, closed-form Hadamard integrals of u^{mu-1} log(pi u^2 w^2)^m.
 *   Prop. (ATM) recombination is done by the caller.
 *
 * Readings where the paper is silent (splitting parameter, cutoffs, fixed u rule,
 * truncation of the near-part product) are listed in the design notes; the parity
 * of this oracle with the paper is pinned by tests/test_oracle_*.py.
 */
#include "ezoracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.141592653589793238462643383279502884
#define OR_EULER_GAMMA 0.577215664901532860606512090082402431

/* ------------------------------------------------------------------------- */
/* Small dense linear algebra for d <= 3                                       */
/* ------------------------------------------------------------------------- */
static double or_det(int d, const double* A) {
  if (d == 1) return A[0];
  if (d == 2) return A[0] * A[3] - A[1] * A[2];
  return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
         A[2] * (A[3] * A[7] - A[4] * A[6]);
}

/* inverse via the adjugate */
static int or_inverse(int d, const double* A, double* Ai) {
  double det = or_det(d, A);
  if (det == 0.0 || !isfinite(det)) return 1;
  if (d == 1) {
    Ai[0] = 1.0 / A[0];
  } else if (d == 2) {
    Ai[0] = A[3] / det;
    Ai[1] = -A[1] / det;
    Ai[2] = -A[2] / det;
    Ai[3] = A[0] / det;
  } else {
    Ai[0] = (A[4] * A[8] - A[5] * A[7]) / det;
    Ai[1] = (A[2] * A[7] - A[1] * A[8]) / det;
    Ai[2] = (A[1] * A[5] - A[2] * A[4]) / det;
    Ai[3] = (A[5] * A[6] - A[3] * A[8]) / det;
    Ai[4] = (A[0] * A[8] - A[2] * A[6]) / det;
    Ai[5] = (A[2] * A[3] - A[0] * A[5]) / det;
    Ai[6] = (A[3] * A[7] - A[4] * A[6]) / det;
    Ai[7] = (A[1] * A[6] - A[0] * A[7]) / det;
    Ai[8] = (A[0] * A[4] - A[1] * A[3]) / det;
  }
  return 0;
}

static void or_transpose(int d, const double* A, double* At) {
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) At[i * d + j] = A[j * d + i];
}

static void or_matvec(int d, const double* M, const double* x, double* y) {
  for (int i = 0; i < d; ++i) {
    double s = 0.0;
    for (int j = 0; j < d; ++j) s += M[i * d + j] * x[j];
    y[i] = s;
  }
}

static double or_dot(int d, const double* a, const double* b) {
  double s = 0.0;
  for (int i = 0; i < d; ++i) s += a[i] * b[i];
  return s;
}

/* compensated (Kahan-Babuska) accumulator */
typedef struct {
  double s, c;
} or_acc;
static void or_acc_add(or_acc* a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x))
    a->c += (a->s - t) + x;
  else
    a->c += (x - t) + a->s;
  a->s = t;
}
static double or_acc_get(const or_acc* a) { return a->s + a->c; }

/* ------------------------------------------------------------------------- */
/* Upper incomplete gamma: Phi_a(t) = t^{-a} Gamma(a,t) = int_1^inf s^{a-1} e^{-ts} ds */
/* ------------------------------------------------------------------------- */

/* Phi_a(t) is evaluated from its defining integral by quadrature and by nothing else
 * (no closed form, continued fraction, series or recurrence in the order a), so that it
 * is a method of its own, independent of any tabulation of Phi built elsewhere.
 *
 * t >= 1: with s = 1 + x, x = e^w,
 *     Phi_a(t) = e^{-t} int_R (1 + e^w)^{a-1} e^w e^{-t e^w} dw,
 *   an integrand analytic in the strip |Im w| < pi/2, decaying like e^w as w -> -inf
 *   and double exponentially as w -> +inf.  The substitution w = c + v - e^{-v} makes
 *   the left tail double exponential too, and the trapezoidal rule in v converges
 *   geometrically in 1/h (Takahasi & Mori's double-exponential idea).  c puts the
 *   integrand's mode near v = 0.  The integrand is unimodal in w: once past its mode
 *   the terms decrease, and the sum stops when they are below 1e-19 of it. */
#define OR_DE_KLO (-30) /* v from -3.75 */
#define OR_DE_KHI 400
static double or_de_x[OR_DE_KHI - OR_DE_KLO + 1]; /* exp(v - e^{-v}) */
static double or_de_j[OR_DE_KHI - OR_DE_KLO + 1]; /* dw/dv = 1 + e^{-v} */

/* The nodes depend on v only: tabulated once when the library is loaded. */
__attribute__((constructor)) static void or_de_init(void) {
  for (int k = OR_DE_KLO; k <= OR_DE_KHI; ++k) {
    double v = k * 0.125, ev = exp(-v);
    or_de_x[k - OR_DE_KLO] = exp(v - ev);
    or_de_j[k - OR_DE_KLO] = 1.0 + ev;
  }
}

static double or_phi_t_ge1(double a, double t) {
  const double h = 0.125;
  double c = a > 0.0 ? log(fmax(a, 1.0) / t) : -log(t + 1.0 - a);
  double ec = exp(c);
  /* (1+x)^{a-1} = (1+x)^n [sqrt(1+x)] with n = floor(a-1) when a is a multiple of 1/2,
     else pow */
  int n = (int)floor(a - 1.0);
  int half = (a - 1.0) - n > 0.25;
  int na = n < 0 ? -n : n;
  int general = fabs(2.0 * a - round(2.0 * a)) > 1e-12;
  double sum = 0.0;
  for (int k = OR_DE_KLO; k <= OR_DE_KHI; ++k) {
    double x = ec * or_de_x[k - OR_DE_KLO];
    double tx = t * x;
    if (tx > 745.0) break;
    double b = 1.0 + x, bp = 1.0;
    if (general) {
      bp = pow(b, a - 1.0);
    } else {
      for (int i = 0; i < na; ++i) bp *= b;
      if (n < 0) bp = 1.0 / bp;
      if (half) bp *= sqrt(b);
    }
    double term = bp * x * exp(-tx) * or_de_j[k - OR_DE_KLO];
    sum += term;
    /* past the mode of (1+x)^{a-1} x e^{-tx} in log x: d/dlog x = (a-1)x/(1+x) + 1 - tx < 0 */
    if ((a - 1.0) * x / (1.0 + x) + 1.0 - tx < 0.0 && term < 1e-19 * sum) break;
  }
  return exp(-t) * h * sum;
}

/* t < 1: split the integral at s = 1/t and scale the upper piece, s = r/t:
 *     Phi_a(t) = int_1^{1/t} s^{a-1} e^{-ts} ds + t^{-a} Phi_a(1).
 * On the finite piece, with s = e^y (0 <= y <= L = log(1/t)), the integrand
 * e^{a y - t e^y} has t e^y <= 1, so it is smooth on [0, L]; composite Gauss-Legendre
 * with 16 nodes on panels of width 1/2 (the last one shorter).  Both pieces are
 * positive, so nothing cancels. */
static double or_gl16_x[16], or_gl16_w[16];
__attribute__((constructor)) static void or_gl16_init(void) { or_gauss_legendre01(16, or_gl16_x, or_gl16_w); }

static double or_phi_t_lt1(double a, double t) {
  const double* gx = or_gl16_x;
  const double* gw = or_gl16_w;
  double L = -log(t);
  double sum = 0.0;
  for (double y0 = 0.0; y0 < L; y0 += 0.5) {
    double wd = fmin(0.5, L - y0);
    double ps = 0.0;
    for (int i = 0; i < 16; ++i) {
      double y = y0 + wd * gx[i];
      ps += gw[i] * exp(a * y - t * exp(y));
    }
    sum += wd * ps;
    /* a < 0: the rest of [0, L] adds at most e^{a y} (L - y) */
    if (a < 0.0 && exp(a * (y0 + wd)) * L < 1e-19 * sum) break;
  }
  return sum + pow(t, -a) * or_phi_t_ge1(a, 1.0);
}

double or_phi(double a, double t) {
  if (t < 0.0 || isnan(t) || !isfinite(a)) return NAN;
  if (t == 0.0) return a < 0.0 ? -1.0 / a : INFINITY;
  return t >= 1.0 ? or_phi_t_ge1(a, t) : or_phi_t_lt1(a, t);
}

/* E_1(t) = Phi_0(t). */
double or_expint_e1(double t) {
  if (!(t > 0.0)) return t == 0.0 ? INFINITY : NAN;
  return or_phi(0.0, t);
}

/* is a a non-positive integer (log case of the regularisation)? returns m >= 0 or -1 */
static int or_log_order(double a) {
  double r = round(a);
  if (fabs(a - r) < 1e-12 && r <= 0.0) return (int)(-r);
  return -1;
}

/* Coefficients r_n (n = 0..nmax) of the entire function Phi^reg_a(t) = sum_n r_n t^n,
 * i.e. Phi_a(t) minus its singular part.  Non-log (a not in -N0):
 *   Phi_a(t) = Gamma(a) t^{-a} - sum_n (-1)^n t^n / (n! (a+n)).
 * Log case a = -m:
 *   Phi_{-m}(t) = ((-1)^m/m!) (psi(m+1) - log t) t^m - sum_{n != m} (-1)^n t^n/(n!(n-m));
 * the removed singular part is ((-1)^{m+1}/m!) t^m log(t/lam^2), matching s_hat of
 * Sec. 3 which uses log(pi |k|^2) = log(t/lam^2). */
static void or_phi_reg_series(double a, double lam, int nmax, double* r) {
  int m = or_log_order(a);
  double fact = 1.0;
  for (int n = 0; n <= nmax; ++n) {
    if (n > 0) fact *= (double)n;
    double sgn = (n % 2 == 0) ? 1.0 : -1.0;
    if (m >= 0 && n == m) {
      double psi = -OR_EULER_GAMMA;
      for (int k = 1; k <= m; ++k) psi += 1.0 / k;
      r[n] = sgn / fact * (psi - 2.0 * log(lam));
    } else {
      r[n] = -sgn / (fact * (a + (double)n));
    }
  }
}

/* ------------------------------------------------------------------------- */
/* Lattice points                                                              */
/* ------------------------------------------------------------------------- */
typedef struct {
  int n, cap;
  int* idx;   /* integer coordinates, d per point */
  double* p;  /* M * idx, d per point */
} or_points;

static void or_points_push(or_points* P, int d, const int* id, const double* x) {
  if (P->n == P->cap) {
    P->cap = P->cap ? 2 * P->cap : 256;
    P->idx = (int*)realloc(P->idx, sizeof(int) * 3 * P->cap);
    P->p = (double*)realloc(P->p, sizeof(double) * 3 * P->cap);
  }
  for (int i = 0; i < d; ++i) {
    P->idx[P->n * 3 + i] = id[i];
    P->p[P->n * 3 + i] = x[i];
  }
  P->n++;
}
static void or_points_free(or_points* P) {
  free(P->idx);
  free(P->p);
  memset(P, 0, sizeof(*P));
}

/* All integer h with |M h - c| <= R; Minv = M^{-1} bounds the box. */
static void or_enumerate(int d, const double* M, const double* Minv, const double* c, double R,
                         or_points* out) {
  double mc[3] = {0, 0, 0};
  or_matvec(d, Minv, c, mc);
  int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  for (int i = 0; i < d; ++i) {
    double rn = 0.0;
    for (int j = 0; j < d; ++j) rn += Minv[i * d + j] * Minv[i * d + j];
    double ext = R * sqrt(rn) + 1e-9;
    lo[i] = (int)floor(mc[i] - ext);
    hi[i] = (int)ceil(mc[i] + ext);
  }
  int id[3] = {0, 0, 0};
  for (id[0] = lo[0]; id[0] <= hi[0]; ++id[0])
    for (id[1] = (d > 1 ? lo[1] : 0); id[1] <= (d > 1 ? hi[1] : 0); ++id[1])
      for (id[2] = (d > 2 ? lo[2] : 0); id[2] <= (d > 2 ? hi[2] : 0); ++id[2]) {
        double fid[3] = {id[0], id[1], id[2]}, x[3];
        or_matvec(d, M, fid, x);
        double r2 = 0.0;
        for (int i = 0; i < d; ++i) r2 += (x[i] - c[i]) * (x[i] - c[i]);
        if (r2 <= R * R) or_points_push(out, d, id, x);
      }
}

static double or_prefactor(double nu, double lam) {
  /* P_nu = pi^{nu/2} / (Gamma(nu/2) lam^nu) */
  return pow(OR_PI, 0.5 * nu) / (tgamma(0.5 * nu) * pow(lam, nu));
}

static int or_gamma_pole(double x) { return x <= 0.0 && fabs(x - round(x)) < 1e-12; }

/* ------------------------------------------------------------------------- */
/* Epstein zeta, general (x, y)                                                */
/* ------------------------------------------------------------------------- */
int or_epstein_zeta(int d, const double* A, double nu, const double* x, const double* y,
                    double lam, double r_real, double r_recip, double* re, double* im) {
  if (d < 1 || d > 3) return 1;
  if (or_gamma_pole(0.5 * nu)) return 2;
  double Ai[9], AiT[9], At[9];
  if (or_inverse(d, A, Ai)) return 1;
  or_transpose(d, Ai, AiT);
  or_transpose(d, A, At);
  double V = fabs(or_det(d, A));
  double P = or_prefactor(nu, lam);
  double a_real = 0.5 * nu, a_rec = 0.5 * (d - nu);

  /* x in Lambda ? */
  double mx[3];
  or_matvec(d, Ai, x, mx);
  int x_in = 1, mxr[3] = {0, 0, 0};
  for (int i = 0; i < d; ++i) {
    mxr[i] = (int)lround(mx[i]);
    if (fabs(mx[i] - mxr[i]) > 1e-12) x_in = 0;
  }

  or_acc sre = {0, 0}, sim = {0, 0};
  /* real space: z in Lambda, 0 < |z - x| <= r_real */
  or_points pts = {0};
  or_enumerate(d, A, Ai, x, r_real, &pts);
  for (int e = 0; e < pts.n; ++e) {
    const int* m = pts.idx + 3 * e;
    const double* z = pts.p + 3 * e;
    if (x_in) {
      int same = 1;
      for (int i = 0; i < d; ++i) same &= (m[i] == mxr[i]);
      if (same) continue;
    }
    double r2 = 0.0;
    for (int i = 0; i < d; ++i) r2 += (z[i] - x[i]) * (z[i] - x[i]);
    double phi = or_phi(a_real, OR_PI * r2 / (lam * lam));
    double arg = 2.0 * OR_PI * or_dot(d, y, z);
    or_acc_add(&sre, phi * cos(arg));
    or_acc_add(&sim, -phi * sin(arg));
  }
  or_points_free(&pts);

  /* reciprocal space: g in Lambda*, |g + y| <= r_recip */
  or_acc rre = {0, 0}, rim = {0, 0};
  double my[3];
  for (int i = 0; i < d; ++i) my[i] = -y[i];
  or_enumerate(d, AiT, At, my, r_recip, &pts);
  for (int e = 0; e < pts.n; ++e) {
    const double* g = pts.p + 3 * e;
    double q[3], q2 = 0.0;
    for (int i = 0; i < d; ++i) {
      q[i] = g[i] + y[i];
      q2 += q[i] * q[i];
    }
    double phi;
    if (q2 == 0.0) {
      if (a_rec >= 0.0) {
        or_points_free(&pts);
        return 2;
      }
      phi = -1.0 / a_rec;
    } else {
      phi = or_phi(a_rec, OR_PI * lam * lam * q2);
    }
    double arg = 2.0 * OR_PI * or_dot(d, x, q);
    or_acc_add(&rre, phi * cos(arg));
    or_acc_add(&rim, -phi * sin(arg));
  }
  or_points_free(&pts);

  double c = pow(lam, (double)d) / V;
  double tre = or_acc_get(&sre) + c * or_acc_get(&rre);
  double tim = or_acc_get(&sim) + c * or_acc_get(&rim);
  if (x_in) {
    double arg = 2.0 * OR_PI * or_dot(d, x, y);
    tre -= (2.0 / nu) * cos(arg);
    tim += (2.0 / nu) * sin(arg);
  }
  *re = P * tre;
  *im = P * tim;
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Epstein zeta in any dimension d <= OR_MAXD (Sec. 6: the method for any d)    */
/* ------------------------------------------------------------------------- */
/* determinant and inverse by Gauss-Jordan elimination with partial pivoting */
static int or_inverse_nd(int d, const double* A, double* Ai, double* det) {
  double M[OR_MAXD * 2 * OR_MAXD];
  int w = 2 * d;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < w; ++j) M[i * w + j] = j < d ? A[i * d + j] : (j - d == i ? 1.0 : 0.0);
  double dt = 1.0;
  for (int c = 0; c < d; ++c) {
    int piv = c;
    for (int r = c + 1; r < d; ++r)
      if (fabs(M[r * w + c]) > fabs(M[piv * w + c])) piv = r;
    if (M[piv * w + c] == 0.0) return 1;
    if (piv != c) {
      for (int j = 0; j < w; ++j) {
        double t = M[c * w + j];
        M[c * w + j] = M[piv * w + j];
        M[piv * w + j] = t;
      }
      dt = -dt;
    }
    double pv = M[c * w + c];
    dt *= pv;
    for (int j = 0; j < w; ++j) M[c * w + j] /= pv;
    for (int r = 0; r < d; ++r) {
      if (r == c) continue;
      double f = M[r * w + c];
      if (f != 0.0)
        for (int j = 0; j < w; ++j) M[r * w + j] -= f * M[c * w + j];
    }
  }
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) Ai[i * d + j] = M[i * w + d + j];
  *det = dt;
  return 0;
}

/* calls f(ctx, z, id) for every integer id with |M id - c| <= R (box from Minv) */
static void or_enumerate_nd(int d, const double* M, const double* Minv, const double* c, double R,
                            void (*f)(void*, const double*, const int*), void* ctx) {
  double mc[OR_MAXD];
  int lo[OR_MAXD], hi[OR_MAXD], id[OR_MAXD];
  for (int i = 0; i < d; ++i) {
    double s = 0.0, rn = 0.0;
    for (int j = 0; j < d; ++j) {
      s += Minv[i * d + j] * c[j];
      rn += Minv[i * d + j] * Minv[i * d + j];
    }
    mc[i] = s;
    double ext = R * sqrt(rn) + 1e-9;
    lo[i] = (int)floor(mc[i] - ext);
    hi[i] = (int)ceil(mc[i] + ext);
    id[i] = lo[i];
  }
  while (1) {
    double z[OR_MAXD], r2 = 0.0;
    for (int i = 0; i < d; ++i) {
      double v = 0.0;
      for (int j = 0; j < d; ++j) v += M[i * d + j] * (double)id[j];
      z[i] = v;
      r2 += (v - c[i]) * (v - c[i]);
    }
    if (r2 <= R * R) f(ctx, z, id);
    int a = d - 1;
    while (a >= 0 && id[a] == hi[a]) {
      id[a] = lo[a];
      --a;
    }
    if (a < 0) break;
    id[a]++;
  }
}

typedef struct {
  int d, x_in;
  const double *x, *y;
  const int* mx;
  double a, lam, nu;
  or_acc re, im;
  int pole;
} or_nd_sum;

static void or_nd_real_term(void* ctx, const double* z, const int* id) {
  or_nd_sum* S = (or_nd_sum*)ctx;
  if (S->x_in) {
    int same = 1;
    for (int i = 0; i < S->d; ++i) same &= id[i] == S->mx[i];
    if (same) return;
  }
  double r2 = 0.0, yz = 0.0;
  for (int i = 0; i < S->d; ++i) {
    r2 += (z[i] - S->x[i]) * (z[i] - S->x[i]);
    yz += S->y[i] * z[i];
  }
  double phi = or_phi(S->a, OR_PI * r2 / (S->lam * S->lam));
  or_acc_add(&S->re, phi * cos(2.0 * OR_PI * yz));
  or_acc_add(&S->im, -phi * sin(2.0 * OR_PI * yz));
}

static void or_nd_recip_term(void* ctx, const double* g, const int* id) {
  (void)id;
  or_nd_sum* S = (or_nd_sum*)ctx;
  double q2 = 0.0, xq = 0.0;
  for (int i = 0; i < S->d; ++i) {
    double q = g[i] + S->y[i];
    q2 += q * q;
    xq += S->x[i] * q;
  }
  double phi;
  if (q2 == 0.0) {
    if (S->a >= 0.0) {
      S->pole = 1;
      return;
    }
    phi = -1.0 / S->a;
  } else {
    phi = or_phi(S->a, OR_PI * S->lam * S->lam * q2);
  }
  or_acc_add(&S->re, phi * cos(2.0 * OR_PI * xq));
  or_acc_add(&S->im, -phi * sin(2.0 * OR_PI * xq));
}

/* The splitting of Z written for any d (the same formula as or_epstein_zeta, with its own
 * linear algebra and enumeration); d <= OR_MAXD. */
int or_epstein_zeta_nd(int d, const double* A, double nu, const double* x, const double* y, double lam,
                       double r_real, double r_recip, double* re, double* im) {
  if (d < 1 || d > OR_MAXD) return 1;
  if (or_gamma_pole(0.5 * nu)) return 2;
  double Ai[OR_MAXD * OR_MAXD], AiT[OR_MAXD * OR_MAXD], At[OR_MAXD * OR_MAXD], det;
  if (or_inverse_nd(d, A, Ai, &det)) return 1;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      AiT[i * d + j] = Ai[j * d + i];
      At[i * d + j] = A[j * d + i];
    }
  double V = fabs(det);
  int mx[OR_MAXD], x_in = 1;
  for (int i = 0; i < d; ++i) {
    double v = 0.0;
    for (int j = 0; j < d; ++j) v += Ai[i * d + j] * x[j];
    mx[i] = (int)lround(v);
    if (fabs(v - mx[i]) > 1e-12) x_in = 0;
  }
  or_nd_sum R = {d, x_in, x, y, mx, 0.5 * nu, lam, nu, {0, 0}, {0, 0}, 0};
  or_enumerate_nd(d, A, Ai, x, r_real, or_nd_real_term, &R);
  double my[OR_MAXD];
  for (int i = 0; i < d; ++i) my[i] = -y[i];
  or_nd_sum K = {d, 0, x, y, mx, 0.5 * (d - nu), lam, nu, {0, 0}, {0, 0}, 0};
  or_enumerate_nd(d, AiT, At, my, r_recip, or_nd_recip_term, &K);
  if (K.pole) return 2;
  double c = pow(lam, (double)d) / V;
  double tre = or_acc_get(&R.re) + c * or_acc_get(&K.re);
  double tim = or_acc_get(&R.im) + c * or_acc_get(&K.im);
  if (x_in) {
    double xy = 0.0;
    for (int i = 0; i < d; ++i) xy += x[i] * y[i];
    tre -= (2.0 / nu) * cos(2.0 * OR_PI * xy);
    tim += (2.0 / nu) * sin(2.0 * OR_PI * xy);
  }
  double P = or_prefactor(nu, lam);
  *re = P * tre;
  *im = P * tim;
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Singular part (Sec. 3)                                                      */
/* ------------------------------------------------------------------------- */
/* coefficient sigma_nu with s_hat_nu(k) = sigma_nu |k|^{nu-d} [log(pi k^2)]^{is_log} */
static double or_sigma(int d, double nu, int* is_log) {
  double mm = 0.5 * (nu - d);
  int m = -1;
  if (fabs(mm - round(mm)) < 1e-12 && round(mm) >= 0.0) m = (int)round(mm);
  if (m >= 0) {
    *is_log = 1;
    double mf = tgamma((double)m + 1.0);
    double sgn = (m % 2 == 0) ? -1.0 : 1.0; /* (-1)^{m+1} */
    return pow(OR_PI, 2.0 * m + 0.5 * d) / tgamma(m + 0.5 * d) * sgn / mf;
  }
  *is_log = 0;
  return pow(OR_PI, nu - 0.5 * d) * tgamma(0.5 * (d - nu)) / tgamma(0.5 * nu);
}

double or_s_hat(int d, double nu, const double* k) {
  int lg;
  double sig = or_sigma(d, nu, &lg);
  double k2 = 0.0;
  for (int i = 0; i < d; ++i) k2 += k[i] * k[i];
  double v = sig * pow(k2, 0.5 * (nu - d));
  if (lg) v *= log(OR_PI * k2);
  return v;
}

int or_epstein_zeta_reg(int d, const double* A, double nu, const double* k, double lam,
                        double r_real, double r_recip, double* out) {
  double x0[3] = {0, 0, 0}, re, im;
  int rc = or_epstein_zeta(d, A, nu, x0, k, lam, r_real, r_recip, &re, &im);
  if (rc) return rc;
  *out = re - or_s_hat(d, nu, k) / fabs(or_det(d, A));
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Gauss-Legendre and Hadamard integrals                                       */
/* ------------------------------------------------------------------------- */
/* P_n(z) and D_n = P_n(z) - P_{n-1}(z) at z = 1 - delta, from the Legendre recurrence
 * rewritten for differences: D_{k+1} = (k D_k - (2k+1) delta P_k) / (k+1), P_{k+1} = P_k + D_{k+1}.
 * It never forms z = 1 - delta, so nodes close to z = 1 keep their relative accuracy. */
static void or_legendre_delta(int n, double delta, double* pn, double* dn) {
  double p = 1.0 - delta, dd = -delta; /* P_1, D_1 */
  if (n == 0) {
    *pn = 1.0;
    *dn = 0.0;
    return;
  }
  for (int k = 1; k < n; ++k) {
    double nd = ((double)k * dd - (2.0 * k + 1.0) * delta * p) / (k + 1.0);
    p += nd;
    dd = nd;
  }
  *pn = p;
  *dn = dd;
}

/* Gauss-Legendre nodes on [0,1], ascending: Newton's method on f(theta) = P_n(cos theta),
 * f'(theta) = -n (P_{n-1} - z P_n) / sin(theta) = -n (delta P_n - D_n) / sin(theta), with
 * delta = 1 - cos(theta) = 2 sin^2(theta/2).  Nodes x = sin^2(theta/2) = delta/2 and weights
 * sin^2(theta) / (n (P_{n-1} - z P_n))^2 (the [-1,1] weight halved) for theta <= pi/2; the
 * upper half by the symmetry x -> 1 - x. */
void or_gauss_legendre01(int n, double* x, double* w) {
  int half = (n + 1) / 2;
  for (int i = 0; i < half; ++i) {
    double th = OR_PI * (i + 0.75) / (n + 0.5);
    if (2 * i + 1 == n) th = 0.5 * OR_PI; /* middle root of odd n: z = 0 */
    double pn, dn;
    for (int it = 0; it < 100 && 2 * i + 1 != n; ++it) {
      double sh = sin(0.5 * th);
      double delta = 2.0 * sh * sh;
      or_legendre_delta(n, delta, &pn, &dn);
      double fp = -(double)n * (delta * pn - dn) / sin(th);
      double step = pn / fp;
      th -= step;
      if (fabs(step) < 1e-16 * th) break;
    }
    double sh = sin(0.5 * th), ch = cos(0.5 * th);
    double delta = 2.0 * sh * sh;
    or_legendre_delta(n, delta, &pn, &dn);
    double q = (double)n * (delta * pn - dn);
    double s = sin(th);
    x[i] = sh * sh;
    w[i] = s * s / (q * q);
    x[n - 1 - i] = ch * ch;
    w[n - 1 - i] = w[i];
  }
}

/* I_m(mu) = finite part of int_0^eps u^{mu-1} L(u)^m du, L(u) = log(pi u^2 w2):
 * I_0 = eps^mu / mu, and integrating by parts
 * I_m = eps^mu L(eps)^m / mu - (2m/mu) I_{m-1}   (Sec. 3, closed forms for m <= 3). */
double or_hadamard(double mu, int m, double eps, double w2) {
  double L = log(OR_PI * eps * eps * w2);
  double em = pow(eps, mu);
  double I = em / mu;
  double Lp = 1.0;
  for (int j = 1; j <= m; ++j) {
    Lp *= L;
    I = em * Lp / mu - (2.0 * j / mu) * I;
  }
  return I;
}

/* ------------------------------------------------------------------------- */
/* n-body lattice sums                                                         */
/* ------------------------------------------------------------------------- */
typedef struct {
  const or_problem* P;
  int d, nsect, nu_tot;
  double Ai[9], AiT[9], At[9], V, vol_fac;
  double pref[OR_MAXNU];
  or_points real;   /* 0 < |z| <= r_real */
  double* g;        /* real.n x n_distinct : Phi_{nu/2}(pi |z|^2 / lam^2) */
  or_points rec;    /* |g| <= r_recip + max_BZ |k| */
  double* phin;     /* rec.n x n_distinct x (2 ell + 1): Phi_{a_j + n}(pi lam^2 |G|^2) for the
                       near-part Taylor coefficients (ray-independent, so computed once) */
  double* u_nodes;
  double* u_w;
  double* v_nodes;
  double* v_w;
} or_ctx;

int or_n_sectors(const or_problem* P) { return P->d * (1 << (P->d - 1)); }

static int or_n_panels(double eps) {
  int np = 0;
  double b = eps;
  while (b < 0.5) {
    b = fmin(2.0 * b, 0.5);
    np++;
  }
  return np;
}

int or_n_u_total(const or_problem* P) {
  return P->u_rule == 2 ? P->n_u * or_n_panels(P->eps) : P->n_u;
}

int or_u_rule(const or_problem* P, double* u, double* w) {
  if (P->u_rule != 1 && P->u_rule != 2) return 1; /* the rule must be explicit */
  double* x = (double*)malloc(sizeof(double) * P->n_u);
  double* wx = (double*)malloc(sizeof(double) * P->n_u);
  or_gauss_legendre01(P->n_u, x, wx);
  if (P->u_rule == 1) {
    for (int i = 0; i < P->n_u; ++i) {
      u[i] = 0.5 * x[i];
      w[i] = 0.5 * wx[i];
    }
  } else {
    double a = P->eps;
    int o = 0;
    while (a < 0.5) {
      double b = fmin(2.0 * a, 0.5);
      for (int i = 0; i < P->n_u; ++i) {
        u[o] = a + (b - a) * x[i];
        w[o] = (b - a) * wx[i];
        o++;
      }
      a = b;
    }
  }
  free(x);
  free(wx);
  return 0;
}

static void or_ctx_free(or_ctx* c) {
  or_points_free(&c->real);
  or_points_free(&c->rec);
  free(c->g);
  free(c->phin);
  free(c->u_nodes);
  free(c->u_w);
  free(c->v_nodes);
  free(c->v_w);
}

static void or_ctx_phin(or_ctx* c) {
  const or_problem* P = c->P;
  int d = c->d, D = 2 * P->ell;
  c->phin = (double*)malloc(sizeof(double) * (c->rec.n + 1) * P->n_distinct * (D + 1));
  for (int e = 0; e < c->rec.n; ++e) {
    double G2 = or_dot(d, c->rec.p + 3 * e, c->rec.p + 3 * e);
    for (int j = 0; j < P->n_distinct; ++j)
      for (int n = 0; n <= D; ++n)
        c->phin[(e * P->n_distinct + j) * (D + 1) + n] =
            G2 == 0.0 ? 0.0 : or_phi(0.5 * (d - P->nu[j]) + n, OR_PI * P->lam * P->lam * G2);
  }
}

static int or_ctx_init(or_ctx* c, const or_problem* P) {
  memset(c, 0, sizeof(*c));
  c->P = P;
  int d = P->d;
  c->d = d;
  if (d < 1 || d > 3 || P->n_distinct < 1 || P->n_distinct > OR_MAXNU || P->n_prod < 1 ||
      P->n_prod > OR_MAXPROD || P->n_u < 1 || (d > 1 && P->n_v < 1) || (P->u_rule != 1 && P->u_rule != 2))
    return 1;
  if (or_inverse(d, P->A, c->Ai)) return 1;
  or_transpose(d, c->Ai, c->AiT);
  or_transpose(d, P->A, c->At);
  c->V = fabs(or_det(d, P->A));
  c->vol_fac = pow(P->lam, (double)d) / c->V;
  c->nsect = or_n_sectors(P);
  for (int j = 0; j < P->n_distinct; ++j) {
    if (or_gamma_pole(0.5 * P->nu[j])) return 2;
    c->pref[j] = or_prefactor(P->nu[j], P->lam);
  }
  double zero[3] = {0, 0, 0};
  or_points all = {0};
  or_enumerate(d, P->A, c->Ai, zero, P->r_real, &all);
  for (int e = 0; e < all.n; ++e) {
    int nz = 0;
    for (int i = 0; i < d; ++i) nz |= all.idx[3 * e + i] != 0;
    if (nz) or_points_push(&c->real, d, all.idx + 3 * e, all.p + 3 * e);
  }
  or_points_free(&all);
  c->g = (double*)malloc(sizeof(double) * (c->real.n + 1) * P->n_distinct);
  for (int e = 0; e < c->real.n; ++e) {
    double r2 = 0.0;
    for (int i = 0; i < d; ++i) r2 += c->real.p[3 * e + i] * c->real.p[3 * e + i];
    for (int j = 0; j < P->n_distinct; ++j)
      c->g[e * P->n_distinct + j] = or_phi(0.5 * P->nu[j], OR_PI * r2 / (P->lam * P->lam));
  }
  /* reciprocal points: cover every k = A^{-T} k~ with k~ in [-1/2,1/2]^d */
  double kmax = 0.0;
  for (int corner = 0; corner < (1 << d); ++corner) {
    double kt[3], k[3];
    for (int i = 0; i < d; ++i) kt[i] = (corner >> i & 1) ? 0.5 : -0.5;
    or_matvec(d, c->AiT, kt, k);
    kmax = fmax(kmax, sqrt(or_dot(d, k, k)));
  }
  or_enumerate(d, c->AiT, c->At, zero, P->r_recip + kmax, &c->rec);
  if (P->u_rule == 2) or_ctx_phin(c);
  int nu_t = or_n_u_total(P);
  c->u_nodes = (double*)malloc(sizeof(double) * nu_t);
  c->u_w = (double*)malloc(sizeof(double) * nu_t);
  or_u_rule(P, c->u_nodes, c->u_w);
  int nv = d > 1 ? P->n_v : 1;
  c->v_nodes = (double*)malloc(sizeof(double) * nv);
  c->v_w = (double*)malloc(sizeof(double) * nv);
  if (d > 1)
    or_gauss_legendre01(nv, c->v_nodes, c->v_w);
  else {
    c->v_nodes[0] = 0.0;
    c->v_w[0] = 1.0;
  }
  return 0;
}

/* Z_{nu_j}(k) at x = 0, k = A^{-T} k~, by the splitting (real part only: the sum is
 * symmetric under z -> -z, so the imaginary part vanishes). */
static double or_zeta_at(const or_ctx* c, int j, const double* k, const double* kt) {
  const or_problem* P = c->P;
  int d = c->d;
  double nu = P->nu[j];
  or_acc sr = {0, 0}, sk = {0, 0};
  for (int e = 0; e < c->real.n; ++e) {
    double mk = 0.0;
    for (int i = 0; i < d; ++i) mk += c->real.idx[3 * e + i] * kt[i];
    or_acc_add(&sr, c->g[e * P->n_distinct + j] * cos(2.0 * OR_PI * mk));
  }
  double a = 0.5 * (d - nu);
  double R2 = P->r_recip * P->r_recip;
  for (int e = 0; e < c->rec.n; ++e) {
    double q2 = 0.0;
    for (int i = 0; i < d; ++i) {
      double q = c->rec.p[3 * e + i] + k[i];
      q2 += q * q;
    }
    if (q2 > R2) continue;
    double phi;
    if (q2 == 0.0) {
      if (a >= 0.0) return NAN;
      phi = -1.0 / a;
    } else {
      phi = or_phi(a, OR_PI * P->lam * P->lam * q2);
    }
    or_acc_add(&sk, phi);
  }
  return c->pref[j] * (or_acc_get(&sr) + c->vol_fac * or_acc_get(&sk) - 2.0 / nu);
}

/* direction of sector s at v: y = sigma^j (p v, 1), sigma^j(y)[i] = y[(i - j) mod d] */
static void or_sector_dir(int d, int s, const double* v, double* ktdir) {
  int half = 1 << (d - 1);
  int j = s / half, pbits = s % half;
  double y[3];
  for (int i = 0; i < d - 1; ++i) y[i] = ((pbits >> i) & 1 ? -1.0 : 1.0) * v[i];
  y[d - 1] = 1.0;
  for (int i = 0; i < d; ++i) ktdir[i] = y[((i - j) % d + d) % d];
}

static void or_products(const or_problem* P, const double* Z, double* f) {
  for (int p = 0; p < P->n_prod; ++p) {
    double v = 1.0;
    for (int j = 0; j < P->n_distinct; ++j)
      for (int e = 0; e < P->expo[p][j]; ++e) v *= Z[j];
    f[p] = v;
  }
}

int or_nbody_node(const or_problem* P, int sector, double u, const double* v, double* f,
                  double* kt_out) {
  or_ctx c;
  int rc = or_ctx_init(&c, P);
  if (rc) {
    or_ctx_free(&c);
    return rc;
  }
  double dir[3], kt[3], k[3], Z[OR_MAXNU];
  or_sector_dir(P->d, sector, v, dir);
  for (int i = 0; i < P->d; ++i) kt[i] = u * dir[i];
  or_matvec(P->d, c.AiT, kt, k);
  for (int j = 0; j < P->n_distinct; ++j) Z[j] = or_zeta_at(&c, j, k, kt);
  or_products(P, Z, f);
  if (kt_out)
    for (int i = 0; i < P->d; ++i) kt_out[i] = kt[i];
  or_ctx_free(&c);
  return 0;
}

/* iterate v multi-index (d-1 axes) */
static int or_n_vnodes(const or_ctx* c) {
  int n = 1;
  for (int i = 0; i < c->d - 1; ++i) n *= c->P->n_v;
  return n;
}
static double or_vnode(const or_ctx* c, int iv, double* v) {
  double w = 1.0;
  for (int i = 0; i < c->d - 1; ++i) {
    int ii = iv % c->P->n_v;
    iv /= c->P->n_v;
    v[i] = c->v_nodes[ii];
    w *= c->v_w[ii];
  }
  return w;
}

static void or_far_line(const or_ctx* c, int s, int iu, double* out) {
  const or_problem* P = c->P;
  int d = c->d;
  double u = c->u_nodes[iu], wu = c->u_w[iu];
  double wpow = 2.0 * wu * pow(u, (double)(d - 1));
  or_acc acc[OR_MAXPROD];
  memset(acc, 0, sizeof(acc));
  int nv = or_n_vnodes(c);
  for (int iv = 0; iv < nv; ++iv) {
    double v[3] = {0, 0, 0};
    double wv = or_vnode(c, iv, v);
    double dir[3], kt[3], k[3], Z[OR_MAXNU], f[OR_MAXPROD];
    or_sector_dir(d, s, v, dir);
    for (int i = 0; i < d; ++i) kt[i] = u * dir[i];
    or_matvec(d, c->AiT, kt, k);
    for (int j = 0; j < P->n_distinct; ++j) Z[j] = or_zeta_at(c, j, k, kt);
    or_products(P, Z, f);
    for (int p = 0; p < P->n_prod; ++p) or_acc_add(&acc[p], wpow * wv * f[p]);
  }
  for (int p = 0; p < P->n_prod; ++p) out[p] = or_acc_get(&acc[p]);
}

/* truncated power series in u: c[0..D] */
static void or_series_mul(const double* a, const double* b, double* out, int D) {
  double tmp[2 * OR_MAXELL + 2];
  for (int i = 0; i <= D; ++i) {
    double s = 0.0;
    for (int j = 0; j <= i; ++j) s += a[j] * b[i - j];
    tmp[i] = s;
  }
  memcpy(out, tmp, sizeof(double) * (D + 1));
}

/* Taylor coefficients C_{k,nu_j}(w) = (w.grad)^{2k} Z^reg(0) / (2k)!, k = 0..ell, by
 * Taylor-mode expansion in u of every term of Z^reg(u w):
 *   real space   g(m) cos(2 pi u z.w)            -> (-1)^k (2 pi z.w)^{2k} / (2k)!
 *   h != 0       Phi_a(t0 + delta(u)),  delta = c (2 u G.w + u^2 |w|^2),
 *                Phi_a(t0 + delta) = sum_n (-1)^n Phi_{a+n}(t0) delta^n / n!
 *                (from Phi_a' = -Phi_{a+1})
 *   h = 0        Phi^reg_a(c |w|^2 u^2) from its entire series. */
static void or_taylor(const or_ctx* c, int j, const double* w, double* C) {
  const or_problem* P = c->P;
  int d = c->d, ell = P->ell, D = 2 * ell;
  double nu = P->nu[j];
  double a = 0.5 * (d - nu);
  double cc = OR_PI * P->lam * P->lam;
  double w2 = or_dot(d, w, w);
  or_acc real[OR_MAXELL + 1], rec[OR_MAXELL + 1];
  memset(real, 0, sizeof(real));
  memset(rec, 0, sizeof(rec));
  for (int e = 0; e < c->real.n; ++e) {
    double zw = or_dot(d, c->real.p + 3 * e, w);
    double g = c->g[e * P->n_distinct + j];
    double x = 2.0 * OR_PI * zw, xp = 1.0, fact = 1.0;
    for (int k = 0; k <= ell; ++k) {
      if (k > 0) {
        xp *= x * x;
        fact *= (2.0 * k - 1.0) * (2.0 * k);
      }
      or_acc_add(&real[k], ((k % 2) ? -1.0 : 1.0) * g * xp / fact);
    }
  }
  double R2 = P->r_recip * P->r_recip;
  for (int e = 0; e < c->rec.n; ++e) {
    const double* G = c->rec.p + 3 * e;
    double G2 = or_dot(d, G, G);
    if (G2 == 0.0 || G2 > R2) continue;
    double t0 = cc * G2;
    double delta[2 * OR_MAXELL + 2] = {0};
    delta[1] = 2.0 * cc * or_dot(d, G, w);
    if (D >= 2) delta[2] = cc * w2;
    double S[2 * OR_MAXELL + 2] = {0}, dp[2 * OR_MAXELL + 2] = {0};
    dp[0] = 1.0; /* delta^0 */
    double fact = 1.0;
    for (int n = 0; n <= D; ++n) {
      if (n > 0) {
        or_series_mul(dp, delta, dp, D);
        fact *= n;
      }
      double coef = ((n % 2) ? -1.0 : 1.0) * c->phin[(e * P->n_distinct + j) * (D + 1) + n] / fact;
      for (int i = 0; i <= D; ++i) S[i] += coef * dp[i];
    }
    for (int k = 0; k <= ell; ++k) or_acc_add(&rec[k], S[2 * k]);
  }
  double r[OR_MAXELL + 1];
  or_phi_reg_series(a, P->lam, ell, r);
  double bp = 1.0;
  for (int k = 0; k <= ell; ++k) {
    or_acc_add(&rec[k], r[k] * bp);
    bp *= cc * w2;
  }
  for (int k = 0; k <= ell; ++k) {
    double v = or_acc_get(&real[k]) + c->vol_fac * or_acc_get(&rec[k]);
    if (k == 0) v -= 2.0 / nu;
    C[k] = c->pref[j] * v;
  }
}

int or_reg_taylor(const or_problem* P, int j, const double* w, double* C) {
  or_ctx c;
  int rc = or_ctx_init(&c, P);
  if (!rc) {
    if (!c.phin) or_ctx_phin(&c);
    or_taylor(&c, j, w, C);
  }
  or_ctx_free(&c);
  return rc;
}

/* Near part of one ray for product p: Hadamard integral over (0, eps) of
 * u^{d-1} prod_i (R_i(u) + S_i(u)), R_i = sum_{k<=ell} C_{k,i} u^{2k}, S_i = s_hat_i(u w)/V,
 * expanded over subsets T of singular factors:
 *   sum_T [prod_{i in T} sigma_i |w|^{nu_i-d} / V] sum_{k<=ell} G_{T,k} I_{m_T}(mu_T + 2k),
 * mu_T = d + sum_{i in T}(nu_i - d), m_T = #log factors in T, G_T = prod_{i not in T} R_i
 * kept in full (each factor is truncated at order 2 ell, their product is not truncated
 * again; this is the reading under which Table "taylor" of Sec. 4.1 is reproduced). */
static double or_near_ray(const or_ctx* c, int p, const double* w, double Ctab[][OR_MAXELL + 1]) {
  const or_problem* P = c->P;
  int d = c->d, ell = P->ell;
  int fac[64], nf = 0;
  for (int j = 0; j < P->n_distinct; ++j)
    for (int e = 0; e < P->expo[p][j]; ++e) fac[nf++] = j;
  if (nf > 20) return NAN;
  int K = ell * nf; /* full product of the order-2ell series */
  double w2 = or_dot(d, w, w);
  double wn = sqrt(w2);
  or_acc acc = {0, 0};
  for (long T = 0; T < (1L << nf); ++T) {
    double coef = 1.0, mu = d;
    int mlog = 0;
    double G[8 * OR_MAXELL + 1] = {0};
    G[0] = 1.0;
    for (int f = 0; f < nf; ++f) {
      int j = fac[f];
      double nu = P->nu[j];
      if (T >> f & 1) {
        int lg;
        double sig = or_sigma(d, nu, &lg);
        coef *= sig * pow(wn, nu - d) / c->V;
        mu += nu - d;
        mlog += lg;
      } else {
        double tmp[8 * OR_MAXELL + 1];
        for (int i = 0; i <= K; ++i) {
          double s = 0.0;
          for (int q = 0; q <= i; ++q) if (i - q <= ell) s += G[q] * Ctab[j][i - q];
          tmp[i] = s;
        }
        memcpy(G, tmp, sizeof(tmp));
      }
    }
    for (int k = 0; k <= K; ++k)
      if (G[k] != 0.0) or_acc_add(&acc, coef * G[k] * or_hadamard(mu + 2.0 * k, mlog, P->eps, w2));
  }
  return or_acc_get(&acc);
}

static void or_near_line(const or_ctx* c, int s, double* out) {
  const or_problem* P = c->P;
  int d = c->d;
  or_acc acc[OR_MAXPROD];
  memset(acc, 0, sizeof(acc));
  int nv = or_n_vnodes(c);
  double Ctab[OR_MAXNU][OR_MAXELL + 1];
  for (int iv = 0; iv < nv; ++iv) {
    double v[3] = {0, 0, 0};
    double wv = or_vnode(c, iv, v);
    double dir[3], w[3];
    or_sector_dir(d, s, v, dir);
    or_matvec(d, c->AiT, dir, w);
    for (int j = 0; j < P->n_distinct; ++j) or_taylor(c, j, w, Ctab[j]);
    for (int p = 0; p < P->n_prod; ++p) or_acc_add(&acc[p], 2.0 * wv * or_near_ray(c, p, w, Ctab));
  }
  for (int p = 0; p < P->n_prod; ++p) out[p] = or_acc_get(&acc[p]);
}

int or_nbody_line(const or_problem* P, int sector, int iu, double* out) {
  or_ctx c;
  int rc = or_ctx_init(&c, P);
  if (rc) {
    or_ctx_free(&c);
    return rc;
  }
  if (sector < 0 || sector >= c.nsect || iu >= or_n_u_total(P)) rc = 1;
  else if (iu >= 0) or_far_line(&c, sector, iu, out);
  else if (P->u_rule == 2) or_near_line(&c, sector, out);
  else
    for (int p = 0; p < P->n_prod; ++p) out[p] = 0.0;
  or_ctx_free(&c);
  return rc;
}

int or_nbody(const or_problem* P, int n_threads, double* out, double* far_lines, double* near_lines) {
  or_ctx c;
  int rc = or_ctx_init(&c, P);
  if (rc) {
    or_ctx_free(&c);
    return rc;
  }
  int nu_t = or_n_u_total(P), ns = c.nsect, np = P->n_prod;
  int nfar = ns * nu_t;
  int nlines = nfar + (P->u_rule == 2 ? ns : 0);
  double* lines = (double*)calloc((size_t)nlines * np, sizeof(double));
  if (n_threads < 1) n_threads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
  for (int L = 0; L < nlines; ++L) {
    if (L < nfar)
      or_far_line(&c, L / nu_t, L % nu_t, lines + (size_t)L * np);
    else
      or_near_line(&c, L - nfar, lines + (size_t)L * np);
  }
  for (int p = 0; p < np; ++p) {
    or_acc acc = {0, 0};
    for (int L = 0; L < nlines; ++L) or_acc_add(&acc, lines[(size_t)L * np + p]);
    out[p] = or_acc_get(&acc);
  }
  if (far_lines) memcpy(far_lines, lines, sizeof(double) * (size_t)nfar * np);
  if (near_lines && P->u_rule == 2) memcpy(near_lines, lines + (size_t)nfar * np, sizeof(double) * ns * np);
  free(lines);
  or_ctx_free(&c);
  return 0;
}
