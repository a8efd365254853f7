// Host side of the C ABI declared in include/ezeta.h: argument checks, lattice
// handles, Gauss-Legendre rules, planning of tables and output segments, and the
// launch sequence (setup kernels -> far/near kernels -> fixed-order reductions).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <array>
#include <vector>

#include "ez_ff.cuh"
#include "ez_kernels.h"
#include "ez_phi.cuh"

using namespace ez;

// ---------------------------------------------------------------------------
// errors and launch accounting
// ---------------------------------------------------------------------------
static thread_local std::string t_err;
static thread_local long long t_launches = 0;

static int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  t_err = buf;
  return code;
}

#define EZ_CUDA(call)                                                                              \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) return fail(EZ_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                                       __FILE__, __LINE__);                                        \
  } while (0)

#define EZ_LAUNCHED()                                                                       \
  do {                                                                                      \
    ++t_launches;                                                                           \
    cudaError_t e_ = cudaGetLastError();                                                    \
    if (e_ != cudaSuccess) return fail(EZ_ECUDA, "launch: %s (line %d)", cudaGetErrorString(e_), __LINE__); \
  } while (0)

extern "C" const char* ez_last_error(void) { return t_err.c_str(); }
extern "C" long long ez_launch_count(int reset) {
  long long v = t_launches;
  if (reset) t_launches = 0;
  return v;
}

// ---------------------------------------------------------------------------
// lattices
// ---------------------------------------------------------------------------
// Matrices are stored row by row with row length d (z_i = sum_j A[i d + j] m_j); for
// d <= 3 only the first d * d entries are used, which is the layout the lattice-sum
// planner and the d <= 3 kernels read.
struct ez_lattice_s {
  int d;
  double A[kMaxDnd * kMaxDnd], Ai[kMaxDnd * kMaxDnd], AiT[kMaxDnd * kMaxDnd], At[kMaxDnd * kMaxDnd], V;
};

// inverse and |det| by Gauss-Jordan elimination with partial pivoting
static bool invert(int d, const double* A, double* X, double* absdet) {
  double M[kMaxDnd][2 * kMaxDnd];
  double det = 1.0;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < 2 * d; ++j) M[i][j] = j < d ? A[i * d + j] : (j - d == i ? 1.0 : 0.0);
  for (int c = 0; c < d; ++c) {
    int p = c;
    for (int r = c + 1; r < d; ++r)
      if (std::fabs(M[r][c]) > std::fabs(M[p][c])) p = r;
    if (M[p][c] == 0.0 || !std::isfinite(M[p][c])) return false;
    if (p != c)
      for (int j = 0; j < 2 * d; ++j) std::swap(M[p][j], M[c][j]);
    det *= M[c][c];
    double inv = 1.0 / M[c][c];
    for (int j = 0; j < 2 * d; ++j) M[c][j] *= inv;
    for (int r = 0; r < d; ++r)
      if (r != c) {
        double f = M[r][c];
        for (int j = 0; j < 2 * d; ++j) M[r][j] -= f * M[c][j];
      }
  }
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) X[i * d + j] = M[i][j + d];
  *absdet = std::fabs(det);
  return std::isfinite(*absdet) && *absdet > 0.0;
}

extern "C" int ez_lattice_create(int d, const double* A, double scale, ez_lattice* out) {
  if (!out || !A) return fail(EZ_EINVAL, "ez_lattice_create: NULL argument");
  if (d < 1 || d > kMaxDnd) return fail(EZ_EINVAL, "ez_lattice_create: d = %d not in 1..%d", d, kMaxDnd);
  if (!(scale > 0.0) || !std::isfinite(scale)) return fail(EZ_EINVAL, "ez_lattice_create: scale = %g", scale);
  for (int i = 0; i < d * d; ++i)
    if (!std::isfinite(A[i])) return fail(EZ_EINVAL, "ez_lattice_create: non-finite A");
  ez_lattice L = new ez_lattice_s();
  L->d = d;
  std::memset(L->A, 0, sizeof L->A);
  for (int i = 0; i < d * d; ++i) L->A[i] = scale * A[i];
  if (!invert(d, L->A, L->Ai, &L->V)) {
    delete L;
    return fail(EZ_EINVAL, "ez_lattice_create: singular lattice matrix");
  }
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      L->AiT[i * d + j] = L->Ai[j * d + i];
      L->At[i * d + j] = L->A[j * d + i];
    }
  *out = L;
  return EZ_OK;
}

extern "C" int ez_lattice_destroy(ez_lattice L) {
  delete L;
  return EZ_OK;
}

extern "C" void ez_quadrature_default(ez_quadrature* q) {
  if (!q) return;
  std::memset(q, 0, sizeof *q);
  q->n_u = 32;
  q->n_v = 32;
  q->eps = 1e-2;
  q->ell = 4;
  q->prec = EZ_FP64;
  q->dedupe = 1;
}

// ---------------------------------------------------------------------------
// Gauss-Legendre on [0, 1].  Newton's method in theta on P_n(cos theta).  The
// Legendre recurrence runs on (P_k, P_k - P_{k-1}) at z = 1 - delta with delta =
// 2 sin^2(theta/2) computed directly, so the nodes next to the endpoints keep full
// relative accuracy (the plain recurrence at z = cos(theta) loses ~ eps/theta^2).
// Nodes with theta <= pi/2 are computed, the rest mirrored (x -> 1 - x).
// ---------------------------------------------------------------------------
static void legendre_near_one(int n, double delta, double* p_n, double* diff_n) {
  // k = 1: P_1 = 1 - delta, P_1 - P_0 = -delta
  double p = 1.0 - delta, df = -delta;
  for (int k = 1; k < n; ++k) {
    const double next = (k * df - (2 * k + 1) * delta * p) / (k + 1);
    p += next;
    df = next;
  }
  *p_n = n ? p : 1.0;
  *diff_n = n ? df : 0.0;
}

static void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; 2 * i < n; ++i) {
    const bool middle = 2 * i + 1 == n;
    double th = middle ? 0.5 * kPi : kPi * (4.0 * i + 3.0) / (4.0 * n + 2.0);
    double pn = 0.0, df = 0.0;
    for (int it = 0; it < 60 && !middle; ++it) {
      const double sh = std::sin(0.5 * th);
      const double delta = 2.0 * sh * sh;
      legendre_near_one(n, delta, &pn, &df);
      const double slope = -n * (delta * pn - df) / std::sin(th);
      const double step = pn / slope;
      th -= step;
      if (std::fabs(step) <= 1e-16 * th) break;
    }
    const double sh = std::sin(0.5 * th), ch = std::cos(0.5 * th);
    const double delta = 2.0 * sh * sh;
    legendre_near_one(n, delta, &pn, &df);
    const double q = n * (delta * pn - df), s = std::sin(th);
    x[i] = sh * sh;
    w[i] = s * s / (q * q);
    x[n - 1 - i] = ch * ch;
    w[n - 1 - i] = w[i];
  }
}

// rules are reused across calls (planning a batch of sums must not recompute them)
static void gauss_legendre01_cached(int n, std::vector<double>& x, std::vector<double>& w) {
  static std::mutex mu;
  static std::vector<std::pair<std::vector<double>, std::vector<double>>> cache;  // index n
  {
    std::lock_guard<std::mutex> lock(mu);
    if ((int)cache.size() > n && !cache[n].first.empty()) {
      x = cache[n].first;
      w = cache[n].second;
      return;
    }
  }
  gauss_legendre01(n, x, w);
  std::lock_guard<std::mutex> lock(mu);
  if ((int)cache.size() <= n) cache.resize(n + 1);
  cache[n] = {x, w};
}

// ---------------------------------------------------------------------------
// planning
// ---------------------------------------------------------------------------
namespace {

constexpr double kTcut = 45.0;       // default cutoffs, FP64 form: exp(-45) ~ 3e-20
constexpr double kTcutMixed = 36.0;  // mixed form (stated bound 1e-10): exp(-36) ~ 2e-16

struct Plan {
  const ez_lattice_s* L;
  ez_sum_spec spec;
  int d, nsect, n_ui, n_v, u_rule, ell, prec;
  double lam, r_real, r_recip, eps;
  int M[3], box[3];
  long long cells;
  int rlo[3], rext[3];
  long long rcap;
  double R2enum;
  std::vector<double> un, uw, vn, vw;
  PhiInfo phi[EZ_MAX_NU];       // reciprocal orders (d - nu)/2, argument pi lam^2 |q|^2
  PhiInfo phi_real[EZ_MAX_NU];  // real-space orders nu/2 for the box g, argument t itself
  bool real_tab;                // the box is large enough for tables to pay (else continued fractions)
  double rser[EZ_MAX_NU][16];
  bool near;
  std::vector<int> alpha, alpha_off;
  std::vector<double> hadw;   // near part, integer exponents: Hadamard weight coefficients
  int hadw_lo = 0, hadw_m1 = 0;
  int nch;            // far segments per line (d = 3: v2 chunks)
  int vchunk;         // d = 3: v2 rows per far-field block
  int m_hp[3];        // mixed form: |m_i| >= m_hp[i] summed in plain binary32
  int n_far_seg, n_far_items, near_per_sector, n_near_seg, n_lines_far, n_lines;
  int hslot;                  // d = 3: 16-byte entries of the folded H of one line group
  int part, n_parts;          // the part of the sum this plan computes
  long long line_lo, line_hi; // its far lines [line_lo, line_hi) of sector * n_ui + iu (d <= 2)
                              // or line groups of j * n_ui + iu (d = 3: the four sectors 4 j + pb)
  bool near_active;           // the near part is computed (part 0 of an eps-split sum)
  size_t smem;
};

double psi_int(int m) {  // digamma(m + 1)
  double s = -0.57721566490153286060651209;
  for (int k = 1; k <= m; ++k) s += 1.0 / k;
  return s;
}

bool is_integer(double x) { return std::fabs(x - std::nearbyint(x)) < 1e-12; }

void fill_phi_host(PhiInfo& P, double a, double t_hi_needed) {
  std::memset(&P, 0, sizeof P);
  P.a = a;
  P.two_a = (int)std::lrint(2.0 * a);
  P.half = is_integer(2.0 * a) ? 1 : 0;
  P.log_m = (is_integer(a) && a <= 0.0) ? (int)std::lrint(-a) : -1;
  P.below1 = a < 1.0 ? 1 : 0;
  P.need_lt = (a < 1.0 && (P.log_m >= 0 || !P.half)) ? 1 : 0;
  P.t_geo_end = kT0 * std::pow(kGeoR, kNGeo);
  const double t_half_end = P.t_geo_end + 0.5 * kNHalf;
  int n_rest;  // intervals after the geometric ones
  if (t_hi_needed <= t_half_end)
    n_rest = (int)std::ceil(std::max(0.0, t_hi_needed - P.t_geo_end) / 0.5) + 1;
  else
    n_rest = kNHalf + (int)std::ceil(t_hi_needed - t_half_end) + 1;
  P.n_int = std::min(kNGeo + n_rest, kMaxInt);
  const int nr = P.n_int - kNGeo;
  P.t_hi = nr <= kNHalf ? P.t_geo_end + 0.5 * nr : t_half_end + (nr - kNHalf);
  P.t_geo_end_f = (float)P.t_geo_end;
  P.t_hi_f = (float)P.t_hi;
  double fact = 1.0;
  if (P.log_m >= 0) {
    const int m = P.log_m;
    double mf = 1.0;
    for (int k = 2; k <= m; ++k) mf *= k;
    P.gam = ((m & 1) ? -1.0 : 1.0) / mf;
    for (int n = 0; n < kNSer; ++n) {
      if (n > 0) fact *= n;
      double sg = (n & 1) ? -1.0 : 1.0;
      P.ser[n] = n == m ? P.gam * psi_int(m) : -sg / (fact * (n - m));
    }
  } else {
    P.gam = std::tgamma(a);
    for (int n = 0; n < kNSer; ++n) {
      if (n > 0) fact *= n;
      double sg = (n & 1) ? -1.0 : 1.0;
      P.ser[n] = -sg / (fact * (a + n));
    }
  }
  P.a_f = (float)a;
  // series lengths: sum_{n >= N} |ser_n| t^n (the terms n >= kNSer add < 1e-18 at t = kT0,
  // bounded by the next one) is increasing in t; breakpoint = largest t <= kT0 (bisection,
  // rounded down to binary32) where it is <= tol.  They depend on a alone: computed once
  // per order and kept (planning runs for every served request).
  struct SerBrk {
    float brk[6], brk_mix[6];
  };
  static std::mutex brk_mu;
  static std::map<double, SerBrk> brk_cache;
  {
    std::lock_guard<std::mutex> lk(brk_mu);
    auto it = brk_cache.find(a);
    if (it != brk_cache.end()) {
      std::memcpy(P.ser_brk, it->second.brk, sizeof P.ser_brk);
      std::memcpy(P.ser_brk_mix, it->second.brk_mix, sizeof P.ser_brk_mix);
      return;
    }
  }
  auto tail = [&](int n0, int n1, double t) {
    double s = 0.0, tn = std::pow(t, n0);
    for (int n = n0; n < n1; ++n, tn *= t) s += std::fabs(P.ser[n]) * tn;
    return s;
  };
  auto brk = [&](int N, double tol) {
    double lo = 0.0, hi = kT0;
    if (tail(N, kNSer, hi) + std::fabs(P.ser[kNSer - 1]) * std::pow(hi, kNSer) <= tol) return (float)hi;
    for (int it = 0; it < 48; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (tail(N, kNSer, mid) + std::fabs(P.ser[kNSer - 1]) * std::pow(mid, kNSer) <= tol)
        lo = mid;
      else
        hi = mid;
    }
    return std::nextafter((float)lo, 0.0f);
  };
  for (int i = 0; i < 6; ++i) P.ser_brk[i] = brk(4 + 2 * i, std::ldexp(1.0, -55));
  for (int i = 0; i < 6; ++i) P.ser_brk_mix[i] = brk(4 + 2 * i, std::ldexp(1.0, -46));
  SerBrk e;
  std::memcpy(e.brk, P.ser_brk, sizeof e.brk);
  std::memcpy(e.brk_mix, P.ser_brk_mix, sizeof e.brk_mix);
  std::lock_guard<std::mutex> lk(brk_mu);
  brk_cache[a] = e;
}

// Mixed form, per order a (cached: planning runs for every served request).
// Last grid points t = kT0 + 0.25 i (t <= 64) with |Phi_a(t)| t > 1e-7 and with |Phi_a(t)| > 1e-6.
struct MixScan {
  double bad_mix, bad_mid;
};
const MixScan& mix_scan(double a) {
  static std::mutex mu;
  static std::map<double, MixScan> cache;
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(a);
  if (it != cache.end()) return it->second;
  MixScan m{kT0, kT0};
  for (int i = 0; kT0 + 0.25 * i <= 64.0; ++i) {
    const double t = kT0 + 0.25 * i;
    const double f = std::fabs(phi_accurate(a, t));
    if (f * t > 1e-7) m.bad_mix = t;
    if (f > 1e-6) m.bad_mid = t;
  }
  return cache[a] = m;
}

// Tail fit of order a beyond t_mix: g(s) = t e^t Phi_a(t), s = t_mix/t in (0, 1], Chebyshev
// interpolation at 24 points in x = 2s - 1, truncated to degree 7 and rewritten in powers of s.
struct TailFit {
  float c[8];
};
const TailFit& tail_fit(double a, float tmix_f) {
  static std::mutex mu;
  static std::map<std::pair<double, float>, TailFit> cache;
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find({a, tmix_f});
  if (it != cache.end()) return it->second;
  const double tmix = tmix_f;
  const int N = 24;
  double gv[N], cc[N];
  for (int k = 0; k < N; ++k) {
    const double xk = std::cos(kPi * (k + 0.5) / N);
    const double sk = 0.5 * (xk + 1.0);
    gv[k] = phi_scaled_large(a, tmix / sk);
  }
  for (int q = 0; q < N; ++q) {
    double acc = 0.0;
    for (int k = 0; k < N; ++k) acc += gv[k] * std::cos(kPi * q * (k + 0.5) / N);
    cc[q] = (q == 0 ? 1.0 : 2.0) * acc / N;
  }
  // sum_{q<8} cc[q] T_q(2s - 1) -> powers of s
  double Tm[8][8] = {{0}};  // Tm[q][i]: coefficient of s^i in T_q(2s - 1)
  Tm[0][0] = 1.0;
  Tm[1][0] = -1.0;
  Tm[1][1] = 2.0;
  for (int q = 2; q < 8; ++q)
    for (int i = 0; i < 8; ++i) {
      double v = -Tm[q - 2][i] - 2.0 * Tm[q - 1][i];
      if (i > 0) v += 4.0 * Tm[q - 1][i - 1];
      Tm[q][i] = v;
    }
  TailFit f;
  for (int i = 0; i < 8; ++i) {
    double v = 0.0;
    for (int q = i; q < 8; ++q) v += cc[q] * Tm[q][i];
    f.c[i] = (float)v;
  }
  return cache[{a, tmix_f}] = f;
}

// regularised h = 0 series (lambda piece of the log case included)
void fill_rser(double* r, double a, double lam, int nmax) {
  int m = (is_integer(a) && a <= 0.0) ? (int)std::lrint(-a) : -1;
  double fact = 1.0;
  for (int n = 0; n <= nmax; ++n) {
    if (n > 0) fact *= n;
    double sg = (n & 1) ? -1.0 : 1.0;
    if (n == m)
      r[n] = sg / fact * (psi_int(m) - 2.0 * std::log(lam));
    else
      r[n] = -sg / (fact * (a + n));
  }
}

// combinations of singular factors: returns false if some mu + 2k == 0
bool near_exponents_ok(const Plan& p, int prod, std::string* why) {
  const ez_sum_spec& s = p.spec;
  int e[EZ_MAX_NU], t[EZ_MAX_NU];
  for (int j = 0; j < s.n_distinct; ++j) {
    e[j] = s.expo[prod][j];
    t[j] = 0;
  }
  while (true) {
    double mu = p.d;
    int deg = 0;
    for (int j = 0; j < s.n_distinct; ++j) {
      mu += t[j] * (s.nu[j] - p.d);
      deg += (e[j] - t[j]) * p.ell;
    }
    deg = std::min(deg, kNearMaxDeg);
    for (int k = 0; k <= deg; ++k)
      if (std::fabs(mu + 2 * k) < 1e-9) {
        char b[160];
        snprintf(b, sizeof b, "Hadamard exponent mu + 2k = 0 (mu = %g, k = %d) in product %d", mu, k, prod);
        *why = b;
        return false;
      }
    int j = 0;
    for (; j < s.n_distinct; ++j) {
      if (t[j] < e[j]) {
        t[j]++;
        break;
      }
      t[j] = 0;
    }
    if (j == s.n_distinct) break;
  }
  return true;
}

double sigma_of(int d, double nu, int* islog);

// x_i -> -x_i maps the lattice onto itself for every axis i (A^{-1} R_i A is an integer
// matrix).  Then Z^reg is even in every component of k and each Taylor coefficient with an
// odd alpha_i vanishes.
static bool reflection_symmetric(const ez_lattice_s* L) {
  const int d = L->d;
  for (int i = 0; i < d; ++i)
    for (int r = 0; r < d; ++r)
      for (int c = 0; c < d; ++c) {
        double s = 0.0;
        for (int k = 0; k < d; ++k) s += L->Ai[r * d + k] * (k == i ? -L->A[k * d + c] : L->A[k * d + c]);
        if (std::fabs(s - std::nearbyint(s)) > 1e-9) return false;
      }
  return true;
}

// Near part with integer exponents: the Hadamard weight of u^{mu'-1} log^m(pi u^2 |w|^2) on
// (0, eps) is eps^{mu'} J_m(mu') with J_0 = 1/mu', J_m = (L^m - 2 m J_{m-1}) / mu', i.e. the
// polynomial sum_i c_{m,i}(mu') L^i in L = log(pi eps^2 |w|^2) with c_{m,m} = 1/mu' and
// c_{m,i} = -2 m c_{m-1,i} / mu' (i < m).  The coefficients eps^{mu'} c_{m,i}(mu') depend on
// mu' alone: tabulated here for every mu' = mu + 2k and m the products need, so that a ray
// only evaluates the polynomial in its own L.
static void hadamard_table(Plan& p) {
  p.hadw.clear();
  const ez_sum_spec& s = p.spec;
  for (int j = 0; j < s.n_distinct; ++j)
    if (!is_integer(s.nu[j])) return;
  int islog[EZ_MAX_NU];
  for (int j = 0; j < s.n_distinct; ++j) sigma_of(p.d, s.nu[j], &islog[j]);
  int lo = 1 << 30, hi = -(1 << 30), mmax = 0;
  for (int pr = 0; pr < s.n_prod; ++pr) {
    int e[EZ_MAX_NU], t[EZ_MAX_NU];
    for (int j = 0; j < s.n_distinct; ++j) {
      e[j] = s.expo[pr][j];
      t[j] = 0;
    }
    while (true) {
      int mu = p.d, deg = 0, ml = 0;
      for (int j = 0; j < s.n_distinct; ++j) {
        mu += t[j] * ((int)std::lrint(s.nu[j]) - p.d);
        deg += (e[j] - t[j]) * p.ell;
        ml += t[j] * islog[j];
      }
      deg = std::min(deg, kNearMaxDeg);
      lo = std::min(lo, mu);
      hi = std::max(hi, mu + 2 * deg);
      mmax = std::max(mmax, ml);
      int j = 0;
      for (; j < s.n_distinct; ++j) {
        if (t[j] < e[j]) {
          t[j]++;
          break;
        }
        t[j] = 0;
      }
      if (j == s.n_distinct) break;
    }
  }
  const int m1 = mmax + 1, n = hi - lo + 1;
  p.hadw_lo = lo;
  p.hadw_m1 = m1;
  p.hadw.assign((size_t)n * m1 * m1, 0.0);
  std::vector<double> c((size_t)m1 * m1);
  for (int mu = lo; mu <= hi; ++mu) {
    if (mu == 0) continue;  // mu + 2k = 0 is refused (EZ_EDOMAIN)
    const double inv = 1.0 / mu, em = std::pow(p.eps, (double)mu);
    std::fill(c.begin(), c.end(), 0.0);
    for (int m = 0; m < m1; ++m) {
      c[m * m1 + m] = inv;
      for (int i = 0; i < m; ++i) c[m * m1 + i] = -2.0 * m * c[(m - 1) * m1 + i] * inv;
    }
    for (int q = 0; q < m1 * m1; ++q) p.hadw[(size_t)(mu - lo) * m1 * m1 + q] = em * c[q];
  }
}

// the d = 3 far kernels read the direction table for the binary64 near-origin term
static bool uses_dirlw(const Plan& p) { return p.d == 3; }

// u_nodes/u_weights (optional, both or neither): an explicit far-field u rule replacing the one
// q describes (the adaptive driver); q.u_rule still decides whether the near part is present.
int make_plan(const ez_lattice_s* L, const ez_sum_spec& spec, const ez_quadrature& qin, Plan& p,
              const std::vector<double>* u_nodes = nullptr, const std::vector<double>* u_weights = nullptr) {
  ez_quadrature q = qin;
  p.L = L;
  p.spec = spec;
  p.d = L->d;
  const int d = p.d;
  if (d > kMaxD) return fail(EZ_EUNSUPPORTED, "lattice sums in d = %d > %d are not built (ez_epstein_zeta is)", d, kMaxD);
  if (spec.n_distinct < 1 || spec.n_distinct > EZ_MAX_NU) return fail(EZ_EINVAL, "n_distinct = %d", spec.n_distinct);
  if (spec.n_prod < 1 || spec.n_prod > EZ_MAX_PROD) return fail(EZ_EINVAL, "n_prod = %d", spec.n_prod);
  int maxfac = 0;
  for (int pr = 0; pr < spec.n_prod; ++pr) {
    int nf = 0;
    for (int j = 0; j < spec.n_distinct; ++j) {
      if (spec.expo[pr][j] < 0) return fail(EZ_EINVAL, "negative exponent count");
      nf += spec.expo[pr][j];
    }
    if (nf > kMaxFactor) return fail(EZ_EINVAL, "product %d has %d > %d factors", pr, nf, kMaxFactor);
    maxfac = std::max(maxfac, nf);
  }
  bool singular = false;
  for (int j = 0; j < spec.n_distinct; ++j) {
    double nu = spec.nu[j];
    if (!std::isfinite(nu)) return fail(EZ_EINVAL, "non-finite exponent");
    if (nu <= 0.0 && is_integer(0.5 * nu)) return fail(EZ_EDOMAIN, "exponent %g is a pole of Gamma(nu/2)", nu);
    // the integrand is analytic in u only when nu - d is a positive odd integer
    if (!is_integer(nu)) {
      singular = true;
    } else {
      const int dn = (int)std::lrint(nu) - d;
      if (dn < 0 || (dn % 2) == 0) singular = true;
    }
  }
  if (q.n_u < 1 || q.n_u > 1 << 20) return fail(EZ_EINVAL, "n_u = %d", q.n_u);
  if (d > 1 && (q.n_v < 1 || q.n_v > 256)) return fail(EZ_EINVAL, "n_v = %d (1..256)", q.n_v);
  p.n_v = d > 1 ? q.n_v : 1;
  p.u_rule = q.u_rule ? q.u_rule : (singular ? 2 : 1);
  if (p.u_rule != 1 && p.u_rule != 2) return fail(EZ_EINVAL, "u_rule = %d", q.u_rule);
  p.eps = q.eps > 0.0 ? q.eps : 1e-2;
  if (!(p.eps < 0.5)) return fail(EZ_EINVAL, "eps = %g", p.eps);
  p.ell = q.ell > 0 ? q.ell : 4;
  if (p.ell > kMaxEll) return fail(EZ_EINVAL, "ell = %d > %d", p.ell, kMaxEll);
  p.prec = q.prec;
  if (p.prec != EZ_FP64 && p.prec != EZ_MIXED) return fail(EZ_EINVAL, "prec = %d", q.prec);
  // default splitting parameter (the result does not depend on lam): the separable
  // real-space contraction costs O(M) per node, the reciprocal sum O(terms).  Measured
  // optima on GB300: lam = 2 V for d = 1, 3 V^{1/2} for d = 2; in 3-D the FP64 form is
  // fastest at the largest lam whose real-space box half-width stays <= 16 (4.5 V^{1/3},
  // capped), the mixed form at 4 V^{1/3} (its reciprocal tails are cheap binary32 work);
  // every default is capped so that the box half-width stays <= 16
  const double tcut = p.prec == EZ_MIXED ? kTcutMixed : kTcut;
  if (q.lambda > 0.0) {
    p.lam = q.lambda;
  } else {
    const double f = d == 1 ? 2.0 : d == 2 ? 3.0 : (p.prec == EZ_MIXED ? 4.0 : 4.5);
    double amax = 0.0;
    for (int i = 0; i < d; ++i) {
      double rn = 0.0;
      for (int j = 0; j < d; ++j) rn += L->Ai[i * d + j] * L->Ai[i * d + j];
      amax = std::max(amax, std::sqrt(rn));
    }
    const double lam_cap = 16.0 / (std::sqrt(tcut / kPi) * amax) * (1.0 - 1e-9);
    p.lam = std::min(f * std::pow(L->V, 1.0 / d), q.r_real > 0.0 ? 1e300 : lam_cap);
  }
  p.r_real = q.r_real > 0.0 ? q.r_real : p.lam * std::sqrt(tcut / kPi);
  p.r_recip = q.r_recip > 0.0 ? q.r_recip : std::sqrt(tcut / kPi) / p.lam;
  p.nsect = d * (1 << (d - 1));
  p.near = p.u_rule == 2;

  // real-space box
  p.cells = 1;
  for (int i = 0; i < 3; ++i) {
    if (i < d) {
      double rn = 0.0;
      for (int j = 0; j < d; ++j) rn += L->Ai[i * d + j] * L->Ai[i * d + j];
      p.M[i] = (int)std::ceil(p.r_real * std::sqrt(rn) + 1e-9);
      if (p.M[i] > 16) return fail(EZ_EINVAL, "real-space box half-width %d > 16 (r_real too large)", p.M[i]);
    } else {
      p.M[i] = 0;
    }
    p.box[i] = 2 * p.M[i] + 1;
    p.cells *= p.box[i];
  }
  // mixed form: along lattice axis i, real-space terms with |m_i| >= m_hp[i] are below
  // 1e-8 of the nearest-neighbour term (|z| >= |m_i| / |row_i(A^{-1})|, Phi decreasing),
  // so the contraction stages sum them in plain binary32
  {
    double dmin2 = 1e300;
    for (int a = -2; a <= 2; ++a)
      for (int b = (d > 1 ? -2 : 0); b <= (d > 1 ? 2 : 0); ++b)
        for (int c = (d > 2 ? -2 : 0); c <= (d > 2 ? 2 : 0); ++c) {
          if (!a && !b && !c) continue;
          const int m[3] = {a, b, c};
          double r2 = 0.0;
          for (int i = 0; i < d; ++i) {
            double z = 0.0;
            for (int j = 0; j < d; ++j) z += L->A[i * d + j] * m[j];
            r2 += z * z;
          }
          dmin2 = std::min(dmin2, r2);
        }
    double ref[EZ_MAX_NU];
    for (int j = 0; j < spec.n_distinct; ++j) ref[j] = std::fabs(phi_accurate(0.5 * spec.nu[j], kPi * dmin2 / (p.lam * p.lam)));
    for (int i = 0; i < 3; ++i) {
      p.m_hp[i] = p.M[i] + 1;
      if (i >= d) continue;
      double rn = 0.0;
      for (int j = 0; j < d; ++j) rn += L->Ai[i * d + j] * L->Ai[i * d + j];
      // smallest m <= M with every |Phi(pi m^2 / (rn lam^2))| <= 1e-8 ref (monotone in m: Phi decreases)
      auto small = [&](int m) {
        for (int j = 0; j < spec.n_distinct; ++j)
          if (std::fabs(phi_accurate(0.5 * spec.nu[j], kPi * (m * m / rn) / (p.lam * p.lam))) > 1e-8 * ref[j])
            return false;
        return true;
      };
      int lo = 0, hi = p.M[i] + 1;  // small(hi) taken as true, small(lo) false
      while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (small(mid))
          hi = mid;
        else
          lo = mid;
      }
      p.m_hp[i] = hi;
    }
  }
  p.real_tab = p.cells * spec.n_distinct >= 4096;
  // reciprocal enumeration: |A^{-T} h| <= r_recip + max_BZ |k|
  double kmax = 0.0;
  for (int c = 0; c < (1 << d); ++c) {
    double s = 0.0;
    for (int i = 0; i < d; ++i) {
      double ki = 0.0;
      for (int j = 0; j < d; ++j) ki += L->AiT[i * d + j] * (((c >> j) & 1) ? 0.5 : -0.5);
      s += ki * ki;
    }
    kmax = std::max(kmax, std::sqrt(s));
  }
  double Renum = p.r_recip + kmax;
  p.R2enum = Renum * Renum;
  p.rcap = 1;
  for (int i = 0; i < 3; ++i) {
    int H = 0;
    if (i < d) {
      double cn = 0.0;
      for (int j = 0; j < d; ++j) cn += L->A[j * d + i] * L->A[j * d + i];
      H = (int)std::ceil(Renum * std::sqrt(cn) + 1e-9);
    }
    p.rlo[i] = -H;
    p.rext[i] = 2 * H + 1;
    p.rcap *= p.rext[i];
  }
  if (p.rcap > (1 << 22)) return fail(EZ_EINVAL, "reciprocal box too large (r_recip)");

  // quadrature rules
  std::vector<double> x, w;
  gauss_legendre01_cached(q.n_u, x, w);
  if (u_nodes && u_weights) {
    if (u_nodes->empty() || u_nodes->size() != u_weights->size() || u_nodes->size() > (1u << 20))
      return fail(EZ_EINVAL, "explicit u rule of %zu nodes", u_nodes->size());
    p.un = *u_nodes;
    p.uw = *u_weights;
  } else if (p.u_rule == 1) {
    p.un.resize(q.n_u);
    p.uw.resize(q.n_u);
    for (int i = 0; i < q.n_u; ++i) {
      p.un[i] = 0.5 * x[i];
      p.uw[i] = 0.5 * w[i];
    }
  } else {
    double a = p.eps;
    while (a < 0.5) {
      double b = std::min(2.0 * a, 0.5);
      for (int i = 0; i < q.n_u; ++i) {
        p.un.push_back(a + (b - a) * x[i]);
        p.uw.push_back((b - a) * w[i]);
      }
      a = b;
    }
  }
  p.n_ui = (int)p.un.size();
  if (d > 1) {
    gauss_legendre01_cached(p.n_v, p.vn, p.vw);
  } else {
    p.vn.assign(1, 0.0);
    p.vw.assign(1, 1.0);
  }

  // Phi tables
  const double c_lam = kPi * p.lam * p.lam;
  for (int j = 0; j < spec.n_distinct; ++j) {
    fill_phi_host(p.phi[j], 0.5 * (d - spec.nu[j]), c_lam * p.r_recip * p.r_recip);
    fill_phi_host(p.phi_real[j], 0.5 * spec.nu[j], kPi * p.r_real * p.r_real / (p.lam * p.lam));
    p.phi_real[j].c_lam = 1.0;
    fill_rser(p.rser[j], 0.5 * (d - spec.nu[j]), p.lam, 15);
  }

  // mixed form: t_mix = first t beyond which every |Phi_a(t)| t <= 1e-7, t_mid = first t
  // beyond which every |Phi_a(t)| <= 1e-6 (all exponents of the sum)
  if (p.prec == EZ_MIXED) {
    double tmix = kT0, tmid = kT0;
    for (int j = 0; j < spec.n_distinct; ++j) {
      // the last grid points t = kT0 + 0.25 i with |Phi_a(t)| t > 1e-7 and |Phi_a(t)| > 1e-6:
      // Phi_a decreases, so within [kT0, t_hi] they are the uncapped ones capped at t_hi
      const MixScan& ms = mix_scan(p.phi[j].a);
      const double t_last = kT0 + 0.25 * std::floor((p.phi[j].t_hi - kT0) / 0.25 + 1e-9);
      tmix = std::max(tmix, std::min(ms.bad_mix, t_last) + 0.25);
      tmid = std::max(tmid, std::min(ms.bad_mid, t_last) + 0.25);
    }
    tmid = std::min(tmid, tmix);
    tmix = (double)(float)tmix;
    for (int j = 0; j < spec.n_distinct; ++j) {
      p.phi[j].t_mix_f = (float)tmix;
      p.phi[j].t_mid_f = (float)tmid;
      const TailFit& tf = tail_fit(p.phi[j].a, (float)tmix);
      for (int i = 0; i < 8; ++i) p.phi[j].tail_p[i] = tf.c[i];
    }
  } else {
    for (int j = 0; j < spec.n_distinct; ++j) p.phi[j].t_mix_f = p.phi[j].t_mid_f = 3.0e38f;
  }

  // near part
  if (p.near) {
    p.alpha.clear();
    p.alpha_off.clear();
    const bool even_only = reflection_symmetric(L);  // odd alpha_i: zero coefficients
    for (int k = 0; k <= p.ell; ++k) {
      p.alpha_off.push_back((int)(p.alpha.size() / 3));
      int K2 = 2 * k;
      for (int a0 = K2; a0 >= 0; --a0)
        for (int a1 = (d > 1 ? K2 - a0 : 0); a1 >= 0; --a1) {
          int a2 = K2 - a0 - a1;
          if (d < 3 && a2 != 0) continue;
          if (d < 2 && a1 != 0) continue;
          if (even_only && ((a0 | a1 | a2) & 1)) continue;
          p.alpha.push_back(a0);
          p.alpha.push_back(a1);
          p.alpha.push_back(a2);
        }
    }
    p.alpha_off.push_back((int)(p.alpha.size() / 3));
    for (int pr = 0; pr < spec.n_prod; ++pr) {
      std::string why;
      if (!near_exponents_ok(p, pr, &why)) return fail(EZ_EDOMAIN, "%s", why.c_str());
    }
    hadamard_table(p);
  }

  // segments.  d = 3: a far-field block takes the four sectors of a line group (axis j,
  // u node) and vchunk rows v2 of them; its 256 threads run n_v * rows nodes per sign p2.
  // vchunk is the largest count whose shared memory fits two blocks per SM (98 KB dynamic
  // + the static reciprocal-list cache and tables, <= 14 KB) that maximises (busy thread slots) x
  // (busy block slots of the last wave, 304 = two blocks per SM of the GPU) for the sum.
  p.vchunk = 1;
  if (d == 3) {
    const long long groups = (long long)d * p.n_ui;
    double best = -1.0;
    p.vchunk = std::min(p.n_v, kVChunkMin);
    for (int c = p.n_v; c >= 1; --c) {
      if (c < kVChunkMin && c < p.n_v) break;
      if (far_smem_bytes(d, spec.n_distinct, p.M, p.n_v, c) > 98 * 1024) continue;
      const int nch = (p.n_v + c - 1) / c;
      double work = 0.0, slots = 0.0;
      for (int k = 0; k < nch; ++k) {
        const long long nn = (long long)p.n_v * std::min(c, p.n_v - k * c);
        work += (double)nn;
        slots += 256.0 * (double)((nn + 255) / 256);
      }
      const double blocks = (double)groups * nch;
      const double score = work / slots * blocks / (304.0 * std::ceil(blocks / 304.0));
      if (score > best + 1e-9) {
        best = score;
        p.vchunk = c;
      }
    }
  }
  p.nch = d == 3 ? (p.n_v + p.vchunk - 1) / p.vchunk : 1;
  // part of the sum: far lines [line_lo, line_hi) of sector * n_ui + iu for d <= 2, line
  // groups [line_lo, line_hi) of j * n_ui + iu for d = 3 (d = 1: items are chunks of 128 u
  // nodes; nodes of a chunk outside the range are computed but their lines are empty)
  p.n_parts = q.n_parts > 1 ? q.n_parts : 1;
  p.part = p.n_parts > 1 ? q.part : 0;
  if (p.part < 0 || p.part >= p.n_parts) return fail(EZ_EINVAL, "part %d of %d", q.part, q.n_parts);
  {
    const long long nl = (long long)(d == 3 ? d : p.nsect) * p.n_ui;
    p.line_lo = nl * p.part / p.n_parts;
    p.line_hi = nl * (p.part + 1) / p.n_parts;
  }
  p.near_active = p.near && p.part == 0;
  if (d == 1) {
    p.n_far_seg = p.n_ui;
    p.n_far_items = p.line_hi > p.line_lo ? (int)((p.line_hi - 1) / 128 - p.line_lo / 128 + 1) : 0;
  } else {
    p.n_far_seg = p.nsect * p.n_ui * p.nch;
    p.n_far_items = (int)((p.line_hi - p.line_lo) * p.nch);
  }
  int nrays = d == 1 ? 1 : (d == 2 ? p.n_v : p.n_v * p.n_v);
  p.near_per_sector = p.near ? (nrays + 127) / 128 : 0;
  p.n_near_seg = p.nsect * p.near_per_sector;
  p.n_lines_far = p.nsect * p.n_ui;
  p.n_lines = p.n_lines_far + (p.near ? p.nsect : 0);
  p.smem = far_smem_bytes(d, spec.n_distinct, p.M, p.n_v, p.vchunk);
  {
    int Mx = 0;
    for (int i = 0; i < d; ++i) Mx = std::max(Mx, p.M[i]);
    p.hslot = d == 3 ? spec.n_distinct * (Mx + 1) * (2 * Mx + 1) : 0;
  }
  return EZ_OK;
}

// sigma_nu of s_hat (Sec. 3)
double sigma_of(int d, double nu, int* islog) {
  const int dn = (int)std::lrint(nu) - d;
  if (is_integer(nu) && dn >= 0 && dn % 2 == 0) {
    int m = dn / 2;
    *islog = 1;
    double mf = std::tgamma(m + 1.0);
    return std::pow(kPi, 2.0 * m + 0.5 * d) / std::tgamma(m + 0.5 * d) * ((m & 1) ? 1.0 : -1.0) / mf;
  }
  *islog = 0;
  return std::pow(kPi, nu - 0.5 * d) * std::tgamma(0.5 * (d - nu)) / std::tgamma(0.5 * nu);
}

// ---------------------------------------------------------------------------
// device arena (grow-only) and pinned staging
// ---------------------------------------------------------------------------
struct Arena {
  std::mutex mu;
  int dev = -1;
  char* d = nullptr;
  size_t dcap = 0;
  char* h = nullptr;
  size_t hcap = 0;
};
Arena g_arena;

int arena_reserve(size_t dbytes, size_t hbytes) {
  int dev = 0;
  EZ_CUDA(cudaGetDevice(&dev));
  if (g_arena.dev != dev) {
    g_arena.d = nullptr;
    g_arena.dcap = 0;
    g_arena.dev = dev;
  }
  if (dbytes > g_arena.dcap) {
    if (g_arena.d) cudaFree(g_arena.d);
    g_arena.d = nullptr;
    size_t want = std::max(dbytes, g_arena.dcap * 2);
    if (cudaMalloc(&g_arena.d, want) != cudaSuccess) {
      cudaGetLastError();
      g_arena.dcap = 0;
      return fail(EZ_ENOMEM, "device allocation of %zu bytes failed", want);
    }
    g_arena.dcap = want;
  }
  if (hbytes > g_arena.hcap) {
    if (g_arena.h) cudaFreeHost(g_arena.h);
    g_arena.h = nullptr;
    size_t want = std::max(hbytes, g_arena.hcap * 2);
    if (cudaMallocHost(&g_arena.h, want) != cudaSuccess) {
      cudaGetLastError();
      g_arena.hcap = 0;
      return fail(EZ_ENOMEM, "pinned allocation of %zu bytes failed", want);
    }
    g_arena.hcap = want;
  }
  return EZ_OK;
}

struct Layout {
  size_t off = 0;
  size_t take(size_t bytes, size_t align = 256) {
    off = (off + align - 1) / align * align;
    size_t o = off;
    off += bytes;
    return o;
  }
};

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The constants uploaded here (__constant__ tables read by phitab_kernel, the far kernels'
// shared-memory attributes) live on each device separately: one flag per device ordinal,
// set under a lock once that device has them.
std::mutex g_init_mu;
bool g_init_dev[64] = {false};
int init_constants() {
  int dev = 0;
  EZ_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(EZ_EINVAL, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_init_mu);
  if (g_init_dev[dev]) return EZ_OK;
  // Chebyshev -> monomial matrix: T_j(x) = sum_i c[j][i] x^i
  double c[kNC][kNC];
  std::memset(c, 0, sizeof c);
  c[0][0] = 1.0;
  if (kNC > 1) c[1][1] = 1.0;
  for (int j = 2; j < kNC; ++j)
    for (int i = 0; i < kNC; ++i) c[j][i] = (i > 0 ? 2.0 * c[j - 1][i - 1] : 0.0) - c[j - 2][i];
  // cosine table of the Chebyshev transform and the Chebyshev points, rounded from
  // long double
  double dct[kNC][kNC], xk[kNC];
  for (int k = 0; k < kNC; ++k) {
    xk[k] = (double)std::cos(3.14159265358979323846264338327950288L * (k + 0.5L) / kNC);
    for (int q = 0; q < kNC; ++q)
      dct[k][q] = (double)std::cos(3.14159265358979323846264338327950288L * k * (q + 0.5L) / kNC);
  }
  EZ_CUDA(upload_cheb2mono(&c[0][0], &dct[0][0], xk));
  EZ_CUDA(far_set_smem_limits());
  EZ_CUDA(upload_inv_int());
  g_init_dev[dev] = true;
  return EZ_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// batched lattice sums: a batch holds the plans of its sums, the packed host
// staging (descriptors, quadrature rules, launch lists) and the device memory of
// every table and output segment.  Running a batch launches every kernel of the
// path (tables are rebuilt on each run); nothing but the result leaves the device.
// ---------------------------------------------------------------------------
struct ez_batch_s {
  int n_req = 0;
  std::vector<Plan> plans;
  bool owns = false;
  char* d = nullptr;
  char* h = nullptr;
  size_t dbytes = 0, hbytes = 0;
  size_t o_work = 0, o_phj = 0;
  int n_phase = 0, max_phase_pairs = 0;
  size_t o_req = 0, o_items = 0, o_rj = 0, o_gj = 0, o_pj = 0, o_tj = 0, o_lreq = 0, o_lseg0 = 0, o_lnseg = 0,
         o_rl0 = 0, o_rnl = 0, o_seg = 0, o_lines = 0, o_out = 0;
  int n_phi = 0, n_tay = 0;
  int n_phi_jobs = 0;  // phitab jobs of a run (groups whose table this batch fills)
  bool phi_built = false;  // an owning batch's Phi tables are filled (by its first run)
  size_t o_hj = 0;
  std::vector<std::pair<int, int>> phi_master;  // per distinct a: (request, nu index) computing the table
  // Phi tables held outside the batch (a server's resident tables), per group: the binary64,
  // binary32 and float-float tables (null: the batch holds the group's table), whether this
  // batch fills it (phitab job), and with how many intervals.  Set after a first layout pass.
  std::vector<std::array<void*, 3>> phi_ext;
  std::vector<char> phi_fill;
  std::vector<int> phi_fill_nint;
  std::vector<cudaEvent_t> phi_ready;  // recorded on the run's stream right after its phitab launch
  struct FarGroup {
    int d, ndm;
    bool mixed;
    size_t begin, end, smem;
  };
  std::vector<FarGroup> far;  // far-field launches: items grouped by (d, precision, exponent class)
  size_t near_begin = 0, near_end = 0;
  long long n_lines = 0;
  std::vector<long long> line0;
  bool ran = false;
  bool lines_fresh = false;  // the lines buffer holds the last run's lines
  bool timing = false;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // start, far begin, far end, end
  // owning batches: a second stream for the setup work that does not feed the far kernels
  cudaStream_t aux = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
};

namespace {

// Phi table slot of a plan: reciprocal order j (slot j) or real-space order j (EZ_MAX_NU + j)
const PhiInfo& phi_slot(const Plan& p, int slot) {
  return slot < EZ_MAX_NU ? p.phi[slot] : p.phi_real[slot - EZ_MAX_NU];
}

// chunks of kTaylorCells cells in the half real-space box after the centre cell
long long taylor_chunks(const Plan& p) { return (p.cells / 2 + kTaylorCells - 1) / kTaylorCells; }

int batch_plan(ez_batch_s& B, int n_req, const ez_lattice* lats, const ez_sum_spec* specs,
               const ez_quadrature* quads) {
  if (n_req < 1) return fail(EZ_EINVAL, "n_req = %d", n_req);
  if (!lats || !specs || !quads) return fail(EZ_EINVAL, "NULL argument");
  int rc = EZ_OK;  // host-only: device constants are set up by the launching entry points
  B.n_req = n_req;
  B.plans.assign(n_req, Plan());
  for (int r = 0; r < n_req; ++r) {
    if (!lats[r]) return fail(EZ_EINVAL, "lattice %d is NULL", r);
    rc = make_plan(lats[r], specs[r], quads[r], B.plans[r]);
    if (rc) return rc;
  }
  return EZ_OK;
}

// layout of buffers (fill = false) or packing of the staging with device addresses (fill = true)
int batch_layout(ez_batch_s& B, bool fill) {
  const int n_req = B.n_req;
  std::vector<Plan>& plans = B.plans;
  std::vector<int> order;
  for (int d = 1; d <= 3; ++d)
    for (int r = 0; r < n_req; ++r)
      if (plans[r].d == d) order.push_back(r);
  // ---- sizes
  long long n_seg = 0;
  long long& n_lines = B.n_lines;
  n_lines = 0;
  size_t n_items_far = 0, n_items_near = 0;
  std::vector<long long> seg_far0(n_req), seg_near0(n_req);
  std::vector<long long>& line0 = B.line0;
  line0.assign(n_req, 0);
  for (int r : order) {
    seg_far0[r] = n_seg;
    n_seg += plans[r].n_far_seg;
    n_items_far += plans[r].n_far_items;
  }
  for (int r : order) {
    seg_near0[r] = n_seg;
    n_seg += plans[r].n_near_seg;
    if (plans[r].near_active) n_items_near += plans[r].n_near_seg;
  }
  for (int r = 0; r < n_req; ++r) {
    line0[r] = n_lines;
    n_lines += plans[r].n_lines;
  }
  Layout dl, hl;
  B.o_req = dl.take(sizeof(ReqDesc) * n_req);
  const size_t h_req = hl.take(sizeof(ReqDesc) * n_req);
  B.o_items = dl.take(sizeof(Item) * (n_items_far + n_items_near));
  const size_t h_items = hl.take(sizeof(Item) * (n_items_far + n_items_near));
  B.o_rj = dl.take(sizeof(RecipJob) * n_req);
  const size_t h_rj = hl.take(sizeof(RecipJob) * n_req);
  B.o_gj = dl.take(sizeof(GboxJob) * n_req);
  const size_t h_gj = hl.take(sizeof(GboxJob) * n_req);
  B.o_hj = dl.take(sizeof(HboxJob) * n_req);
  const size_t h_hj = hl.take(sizeof(HboxJob) * n_req);
  int& n_phi = B.n_phi;
  int& n_tay = B.n_tay;
  std::vector<std::vector<int>> phi_group;  // Phi table group of each (request, slot), -1 unused
  n_phi = n_tay = 0;
  for (int r = 0; r < n_req; ++r)
    if (plans[r].near_active) n_tay += plans[r].spec.n_distinct;
  // Phi tables are tabulated in t itself (reciprocal vectors are stored scaled), so they
  // depend on the order a alone: one table per distinct a, computed with the most intervals
  // any member needs and read by every member (slot j < EZ_MAX_NU: reciprocal order j; slot
  // EZ_MAX_NU + j: real-space order j)
  {
    std::vector<std::vector<std::pair<int, int>>> groups;
    for (int r = 0; r < n_req; ++r)
      for (int k = 0; k < (plans[r].real_tab ? 2 : 1); ++k)
        for (int j = 0; j < plans[r].spec.n_distinct; ++j) {
          const int slot = k * EZ_MAX_NU + j;
          const PhiInfo& P = phi_slot(plans[r], slot);
          int g = 0;
          for (; g < (int)groups.size(); ++g) {
            const PhiInfo& Q = phi_slot(plans[groups[g][0].first], groups[g][0].second);
            if (Q.a == P.a && Q.t_geo_end == P.t_geo_end) break;
          }
          if (g == (int)groups.size()) groups.emplace_back();
          groups[g].push_back({r, slot});
        }
    B.phi_master.clear();
    phi_group.assign(n_req, std::vector<int>(2 * EZ_MAX_NU, -1));
    for (int g = 0; g < (int)groups.size(); ++g) {
      size_t m = 0;
      for (size_t i = 1; i < groups[g].size(); ++i)
        if (phi_slot(plans[groups[g][i].first], groups[g][i].second).n_int >
            phi_slot(plans[groups[g][m].first], groups[g][m].second).n_int)
          m = i;
      B.phi_master.push_back(groups[g][m]);
      for (auto& rs : groups[g]) phi_group[rs.first][rs.second] = g;
    }
    n_phi = (int)B.phi_master.size();
  }
  const bool ext = (int)B.phi_ext.size() == n_phi;  // resident tables supplied for these groups
  B.n_phi_jobs = 0;
  for (int g = 0; g < n_phi; ++g) B.n_phi_jobs += (!ext || !B.phi_ext[g][0] || B.phi_fill[g]) ? 1 : 0;
  B.o_pj = dl.take(sizeof(PhiJob) * std::max(B.n_phi_jobs, 1));
  const size_t h_pj = hl.take(sizeof(PhiJob) * std::max(B.n_phi_jobs, 1));
  B.o_tj = dl.take(sizeof(TaylorJob) * std::max(n_tay, 1));
  const size_t h_tj = hl.take(sizeof(TaylorJob) * std::max(n_tay, 1));
  B.o_lreq = dl.take(sizeof(int) * n_lines);
  const size_t h_lreq = hl.take(sizeof(int) * n_lines);
  B.o_lseg0 = dl.take(sizeof(long long) * n_lines);
  const size_t h_lseg0 = hl.take(sizeof(long long) * n_lines);
  B.o_lnseg = dl.take(sizeof(int) * n_lines);
  const size_t h_lnseg = hl.take(sizeof(int) * n_lines);
  B.o_rl0 = dl.take(sizeof(long long) * n_req);
  const size_t h_rl0 = hl.take(sizeof(long long) * n_req);
  B.o_rnl = dl.take(sizeof(int) * n_req);
  const size_t h_rnl = hl.take(sizeof(int) * n_req);
  // phase tables: one per distinct (d, u rule, n_u, eps, n_v) among the d <= 2 sums
  std::vector<int> phase_of(n_req, -1), phase_rep, phase_mp1;
  for (int r = 0; r < n_req; ++r) {
    const Plan& p = plans[r];
    if (p.d > 2) continue;
    int Mx = std::max(p.M[0], p.d > 1 ? p.M[1] : 0);
    int g = -1;
    for (int q = 0; q < (int)phase_rep.size(); ++q) {
      const Plan& o = plans[phase_rep[q]];
      if (o.d == p.d && o.u_rule == p.u_rule && o.n_ui == p.n_ui && o.n_v == p.n_v && o.eps == p.eps &&
          o.un == p.un) {
        g = q;
        break;
      }
    }
    if (g < 0) {
      g = (int)phase_rep.size();
      phase_rep.push_back(r);
      phase_mp1.push_back(Mx + 1);
    }
    phase_mp1[g] = std::max(phase_mp1[g], Mx + 1);
    phase_of[r] = g;
  }
  B.n_phase = (int)phase_rep.size();
  B.max_phase_pairs = 0;
  for (int g = 0; g < B.n_phase; ++g)
    B.max_phase_pairs = std::max(B.max_phase_pairs, plans[phase_rep[g]].n_ui * plans[phase_rep[g]].n_v);
  B.o_phj = dl.take(sizeof(PhaseJob) * std::max(B.n_phase, 1));
  const size_t h_phj = hl.take(sizeof(PhaseJob) * std::max(B.n_phase, 1));
  std::vector<size_t> o_un(n_req), o_uw(n_req), o_vn(n_req), o_vw(n_req), o_al(n_req), o_alo(n_req), o_hw(n_req);
  std::vector<size_t> h_un(n_req), h_uw(n_req), h_vn(n_req), h_vw(n_req), h_al(n_req), h_alo(n_req), h_hw(n_req);
  std::vector<size_t> o_vff(n_req), h_vff(n_req), o_vwff(n_req), h_vwff(n_req);
  std::vector<size_t> o_rec(n_req), o_recf(n_req), o_reclo(n_req), o_rectmp(n_req), o_gbox(n_req), o_tay(n_req),
      o_phig(n_req), o_gboxff(n_req), o_tpart(n_req), o_hbox(n_req), o_dirlw(n_req);
  std::vector<std::vector<size_t>> o_tab(n_req), o_tabf(n_req), o_tabff(n_req);
  for (int r = 0; r < n_req; ++r) {
    Plan& p = plans[r];
    o_un[r] = dl.take(sizeof(double) * p.n_ui);
    h_un[r] = hl.take(sizeof(double) * p.n_ui);
    o_uw[r] = dl.take(sizeof(double) * p.n_ui);
    h_uw[r] = hl.take(sizeof(double) * p.n_ui);
    o_vn[r] = dl.take(sizeof(double) * p.vn.size());
    h_vn[r] = hl.take(sizeof(double) * p.vn.size());
    o_vw[r] = dl.take(sizeof(double) * p.vw.size());
    h_vw[r] = hl.take(sizeof(double) * p.vw.size());
    o_vff[r] = dl.take(sizeof(float2) * p.vn.size());
    h_vff[r] = hl.take(sizeof(float2) * p.vn.size());
    o_vwff[r] = dl.take(sizeof(float2) * p.vw.size());
    h_vwff[r] = hl.take(sizeof(float2) * p.vw.size());
    o_al[r] = dl.take(sizeof(int) * std::max<size_t>(p.alpha.size(), 1));
    h_al[r] = hl.take(sizeof(int) * std::max<size_t>(p.alpha.size(), 1));
    o_alo[r] = dl.take(sizeof(int) * std::max<size_t>(p.alpha_off.size(), 1));
    h_alo[r] = hl.take(sizeof(int) * std::max<size_t>(p.alpha_off.size(), 1));
    o_hw[r] = dl.take(sizeof(double) * std::max<size_t>(p.hadw.size(), 1));
    h_hw[r] = hl.take(sizeof(double) * std::max<size_t>(p.hadw.size(), 1));
  }
  // everything above is uploaded as one prefix: device and staging offsets must agree
  if (dl.off != hl.off || B.o_items != h_items || B.o_rnl != h_rnl ||
      (n_req > 0 && (o_alo[n_req - 1] != h_alo[n_req - 1] || o_un[n_req - 1] != h_un[n_req - 1] ||
                     o_hw[n_req - 1] != h_hw[n_req - 1])))
    return fail(EZ_EINVAL, "internal: staging layout mismatch");
  // device-only tables and outputs
  for (int r = 0; r < n_req; ++r) {
    Plan& p = plans[r];
    o_rec[r] = dl.take(sizeof(G4) * p.rcap);
    o_recf[r] = dl.take(sizeof(float4) * p.rcap);
    o_reclo[r] = dl.take(sizeof(float4) * p.rcap);
    o_rectmp[r] = dl.take(sizeof(G4) * p.rcap);
    o_gbox[r] = dl.take(sizeof(double) * p.cells * p.spec.n_distinct);
    o_gboxff[r] = p.prec == EZ_MIXED ? dl.take(sizeof(float2) * p.cells * p.spec.n_distinct) : 0;
    o_hbox[r] = p.d == 3 ? dl.take(16 * (size_t)p.hslot * std::max<long long>(p.line_hi - p.line_lo, 1)) : 0;
    o_dirlw[r] = uses_dirlw(p) ? dl.take(sizeof(double4) * 12 * (size_t)p.n_v * p.n_v) : 0;
    o_tab[r].assign(2 * EZ_MAX_NU, 0);
    o_tabf[r].assign(2 * EZ_MAX_NU, 0);
    o_tabff[r].assign(2 * EZ_MAX_NU, 0);
    const size_t na = p.alpha.size() / 3;
    o_tay[r] = dl.take(sizeof(double) * std::max<size_t>(na, 1) * p.spec.n_distinct);
    o_phig[r] = p.near ? dl.take(sizeof(double) * p.rcap * (2 * p.ell + 1) * p.spec.n_distinct) : 0;
    o_tpart[r] = p.near ? dl.take(sizeof(double) * std::max<long long>(taylor_chunks(p), 1) * std::max<size_t>(na, 1) *
                                  p.spec.n_distinct)
                        : 0;
  }
  // the Phi tables: one per group, read by every (request, slot) of the group
  std::vector<size_t> o_gtab(n_phi, 0), o_gtabf(n_phi, 0), o_gtabff(n_phi, 0);
  for (int g = 0; g < n_phi; ++g) {
    if (ext && B.phi_ext[g][0]) continue;
    const int ni = phi_slot(plans[B.phi_master[g].first], B.phi_master[g].second).n_int;
    o_gtab[g] = dl.take(sizeof(double) * kRec * ni);
    o_gtabf[g] = dl.take(sizeof(float) * kRec * ni);
    o_gtabff[g] = dl.take(sizeof(float) * kRecFF * ni);
  }
  for (int r = 0; r < n_req; ++r)
    for (int slot = 0; slot < 2 * EZ_MAX_NU; ++slot) {
      const int g = phi_group[r][slot];
      if (g < 0) continue;
      o_tab[r][slot] = o_gtab[g];
      o_tabf[r][slot] = o_gtabf[g];
      o_tabff[r][slot] = o_gtabff[g];
    }
  std::vector<size_t> o_phase(B.n_phase), o_phaseff(B.n_phase, 0);
  std::vector<char> phase_mixed(B.n_phase, 0);
  for (int r = 0; r < n_req; ++r)
    if (phase_of[r] >= 0 && plans[r].prec == EZ_MIXED) phase_mixed[phase_of[r]] = 1;
  for (int g = 0; g < B.n_phase; ++g) {
    const Plan& p = plans[phase_rep[g]];
    const size_t n = (size_t)p.n_ui * p.n_v * phase_mp1[g];
    o_phase[g] = dl.take(sizeof(double2) * n);
    if (phase_mixed[g]) o_phaseff[g] = dl.take(sizeof(float4) * n);
  }
  B.o_seg = dl.take(sizeof(double) * EZ_MAX_PROD * std::max<long long>(n_seg, 1));
  B.o_lines = dl.take(sizeof(double) * EZ_MAX_PROD * n_lines);
  B.o_out = dl.take(sizeof(double) * EZ_MAX_PROD * n_req);
  B.o_work = dl.take(sizeof(unsigned long long) * 3 * n_req);

  if (!fill) {
    B.dbytes = dl.off;
    B.hbytes = hl.off;
    return EZ_OK;
  }
  char* D = B.d;
  char* Hs = B.h;
  auto dptr = [&](size_t o) { return (void*)(D + o); };
  // table k (0 binary64, 1 binary32, 2 float-float) of (request r, slot): resident or the batch's
  auto tab_ptr = [&](int r, int slot, int k) -> void* {
    const int g = phi_group[r][slot];
    if (ext && g >= 0 && B.phi_ext[g][0]) return B.phi_ext[g][k];
    return dptr(k == 0 ? o_tab[r][slot] : k == 1 ? o_tabf[r][slot] : o_tabff[r][slot]);
  };
  // ---- fill host staging
  ReqDesc* reqs = (ReqDesc*)(Hs + h_req);
  Item* items = (Item*)(Hs + h_items);
  RecipJob* rjobs = (RecipJob*)(Hs + h_rj);
  GboxJob* gjobs = (GboxJob*)(Hs + h_gj);
  HboxJob* hjobs = (HboxJob*)(Hs + h_hj);
  PhiJob* pjobs = (PhiJob*)(Hs + h_pj);
  TaylorJob* tjobs = (TaylorJob*)(Hs + h_tj);
  int* lreq = (int*)(Hs + h_lreq);
  long long* lseg0 = (long long*)(Hs + h_lseg0);
  int* lnseg = (int*)(Hs + h_lnseg);
  long long* rl0 = (long long*)(Hs + h_rl0);
  int* rnl = (int*)(Hs + h_rnl);
  int itj = 0;
  for (int r = 0; r < n_req; ++r) {
    Plan& p = plans[r];
    const ez_lattice_s* L = p.L;
    ReqDesc& R = reqs[r];
    std::memset(&R, 0, sizeof R);
    R.d = p.d;
    R.nsect = p.nsect;
    R.n_ui = p.n_ui;
    R.n_v = p.n_v;
    R.u_rule = p.u_rule;
    R.n_distinct = p.spec.n_distinct;
    R.n_prod = p.spec.n_prod;
    R.ell = p.ell;
    R.prec = p.prec;
    std::memcpy(R.expo, p.spec.expo, sizeof R.expo);
    std::memcpy(R.A, L->A, sizeof R.A);
    std::memcpy(R.AiT, L->AiT, sizeof R.AiT);
    R.V = L->V;
    R.lam = p.lam;
    R.c_phys = kPi * p.lam * p.lam;
    const double sc = std::sqrt(R.c_phys);  // reciprocal vectors in units of 1/s
    R.inv_s = 1.0 / sc;
    for (int i = 0; i < 9; ++i) R.AiTs[i] = sc * L->AiT[i];
    R.c_lam = 1.0;
    R.vol_fac = std::pow(p.lam, p.d) / L->V;
    R.R2_recip = R.c_phys * p.r_recip * p.r_recip;
    R.eps = p.eps;
    R.inv_eps = 1.0 / p.eps;
    for (int j = 0; j < p.spec.n_distinct; ++j) {
      double nu = p.spec.nu[j];
      R.nu[j] = nu;
      R.two_over_nu[j] = 2.0 / nu;
      R.pref[j] = std::pow(kPi, 0.5 * nu) / (std::tgamma(0.5 * nu) * std::pow(p.lam, nu));
      R.sig[j] = sigma_of(p.d, nu, &R.islog[j]);
      R.phi[j] = p.phi[j];
      R.phi[j].c_lam = R.c_lam;
      R.phi[j].tab = (const double*)tab_ptr(r, j, 0);
      R.phi[j].tabf = (const float*)tab_ptr(r, j, 1);
      R.phi[j].tabff = (const float*)tab_ptr(r, j, 2);
    }
    for (int i = 0; i < 3; ++i) {
      R.M[i] = p.M[i];
      R.box[i] = p.box[i];
    }
    R.vchunk = p.vchunk;
    for (int i = 0; i < 3; ++i) R.m_hp[i] = p.m_hp[i];
    R.gbox = (const double*)dptr(o_gbox[r]);
    R.rec = (const G4*)dptr(o_rec[r]);
    R.recf = (const float4*)dptr(o_recf[r]);
    R.reclo = (const float4*)dptr(o_reclo[r]);
    R.R2f = (float)R.R2_recip;
    R.work = (unsigned long long*)dptr(B.o_work) + 3 * r;
    R.c_lam_f = 1.0f;
    R.c_lam_ff = make_float2(1.0f, 0.0f);
    R.near_int_mu = 1;
    for (int j = 0; j < p.spec.n_distinct; ++j) R.near_int_mu &= is_integer(p.spec.nu[j]) ? 1 : 0;
    R.order_chain = p.spec.n_distinct >= 3;
    for (int j = 1; j < p.spec.n_distinct; ++j) R.order_chain &= p.spec.nu[j] == p.spec.nu[0] + 2.0 * j;
    R.n_rec = 0;
    R.u_nodes = (const double*)dptr(o_un[r]);
    R.u_w = (const double*)dptr(o_uw[r]);
    R.v_nodes = (const double*)dptr(o_vn[r]);
    R.v_w = (const double*)dptr(o_vw[r]);
    R.v_ff = (const float2*)dptr(o_vff[r]);
    R.vw_ff = (const float2*)dptr(o_vwff[r]);
    {
      float2* vf = (float2*)(Hs + h_vff[r]);
      float2* wf = (float2*)(Hs + h_vwff[r]);
      for (size_t i = 0; i < p.vn.size(); ++i) ff_split(p.vn[i], vf[i].x, vf[i].y);
      for (size_t i = 0; i < p.vw.size(); ++i) ff_split(p.vw[i], wf[i].x, wf[i].y);
      for (int j = 0; j < p.spec.n_distinct; ++j) {
        ff_split(R.pref[j], R.pref_ff[j].x, R.pref_ff[j].y);
        ff_split(R.two_over_nu[j], R.tov_ff[j].x, R.tov_ff[j].y);
      }
      ff_split(R.vol_fac, R.vol_ff.x, R.vol_ff.y);
    }
    if (phase_of[r] >= 0) {
      R.phase = (const double2*)dptr(o_phase[phase_of[r]]);
      R.phaseff = o_phaseff[phase_of[r]] ? (const float4*)dptr(o_phaseff[phase_of[r]]) : nullptr;
      R.phase_mp1 = phase_mp1[phase_of[r]];
    }
    std::memcpy(Hs + h_un[r], p.un.data(), sizeof(double) * p.n_ui);
    std::memcpy(Hs + h_uw[r], p.uw.data(), sizeof(double) * p.n_ui);
    std::memcpy(Hs + h_vn[r], p.vn.data(), sizeof(double) * p.vn.size());
    std::memcpy(Hs + h_vw[r], p.vw.data(), sizeof(double) * p.vw.size());
    R.n_alpha = (int)(p.alpha.size() / 3);
    R.alpha = (const int*)dptr(o_al[r]);
    R.alpha_off = (const int*)dptr(o_alo[r]);
    R.taylor = (const double*)dptr(o_tay[r]);
    if (!p.alpha.empty()) {
      std::memcpy(Hs + h_al[r], p.alpha.data(), sizeof(int) * p.alpha.size());
      std::memcpy(Hs + h_alo[r], p.alpha_off.data(), sizeof(int) * p.alpha_off.size());
    }
    R.dirlw = o_dirlw[r] ? (const double4*)dptr(o_dirlw[r]) : nullptr;
    R.hadw = p.hadw.empty() ? nullptr : (const double*)dptr(o_hw[r]);
    R.hadw_lo = p.hadw_lo;
    R.hadw_m1 = p.hadw_m1;
    if (!p.hadw.empty()) std::memcpy(Hs + h_hw[r], p.hadw.data(), sizeof(double) * p.hadw.size());
    RecipJob& RJ = rjobs[r];
    RJ.req = r;
    for (int i = 0; i < 3; ++i) {
      RJ.lo[i] = p.rlo[i];
      RJ.ext[i] = p.rext[i];
    }
    RJ.R2 = R.c_phys * p.R2enum;
    RJ.cap = (int)p.rcap;
    RJ.out = (G4*)dptr(o_rec[r]);
    RJ.outf = (float4*)dptr(o_recf[r]);
    RJ.outlo = (float4*)dptr(o_reclo[r]);
    RJ.tmp = (G4*)dptr(o_rectmp[r]);
    GboxJob& GJ = gjobs[r];
    std::memset(&GJ, 0, sizeof GJ);
    GJ.req = r;
    GJ.x_in_lattice = 1;
    GJ.R2 = p.r_real * p.r_real;
    GJ.out = (double*)dptr(o_gbox[r]);
    GJ.use_tab = p.real_tab ? 1 : 0;
    for (int j = 0; p.real_tab && j < p.spec.n_distinct; ++j) {
      GJ.phi[j] = p.phi_real[j];
      GJ.phi[j].tab = (const double*)tab_ptr(r, EZ_MAX_NU + j, 0);
      GJ.phi[j].tabf = nullptr;
      GJ.phi[j].tabff = nullptr;
    }
    GJ.outff = o_gboxff[r] ? (float2*)dptr(o_gboxff[r]) : nullptr;
    R.gboxff = o_gboxff[r] ? (const float2*)dptr(o_gboxff[r]) : nullptr;
    HboxJob& HJ = hjobs[r];
    HJ.req = r;
    HJ.g_lo = p.d == 3 ? (int)p.line_lo : 0;
    HJ.g_hi = p.d == 3 ? (int)p.line_hi : 0;
    HJ.out = p.d == 3 && p.prec != EZ_MIXED ? (double2*)dptr(o_hbox[r]) : nullptr;
    HJ.outff = p.d == 3 && p.prec == EZ_MIXED ? (float4*)dptr(o_hbox[r]) : nullptr;
    R.hbox = HJ.out;
    R.hboxff = HJ.outff;
    R.hslot = p.hslot;
    R.hg_lo = HJ.g_lo;
    if (p.near_active)
      for (int j = 0; j < p.spec.n_distinct; ++j) {
        TaylorJob& T = tjobs[itj++];
        T.req = r;
        T.nu_index = j;
        T.phiG = (double*)dptr(o_phig[r]) + (size_t)j * p.rcap * (2 * p.ell + 1);
        std::memcpy(T.rser, p.rser[j], sizeof T.rser);
        T.out = (double*)dptr(o_tay[r]) + (size_t)j * R.n_alpha;
        T.part = (double*)dptr(o_tpart[r]);
        T.n_chunk = (int)taylor_chunks(p);
      }
  }
  for (int g = 0, jb = 0; g < n_phi; ++g) {
    if (ext && B.phi_ext[g][0] && !B.phi_fill[g]) continue;  // resident and already filled
    const int r = B.phi_master[g].first, j = B.phi_master[g].second;
    PhiJob& J = pjobs[jb++];
    const PhiInfo& P = phi_slot(plans[r], j);
    J.a = P.a;
    J.c_lam = 1.0;  // tables in t (reciprocal vectors scaled, real-space argument t itself)
    J.t_geo_end = P.t_geo_end;
    J.n_int = (ext && B.phi_ext[g][0]) ? B.phi_fill_nint[g] : P.n_int;
    J.out = (double*)tab_ptr(r, j, 0);
    J.outf = (float*)tab_ptr(r, j, 1);
    J.outff = (float*)tab_ptr(r, j, 2);
  }
  {
    PhaseJob* phj = (PhaseJob*)(Hs + h_phj);
    for (int g = 0; g < B.n_phase; ++g) {
      const int r = phase_rep[g];
      const Plan& p = plans[r];
      phj[g].n_ui = p.n_ui;
      phj[g].n_v = p.d == 1 ? 1 : p.n_v;
      phj[g].mp1 = phase_mp1[g];
      phj[g].u = (const double*)dptr(o_un[r]);
      phj[g].v = p.d == 1 ? nullptr : (const double*)dptr(o_vn[r]);
      phj[g].out = (double2*)dptr(o_phase[g]);
      phj[g].outff = o_phaseff[g] ? (float4*)dptr(o_phaseff[g]) : nullptr;
    }
  }
  // items (far: grouped by d, precision and exponent class, one launch per group; near after)
  size_t ii = 0;
  B.far.clear();
  for (int d = 1; d <= 3; ++d)
    for (int mixed = 0; mixed < 2; ++mixed)
      for (int ndm : {1, 4, 8}) {
        ez_batch_s::FarGroup g{d, ndm, mixed != 0, ii, ii, 0};
        for (int r : order) {
          Plan& p = plans[r];
          if (p.d != d || (p.prec == EZ_MIXED) != (mixed != 0) || far_nd_class(p.spec.n_distinct) != ndm) continue;
          g.smem = std::max(g.smem, p.smem);
          if (d == 1) {
            for (int c = (int)(p.line_lo / 128); c * 128LL < p.line_hi; ++c)
              items[ii++] = Item{r, 0, c * 128, c, seg_far0[r] + c * 128};
          } else {
            for (long long L = p.line_lo; L < p.line_hi; ++L) {
              // d = 3: L is a line group (axis j, u node); the item covers sectors 4 j .. 4 j + 3
              const int s = (int)(L / p.n_ui) * (d == 3 ? 4 : 1), iu = (int)(L % p.n_ui);
              const long long Ls = (long long)s * p.n_ui + iu;
              for (int c = 0; c < p.nch; ++c) items[ii++] = Item{r, s, iu, c, seg_far0[r] + Ls * p.nch + c};
            }
          }
        }
        g.end = ii;
        if (g.end > g.begin) B.far.push_back(g);
      }
  B.near_begin = ii;
  for (int r : order) {
    Plan& p = plans[r];
    if (!p.near_active) continue;
    long long s0 = seg_near0[r];
    for (int s = 0; s < p.nsect; ++s)
      for (int c = 0; c < p.near_per_sector; ++c) items[ii++] = Item{r, s, 0, c, s0++};
  }
  B.near_end = ii;
  // lines
  for (int r = 0; r < n_req; ++r) {
    Plan& p = plans[r];
    long long L0 = line0[r];
    rl0[r] = L0;
    rnl[r] = p.n_lines;
    for (int s = 0; s < p.nsect; ++s)
      for (int iu = 0; iu < p.n_ui; ++iu) {
        long long L = L0 + (long long)s * p.n_ui + iu;
        const long long Lr = (long long)s * p.n_ui + iu;
        lreq[L] = r;
        lseg0[L] = seg_far0[r] + Lr * p.nch;
        const long long Lp = p.d == 3 ? (long long)(s / 4) * p.n_ui + iu : Lr;  // line (group) of the part range
        lnseg[L] = (Lp >= p.line_lo && Lp < p.line_hi) ? p.nch : 0;  // lines of other parts are empty
      }
    if (p.near)
      for (int s = 0; s < p.nsect; ++s) {
        long long L = L0 + p.n_lines_far + s;
        lreq[L] = r;
        lseg0[L] = seg_near0[r] + (long long)s * p.near_per_sector;
        lnseg[L] = p.near_active ? p.near_per_sector : 0;
      }
  }
  return EZ_OK;
}

int batch_launch(ez_batch_s& B, cudaStream_t stream) {
  char* D = B.d;
  auto dptr = [&](size_t o) { return (void*)(D + o); };
  if (B.timing) EZ_CUDA(cudaEventRecord(B.ev[0], stream));
  EZ_CUDA(cudaMemsetAsync(dptr(B.o_work), 0, sizeof(unsigned long long) * 3 * B.n_req, stream));
  ReqDesc* dreqs = (ReqDesc*)dptr(B.o_req);
  enum_recip_kernel<<<B.n_req, 512, 0, stream>>>(dreqs, (const RecipJob*)dptr(B.o_rj));
  EZ_LAUNCHED();
  {
    long long max_rcap = 0;
    for (auto& p : B.plans) max_rcap = std::max(max_rcap, p.rcap);
    sort_recip_kernel<<<dim3((unsigned)((max_rcap + 255) / 256), B.n_req), 256, 0, stream>>>(
        dreqs, (const RecipJob*)dptr(B.o_rj));
    EZ_LAUNCHED();
  }
  int max_int = 0;
  for (auto& m : B.phi_master) max_int = std::max(max_int, phi_slot(B.plans[m.first], m.second).n_int);
  for (size_t g = 0; g < B.phi_fill_nint.size(); ++g)
    if (B.phi_fill[g]) max_int = std::max(max_int, B.phi_fill_nint[g]);
  // the Phi tables depend on the orders alone: a batch that owns its memory fills them on
  // its first run and keeps them (its runs are ordered on one stream at a time)
  if (B.n_phi_jobs > 0 && !(B.owns && B.phi_built)) {
    phitab_kernel<<<dim3((max_int + kPhiIv - 1) / kPhiIv, B.n_phi_jobs), kPhiIv * kNC, 0, stream>>>(
        (const PhiJob*)dptr(B.o_pj));
    EZ_LAUNCHED();
    if (B.owns) B.phi_built = true;
  }
  for (cudaEvent_t e : B.phi_ready) EZ_CUDA(cudaEventRecord(e, stream));
  // the real-space box reads the real-order Phi tables: after phitab
  long long max_cells = 0;
  for (auto& p : B.plans) max_cells = std::max(max_cells, p.cells * p.spec.n_distinct);
  gbox_kernel<<<dim3((unsigned)((max_cells + 255) / 256), B.n_req), 256, 0, stream>>>(dreqs, (const GboxJob*)dptr(B.o_gj), B.n_req);
  EZ_LAUNCHED();
  // the near part's Taylor tensors (after the box and the tables) run on the batch's second
  // stream while the main stream builds H and the direction table; joined before the far
  // kernels (whose timing window stays free of them)
  const bool fork = B.aux && B.n_tay;
  cudaStream_t ts = fork ? B.aux : stream;
  if (fork) {
    EZ_CUDA(cudaEventRecord(B.fork_ev, stream));
    EZ_CUDA(cudaStreamWaitEvent(B.aux, B.fork_ev, 0));
  }
  if (B.n_tay) {
    long long max_rec = 0;
    for (auto& p : B.plans)
      if (p.near) max_rec = std::max(max_rec, p.rcap);
    phiseq_kernel<<<dim3((unsigned)((max_rec + 127) / 128), B.n_tay), 128, 0, ts>>>(dreqs, (const TaylorJob*)dptr(B.o_tj), B.n_tay);
    EZ_LAUNCHED();
    int max_alpha = 0;
    long long max_chunk = 0;
    for (auto& p : B.plans)
      if (p.near) {
        max_alpha = std::max(max_alpha, (int)(p.alpha.size() / 3));
        max_chunk = std::max(max_chunk, taylor_chunks(p));
      }
    if (max_chunk > 0) {
      taylor_real_kernel<<<dim3((unsigned)max_chunk, B.n_tay), 128, 0, ts>>>(dreqs, (const TaylorJob*)dptr(B.o_tj),
                                                                                  B.n_tay);
      EZ_LAUNCHED();
    }
    taylor_kernel<<<dim3(max_alpha, B.n_tay), 128, 0, ts>>>(dreqs, (const TaylorJob*)dptr(B.o_tj), B.n_tay);
    EZ_LAUNCHED();
  }
  if (fork) EZ_CUDA(cudaEventRecord(B.join_ev, B.aux));
  {  // H of every line group: column chunks (jn, ma, mb >= 0) x axes x requests
    long long max_cols = 0;
    bool mixed_any = false, f64_any = false;
    for (auto& p : B.plans)
      if (p.d == 3 && p.line_hi > p.line_lo) {
        int Mx = 0;
        for (int i = 0; i < 3; ++i) Mx = std::max(Mx, p.M[i]);
        max_cols = std::max(max_cols, (long long)p.spec.n_distinct * (Mx + 1) * (Mx + 1));
        (p.prec == EZ_MIXED ? mixed_any : f64_any) = true;
      }
    if (max_cols > 0) {
      EZ_CUDA(launch_hbox(mixed_any, f64_any, (unsigned)((max_cols + kHboxColsHost - 1) / kHboxColsHost), B.n_req,
                          dreqs, (const HboxJob*)dptr(B.o_hj), stream));
      t_launches += (mixed_any ? 1 : 0) + (f64_any ? 1 : 0);
    }
  }
  {
    long long max_dirs = 0;
    for (auto& p : B.plans)
      if (uses_dirlw(p)) max_dirs = std::max(max_dirs, 12LL * p.n_v * p.n_v);
    if (max_dirs > 0) {
      dirlw_kernel<<<dim3((unsigned)((max_dirs + 255) / 256), B.n_req), 256, 0, stream>>>(dreqs);
      EZ_LAUNCHED();
    }
  }
  if (B.n_phase) {
    phase_kernel<<<dim3((unsigned)((B.max_phase_pairs + 127) / 128), B.n_phase), 128, 0, stream>>>(
        (const PhaseJob*)dptr(B.o_phj));
    EZ_LAUNCHED();
  }
  if (fork) EZ_CUDA(cudaStreamWaitEvent(stream, B.join_ev, 0));
  Item* ditems = (Item*)dptr(B.o_items);
  double* dseg = (double*)dptr(B.o_seg);
  if (B.timing) EZ_CUDA(cudaEventRecord(B.ev[1], stream));
  for (const auto& g : B.far) {
    if (g.d == 3 && g.smem > 200 * 1024) return fail(EZ_EINVAL, "far kernel needs %zu bytes of shared memory", g.smem);
    EZ_CUDA(launch_far(g.d, g.mixed, g.ndm, (unsigned)(g.end - g.begin), g.smem, stream, dreqs, ditems + g.begin, dseg));
    EZ_LAUNCHED();
  }
  if (B.timing) EZ_CUDA(cudaEventRecord(B.ev[2], stream));
  if (B.near_end > B.near_begin) {
    near_kernel<<<(unsigned)(B.near_end - B.near_begin), 128, 0, stream>>>(dreqs, ditems + B.near_begin, dseg);
    EZ_LAUNCHED();
  }
  // the totals straight from the segments (lines_kernel's order of additions); the lines
  // themselves are written only when a caller asks for them (batch_make_lines)
  double* dout = (double*)dptr(B.o_out);
  total_kernel<<<B.n_req, 128, 0, stream>>>(dreqs, (const long long*)dptr(B.o_rl0), (const int*)dptr(B.o_rnl),
                                            B.n_req, (const long long*)dptr(B.o_lseg0), (const int*)dptr(B.o_lnseg),
                                            dseg, dout);
  EZ_LAUNCHED();
  if (B.timing) EZ_CUDA(cudaEventRecord(B.ev[3], stream));
  B.ran = true;
  B.lines_fresh = false;
  return EZ_OK;
}

// the per-line partial sums of the last run, from its segments (kept until the next run)
int batch_make_lines(ez_batch_s& B, cudaStream_t stream) {
  if (B.lines_fresh || B.n_lines == 0) return EZ_OK;
  char* base = B.d;
  auto dptr = [&](size_t o) { return base + o; };
  lines_kernel<<<(unsigned)((B.n_lines + 127) / 128), 128, 0, stream>>>(
      (const ReqDesc*)dptr(B.o_req), (const int*)dptr(B.o_lreq), (const long long*)dptr(B.o_lseg0),
      (const int*)dptr(B.o_lnseg), (int)B.n_lines, (const double*)dptr(B.o_seg), (double*)dptr(B.o_lines));
  EZ_LAUNCHED();
  B.lines_fresh = true;
  return EZ_OK;
}

}  // namespace

extern "C" int ez_batch_create(int n_req, const ez_lattice* lats, const ez_sum_spec* specs,
                               const ez_quadrature* quads, void* stream, ez_batch* out) {
  if (!out) return fail(EZ_EINVAL, "NULL argument");
  int rc0 = init_constants();
  if (rc0) return rc0;
  ez_batch B = new ez_batch_s();
  int rc = batch_plan(*B, n_req, lats, specs, quads);
  if (!rc) rc = batch_layout(*B, false);
  if (!rc) {
    if (cudaMalloc(&B->d, B->dbytes) != cudaSuccess) {
      cudaGetLastError();
      B->d = nullptr;
      rc = fail(EZ_ENOMEM, "device allocation of %zu bytes failed", B->dbytes);
    } else if (cudaMallocHost(&B->h, B->hbytes) != cudaSuccess) {
      cudaGetLastError();
      B->h = nullptr;
      rc = fail(EZ_ENOMEM, "pinned allocation of %zu bytes failed", B->hbytes);
    }
    B->owns = true;
    // the second stream (optional: without it every kernel runs on the caller's stream)
    if (cudaStreamCreateWithFlags(&B->aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&B->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&B->join_ev, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      if (B->aux) cudaStreamDestroy(B->aux);
      if (B->fork_ev) cudaEventDestroy(B->fork_ev);
      if (B->join_ev) cudaEventDestroy(B->join_ev);
      B->aux = nullptr;
      B->fork_ev = B->join_ev = nullptr;
    }
  }
  if (!rc) rc = batch_layout(*B, true);
  if (!rc) {
    cudaError_t e = cudaMemcpyAsync(B->d, B->h, B->hbytes, cudaMemcpyHostToDevice, (cudaStream_t)stream);
    if (e != cudaSuccess) rc = fail(EZ_ECUDA, "upload: %s", cudaGetErrorString(e));
  }
  if (rc) {
    ez_batch_destroy(B);
    return rc;
  }
  *out = B;
  return EZ_OK;
}

extern "C" int ez_batch_run(ez_batch B, double* out, void* stream_) {
  if (!B) return fail(EZ_EINVAL, "NULL batch");
  cudaStream_t stream = (cudaStream_t)stream_;
  int rc = batch_launch(*B, stream);
  if (rc) return rc;
  if (out) {
    EZ_CUDA(cudaMemcpyAsync(out, B->d + B->o_out, sizeof(double) * EZ_MAX_PROD * B->n_req, cudaMemcpyDefault, stream));
    if (!is_device_ptr(out)) EZ_CUDA(cudaStreamSynchronize(stream));
  }
  return EZ_OK;
}

extern "C" long long ez_batch_n_lines(ez_batch B) { return B ? B->n_lines : -1; }

extern "C" int ez_batch_lines(ez_batch B, double* lines, long long* line_offsets, void* stream_) {
  if (!B || !B->ran) return fail(EZ_EINVAL, "batch has not run");
  cudaStream_t stream = (cudaStream_t)stream_;
  if (lines) {
    int rc = batch_make_lines(*B, stream);
    if (rc) return rc;
    EZ_CUDA(cudaMemcpyAsync(lines, B->d + B->o_lines, sizeof(double) * EZ_MAX_PROD * B->n_lines, cudaMemcpyDefault, stream));
    if (!is_device_ptr(lines)) EZ_CUDA(cudaStreamSynchronize(stream));
  }
  if (line_offsets)
    for (int r = 0; r <= B->n_req; ++r) line_offsets[r] = r < B->n_req ? B->line0[r] : B->n_lines;
  return EZ_OK;
}

extern "C" int ez_batch_timing(ez_batch B, int enable, float* far_ms, float* total_ms) {
  if (!B) return fail(EZ_EINVAL, "NULL batch");
  if ((far_ms || total_ms) && B->timing && B->ran) {
    EZ_CUDA(cudaEventSynchronize(B->ev[3]));
    if (far_ms) EZ_CUDA(cudaEventElapsedTime(far_ms, B->ev[1], B->ev[2]));
    if (total_ms) EZ_CUDA(cudaEventElapsedTime(total_ms, B->ev[0], B->ev[3]));
  } else {
    if (far_ms) *far_ms = -1.f;
    if (total_ms) *total_ms = -1.f;
  }
  if (enable && !B->ev[0])
    for (int i = 0; i < 4; ++i) EZ_CUDA(cudaEventCreate(&B->ev[i]));
  B->timing = enable != 0;
  return EZ_OK;
}

// FP64 flops of the far-field kernels of the last run: counted reciprocal terms
// ((3d - 1) per in-range term, 2n + 1 per evaluated polynomial of n coefficients)
// plus the per-node and per-block real-space and bookkeeping costs of the design.
extern "C" int ez_batch_far_flops(ez_batch B, double* flops, long long* terms, long long* coefs) {
  if (!B || !B->ran) return fail(EZ_EINVAL, "batch has not run");
  std::vector<unsigned long long> w(3 * B->n_req);
  EZ_CUDA(cudaMemcpy(w.data(), B->d + B->o_work, sizeof(unsigned long long) * w.size(), cudaMemcpyDeviceToHost));
  double total = 0.0;
  long long nt = 0, nc = 0;
  for (int r = 0; r < B->n_req; ++r) {
    const Plan& p = B->plans[r];
    const int d = p.d, nd = p.spec.n_distinct;
    int nfac = 0;
    for (int pr = 0; pr < p.spec.n_prod; ++pr)
      for (int j = 0; j < nd; ++j) nfac += p.spec.expo[pr][j];
    const double t = (double)w[3 * r], c = (double)w[3 * r + 1], qt = (double)w[3 * r + 2];
    nt += (long long)w[3 * r];
    nc += (long long)w[3 * r + 1];
    // |G + k|^2 (3d - 1 flops) where it was formed, 2 flops per coefficient (argument and
    // Horner steps), one accumulation per term and order
    double per_term = (3.0 * d - 1.0) * qt + 2.0 * c + 1.0 * t * nd;
    double nodes = (double)p.nsect * p.n_ui * (d == 1 ? 1 : (d == 2 ? p.n_v : (double)p.n_v * p.n_v));
    double per_node = 2.0 * d * d + 4.0 * nd + nfac + 2.0;  // k, assembly, products, weight
    double blocks = 0.0, per_block = 0.0;
    if (d == 1) {
      per_node += p.M[0] * (6.0 + 2.0 * nd);
    } else if (d == 2) {
      const double Ma = 0.5 * (p.M[0] + p.M[1]), Mc = Ma;
      per_node += Ma * (6.0 + 4.0 * nd) + 2.0 * nd;
      blocks = (double)p.nsect * p.n_ui;
      per_block = nd * (Ma + 1) * Mc * 4.0;
    } else {
      // a block covers the four sectors of a line group: the two nodes p1 = +-1 of a
      // (v1, v2, p2) share one pass over ma (two FMAs), B_{+-} one pass over mb (four);
      // H is built by hbox_kernel, outside the far kernel
      const double Mm = (p.M[0] + p.M[1] + p.M[2]) / 3.0;
      per_node += Mm * 2.0 * nd + 3.0 * nd;
      blocks = (double)d * p.n_ui * p.nch;
      const double nv2 = std::min(p.vchunk, p.n_v);
      per_block = (Mm + 1) * p.n_v * 6.0 + (Mm + 1) * nv2 * 6.0 + nd * (Mm + 1) * nv2 * (Mm * 8.0 + 4.0);
    }
    total += per_term + nodes * per_node + blocks * per_block;
  }
  if (flops) *flops = total;
  if (terms) *terms = nt;
  if (coefs) *coefs = nc;
  return EZ_OK;
}

extern "C" int ez_batch_sizes(ez_batch B, long long* device_bytes, long long* staging_bytes) {
  if (!B) return fail(EZ_EINVAL, "NULL batch");
  if (device_bytes) *device_bytes = (long long)B->dbytes;
  if (staging_bytes) *staging_bytes = (long long)B->hbytes;
  return EZ_OK;
}

extern "C" int ez_batch_destroy(ez_batch B) {
  if (!B) return EZ_OK;
  for (int i = 0; i < 4; ++i)
    if (B->ev[i]) cudaEventDestroy(B->ev[i]);
  if (B->aux) {
    cudaStreamSynchronize(B->aux);
    cudaStreamDestroy(B->aux);
  }
  if (B->fork_ev) cudaEventDestroy(B->fork_ev);
  if (B->join_ev) cudaEventDestroy(B->join_ev);
  if (B->owns) {
    if (B->d) cudaFree(B->d);
    if (B->h) cudaFreeHost(B->h);
  }
  delete B;
  return EZ_OK;
}

// one-shot path: the batch lives in the shared arena for the duration of the call
static int run_batch(ez_batch_s& B, double* out, double* lines_out, long long* line_offsets, cudaStream_t stream);

static int run_sums(int n_req, const ez_lattice* lats, const ez_sum_spec* specs, const ez_quadrature* quads,
                    double* out, double* lines_out, long long* line_offsets, cudaStream_t stream) {
  if (!out) return fail(EZ_EINVAL, "NULL argument");
  ez_batch_s B;
  int rc = batch_plan(B, n_req, lats, specs, quads);
  if (rc) return rc;
  return run_batch(B, out, lines_out, line_offsets, stream);
}

// runs the planned batch B (plans set, n_req = plans.size()) in the shared arena
static int run_batch(ez_batch_s& B, double* out, double* lines_out, long long* line_offsets, cudaStream_t stream) {
  int rc0 = init_constants();
  if (rc0) return rc0;
  const int n_req = B.n_req;
  int rc = batch_layout(B, false);
  if (rc) return rc;
  std::lock_guard<std::mutex> lock(g_arena.mu);
  rc = arena_reserve(B.dbytes, B.hbytes);
  if (rc) return rc;
  B.d = g_arena.d;
  B.h = g_arena.h;
  B.owns = false;
  rc = batch_layout(B, true);
  if (rc) return rc;
  EZ_CUDA(cudaMemcpyAsync(B.d, B.h, B.hbytes, cudaMemcpyHostToDevice, stream));
  rc = batch_launch(B, stream);
  if (rc) return rc;
  EZ_CUDA(cudaMemcpyAsync(out, B.d + B.o_out, sizeof(double) * EZ_MAX_PROD * n_req, cudaMemcpyDefault, stream));
  if (lines_out) {
    rc = batch_make_lines(B, stream);
    if (rc) return rc;
    EZ_CUDA(cudaMemcpyAsync(lines_out, B.d + B.o_lines, sizeof(double) * EZ_MAX_PROD * B.n_lines, cudaMemcpyDefault, stream));
  }
  if (line_offsets)
    for (int r = 0; r <= n_req; ++r) line_offsets[r] = r < n_req ? B.line0[r] : B.n_lines;
  EZ_CUDA(cudaStreamSynchronize(stream));
  return EZ_OK;
}

extern "C" int ez_lattice_sums(int n_req, const ez_lattice* lats, const ez_sum_spec* specs,
                               const ez_quadrature* quads, double* out, double* lines, long long* line_offsets,
                               void* stream) {
  return run_sums(n_req, lats, specs, quads, out, lines, line_offsets, (cudaStream_t)stream);
}

extern "C" int ez_layout(int d, const ez_sum_spec* spec, const ez_quadrature* q, int* n_sectors, int* n_u_total,
                         int* u_rule_used) {
  if (!spec || !q) return fail(EZ_EINVAL, "NULL argument");
  ez_lattice_s L;
  L.d = d;
  if (d < 1 || d > 3) return fail(EZ_EINVAL, "d = %d", d);
  double I[9] = {0};
  for (int i = 0; i < d; ++i) I[i * d + i] = 1.0;
  std::memcpy(L.A, I, sizeof I);
  std::memcpy(L.Ai, I, sizeof I);
  std::memcpy(L.AiT, I, sizeof I);
  std::memcpy(L.At, I, sizeof I);
  L.V = 1.0;
  Plan p;
  int rc = make_plan(&L, *spec, *q, p);
  if (rc) return rc;
  if (n_sectors) *n_sectors = p.nsect;
  if (n_u_total) *n_u_total = p.n_ui;
  if (u_rule_used) *u_rule_used = p.u_rule;
  return EZ_OK;
}

extern "C" int ez_plan_describe(ez_lattice lat, const ez_sum_spec* spec, const ez_quadrature* q, ez_plan_info* out) {
  if (!lat || !spec || !q || !out) return fail(EZ_EINVAL, "NULL argument");
  Plan p;
  int rc = make_plan(lat, *spec, *q, p);
  if (rc) return rc;
  std::memset(out, 0, sizeof *out);
  out->lambda = p.lam;
  out->r_real = p.r_real;
  out->r_recip = p.r_recip;
  for (int i = 0; i < 3; ++i) {
    out->M[i] = p.M[i];
    out->m_hp[i] = p.m_hp[i];
  }
  out->n_sectors = p.nsect;
  out->n_u_total = p.n_ui;
  out->u_rule = p.u_rule;
  out->vchunk = p.vchunk;
  out->n_chunks = p.nch;
  out->line_lo = p.line_lo;
  out->line_hi = p.line_hi;
  out->n_far_items = p.n_far_items;
  out->far_smem_bytes = p.smem;
  out->t_mix = p.phi[0].t_mix_f;
  out->t_mid = p.phi[0].t_mid_f;
  out->n_alpha = p.near ? (int)(p.alpha.size() / 3) : 0;
  return EZ_OK;
}

extern "C" int ez_lattice_sum_nbody(ez_lattice lat, const double* nu, int n, const ez_quadrature* q, double* value,
                                    double* err_est, void* stream) {
  if (!lat || !nu || !q || !value) return fail(EZ_EINVAL, "NULL argument");
  if (n < 1 || n > kMaxFactor) return fail(EZ_EINVAL, "n = %d not in 1..%d", n, kMaxFactor);
  ez_sum_spec s;
  std::memset(&s, 0, sizeof s);
  s.n_prod = 1;
  if (q->dedupe == 0) {
    if (n > EZ_MAX_NU) return fail(EZ_EINVAL, "dedupe = 0 supports n <= %d", EZ_MAX_NU);
    s.n_distinct = n;
    for (int i = 0; i < n; ++i) {
      s.nu[i] = nu[i];
      s.expo[0][i] = 1;
    }
  } else {
    for (int i = 0; i < n; ++i) {
      int j = 0;
      for (; j < s.n_distinct; ++j)
        if (s.nu[j] == nu[i]) break;
      if (j == s.n_distinct) {
        if (s.n_distinct == EZ_MAX_NU) return fail(EZ_EINVAL, "more than %d distinct exponents", EZ_MAX_NU);
        s.nu[s.n_distinct++] = nu[i];
      }
      s.expo[0][j]++;
    }
  }
  // with err_est: the same sum on the embedded coarse rule (half the u nodes per panel and
  // half the v nodes per axis, same panels, near part and cutoffs) in the same batch
  ez_lattice ls[2] = {lat, lat};
  ez_sum_spec ss[2] = {s, s};
  ez_quadrature qs[2] = {*q, *q};
  qs[1].n_u = std::max(1, (q->n_u + 1) / 2);
  qs[1].n_v = std::max(1, (q->n_v + 1) / 2);
  const int nreq = err_est ? 2 : 1;
  double out[2 * EZ_MAX_PROD];
  int rc = run_sums(nreq, ls, ss, qs, out, nullptr, nullptr, (cudaStream_t)stream);
  if (rc) return rc;
  double e = err_est ? std::fabs(out[0] - out[EZ_MAX_PROD]) : 0.0;
  if (is_device_ptr(value))
    EZ_CUDA(cudaMemcpyAsync(value, out, sizeof(double), cudaMemcpyHostToDevice, (cudaStream_t)stream));
  else
    *value = out[0];
  if (err_est) {
    if (is_device_ptr(err_est))
      EZ_CUDA(cudaMemcpyAsync(err_est, &e, sizeof(double), cudaMemcpyHostToDevice, (cudaStream_t)stream));
    else
      *err_est = e;
  }
  if (is_device_ptr(value) || (err_est && is_device_ptr(err_est)))
    EZ_CUDA(cudaStreamSynchronize((cudaStream_t)stream));  // the copies read host stack values
  return EZ_OK;
}

// ---------------------------------------------------------------------------
// Adaptive u integration (Sec. 3: the far-field u integral by standard adaptive quadrature
// with recursive interval subdivision).  Global and in rounds, so every round is one batched
// launch: round 0 takes the n-point Gauss-Legendre rule on each starting panel (the graded
// panels [eps, 2 eps], ..., [., 1/2] with the near part on (0, eps) for u_rule 2; [0, 1/4],
// [1/4, 1/2] for u_rule 1); every later round evaluates the two halves of each open panel,
// estimates the panel's error as |Q(panel) - Q(left) - Q(right)| (largest over the products,
// relative to the running total) and closes the panel with Q(left) + Q(right) when that is
// below tol times the panel's share of the interval, else keeps both halves open.
// ---------------------------------------------------------------------------
namespace {
struct UPanel {
  double a, b;
  double q[EZ_MAX_PROD];  // n-point Gauss-Legendre value of the panel (all sectors and v nodes)
  double e[EZ_MAX_PROD];  // error estimate carried by an open panel (half of its parent's)
};

// one batched evaluation of the n-point rule on every panel of `panels` (and of the near part
// when `near`): each panel's value summed over sectors in a fixed order, compensated
int eval_panels(ez_lattice lat, const ez_sum_spec& spec, const ez_quadrature& q, int n, std::vector<UPanel>& panels,
                bool near, double* near_val, long long* nodes, cudaStream_t stream) {
  std::vector<double> gx, gw, un, uw;
  gauss_legendre01_cached(n, gx, gw);
  for (const UPanel& P : panels)
    for (int i = 0; i < n; ++i) {
      un.push_back(P.a + (P.b - P.a) * gx[i]);
      uw.push_back((P.b - P.a) * gw[i]);
    }
  ez_batch_s B;
  B.n_req = 1;
  B.plans.resize(1);
  int rc = make_plan(lat, spec, q, B.plans[0], &un, &uw);
  if (rc) return rc;
  Plan& p = B.plans[0];
  if (!near) p.near_active = false;
  rc = batch_layout(B, false);
  if (rc) return rc;
  std::vector<double> lines((size_t)B.n_lines * EZ_MAX_PROD), out(EZ_MAX_PROD);
  rc = run_batch(B, out.data(), lines.data(), nullptr, stream);
  if (rc) return rc;
  const int np = spec.n_prod, nsect = p.nsect, nui = p.n_ui;
  for (size_t k = 0; k < panels.size(); ++k)
    for (int pr = 0; pr < np; ++pr) {
      double sum = 0.0, c = 0.0;
      for (int sct = 0; sct < nsect; ++sct)
        for (int i = 0; i < n; ++i) {
          const double x = lines[((size_t)sct * nui + k * n + i) * EZ_MAX_PROD + pr];
          const double t = sum + x;
          c += std::fabs(sum) >= std::fabs(x) ? (sum - t) + x : (x - t) + sum;
          sum = t;
        }
      panels[k].q[pr] = sum + c;
    }
  if (near_val)
    for (int pr = 0; pr < np; ++pr) {
      double sum = 0.0;
      if (near && p.near)
        for (int sct = 0; sct < nsect; ++sct) sum += lines[((size_t)nsect * nui + sct) * EZ_MAX_PROD + pr];
      near_val[pr] = sum;
    }
  if (nodes) *nodes += (long long)nui;
  return EZ_OK;
}
}  // namespace

extern "C" int ez_lattice_sum_adaptive(ez_lattice lat, const ez_sum_spec* spec, const ez_quadrature* q, double tol,
                                       int max_rounds, double* value, double* err_est, long long* n_u_used,
                                       void* stream_) {
  cudaStream_t stream = (cudaStream_t)stream_;
  if (!lat || !spec || !q || !value) return fail(EZ_EINVAL, "NULL argument");
  if (!(tol > 0.0) || !(tol < 1.0)) return fail(EZ_EINVAL, "tol = %g not in (0, 1)", tol);
  if (max_rounds < 2 || max_rounds > 60) return fail(EZ_EINVAL, "max_rounds = %d not in 2..60", max_rounds);
  if (q->n_parts > 1) return fail(EZ_EINVAL, "the adaptive rule integrates the whole sum (n_parts = %d)", q->n_parts);
  Plan p0;
  int rc = make_plan(lat, *spec, *q, p0);
  if (rc) return rc;
  const int np = spec->n_prod, n = q->n_u;
  std::vector<UPanel> open;
  double lo = 0.0;
  if (p0.u_rule == 2) {
    lo = p0.eps;
    for (double a = p0.eps; a < 0.5;) {
      const double b = std::min(2.0 * a, 0.5);
      open.push_back(UPanel{a, b, {0, 0, 0, 0}, {0, 0, 0, 0}});
      a = b;
    }
  } else {
    open.push_back(UPanel{0.0, 0.25, {0, 0, 0, 0}, {0, 0, 0, 0}});
    open.push_back(UPanel{0.25, 0.5, {0, 0, 0, 0}, {0, 0, 0, 0}});
  }
  const double len = 0.5 - lo;
  double near_val[EZ_MAX_PROD] = {0, 0, 0, 0}, done[EZ_MAX_PROD] = {0, 0, 0, 0}, err[EZ_MAX_PROD] = {0, 0, 0, 0};
  long long nodes = 0;
  rc = eval_panels(lat, *spec, *q, n, open, p0.u_rule == 2, near_val, &nodes, stream);
  if (rc) return rc;
  for (int round = 1; round < max_rounds && !open.empty(); ++round) {
    std::vector<UPanel> halves;
    for (const UPanel& P : open) {
      const double m = 0.5 * (P.a + P.b);
      halves.push_back(UPanel{P.a, m, {0, 0, 0, 0}, {0, 0, 0, 0}});
      halves.push_back(UPanel{m, P.b, {0, 0, 0, 0}, {0, 0, 0, 0}});
    }
    rc = eval_panels(lat, *spec, *q, n, halves, false, nullptr, &nodes, stream);
    if (rc) return rc;
    // running total for the relative criterion: near part, closed panels, halves of open ones
    double total[EZ_MAX_PROD];
    for (int pr = 0; pr < np; ++pr) {
      total[pr] = near_val[pr] + done[pr];
      for (const UPanel& h : halves) total[pr] += h.q[pr];
    }
    std::vector<UPanel> next;
    for (size_t k = 0; k < open.size(); ++k) {
      const UPanel& P = open[k];
      UPanel L = halves[2 * k], R = halves[2 * k + 1];
      double worst = 0.0;
      for (int pr = 0; pr < np; ++pr) {
        const double e = std::fabs(P.q[pr] - L.q[pr] - R.q[pr]);
        worst = std::max(worst, e / std::max(std::fabs(total[pr]), 1e-300));
        L.e[pr] = R.e[pr] = 0.5 * e;
      }
      if (worst <= tol * (P.b - P.a) / len) {
        for (int pr = 0; pr < np; ++pr) {
          done[pr] += L.q[pr] + R.q[pr];
          err[pr] += L.e[pr] + R.e[pr];
        }
      } else {
        next.push_back(L);
        next.push_back(R);
      }
    }
    open.swap(next);
  }
  // panels still open when the rounds ran out: their values and carried estimates count
  for (const UPanel& P : open)
    for (int pr = 0; pr < np; ++pr) {
      done[pr] += P.q[pr];
      err[pr] += P.e[pr];
    }
  for (int pr = 0; pr < np; ++pr) {
    value[pr] = near_val[pr] + done[pr];
    if (err_est) err_est[pr] = err[pr];
  }
  if (n_u_used) *n_u_used = nodes;
  return EZ_OK;
}

extern "C" int ez_atm_energy(ez_lattice lat, const ez_quadrature* q, double* energy, double* parts, void* stream) {
  if (!lat || !q || !energy) return fail(EZ_EINVAL, "NULL argument");
  ez_sum_spec s;
  std::memset(&s, 0, sizeof s);
  s.n_distinct = 4;
  s.nu[0] = -1.0;
  s.nu[1] = 1.0;
  s.nu[2] = 3.0;
  s.nu[3] = 5.0;
  s.n_prod = 3;
  s.expo[0][2] = 3;  // (3,3,3)
  s.expo[1][0] = 1;  // (-1,5,5)
  s.expo[1][3] = 2;
  s.expo[2][1] = 1;  // (1,3,5)
  s.expo[2][2] = 1;
  s.expo[2][3] = 1;
  double out[EZ_MAX_PROD];
  int rc = run_sums(1, &lat, &s, q, out, nullptr, nullptr, (cudaStream_t)stream);
  if (rc) return rc;
  *energy = out[0] / 24.0 - 3.0 * out[1] / 16.0 + 3.0 * out[2] / 8.0;
  if (parts)
    for (int i = 0; i < 3; ++i) parts[i] = out[i];
  return EZ_OK;
}

// ---------------------------------------------------------------------------
// Epstein zeta at many y
// ---------------------------------------------------------------------------
// d > 3: the real-space ball enumerated once as rows of lattice points (nd_rows_kernel,
// nd_scan_kernel, nd_fill_kernel), then one thread per y (epstein_nd_kernel, which enumerates
// its own reciprocal ball).  Splitting parameter lam = V^{1/d}, cutoffs pi |z - x|^2 / lam^2 <= T
// and pi lam^2 |g + y|^2 <= T.  The row counts are taken in a first pass (one synchronisation)
// so that the cell list is allocated at its exact size.
static int epstein_nd(const ez_lattice_s* L, double nu, const double* x, const double* y, size_t m, double* re,
                      double* im, cudaStream_t stream) {
  const int d = L->d;
  const double lam = std::pow(L->V, 1.0 / d);
  const double s = std::sqrt(kPi) * lam;
  const double r_real = lam * std::sqrt(kTcut / kPi);
  NdBallJob JR;
  std::memset(&JR, 0, sizeof JR);
  JR.d = d;
  // real space: the ball |z - x| <= r_real inside the box round(A^{-1} x) + [-M, M]^d
  int mx[kMaxDnd], Mr[kMaxDnd];
  double xt[kMaxDnd];
  bool x_in = true, x_zero = true;
  for (int i = 0; i < d; ++i) {
    double v = 0.0, rn = 0.0;
    for (int j = 0; j < d; ++j) {
      v += L->Ai[i * d + j] * x[j];
      rn += L->Ai[i * d + j] * L->Ai[i * d + j];
    }
    xt[i] = v;
    mx[i] = (int)std::lrint(v);
    if (std::fabs(v - mx[i]) > 1e-12) x_in = false;
    if (x[i] != 0.0) x_zero = false;
    Mr[i] = (int)std::ceil(r_real * std::sqrt(rn) + 0.5 + 1e-9);
    if (2 * Mr[i] + 1 > kNdMaxExt)
      return fail(EZ_EINVAL, "real-space box half-width %d too large (lattice too skewed)", Mr[i]);
  }
  for (int i = 0; i < d * d; ++i) JR.M[i] = L->A[i];
  for (int i = 0; i < d; ++i) {
    JR.c[i] = x[i];
    JR.lo[i] = mx[i] - Mr[i];
    JR.ext[i] = 2 * Mr[i] + 1;
    JR.cid[i] = mx[i];
  }
  JR.R2 = r_real * r_real;
  JR.a = 0.5 * nu;
  JR.pi_over_lam2 = kPi / (lam * lam);
  JR.skip_center = x_in ? 1 : 0;
  JR.n_prefix = 1;
  for (int l = 0; l + 1 < d; ++l) JR.n_prefix *= JR.ext[l];
  // reciprocal space: Cholesky factor (upper) of the Gram matrix of B = s A^{-T}
  double Rk[kMaxDnd * kMaxDnd] = {0};
  {
    double G[kMaxDnd * kMaxDnd];
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) {
        double g = 0.0;
        for (int k = 0; k < d; ++k) g += (s * L->AiT[k * d + i]) * (s * L->AiT[k * d + j]);
        G[i * d + j] = g;
      }
    for (int i = 0; i < d; ++i) {
      double dg = G[i * d + i];
      for (int k = 0; k < i; ++k) dg -= Rk[k * d + i] * Rk[k * d + i];
      if (!(dg > 0.0)) return fail(EZ_EINVAL, "dual Gram matrix is not positive definite");
      Rk[i * d + i] = std::sqrt(dg);
      for (int j = i + 1; j < d; ++j) {
        double v = G[i * d + j];
        for (int k = 0; k < i; ++k) v -= Rk[k * d + i] * Rk[k * d + j];
        Rk[i * d + j] = v / Rk[i * d + i];
      }
    }
  }
  PhiInfo phi;
  fill_phi_host(phi, 0.5 * (d - nu), kTcut);
  phi.c_lam = 1.0;
  // per-thread phase tables in shared memory: every offset, or above 1 KB per thread (64
  // entries: d = 6 boxes) the non-negative ones only, which doubles the resident warps
  int phase_len = 0;
  for (int i = 0; i < d; ++i) phase_len += 2 * Mr[i] + 1;
  const bool half_phases = phase_len > 64;
  if (half_phases) {
    phase_len = 0;
    for (int i = 0; i < d; ++i) phase_len += Mr[i] + 1;
  }
  unsigned threads = 128;
  while (threads > 32 && (size_t)phase_len * 16 * threads > (size_t)220 * 1024) threads /= 2;
  const size_t smem = (size_t)phase_len * 16 * threads;

  const bool y_dev = is_device_ptr(y), re_dev = is_device_ptr(re), im_dev = im && is_device_ptr(im);
  Layout dl, hl;
  const size_t o_jr = dl.take(sizeof(NdBallJob)), h_jr = hl.take(sizeof(NdBallJob));
  const size_t h_cnt = hl.take(4 * sizeof(int));
  const size_t o_k0r = dl.take(sizeof(int) * JR.n_prefix), o_nr = dl.take(sizeof(int) * JR.n_prefix);
  const size_t o_rowr = dl.take(sizeof(int4) * JR.n_prefix);
  const size_t o_cnt = dl.take(4 * sizeof(int));
  const size_t phase1 = dl.off;
  std::lock_guard<std::mutex> lock(g_arena.mu);
  // uploads the job and enumerates the rows (counts_only: the counts alone)
  auto run_rows = [&](bool counts_only) -> int {
    char* D = g_arena.d;
    char* Hs = g_arena.h;
    JR.row_k0 = (int*)(D + o_k0r);
    JR.row_n = (int*)(D + o_nr);
    JR.rows = (int4*)(D + o_rowr);
    JR.counts = (int*)(D + o_cnt);
    if (counts_only) JR.cell_cap = 0;
    std::memcpy(Hs + h_jr, &JR, sizeof JR);
    EZ_CUDA(cudaMemcpyAsync(D + o_jr, Hs + h_jr, sizeof JR, cudaMemcpyHostToDevice, stream));
    const NdBallJob* jd = (const NdBallJob*)(D + o_jr);
    nd_rows_kernel<<<(unsigned)((JR.n_prefix + 255) / 256), 256, 0, stream>>>(jd);
    EZ_LAUNCHED();
    nd_scan_kernel<<<1, 1024, 0, stream>>>(jd);
    EZ_LAUNCHED();
    if (!counts_only) {
      nd_fill_kernel<<<4 * 152, 256, 0, stream>>>(jd);
      EZ_LAUNCHED();
    }
    return EZ_OK;
  };
  int rc = arena_reserve(phase1, hl.off);
  if (rc) return rc;
  rc = run_rows(true);
  if (rc) return rc;
  EZ_CUDA(cudaMemcpyAsync(g_arena.h + h_cnt, g_arena.d + o_cnt, 2 * sizeof(int), cudaMemcpyDeviceToHost, stream));
  EZ_CUDA(cudaStreamSynchronize(stream));
  int cnt[2];
  std::memcpy(cnt, g_arena.h + h_cnt, sizeof cnt);
  const long long cells_r = std::max(cnt[1], 1);
  const size_t o_g = dl.take(sizeof(double) * cells_r);
  const size_t o_pj = dl.take(sizeof(PhiJob)), h_pj = hl.take(sizeof(PhiJob));
  const size_t o_tab = dl.take(sizeof(double) * kRec * phi.n_int);
  const size_t o_st = dl.take(sizeof(int));
  const size_t o_y = y_dev ? 0 : dl.take(sizeof(double) * m * d);
  const size_t o_re = re_dev ? 0 : dl.take(sizeof(double) * m);
  const size_t o_im = (!im || im_dev) ? 0 : dl.take(sizeof(double) * m);
  rc = arena_reserve(dl.off, hl.off);
  if (rc) return rc;
  char* D = g_arena.d;
  char* Hs = g_arena.h;
  JR.cell_cap = cells_r;
  JR.out = (double*)(D + o_g);
  rc = run_rows(false);
  if (rc) return rc;
  PhiJob& PJ = *(PhiJob*)(Hs + h_pj);
  std::memset(&PJ, 0, sizeof PJ);
  PJ.a = phi.a;
  PJ.c_lam = 1.0;
  PJ.t_geo_end = phi.t_geo_end;
  PJ.n_int = phi.n_int;
  PJ.out = (double*)(D + o_tab);
  EZ_CUDA(cudaMemcpyAsync(D + o_pj, &PJ, sizeof PJ, cudaMemcpyHostToDevice, stream));
  EZ_CUDA(cudaMemsetAsync(D + o_st, 0, sizeof(int), stream));
  if (!y_dev) EZ_CUDA(cudaMemcpyAsync(D + o_y, y, sizeof(double) * m * d, cudaMemcpyHostToDevice, stream));
  phitab_kernel<<<dim3((phi.n_int + kPhiIv - 1) / kPhiIv, 1), kPhiIv * kNC, 0, stream>>>((const PhiJob*)(D + o_pj));
  EZ_LAUNCHED();
  NdEpsteinArgs A;
  std::memset(&A, 0, sizeof A);
  A.d = d;
  A.m = (int)m;
  A.pref = std::pow(kPi, 0.5 * nu) / (std::tgamma(0.5 * nu) * std::pow(lam, nu));
  A.vol_fac = std::pow(lam, d) / L->V;
  A.R2_recip = kTcut;
  A.two_over_nu = 2.0 / nu;
  for (int i = 0; i < d * d; ++i) {
    A.At[i] = L->At[i];
    A.Rk[i] = Rk[i];
  }
  for (int i = 0; i < d; ++i) {
    A.xt[i] = xt[i];
    A.M[i] = Mr[i];
    A.mx[i] = mx[i];
  }
  A.x_zero = x_zero ? 1 : 0;
  A.x_in_lattice = x_in ? 1 : 0;
  A.phase_len = phase_len;
  A.half_phases = half_phases ? 1 : 0;
  A.rows = JR.rows;
  A.rcounts = JR.counts;
  A.g = JR.out;
  A.phi = phi;
  A.phi.tab = (const double*)(D + o_tab);
  A.y = y_dev ? y : (const double*)(D + o_y);
  A.re = re_dev ? re : (double*)(D + o_re);
  A.im = im ? (im_dev ? im : (double*)(D + o_im)) : nullptr;
  A.status = (int*)(D + o_st);
  EZ_CUDA(launch_epstein_nd(A, threads, smem, stream));
  ++t_launches;
  if (!re_dev) EZ_CUDA(cudaMemcpyAsync(re, D + o_re, sizeof(double) * m, cudaMemcpyDeviceToHost, stream));
  if (im && !im_dev) EZ_CUDA(cudaMemcpyAsync(im, D + o_im, sizeof(double) * m, cudaMemcpyDeviceToHost, stream));
  EZ_CUDA(cudaMemcpyAsync(Hs + h_cnt, D + o_st, sizeof(int), cudaMemcpyDeviceToHost, stream));
  EZ_CUDA(cudaStreamSynchronize(stream));
  int status;
  std::memcpy(&status, Hs + h_cnt, sizeof status);
  if (status) return fail(EZ_EDOMAIN, "some y lie in the reciprocal lattice with nu <= d (pole)");
  return EZ_OK;
}

extern "C" int ez_epstein_zeta(ez_lattice L, double nu, const double* x, const double* y, size_t m, double* re,
                               double* im, int prec, void* stream_) {
  cudaStream_t stream = (cudaStream_t)stream_;
  if (!L || !x || (m && (!y || !re))) return fail(EZ_EINVAL, "NULL argument");
  if (m == 0) return EZ_OK;
  if (m > (size_t)1 << 31) return fail(EZ_EINVAL, "m too large");
  if (prec != EZ_FP64 && prec != EZ_MIXED) return fail(EZ_EINVAL, "prec = %d", prec);
  if (prec == EZ_MIXED) return fail(EZ_EUNSUPPORTED, "mixed precision not built yet");
  if (!std::isfinite(nu)) return fail(EZ_EINVAL, "exponent %g is not finite", nu);
  if (nu <= 0.0 && is_integer(0.5 * nu)) return fail(EZ_EDOMAIN, "exponent %g is a pole of Gamma(nu/2)", nu);
  int rc = init_constants();
  if (rc) return rc;
  if (L->d > kMaxD) return epstein_nd(L, nu, x, y, m, re, im, stream);
  const int d = L->d;
  ez_sum_spec s;
  std::memset(&s, 0, sizeof s);
  s.n_distinct = 1;
  s.nu[0] = nu;
  s.n_prod = 1;
  s.expo[0][0] = 1;
  ez_quadrature q;
  ez_quadrature_default(&q);
  q.n_u = 1;
  q.n_v = 1;
  q.u_rule = 1;
  q.lambda = std::pow(L->V, 1.0 / d);  // per-thread real-space box: keep it small
  Plan p;
  rc = make_plan(L, s, q, p);
  if (rc) return rc;
  // box around round(A^{-1} x)
  double xt[3] = {0, 0, 0};
  int mx[3] = {0, 0, 0};
  bool x_in = true;
  for (int i = 0; i < d; ++i) {
    double v = 0.0;
    for (int j = 0; j < d; ++j) v += L->Ai[i * d + j] * x[j];
    xt[i] = v;
    mx[i] = (int)std::lrint(v);
    if (std::fabs(v - mx[i]) > 1e-12) x_in = false;
  }
  p.cells = 1;
  for (int i = 0; i < 3; ++i) {
    if (i < d) {
      double rn = 0.0;
      for (int j = 0; j < d; ++j) rn += L->Ai[i * d + j] * L->Ai[i * d + j];
      p.M[i] = (int)std::ceil(p.r_real * std::sqrt(rn) + 0.5 + 1e-9);
      if (p.M[i] > 24) return fail(EZ_EINVAL, "real-space box too large");
    }
    p.box[i] = 2 * p.M[i] + 1;
    p.cells *= p.box[i];
  }
  const bool y_dev = is_device_ptr(y), re_dev = is_device_ptr(re), im_dev = im && is_device_ptr(im);
  Layout dl, hl;
  const size_t o_req = dl.take(sizeof(ReqDesc)), h_req = hl.take(sizeof(ReqDesc));
  const size_t o_rj = dl.take(sizeof(RecipJob)), h_rj = hl.take(sizeof(RecipJob));
  const size_t o_gj = dl.take(sizeof(GboxJob)), h_gj = hl.take(sizeof(GboxJob));
  const size_t o_pj = dl.take(sizeof(PhiJob)), h_pj = hl.take(sizeof(PhiJob));
  const size_t o_rec = dl.take(sizeof(G4) * p.rcap);
  const size_t o_recf = dl.take(sizeof(float4) * p.rcap);
  const size_t o_gbox = dl.take(sizeof(double) * p.cells);
  const size_t o_tab = dl.take(sizeof(double) * kRec * p.phi[0].n_int);
  const size_t o_st = dl.take(sizeof(int));
  const size_t o_y = y_dev ? 0 : dl.take(sizeof(double) * m * d);
  const size_t o_re = re_dev ? 0 : dl.take(sizeof(double) * m);
  const size_t o_im = (!im || im_dev) ? 0 : dl.take(sizeof(double) * m);
  std::lock_guard<std::mutex> lock(g_arena.mu);
  rc = arena_reserve(dl.off, hl.off);
  if (rc) return rc;
  char* D = g_arena.d;
  char* Hs = g_arena.h;
  ReqDesc& R = *(ReqDesc*)(Hs + h_req);
  std::memset(&R, 0, sizeof R);
  R.d = d;
  R.n_distinct = 1;
  R.nu[0] = nu;
  std::memcpy(R.A, L->A, sizeof R.A);
  std::memcpy(R.AiT, L->AiT, sizeof R.AiT);
  for (int i = 0; i < 9; ++i) R.AiTs[i] = std::sqrt(kPi) * p.lam * L->AiT[i];  // scaled units
  R.lam = p.lam;
  for (int i = 0; i < 3; ++i) {
    R.M[i] = p.M[i];
    R.box[i] = p.box[i];
  }
  R.rec = (const G4*)(D + o_rec);
  R.gbox = (const double*)(D + o_gbox);
  RecipJob& RJ = *(RecipJob*)(Hs + h_rj);
  RJ.req = 0;
  for (int i = 0; i < 3; ++i) {
    RJ.lo[i] = p.rlo[i];
    RJ.ext[i] = p.rext[i];
  }
  RJ.R2 = kPi * p.lam * p.lam * p.R2enum;
  RJ.cap = (int)p.rcap;
  RJ.out = (G4*)(D + o_rec);
  RJ.outf = (float4*)(D + o_recf);
  RJ.outlo = nullptr;
  RJ.tmp = nullptr;
  GboxJob& GJ = *(GboxJob*)(Hs + h_gj);
  std::memset(&GJ, 0, sizeof GJ);
  GJ.req = 0;
  for (int i = 0; i < d; ++i) {
    GJ.x[i] = x[i];
    GJ.mx[i] = mx[i];
  }
  GJ.x_in_lattice = x_in ? 1 : 0;
  GJ.R2 = p.r_real * p.r_real;
  GJ.out = (double*)(D + o_gbox);
  PhiJob& PJ = *(PhiJob*)(Hs + h_pj);
  PJ.a = p.phi[0].a;
  PJ.c_lam = 1.0;  // the table in t
  PJ.t_geo_end = p.phi[0].t_geo_end;
  PJ.n_int = p.phi[0].n_int;
  PJ.out = (double*)(D + o_tab);
  PJ.outf = nullptr;
  PJ.outff = nullptr;
  EZ_CUDA(cudaMemcpyAsync(D, Hs, hl.off, cudaMemcpyHostToDevice, stream));
  EZ_CUDA(cudaMemsetAsync(D + o_st, 0, sizeof(int), stream));
  if (!y_dev) EZ_CUDA(cudaMemcpyAsync(D + o_y, y, sizeof(double) * m * d, cudaMemcpyHostToDevice, stream));
  enum_recip_kernel<<<1, 512, 0, stream>>>((ReqDesc*)(D + o_req), (const RecipJob*)(D + o_rj));
  EZ_LAUNCHED();
  gbox_kernel<<<dim3((unsigned)((p.cells + 255) / 256), 1), 256, 0, stream>>>((const ReqDesc*)(D + o_req),
                                                                              (const GboxJob*)(D + o_gj), 1);
  EZ_LAUNCHED();
  phitab_kernel<<<dim3((p.phi[0].n_int + kPhiIv - 1) / kPhiIv, 1), kPhiIv * kNC, 0, stream>>>((const PhiJob*)(D + o_pj));
  EZ_LAUNCHED();
  EpsteinArgs A;
  std::memset(&A, 0, sizeof A);
  A.d = d;
  A.m = (int)m;
  A.nu = nu;
  A.pref = std::pow(kPi, 0.5 * nu) / (std::tgamma(0.5 * nu) * std::pow(p.lam, nu));
  A.vol_fac = std::pow(p.lam, d) / L->V;
  A.c_lam = 1.0;
  A.lam = p.lam;
  A.R2_recip = kPi * p.lam * p.lam * p.r_recip * p.r_recip;
  A.two_over_nu = 2.0 / nu;
  std::memcpy(A.A, L->A, sizeof A.A);
  // reciprocal space in scaled units s = sqrt(pi) lam: y~ = s A^{-T} y_reduced, and x / s in the
  // phases x.(g + y) = (x / s).(g~ + y~)
  for (int i = 0; i < 9; ++i) A.AiT[i] = std::sqrt(kPi) * p.lam * L->AiT[i];
  std::memcpy(A.At, L->At, sizeof A.At);
  for (int i = 0; i < d; ++i) {
    A.x[i] = x[i] / (std::sqrt(kPi) * p.lam);
    A.xt[i] = xt[i];
    A.mx[i] = mx[i];
  }
  A.x_in_lattice = x_in ? 1 : 0;
  for (int i = 0; i < 3; ++i) {
    A.M[i] = p.M[i];
    A.box[i] = p.box[i];
  }
  A.gbox = (const double*)(D + o_gbox);
  A.rq = (const ReqDesc*)(D + o_req);
  A.phi = p.phi[0];
  A.phi.c_lam = A.c_lam;
  A.phi.tab = (const double*)(D + o_tab);
  A.c_lam_f = (float)A.c_lam;
  A.R2f = (float)A.R2_recip;
  A.y = y_dev ? y : (const double*)(D + o_y);
  A.re = re_dev ? re : (double*)(D + o_re);
  A.im = im ? (im_dev ? im : (double*)(D + o_im)) : nullptr;
  A.status = (int*)(D + o_st);
  epstein_kernel<<<(unsigned)((m + 127) / 128), 128, 0, stream>>>(A);
  EZ_LAUNCHED();
  if (!re_dev) EZ_CUDA(cudaMemcpyAsync(re, D + o_re, sizeof(double) * m, cudaMemcpyDeviceToHost, stream));
  if (im && !im_dev) EZ_CUDA(cudaMemcpyAsync(im, D + o_im, sizeof(double) * m, cudaMemcpyDeviceToHost, stream));
  int status = 0;
  EZ_CUDA(cudaMemcpyAsync(&status, D + o_st, sizeof(int), cudaMemcpyDeviceToHost, stream));
  EZ_CUDA(cudaStreamSynchronize(stream));
  if (status) return fail(EZ_EDOMAIN, "some y lie in the reciprocal lattice with nu <= d (pole)");
  return EZ_OK;
}

// ---------------------------------------------------------------------------
// Epstein zeta with a static scratch area (no allocation at all).
//
// Some callers cannot allocate device memory at the moment they need a value:
// code running inside an allocator or a memory-pool callback, real-time threads
// that must not enter the driver's allocator (cudaMalloc can synchronise the
// device and take locks), and processes whose device memory is fully reserved
// by another framework.  This entry point computes what ez_epstein_zeta computes
// but keeps every piece of scratch (descriptors, reciprocal-lattice list,
// real-space box, Phi table, status flag) in the file-scope array below, which
// every GPU that loads this library holds until the process exits.
// ---------------------------------------------------------------------------
namespace {
constexpr size_t kStaticScratchBytes = 256 * 1024;
}  // namespace

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

namespace {
std::mutex g_static_mu;
void* g_static_addr[64] = {nullptr};  // device address of g_static_scratch, per device ordinal

// Resolves the device address of the static scratch on the current device (first call
// per device only).  In host code the symbol is a host-side stand-in, never a device address.
int static_scratch_address(void** out) {
  int dev = 0;
  EZ_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(EZ_EINVAL, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
      return fail(EZ_ECUDA, "cudaGetSymbolAddress(static scratch): %s", cudaGetErrorString(e));
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return EZ_OK;
}
}  // namespace

extern "C" int ez_epstein_zeta_static(ez_lattice L, double nu, const double* x, const double* y, size_t m,
                                      double* re, double* im, void* stream_) {
  cudaStream_t stream = (cudaStream_t)stream_;
  if (!L || !x || (m && (!y || !re))) return fail(EZ_EINVAL, "NULL argument");
  if (m == 0) return EZ_OK;
  if (m > (size_t)1 << 31) return fail(EZ_EINVAL, "m too large");
  if (!is_device_ptr(y) || !is_device_ptr(re) || (im && !is_device_ptr(im)))
    return fail(EZ_EINVAL, "ez_epstein_zeta_static takes device buffers for y, re and im "
                           "(host buffers would need staging memory)");
  if (L->d > kMaxD) return fail(EZ_EUNSUPPORTED, "ez_epstein_zeta_static: d = %d > %d (ez_epstein_zeta takes it)", L->d, kMaxD);
  if (!std::isfinite(nu)) return fail(EZ_EINVAL, "exponent %g is not finite", nu);
  if (nu <= 0.0 && is_integer(0.5 * nu)) return fail(EZ_EDOMAIN, "exponent %g is a pole of Gamma(nu/2)", nu);
  int rc = init_constants();
  if (rc) return rc;
  const int d = L->d;
  ez_sum_spec s;
  std::memset(&s, 0, sizeof s);
  s.n_distinct = 1;
  s.nu[0] = nu;
  s.n_prod = 1;
  s.expo[0][0] = 1;
  ez_quadrature q;
  ez_quadrature_default(&q);
  q.n_u = 1;
  q.n_v = 1;
  q.u_rule = 1;
  q.lambda = std::pow(L->V, 1.0 / d);  // per-thread real-space box: keep it small
  Plan p;
  rc = make_plan(L, s, q, p);
  if (rc) return rc;
  double xt[3] = {0, 0, 0};
  int mx[3] = {0, 0, 0};
  bool x_in = true;
  for (int i = 0; i < d; ++i) {
    double v = 0.0;
    for (int j = 0; j < d; ++j) v += L->Ai[i * d + j] * x[j];
    xt[i] = v;
    mx[i] = (int)std::lrint(v);
    if (std::fabs(v - mx[i]) > 1e-12) x_in = false;
  }
  p.cells = 1;
  for (int i = 0; i < 3; ++i) {
    if (i < d) {
      double rn = 0.0;
      for (int j = 0; j < d; ++j) rn += L->Ai[i * d + j] * L->Ai[i * d + j];
      p.M[i] = (int)std::ceil(p.r_real * std::sqrt(rn) + 0.5 + 1e-9);
      if (p.M[i] > 24) return fail(EZ_EINVAL, "real-space box too large");
    }
    p.box[i] = 2 * p.M[i] + 1;
    p.cells *= p.box[i];
  }
  Layout dl;
  const size_t o_req = dl.take(sizeof(ReqDesc));
  const size_t o_rj = dl.take(sizeof(RecipJob));
  const size_t o_gj = dl.take(sizeof(GboxJob));
  const size_t o_pj = dl.take(sizeof(PhiJob));
  const size_t o_rec = dl.take(sizeof(G4) * p.rcap);
  const size_t o_recf = dl.take(sizeof(float4) * p.rcap);
  const size_t o_gbox = dl.take(sizeof(double) * p.cells);
  const size_t o_tab = dl.take(sizeof(double) * kRec * p.phi[0].n_int);
  const size_t o_st = dl.take(sizeof(int));
  if (dl.off > kStaticScratchBytes)
    return fail(EZ_EINVAL, "this lattice and exponent need %zu bytes of scratch; the static area of "
                           "ez_epstein_zeta_static holds %zu bytes (use ez_epstein_zeta)",
                dl.off, kStaticScratchBytes);
  void* base = nullptr;
  rc = static_scratch_address(&base);
  if (rc) return rc;
  char* D = (char*)base;
  // descriptors on the host stack, copied into the static area (pageable copies are
  // staged by the driver before cudaMemcpyAsync returns)
  ReqDesc R;
  std::memset(&R, 0, sizeof R);
  R.d = d;
  R.n_distinct = 1;
  R.nu[0] = nu;
  std::memcpy(R.A, L->A, sizeof R.A);
  std::memcpy(R.AiT, L->AiT, sizeof R.AiT);
  for (int i = 0; i < 9; ++i) R.AiTs[i] = std::sqrt(kPi) * p.lam * L->AiT[i];  // scaled units
  R.lam = p.lam;
  for (int i = 0; i < 3; ++i) {
    R.M[i] = p.M[i];
    R.box[i] = p.box[i];
  }
  R.rec = (const G4*)(D + o_rec);
  R.gbox = (const double*)(D + o_gbox);
  RecipJob RJ;
  std::memset(&RJ, 0, sizeof RJ);
  RJ.req = 0;
  for (int i = 0; i < 3; ++i) {
    RJ.lo[i] = p.rlo[i];
    RJ.ext[i] = p.rext[i];
  }
  RJ.R2 = kPi * p.lam * p.lam * p.R2enum;
  RJ.cap = (int)p.rcap;
  RJ.out = (G4*)(D + o_rec);
  RJ.outf = (float4*)(D + o_recf);
  GboxJob GJ;
  std::memset(&GJ, 0, sizeof GJ);
  GJ.req = 0;
  for (int i = 0; i < d; ++i) {
    GJ.x[i] = x[i];
    GJ.mx[i] = mx[i];
  }
  GJ.x_in_lattice = x_in ? 1 : 0;
  GJ.R2 = p.r_real * p.r_real;
  GJ.out = (double*)(D + o_gbox);
  PhiJob PJ;
  std::memset(&PJ, 0, sizeof PJ);
  PJ.a = p.phi[0].a;
  PJ.c_lam = 1.0;  // the table in t
  PJ.t_geo_end = p.phi[0].t_geo_end;
  PJ.n_int = p.phi[0].n_int;
  PJ.out = (double*)(D + o_tab);
  EZ_CUDA(cudaMemcpyAsync(D + o_req, &R, sizeof R, cudaMemcpyHostToDevice, stream));
  EZ_CUDA(cudaMemcpyAsync(D + o_rj, &RJ, sizeof RJ, cudaMemcpyHostToDevice, stream));
  EZ_CUDA(cudaMemcpyAsync(D + o_gj, &GJ, sizeof GJ, cudaMemcpyHostToDevice, stream));
  EZ_CUDA(cudaMemcpyAsync(D + o_pj, &PJ, sizeof PJ, cudaMemcpyHostToDevice, stream));
  EZ_CUDA(cudaMemsetAsync(D + o_st, 0, sizeof(int), stream));  // the pole flag must start at zero
  enum_recip_kernel<<<1, 512, 0, stream>>>((ReqDesc*)(D + o_req), (const RecipJob*)(D + o_rj));
  EZ_LAUNCHED();
  gbox_kernel<<<dim3((unsigned)((p.cells + 255) / 256), 1), 256, 0, stream>>>((const ReqDesc*)(D + o_req),
                                                                              (const GboxJob*)(D + o_gj), 1);
  EZ_LAUNCHED();
  phitab_kernel<<<dim3((p.phi[0].n_int + kPhiIv - 1) / kPhiIv, 1), kPhiIv * kNC, 0, stream>>>((const PhiJob*)(D + o_pj));
  EZ_LAUNCHED();
  EpsteinArgs A;
  std::memset(&A, 0, sizeof A);
  A.d = d;
  A.m = (int)m;
  A.nu = nu;
  A.pref = std::pow(kPi, 0.5 * nu) / (std::tgamma(0.5 * nu) * std::pow(p.lam, nu));
  A.vol_fac = std::pow(p.lam, d) / L->V;
  A.c_lam = 1.0;
  A.lam = p.lam;
  A.R2_recip = kPi * p.lam * p.lam * p.r_recip * p.r_recip;
  A.two_over_nu = 2.0 / nu;
  std::memcpy(A.A, L->A, sizeof A.A);
  // reciprocal space in scaled units s = sqrt(pi) lam: y~ = s A^{-T} y_reduced, and x / s in the
  // phases x.(g + y) = (x / s).(g~ + y~)
  for (int i = 0; i < 9; ++i) A.AiT[i] = std::sqrt(kPi) * p.lam * L->AiT[i];
  std::memcpy(A.At, L->At, sizeof A.At);
  for (int i = 0; i < d; ++i) {
    A.x[i] = x[i] / (std::sqrt(kPi) * p.lam);
    A.xt[i] = xt[i];
    A.mx[i] = mx[i];
  }
  A.x_in_lattice = x_in ? 1 : 0;
  for (int i = 0; i < 3; ++i) {
    A.M[i] = p.M[i];
    A.box[i] = p.box[i];
  }
  A.gbox = (const double*)(D + o_gbox);
  A.rq = (const ReqDesc*)(D + o_req);
  A.phi = p.phi[0];
  A.phi.c_lam = A.c_lam;
  A.phi.tab = (const double*)(D + o_tab);
  A.c_lam_f = (float)A.c_lam;
  A.R2f = (float)A.R2_recip;
  A.y = y;
  A.re = re;
  A.im = im;
  A.status = (int*)(D + o_st);
  epstein_kernel<<<(unsigned)((m + 127) / 128), 128, 0, stream>>>(A);
  EZ_LAUNCHED();
  int status = 0;
  EZ_CUDA(cudaMemcpyAsync(&status, D + o_st, sizeof(int), cudaMemcpyDeviceToHost, stream));
  EZ_CUDA(cudaStreamSynchronize(stream));
  if (status) return fail(EZ_EDOMAIN, "some y lie in the reciprocal lattice with nu <= d (pole)");
  return EZ_OK;
}

// ---------------------------------------------------------------------------
// Serving: continuous batching (ez_server_*, see ezeta.h).
// ---------------------------------------------------------------------------
#include <condition_variable>
#include <deque>
#include <thread>
#include <unordered_set>

#include <time.h>

namespace {

double mono_now() {
  timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

struct SrvReq {
  unsigned long long ticket = 0, tag = 0;
  std::shared_ptr<ez_lattice_s> lat;  // stable address: the plans point at it
  ez_sum_spec spec;
  ez_quadrature quad;
  int flags = 0;
  Plan plan, plan_coarse;  // made by ez_server_submit on the submitting thread
  double t_submit = 0.0;
  size_t est_bytes = 0;  // device bytes of a tick holding this request alone
  int status = EZ_OK;    // planning error, reported as the result
};

struct Tick {
  bool busy = false;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  char* d = nullptr;   // device memory of the tick, stream-ordered from the server's pool
  size_t dbytes = 0;   // its size, counted against the budget until the tick completes
  char* h = nullptr;
  size_t hcap = 0;
  double* hout = nullptr;
  size_t hout_cap = 0;
  std::vector<SrvReq> reqs;
  std::vector<int> slot, slot_coarse;  // batch index of each request (and of its coarse rule, or -1)
  ez_batch_s batch;
  double t_start = 0.0;
  int error = EZ_OK;
};

}  // namespace

struct ez_server_s {
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<SrvReq> pending;
  std::deque<ez_result> done;
  std::unordered_set<unsigned long long> open;  // submitted and not yet completed
  size_t budget = 0;
  int n_streams = 1, max_batch = 1, max_pending = 1, flags = 0, device = 0;
  std::vector<Tick> ticks;
  std::thread worker;
  bool stop = false, exited = false;
  unsigned long long next_ticket = 1;
  ez_serve_stats st;
  int n_busy = 0;
  double busy_since = 0.0;
  cudaMemPool_t pool = nullptr;      // device memory of the ticks (stream-ordered, no device sync)
  std::vector<void*> retired_host;   // outgrown pinned staging, freed when the server is destroyed
  // resident Phi tables, one per order a, kMaxInt intervals: they depend on a alone
  // (tables in t), so every later tick reads them instead of building its own
  struct PhiRes {
    char* p = nullptr;
    size_t bytes = 0;
    cudaEvent_t ready = nullptr;  // after the phitab launch that filled it
  };
  std::map<double, PhiRes> phi_res;  // key: the order a
  size_t phi_res_bytes = 0;
};

namespace {

bool dryrun(const ez_server_s* S) { return (S->flags & EZ_SERVER_DRYRUN) != 0; }

size_t held_bytes(const ez_server_s* S) {
  size_t b = S->phi_res_bytes;
  for (const Tick& T : S->ticks) b += T.dbytes;
  return b;
}

void push_result(ez_server_s* S, const SrvReq& q, int status, const double* v, const double* vc, double t_start,
                 double t_done) {
  ez_result r;
  std::memset(&r, 0, sizeof r);
  r.ticket = q.ticket;
  r.tag = q.tag;
  r.status = status;
  for (int p = 0; p < EZ_MAX_PROD; ++p) {
    r.value[p] = v ? v[p] : std::nan("");
    r.err_est[p] = (v && vc) ? std::fabs(v[p] - vc[p]) : std::nan("");
  }
  r.t_submit = q.t_submit;
  r.t_start = t_start;
  r.t_done = t_done;
  S->done.push_back(r);
  S->open.erase(q.ticket);
  S->st.completed++;
  if (status != EZ_OK) S->st.failed++;
}

// grows a pinned host buffer geometrically; the outgrown one is kept until the server is
// destroyed (freeing pinned memory would synchronise the device under the running ticks)
template <typename P>
int grow_pinned(ez_server_s* S, P*& buf, size_t& cap, size_t need, const char* what) {
  if (need <= cap) return EZ_OK;
  const size_t ncap = std::max(need, 2 * cap);
  void* nb = nullptr;
  if (cudaMallocHost(&nb, ncap) != cudaSuccess) {
    cudaGetLastError();
    return fail(EZ_ENOMEM, "pinned %s of %zu bytes failed", what, ncap);
  }
  if (buf) S->retired_host.push_back((void*)buf);
  buf = (P*)nb;
  cap = ncap;
  return EZ_OK;
}

// launches one tick for T.reqs (called without the lock; only the worker touches T).  The
// plans come from ez_server_submit; a request with EZ_REQ_ERR_EST adds its coarse-rule plan.
// The tick's device memory comes from the server's pool in stream order and goes back to it
// in stream order after the results are copied out: nothing here synchronises the device.
int launch_tick(ez_server_s* S, Tick& T) {
  const int n = (int)T.reqs.size();
  T.batch = ez_batch_s();
  T.slot.assign(n, -1);
  T.slot_coarse.assign(n, -1);
  std::vector<Plan>& plans = T.batch.plans;
  for (int i = 0; i < n; ++i) {
    T.slot[i] = (int)plans.size();
    plans.push_back(T.reqs[i].plan);
    if (T.reqs[i].flags & EZ_REQ_ERR_EST) {
      T.slot_coarse[i] = (int)plans.size();
      plans.push_back(T.reqs[i].plan_coarse);
    }
  }
  T.batch.n_req = (int)plans.size();
  int rc = batch_layout(T.batch, false);
  if (rc) return rc;
  T.dbytes = T.batch.dbytes;
  if (dryrun(S)) return EZ_OK;  // account the memory a real tick would hold
  // resident Phi tables: read those of earlier ticks (after their fill, which may run on
  // another stream), build the missing ones into new resident tables in this tick
  std::vector<cudaEvent_t> waits;
  std::vector<double> fresh;  // resident tables created by this tick (dropped again if it fails)
  auto drop_fresh = [&]() {
    for (double key : fresh) {
      auto it = S->phi_res.find(key);
      if (it == S->phi_res.end()) continue;
      cudaFreeAsync(it->second.p, T.stream);
      if (it->second.ready) cudaEventDestroy(it->second.ready);
      S->phi_res_bytes -= it->second.bytes;
      S->phi_res.erase(it);
    }
    fresh.clear();
  };
  {
    ez_batch_s& B = T.batch;
    const int ng = B.n_phi;
    B.phi_ext.assign(ng, {nullptr, nullptr, nullptr});
    B.phi_fill.assign(ng, 0);
    B.phi_fill_nint.assign(ng, 0);
    B.phi_ready.clear();
    const size_t b64 = sizeof(double) * kRec * kMaxInt, b32 = sizeof(float) * kRec * kMaxInt,
                 bff = sizeof(float) * kRecFF * kMaxInt;
    for (int g = 0; g < ng; ++g) {
      const PhiInfo& P = phi_slot(B.plans[B.phi_master[g].first], B.phi_master[g].second);
      auto it = S->phi_res.find(P.a);
      if (it == S->phi_res.end()) {
        ez_server_s::PhiRes e;
        e.bytes = b64 + b32 + bff;
        if (cudaMallocFromPoolAsync((void**)&e.p, e.bytes, S->pool, T.stream) != cudaSuccess) {
          cudaGetLastError();
          drop_fresh();
          return fail(EZ_ENOMEM, "resident Phi table of %zu bytes failed", e.bytes);
        }
        if (cudaEventCreateWithFlags(&e.ready, cudaEventDisableTiming) != cudaSuccess) {
          cudaGetLastError();
          cudaFreeAsync(e.p, T.stream);
          drop_fresh();
          return fail(EZ_ECUDA, "event creation failed");
        }
        it = S->phi_res.emplace(P.a, e).first;
        fresh.push_back(P.a);
        S->phi_res_bytes += e.bytes;
        B.phi_fill[g] = 1;
        B.phi_fill_nint[g] = kMaxInt;
        B.phi_ready.push_back(e.ready);
        S->st.phi_tables_built++;
      } else {
        waits.push_back(it->second.ready);
        S->st.phi_tables_reused++;
      }
      char* base = it->second.p;
      B.phi_ext[g] = {base, base + b64, base + b64 + b32};
    }
    rc = batch_layout(B, false);  // without the resident tables
    if (rc) {
      drop_fresh();
      return rc;
    }
    T.dbytes = B.dbytes;
  }
  if (cudaMallocFromPoolAsync((void**)&T.d, T.batch.dbytes, S->pool, T.stream) != cudaSuccess) {
    cudaGetLastError();
    T.d = nullptr;
    T.dbytes = 0;
    drop_fresh();
    return fail(EZ_ENOMEM, "tick allocation of %zu bytes failed", T.batch.dbytes);
  }
  const size_t ob = sizeof(double) * EZ_MAX_PROD * T.batch.n_req;
  rc = grow_pinned(S, T.h, T.hcap, T.batch.hbytes, "staging");
  if (!rc) rc = grow_pinned(S, T.hout, T.hout_cap, ob, "output");
  if (!rc) {
    T.batch.d = T.d;
    T.batch.h = T.h;
    T.batch.owns = false;
    rc = batch_layout(T.batch, true);
  }
  if (!rc && cudaMemcpyAsync(T.d, T.h, T.batch.hbytes, cudaMemcpyHostToDevice, T.stream) != cudaSuccess)
    rc = fail(EZ_ECUDA, "staging upload failed");
  for (cudaEvent_t e : waits)
    if (!rc && cudaStreamWaitEvent(T.stream, e, 0) != cudaSuccess) rc = fail(EZ_ECUDA, "stream wait failed");
  if (!rc) rc = batch_launch(T.batch, T.stream);
  if (!rc && cudaMemcpyAsync(T.hout, T.d + T.batch.o_out, ob, cudaMemcpyDeviceToHost, T.stream) != cudaSuccess)
    rc = fail(EZ_ECUDA, "result download failed");
  cudaFreeAsync(T.d, T.stream);  // back to the pool once the stream has passed this point
  T.d = nullptr;
  if (rc) {
    cudaGetLastError();
    drop_fresh();
    return rc;
  }
  EZ_CUDA(cudaEventRecord(T.done, T.stream));
  return EZ_OK;
}

void server_loop(ez_server_s* S) {
  if (!dryrun(S)) cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lock(S->mu);
  while (true) {
    bool progressed = false;
    // completions
    for (Tick& T : S->ticks) {
      if (!T.busy) continue;
      bool fin = true;
      int err = T.error;
      if (!dryrun(S) && !err) {
        cudaError_t q = cudaEventQuery(T.done);
        if (q == cudaErrorNotReady) fin = false;
        else if (q != cudaSuccess) err = EZ_ECUDA;
      }
      if (!fin) continue;
      const double now = mono_now();
      const bool vals = !err && !dryrun(S);
      for (size_t i = 0; i < T.reqs.size(); ++i)
        push_result(S, T.reqs[i], err, vals ? T.hout + (size_t)T.slot[i] * EZ_MAX_PROD : nullptr,
                    vals && T.slot_coarse[i] >= 0 ? T.hout + (size_t)T.slot_coarse[i] * EZ_MAX_PROD : nullptr,
                    T.t_start, now);
      T.reqs.clear();
      T.dbytes = 0;
      T.busy = false;
      T.error = EZ_OK;
      if (--S->n_busy == 0) S->st.busy_seconds += now - S->busy_since;
      progressed = true;
    }
    if (progressed) S->cv_done.notify_all();
    if (S->stop && S->n_busy == 0) break;
    // admission: FIFO, as long as a stream is free and the device memory fits
    for (Tick& T : S->ticks) {
      if (T.busy || S->pending.empty() || S->stop) continue;
      size_t others = 0;
      for (const Tick& U : S->ticks)
        if (&U != &T) others += U.dbytes;
      const size_t room = S->budget > others ? S->budget - others : 0;
      size_t sum = 0;
      std::vector<SrvReq> take;
      while (!S->pending.empty() && (int)take.size() < S->max_batch) {
        SrvReq& q = S->pending.front();
        if (q.status != EZ_OK) {
          push_result(S, q, q.status, nullptr, nullptr, 0.0, mono_now());
          S->pending.pop_front();
          progressed = true;
          continue;
        }
        if (q.est_bytes > S->budget) {
          push_result(S, q, EZ_ENOMEM, nullptr, nullptr, 0.0, mono_now());
          S->pending.pop_front();
          progressed = true;
          continue;
        }
        if (sum + q.est_bytes > room && !take.empty()) break;
        if (sum + q.est_bytes > room) break;  // wait for other ticks to release memory
        sum += q.est_bytes;
        take.push_back(std::move(q));
        S->pending.pop_front();
      }
      if (take.empty()) continue;
      T.reqs = std::move(take);
      T.busy = true;
      T.t_start = mono_now();
      if (S->n_busy++ == 0) S->busy_since = T.t_start;
      S->st.ticks++;
      S->st.max_batch_seen = std::max<long long>(S->st.max_batch_seen, (long long)T.reqs.size());
      lock.unlock();
      const int rc = launch_tick(S, T);
      lock.lock();
      if (rc) T.error = rc;
      S->st.peak_device_bytes = std::max<long long>(S->st.peak_device_bytes, (long long)held_bytes(S));
      progressed = true;
    }
    if (progressed) S->cv_done.notify_all();
    if (!progressed) S->cv_work.wait_for(lock, std::chrono::microseconds(S->n_busy ? 20 : 2000));
  }
  S->exited = true;
  S->cv_done.notify_all();
}

}  // namespace

extern "C" int ez_server_create(size_t mem_budget_bytes, int n_streams, int max_batch, int max_pending, int flags,
                                ez_server* out) {
  if (!out) return fail(EZ_EINVAL, "NULL argument");
  if (mem_budget_bytes == 0 || n_streams < 1 || n_streams > 16 || max_batch < 1 || max_batch > 65536 ||
      max_pending < 1)
    return fail(EZ_EINVAL, "server limits: budget %zu, streams %d, batch %d, pending %d", mem_budget_bytes,
                n_streams, max_batch, max_pending);
  ez_server S = new ez_server_s();
  std::memset(&S->st, 0, sizeof S->st);
  S->budget = mem_budget_bytes;
  S->n_streams = n_streams;
  S->max_batch = max_batch;
  S->max_pending = max_pending;
  S->flags = flags;
  S->ticks.resize(n_streams);
  if (!dryrun(S)) {
    int rc = init_constants();
    if (rc) {
      delete S;
      return rc;
    }
    cudaGetDevice(&S->device);
    // a pool of its own: ticks allocate and free in stream order (no device synchronisation);
    // it keeps up to the budget for reuse, and never makes one stream wait for another to
    // reuse memory (only memory whose release the GPU has already passed is reused)
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = S->device;
    unsigned long long keep = mem_budget_bytes;
    int no = 0;
    if (cudaMemPoolCreate(&S->pool, &props) != cudaSuccess ||
        cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess ||
        cudaMemPoolSetAttribute(S->pool, cudaMemPoolReuseAllowInternalDependencies, &no) != cudaSuccess) {
      cudaGetLastError();
      S->exited = true;  // no worker yet
      ez_server_destroy(S, 0);
      return fail(EZ_ECUDA, "device memory pool creation failed");
    }
    for (Tick& T : S->ticks) {
      if (cudaStreamCreateWithFlags(&T.stream, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&T.done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        S->exited = true;  // no worker yet
        ez_server_destroy(S, 0);
        return fail(EZ_ECUDA, "stream/event creation failed");
      }
    }
  }
  S->worker = std::thread(server_loop, S);
  *out = S;
  return EZ_OK;
}

extern "C" int ez_server_submit(ez_server S, const ez_request* req, unsigned long long* ticket) {
  if (!S || !req) return fail(EZ_EINVAL, "NULL argument");
  SrvReq q;
  const int d = req->d;
  if (d < 1 || d > 3) return fail(EZ_EINVAL, "request d = %d", d);
  if (req->flags & ~EZ_REQ_ERR_EST) return fail(EZ_EINVAL, "request flags %d", req->flags);
  q.lat = std::make_shared<ez_lattice_s>();
  ez_lattice_s& L = *q.lat;
  std::memset(&L, 0, sizeof L);
  L.d = d;
  std::memcpy(L.A, req->A, sizeof(double) * d * d);
  if (!invert(d, L.A, L.Ai, &L.V)) return fail(EZ_EINVAL, "singular lattice matrix");
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      L.AiT[i * d + j] = L.Ai[j * d + i];
      L.At[i * d + j] = L.A[j * d + i];
    }
  q.spec = req->spec;
  q.quad = req->quad;
  q.tag = req->tag;
  q.flags = req->flags;
  {  // plan it here, on the submitting thread: validity, device footprint, and the plans the
     // worker launches (it never plans)
    int rc = make_plan(q.lat.get(), q.spec, q.quad, q.plan);
    ez_batch_s B;
    if (!rc) {
      B.n_req = 1;
      B.plans.assign(1, q.plan);
      if (q.flags & EZ_REQ_ERR_EST) {
        ez_quadrature qc = q.quad;
        qc.n_u = std::max(1, (q.quad.n_u + 1) / 2);
        qc.n_v = std::max(1, (q.quad.n_v + 1) / 2);
        rc = make_plan(q.lat.get(), q.spec, qc, q.plan_coarse);
        B.n_req = 2;
        B.plans.push_back(q.plan_coarse);
      }
    }
    if (!rc) rc = batch_layout(B, false);
    q.status = rc;
    q.est_bytes = rc ? 0 : B.dbytes;
  }
  std::lock_guard<std::mutex> lock(S->mu);
  if (S->stop) return fail(EZ_EINVAL, "server is shutting down");
  if ((int)S->pending.size() >= S->max_pending) return fail(EZ_EBUSY, "queue full (%d pending)", S->max_pending);
  q.ticket = S->next_ticket++;
  q.t_submit = mono_now();
  if (ticket) *ticket = q.ticket;
  S->open.insert(q.ticket);
  S->pending.push_back(std::move(q));
  S->st.submitted++;
  S->cv_work.notify_one();
  return EZ_OK;
}

extern "C" int ez_server_poll(ez_server S, ez_result* out, int max_results, int* n_out) {
  if (!S || (!out && max_results > 0)) return fail(EZ_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lock(S->mu);
  int n = 0;
  while (n < max_results && !S->done.empty()) {
    out[n++] = S->done.front();
    S->done.pop_front();
  }
  if (n_out) *n_out = n;
  return EZ_OK;
}

extern "C" int ez_server_wait(ez_server S, unsigned long long ticket, int timeout_ms, ez_result* out) {
  if (!S || !out) return fail(EZ_EINVAL, "NULL argument");
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(std::max(0, timeout_ms));
  std::unique_lock<std::mutex> lock(S->mu);
  while (true) {
    for (auto it = S->done.begin(); it != S->done.end(); ++it)
      if (it->ticket == ticket) {
        *out = *it;
        S->done.erase(it);
        return EZ_OK;
      }
    if (!S->open.count(ticket)) return fail(EZ_EINVAL, "unknown or already collected ticket %llu", ticket);
    if (S->cv_done.wait_until(lock, deadline) == std::cv_status::timeout) {
      for (auto it = S->done.begin(); it != S->done.end(); ++it)
        if (it->ticket == ticket) {
          *out = *it;
          S->done.erase(it);
          return EZ_OK;
        }
      return fail(EZ_ETIMEOUT, "ticket %llu not done after %d ms", ticket, timeout_ms);
    }
  }
}

extern "C" int ez_server_stats(ez_server S, ez_serve_stats* out) {
  if (!S || !out) return fail(EZ_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lock(S->mu);
  *out = S->st;
  if (S->n_busy) out->busy_seconds += mono_now() - S->busy_since;
  return EZ_OK;
}

extern "C" int ez_server_destroy(ez_server S, int timeout_ms) {
  if (!S) return EZ_OK;
  {
    std::unique_lock<std::mutex> lock(S->mu);
    S->stop = true;
    S->pending.clear();
    S->cv_work.notify_all();
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(std::max(0, timeout_ms));
    while (!S->exited)
      if (S->cv_done.wait_until(lock, deadline) == std::cv_status::timeout && !S->exited)
        return fail(EZ_ETIMEOUT, "server ticks still running after %d ms", timeout_ms);
  }
  if (S->worker.joinable()) S->worker.join();
  for (Tick& T : S->ticks)
    if (T.stream) cudaStreamSynchronize(T.stream);
  // the resident tables go back to the pool while the streams still exist
  cudaStream_t s0 = S->ticks.empty() ? nullptr : S->ticks[0].stream;
  for (auto& kv : S->phi_res) {
    if (kv.second.p && s0) cudaFreeAsync(kv.second.p, s0);
    if (kv.second.ready) cudaEventDestroy(kv.second.ready);
  }
  S->phi_res.clear();
  if (s0) cudaStreamSynchronize(s0);
  for (Tick& T : S->ticks) {
    if (T.h) cudaFreeHost(T.h);
    if (T.hout) cudaFreeHost(T.hout);
    if (T.done) cudaEventDestroy(T.done);
    if (T.stream) cudaStreamDestroy(T.stream);
  }
  for (void* p : S->retired_host) cudaFreeHost(p);
  if (S->pool) cudaMemPoolDestroy(S->pool);
  delete S;
  return EZ_OK;
}
