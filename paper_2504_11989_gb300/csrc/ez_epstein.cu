// Z_{Lambda,nu}(x, y) for many y (Def. "Epstein zeta function"), by the
// incomplete-gamma splitting with parameter lam:
//   Z = P_nu [ sum_{z != x} g(z) e^{-2 pi i y.z}
//            + lam^d/V sum_{g*} Phi_{(d-nu)/2}(pi lam^2 |g* + y|^2) e^{-2 pi i x.(g* + y)}
//            - [x in Lambda] (2/nu) e^{-2 pi i x.y} ],   g(z) = Phi_{nu/2}(pi |z - x|^2 / lam^2).
// y is first reduced modulo Lambda* (Z is periodic in y).  The real-space sum over the box
// m in round(A^{-1}x) + [-M, M]^d is contracted axis by axis with per-axis phase powers.
#include "ez_kernels.h"
#include "ez_phi.cuh"

namespace ez {

namespace {
constexpr int kMaxBox = 2 * 24 + 1;
__device__ __forceinline__ double2 cmul2(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
}  // namespace

__global__ void __launch_bounds__(128) epstein_kernel(EpsteinArgs P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.m) return;
  const int d = P.d;
  double y[3] = {0.0, 0.0, 0.0}, yt[3] = {0.0, 0.0, 0.0}, yr[3] = {0.0, 0.0, 0.0};
  for (int c = 0; c < d; ++c) y[c] = P.y[(size_t)i * d + c];
  for (int c = 0; c < d; ++c) {  // A^T y, reduced to [-1/2, 1/2]
    double s = 0.0;
    for (int q = 0; q < d; ++q) s = fma(P.At[c * d + q], y[q], s);
    yt[c] = s - rint(s);
  }
  for (int c = 0; c < d; ++c) {
    double s = 0.0;
    for (int q = 0; q < d; ++q) s = fma(P.AiT[c * d + q], yt[q], s);
    yr[c] = s;
  }
  // ---- real space: sum_m g(m) e^{-2 pi i yt.(m + mx)}
  double2 ph[3][kMaxBox];
  for (int c = 0; c < 3; ++c) {
    const int Mc = c < d ? P.M[c] : 0;
    double sn, cs;
    sincospi(-2.0 * yt[c], &sn, &cs);
    const double2 e1 = make_double2(cs, sn);
    double2 e = make_double2(1.0, 0.0);
    ph[c][Mc] = e;
    for (int m = 1; m <= Mc; ++m) {
      e = cmul2(e, e1);
      ph[c][Mc + m] = e;
      ph[c][Mc - m] = make_double2(e.x, -e.y);
    }
  }
  double sre = 0.0, sim = 0.0;
  const int b0 = P.box[0], b1 = d > 1 ? P.box[1] : 1, b2 = d > 2 ? P.box[2] : 1;
  for (int m0 = 0; m0 < b0; ++m0) {
    double r1 = 0.0, i1 = 0.0;
    for (int m1 = 0; m1 < b1; ++m1) {
      const double* g = P.gbox + ((size_t)m0 * b1 + m1) * b2;
      double r2 = 0.0, i2 = 0.0;
      for (int m2 = 0; m2 < b2; ++m2) {
        const double gv = g[m2];
        const double2 e = ph[2][m2];
        r2 = fma(gv, e.x, r2);
        i2 = fma(gv, e.y, i2);
      }
      const double2 e = ph[1][m1];
      r1 += r2 * e.x - i2 * e.y;
      i1 += r2 * e.y + i2 * e.x;
    }
    const double2 e = ph[0][m0];
    sre += r1 * e.x - i1 * e.y;
    sim += r1 * e.y + i1 * e.x;
  }
  {  // common factor e^{-2 pi i yt.mx}
    double s = 0.0;
    for (int c = 0; c < d; ++c) s = fma(yt[c], (double)P.mx[c], s);
    s -= rint(s);
    double sn, cs;
    sincospi(-2.0 * s, &sn, &cs);
    const double tr = sre * cs - sim * sn, ti = sre * sn + sim * cs;
    sre = tr;
    sim = ti;
  }
  // ---- reciprocal space: sum over |g* + yr| <= R of Phi * e^{-2 pi i x.(g* + yr)}
  double rre = 0.0, rim = 0.0;
  const ReqDesc* R = P.rq;
  const int nrec = R->n_rec;
  bool pole = false;
  for (int h = 0; h < nrec; ++h) {
    const G4 G = ldg_g4(R->rec + h);
    double q[3] = {G.x + yr[0], G.y + yr[1], G.z + yr[2]};
    double qq = 0.0;
    for (int c = 0; c < d; ++c) qq = fma(q[c], q[c], qq);
    if (qq > P.R2_recip) continue;
    double phi;
    if (qq == 0.0) {
      if (P.phi.a >= 0.0) {
        pole = true;
        continue;
      }
      phi = -1.0 / P.phi.a;
    } else {
      int nused;
      phi = phi_eval_qq(P.phi, qq, P.c_lam_f * (float)qq, nused);
    }
    if (P.x_in_lattice && P.xt[0] == 0.0 && P.xt[1] == 0.0 && P.xt[2] == 0.0) {
      rre += phi;
    } else {
      double xq = 0.0;
      for (int c = 0; c < d; ++c) xq = fma(P.x[c], q[c], xq);
      double sn, cs;
      sincospi(-2.0 * xq, &sn, &cs);
      rre = fma(phi, cs, rre);
      rim = fma(phi, sn, rim);
    }
  }
  double tre = sre + P.vol_fac * rre, tim = sim + P.vol_fac * rim;
  if (P.x_in_lattice) {
    double xy = 0.0;
    for (int c = 0; c < d; ++c) xy = fma(P.x[c], yr[c], xy);
    double sn, cs;
    sincospi(-2.0 * xy, &sn, &cs);
    tre -= P.two_over_nu * cs;
    tim -= P.two_over_nu * sn;
  }
  if (pole) {
    tre = tim = __longlong_as_double(0x7ff8000000000000LL);
    atomicOr(P.status, 1);
  }
  P.re[i] = P.pref * tre;
  if (P.im) P.im[i] = P.pref * tim;
}

}  // namespace ez
