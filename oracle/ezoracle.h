/*
 * ezoracle.h -- plain FP64 CPU oracle for the Epstein zeta method of
 * "Epstein zeta method for many-body lattice sums" (Buchheit & Busse).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library.  It shares no
 * code, header, table or constant generator with the CUDA library.
 *
 * Conventions: lattice matrix A is row-major (A[i*d+j] = component i of basis
 * vector j), Lambda = A Z^d, reciprocal lattice A^{-T} Z^d (Def. "Lattices").
 * All arithmetic is IEEE double.
 */
#ifndef EZORACLE_H
#define EZORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define OR_MAXNU 8
#define OR_MAXPROD 4
#define OR_MAXELL 8
#define OR_MAXD 6 /* largest dimension of or_epstein_zeta_nd */

/* Phi_a(t) = t^{-a} Gamma(a,t) for real a, t >= 0; Phi_a(0) = -1/a (a < 0). */
double or_phi(double a, double t);
/* E_1(t), t > 0. */
double or_expint_e1(double t);
/* Gauss-Legendre rule with n nodes on [0,1] (ascending). */
void or_gauss_legendre01(int n, double* x, double* w);
/* Hadamard finite-part integral of u^{mu-1} log(pi u^2 w2)^m over (0, eps). */
double or_hadamard(double mu, int m, double eps, double w2);

/* Z_{Lambda,nu}(x, y) by the incomplete-gamma splitting with parameter lam and
 * real/reciprocal cutoffs |z - x| <= r_real, |g + y| <= r_recip.
 * Returns 0 on success, 2 on a pole (y in Lambda* with nu <= d, or Gamma(nu/2) pole). */
int or_epstein_zeta(int d, const double* A, double nu, const double* x, const double* y,
                    double lam, double r_real, double r_recip, double* re, double* im);

/* The same for any dimension 1 <= d <= OR_MAXD (A row-major d x d); its own linear algebra
 * (Gauss-Jordan) and lattice enumeration. */
int or_epstein_zeta_nd(int d, const double* A, double nu, const double* x, const double* y,
                       double lam, double r_real, double r_recip, double* re, double* im);

/* Regularised Z^reg_{Lambda,nu}(k) = Z(k) - s_hat_nu(k)/V at x = 0 (Sec. 3). */
int or_epstein_zeta_reg(int d, const double* A, double nu, const double* k, double lam,
                        double r_real, double r_recip, double* out);

/* s_hat_nu(k) of Sec. 3 (power or logarithmic singularity), not divided by V. */
double or_s_hat(int d, double nu, const double* k);

typedef struct {
  int d;
  double A[9];
  double lam, r_real, r_recip;
  int n_distinct;
  double nu[OR_MAXNU];
  int n_prod;
  int expo[OR_MAXPROD][OR_MAXNU]; /* product p = prod_j Z_{nu_j}^{expo[p][j]} */
  int u_rule;                     /* 1: GL on [0,1/2] (n_u nodes); 2: eps-split, n_u nodes per panel
                                     (no automatic choice: anything else is an error) */
  int n_u, n_v;
  double eps;
  int ell;
} or_problem;

/* Number of Duffy sectors d*2^(d-1) and far-field u nodes of a problem. */
int or_n_sectors(const or_problem* P);
int or_n_u_total(const or_problem* P);
/* u nodes (abscissae in (0,1/2)) and weights of the far-field u rule. */
int or_u_rule(const or_problem* P, double* u, double* w);

/* Lattice sums: out[p] for each product.  far_lines (n_sect*n_u_total*n_prod) and
 * near_lines (n_sect*n_prod) receive the per-line partial sums when non-NULL.
 * n_threads > 1 parallelises over lines (fixed-order final sum). */
int or_nbody(const or_problem* P, int n_threads, double* out, double* far_lines, double* near_lines);
/* One line: far line (sector, iu) for iu >= 0, near line of the sector for iu < 0. */
int or_nbody_line(const or_problem* P, int sector, int iu, double* out);
/* Integrand of product p at one Duffy node, without weights: prod Z(k).  Also returns k~. */
int or_nbody_node(const or_problem* P, int sector, double u, const double* v, double* f, double* kt);
/* Taylor coefficients C_{k,nu_j}(w), k=0..ell, of Z^reg along direction w (Sec. 3). */
int or_reg_taylor(const or_problem* P, int j, const double* w, double* C);

#ifdef __cplusplus
}
#endif
#endif
