// Internal definitions of the GB300 Epstein zeta library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/ezeta.h"

namespace ez {

constexpr double kPi = 3.141592653589793238462643383279502884;

// ---------------------------------------------------------------------------
// Tables of Phi_a(t) = t^{-a} Gamma(a,t) for the reciprocal-space hot loop.
// t in [kT0, t_hi]: piecewise polynomials in x = (t - t_mid)/h on kNGeo geometric
//   intervals [kT0 r^i, kT0 r^{i+1}] (r = kGeoR), then kNHalf intervals of width 1/2, then
//   unit-width intervals up to t_hi (beyond t ~ 45 Phi is below the table floor and the
//   records hold one coefficient: only their count matters there).  Record of an interval (kRec doubles, 16-byte aligned): the number n of
//   coefficients kept (4, 8, 12 or 16, an int in the first slot), s = c/h and
//   o = -t_mid/h so that x = fma(|q|^2, s, o) with t = c |q|^2, one pad slot, then
//   b_0 .. b_{kNC-1} (monomials in x; b_j = 0 for j >= n).  n is the shortest length whose Chebyshev
//   tail is below max(2^-53 max|Phi|, 1e-19) on the interval: 1 (a constant), 4, 8, 12 or 16.
//   The float-float copy (kRecFF floats: n, J, s hi/lo, m hi/lo, 0, 0, then (hi, lo) pairs)
//   also holds J (even, 2 <= J <= n): the coefficients j >= J sum to <= 2^-30 min|Phi| on the
//   interval and are evaluated in binary32.
// t < kT0: series of the entire part plus the singular term.
// t > t_hi: asymptotic expansion e^{-t}/t (1 + (a-1)/t + (a-1)(a-2)/t^2 + ...).
// ---------------------------------------------------------------------------
constexpr int kNC = 16;
constexpr int kRec = kNC + 4;
constexpr int kNGeo = 5;
constexpr double kT0 = 0.5;
constexpr double kGeoR = 1.4;
constexpr int kNSer = 16;  // t < 1/2: 0.5^16/16! ~ 7e-19
constexpr int kNHalf = 100;  // intervals of width 1/2 after the geometric ones
constexpr int kMaxInt = 420;  // intervals per table (t_hi <= ~366)
// Float-float table of the mixed form (kRecFF floats per interval, 16-byte aligned):
// int n (shortest length in {4, 8, 12, 16} with Chebyshev tail below 2^-47 max|Phi|), pad,
// s = c/h and m = t_mid/c as float-float pairs, two pads, then b_0 .. b_{kNC-1} as
// (hi, lo) pairs.  x = s (|q|^2 - m): |q|^2 and m lie within a factor 2 of each other on
// the interval, so the leading difference is exact (Sterbenz).
constexpr int kRecFF = 8 + 2 * kNC;

// reciprocal-space record: (G_0, G_1, G_2, |G|^2) with G = A^{-T} h
struct alignas(32) G4 {
  double x, y, z, w;
};

struct PhiInfo {
  double a;           // order
  double c_lam;       // t = c_lam |q|^2
  int log_m;          // a = -log_m (log case) or -1
  int two_a;          // 2a rounded (exact when half != 0)
  double gam;         // Gamma(a) (non-log) or (-1)^m/m! (log)
  double t_geo_end;   // kT0 * kGeoR^kNGeo
  double t_hi;        // end of the tabulated range
  float t_geo_end_f, t_hi_f;
  float t_mix_f;      // mixed form: terms with t >= t_mix_f are evaluated in binary32
  float t_mid_f;      // mixed form: t_mid_f <= t < t_mix_f: binary64 argument, binary32 polynomial
  float tail_p[8];    // mixed form, t >= t_mix_f: Phi_a(t) = e^{-t} t^{-1} sum_k tail_p[k] (t_mix_f/t)^k
  int n_int;          // number of intervals
  const double* tab;  // n_int * kRec doubles (device)
  const float* tabf;  // binary32 table (own polynomial lengths) for the mixed form (device)
  const float* tabff; // float-float table (n_int * kRecFF floats) for the mixed form (device)
  double ser[kNSer];  // entire part for t < kT0
  float a_f;             // a in binary32 (exact for the half-integer orders of integer exponents)
  int half;              // 2a is an integer: t^{-a} by square roots and integer powers, else exp/log
  // t < kT0: below ser_brk[i] the series needs only N = 4 + 2 i terms (i < 6; N = kNSer
  // above ser_brk[5]): the dropped terms sum to <= 2^-55 in absolute value.
  float ser_brk[6];
  float ser_brk_mix[6];  // the same for 2^-46 (the mixed form's binary64 order chain)
  int below1;   // a < 1: the mixed form's binary64 order chain takes its series
  int need_lt;  // a < 1 with a log term or a non-half-integer order: log t is needed
};
static_assert(sizeof(PhiInfo) % sizeof(double) == 0, "PhiInfo is copied to shared memory in doubles");

// ---------------------------------------------------------------------------
// One lattice sum as seen by the kernels (device resident).
// ---------------------------------------------------------------------------
constexpr int kMaxD = 3;    // lattice sums (Duffy nodes, near part, serving)
constexpr int kMaxDnd = 6;  // the Epstein zeta function alone (any dimension up to this)
constexpr int kMaxFactor = 64;
constexpr int kNearMaxDeg = 64;  // u^2 degree of products in the near part
constexpr int kNearPowE = 8;      // near part: powers C^r tabulated per ray up to this r
constexpr int kNearPowCache = 96; // ... in at most this many coefficients (else products factor by factor)
constexpr int kMaxEll = 8;       // largest Taylor order parameter ell of the near part
constexpr int kInvIntHalf = 256; // near part: table of 1/n for |n| <= kInvIntHalf
constexpr int kVChunkMin = 8;   // d = 3: fewest v2 rows per far-field block
constexpr int kMaxBoxM = 16;    // largest real-space box half-width M_i

struct ReqDesc {
  int d, nsect, n_ui, n_v, u_rule, n_distinct, n_prod, ell, prec;
  int expo[EZ_MAX_PROD][EZ_MAX_NU];
  double A[9], AiT[9];
  // Reciprocal space is stored in scaled units: every reciprocal vector (the list G, the node
  // k, the cutoff) is multiplied by s = sqrt(pi) lam, so that |G~ + k~|^2 is the argument t of
  // Phi itself.  The Phi tables then depend on the order a alone (shared by every sum).
  double AiTs[9];        // s A^{-T}: k~ = s A^{-T} k_reduced, G~ = s A^{-T} h
  double c_phys, inv_s;  // pi lam^2 = s^2 and 1/s (Taylor tensors are taken in physical k)
  double V, lam, c_lam, vol_fac, R2_recip, eps;  // c_lam = 1 (scaled units), R2_recip = (s r_recip)^2
  double nu[EZ_MAX_NU], pref[EZ_MAX_NU], two_over_nu[EZ_MAX_NU];
  double sig[EZ_MAX_NU];  // singular coefficient sigma_nu of s_hat
  int islog[EZ_MAX_NU];
  int near_int_mu;        // every nu_j is an integer: the Hadamard exponents mu + 2k are integers
  // real space: full box prod_i (2 M_i + 1), g = 0 outside the ball and at m = 0
  int M[3], box[3];
  int vchunk;          // d = 3: v2 rows per far-field block
  int m_hp[3];         // mixed form: real-space terms with |m_i| >= m_hp[i] are summed in binary32
  const double* gbox;  // [n_distinct][box0][box1][box2]
  const float2* gboxff; // the same as float-float (hi, lo), for the mixed form
  // d = 3: folded H(ma, mb) per line group G = j n_ui + iu in [hg_lo, hg_lo + groups), hslot
  // 16-byte entries per group: double2 (FP64 form, hbox) or float-float complex (hboxff)
  const double2* hbox;
  const float4* hboxff;
  int hslot, hg_lo;
  // reciprocal space: all h with |A^{-T} h| <= r_recip + max_BZ |k|
  int n_rec;
  const G4* rec;      // (G_0, G_1, G_2, |G|^2)
  const float4* recf; // the same in binary32, for the cutoff screen
  const float4* reclo; // G - (double)recf (binary32): recf + reclo is G as float-float
  float R2f, c_lam_f;
  float2 c_lam_ff;    // c_lam as float-float
  int order_chain;     // mixed form: nu_j = nu_0 + 2j (>= 3 exponents), so the reciprocal orders
                       // a_j = a_0 - j are linked by t Phi_{a+1} = a Phi_a + e^{-t}
  PhiInfo phi[EZ_MAX_NU];
  // quadrature
  const double* u_nodes;
  const double* u_w;
  const double* v_nodes;
  const double* v_w;
  const float2* v_ff;   // v nodes and weights as float-float, for the mixed form
  const float2* vw_ff;
  // float-float copies of the per-exponent constants, for the mixed form
  float2 pref_ff[EZ_MAX_NU], tov_ff[EZ_MAX_NU], vol_ff;
  double inv_eps;           // 1 / eps (near part)
  // d <= 2: powers e^{2 pi i m u v}, m = 0..phase_mp1-1, per (u node, v node); shared by every
  // sum of a batch with the same quadrature (the phases do not depend on the lattice)
  const double2* phase;
  const float4* phaseff;  // the same as float-float complex (re hi, re lo, im hi, im lo)
  int phase_mp1;
  // near part
  int n_alpha;            // multi-indices with |alpha| even <= 2 ell
  const int* alpha;       // [n_alpha][3]
  const int* alpha_off;   // start of |alpha| = 2k blocks, k = 0..ell+1
  const double* taylor;   // [n_distinct][n_alpha] : d^alpha Z^reg(0) / alpha!
  // integer exponents: eps^{mu'} J_m(mu') = sum_{i <= m} hadw[((mu' - hadw_lo) m1 + m) m1 + i] L^i
  // (m1 = hadw_m1); null otherwise (real exponents: the recurrence per ray)
  const double* hadw;
  int hadw_lo, hadw_m1;
  // d = 3: (log |w|^2, |w|^2, 1/|w|^2, |w|) of the scaled node direction
  // w = sigma^j(p1 v1, p2 v2, 1) mapped by A^{-T} (k = u w), index
  // (((j 2 + [p1 < 0]) 2 + [p2 < 0]) n_v + v2) n_v + v1: t, log t, 1/t and sqrt t of the
  // h = 0 term follow from u of the block (binary64)
  const double4* dirlw;
  // output slices
  int far_item0, n_far_items, near_item0, n_near_items;
  int line0;  // first line (far lines then near lines)
  unsigned long long* work;  // [2]: in-range reciprocal terms, sum of polynomial lengths
};

// Work item of a far-field or near-field launch.
struct Item {
  int req, sector, iu, chunk;
  long long seg;  // first output segment of this item
  __host__ __device__ long long chunk_seg() const { return seg; }
};

}  // namespace ez
