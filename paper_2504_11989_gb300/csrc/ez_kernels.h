// Kernel entry points and setup job records of the Epstein zeta library.
#pragma once

#include "ez_internal.h"

namespace ez {

struct RecipJob {
  int req;
  int lo[3], ext[3];
  double R2;
  int cap;
  G4* out;
  float4* outf;
  float4* outlo;  // low parts of the float-float G (may be null)
  G4* tmp;        // non-null: enumerate into tmp; sort_recip_kernel then writes out/outf/outlo
};

struct GboxJob {
  int req;
  double x[3];  // centre (0 for the n-body path)
  int mx[3];    // integer offset of the box centre (round(A^{-1} x))
  int x_in_lattice;
  double R2;
  double* out;
  float2* outff;  // float-float copy (may be null)
  int use_tab;    // 1: g from the tables of the real-space orders in phi (c_lam = 1, argument t)
  PhiInfo phi[EZ_MAX_NU];
};

// d = 3 far field: H of the line groups [g_lo, g_hi) of one request (slot G - g_lo)
struct HboxJob {
  int req, g_lo, g_hi;
  double2* out;   // FP64 form
  float4* outff;  // mixed form (float-float complex); exactly one of out / outff is set
};

struct PhiJob {
  double a;
  double c_lam;
  double t_geo_end;
  int n_int;
  double* out;
  float* outf;
  float* outff;  // float-float table (may be null)
};


struct TaylorJob {
  int req, nu_index;
  double* phiG;   // [n_rec_cap][2 ell + 1]
  double rser[16];  // entire series of the regularised h = 0 term (lambda piece included)
  double* out;    // [n_alpha]
  double* part;   // first job of a request: real-space partial moments [n_chunk][n_alpha][n_distinct]
  int n_chunk;    // chunks of kTaylorCells cells of the half box
};
constexpr int kTaylorCells = 64;

struct PhaseJob {
  int n_ui, n_v, mp1;
  const double* u;
  const double* v;  // NULL for d = 1 (v = 1)
  double2* out;     // [n_ui][n_v][mp1]
  float4* outff;    // float-float copy (may be null)
};

struct EpsteinArgs {
  int d, m;
  double nu, pref, vol_fac, c_lam, lam, R2_recip, two_over_nu;
  double A[9], AiT[9], At[9];  // AiT scaled by s = sqrt(pi) lam (reciprocal vectors in scaled units)
  double x[3], xt[3];  // x / s (paired with scaled reciprocal vectors in the phases) and A^{-1} x
  int x_in_lattice;
  int M[3], box[3], mx[3];
  const double* gbox;
  int n_rec_cap;
  const ReqDesc* rq;  // for n_rec and the reciprocal list
  float c_lam_f, R2f;
  PhiInfo phi;
  const double* y;
  double* re;
  double* im;
  int* status;
};

__global__ void enum_recip_kernel(ReqDesc* reqs, const RecipJob* jobs);
__global__ void sort_recip_kernel(const ReqDesc* reqs, const RecipJob* jobs);
__global__ void gbox_kernel(const ReqDesc* reqs, const GboxJob* jobs, int n_jobs);
constexpr int kHboxColsHost = 32;  // hbox_kernel: columns per block (kHboxCols)
cudaError_t launch_hbox(bool mixed_any, bool f64_any, unsigned col_chunks, int n_req, const ReqDesc* reqs,
                        const HboxJob* jobs, cudaStream_t st);
__global__ void phitab_kernel(const PhiJob* jobs);
__global__ void taylor_kernel(const ReqDesc* reqs, const TaylorJob* jobs, int n_jobs);
__global__ void taylor_real_kernel(const ReqDesc* reqs, const TaylorJob* jobs, int n_jobs);
__global__ void phiseq_kernel(const ReqDesc* reqs, const TaylorJob* jobs, int n_jobs);

// far-field kernels (d = 1, 2, 3): binary64 or mixed form, at most ndm distinct exponents
inline int far_nd_class(int nd) { return nd <= 1 ? 1 : (nd <= 4 ? 4 : 8); }
cudaError_t launch_far(int d, bool mixed, int ndm, unsigned grid, size_t smem, cudaStream_t st,
                       const ReqDesc* reqs, const Item* items, double* seg);
cudaError_t far_set_smem_limits();
cudaError_t upload_inv_int();
__global__ void near_kernel(const ReqDesc* reqs, const Item* items, double* seg);
__global__ void lines_kernel(const ReqDesc* reqs, const int* line_req, const long long* line_seg0,
                             const int* line_nseg, int n_lines, const double* seg, double* lines);
__global__ void total_kernel(const ReqDesc* reqs, const long long* req_line0, const int* req_nlines,
                             int n_req, const long long* line_seg0, const int* line_nseg, const double* seg,
                             double* out);
__global__ void epstein_kernel(EpsteinArgs args);
__global__ void phase_kernel(const PhaseJob* jobs);
__global__ void dirlw_kernel(const ReqDesc* reqs);

// ---- the Epstein zeta function in any dimension d <= kMaxDnd ----
// Lattice points id in the box lo + [0, ext) with |M id - c|^2 <= R2, stored as rows along the
// last axis: one record per non-empty row, in lexicographic order of the row's prefix
// (id_0 .. id_{d-2}).  Record (int4): x = offset of the row's first cell, y = k0 | n << 16 (the
// row holds id_{d-1} = lo_{d-1} + k0 + [0, n)), z = prefix, 6 bits per axis (axis l at bit 6 l,
// index id_l - lo_l), w = the first prefix axis at which the row differs from the previous one.
constexpr int kNdMaxExt = 63;  // box extent per axis (6-bit prefix fields)
struct NdBallJob {
  int d;
  double M[kMaxDnd * kMaxDnd];  // z_i = sum_j M[i d + j] id_j
  double c[kMaxDnd];
  double R2;
  int lo[kMaxDnd], ext[kMaxDnd];
  long long n_prefix;  // prod_{l < d - 1} ext_l (1 for d = 1)
  int* row_k0;         // [n_prefix] scratch
  int* row_n;          // [n_prefix] scratch
  int4* rows;          // [n_prefix]: the non-empty rows
  int* counts;         // [2]: rows, cells
  long long cell_cap;  // cells the output holds (0: count only, no output)
  double a, pi_over_lam2;  // g = Phi_a(pi_over_lam2 |z - c|^2)
  int skip_center;         // the cell id == cid is left out (x in the lattice)
  int cid[kMaxDnd];
  double* out;             // [cell] g
};

struct NdEpsteinArgs {
  int d, m;
  double pref, vol_fac, R2_recip, two_over_nu;
  double At[kMaxDnd * kMaxDnd];  // A^T: reduced coordinates yt = A^T y
  double Rk[kMaxDnd * kMaxDnd];  // upper triangular, R^T R = B^T B with B = sqrt(pi) lam A^{-T}
  double xt[kMaxDnd];            // A^{-1} x
  int x_zero, x_in_lattice;
  int M[kMaxDnd], mx[kMaxDnd];   // real-space box mx - M + [0, 2 M]
  int phase_len;                 // per-thread phase entries in shared memory: sum_l (2 M_l + 1),
                                 // or sum_l (M_l + 1) with half_phases
  int half_phases;               // tables of the non-negative offsets only (large boxes)
  const int4* rows;
  const int* rcounts;  // [0]: real-space rows
  const double* g;
  PhiInfo phi;         // order (d - nu) / 2, argument t = pi lam^2 |g* + y|^2
  const double* y;
  double* re;
  double* im;
  int* status;
};
__global__ void nd_rows_kernel(const NdBallJob* job);
__global__ void nd_scan_kernel(const NdBallJob* job);
__global__ void nd_fill_kernel(const NdBallJob* job);
cudaError_t launch_epstein_nd(const NdEpsteinArgs& args, unsigned threads, size_t smem, cudaStream_t st);

size_t far_smem_bytes(int d, int n_distinct, const int* M, int n_v, int vchunk);
// Chebyshev -> monomial matrix (kNC x kNC), cosine table of the transform (kNC x kNC),
// Chebyshev points (kNC)
cudaError_t upload_cheb2mono(const double* host_matrix, const double* dct, const double* xk);
constexpr int kPhiIv = 8;  // phitab_kernel: intervals per block

}  // namespace ez
