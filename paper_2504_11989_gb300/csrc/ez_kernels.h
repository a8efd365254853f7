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
__global__ void hbox_kernel(const ReqDesc* reqs, const HboxJob* jobs);
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
                             int n_req, const double* lines, double* out);
__global__ void epstein_kernel(EpsteinArgs args);
__global__ void phase_kernel(const PhaseJob* jobs);

size_t far_smem_bytes(int d, int n_distinct, const int* M, int n_v, int vchunk);
// Chebyshev -> monomial matrix (kNC x kNC), cosine table of the transform (kNC x kNC),
// Chebyshev points (kNC)
cudaError_t upload_cheb2mono(const double* host_matrix, const double* dct, const double* xk);
constexpr int kPhiIv = 8;  // phitab_kernel: intervals per block

}  // namespace ez
