// Setup kernels: lattice-point tables, incomplete-gamma tables and Taylor
// tensors of Z^reg at the origin.  All of them run once per lattice sum.
#include "ez_ff.cuh"
#include "ez_kernels.h"
#include "ez_phi.cuh"

namespace ez {

// ---------------------------------------------------------------------------
// Reciprocal lattice points h with |A^{-T} h| <= R (box lo..hi), compacted in
// lexicographic order by one block (ordered prefix sums), written in scaled units
// G~ = s A^{-T} h as (G~_0, G~_1, G~_2, |G~|^2) (J.R2 is scaled too).  The count goes to
// req->n_rec.
// ---------------------------------------------------------------------------
__global__ void enum_recip_kernel(ReqDesc* reqs, const RecipJob* jobs) {
  const RecipJob J = jobs[blockIdx.x];
  ReqDesc* R = reqs + J.req;
  const int d = R->d;
  const long long total = (long long)J.ext[0] * J.ext[1] * J.ext[2];
  __shared__ int warp_sums[32];
  __shared__ int base;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (long long start = 0; start < total; start += blockDim.x) {
    long long idx = start + threadIdx.x;
    int keep = 0;
    double G[3] = {0, 0, 0}, G2 = 0.0;
    if (idx < total) {
      int h[3];
      long long r = idx;
      h[2] = (int)(r % J.ext[2]) + J.lo[2];
      r /= J.ext[2];
      h[1] = (int)(r % J.ext[1]) + J.lo[1];
      r /= J.ext[1];
      h[0] = (int)r + J.lo[0];
      for (int i = 0; i < d; ++i) {
        double s = 0.0;
        for (int k = 0; k < d; ++k) s = fma(R->AiTs[i * d + k], (double)h[k], s);
        G[i] = s;
        G2 = fma(s, s, G2);
      }
      keep = G2 <= J.R2;
    }
    unsigned ballot = __ballot_sync(0xffffffffu, keep);
    int before = __popc(ballot & ((1u << lane) - 1u));
    if (lane == 0) warp_sums[wid] = __popc(ballot);
    __syncthreads();
    int off = 0;
    for (int w = 0; w < wid; ++w) off += warp_sums[w];
    if (keep) {
      int pos = base + off + before;
      if (pos < J.cap && J.tmp) {
        J.tmp[pos] = G4{G[0], G[1], G[2], G2};
      } else if (pos < J.cap) {
        J.out[pos] = G4{G[0], G[1], G[2], G2};
        J.outf[pos] = make_float4((float)G[0], (float)G[1], (float)G[2], (float)G2);
        if (J.outlo)
          J.outlo[pos] = make_float4((float)(G[0] - (double)(float)G[0]), (float)(G[1] - (double)(float)G[1]),
                                     (float)(G[2] - (double)(float)G[2]), 0.0f);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int tot = 0;
      for (int w = 0; w < nw; ++w) tot += warp_sums[w];
      base += tot;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) R->n_rec = min(base, J.cap);
}

// ---------------------------------------------------------------------------
// Reciprocal points of a request in ascending order of |G|^2 (ties: enumeration order),
// by rank: one thread per point counts the points before it (the keys are staged in
// shared memory in chunks).  Writes the binary64 list and its float and float-float
// copies.  Grid: (points / blockDim, requests).
// ---------------------------------------------------------------------------
__global__ void sort_recip_kernel(const ReqDesc* reqs, const RecipJob* jobs) {
  const RecipJob J = jobs[blockIdx.y];
  if (!J.tmp) return;
  const int n = reqs[J.req].n_rec;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if ((long long)blockIdx.x * blockDim.x >= n) return;  // whole block past the end (uniform)
  constexpr int kChunk = 1024;
  __shared__ double key[kChunk];
  const G4 G = i < n ? J.tmp[i] : G4{0.0, 0.0, 0.0, 0.0};
  int rank = 0;
  for (int base = 0; base < n; base += kChunk) {
    const int m = min(kChunk, n - base);
    __syncthreads();
    for (int q = threadIdx.x; q < m; q += blockDim.x) key[q] = J.tmp[base + q].w;
    __syncthreads();
    if (i < n)
      for (int q = 0; q < m; ++q) {
        const double w = key[q];
        rank += (w < G.w || (w == G.w && base + q < i)) ? 1 : 0;
      }
  }
  if (i >= n) return;
  J.out[rank] = G;
  const float hx = (float)G.x, hy = (float)G.y, hz = (float)G.z;
  J.outf[rank] = make_float4(hx, hy, hz, (float)G.w);
  if (J.outlo)
    J.outlo[rank] = make_float4((float)(G.x - (double)hx), (float)(G.y - (double)hy), (float)(G.z - (double)hz), 0.0f);
}

// ---------------------------------------------------------------------------
// Real-space box: g_nu(m) = Phi_{nu/2}(pi |A m - x|^2 / lam^2) for 0 < |A m - x| <= R,
// zero elsewhere.  One thread per (box cell, distinct nu).
// ---------------------------------------------------------------------------
__global__ void gbox_kernel(const ReqDesc* reqs, const GboxJob* jobs, int n_jobs) {
  int jid = blockIdx.y;
  if (jid >= n_jobs) return;
  const GboxJob& J = jobs[jid];
  const ReqDesc* R = reqs + J.req;
  const int d = R->d;
  const long long cells = (long long)R->box[0] * R->box[1] * R->box[2];
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= cells * R->n_distinct) return;
  int jn = (int)(idx / cells);
  long long c = idx % cells;
  int m[3];
  m[2] = (int)(c % R->box[2]) - R->M[2];
  c /= R->box[2];
  m[1] = (int)(c % R->box[1]) - R->M[1];
  c /= R->box[1];
  m[0] = (int)c - R->M[0];
  double r2 = 0.0;
  bool center = true;
  for (int i = 0; i < d; ++i) {
    double s = -J.x[i];
    for (int k = 0; k < d; ++k) s = fma(R->A[i * d + k], (double)(m[k] + J.mx[k]), s);
    r2 = fma(s, s, r2);
    center &= (m[i] + J.mx[i]) == J.mx[i];
  }
  double g = 0.0;
  bool excluded = J.x_in_lattice ? center : false;
  if (!excluded && r2 <= J.R2 && r2 > 0.0) {
    const double t = kPi * r2 / (R->lam * R->lam);
    g = J.use_tab ? phi_eval(J.phi[jn], t) : phi_accurate(0.5 * R->nu[jn], t);
  }
  J.out[idx] = g;
  if (J.outff) {
    float hi, lo;
    ff_split(g, hi, lo);
    J.outff[idx] = make_float2(hi, lo);
  }
}

// ---------------------------------------------------------------------------
// Phi_a tables: kNC threads per (distinct a, interval), kPhiIv intervals per block.
// Chebyshev interpolation at the kNC Chebyshev points of the interval, then
// conversion to monomials in x in [-1, 1].  The cosine table of the transform, the
// Chebyshev points and the conversion matrix are uploaded once (constant memory) and
// staged in shared memory per block.
// ---------------------------------------------------------------------------
__constant__ double c_cheb2mono[kNC * kNC];  // [j][i]: coefficient of x^i in T_j(x)
__constant__ double c_dct[kNC * kNC];        // [k][q]: cos(pi k (q + 1/2) / kNC)
__constant__ double c_cheb_x[kNC];           // cos(pi (k + 1/2) / kNC)

cudaError_t upload_cheb2mono(const double* m, const double* dct, const double* xk) {
  cudaError_t e = cudaMemcpyToSymbol(c_cheb2mono, m, sizeof(double) * kNC * kNC);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_dct, dct, sizeof(double) * kNC * kNC);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_cheb_x, xk, sizeof(double) * kNC);
  return e;
}

// midpoint and half-width of interpolation interval iv (geometric, then unit width)
__device__ __forceinline__ void phi_interval_bounds(int iv, double t_geo_end, double& tm, double& h) {
  double lo, hi;
  if (iv < kNGeo) {
    lo = kT0 * pow(kGeoR, (double)iv);
    hi = lo * kGeoR;
  } else {
    const int k = iv - kNGeo;  // half-width intervals, then unit width
    lo = k < kNHalf ? t_geo_end + 0.5 * k : t_geo_end + 0.5 * kNHalf + (k - kNHalf);
    hi = lo + (k < kNHalf ? 0.5 : 1.0);
  }
  tm = 0.5 * (lo + hi);
  h = 0.5 * (hi - lo);
}

__global__ void __launch_bounds__(kPhiIv * kNC) phitab_kernel(const PhiJob* jobs) {
  const PhiJob J = jobs[blockIdx.y];
  __shared__ double sdct[kNC * kNC], sc2m[kNC * kNC];
  for (int i = threadIdx.x; i < kNC * kNC; i += blockDim.x) {
    sdct[i] = c_dct[i];
    sc2m[i] = c_cheb2mono[i];
  }
  const int sub = threadIdx.x / kNC, k = threadIdx.x - sub * kNC;
  const int iv = blockIdx.x * kPhiIv + sub;
  const bool live = iv < J.n_int;  // every thread reaches the barriers
  double tm = 0.0, h = 1.0;
  if (live) phi_interval_bounds(iv, J.t_geo_end, tm, h);
  __shared__ double fs[kPhiIv][kNC], cjs[kPhiIv][kNC], babs[kPhiIv][kNC];
  __shared__ int nkeep[kPhiIv], nkeep_f[kPhiIv], nkeep_ff[kPhiIv], jsplit[kPhiIv];
  double* f = fs[sub];
  double* cj = cjs[sub];
  f[k] = live ? phi_accurate(J.a, tm + h * c_cheb_x[k]) : 0.0;
  __syncthreads();
  double s = 0.0;
  for (int q = 0; q < kNC; ++q) s += f[q] * sdct[k * kNC + q];
  cj[k] = (k == 0 ? 1.0 : 2.0) * s / kNC;
  __syncthreads();
  if (k == 0) {
    // shortest length n in {4, 8, 12, 16} whose Chebyshev tail is below the tolerance:
    // binary64 table max(2^-53 max|Phi|, 1e-19), binary32 table 2^-26 max|Phi|
    double fm = 0.0;
    for (int q = 0; q < kNC; ++q) fm = fmax(fm, fabs(f[q]));
    const double tol = fmax(fm / 9007199254740992.0, 1e-19);  // 2^-53 max|Phi|
    const double tolf = fm / 67108864.0;
    const double tolff = fm / 140737488355328.0;  // 2^-47: float-float table
    int n = kNC, nf = kNC, nff = kNC;
    for (int cand = kNC - 4; cand >= 4; cand -= 4) {
      double tail = 0.0;
      for (int q = cand; q < kNC; ++q) tail += fabs(cj[q]);
      if (tail <= tol) n = cand;
      if (tail <= tolf) nf = cand;
      if (tail <= tolff) nff = cand;
    }
    // binary64 table: a single coefficient where the whole non-constant part is below the
    // tolerance (far tails, |Phi| < ~1e-19: one load instead of a Horner scheme)
    double tail1 = 0.0;
    for (int q = 1; q < kNC; ++q) tail1 += fabs(cj[q]);
    if (tail1 <= tol) n = 1;
    nkeep[sub] = n;
    nkeep_f[sub] = nf;
    nkeep_ff[sub] = nff;
  }
  __syncthreads();
  const int n = nkeep[sub], nf = nkeep_f[sub], nff = nkeep_ff[sub];
  double b = 0.0, bf = 0.0, bff = 0.0;
  for (int j = k; j < n; ++j) b += cj[j] * sc2m[j * kNC + k];
  for (int j = k; j < nf; ++j) bf += cj[j] * sc2m[j * kNC + k];
  for (int j = k; j < nff; ++j) bff += cj[j] * sc2m[j * kNC + k];
  // J (float-float records): the coefficients j >= J (x in [-1, 1]) sum to <= 2^-30
  // min|Phi| on the interval
  babs[sub][k] = fabs(bff);
  __syncthreads();
  if (k == 0) {
    double fmn = fabs(f[0]);
    for (int q = 1; q < kNC; ++q) fmn = fmin(fmn, fabs(f[q]));
    const double thr = ldexp(fmn, -30);
    int Jb = nff;
    double tl = 0.0;
    for (int Jc = nff - 2; Jc >= 2; Jc -= 2) {
      tl += babs[sub][Jc] + babs[sub][Jc + 1];
      if (tl > thr) break;
      Jb = Jc;
    }
    jsplit[sub] = Jb;
  }
  __syncthreads();
  if (!live) return;
  if (J.outff) {
    float* rff = J.outff + (size_t)iv * kRecFF;
    ff_split(bff, rff[8 + 2 * k], rff[9 + 2 * k]);
    if (k == 0) {
      reinterpret_cast<int*>(rff)[0] = nff;
      reinterpret_cast<int*>(rff)[1] = jsplit[sub];
      ff_split(J.c_lam / h, rff[2], rff[3]);
      ff_split(tm / J.c_lam, rff[4], rff[5]);
      rff[6] = rff[7] = 0.0f;
    }
  }
  double* r = J.out + (size_t)iv * kRec;
  r[4 + k] = b;
  if (J.outf) J.outf[(size_t)iv * kRec + 4 + k] = (float)bf;
  if (k == 0) {
    reinterpret_cast<int*>(r)[0] = n;
    reinterpret_cast<int*>(r)[1] = 0;
    r[1] = J.c_lam / h;
    r[2] = -tm / h;
    r[3] = 0.0;
    if (J.outf) {
      float* rf = J.outf + (size_t)iv * kRec;
      reinterpret_cast<int*>(rf)[0] = nf;
      rf[1] = (float)(J.c_lam / h);
      rf[2] = (float)(-tm / h);
      rf[3] = 0.0f;
    }
  }
}

// ---------------------------------------------------------------------------
// Taylor tensors of Z^reg_nu at k = 0:  D[alpha] = d^alpha Z^reg(0) / alpha!, |alpha|
// even <= 2 ell.  One thread per (request, distinct nu, alpha); serial sums in a
// fixed order (deterministic).  Terms (P_nu, c = pi lam^2):
//   real space   P_nu sum_m g(m) (-1)^K (2 pi)^{2K} z^alpha / alpha!,    2K = |alpha|
//   h != 0       P_nu lam^d/V sum_n (-1)^n Phi_{a+n}(c|G|^2) c^n / n! [k^alpha](2 G.k + |k|^2)^n
//   h = 0        P_nu lam^d/V r_K c^K K!/prod (alpha_i/2)!  (alpha all even)
//   constant     -P_nu 2/nu at alpha = 0.
// ---------------------------------------------------------------------------
__device__ double binom(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}
__device__ double factd(int n) {
  double r = 1.0;
  for (int i = 2; i <= n; ++i) r *= i;
  return r;
}

constexpr int kTaylorThreads = 128;

// Real-space moments of the Taylor tensors, per chunk of kTaylorCells cells of the half
// box after the centre cell (g(-m) = g(m) and the monomials are even): the block tabulates
// the powers z_i^e of its cells and their g values in shared memory, then thread alpha
// sums g(m) z^alpha over the chunk in cell order for every exponent.  One block per
// (chunk, request); the partial moments are added over the chunks in chunk order by
// taylor_kernel.
__global__ void __launch_bounds__(kTaylorThreads) taylor_real_kernel(const ReqDesc* reqs, const TaylorJob* jobs,
                                                                     int n_jobs) {
  const int jid = blockIdx.y;
  if (jid >= n_jobs) return;
  const TaylorJob J = jobs[jid];
  if (J.nu_index != 0 || (int)blockIdx.x >= J.n_chunk) return;
  const ReqDesc* R = reqs + J.req;
  const int d = R->d, nd = R->n_distinct, ne = 2 * R->ell + 1;
  __shared__ double pw[3][2 * kMaxEll + 1][kTaylorCells];
  __shared__ double gv[EZ_MAX_NU][kTaylorCells];
  const long long cells = (long long)R->box[0] * R->box[1] * R->box[2];
  const long long c0 = cells / 2 + 1 + (long long)blockIdx.x * kTaylorCells;
  const int nc = (int)min((long long)kTaylorCells, cells - c0);
  // the cells inside the ball (g != 0, the same for every exponent), compacted in cell order:
  // skipping g = 0 leaves every sum bitwise unchanged
  const int c = threadIdx.x, lane = c & 31, wid = c >> 5;
  __shared__ int s_live[kTaylorThreads / 32];
  double z[3] = {0.0, 0.0, 0.0};
  bool live = false;
  long long idx = 0;
  if (c < nc) {
    idx = c0 + c;
    live = R->gbox[idx] != 0.0;
  }
  const unsigned lm = __ballot_sync(0xffffffffu, live);
  if (lane == 0) s_live[wid] = __popc(lm);
  __syncthreads();
  int pos = __popc(lm & ((1u << lane) - 1u)), nlive = 0;
  for (int w = 0; w < kTaylorThreads / 32; ++w) {
    if (w < wid) pos += s_live[w];
    nlive += s_live[w];
  }
  if (live) {
    long long cc = idx;
    int m[3];
    m[2] = (int)(cc % R->box[2]) - R->M[2];
    cc /= R->box[2];
    m[1] = (int)(cc % R->box[1]) - R->M[1];
    cc /= R->box[1];
    m[0] = (int)cc - R->M[0];
    for (int i = 0; i < d; ++i) {
      double zi = 0.0;
      for (int k = 0; k < d; ++k) zi = fma(R->A[i * d + k], (double)m[k], zi);
      z[i] = zi;
    }
    for (int jn = 0; jn < nd; ++jn) gv[jn][pos] = R->gbox[(size_t)jn * cells + idx];
    for (int i = 0; i < 3; ++i) {
      double p = 1.0;
      for (int e = 0; e < ne; ++e) {
        pw[i][e][pos] = p;
        p *= z[i];
      }
    }
  }
  __syncthreads();
  for (int ia = threadIdx.x; ia < R->n_alpha; ia += blockDim.x) {
    const int* al = R->alpha + 3 * ia;
    const int a0 = al[0], a1 = al[1], a2 = al[2];
    double acc[EZ_MAX_NU];
#pragma unroll
    for (int jn = 0; jn < EZ_MAX_NU; ++jn) acc[jn] = 0.0;
    for (int q = 0; q < nlive; ++q) {
      const double mono = pw[0][a0][q] * pw[1][a1][q] * pw[2][a2][q];
#pragma unroll
      for (int jn = 0; jn < EZ_MAX_NU; ++jn)
        if (jn < nd) acc[jn] = fma(gv[jn][q], mono, acc[jn]);
    }
    double* o = J.part + ((size_t)blockIdx.x * R->n_alpha + ia) * nd;
    for (int jn = 0; jn < nd; ++jn) o[jn] = acc[jn];
  }
}

// One block of kTaylorThreads per (request, alpha), every distinct nu of the request at
// once (grid y runs over the request's Taylor jobs; the blocks of all but its first job
// return at once).  Real space: the half-box moments of taylor_real_kernel, doubled.
// Reciprocal space: the k^alpha coefficients of each lattice point serve every exponent.
// Fixed-order block reduction.
__global__ void __launch_bounds__(kTaylorThreads) taylor_kernel(const ReqDesc* reqs, const TaylorJob* jobs,
                                                                int n_jobs) {
  const int jid = blockIdx.y;
  if (jid >= n_jobs) return;
  const TaylorJob J0 = jobs[jid];
  if (J0.nu_index != 0) return;
  const ReqDesc* R = reqs + J0.req;
  const int ia = blockIdx.x;
  if (ia >= R->n_alpha) return;
  const int d = R->d, nd = R->n_distinct;
  const int* al = R->alpha + 3 * ia;
  const int alpha[3] = {al[0], al[1], al[2]};
  const int K2 = alpha[0] + alpha[1] + alpha[2];
  const int K = K2 / 2;
  const double afact = factd(alpha[0]) * factd(alpha[1]) * factd(alpha[2]);
  const double c = R->c_phys;  // the tensors are derivatives in physical k
  double sreal[EZ_MAX_NU], srec[EZ_MAX_NU];
#pragma unroll
  for (int jn = 0; jn < EZ_MAX_NU; ++jn) sreal[jn] = srec[jn] = 0.0;
  // real space: 2 sum_{m > 0} g(m) z^alpha, the chunk moments of taylor_real_kernel
  for (int ch = threadIdx.x; ch < J0.n_chunk; ch += blockDim.x) {
    const double* pp = J0.part + ((size_t)ch * R->n_alpha + ia) * nd;
#pragma unroll
    for (int jn = 0; jn < EZ_MAX_NU; ++jn)
      if (jn < nd) sreal[jn] += pp[jn];
  }
  // reciprocal space, h != 0
  const int stride = 2 * R->ell + 1;
  for (int hi = threadIdx.x; hi < R->n_rec; hi += blockDim.x) {
    const G4 G = R->rec[hi];
    if (G.w == 0.0 || G.w > R->R2_recip) continue;
    const double Gv[3] = {G.x * R->inv_s, G.y * R->inv_s, G.z * R->inv_s};  // physical G
    for (int n = K; n <= K2; ++n) {
      const int jj = 2 * n - K2;  // number of linear factors
      // coefficient of k^alpha in (2 G.k)^jj (|k|^2)^(n-jj)
      double coef = 0.0;
      int b[3];
      for (b[0] = 0; b[0] <= alpha[0]; ++b[0])
        for (b[1] = 0; b[1] <= alpha[1]; ++b[1]) {
          b[2] = jj - b[0] - b[1];
          if (b[2] < 0 || b[2] > alpha[2]) continue;
          bool even = true;
          for (int i = 0; i < 3; ++i) even &= ((alpha[i] - b[i]) & 1) == 0;
          if (!even) continue;
          double lin = factd(jj);
          double quad = factd(n - jj);
          for (int i = 0; i < 3; ++i) {
            lin /= factd(b[i]);
            for (int e = 0; e < b[i]; ++e) lin *= 2.0 * Gv[i];
            quad /= factd((alpha[i] - b[i]) / 2);
          }
          coef += lin * quad;
        }
      if (coef == 0.0) continue;
      double cn = 1.0;
      for (int e = 0; e < n; ++e) cn *= c;
      const double f = ((n & 1) ? -1.0 : 1.0) * cn / factd(n) * binom(n, jj) * coef;
#pragma unroll
      for (int jn = 0; jn < EZ_MAX_NU; ++jn)
        if (jn < nd) srec[jn] = fma(jobs[jid + jn].phiG[(size_t)hi * stride + n], f, srec[jn]);
    }
  }
  // fixed-order block reduction of (sreal, srec) per exponent
  __shared__ double red[2 * EZ_MAX_NU][kTaylorThreads];
#pragma unroll
  for (int jn = 0; jn < EZ_MAX_NU; ++jn) {
    red[2 * jn][threadIdx.x] = sreal[jn];
    red[2 * jn + 1][threadIdx.x] = srec[jn];
  }
  __syncthreads();
  for (int w = kTaylorThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int q = 0; q < 2 * nd; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x >= nd) return;
  const int jn = threadIdx.x;
  const TaylorJob J = jobs[jid + jn];
  double twopi_pow = 1.0;
  for (int e = 0; e < K2; ++e) twopi_pow *= 2.0 * kPi;
  const double sr = 2.0 * red[2 * jn][0] * ((K & 1) ? -1.0 : 1.0) * twopi_pow / afact;
  double sk = red[2 * jn + 1][0];
  // h = 0: regularised entire series
  const bool all_even = ((alpha[0] | alpha[1] | alpha[2]) & 1) == 0;
  if (all_even && K <= R->ell) {
    double cK = 1.0;
    for (int e = 0; e < K; ++e) cK *= c;
    sk += J.rser[K] * cK * factd(K) / (factd(alpha[0] / 2) * factd(alpha[1] / 2) * factd(alpha[2] / 2));
  }
  double v = sr + R->vol_fac * sk;
  if (K2 == 0) v -= 2.0 / R->nu[jn];
  J.out[ia] = R->pref[jn] * v;
}

__global__ void phiseq_kernel(const ReqDesc* reqs, const TaylorJob* jobs, int n_jobs) {
  int jid = blockIdx.y;
  if (jid >= n_jobs) return;
  const TaylorJob J = jobs[jid];
  const ReqDesc* R = reqs + J.req;
  int hi = blockIdx.x * blockDim.x + threadIdx.x;
  if (hi >= R->n_rec) return;
  const double a = 0.5 * (R->d - R->nu[J.nu_index]);
  const double t = R->c_lam * R->rec[hi].w;
  const int stride = 2 * R->ell + 1;
  for (int n = 0; n < stride; ++n) J.phiG[(size_t)hi * stride + n] = t > 0.0 ? phi_accurate(a + n, t) : 0.0;
}

// Phase powers e^{2 pi i m u v} (m < mp1) for every (u node, v node) of a quadrature;
// one thread per node pair, sincospi once and complex rotations after.
__global__ void phase_kernel(const PhaseJob* jobs) {
  const PhaseJob J = jobs[blockIdx.y];
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)J.n_ui * J.n_v) return;
  const int iu = (int)(i / J.n_v), iv = (int)(i % J.n_v);
  const double arg = J.v ? J.u[iu] * J.v[iv] : J.u[iu];
  double sn, cs;
  sincospi(2.0 * arg, &sn, &cs);
  double2* o = J.out + (size_t)i * J.mp1;
  float4* off = J.outff ? J.outff + (size_t)i * J.mp1 : nullptr;
  double2 e = make_double2(1.0, 0.0);
  for (int m = 0; m < J.mp1; ++m) {
    if (m) e = make_double2(fma(e.x, cs, -e.y * sn), fma(e.x, sn, e.y * cs));
    o[m] = e;
    if (off) {
      float4 f;
      ff_split(e.x, f.x, f.y);
      ff_split(e.y, f.z, f.w);
      off[m] = f;
    }
  }
}

// d = 3: (log |w|^2, |w|^2, 1/|w|^2, |w|) of every scaled node direction
// w = p1 v1 A^{-T} e_a + p2 v2 A^{-T} e_b + A^{-T} e_c (axes a = j, b = j + 1, c = j + 2 mod 3,
// scaled by sqrt(pi) lam), so that the far kernels get t = u^2 |w|^2, log t = 2 log u +
// log |w|^2, 1/t = u^{-2} / |w|^2 and sqrt t = u |w| of the h = 0 term without a logarithm,
// a division or a square root per node.
__global__ void dirlw_kernel(const ReqDesc* reqs) {
  const ReqDesc* R = reqs + blockIdx.y;
  if (!R->dirlw) return;
  const int nv = R->n_v;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 12LL * nv * nv) return;
  const int v1 = (int)(i % nv);
  long long r = i / nv;
  const int v2 = (int)(r % nv);
  r /= nv;
  const int s2 = (int)(r % 2);
  r /= 2;
  const int s1 = (int)(r % 2), j = (int)(r / 2);
  const int ax_a = j, ax_b = (j + 1) % 3, ax_c = (j + 2) % 3;
  const double a = s1 ? -R->v_nodes[v1] : R->v_nodes[v1];
  const double b = s2 ? -R->v_nodes[v2] : R->v_nodes[v2];
  double w2 = 0.0;
  for (int c = 0; c < 3; ++c) {
    const double wc = fma(R->AiTs[c * 3 + ax_a], a, fma(R->AiTs[c * 3 + ax_b], b, R->AiTs[c * 3 + ax_c]));
    w2 = fma(wc, wc, w2);
  }
  const_cast<double4*>(R->dirlw)[i] = make_double4(log(w2), w2, 1.0 / w2, sqrt(w2));
}

}  // namespace ez
