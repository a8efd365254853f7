// Z_{Lambda,nu}(x, y) in any dimension d <= kMaxDnd (Sec. 6: the method is not tied to
// d <= 3), by the same incomplete-gamma splitting as the d <= 3 kernel:
//   Z = P_nu [ sum_{z != x} Phi_{nu/2}(pi |z - x|^2 / lam^2) e^{-2 pi i y.z}
//            + lam^d/V sum_{g*} Phi_{(d-nu)/2}(pi lam^2 |g* + y|^2) e^{-2 pi i x.(g* + y)}
//            - [x in Lambda] (2/nu) e^{-2 pi i x.y} ].
// In d dimensions a ball fills a vanishing part of its bounding box (about 8 % for d = 6), so
// neither sum runs over a box.
// Real space (the same ball for every y): enumerated once per call as rows along the last
// lattice axis (nd_rows_kernel: the range of each row from the quadratic |z - x|^2 <= r^2,
// nd_scan_kernel: offsets in one deterministic order, nd_fill_kernel: the g values).  Per y the
// sum is contracted axis by axis over the rows: the row sums take the last axis' phases from a
// per-thread table in shared memory (for large boxes the non-negative offsets only, the others
// as conjugates), and a row whose prefix differs from the previous one at
// axis l closes the partial sums of axes d-2 .. l, each multiplied by its axis' phase (a nested
// Horner scheme over the ball, one complex product per closed level).
// Reciprocal space (a different ball for every y): enumerated per thread by the Fincke-Pohst
// recursion on the Cholesky factor R of the dual Gram matrix (scaled units: R^T R = B^T B,
// B = sqrt(pi) lam A^{-T}), so that pi lam^2 |g* + y|^2 = |R (h + yt)|^2 with yt = A^T y reduced
// to [-1/2, 1/2]^d: the admissible interval of h_I follows from h_{I+1} .. h_{d-1}, and only the
// points inside the ball are visited, whatever the shape of the basis.
#include "ez_kernels.h"
#include "ez_phi.cuh"

namespace ez {

namespace {
__device__ __forceinline__ double2 cmul2(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

// s += b with the rounding error of the addition (Knuth's TwoSum) collected in e
__device__ __forceinline__ void two_sum_acc(double& s, double& e, double b) {
  const double t = s + b;
  const double bv = t - s;
  e += (s - (t - bv)) + (b - bv);
  s = t;
}

// lattice point of the row `prefix` (indices id_l, l < d - 1) at last-axis index t:
// z_i = sum_j M[i d + j] id_j in the order j = 0 .. d-1
__device__ __forceinline__ void nd_point(const NdBallJob& J, const int* id, double* z) {
  const int d = J.d;
  for (int i = 0; i < d; ++i) {
    double v = 0.0;
    for (int j = 0; j < d; ++j) v = fma(J.M[i * d + j], (double)id[j], v);
    z[i] = v;
  }
}

__device__ __forceinline__ double nd_r2(const NdBallJob& J, const int* id) {
  double z[kMaxDnd];
  nd_point(J, id, z);
  double r2 = 0.0;
  for (int i = 0; i < J.d; ++i) {
    const double w = z[i] - J.c[i];
    r2 = fma(w, w, r2);
  }
  return r2;
}

// prefix index p -> id_l (l < d - 1), the last prefix axis fastest
__device__ __forceinline__ void nd_decode_prefix(const NdBallJob& J, long long p, int* id) {
  for (int l = J.d - 2; l >= 0; --l) {
    const int e = J.ext[l];
    id[l] = J.lo[l] + (int)(p % e);
    p /= e;
  }
}
}  // namespace

// one thread per row: the range of the last index with |z - c|^2 <= R2
__global__ void nd_rows_kernel(const NdBallJob* job) {
  const NdBallJob& J = *job;
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= J.n_prefix) return;
  const int d = J.d, L = d - 1;
  int id[kMaxDnd];
  nd_decode_prefix(J, p, id);
  // |z0 + t b|^2 <= R2 with z0 = M (prefix, 0) - c and b = column d-1 of M
  double bb = 0.0, zb = 0.0, zz = 0.0;
  for (int i = 0; i < d; ++i) {
    double v = -J.c[i];
    for (int j = 0; j < L; ++j) v = fma(J.M[i * d + j], (double)id[j], v);
    const double b = J.M[i * d + L];
    bb = fma(b, b, bb);
    zb = fma(v, b, zb);
    zz = fma(v, v, zz);
  }
  const double disc = zb * zb - bb * (zz - J.R2);
  int t0 = 1, t1 = 0;
  const int tlo = J.lo[L], thi = J.lo[L] + J.ext[L] - 1;
  if (disc >= 0.0) {
    const double sq = sqrt(disc);
    const double a = (-zb - sq) / bb, b = (-zb + sq) / bb;
    t0 = (int)fmin(fmax(floor(a), (double)tlo), (double)thi + 1.0);
    t1 = (int)fmax(fmin(ceil(b), (double)thi), (double)tlo - 1.0);
    // the same test as the cells' own (the quadratic only brackets the range)
    for (; t0 <= t1; ++t0) {
      id[L] = t0;
      if (nd_r2(J, id) <= J.R2) break;
    }
    for (; t1 >= t0; --t1) {
      id[L] = t1;
      if (nd_r2(J, id) <= J.R2) break;
    }
  }
  J.row_k0[p] = t0 - tlo;
  J.row_n[p] = t1 >= t0 ? t1 - t0 + 1 : 0;
}

// one block of 1024 threads: offsets of the non-empty rows and cells in prefix order, the row
// records and the counts.  Each thread takes a contiguous range of prefixes.
__global__ void __launch_bounds__(1024) nd_scan_kernel(const NdBallJob* job) {
  const NdBallJob& J = *job;
  __shared__ long long s_cells[1024];
  __shared__ int s_rows[1024];
  const int tid = threadIdx.x, nt = blockDim.x;
  const long long n = J.n_prefix;
  const long long chunk = (n + nt - 1) / nt;
  const long long beg = min(n, (long long)tid * chunk), end = min(n, beg + chunk);
  long long cells = 0;
  int rows = 0;
  for (long long p = beg; p < end; ++p) {
    const int k = J.row_n[p];
    cells += k;
    rows += k > 0;
  }
  s_cells[tid] = cells;
  s_rows[tid] = rows;
  __syncthreads();
  if (tid == 0) {  // exclusive scan (1024 entries)
    long long c = 0;
    int r = 0;
    for (int i = 0; i < nt; ++i) {
      const long long ci = s_cells[i];
      const int ri = s_rows[i];
      s_cells[i] = c;
      s_rows[i] = r;
      c += ci;
      r += ri;
    }
    J.counts[0] = r;
    J.counts[1] = (int)min(c, (long long)0x7fffffff);
  }
  __syncthreads();
  const int d = J.d;
  if (J.cell_cap > 0) {
    long long c = s_cells[tid];
    int r = s_rows[tid];
    for (long long p = beg; p < end; ++p) {
      const int k = J.row_n[p];
      if (k == 0) continue;
      int packed = 0;
      long long q = p;
      for (int l = d - 2; l >= 0; --l) {
        packed |= (int)(q % J.ext[l]) << (6 * l);
        q /= J.ext[l];
      }
      J.rows[r] = make_int4((int)c, J.row_k0[p] | (k << 16), packed, 0);
      c += k;
      ++r;
    }
  }
  __syncthreads();
  if (J.cell_cap > 0) {
    const int nrows = J.counts[0];
    for (int r = tid + 1; r < nrows; r += nt) {
      const int a = J.rows[r - 1].z, b = J.rows[r].z;
      int lev = 0;
      while (lev < d - 2 && ((a >> (6 * lev)) & 63) == ((b >> (6 * lev)) & 63)) ++lev;
      J.rows[r].w = lev;
    }
  }
}

// one warp per row: the cells' g values
__global__ void nd_fill_kernel(const NdBallJob* job) {
  const NdBallJob& J = *job;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, n_warps = (gridDim.x * blockDim.x) >> 5;
  const int nrows = J.counts[0], d = J.d, L = d - 1;
  for (int r = warp; r < nrows; r += n_warps) {
    const int4 R = J.rows[r];
    int id[kMaxDnd];
    for (int l = 0; l < L; ++l) id[l] = J.lo[l] + ((R.z >> (6 * l)) & 63);
    const int k0 = R.y & 0xffff, n = R.y >> 16;
    for (int k = lane; k < n; k += 32) {
      id[L] = J.lo[L] + k0 + k;
      const long long cell = (long long)R.x + k;
      if (cell >= J.cell_cap) continue;
      double z[kMaxDnd];
      nd_point(J, id, z);
      bool center = J.skip_center != 0;
      for (int i = 0; i < d; ++i) center = center && id[i] == J.cid[i];
      double r2 = 0.0;
      for (int i = 0; i < d; ++i) {
        const double w = z[i] - J.c[i];
        r2 = fma(w, w, r2);
      }
      J.out[cell] = center ? 0.0 : phi_accurate(J.a, J.pi_over_lam2 * r2);
    }
  }
}

// Reciprocal sum of one y: accumulators (TwoSum-compensated across level-0 runs)
struct RecipAcc {
  double re, im, ere, eim;
  bool pole;
};

// Level I of the Fincke-Pohst recursion: S = sum_{k > I} (R (h + yt))_k^2 so far; h_{I+1..D-1}
// fixed.  (R (h + yt))_I = R_II h_I + u_I with u_I = sum_{j >= I} R_Ij yt_j + sum_{j > I} R_Ij h_j.
template <int D, int I>
__device__ __forceinline__ void fp_level(const NdEpsteinArgs& P, const double (&yt)[D], int (&h)[D], double S,
                                         RecipAcc& acc) {
  double u = 0.0;
#pragma unroll
  for (int j = D - 1; j >= I; --j) u = fma(P.Rk[I * D + j], j > I ? (double)h[j] + yt[j] : yt[j], u);
  const double rem = P.R2_recip - S;
  if (rem < 0.0) return;
  const double rii = P.Rk[I * D + I];
  const double r = sqrt(rem) * (1.0 + 1e-12) + 1e-12;  // bracket; the points are tested below
  const int lo = (int)ceil((-u - r) / rii), hi = (int)floor((-u + r) / rii);
  if constexpr (I > 0) {
    for (h[I] = lo; h[I] <= hi; ++h[I]) {
      const double v = fma(rii, (double)h[I], u);
      fp_level<D, I - 1>(P, yt, h, fma(v, v, S), acc);
    }
  } else {
    // the run h_0 = lo .. hi: phases e^{-2 pi i xt.(h + yt)} with xt = A^{-1} x
    double base = 0.0;
    if (!P.x_zero) {
#pragma unroll
      for (int k = D - 1; k >= 1; --k) base = fma(P.xt[k], (double)h[k] + yt[k], base);
      base = fma(P.xt[0], yt[0], base);
      base -= rint(base);
    }
    double pre = 0.0, pim = 0.0;
    for (int h0 = lo; h0 <= hi; ++h0) {
      const double v = fma(rii, (double)h0, u);
      const double qq = fma(v, v, S);
      if (qq > P.R2_recip) continue;
      double phi;
      if (qq == 0.0) {
        if (P.phi.a >= 0.0) {
          acc.pole = true;
          continue;
        }
        phi = -1.0 / P.phi.a;
      } else {
        int nused;
        phi = phi_eval_qq(P.phi, qq, (float)qq, nused);
      }
      if (P.x_zero) {
        pre += phi;
      } else {
        double sn, cs;
        sincospi(-2.0 * fma(P.xt[0], (double)h0, base), &sn, &cs);
        pre = fma(phi, cs, pre);
        pim = fma(phi, sn, pim);
      }
    }
    two_sum_acc(acc.re, acc.ere, pre);
    two_sum_acc(acc.im, acc.eim, pim);
  }
}

// one thread per y; phase tables of the d axes in shared memory, entry e of thread tid at
// [e * blockDim + tid]
template <int D, bool HALF>
__global__ void __launch_bounds__(128) epstein_nd_kernel(NdEpsteinArgs P) {
  extern __shared__ double2 sph[];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.m) return;
  const int tid = threadIdx.x, nt = blockDim.x;
  double y[D], yt[D];
#pragma unroll
  for (int c = 0; c < D; ++c) y[c] = P.y[(size_t)i * D + c];
#pragma unroll
  for (int c = 0; c < D; ++c) {  // A^T y, reduced to [-1/2, 1/2]
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < D; ++q) s = fma(P.At[c * D + q], y[q], s);
    yt[c] = s - rint(s);
  }
  // phases e^{-2 pi i yt_c o} of the offsets o = k - M_c: all of [-M_c, M_c], or (HALF, for
  // large boxes) [0, M_c] only, a negative offset taking the conjugate of -o (half the shared
  // memory per thread, twice the resident warps)
  int base[D];
  {
    int b = 0;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      base[c] = b;
      const int Mc = P.M[c];
      const int z = HALF ? 0 : Mc;  // slot of offset 0
      double sn, cs;
      sincospi(-2.0 * yt[c], &sn, &cs);
      const double2 e1 = make_double2(cs, sn);
      double2 e = make_double2(1.0, 0.0);
      sph[(size_t)(b + z) * nt + tid] = e;
      for (int k = 1; k <= Mc; ++k) {
        e = cmul2(e, e1);
        sph[(size_t)(b + z + k) * nt + tid] = e;
        if (!HALF) sph[(size_t)(b + z - k) * nt + tid] = make_double2(e.x, -e.y);
      }
      b += HALF ? Mc + 1 : 2 * Mc + 1;
    }
  }
  // phase of box index k (offset k - M_c) on axis c
  auto phase = [&](int c, int k) {
    if (!HALF) return sph[(size_t)(base[c] + k) * nt + tid];
    const int o = k - P.M[c];
    const double2 e = sph[(size_t)(base[c] + (o >= 0 ? o : -o)) * nt + tid];
    return o >= 0 ? e : make_double2(e.x, -e.y);
  };
  // ---- real space over the rows
  static_assert(D >= 2, "rows need a prefix axis");
  double2 acc[D - 1];
  int pidx[D - 1];
#pragma unroll
  for (int l = 0; l < D - 1; ++l) {
    acc[l] = make_double2(0.0, 0.0);
    pidx[l] = 0;
  }
  double2 tot = make_double2(0.0, 0.0), rs = make_double2(0.0, 0.0);
  const int nrows = *P.rcounts;
  // close the partial sums of prefix axes D-2 .. lev of the previous row
  auto close_levels = [&](int lev) {
#pragma unroll
    for (int l = D - 2; l >= 0; --l) {
      if (l >= lev) {
        const double2 v = l == D - 2 ? rs : acc[l];
        if (l < D - 2) acc[l] = make_double2(0.0, 0.0);
        const double2 cv = cmul2(v, phase(l, pidx[l]));
        if (l > 0) {
          acc[l - 1].x += cv.x;
          acc[l - 1].y += cv.y;
        } else {
          tot.x += cv.x;
          tot.y += cv.y;
        }
      }
    }
  };
  for (int r = 0; r < nrows; ++r) {
    const int4 R = __ldg(P.rows + r);
    if (r > 0) close_levels(R.w);
#pragma unroll
    for (int l = 0; l < D - 1; ++l) pidx[l] = (R.z >> (6 * l)) & 63;
    const int k0 = R.y & 0xffff, n = R.y >> 16;
    const double* g = P.g + R.x;
    double sr = 0.0, si = 0.0;
    if constexpr (HALF) {
      const int Ml = P.M[D - 1];
      const double2* ph = sph + (size_t)base[D - 1] * nt + tid;
      int k = 0;
      for (; k < n && k0 + k < Ml; ++k) {  // negative offsets: conjugates
        const double gv = __ldg(g + k);
        const double2 e = ph[(size_t)(Ml - k0 - k) * nt];
        sr = fma(gv, e.x, sr);
        si = fma(-gv, e.y, si);
      }
      for (; k < n; ++k) {
        const double gv = __ldg(g + k);
        const double2 e = ph[(size_t)(k0 + k - Ml) * nt];
        sr = fma(gv, e.x, sr);
        si = fma(gv, e.y, si);
      }
    } else {
      const double2* ph = sph + (size_t)(base[D - 1] + k0) * nt + tid;
      for (int k = 0; k < n; ++k) {
        const double gv = __ldg(g + k);
        const double2 e = ph[(size_t)k * nt];
        sr = fma(gv, e.x, sr);
        si = fma(gv, e.y, si);
      }
    }
    rs = make_double2(sr, si);
  }
  if (nrows > 0) close_levels(0);
  {  // common factor e^{-2 pi i yt.mx}
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < D; ++c) s = fma(yt[c], (double)P.mx[c], s);
    s -= rint(s);
    double sn, cs;
    sincospi(-2.0 * s, &sn, &cs);
    tot = cmul2(tot, make_double2(cs, sn));
  }
  // ---- reciprocal space: sum over |R (h + yt)|^2 <= R2 of Phi * e^{-2 pi i xt.(h + yt)}
  RecipAcc ra{0.0, 0.0, 0.0, 0.0, false};
  {
    int h[D];
    fp_level<D, D - 1>(P, yt, h, 0.0, ra);
  }
  const double rre = ra.re + ra.ere, rim = ra.im + ra.eim;
  const bool pole = ra.pole;
  double tre = tot.x + P.vol_fac * rre, tim = tot.y + P.vol_fac * rim;
  if (P.x_in_lattice) {
    double xy = 0.0;
#pragma unroll
    for (int c = 0; c < D; ++c) xy = fma(P.xt[c], yt[c], xy);
    xy -= rint(xy);
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

cudaError_t launch_epstein_nd(const NdEpsteinArgs& a, unsigned threads, size_t smem, cudaStream_t st) {
  const unsigned grid = (unsigned)((a.m + threads - 1) / threads);
  switch (a.d * 2 + (a.half_phases ? 1 : 0)) {
#define EZ_ND_CASE(DD, HH)                                                                          \
  case DD * 2 + HH: {                                                                               \
    cudaError_t e = cudaFuncSetAttribute(epstein_nd_kernel<DD, HH>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                         (int)smem);                                                \
    if (e != cudaSuccess) return e;                                                                 \
    epstein_nd_kernel<DD, HH><<<grid, threads, smem, st>>>(a);                                      \
    return cudaGetLastError();                                                                      \
  }
    EZ_ND_CASE(4, 0)
    EZ_ND_CASE(4, 1)
    EZ_ND_CASE(5, 0)
    EZ_ND_CASE(5, 1)
    EZ_ND_CASE(6, 0)
    EZ_ND_CASE(6, 1)
#undef EZ_ND_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace ez
