// Far-field, near-field and reduction kernels of the n-body lattice sums
// (Thm "Epstein representation", Cor. "Duffy transformation", Sec. 3).
//
// Far field: a block owns one Duffy line (sector s, u node) for d <= 2; for d = 3 the
// four sectors of one axis j and u node (a line group), vchunk v2 rows of them.  On a
// line k~ = u sigma^j(p1 v1, p2 v2, 1), so the real-space sum of every node factorises
// over the axes:
//   sum_m g(m) e^{2 pi i m.k~} = sum_{ma} Ea(ma, v1) B(ma, v2),
//   B(ma, v2) = sum_{mb} Eb(mb, v2) H(ma, mb),  H(ma, mb) = sum_{mc} g(m) e^{2 pi i mc u},
// H once per line group (d = 3) or per block, B once per block in shared memory;
// g(-m) = g(m) folds ma < 0.
// The reciprocal sum runs per node over the compacted list of A^{-T} h.
#include <cstdio>
#include <type_traits>

#include "ez_ff.cuh"
#include "ez_kernels.h"
#include "ez_phi.cuh"

namespace ez {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

template <int NT>
__device__ __forceinline__ void block_reduce_store(double (&v)[EZ_MAX_PROD], int np, double scale,
                                                   double* out) {
  __shared__ double red[NT / 32][EZ_MAX_PROD];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int p = 0; p < EZ_MAX_PROD; ++p) {
    double x = v[p];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) red[wid][p] = x;
  }
  __syncthreads();
  if (threadIdx.x < EZ_MAX_PROD) {
    double s = 0.0;
    for (int w = 0; w < NT / 32; ++w) s += red[w][threadIdx.x];
    if (threadIdx.x < np) out[threadIdx.x] = scale * s;
  }
}

// adds the block's work counts to the request's counters (one atomic per warp)
// work[0]: in-range reciprocal terms, work[1]: polynomial coefficients evaluated,
// work[2]: terms whose |G + k|^2 was formed (the FP64 form skips it for constant records)
__device__ __forceinline__ void count_work(const ReqDesc* R, unsigned terms, unsigned coefs, unsigned qterms) {
  unsigned long long t = terms, c = coefs, q = qterms;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    t += __shfl_down_sync(0xffffffffu, t, o);
    c += __shfl_down_sync(0xffffffffu, c, o);
    q += __shfl_down_sync(0xffffffffu, q, o);
  }
  if ((threadIdx.x & 31) == 0 && R->work) {
    atomicAdd(R->work, t);
    atomicAdd(R->work + 1, c);
    atomicAdd(R->work + 2, q);
  }
}

__device__ __forceinline__ void load_phi(PhiInfo* sphi, const ReqDesc* R, int nd) {
  const int words = (int)(sizeof(PhiInfo) / sizeof(double));
  const double* src = reinterpret_cast<const double*>(R->phi);
  double* dst = reinterpret_cast<double*>(sphi);
  for (int i = threadIdx.x; i < nd * words; i += blockDim.x) dst[i] = src[i];
}

// Mixed form: the first kRecCache points of the |G|-sorted reciprocal list, staged in
// shared memory once per block: every node of the block walks the list in the same order,
// so each load is a broadcast from shared memory.
// FP64 form, d = 3, >= 4 exponents: the points of the list that can lie within the cutoff for
// some node of the block (a candidate list, in list order, built per block and sign p2 by
// rec_candidates; measured faster there, slower for one exponent and in the mixed form, whose
// walk already stops at the |G| bound of the node).  n = -1 (FP64) or n = n_rec (mixed) walks
// the whole list.
constexpr int kRecCache = 256;
struct RecCacheF64 {  // the FP64 form reads the points through the read-only cache (measured faster)
  int idx[kRecCache];
  int n;
};
struct RecCacheMix {
  float4 f[kRecCache];   // binary32 hi parts and |G|^2
  float4 lo[kRecCache];  // low parts of the float-float G
  int idx[kRecCache];    // list index of entry i
  int n;                 // entries to walk (entries >= kRecCache are list entries, read from global)
};

__device__ __forceinline__ void load_rec_cache(RecCacheF64& c, const ReqDesc*) {
  if (threadIdx.x == 0) c.n = -1;
}
__device__ __forceinline__ void load_rec_cache(RecCacheMix& c, const ReqDesc* R) {
  const int n = min(R->n_rec, kRecCache);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    c.f[i] = __ldg(R->recf + i);
    c.lo[i] = __ldg(R->reclo + i);
    c.idx[i] = i;
  }
  if (threadIdx.x == 0) c.n = R->n_rec;
}

// min over alpha in [-1, 1], beta in [b0, b1] of |w + alpha da + beta db|^2: the stationary
// point if it is inside, else the minimum over the four edges (each a clamped 1-D problem)
__device__ __forceinline__ double para_dist2(const double* w, const double* da, const double* db, double b0,
                                             double b1) {
  const double aa = da[0] * da[0] + da[1] * da[1] + da[2] * da[2];
  const double ab = da[0] * db[0] + da[1] * db[1] + da[2] * db[2];
  const double bb = db[0] * db[0] + db[1] * db[1] + db[2] * db[2];
  const double wa = w[0] * da[0] + w[1] * da[1] + w[2] * da[2];
  const double wb = w[0] * db[0] + w[1] * db[1] + w[2] * db[2];
  const double ww = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  auto q = [&](double al, double be) { return ww + 2.0 * (al * wa + be * wb) + al * al * aa + 2.0 * al * be * ab + be * be * bb; };
  double best = 1e300;
  const double det = aa * bb - ab * ab;
  if (det > 0.0) {
    const double al = (-wa * bb + wb * ab) / det, be = (-wb * aa + wa * ab) / det;
    if (al >= -1.0 && al <= 1.0 && be >= b0 && be <= b1) best = q(al, be);
  }
  for (int e = 0; e < 2; ++e) {
    const double al = e ? 1.0 : -1.0;  // edges alpha = -+1
    const double be = bb > 0.0 ? fmin(fmax(-(wb + al * ab) / bb, b0), b1) : b0;
    best = fmin(best, q(al, be));
    const double bf = e ? b1 : b0;  // edges beta = b0, b1
    const double a2 = aa > 0.0 ? fmin(fmax(-(wa + bf * ab) / aa, -1.0), 1.0) : 0.0;
    best = fmin(best, q(a2, bf));
  }
  return fmax(best, 0.0);
}

// Candidate list of the block: list points G with |G + k| <= r_recip (1 + 1e-5) for some
// k = c0 + alpha da + beta db, alpha in [-1, 1], beta in [b0, b1] (every node of the block at
// one sign p2; the margin is far above the binary32 rounding of the per-node cutoff test, so
// the nodes skip exactly the points they would have skipped in the whole list).  Kept in list
// order; more than kRecCache candidates fall back to the whole list.  Call with every thread.
template <class RC>
__device__ __noinline__ void rec_candidates(RC& rc, const ReqDesc* R, const double* c0, const double* da, const double* db,
                               double b0, double b1) {
  __shared__ int s_cnt[8], s_total;
  constexpr bool kMix = std::is_same<RC, RecCacheMix>::value;
  const int nrec = R->n_rec, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const double r2m = R->R2_recip * (1.0 + 2e-5);
  if (threadIdx.x == 0) s_total = 0;
  __syncthreads();
  for (int base = 0; base < nrec; base += 256) {
    const int h = base + (int)threadIdx.x;
    bool in = false;
    if (h < nrec) {
      const G4 G = ldg_g4(R->rec + h);
      const double w[3] = {G.x + c0[0], G.y + c0[1], G.z + c0[2]};
      in = para_dist2(w, da, db, b0, b1) <= r2m;
    }
    const unsigned m = __ballot_sync(0xffffffffu, in);
    if (lane == 0) s_cnt[wid] = __popc(m);
    __syncthreads();
    int off = s_total;
    for (int q = 0; q < wid; ++q) off += s_cnt[q];
    off += __popc(m & ((1u << lane) - 1u));
    if (in && off < kRecCache) {
      rc.idx[off] = h;
      if constexpr (kMix) {
        rc.f[off] = __ldg(R->recf + h);
        rc.lo[off] = __ldg(R->reclo + h);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0)
      for (int q = 0; q < 8; ++q) s_total += s_cnt[q];
    __syncthreads();
  }
  if (s_total > kRecCache) {
    if constexpr (kMix) {
      load_rec_cache(rc, R);
    } else if (threadIdx.x == 0) {
      rc.n = -1;
    }
  } else if (threadIdx.x == 0) {
    rc.n = s_total;
  }
  __syncthreads();
}

// The direction-table entry of a d = 3 node (null elsewhere) and its block's u: the h = 0
// term has t = u^2 |w|^2, log t = 2 log u + log |w|^2, 1/t = u^{-2} / |w|^2, sqrt t = u |w|.
struct NodeDir {
  const double4* w;  // (log |w|^2, |w|^2, 1/|w|^2, |w|) or null
  const double* ub;  // the block's (u, u^2, 2 log u, 1/u^2) in shared memory (with w)
};

// log t, 1/t and sqrt t of a term with t < kT0 for the orders that take their series (every
// order, or with an order chain those below 1; the chain's recurrence needs 1/t): from the
// direction table (the h = 0 term of a d = 3 node), else computed where needed
__device__ __forceinline__ void small_t_aux(const PhiInfo* sphi, int nd, bool chain, double t, const NodeDir& nd0,
                                            bool h0, double& lt, double& it, double& st) {
  if (h0 && nd0.w) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(nd0.w));
    const double2 b = __ldg(reinterpret_cast<const double2*>(nd0.w) + 1);
    lt = nd0.ub[2] + a.x;
    it = nd0.ub[3] * b.x;
    st = nd0.ub[0] * b.y;
    return;
  }
  bool need_lt = false, need_it = chain, need_st = false;
  for (int j = 0; j < nd; ++j) {
    const PhiInfo& P = sphi[j];
    if (chain && !P.below1) continue;
    need_lt |= P.log_m >= 0 || !P.half;
    need_it |= P.half && P.log_m < 0 && P.two_a > 0;
    need_st |= P.half && P.log_m < 0 && (P.two_a & 1);
  }
  lt = need_lt ? log(t) : 0.0;
  it = need_it ? 1.0 / t : 0.0;
  st = need_st ? sqrt(t) : 0.0;
}

// h = 0 term near k = 0 (t < kT0) of an order chain (orders a_j = a_0 + (nd-1-j), lowest
// a_0 < 0), in binary64: the orders a < 1 by their series (log t and 1/t given by the
// caller), e^{-t} = t Phi_{a_0+1} - a_0 Phi_{a_0} from the two lowest (a sum of positive
// terms), and every order a >= 1 upward by Phi_a = ((a-1) Phi_{a-1} + e^{-t}) / t, also
// positive terms.  brk: the series breakpoints (2^-55 FP64 form, 2^-46 mixed form).
template <int NDM>
__device__ __forceinline__ void chain_values(const PhiInfo* sphi, int nd, double t, double lt, double it, double st,
                                             const float* const* brk, double (&v)[NDM], unsigned& coefs) {
  double prev = 0.0, E = 0.0;
#pragma unroll
  for (int j = NDM - 1; j >= 0; --j)
    if (j < nd) {
      const PhiInfo& P = sphi[j];
      double x;
      if (P.below1) {
        int n;
        x = phi_small_shared(P, t, lt, it, st, n, brk[j]);
        coefs += n;
        if (j == nd - 2) E = fma(t, x, -sphi[nd - 1].a * prev);
      } else {
        x = fma(sphi[j + 1].a, prev, E) * it;
      }
      prev = x;
      v[j] = x;
    }
}

// reciprocal sum at k (x = 0), FP64 form: acc[j] += Phi_{a_j}(pi lam^2 |G + k|^2) over
// |G + k| <= R, every value binary64.  The cutoff test, the branch and the table interval
// are taken in binary32 (a term within ~1e-7 relative of the cutoff radius may fall either
// way: it is below the truncation tolerance by the choice of the radius).
// nd0: the node's direction-table entry (d = 3; its h = 0 term's log t, 1/t, sqrt t).
// With an order chain the terms with t < kT0 take the chain (chain_values), log t and 1/t
// shared by the orders; other orders evaluate their t < kT0 terms one by one (phi_small).
// K2: k holds 2k (the d = 3 kernel forms it from doubled constants; scaling by powers of two
// is exact, so every value is the same as from k).
template <int D, int NDM, bool K2 = false>
__device__ __forceinline__ void recip_sum(const ReqDesc* R, const PhiInfo* sphi, int nd, const double* k,
                                          const float* kf, double* acc, unsigned& terms, unsigned& coefs,
                                          unsigned& qterms, const RecCacheF64& rc, const NodeDir& nd0) {
  const bool chain = NDM >= 3 && R->order_chain && sphi[nd - 1].a < 0.0;
  const bool list = rc.n >= 0;
  const int nrec = list ? rc.n : R->n_rec;
  const float R2f = R->R2f, cf = R->c_lam_f;
  const G4* rec = R->rec;
  const float4* recf = R->recf;
  // |G + k|^2 = |G|^2 + |k|^2 + 2 G.k: with 2k and |k|^2 per node, d FMAs and one add per
  // term (for k in the reduced cell |G + k| is not much smaller than |G|: no cancellation
  // beyond a few ulp)
  double k2v[3] = {0.0, 0.0, 0.0}, kk2 = 0.0;
  if constexpr (K2) {
    double q2 = 0.0;  // |2k|^2
#pragma unroll
    for (int i = 0; i < D; ++i) {
      k2v[i] = k[i];
      q2 = fma(k[i], k[i], q2);
    }
    kk2 = 0.25 * q2;
  } else {
#pragma unroll
    for (int i = 0; i < D; ++i) {
      k2v[i] = 2.0 * k[i];
      kk2 = fma(k[i], k[i], kk2);
    }
  }
  for (int hh = 0; hh < nrec; ++hh) {
    const int h = list ? rc.idx[hh] : hh;
    const float4 Gf = __ldg(recf + h);
    float qqf;
    if (D == 1) {
      const float a = Gf.x + kf[0];
      qqf = a * a;
    } else if (D == 2) {
      const float a = Gf.x + kf[0], b = Gf.y + kf[1];
      qqf = fmaf(a, a, b * b);
    } else {
      const float a = Gf.x + kf[0], b = Gf.y + kf[1], c = Gf.z + kf[2];
      qqf = fmaf(a, a, fmaf(b, b, c * c));
    }
    if (qqf <= R2f) {
      const float tf = cf * qqf;
      // the binary64 |G + k|^2 only where an order needs it: a constant record (Phi below
      // the table floor on the interval, picked by the binary32 t) is one load
      double qq = 0.0;
      bool have_qq = false;
      ++terms;
      if (chain && tf < (float)kT0) {
        const G4 G = ldg_g4(rec + h);
        qq = fma(k2v[0], G.x, G.w + kk2);
        if (D >= 2) qq = fma(k2v[1], G.y, qq);
        if (D >= 3) qq = fma(k2v[2], G.z, qq);
        ++qterms;
        // qq > 0 and |G|^2 == 0 as integer tests on the binary64 words (neither value is a
        // NaN; a positive double has a positive bit pattern): off the FP64 pipe
        if (__double_as_longlong(qq) > 0) {
          const double t = D == 3 ? qq : sphi[0].c_lam * qq;  // c_lam = 1 (scaled units); d = 3 skips it
          double lt, it, st;
          small_t_aux(sphi, nd, true, t, nd0, __double_as_longlong(G.w) == 0, lt, it, st);
          const float* brk[NDM];
#pragma unroll
          for (int j = 0; j < NDM; ++j) brk[j] = sphi[j].ser_brk;
          double v[NDM];
          chain_values<NDM>(sphi, nd, t, lt, it, st, brk, v, coefs);
#pragma unroll
          for (int j = 0; j < NDM; ++j)
            if (j < nd) acc[j] += v[j];
          continue;
        }
        have_qq = true;
      }
      if (chain && tf >= (float)kT0 && tf <= sphi[0].t_hi_f) {
        // the two lowest orders from their tables, e^{-t} = t Phi_{a0+1} - a0 Phi_{a0} from them
        // (positive terms, a0 < 0) and every higher order upward by Phi_a = ((a-1) Phi_{a-1} +
        // e^{-t}) / t, also positive terms: half the table records per term.  Where both
        // records are constants (Phi below the table floor) every order takes its constant.
        const int i = min(phi_interval(tf, sphi[0].t_geo_end_f), sphi[0].n_int - 1);
        const double* r0 = sphi[nd - 1].tab + (size_t)i * kRec;
        const double* r1 = sphi[nd - 2].tab + (size_t)i * kRec;
        const double2 so0 = __ldg(reinterpret_cast<const double2*>(r0));
        const double2 so1 = __ldg(reinterpret_cast<const double2*>(r1));
        const bool c0 = __double2loint(so0.x) == 1, c1 = __double2loint(so1.x) == 1;
        if (!(c0 && c1)) {
          const G4 G = ldg_g4(rec + h);
          qq = fma(k2v[0], G.x, G.w + kk2);
          if (D >= 2) qq = fma(k2v[1], G.y, qq);
          if (D >= 3) qq = fma(k2v[2], G.z, qq);
          ++qterms;
          const double t = D == 3 ? qq : sphi[0].c_lam * qq;  // c_lam = 1 (scaled units); d = 3 skips it
          int n0 = 0, n1 = 0;
          const double v0 = c0 ? __ldg(r0 + 4) : phi_poly(r0, fma(qq, so0.y, __ldg(r0 + 2)), n0);
          const double v1 = c1 ? __ldg(r1 + 4) : phi_poly(r1, fma(qq, so1.y, __ldg(r1 + 2)), n1);
          coefs += n0 + n1;
          acc[nd - 1] += v0;
          acc[nd - 2] += v1;
          const double E = fma(t, v1, -sphi[nd - 1].a * v0);
          const double it = 1.0 / t;
          double prev = v1;
#pragma unroll
          for (int j = NDM - 3; j >= 0; --j)
            if (j <= nd - 3) {
              prev = fma(sphi[j + 1].a, prev, E) * it;
              acc[j] += prev;
            }
          continue;
        }
      }
#pragma unroll
      for (int j = 0; j < NDM; ++j)
        if (j < nd) {
          const PhiInfo& P = sphi[j];
          if (tf >= (float)kT0 && tf <= P.t_hi_f) {
            const int i = min(phi_interval(tf, P.t_geo_end_f), P.n_int - 1);
            const double* r = P.tab + (size_t)i * kRec;
            const double2 so = __ldg(reinterpret_cast<const double2*>(r));  // (n|pad, s)
            if (__double2loint(so.x) == 1) {
              acc[j] += __ldg(r + 4);
              continue;
            }
          }
          if (!have_qq) {
            const G4 G = ldg_g4(rec + h);
            qq = fma(k2v[0], G.x, G.w + kk2);
            if (D >= 2) qq = fma(k2v[1], G.y, qq);
            if (D >= 3) qq = fma(k2v[2], G.z, qq);
            have_qq = true;
            ++qterms;
          }
          int n;
          acc[j] += phi_eval_qq(P, qq, tf, n);
          coefs += n;
        }
    }
  }
}

// 1/x to ~1 ulp for normal x > 0 (one MUFU operation; binary32 tail and middle-range terms)
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Mixed form, binary32 tail term for every exponent: Phi_a(t) = e^{-t} t^{-1} P_a(t_mix/t).
// With an order chain (orders a_j = a_0 - j) only the lowest order uses its fit; the others
// follow upward from t Phi_{a+1} = a Phi_a + e^{-t} (stable for t > t_mix > |a|).
template <int NDM>
__device__ __forceinline__ void tails_f(const PhiInfo* sphi, int nd, bool chain, float E, float r, float sv,
                                        float* st) {
  float prev = 0.0f;
#pragma unroll
  for (int j = NDM - 1; j >= 0; --j)
    if (j < nd) {
      const float v = (!chain || j == nd - 1) ? E * r * phi_tail_poly(sphi[j], sv)
                                              : fmaf(sphi[j + 1].a_f, prev, E) * r;
      prev = v;
      st[j] += v;
    }
}

// the mixed form's binary64 near-origin term: the chain, or every order by its series,
// with log t, 1/t and sqrt t from the direction-table entry w (the h = 0 term of a d = 3
// node: t = u^2 |w|^2) or computed; the values split into float-float and added to hs.
// Out of line: it keeps the transcendental code out of the registers of the caller's loop.
template <int NDM>
__device__ __noinline__ void small_terms_f64(const PhiInfo* sphi, int nd, bool chain, double t, const double4* w,
                                             const double* ub, ff* hs, unsigned& coefs) {
  double lt, it, st;
  const NodeDir nd0{w, ub};
  small_t_aux(sphi, nd, chain, t, nd0, w != nullptr, lt, it, st);
  double v[NDM];
  if (chain) {
    const float* brk[NDM];
#pragma unroll
    for (int j = 0; j < NDM; ++j) brk[j] = sphi[j].ser_brk_mix;
    chain_values<NDM>(sphi, nd, t, lt, it, st, brk, v, coefs);
  } else {
#pragma unroll
    for (int j = 0; j < NDM; ++j)
      if (j < nd) {
        int n;
        v[j] = phi_small_shared(sphi[j], t, lt, it, st, n, sphi[j].ser_brk_mix);
        coefs += n;
      }
  }
#pragma unroll
  for (int j = 0; j < NDM; ++j)
    if (j < nd) {
      float hi, lo;
      ff_split_trunc(v[j], hi, lo);
      hs[j] = ff_add(hs[j], ff{hi, lo});
    }
}

// Mixed form of the same sum.  Terms by t = pi lam^2 |G + k|^2 (binary32 screen):
//  * t >= t_mix (|Phi| t <= 1e-7 beyond it): binary32, e^{-t} t^{-1} P(t_mix/t);
//  * t_mid <= t < t_mix (|Phi| <= 1e-6): float-float argument, binary32 polynomial;
//  * kT0 <= t < t_mid (the heads): float-float |G + k|^2, argument and Horner scheme on
//    the float-float table (~46 bits, no binary64 instruction);
//  * t < kT0 (the h = 0 term near k = 0: series and singular part) or beyond the table:
//    binary64 as in the FP64 form, from |G + k|^2 formed in binary64 of the float-float k.
// The list is sorted by |G|: once |G| > sqrt(t_mix / c) + |k|, every remaining term is a
// binary32 tail, evaluated by a short loop that skips the points beyond the cutoff.  Tails
// are summed in binary32, the middle range with Kahan compensation, heads in float-float.
// nd0: the node's direction-table entry (d = 3): t, log t, 1/t and sqrt t of its h = 0 term.
template <int D, int NDM>
__device__ __forceinline__ void recip_sum_mixed(const ReqDesc* R, const PhiInfo* sphi, int nd, const ff* kff,
                                                ff* A, unsigned& terms, unsigned& coefs, const RecCacheMix& rc,
                                                const NodeDir& nd0) {
  const int nrec = rc.n;
  const float R2f = R->R2f, cf = R->c_lam_f;
  const float tmix = sphi[0].t_mix_f, tmid = sphi[0].t_mid_f;
  const float t_hi = sphi[0].t_hi_f, t_geo = sphi[0].t_geo_end_f;
  const int last = sphi[0].n_int - 1;
  const float* tabff0 = sphi[0].tabff;
  const float4* recf = R->recf;
  const float4* reclo = R->reclo;
  const bool chain = NDM >= 3 && R->order_chain;
  // binary64 near-origin terms: the order chain, or (a log-case or real order) every order
  // by its series with log t shared; else each order on its own (phi_eval_qq)
  const bool chain64 = chain && sphi[nd - 1].a < 0.0;
  bool shared = chain64;
  for (int j = 0; j < nd; ++j) shared |= sphi[j].log_m >= 0 || !sphi[j].half;
  float kf[3] = {0.0f, 0.0f, 0.0f}, klo[3] = {0.0f, 0.0f, 0.0f}, kn2 = 0.0f;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    kf[i] = kff[i].hi;
    klo[i] = kff[i].lo;
    kn2 = fmaf(kf[i], kf[i], kn2);
  }
  // |G| beyond which t > t_mix for this k, and beyond which |G + k| > R (relative margins
  // for the binary32 rounding)
  const float kn = sqrtf(kn2);
  const float gb = (sqrtf(tmix / cf) + kn) * 1.0001f;
  const float gb2 = gb * gb;
  const float gc = (sqrtf(R2f) + kn) * 1.0001f;
  const float gc2 = gc * gc;
  float sf[NDM], cpf[NDM], st[NDM];
  ff hs[NDM];
#pragma unroll
  for (int j = 0; j < NDM; ++j) {
    sf[j] = cpf[j] = st[j] = 0.0f;
    hs[j] = ff{0.0f, 0.0f};
  }
  int h = 0;
  for (; h < nrec; ++h) {
    const float4 Gf = h < kRecCache ? rc.f[h] : __ldg(recf + h);
    if (Gf.w > gb2) break;
    float qqf;
    if (D == 1) {
      const float a = Gf.x + kf[0];
      qqf = a * a;
    } else if (D == 2) {
      const float a = Gf.x + kf[0], b = Gf.y + kf[1];
      qqf = fmaf(a, a, b * b);
    } else {
      const float a = Gf.x + kf[0], b = Gf.y + kf[1], c = Gf.z + kf[2];
      qqf = fmaf(a, a, fmaf(b, b, c * c));
    }
    if (qqf > R2f) continue;
    const float tf = cf * qqf;
    if (tf >= tmix) {
      const float r = rcp_approx(tf), E = __expf(-tf), sv = tmix * r;
      tails_f<NDM>(sphi, nd, chain, E, r, sv, st);
      continue;
    }
    // binary64: the incomplete gamma near the origin (t < kT0, the h = 0 term near k = 0:
    // entire series plus singular part, as in the FP64 form), t = 0, and beyond the table
    if (tf < (float)kT0 || tf > t_hi) {
      if (shared && tf < (float)kT0 && Gf.w == 0.0f && nd0.w) {  // the h = 0 term from the direction table
        ++terms;
        const double t0 = nd0.ub[1] * __ldg(reinterpret_cast<const double*>(nd0.w) + 1);
        small_terms_f64<NDM>(sphi, nd, chain64, t0, nd0.w, nd0.ub, hs, coefs);
        continue;
      }
      const G4 G = ldg_g4(R->rec + (h < kRecCache ? rc.idx[h] : h));
      const double q0 = G.x + ((double)kf[0] + (double)klo[0]);
      double qq = q0 * q0;
      if (D >= 2) {
        const double q1 = G.y + ((double)kf[1] + (double)klo[1]);
        qq = fma(q1, q1, qq);
      }
      if (D >= 3) {
        const double q2 = G.z + ((double)kf[2] + (double)klo[2]);
        qq = fma(q2, q2, qq);
      }
      ++terms;
      if (shared && tf < (float)kT0 && qq > 0.0) {
        small_terms_f64<NDM>(sphi, nd, chain64, sphi[0].c_lam * qq, nullptr, nullptr, hs, coefs);
        continue;
      }
#pragma unroll
      for (int j = 0; j < NDM; ++j)
        if (j < nd) {
          int n;
          float hi, lo;
          ff_split(phi_eval_qq(sphi[j], qq, tf, n), hi, lo);
          hs[j] = ff_add(hs[j], ff{hi, lo});
          coefs += n;
        }
      continue;
    }
    // float-float |G + k|^2 and x = s (|q|^2 - m) (s, m shared by every exponent)
    const float4 Gl = h < kRecCache ? rc.lo[h] : __ldg(reclo + h);
    ff qq = ff_sqr(ff_add4(Gf.x, Gl.x, kf[0], klo[0]));
    if (D >= 2) qq = ff_add(qq, ff_sqr(ff_add4(Gf.y, Gl.y, kf[1], klo[1])));
    if (D >= 3) qq = ff_add(qq, ff_sqr(ff_add4(Gf.z, Gl.z, kf[2], klo[2])));
    const int iv = min(phi_interval(tf, t_geo), last);
    const float4 hd = __ldg(reinterpret_cast<const float4*>(tabff0 + (size_t)iv * kRecFF));      // n, 0, s
    const float4 hm = __ldg(reinterpret_cast<const float4*>(tabff0 + (size_t)iv * kRecFF) + 1);  // m, 0, 0
    const ff dq = ff_two_sum(__fsub_rn(qq.hi, hm.x), __fsub_rn(qq.lo, hm.y));  // leading difference exact
    const ff x = ff_mul(dq, ff{hd.z, hd.w});
    if (tf >= tmid) {
      // descending j = ascending order; with a chain only the two lowest orders use the
      // table, the others follow from t Phi_{a+1} = a Phi_a + e^{-t}
      float prev = 0.0f, Ef = 0.0f;
      const float rt = chain ? rcp_approx(tf) : 0.0f;
#pragma unroll
      for (int j = NDM - 1; j >= 0; --j)
        if (j < nd) {
          float v;
          if (!chain || j >= nd - 2) {
            v = phi_poly_f(sphi[j].tabf + (size_t)iv * kRec, x.hi);
            if (chain && j == nd - 2) Ef = fmaf(tf, v, -sphi[nd - 1].a_f * prev);
          } else {
            v = fmaf(sphi[j + 1].a_f, prev, Ef) * rt;
          }
          prev = v;
          const float y = v - cpf[j];  // Kahan: sf + cpf carries the middle range
          const float t = sf[j] + y;
          cpf[j] = (t - sf[j]) - y;
          sf[j] = t;
        }
      continue;
    }
    ++terms;
    {
      ff prev{0.0f, 0.0f}, E{0.0f, 0.0f}, rt{0.0f, 0.0f};
      if (chain) {
        const ff tff = ff_mul(ff{R->c_lam_ff.x, R->c_lam_ff.y}, qq);
        rt = ff_rcp(tff);
        E = tff;  // holds t until the two table orders are known
      }
#pragma unroll
      for (int j = NDM - 1; j >= 0; --j)
        if (j < nd) {
          ff v;
          if (!chain || j >= nd - 2) {
            int n;
            v = phi_poly_ff(sphi[j].tabff + (size_t)iv * kRecFF, x, n);
            coefs += n;
            if (chain && j == nd - 2) {  // e^{-t} = t Phi_{a+1} - a Phi_a with a the lowest order
              const ff ap = ff_mul(ff{sphi[nd - 1].a_f, 0.0f}, prev);
              E = ff_add(ff_mul(E, v), ff{-ap.hi, -ap.lo});
            }
          } else {
            v = ff_mul(ff_add(ff_mul(ff{sphi[j + 1].a_f, 0.0f}, prev), E), rt);
          }
          prev = v;
          hs[j] = ff_add(hs[j], v);
        }
    }
  }
  // the rest: binary32 tails only, up to the cutoff
#pragma unroll 2
  for (; h < nrec; ++h) {
    const float4 Gf = h < kRecCache ? rc.f[h] : __ldg(recf + h);
    if (Gf.w > gc2) break;
    float qqf;
    if (D == 1) {
      const float a = Gf.x + kf[0];
      qqf = a * a;
    } else if (D == 2) {
      const float a = Gf.x + kf[0], b = Gf.y + kf[1];
      qqf = fmaf(a, a, b * b);
    } else {
      const float a = Gf.x + kf[0], b = Gf.y + kf[1], c = Gf.z + kf[2];
      qqf = fmaf(a, a, fmaf(b, b, c * c));
    }
    if (qqf > R2f) continue;  // outside the cutoff (neighbouring nodes mostly agree: little divergence)
    const float tf = cf * qqf;
    const float r = rcp_approx(tf), sv = tmix * r;
    tails_f<NDM>(sphi, nd, chain, __expf(-tf), r, sv, st);
  }
#pragma unroll
  for (int j = 0; j < NDM; ++j)
    if (j < nd) A[j] = ff_add_f(ff_add_f(ff_add_f(hs[j], sf[j]), -cpf[j]), st[j]);
}

// Mixed form, node assembly in float-float: Z_j = P_j (Zr_j + (lam^d/V) A_j - 2/nu_j)
// (Zr: real-space part incl. the m = 0 column, A: reciprocal sum), then every product
// prod_j Z_j^{e_pj} times the node weight w added to wsum.
template <int NDM>
__device__ __forceinline__ void assemble_mixed(const ReqDesc* R, int nd, int np, const ff* Zr, const ff* A, ff w,
                                               ff (&wsum)[EZ_MAX_PROD]) {
  ff Z[NDM];
  const ff vol{R->vol_ff.x, R->vol_ff.y};
#pragma unroll
  for (int j = 0; j < NDM; ++j)
    if (j < nd) {
      ff t = ff_add(Zr[j], ff_mul(vol, A[j]));
      t = ff_add(t, ff{-R->tov_ff[j].x, -R->tov_ff[j].y});
      Z[j] = ff_mul(ff{R->pref_ff[j].x, R->pref_ff[j].y}, t);
    }
#pragma unroll
  for (int p = 0; p < EZ_MAX_PROD; ++p) {
    if (p >= np) break;
    ff f{1.0f, 0.0f};
#pragma unroll
    for (int j = 0; j < NDM; ++j)
      if (j < nd)
        for (int q = 0; q < R->expo[p][j]; ++q) f = ff_mul(f, Z[j]);
    wsum[p] = ff_add(wsum[p], ff_mul(w, f));
  }
}

// float-float of a binary64 value held in a register (per block or per node setup)
__device__ __forceinline__ ff ffd(double x) {
  ff r;
  ff_split(x, r.hi, r.lo);
  return r;
}

// Products of the node's zeta values, weighted and accumulated per product.  FIRST: each
// product starts from its first factor (the d = 3 kernel: one binary64 multiplication fewer
// per product); the d = 1, 2 kernels keep the loop from 1, which holds fewer registers there.
template <int NDM, bool FIRST = false>
__device__ __forceinline__ void products(const ReqDesc* R, int nd, int np, const double* Z, double w,
                                         double (&acc)[EZ_MAX_PROD]) {
#pragma unroll
  for (int p = 0; p < EZ_MAX_PROD; ++p) {
    if (p >= np) break;
    double f = 1.0;
    if constexpr (FIRST) {
      bool first = true;
#pragma unroll
      for (int j = 0; j < NDM; ++j)
        if (j < nd) {
          int e = R->expo[p][j];
          if (e > 0 && first) {
            f = Z[j];
            first = false;
            --e;
          }
          for (int q = 0; q < e; ++q) f *= Z[j];
        }
    } else {
      for (int j = 0; j < nd; ++j) {
        const int e = R->expo[p][j];
        for (int q = 0; q < e; ++q) f *= Z[j];
      }
    }
    acc[p] = fma(w, f, acc[p]);
  }
}

size_t far_smem_bytes(int d, int nd, const int* M, int n_v, int vchunk) {
  int Mx = 0;
  for (int i = 0; i < d; ++i) Mx = M[i] > Mx ? M[i] : Mx;
  size_t n = 0;
  if (d == 3)  // Ea, Eb, H, B_{+-}, 8 bytes per (exponent, thread) for the p1 = -1 node, k parts
    n = (size_t)(Mx + 1) * n_v + (size_t)(Mx + 1) * vchunk + (size_t)nd * (Mx + 1) * (2 * Mx + 1) +
        2 * (size_t)nd * (Mx + 1) * vchunk + (size_t)nd * 128 + ((size_t)(n_v + 2 * vchunk) * 24 + 15) / 16;
  else if (d == 2)
    n = (size_t)(Mx + 1) + (size_t)nd * (Mx + 1);
  return n * sizeof(double2);
}

// Compensated dot product step (the Dot2 scheme of Ogita, Rump and Oishi, 2005, on
// float-float operands): s + c += (a_hi + a_lo)(b_hi + b_lo).  The leading product and
// the running sum are split exactly (two_prod, two_sum); the cross terms and the errors
// go to c.  ~12 binary32 instructions, result as if accumulated with ~48 bits.
__device__ __forceinline__ void dot2_acc(float& s, float& c, float a_hi, float a_lo, float b_hi, float b_lo) {
  const float p = __fmul_rn(a_hi, b_hi);
  float e = __fmaf_rn(a_hi, b_hi, -p);
  e = __fmaf_rn(a_hi, b_lo, __fmaf_rn(a_lo, b_hi, e));
  const ff t = ff_two_sum(s, p);
  s = t.hi;
  c = __fadd_rn(c, __fadd_rn(t.lo, e));
}

__device__ __forceinline__ float4 ff_complex(double2 z) {
  float4 r;
  ff_split(z.x, r.x, r.y);
  ff_split(z.y, r.z, r.w);
  return r;
}

// ------------------------------------------------------------------------- d = 3
// A line group is the axis j of the Duffy sector and the u node: its four sectors (sign
// patterns p1, p2 of k~ = u sigma^j(p1 v1, p2 v2, 1)) share H(ma, mb) = sum_mc g(m)
// e^{2 pi i mc u}, which depends on neither the signs nor v.  It is built once per
// (request, line group) by hbox_kernel and stored folded over mb:
//   H(ma, 0) at mb = 0,  Hs = H(ma, mb) + H(ma, -mb) at +mb,  Hd = H(ma, mb) - H(ma, -mb) at -mb,
// as double2 summed in binary64 (FP64 form) or as float-float complex (mixed form: re hi,
// re lo, im hi, im lo) from compensated binary32 dot products.
// Grid: (chunk of kHboxCols columns (jn, ma, mb >= 0), axis j, job).  A block stages its
// columns' g values along the c axis (both signs of mb) in shared memory once, then computes
// H for every u node of the axis from them, kHboxU nodes at a time with their phases
// e^{2 pi i mc u} tabulated; each (column, u node) entry is the same sum, in the same order,
// as a direct evaluation.  The box is read once per (request, axis) instead of once per line
// group.
constexpr int kHboxCols = kHboxColsHost, kHboxU = 32;
template <bool MIXED>
__global__ void __launch_bounds__(256) hbox_kernel(const ReqDesc* __restrict__ reqs, const HboxJob* __restrict__ jobs) {
  using GT = typename std::conditional<MIXED, float2, double>::type;
  using ET = typename std::conditional<MIXED, float4, double2>::type;
  __shared__ GT sg[kHboxCols][2][2 * kMaxBoxM + 1];  // [column][+mb, -mb][mc + Mc]
  __shared__ ET sE[kHboxU][kMaxBoxM + 1];            // [u node of the tile][mc]
  const HboxJob& J = jobs[blockIdx.z];
  if (MIXED ? !J.outff : !J.out) return;
  const ReqDesc* R = reqs + J.req;
  const int j = blockIdx.y, n_ui = R->n_ui, nd = R->n_distinct;
  const int iu_lo = max(0, J.g_lo - j * n_ui), iu_hi = min(n_ui, J.g_hi - j * n_ui);
  if (iu_hi <= iu_lo) return;
  const int ax_a = j, ax_b = (j + 1) % 3, ax_c = (j + 2) % 3;
  const int Ma = R->M[ax_a], Mb = R->M[ax_b], Mc = R->M[ax_c];
  const int nHp = (Ma + 1) * (Mb + 1), ncols = nd * nHp;
  const int c0 = blockIdx.x * kHboxCols;
  if (c0 >= ncols) return;
  const int nc = min(kHboxCols, ncols - c0);
  const int st[3] = {R->box[1] * R->box[2], R->box[2], 1};
  const int sta = st[ax_a], stb = st[ax_b], stc = st[ax_c];
  const int gbase = R->M[0] * st[0] + R->M[1] * st[1] + R->M[2] * st[2];
  const long long cells = (long long)R->box[0] * R->box[1] * R->box[2];
  const int nz = 2 * Mc + 1;
  for (int e = threadIdx.x; e < nc * 2 * nz; e += blockDim.x) {
    const int col = e / (2 * nz), r = e - col * 2 * nz, sgn = r / nz, z = r - sgn * nz;
    const int c = c0 + col, jn = c / nHp, q = c - jn * nHp, ma = q / (Mb + 1), mb = q - ma * (Mb + 1);
    const long long off = (long long)jn * cells + gbase + ma * sta + (sgn ? -mb : mb) * stb + (z - Mc) * stc;
    if constexpr (MIXED)
      sg[col][sgn][z] = R->gboxff[off];
    else
      sg[col][sgn][z] = R->gbox[off];
  }
  const int nH = (Ma + 1) * (2 * Mb + 1);
  for (int t0 = iu_lo; t0 < iu_hi; t0 += kHboxU) {
    const int nt = min(kHboxU, iu_hi - t0);
    __syncthreads();  // the columns are staged; the previous tile's phases are used up
    for (int e = threadIdx.x; e < nt * (Mc + 1); e += blockDim.x) {
      const int t = e / (Mc + 1), mc = e - t * (Mc + 1);
      double sn, cs;
      sincospi(2.0 * ((double)mc * R->u_nodes[t0 + t]), &sn, &cs);
      if constexpr (MIXED)
        sE[t][mc] = ff_complex(make_double2(cs, sn));
      else
        sE[t][mc] = make_double2(cs, sn);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nc * nt; e += blockDim.x) {
      const int t = e / nc, col = e - t * nc;
      const int c = c0 + col, jn = c / nHp, q = c - jn * nHp, ma = q / (Mb + 1), mb = q - ma * (Mb + 1);
      const GT* gp_ = &sg[col][0][Mc];
      const GT* gm_ = &sg[col][1][Mc];
      const ET* Ec = sE[t];
      const size_t base =
          (size_t)(j * n_ui + t0 + t - J.g_lo) * R->hslot + (size_t)jn * nH + ma * (2 * Mb + 1) + Mb;
      if constexpr (MIXED) {
        // compensated dot products in binary32 on the float-float box; |mc| >= m_hp (below
        // 1e-8) in plain binary32
        float s0 = gp_[0].x, c0f = gp_[0].y, s1 = 0.0f, c1 = 0.0f, s2 = gm_[0].x, c2 = gm_[0].y, s3 = 0.0f, c3 = 0.0f;
        const int mc_hp = min(Mc + 1, R->m_hp[ax_c]);
        for (int mc = 1; mc < mc_hp; ++mc) {
          const float4 E = Ec[mc];
          const float2 a = gp_[mc], b = gp_[-mc], cc = gm_[mc], dd = gm_[-mc];
          dot2_acc(s0, c0f, a.x, a.y, E.x, E.y);
          dot2_acc(s0, c0f, b.x, b.y, E.x, E.y);
          dot2_acc(s1, c1, a.x, a.y, E.z, E.w);
          dot2_acc(s1, c1, -b.x, -b.y, E.z, E.w);
          dot2_acc(s2, c2, cc.x, cc.y, E.x, E.y);
          dot2_acc(s2, c2, dd.x, dd.y, E.x, E.y);
          dot2_acc(s3, c3, cc.x, cc.y, E.z, E.w);
          dot2_acc(s3, c3, -dd.x, -dd.y, E.z, E.w);
        }
        float q0 = 0.0f, q1 = 0.0f, q2 = 0.0f, q3 = 0.0f;
        for (int mc = mc_hp; mc <= Mc; ++mc) {
          const float4 E = Ec[mc];
          const float a = gp_[mc].x, b = gp_[-mc].x, cc = gm_[mc].x, dd = gm_[-mc].x;
          q0 = fmaf(a + b, E.x, q0);
          q1 = fmaf(a - b, E.z, q1);
          q2 = fmaf(cc + dd, E.x, q2);
          q3 = fmaf(cc - dd, E.z, q3);
        }
        const ff pr = ff_two_sum(s0, c0f + q0), pi = ff_two_sum(s1, c1 + q1);
        const ff mr = ff_two_sum(s2, c2 + q2), mi = ff_two_sum(s3, c3 + q3);
        if (mb == 0) {
          J.outff[base] = make_float4(pr.hi, pr.lo, pi.hi, pi.lo);
        } else {
          const ff sr = ff_add(pr, mr), si = ff_add(pi, mi);
          const ff dr = ff_add(pr, ff{-mr.hi, -mr.lo}), di = ff_add(pi, ff{-mi.hi, -mi.lo});
          J.outff[base + mb] = make_float4(sr.hi, sr.lo, si.hi, si.lo);
          J.outff[base - mb] = make_float4(dr.hi, dr.lo, di.hi, di.lo);
        }
      } else {
        // H(ma, +-mb): real parts pair g(+mc) + g(-mc) with cos, imaginary parts the difference with sin
        double pr = gp_[0], pi = 0.0, mr = gm_[0], mi = 0.0;
        for (int mc = 1; mc <= Mc; ++mc) {
          const double2 E = Ec[mc];
          const double a = gp_[mc], b = gp_[-mc], cc = gm_[mc], dd = gm_[-mc];
          pr = fma(a + b, E.x, pr);
          pi = fma(a - b, E.y, pi);
          mr = fma(cc + dd, E.x, mr);
          mi = fma(cc - dd, E.y, mi);
        }
        double2 hs, hd;
        if (mb == 0) {
          hs = make_double2(pr, pi);
          hd = hs;
        } else {
          hs = make_double2(pr + mr, pi + mi);
          hd = make_double2(pr - mr, pi - mi);
        }
        J.out[base + mb] = hs;
        if (mb) J.out[base - mb] = hd;
      }
    }
  }
}

cudaError_t launch_hbox(bool mixed_any, bool f64_any, unsigned col_chunks, int n_req, const ReqDesc* reqs,
                        const HboxJob* jobs, cudaStream_t st) {
  const dim3 grid(col_chunks, 3, (unsigned)n_req);
  if (f64_any) {
    hbox_kernel<false><<<grid, 256, 0, st>>>(reqs, jobs);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (mixed_any) {
    hbox_kernel<true><<<grid, 256, 0, st>>>(reqs, jobs);
    return cudaGetLastError();
  }
  return cudaSuccess;
}

// Far field, d = 3.  Block: the four sectors of one line group and vchunk rows v2, all n_v
// values of v1.  With the p = +1 phases Ea(ma, v1) = e^{2 pi i ma u v1}, Eb(mb, v2) =
// e^{2 pi i mb u v2} (p = -1 conjugates them):
//   B_p2(ma, v2) = X + p2 Y,  X = H(ma, 0) + sum_{mb >= 1} Hs Re Eb,  Y = i sum_{mb >= 1} Hd Im Eb,
//   Zr_{p1 p2}(v1, v2) = B_p2(0, v2) + 2 (S0 - p1 S1),  S0 = sum_{ma >= 1} Re Ea Re B_p2,
//   S1 = sum_{ma >= 1} Im Ea Im B_p2,
// so one pass over mb gives both B of a v2 row and one pass over ma both nodes (p1 = +-1) of
// a (v1, v2, p2).  Shared memory (16-byte entries): Ea[(Ma+1) n_v], Eb[(Mb+1) vchunk],
// H[nd (Ma+1) (2Mb+1)] (copied from the line group's slot), B[2][nd (Ma+1) vchunk], then
// one 8-byte slot per (exponent, thread) holding the real-space part of the p1 = -1 node
// while the p1 = +1 node runs (registers are the limit of this kernel), and (mixed form)
// the float-float parts of k = p1 kA(v1) + kB_p2(v2): kA = u v1 A^{-T} e_a,
// kB = p2 u v2 A^{-T} e_b + u A^{-T} e_c.
// FP64 form: every entry binary64.  Mixed form: float-float complex entries; B and the
// per-node sums are compensated dot products in binary32, |m| >= m_hp in plain binary32.
template <int NT>
__device__ __forceinline__ void block_reduce_store2(double (&v)[EZ_MAX_PROD], double (&w)[EZ_MAX_PROD], int np,
                                                    double scale, double* out_v, double* out_w) {
  __shared__ double red[NT / 32][2 * EZ_MAX_PROD];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int p = 0; p < EZ_MAX_PROD; ++p) {
    double x = v[p], y = w[p];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      x += __shfl_down_sync(0xffffffffu, x, o);
      y += __shfl_down_sync(0xffffffffu, y, o);
    }
    if (lane == 0) {
      red[wid][p] = x;
      red[wid][EZ_MAX_PROD + p] = y;
    }
  }
  __syncthreads();
  if (threadIdx.x < 2 * EZ_MAX_PROD) {
    double s = 0.0;
    for (int q = 0; q < NT / 32; ++q) s += red[q][threadIdx.x];
    const int p = threadIdx.x % EZ_MAX_PROD;
    if (p < np) (threadIdx.x < EZ_MAX_PROD ? out_v : out_w)[p] = scale * s;
  }
  __syncthreads();  // red is reused by the next call
}

template <bool MIXED, int NDM>
__global__ void __launch_bounds__(256, (MIXED && NDM == 1) ? 3 : 2) far_kernel_d3(const ReqDesc* __restrict__ reqs,
                                                       const Item* __restrict__ items, double* __restrict__ seg) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ PhiInfo sphi[NDM];
  const Item it = items[blockIdx.x];
  const ReqDesc* R = reqs + it.req;
  const int nd = R->n_distinct, np = R->n_prod, nv = R->n_v, vch = R->vchunk;
  load_phi(sphi, R, nd);
  __shared__ typename std::conditional<MIXED, RecCacheMix, RecCacheF64>::type rcache;
  if constexpr (MIXED || NDM < 4) load_rec_cache(rcache, R);  // the whole list (else candidates per pass)

  const int j = it.sector >> 2;
  const int ax_a = j, ax_b = (j + 1) % 3;
  const double u = R->u_nodes[it.iu];
  const double wblk = 2.0 * R->u_w[it.iu] * u * u;
  const int Ma = R->M[ax_a], Mb = R->M[ax_b];
  const int v2_0 = it.chunk * vch, nv2 = min(vch, nv - v2_0);
  // segments of the four sectors 4 j + pb (pb = 1: p1 = -1, pb = 2: p2 = -1) of this chunk
  const long long sstride = (long long)R->n_ui * ((nv + vch - 1) / vch);

  double2* Ea = reinterpret_cast<double2*>(smem_raw);
  double2* Eb = Ea + (Ma + 1) * nv;
  double2* H = Eb + (Mb + 1) * vch;
  const int nH = (Ma + 1) * (2 * Mb + 1);
  double2* B = H + nd * nH;
  const int nBs = nd * (Ma + 1) * vch;  // entries of one B_p2
  float4* Ea4 = reinterpret_cast<float4*>(Ea);
  float4* Eb4 = reinterpret_cast<float4*>(Eb);
  float4* H4 = reinterpret_cast<float4*>(H);
  float4* B4 = reinterpret_cast<float4*>(B);
  double* zsm = reinterpret_cast<double*>(B + 2 * nBs);  // [nd][256]
  float2* zsm2 = reinterpret_cast<float2*>(zsm);
  float2* kA = reinterpret_cast<float2*>(zsm + nd * 256);  // [n_v][3]
  float2* kB = kA + 3 * nv;                                 // [2][vchunk][3]

  {  // H of the line group: nd nH 16-byte entries, contiguous in its slot
    const float4* src = reinterpret_cast<const float4*>(MIXED ? (const void*)R->hboxff : (const void*)R->hbox) +
                        (size_t)(j * R->n_ui + it.iu - R->hg_lo) * R->hslot;
    for (int e = threadIdx.x; e < nd * nH; e += blockDim.x) H4[e] = __ldg(src + e);
  }
  // (u, u^2, 2 log u, 1/u^2) of the block: the h = 0 term's t, log t, 1/t, sqrt t with the
  // direction table
  __shared__ double s_ublk[4];
  if (threadIdx.x == 0) {
    s_ublk[0] = u;
    s_ublk[1] = u * u;
    s_ublk[2] = R->dirlw ? 2.0 * log(u) : 0.0;
    s_ublk[3] = 1.0 / (u * u);
  }
  for (int v1 = threadIdx.x; v1 < nv; v1 += blockDim.x) {
    double sn, cs;
    sincospi(2.0 * (u * R->v_nodes[v1]), &sn, &cs);
    const double2 e1 = make_double2(cs, sn);
    double2 e = make_double2(1.0, 0.0);
    for (int ma = 0; ma <= Ma; ++ma) {
      if (ma) e = cmul(e, e1);
      if constexpr (MIXED)
        Ea4[ma * nv + v1] = ff_complex(e);
      else
        Ea[ma * nv + v1] = e;
    }
  }
  for (int v2l = threadIdx.x; v2l < nv2; v2l += blockDim.x) {
    double sn, cs;
    sincospi(2.0 * (u * R->v_nodes[v2_0 + v2l]), &sn, &cs);
    const double2 e1 = make_double2(cs, sn);
    double2 e = make_double2(1.0, 0.0);
    for (int mb = 0; mb <= Mb; ++mb) {
      if (mb) e = cmul(e, e1);
      if constexpr (MIXED)
        Eb4[mb * vch + v2l] = ff_complex(e);
      else
        Eb[mb * vch + v2l] = e;
    }
  }
  if constexpr (MIXED) {
    const int ax_c = (j + 2) % 3;
    for (int e = threadIdx.x; e < nv + 2 * nv2; e += blockDim.x) {
      if (e < nv) {
        const float2 a1 = __ldg(R->v_ff + e);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const ff t = ff_mul(ffd(R->AiTs[i * 3 + ax_a] * u), ff{a1.x, a1.y});
          kA[e * 3 + i] = make_float2(t.hi, t.lo);
        }
      } else {
        const int q = e - nv, s2 = q / nv2, v2l = q - s2 * nv2;
        const float2 a2 = __ldg(R->v_ff + v2_0 + v2l);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const ff t = ff_add(ff_mul(ffd(R->AiTs[i * 3 + ax_b] * (s2 ? -u : u)), ff{a2.x, a2.y}),
                              ffd(R->AiTs[i * 3 + ax_c] * u));
          kB[(s2 * vch + v2l) * 3 + i] = make_float2(t.hi, t.lo);
        }
      }
    }
  } else {
    // binary32 parts of k for the cutoff screen (k = kb + p1 ka per node): the binary32
    // roundings of the binary64 parts the node loop forms, one conversion per part and block
    const int ax_c = (j + 2) % 3;
    float* kAf = reinterpret_cast<float*>(kA);
    float* kBf = reinterpret_cast<float*>(kB);
    for (int e = threadIdx.x; e < nv + 2 * nv2; e += blockDim.x) {
      if (e < nv) {
        const double kta = u * R->v_nodes[e];
#pragma unroll
        for (int i = 0; i < 3; ++i) kAf[e * 3 + i] = (float)(R->AiTs[i * 3 + ax_a] * kta);
      } else {
        const int q = e - nv, s2 = q / nv2, v2l = q - s2 * nv2;
        const double ktb = u * (s2 ? -R->v_nodes[v2_0 + v2l] : R->v_nodes[v2_0 + v2l]);
#pragma unroll
        for (int i = 0; i < 3; ++i)
          kBf[(s2 * vch + v2l) * 3 + i] = (float)fma(R->AiTs[i * 3 + ax_b], ktb, R->AiTs[i * 3 + ax_c] * u);
      }
    }
  }
  // pref_j vol_fac per exponent: the FP64 node value is one FMA on the scaled B (below)
  __shared__ double s_pv[NDM];
  if (threadIdx.x < nd && threadIdx.x < NDM) s_pv[threadIdx.x] = R->pref[threadIdx.x] * R->vol_fac;
  __syncthreads();

  // B_{+-}(ma, v2) = X +- Y: one thread per (jn, ma, v2)
  const int nB = (Ma + 1) * nv2;
  for (int e = threadIdx.x; e < nd * nB; e += blockDim.x) {
    const int jn = e / nB, r = e - jn * nB;
    const int ma = r / nv2, v2l = r - ma * nv2;
    const int hb = (jn * (Ma + 1) + ma) * (2 * Mb + 1) + Mb;
    const int bo = (jn * (Ma + 1) + ma) * vch + v2l;
    if constexpr (MIXED) {
      const float4* h = H4 + hb;
      float xr = h[0].x, cxr = h[0].y, xi = h[0].z, cxi = h[0].w;
      float yr = 0.0f, cyr = 0.0f, yi = 0.0f, cyi = 0.0f;
      const int mb_hp = min(Mb + 1, R->m_hp[ax_b]);
      for (int mb = 1; mb < mb_hp; ++mb) {
        const float4 E = Eb4[mb * vch + v2l];
        const float4 hs = h[mb], hd = h[-mb];
        dot2_acc(xr, cxr, hs.x, hs.y, E.x, E.y);
        dot2_acc(yr, cyr, -hd.z, -hd.w, E.z, E.w);
        dot2_acc(xi, cxi, hs.z, hs.w, E.x, E.y);
        dot2_acc(yi, cyi, hd.x, hd.y, E.z, E.w);
      }
      for (int mb = mb_hp; mb <= Mb; ++mb) {  // below 1e-8: binary32
        const float4 E = Eb4[mb * vch + v2l];
        const float4 hs = h[mb], hd = h[-mb];
        cxr = fmaf(hs.x, E.x, cxr);
        cyr = fmaf(-hd.z, E.z, cyr);
        cxi = fmaf(hs.z, E.x, cxi);
        cyi = fmaf(hd.x, E.z, cyi);
      }
      const ff pr = ff_two_sum(xr, yr), pi = ff_two_sum(xi, yi);
      const ff mr = ff_two_sum(xr, -yr), mi = ff_two_sum(xi, -yi);
      const ff bpr = ff_fast_two_sum(pr.hi, pr.lo + (cxr + cyr)), bpi = ff_fast_two_sum(pi.hi, pi.lo + (cxi + cyi));
      const ff bmr = ff_fast_two_sum(mr.hi, mr.lo + (cxr - cyr)), bmi = ff_fast_two_sum(mi.hi, mi.lo + (cxi - cyi));
      B4[bo] = make_float4(bpr.hi, bpr.lo, bpi.hi, bpi.lo);
      B4[nBs + bo] = make_float4(bmr.hi, bmr.lo, bmi.hi, bmi.lo);
    } else {
      const double2* h = H + hb;
      double xr = h[0].x, xi = h[0].y, yr = 0.0, yi = 0.0;
      for (int mb = 1; mb <= Mb; ++mb) {
        const double2 E = Eb[mb * vch + v2l];
        const double2 hs = h[mb], hd = h[-mb];
        xr = fma(hs.x, E.x, xr);
        yr = fma(-hd.y, E.y, yr);
        xi = fma(hs.y, E.x, xi);
        yi = fma(hd.x, E.y, yi);
      }
      // scaled by pref_j, with -pref_j 2/nu_j in the real part of the m_a = 0 entry: the
      // node's Z_j = pref_j (Zp_j + vol_fac acc_j - 2/nu_j) is then one FMA on its Zp_j
      const double pf = R->pref[jn], c = ma == 0 ? pf * R->two_over_nu[jn] : 0.0;
      B[bo] = make_double2(fma(pf, xr + yr, -c), pf * (xi + yi));
      B[nBs + bo] = make_double2(fma(pf, xr - yr, -c), pf * (xi - yi));
    }
  }
  __syncthreads();

  const int ax_c = (j + 2) % 3;
  // 2 A^{-T} columns: the FP64 node loop forms 2k directly (exact scaling)
  double kca[3], kcb[3], kcc[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    kca[i] = 2.0 * R->AiTs[i * 3 + ax_a];
    kcb[i] = 2.0 * R->AiTs[i * 3 + ax_b];
    kcc[i] = 2.0 * R->AiTs[i * 3 + ax_c];
  }
  unsigned terms = 0, coefs = 0, qterms = 0;
  const int nn = nv * nv2;
  for (int s2 = 0; s2 < 2; ++s2) {  // p2 = +1, -1
    if constexpr (!MIXED && NDM >= 4) {  // candidates: k = u A^{-T} (alpha e_a + p2 beta e_b + e_c), alpha = p1 v1, beta = v2
      double c0[3], da[3], db[3];
      const double hu = 0.5 * u;  // the constants are doubled
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        c0[i] = kcc[i] * hu;
        da[i] = kca[i] * hu;
        db[i] = kcb[i] * (s2 ? -hu : hu);
      }
      double b0 = R->v_nodes[v2_0], b1 = b0;
      for (int q = 1; q < nv2; ++q) {
        b0 = fmin(b0, R->v_nodes[v2_0 + q]);
        b1 = fmax(b1, R->v_nodes[v2_0 + q]);
      }
      rec_candidates(rcache, R, c0, da, db, b0, b1);
    }
    double wsum[EZ_MAX_PROD] = {0.0, 0.0, 0.0, 0.0}, wneg[EZ_MAX_PROD] = {0.0, 0.0, 0.0, 0.0};
    if constexpr (MIXED) {
      const double4* dirlw = R->dirlw;
      ff ws[EZ_MAX_PROD] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
      ff wn[EZ_MAX_PROD] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
      const int ma_hp = min(Ma + 1, R->m_hp[ax_a]);
      const float4* Bs = B4 + s2 * nBs;
      for (int n = threadIdx.x; n < nn; n += blockDim.x) {
        const int v2l = n / nv, v1 = n - v2l * nv;
        const float2 w1 = __ldg(R->vw_ff + v1), w2 = __ldg(R->vw_ff + v2_0 + v2l);
        // S0 and S1 per exponent: two independent compensated chains, interleaved over the exponents
        ff Zp[NDM], A[NDM];
        float s0[NDM], c0[NDM], s1[NDM], c1[NDM];
#pragma unroll
        for (int jn = 0; jn < NDM; ++jn) s0[jn] = c0[jn] = s1[jn] = c1[jn] = 0.0f;
        const float4* bcol = Bs + v2l;
        for (int ma = 1; ma < ma_hp; ++ma) {
          const float4 E = Ea4[ma * nv + v1];
#pragma unroll
          for (int jn = 0; jn < NDM; ++jn)
            if (jn < nd) {
              const float4 bb = bcol[(jn * (Ma + 1) + ma) * vch];
              dot2_acc(s0[jn], c0[jn], E.x, E.y, bb.x, bb.y);
              dot2_acc(s1[jn], c1[jn], E.z, E.w, bb.z, bb.w);
            }
        }
        for (int ma = ma_hp; ma <= Ma; ++ma) {  // below 1e-8: binary32
          const float4 E = Ea4[ma * nv + v1];
#pragma unroll
          for (int jn = 0; jn < NDM; ++jn)
            if (jn < nd) {
              const float4 bb = bcol[(jn * (Ma + 1) + ma) * vch];
              c0[jn] = fmaf(E.x, bb.x, c0[jn]);
              c1[jn] = fmaf(E.z, bb.z, c1[jn]);
            }
        }
#pragma unroll
        for (int jn = 0; jn < NDM; ++jn)
          if (jn < nd) {
            const float4 b0 = bcol[jn * (Ma + 1) * vch];
            const ff tp = ff_two_sum(s0[jn], -s1[jn]), tm = ff_two_sum(s0[jn], s1[jn]);
            const ff Sp = ff_fast_two_sum(tp.hi, tp.lo + (c0[jn] - c1[jn]));
            const ff Sm = ff_fast_two_sum(tm.hi, tm.lo + (c0[jn] + c1[jn]));
            Zp[jn] = ff_add(ff{2.0f * Sp.hi, 2.0f * Sp.lo}, ff{b0.x, b0.y});
            const ff zm = ff_add(ff{2.0f * Sm.hi, 2.0f * Sm.lo}, ff{b0.x, b0.y});
            zsm2[jn * 256 + threadIdx.x] = make_float2(zm.hi, zm.lo);
          }
        const ff w = ff_mul(ff{w1.x, w1.y}, ff{w2.x, w2.y});
        ff ka[3], kb[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const float2 a = kA[v1 * 3 + i], b = kB[(s2 * vch + v2l) * 3 + i];
          ka[i] = ff{a.x, a.y};
          kb[i] = ff{b.x, b.y};
        }
#pragma unroll 1
        for (int q = 0; q < 2; ++q) {  // p1 = +1, then p1 = -1 (ka and Zp change, ws/wn swap)
          ff k[3];
#pragma unroll
          for (int i = 0; i < 3; ++i) k[i] = ff_add(kb[i], ka[i]);
          const NodeDir nd0{dirlw ? dirlw + (((size_t)(j * 2 + q) * 2 + s2) * nv + v2_0 + v2l) * nv + v1 : nullptr,
                            s_ublk};
          recip_sum_mixed<3, NDM>(R, sphi, nd, k, A, terms, coefs, rcache, nd0);
          assemble_mixed<NDM>(R, nd, np, Zp, A, w, ws);
#pragma unroll
          for (int i = 0; i < 3; ++i) ka[i] = ff{-ka[i].hi, -ka[i].lo};
#pragma unroll
          for (int jn = 0; jn < NDM; ++jn)
            if (jn < nd) {
              const float2 z = zsm2[jn * 256 + threadIdx.x];
              Zp[jn] = ff{z.x, z.y};
            }
#pragma unroll
          for (int p = 0; p < EZ_MAX_PROD; ++p) {
            const ff t = ws[p];
            ws[p] = wn[p];
            wn[p] = t;
          }
        }
      }
#pragma unroll
      for (int p = 0; p < EZ_MAX_PROD; ++p) {
        wsum[p] = (double)ws[p].hi + (double)ws[p].lo;
        wneg[p] = (double)wn[p].hi + (double)wn[p].lo;
      }
    } else {
      const double2* Bs = B + s2 * nBs;
      const double4* dirlw = R->dirlw;
      for (int n = threadIdx.x; n < nn; n += blockDim.x) {
        const int v2l = n / nv, v1 = n - v2l * nv;
        const double kta = u * R->v_nodes[v1];
        const double ktb = u * (s2 ? -R->v_nodes[v2_0 + v2l] : R->v_nodes[v2_0 + v2l]);
        const double wv = R->v_w[v1] * R->v_w[v2_0 + v2l];
        // 2k = 2kb + 2ka (p1 = +1), then 2kb - 2ka
        double ka[3], kb[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          ka[i] = kca[i] * kta;
          kb[i] = fma(kcb[i], ktb, kcc[i] * u);
        }
        double Zp[NDM];
#pragma unroll
        for (int jn = 0; jn < NDM; ++jn) {
          Zp[jn] = 0.0;
          if (jn < nd) {
            const double2* b = Bs + jn * (Ma + 1) * vch + v2l;
            double s0 = 0.0, s1 = 0.0;
            for (int ma = 1; ma <= Ma; ++ma) {
              const double2 E = Ea[ma * nv + v1];
              const double2 bb = b[ma * vch];
              s0 = fma(E.x, bb.x, s0);
              s1 = fma(E.y, bb.y, s1);
            }
            const double t0 = fma(2.0, s0, b[0].x);
            Zp[jn] = fma(-2.0, s1, t0);
            zsm[jn * 256 + threadIdx.x] = fma(2.0, s1, t0);
          }
        }
#pragma unroll 1
        for (int q = 0; q < 2; ++q) {  // p1 = +1, then p1 = -1 (ka and Zp change, wsum/wneg swap)
          double k[3], acc[NDM], Z[NDM];
#pragma unroll
          for (int i = 0; i < 3; ++i) k[i] = kb[i] + ka[i];
#pragma unroll
          for (int jn = 0; jn < NDM; ++jn) acc[jn] = 0.0;
          float kf[3];
          {
            const float* kaf = reinterpret_cast<const float*>(kA) + v1 * 3;
            const float* kbf = reinterpret_cast<const float*>(kB) + (s2 * vch + v2l) * 3;
#pragma unroll
            for (int i = 0; i < 3; ++i) kf[i] = q ? kbf[i] - kaf[i] : kbf[i] + kaf[i];
          }
          const NodeDir nd0{dirlw ? dirlw + (((size_t)(j * 2 + q) * 2 + s2) * nv + v2_0 + v2l) * nv + v1 : nullptr,
                            s_ublk};
          recip_sum<3, NDM, true>(R, sphi, nd, k, kf, acc, terms, coefs, qterms, rcache, nd0);
#pragma unroll
          for (int jn = 0; jn < NDM; ++jn)
            if (jn < nd) Z[jn] = fma(s_pv[jn], acc[jn], Zp[jn]);
          products<NDM, true>(R, nd, np, Z, wv, wsum);
#pragma unroll
          for (int i = 0; i < 3; ++i) ka[i] = -ka[i];
#pragma unroll
          for (int jn = 0; jn < NDM; ++jn)
            if (jn < nd) Zp[jn] = zsm[jn * 256 + threadIdx.x];
#pragma unroll
          for (int p = 0; p < EZ_MAX_PROD; ++p) {
            const double t = wsum[p];
            wsum[p] = wneg[p];
            wneg[p] = t;
          }
        }
      }
    }
    double* o = seg + (size_t)it.chunk_seg() * EZ_MAX_PROD;
    block_reduce_store2<256>(wsum, wneg, np, wblk, o + (size_t)(2 * s2) * sstride * EZ_MAX_PROD,
                             o + (size_t)(2 * s2 + 1) * sstride * EZ_MAX_PROD);
  }
  count_work(R, terms, coefs, MIXED ? terms : qterms);
}

// ------------------------------------------------------------------------- d = 2

template <bool MIXED, int NDM>
__device__ __forceinline__ void far_d2_body(const ReqDesc* __restrict__ reqs, const Item* __restrict__ items,
                                            double* __restrict__ seg) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ PhiInfo sphi[NDM];
  const Item it = items[blockIdx.x];
  const ReqDesc* R = reqs + it.req;
  const int nd = R->n_distinct, np = R->n_prod, nv = R->n_v;
  load_phi(sphi, R, nd);
  __shared__ typename std::conditional<MIXED, RecCacheMix, RecCacheF64>::type rcache;
  load_rec_cache(rcache, R);
  const int j = it.sector >> 1;
  const double p1 = (it.sector & 1) ? -1.0 : 1.0;
  const int ax_a = j, ax_c = 1 - j;
  const double u = R->u_nodes[it.iu];
  const double wblk = 2.0 * R->u_w[it.iu] * u;
  const int Ma = R->M[ax_a], Mc = R->M[ax_c];
  const int st[2] = {R->box[1], 1};
  const int sta = st[ax_a], stc = st[ax_c];
  const int gbase = R->M[0] * st[0] + R->M[1] * st[1];
  const long long cells = (long long)R->box[0] * R->box[1];
  double2* Ec = reinterpret_cast<double2*>(smem_raw);
  double2* H = Ec + (Mc + 1);
  if (threadIdx.x <= Mc) {
    double sn, cs;
    sincospi(2.0 * ((double)threadIdx.x * u), &sn, &cs);
    Ec[threadIdx.x] = make_double2(cs, sn);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nd * (Ma + 1); e += blockDim.x) {
    const int jn = e / (Ma + 1), ma = e - jn * (Ma + 1);
    const double* g = R->gbox + (size_t)jn * cells + gbase + ma * sta;
    double hr = g[0], hi = 0.0;
    for (int mc = 1; mc <= Mc; ++mc) {
      const double gp = g[mc * stc], gm = g[-mc * stc];
      hr = fma(gp + gm, Ec[mc].x, hr);
      hi = fma(gp - gm, Ec[mc].y, hi);
    }
    if constexpr (MIXED)
      reinterpret_cast<float4*>(H)[e] = ff_complex(make_double2(hr, hi));
    else
      H[e] = make_double2(hr, hi);
  }
  __syncthreads();
  const double kca0 = R->AiTs[0 * 2 + ax_a], kca1 = R->AiTs[1 * 2 + ax_a];
  const double kcc0 = R->AiTs[0 * 2 + ax_c], kcc1 = R->AiTs[1 * 2 + ax_c];
  double wsum[EZ_MAX_PROD] = {0.0, 0.0, 0.0, 0.0};
  unsigned terms = 0, coefs = 0, qterms = 0;
  if constexpr (MIXED) {
    // k = alpha v + gamma in float-float; real space by compensated dot products on the
    // float-float phase table (conjugated for p1 = -1) and H
    const float4* H4 = reinterpret_cast<const float4*>(H);
    const ff al[2] = {ffd(kca0 * (u * p1)), ffd(kca1 * (u * p1))};
    const ff ga[2] = {ffd(kcc0 * u), ffd(kcc1 * u)};
    const float sg = (float)p1;
    const int ma_hp = min(Ma + 1, R->m_hp[ax_a]);
    ff ws[EZ_MAX_PROD] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
    for (int v = threadIdx.x; v < nv; v += blockDim.x) {
      const float2 a = __ldg(R->v_ff + v), wv = __ldg(R->vw_ff + v);
      const ff x{a.x, a.y};
      const ff k[2] = {ff_add(ff_mul(al[0], x), ga[0]), ff_add(ff_mul(al[1], x), ga[1])};
      const float4* ph = R->phaseff + ((size_t)it.iu * nv + v) * R->phase_mp1;
      float s[NDM], c[NDM], s1[NDM], c1[NDM];  // real and imaginary product chains
#pragma unroll
      for (int jn = 0; jn < NDM; ++jn) s[jn] = c[jn] = s1[jn] = c1[jn] = 0.0f;
      for (int ma = 1; ma < ma_hp; ++ma) {
        const float4 e = __ldg(ph + ma);
#pragma unroll
        for (int jn = 0; jn < NDM; ++jn)
          if (jn < nd) {
            const float4 hh = H4[jn * (Ma + 1) + ma];
            dot2_acc(s[jn], c[jn], e.x, e.y, hh.x, hh.y);
            dot2_acc(s1[jn], c1[jn], -sg * e.z, -sg * e.w, hh.z, hh.w);
          }
      }
      for (int ma = ma_hp; ma <= Ma; ++ma) {  // below 1e-8: binary32
        const float4 e = __ldg(ph + ma);
#pragma unroll
        for (int jn = 0; jn < NDM; ++jn)
          if (jn < nd) {
            const float4 hh = H4[jn * (Ma + 1) + ma];
            c[jn] = fmaf(e.x, hh.x, fmaf(-sg * e.z, hh.z, c[jn]));
          }
      }
      ff Zr[NDM], A[NDM];
#pragma unroll
      for (int jn = 0; jn < NDM; ++jn)
        if (jn < nd) {
          const ff t = ff_two_sum(s[jn], s1[jn]);
          const ff S = ff_fast_two_sum(t.hi, t.lo + (c[jn] + c1[jn]));
          const float4 h0 = H4[jn * (Ma + 1)];
          Zr[jn] = ff_add(ff{2.0f * S.hi, 2.0f * S.lo}, ff{h0.x, h0.y});
        }
      recip_sum_mixed<2, NDM>(R, sphi, nd, k, A, terms, coefs, rcache, NodeDir{nullptr, nullptr});
      assemble_mixed<NDM>(R, nd, np, Zr, A, ff{wv.x, wv.y}, ws);
    }
#pragma unroll
    for (int p = 0; p < EZ_MAX_PROD; ++p) wsum[p] = (double)ws[p].hi + (double)ws[p].lo;
  } else
  for (int v = threadIdx.x; v < nv; v += blockDim.x) {
    const double kta = u * (p1 * R->v_nodes[v]);
    const double wv = R->v_w[v];
    double k[2] = {fma(kca0, kta, kcc0 * u), fma(kca1, kta, kcc1 * u)};
    // e^{2 pi i ma kta} = (e^{2 pi i ma u v})^* for p1 = -1: conjugation is exact in the table
    const double2* ph = R->phase + ((size_t)it.iu * nv + v) * R->phase_mp1;
    const double sgn = p1;
    double sr[NDM], Z[NDM], acc[NDM];
#pragma unroll
    for (int jn = 0; jn < NDM; ++jn) sr[jn] = acc[jn] = 0.0;
    for (int ma = 1; ma <= Ma; ++ma) {
      const double2 e = ph[ma];
      const double ey = sgn * e.y;
#pragma unroll
      for (int jn = 0; jn < NDM; ++jn)
        if (jn < nd) {
          const double2 hh = H[jn * (Ma + 1) + ma];
          sr[jn] = fma(e.x, hh.x, fma(-ey, hh.y, sr[jn]));
        }
    }
#pragma unroll
    for (int jn = 0; jn < NDM; ++jn)
      if (jn < nd) Z[jn] = fma(2.0, sr[jn], H[jn * (Ma + 1)].x);
    const float kf[2] = {(float)k[0], (float)k[1]};
    recip_sum<2, NDM>(R, sphi, nd, k, kf, acc, terms, coefs, qterms, rcache, NodeDir{nullptr, nullptr});
#pragma unroll
    for (int jn = 0; jn < NDM; ++jn)
      if (jn < nd) Z[jn] = R->pref[jn] * (Z[jn] + R->vol_fac * acc[jn] - R->two_over_nu[jn]);
    products<NDM>(R, nd, np, Z, wv, wsum);
  }
  count_work(R, terms, coefs, MIXED ? terms : qterms);
  block_reduce_store<128>(wsum, np, wblk, seg + (size_t)it.chunk_seg() * EZ_MAX_PROD);
}

template <bool MIXED, int NDM>
__global__ void __launch_bounds__(128) far_kernel_d2(const ReqDesc* __restrict__ reqs, const Item* __restrict__ items,
                                                     double* __restrict__ seg) {
  far_d2_body<MIXED, NDM>(reqs, items, seg);
}
// the single-exponent mixed variant trades a few spills for 32 resident warps per SM
__global__ void __launch_bounds__(128, 8) far_kernel_d2_mixed1(const ReqDesc* __restrict__ reqs,
                                                               const Item* __restrict__ items,
                                                               double* __restrict__ seg) {
  far_d2_body<true, 1>(reqs, items, seg);
}

// ------------------------------------------------------------------------- d = 1
template <bool MIXED, int NDM>
__global__ void __launch_bounds__(128) far_kernel_d1(const ReqDesc* __restrict__ reqs,
                                                       const Item* __restrict__ items, double* __restrict__ seg) {
  __shared__ PhiInfo sphi[NDM];
  const Item it = items[blockIdx.x];
  const ReqDesc* R = reqs + it.req;
  const int nd = R->n_distinct, np = R->n_prod;
  load_phi(sphi, R, nd);
  __shared__ typename std::conditional<MIXED, RecCacheMix, RecCacheF64>::type rcache;
  load_rec_cache(rcache, R);
  __syncthreads();
  const int iu = it.iu + threadIdx.x;
  if (iu >= R->n_ui) return;
  const double u = R->u_nodes[iu];
  const double w = 2.0 * R->u_w[iu];
  const int M = R->M[0];
  unsigned terms = 0, coefs = 0, qterms = 0;
  double f[EZ_MAX_PROD] = {0.0, 0.0, 0.0, 0.0};
  if constexpr (MIXED) {
    const ff k[1] = {ffd(R->AiTs[0] * u)};
    const float4* ph = R->phaseff + (size_t)iu * R->phase_mp1;
    float s[NDM], c[NDM];
#pragma unroll
    for (int jn = 0; jn < NDM; ++jn) s[jn] = c[jn] = 0.0f;
    for (int m = 1; m <= M; ++m) {
      const float4 e = __ldg(ph + m);
#pragma unroll
      for (int jn = 0; jn < NDM; ++jn)
        if (jn < nd) {
          const float2 g = __ldg(R->gboxff + (size_t)jn * R->box[0] + M + m);
          dot2_acc(s[jn], c[jn], g.x, g.y, e.x, e.y);
        }
    }
    ff Zr[NDM], A[NDM];
#pragma unroll
    for (int jn = 0; jn < NDM; ++jn)
      if (jn < nd) {
        const ff S = ff_two_sum(s[jn], c[jn]);
        Zr[jn] = ff{2.0f * S.hi, 2.0f * S.lo};
      }
    recip_sum_mixed<1, NDM>(R, sphi, nd, k, A, terms, coefs, rcache, NodeDir{nullptr, nullptr});
    ff ws[EZ_MAX_PROD] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
    assemble_mixed<NDM>(R, nd, np, Zr, A, ffd(w), ws);
#pragma unroll
    for (int p = 0; p < EZ_MAX_PROD; ++p) f[p] = (double)ws[p].hi + (double)ws[p].lo;
  } else {
  double k[1] = {R->AiTs[0] * u};
  const double2* ph = R->phase + (size_t)iu * R->phase_mp1;
  double sr[NDM], acc[NDM], Z[NDM];
#pragma unroll
  for (int jn = 0; jn < NDM; ++jn) sr[jn] = acc[jn] = 0.0;
  for (int m = 1; m <= M; ++m) {
    const double ex = ph[m].x;
#pragma unroll
    for (int jn = 0; jn < NDM; ++jn)
      if (jn < nd) sr[jn] = fma(R->gbox[(size_t)jn * R->box[0] + M + m], ex, sr[jn]);
  }
  const float kf[1] = {(float)k[0]};
  recip_sum<1, NDM>(R, sphi, nd, k, kf, acc, terms, coefs, qterms, rcache, NodeDir{nullptr, nullptr});
#pragma unroll
  for (int jn = 0; jn < NDM; ++jn)
    if (jn < nd) Z[jn] = R->pref[jn] * (2.0 * sr[jn] + R->vol_fac * acc[jn] - R->two_over_nu[jn]);
  products<NDM>(R, nd, np, Z, w, f);
  }
  double* o = seg + (size_t)(it.chunk_seg() + threadIdx.x) * EZ_MAX_PROD;
  for (int p = 0; p < np; ++p) o[p] = f[p];
  if (R->work) {  // lanes beyond n_ui left early: sum over the lanes still active
    const unsigned am = __activemask();
    const unsigned t = __reduce_add_sync(am, terms), c = __reduce_add_sync(am, coefs);
    const unsigned q = __reduce_add_sync(am, MIXED ? terms : qterms);
    if ((int)(threadIdx.x & 31) == __ffs(am) - 1) {
      atomicAdd(R->work, (unsigned long long)t);
      atomicAdd(R->work + 1, (unsigned long long)c);
      atomicAdd(R->work + 2, (unsigned long long)q);
    }
  }
}


// ------------------------------------------------------------------------- near part
// One thread per ray (sector, v): C_{k,nu}(w) = sum_{|alpha| = 2k} D_nu[alpha] w^alpha, then
// every product expanded over how many of each factor's singular parts s_hat/V enter,
// integrated on (0, eps) in closed form (Hadamard finite part):
//   I_m(mu) = eps^mu J_m,  J_0 = 1/mu,  J_m = L^m/mu - (2m/mu) J_{m-1},  L = log(pi eps^2 |w|^2).
// 1/n for |n| <= kInvIntHalf (n = 0 unused), filled once by upload_inv_int
__constant__ double c_inv_int[2 * kInvIntHalf + 1];

cudaError_t upload_inv_int() {
  double t[2 * kInvIntHalf + 1];
  for (int n = -kInvIntHalf; n <= kInvIntHalf; ++n) t[n + kInvIntHalf] = n ? 1.0 / n : 0.0;
  return cudaMemcpyToSymbol(c_inv_int, t, sizeof t);
}

__device__ double ipow(double x, int e) {
  double r = 1.0, b = x;
  int k = e < 0 ? -e : e;
  while (k) {
    if (k & 1) r *= b;
    b *= b;
    k >>= 1;
  }
  return e < 0 ? 1.0 / r : r;
}

// Number type of the near part (binary64 in both forms: the near part is the
// integral of the singular subtraction at k -> 0).
__device__ __forceinline__ double nfma(double a, double b, double c) { return fma(a, b, c); }
template <typename N>
__device__ __forceinline__ N nfrom(double x);
template <>
__device__ __forceinline__ double nfrom<double>(double x) {
  return x;
}
// exact conversion of an integer |v| < 2^48 (binomial products, small multipliers)
template <typename N>
__device__ __forceinline__ N nint(long long v);
template <>
__device__ __forceinline__ double nint<double>(long long v) {
  return (double)v;
}
__device__ __forceinline__ double nto(double x) { return x; }
__device__ __forceinline__ double ninv(double, int mk) {
  return (mk >= -kInvIntHalf && mk <= kInvIntHalf) ? c_inv_int[mk + kInvIntHalf] : 1.0 / (double)mk;
}
template <typename N>
__device__ __forceinline__ N npow(N x, int e) {  // e >= 0
  N r = nint<N>(1);
  while (e) {
    if (e & 1) r = r * x;
    x = x * x;
    e >>= 1;
  }
  return r;
}
// eps or 1/eps of the near part (set on the host)
template <typename N>
__device__ __forceinline__ N neps(const ReqDesc* R, bool inv);
template <>
__device__ __forceinline__ double neps<double>(const ReqDesc* R, bool inv) {
  return inv ? R->inv_eps : R->eps;
}
__device__ __forceinline__ double ntaylor(const ReqDesc* R, int jn, int ia, double) {
  return R->taylor[(size_t)jn * R->n_alpha + ia];
}

// sig_w[j] = sigma_j |w|^{nu_j - d} / V (per ray, shared by every product and subset)
template <typename N>
__device__ N near_product(const ReqDesc* R, int p, const N (*C)[kMaxEll + 1], const N* sig_w, N L, const N* PW,
                         const int (*pw_off)[kNearPowE + 1]) {
  const int nd = R->n_distinct, d = R->d, ell = R->ell;
  int e[EZ_MAX_NU], t[EZ_MAX_NU];
  for (int j = 0; j < nd; ++j) {
    e[j] = R->expo[p][j];
    t[j] = 0;
  }
  N total = nint<N>(0);
  N G[kNearMaxDeg + 1], T[kNearMaxDeg + 1];
  const N eps = neps<N>(R, false), inv_eps = neps<N>(R, true), eps2 = eps * eps;
  const bool int_mu = R->near_int_mu != 0;  // every nu_j - d an integer: integer mu, tabulated 1/n
  while (true) {
    N coef = nint<N>(1);
    long long mult = 1;  // product of binomials (exact integers)
    int mu = d, mlog = 0;
    double mu_r = d;  // real mu (non-integer exponents)
    for (int j = 0; j < nd; ++j) {
      if (t[j]) {
        long long bj = 1;
        for (int i = 1; i <= t[j]; ++i) bj = bj * (e[j] - t[j] + i) / i;
        mult *= bj;
        for (int i = 0; i < t[j]; ++i) coef = coef * sig_w[j];
        if (int_mu) mu += t[j] * ((int)lrint(R->nu[j]) - d);
        mu_r += t[j] * (R->nu[j] - d);
        mlog += t[j] * R->islog[j];
      }
    }
    int deg = 0;
    G[0] = nint<N>(1);
    if (PW) {  // products of the tabulated powers C_j^r (one convolution per further factor j)
      deg = -1;
      for (int j = 0; j < nd; ++j) {
        const int r = e[j] - t[j];
        if (r == 0) continue;
        const N* src = r == 1 ? C[j] : PW + pw_off[j][r];
        const int sdeg = min(ell * r, kNearMaxDeg);
        if (deg < 0) {
          for (int i = 0; i <= sdeg; ++i) G[i] = src[i];
          deg = sdeg;
          continue;
        }
        const int nd2 = min(deg + sdeg, kNearMaxDeg);
        for (int i = 0; i <= nd2; ++i) {
          N s = nint<N>(0);
          for (int q = max(0, i - sdeg); q <= min(i, deg); ++q) s = nfma(G[q], src[i - q], s);
          T[i] = s;
        }
        deg = nd2;
        for (int i = 0; i <= deg; ++i) G[i] = T[i];
      }
      if (deg < 0) {
        G[0] = nint<N>(1);
        deg = 0;
      }
    } else {
      for (int j = 0; j < nd; ++j)
        for (int r = 0; r < e[j] - t[j]; ++r) {
          const int nd2 = min(deg + ell, kNearMaxDeg);
          for (int i = 0; i <= nd2; ++i) {
            N s = nint<N>(0);
            for (int q = max(0, i - ell); q <= min(i, deg); ++q) s = nfma(G[q], C[j][i - q], s);
            T[i] = s;
          }
          deg = nd2;
          for (int i = 0; i <= deg; ++i) G[i] = T[i];
        }
    }
    N sumk = nint<N>(0);
    if (R->hadw) {  // integer mu: tabulated coefficients of the weight's polynomial in L
      const int m1 = R->hadw_m1;
      const double* q = R->hadw + ((size_t)(mu - R->hadw_lo) * m1 + mlog) * m1;
      for (int k = 0; k <= deg; ++k, q += 2 * m1 * m1) {
        N W = q[mlog];
        for (int i = mlog - 1; i >= 0; --i) W = nfma(W, L, q[i]);
        sumk = nfma(G[k], W, sumk);
      }
      total = nfma(nint<N>(mult) * coef, sumk, total);
    } else {
    N epm = int_mu ? (mu >= 0 ? npow(eps, mu) : npow(inv_eps, -mu)) : exp(mu_r * log(eps));
    for (int k = 0; k <= deg; ++k) {
      // J_0 = 1/mu_k, J_i = (L^i - 2 i J_{i-1}) / mu_k with 1/mu_k from the table of
      // reciprocals of small integers (no division in the loop) when mu is an integer
      const int mk = mu + 2 * k;
      const N inv = int_mu ? ninv(epm, mk) : 1.0 / (mu_r + 2 * k);
      N J = inv, Lp = nint<N>(1);
      for (int i = 1; i <= mlog; ++i) {
        Lp = Lp * L;
        J = (Lp + J * nint<N>(-2 * i)) * inv;
      }
      sumk = nfma(G[k], epm * J, sumk);
      epm = epm * eps2;
    }
    total = nfma(nint<N>(mult) * coef, sumk, total);
    }
    int j = 0;
    for (; j < nd; ++j) {
      if (t[j] < e[j]) {
        t[j]++;
        break;
      }
      t[j] = 0;
    }
    if (j == nd) break;
  }
  return total;
}

// one ray: C_k(w) of every exponent, then every product's near integral (scale 2 w_v)
template <typename N>
__device__ void near_core(const ReqDesc* R, const N* wN, N L, const N* sig_w, double scale,
                          double (&val)[EZ_MAX_PROD]) {
  const int ell = R->ell, nd = R->n_distinct, np = R->n_prod;
  // C_k(w) = sum_{|alpha| = 2k} D[alpha] w^alpha: one monomial per alpha (powers of w
  // tabulated once), shared by every exponent
  N pw[3][2 * kMaxEll + 1];
  for (int i = 0; i < 3; ++i) {
    pw[i][0] = nint<N>(1);
    for (int q = 1; q <= 2 * ell; ++q) pw[i][q] = pw[i][q - 1] * wN[i];
  }
  N C[EZ_MAX_NU][kMaxEll + 1];
  for (int jn = 0; jn < nd; ++jn)
    for (int kk = 0; kk <= ell; ++kk) C[jn][kk] = nint<N>(0);
  for (int kk = 0; kk <= ell; ++kk)
    for (int ia = R->alpha_off[kk]; ia < R->alpha_off[kk + 1]; ++ia) {
      const int* al = R->alpha + 3 * ia;
      const N mono = pw[0][al[0]] * pw[1][al[1]] * pw[2][al[2]];
      for (int jn = 0; jn < nd; ++jn) C[jn][kk] = nfma(ntaylor(R, jn, ia, mono), mono, C[jn][kk]);
    }
  // powers C_j^r, 2 <= r <= max over the products of e_pj, tabulated once per ray when they fit
  N PW[kNearPowCache];
  int pw_off[EZ_MAX_NU][kNearPowE + 1];
  bool use_pw = true;
  int used = 0;
  for (int jn = 0; jn < nd && use_pw; ++jn) {
    int emax = 0;
    for (int p = 0; p < np; ++p) emax = max(emax, R->expo[p][jn]);
    if (emax > kNearPowE) {
      use_pw = false;
      break;
    }
    for (int r = 2; r <= emax; ++r) {
      const int dg = min(ell * r, kNearMaxDeg), dp = min(ell * (r - 1), kNearMaxDeg);
      if (used + dg + 1 > kNearPowCache) {
        use_pw = false;
        break;
      }
      const N* prev = r == 2 ? C[jn] : PW + pw_off[jn][r - 1];
      N* dst = PW + used;
      for (int i = 0; i <= dg; ++i) {  // C^r = C^{r-1} C, truncated at kNearMaxDeg
        N sv = nint<N>(0);
        for (int q = max(0, i - ell); q <= min(i, dp); ++q) sv = nfma(prev[q], C[jn][i - q], sv);
        dst[i] = sv;
      }
      pw_off[jn][r] = used;
      used += dg + 1;
    }
  }
  for (int p = 0; p < np; ++p) val[p] = scale * nto(near_product<N>(R, p, C, sig_w, L, use_pw ? PW : nullptr, pw_off));
}

// per-ray inputs in binary64 (both forms)
__device__ void near_ray_f64(const ReqDesc* R, const double* dir, double wv, double (&val)[EZ_MAX_PROD]) {
  const int d = R->d, nd = R->n_distinct;
  double w[3] = {0.0, 0.0, 0.0}, w2 = 0.0;
  for (int i = 0; i < d; ++i) {
    double s = 0.0;
    for (int q = 0; q < d; ++q) s = fma(R->AiT[i * d + q], dir[q], s);
    w[i] = s;
    w2 = fma(s, s, w2);
  }
  const double L = log(kPi * R->eps * R->eps * w2);
  const double wn = sqrt(w2), inv_wn = 1.0 / wn, inv_V = 1.0 / R->V;
  double sig_w[EZ_MAX_NU];
  for (int jn = 0; jn < nd; ++jn) {
    const double dr = R->nu[jn] - d;
    const int dn = (int)lrint(dr);
    const double pw = fabs(dr - dn) < 1e-12 ? (dn >= 0 ? ipow(wn, dn) : ipow(inv_wn, -dn)) : exp(dr * log(wn));
    sig_w[jn] = R->sig[jn] * pw * inv_V;
  }
  near_core<double>(R, w, L, sig_w, 2.0 * wv, val);
}

__global__ void __launch_bounds__(128) near_kernel(const ReqDesc* __restrict__ reqs, const Item* __restrict__ items,
                                                   double* __restrict__ seg) {
  const Item it = items[blockIdx.x];
  const ReqDesc* R = reqs + it.req;
  const int d = R->d, nv = R->n_v, np = R->n_prod;
  const int nrays = d == 1 ? 1 : (d == 2 ? nv : nv * nv);
  const int r = it.chunk * blockDim.x + threadIdx.x;
  double val[EZ_MAX_PROD] = {0.0, 0.0, 0.0, 0.0};
  if (r < nrays) {
    double v[2] = {0.0, 0.0}, wv = 1.0;
    if (d >= 2) {
      v[0] = R->v_nodes[r % nv];
      wv *= R->v_w[r % nv];
    }
    if (d == 3) {
      v[1] = R->v_nodes[r / nv];
      wv *= R->v_w[r / nv];
    }
    const int half = 1 << (d - 1);
    const int j = it.sector / half, pb = it.sector % half;
    double y[3], dir[3];
    for (int i = 0; i < d - 1; ++i) y[i] = (((pb >> i) & 1) ? -1.0 : 1.0) * v[i];
    y[d - 1] = 1.0;
    for (int i = 0; i < d; ++i) dir[i] = y[((i - j) % d + d) % d];
    near_ray_f64(R, dir, wv, val);
  }
  block_reduce_store<128>(val, np, 1.0, seg + (size_t)it.chunk_seg() * EZ_MAX_PROD);
}

__global__ void lines_kernel(const ReqDesc* reqs, const int* line_req, const long long* line_seg0,
                             const int* line_nseg, int n_lines, const double* seg, double* lines) {
  const int L = blockIdx.x * blockDim.x + threadIdx.x;
  if (L >= n_lines) return;
  const int np = reqs[line_req[L]].n_prod;
  for (int p = 0; p < EZ_MAX_PROD; ++p) {
    double s = 0.0;
    if (p < np)
      for (int q = 0; q < line_nseg[L]; ++q) s += seg[(size_t)(line_seg0[L] + q) * EZ_MAX_PROD + p];
    lines[(size_t)L * EZ_MAX_PROD + p] = s;
  }
}

// Compensated (Neumaier) sum of a request's lines, each line formed from its segments in
// the order lines_kernel adds them (the total does not depend on whether the lines are
// written).  One block of 128 threads per request:
// thread (slot j, product p) sums lines j, j + 32, j + 64, ... in order (eight at a time,
// each group plainly and the groups with compensation); the 32 partial sums of each product
// are then added in slot order.  The order is fixed, so the result does not depend on the
// batch the request runs in.
__device__ __forceinline__ void neumaier_add(double& s, double& c, double x) {
  const double t = s + x;
  c += fabs(s) >= fabs(x) ? (s - t) + x : (x - t) + s;
  s = t;
}

__global__ void total_kernel(const ReqDesc* reqs, const long long* req_line0, const int* req_nlines, int n_req,
                             const long long* line_seg0, const int* line_nseg, const double* seg, double* out) {
  static_assert(EZ_MAX_PROD == 4, "128 threads = 32 slots x 4 products");
  const int r = blockIdx.x;
  if (r >= n_req) return;
  const int p = threadIdx.x & 3, j = threadIdx.x >> 2;
  const int nl = req_nlines[r];
  const long long l0 = req_line0[r];
  // line q of the request: its segments added in order from 0, as lines_kernel adds them
  auto line = [&](int q) {
    const long long L = l0 + q;
    const double* sp = seg + (size_t)line_seg0[L] * EZ_MAX_PROD + p;
    const int ns = line_nseg[L];
    double v = 0.0;
    for (int k = 0; k < ns; ++k) v += sp[(size_t)k * EZ_MAX_PROD];
    return v;
  };
  // groups of eight of the thread's lines summed plainly, each group added with Neumaier's
  // compensation (error <= 8 ulp of the group's magnitude, at a third of the binary64
  // operations of a compensated step per line)
  double s = 0.0, c = 0.0;
  int q = j;
  for (; q + 7 * 32 < nl; q += 8 * 32) {
    double g = line(q);
#pragma unroll
    for (int k = 1; k < 8; ++k) g += line(q + k * 32);
    neumaier_add(s, c, g);
  }
  for (; q < nl; q += 32) neumaier_add(s, c, line(q));
  __shared__ double ps[128], pc[128];
  ps[threadIdx.x] = s;
  pc[threadIdx.x] = c;
  __syncthreads();
  if (j == 0) {
    double S = 0.0, C = 0.0;
    for (int q = 0; q < 32; ++q) {
      neumaier_add(S, C, ps[q * 4 + p]);
      C += pc[q * 4 + p];
    }
    out[(size_t)r * EZ_MAX_PROD + p] = p < reqs[r].n_prod ? S + C : 0.0;
  }
}

// ------------------------------------------------------------------------- launch
// Far-field variants: binary64 or mixed form, at most NDM in {1, 4, 8} distinct exponents
// (the per-node arrays are sized by NDM, which keeps the register count of the common
// single-exponent sums low).
template <bool MIXED, int NDM>
static cudaError_t launch_far_t(int d, unsigned grid, size_t smem, cudaStream_t st, const ReqDesc* reqs,
                                const Item* items, double* seg) {
  if (d == 1)
    far_kernel_d1<MIXED, NDM><<<grid, 128, 0, st>>>(reqs, items, seg);
  else if (d == 2 && MIXED && NDM == 1)
    far_kernel_d2_mixed1<<<grid, 128, smem, st>>>(reqs, items, seg);
  else if (d == 2)
    far_kernel_d2<MIXED, NDM><<<grid, 128, smem, st>>>(reqs, items, seg);
  else
    far_kernel_d3<MIXED, NDM><<<grid, 256, smem, st>>>(reqs, items, seg);
  return cudaGetLastError();
}

cudaError_t launch_far(int d, bool mixed, int ndm, unsigned grid, size_t smem, cudaStream_t st,
                       const ReqDesc* reqs, const Item* items, double* seg) {
  if (mixed) {
    if (ndm == 1) return launch_far_t<true, 1>(d, grid, smem, st, reqs, items, seg);
    if (ndm == 4) return launch_far_t<true, 4>(d, grid, smem, st, reqs, items, seg);
    return launch_far_t<true, 8>(d, grid, smem, st, reqs, items, seg);
  }
  if (ndm == 1) return launch_far_t<false, 1>(d, grid, smem, st, reqs, items, seg);
  if (ndm == 4) return launch_far_t<false, 4>(d, grid, smem, st, reqs, items, seg);
  return launch_far_t<false, 8>(d, grid, smem, st, reqs, items, seg);
}

template <bool MIXED, int NDM>
static cudaError_t far_smem_limits_t() {
  cudaError_t e = cudaFuncSetAttribute(far_kernel_d3<MIXED, NDM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       200 * 1024);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(far_kernel_d2<MIXED, NDM>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
}

cudaError_t far_set_smem_limits() {
  cudaError_t e = cudaFuncSetAttribute(far_kernel_d2_mixed1, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
  if (e != cudaSuccess) return e;
  if ((e = far_smem_limits_t<false, 1>()) != cudaSuccess) return e;
  if ((e = far_smem_limits_t<false, 4>()) != cudaSuccess) return e;
  if ((e = far_smem_limits_t<false, 8>()) != cudaSuccess) return e;
  if ((e = far_smem_limits_t<true, 1>()) != cudaSuccess) return e;
  if ((e = far_smem_limits_t<true, 4>()) != cudaSuccess) return e;
  return far_smem_limits_t<true, 8>();
}

}  // namespace ez
