// cs_cta_elliptic.cuh -- the round-cone fused solve and IFT adjoint for
// instances beyond one warp (nv up to 128, m up to 1024 rows = 341
// contacts), one 256-thread CTA per instance (device code).
//
// The method of cs_elliptic.cuh (Section III-A, Eqs. 2-5 with Eqs. 6-10 and
// 17): each contact's zone, gradient in float-pair arithmetic and 3 x 3
// Hessian block from cone_eval(); H = M + sum_c J_c^T hess_c J_c; the convex
// line search by safeguarded Newton on phi' with the quadratic model near
// convergence; Newton directions from one FP32 solve of the compensated
// residual; the adjoint from a refined solve; the cone parameters'
// gradients.  The work is spread over the block: rows as in
// the CTA solver (thread t owns rows t + 256 u), contact c owned by thread
// c mod 256 (at most two per thread), the Newton matrix in 4 x 4 register
// blocks split over contact groups, and the CTA solver's factor, triangular
// solves and split-K products.
#pragma once

#include "cs_cta.cuh"
#include "cs_elliptic.cuh"

namespace csk {

// Vector slots beyond the CTA solver's own (CtaVec).
enum CtaEllVec {
  CE_RLO = C_PP + 1,  // low part of the residual r
  CE_S1, CE_S2,       // J^T lambda pair in the refined solve
  CE_RHO,             // the refined solve's correction
  CE_NVEC
};

// Shared-memory geometry: the CTA solver's, then u and J x as pairs per row,
// mu, the six Hessian entries and phi per contact.
struct CtaEllGeo {
  CtaGeo g;
  int ncap, oUh, oUl, oXh, oXl, oMu, oHB, oPhi, words;
  __host__ __device__ static CtaEllGeo make(int nv_max, int m_max) {
    CtaEllGeo e;
    e.g = CtaGeo::make(nv_max, m_max, CE_NVEC);
    const int mcap = e.g.mcap;
    e.ncap = (mcap / 3 + 31) & ~31;
    e.oUh = (e.g.words + 31) & ~31;
    e.oUl = e.oUh + mcap;
    e.oXh = e.oUl + mcap;
    e.oXl = e.oXh + mcap;
    e.oMu = e.oXl + mcap;
    e.oHB = e.oMu + e.ncap;
    e.oPhi = e.oHB + 6 * e.ncap;
    e.words = e.oPhi + e.ncap;
    return e;
  }
  __host__ __device__ size_t bytes() const { return ((size_t)words * 4 + 127) & ~(size_t)127; }
};

template <int MTC>
struct CtaElliptic {
  // contact slots per thread: m <= 256 MTC rows, so at most 256 MTC / 3 contacts
  static constexpr int MCTC = (MTC * kCtaThreads / 3 + kCtaThreads - 1) / kCtaThreads;
  CtaSolver<MTC> S;
  CtaEllGeo eg;
  int nc;
  uint32_t zbits;  // 2 bits per contact slot: its zone

  __device__ __forceinline__ float* Uh() { return S.sm + eg.oUh; }
  __device__ __forceinline__ float* Ul() { return S.sm + eg.oUl; }
  __device__ __forceinline__ float* Xh() { return S.sm + eg.oXh; }
  __device__ __forceinline__ float* Xl() { return S.sm + eg.oXl; }
  __device__ __forceinline__ float* Mu() { return S.sm + eg.oMu; }
  __device__ __forceinline__ float* HB(int k) { return S.sm + eg.oHB + k * eg.ncap; }
  __device__ __forceinline__ float* Phi() { return S.sm + eg.oPhi; }
  __device__ __forceinline__ int con(int u) const { return S.tid + kCtaThreads * u; }

  __device__ __forceinline__ bool load(const EParams& EP, const cs_inst& e) {
    if (!S.load(EP.P, e)) return false;  // the same answer on every thread
    if (S.m % 3) return false;
    nc = S.m / 3;
    for (int c = S.tid; c < eg.ncap; c += kCtaThreads)
      Mu()[c] = c < nc ? __ldg(EP.mu + e.off_r + 3 * c) : 0.f;
    __syncthreads();
    return true;
  }

  // Per-row pairs x = J (vh + vl) (optionally minus aref) into (Ah, Al).
  __device__ __forceinline__ void rows_to_smem(const float* vh, const float* vl, bool minus_aref,
                                               float* Ah, float* Al) {
    float s[MTC], c[MTC];
    S.rows_dot(vh, vl, true, s, c);
#pragma unroll
    for (int u = 0; u < MTC; ++u) {
      if (S.row_valid(u)) {
        float t, te, hi, lo;
        two_sum(s[u], minus_aref ? -S.aref_r[u] : 0.f, t, te);
        norm_pair(t, __fadd_rn(te, c[u]), hi, lo);
        Ah[S.row(u)] = hi;
        Al[S.row(u)] = lo;
      }
    }
    __syncthreads();
  }

  // ------------------------------------------------------------ residual
  // At a = C_AH + C_AL: u (pairs) per row, each contact's zone, gradient (F,
  // Flo per row), Hessian block and phi; the active-row list (the three rows
  // of every contact not in zone 0, in contact order); r = M a - qfrc +
  // J^T grad (compensated: C_R + CE_RLO), C_MAQ = M a - qfrc.
  __device__ __forceinline__ float residual(float* scale, bool* bad) {
    const int tid = S.tid, lane = S.lane, warp = S.warp, nv = S.nv;
    const float* vh = S.V(C_AH);
    const float* vl = S.V(C_AL);
    rows_to_smem(vh, vl, true, Uh(), Ul());
    float* F = S.Fs();
    float* Fl = S.Flo();
    int* idx = S.Idx();
    const float* Dm_ = S.Ds();
    float* Rd = S.Red() + 5 * kCtaWarps;  // compaction counts
    int base = 0;
    float fm = 0.f;
    zbits = 0;
#pragma unroll
    for (int u = 0; u < MCTC; ++u) {
      const int c = con(u);
      const bool valid = c < nc;
      Cone o;
      o.zone = 0;
      if (valid) {
        float uh[3], ul[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          uh[q] = Uh()[3 * c + q];
          ul[q] = Ul()[3 * c + q];
        }
        cone_eval(uh, ul, Dm_[3 * c], Dm_[3 * c + 1], Mu()[c], true, o);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          F[3 * c + q] = o.g[q];
          Fl[3 * c + q] = o.gl[q];
          fm = fmaxf(fm, fabsf(o.g[q]));
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) HB(k)[c] = o.h[k];
        Phi()[c] = o.phi;
      }
      const bool on = valid && o.zone != 0;
      zbits |= (uint32_t)o.zone << (2 * u);
      // block-wide compaction in contact order
      const unsigned bal = __ballot_sync(kFull, on);
      if (lane == 0) Rd[warp] = __int_as_float(__popc(bal));
      __syncthreads();
      int before = base, total = base;
#pragma unroll
      for (int w = 0; w < kCtaWarps; ++w) {
        const int cw = __float_as_int(Rd[w]);
        if (w < warp) before += cw;
        total += cw;
      }
      if (on) {
        const int pos = 3 * (before + __popc(bal & ((1u << lane) - 1u)));
        idx[pos] = 3 * c;
        idx[pos + 1] = 3 * c + 1;
        idx[pos + 2] = 3 * c + 2;
      }
      base = total;
      __syncthreads();
    }
    S.nact = 3 * base;
    S.fmax = S.block_max(fm);
    const float* Jm = S.Js();
    const float* Mm = S.Ms();
    const int JS = S.geo.JS, MS = S.geo.MS;
    S.split_dot(nv, S.nact, true,
                [&](int j, int q, float& a, float& h, float& l) {
                  const int i = idx[q];
                  a = Jm[i * JS + j];
                  h = F[i];
                  l = Fl[i];
                },
                S.V(C_X), S.V(C_MP));  // J^T grad (pair)
    S.split_dot(nv, nv, true,
                [&](int j, int k, float& a, float& h, float& l) {
                  a = Mm[j * MS + k];
                  h = vh[k];
                  l = vl[k];
                },
                S.V(C_R), S.V(C_MAQ));  // M a (pair)
    float rloc = 0.f, msm = 0.f, jsm = 0.f;
    bool nonfinite = false;
    if (tid < nv) {
      const float ms = S.V(C_R)[tid], mc = S.V(C_MAQ)[tid];
      const float js = S.V(C_X)[tid], jc = S.V(C_MP)[tid];
      float t1, e1, t2, e2;
      two_sum(ms, -S.V(C_QF)[tid], t1, e1);
      const float lo1 = __fadd_rn(e1, mc);
      const float maq = __fadd_rn(t1, lo1);
      two_sum(t1, js, t2, e2);
      const float lo2 = __fadd_rn(lo1, __fadd_rn(e2, jc));
      const float r = __fadd_rn(t2, lo2);
      // thread tid reads and overwrites only entry tid of these slots
      S.V(C_R)[tid] = r;
      S.V(CE_RLO)[tid] = __fsub_rn(lo2, __fsub_rn(r, t2));
      S.V(C_MAQ)[tid] = maq;
      rloc = fabsf(r);
      msm = fabsf(ms);
      jsm = fabsf(js);
      nonfinite = !(rloc < CUDART_INF_F);
    }
    for (int j = nv + tid; j < S.geo.nvcap; j += kCtaThreads) {
      S.V(C_R)[j] = 0.f;
      S.V(CE_RLO)[j] = 0.f;
      S.V(C_MAQ)[j] = 0.f;
    }
    const float rm = S.block_max(rloc);
    const float sc = fmaxf(fmaxf(1.f, S.qmax), fmaxf(S.block_max(msm), S.block_max(jsm)));
    *scale = sc;
    *bad = S.block_any(nonfinite) || !(sc < CUDART_INF_F);
    return rm;
  }

  // ----------------------------------------------------- Newton matrix
  // H = M + sum over contacts not in zone 0 of J_c^T hess_c J_c (Eq. 9) into
  // Ls(), then factor.  4 x 4 register blocks of the lower triangle, split
  // over groups of contacts when there are few blocks.
  __device__ __forceinline__ bool assemble_and_factor() {
    const float* Mm = S.Ms();
    const float* Jm = S.Js();
    const int* idx = S.Idx();
    float* L = S.Ls();
    float* scr = S.Scr();
    const int nvc = S.geo.nvcap, MS = S.geo.MS, JS = S.geo.JS;
    const int nb = nvc >> 2;
    const int nbl = nb * (nb + 1) / 2;
    const int R = max(1, min(kCtaThreads / nbl, 16));
    const int items = nbl * R;
    const int ncon = S.nact / 3;
#pragma unroll 1
    for (int w = S.tid; w < items; w += kCtaThreads) {
      const int blk = w % nbl, grp = w / nbl;
      int bj = 0;
      while ((bj + 1) * (bj + 2) / 2 <= blk) ++bj;
      const int bk = blk - bj * (bj + 1) / 2;
      const int cj = 4 * bj, ck = 4 * bk;
      float acc[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
#pragma unroll 2
      for (int q = grp; q < ncon; q += R) {
        const int r0 = idx[3 * q];
        const int c = r0 / 3;
        const float h00 = HB(0)[c], h01 = HB(1)[c], h02 = HB(2)[c];
        const float h11 = HB(3)[c], h12 = HB(4)[c], h22 = HB(5)[c];
        float x[3][4], y[3][4];
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          const float* Ji = Jm + (r0 + p) * JS;
#pragma unroll
          for (int a = 0; a < 4; ++a) x[p][a] = Ji[cj + a];
#pragma unroll
          for (int b = 0; b < 4; ++b) y[p][b] = Ji[ck + b];
        }
        // z_p = hess_c y (per column b), then acc += x_p z_p^T
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const float z0 = __fmaf_rn(h00, y[0][b], __fmaf_rn(h01, y[1][b], h02 * y[2][b]));
          const float z1 = __fmaf_rn(h01, y[0][b], __fmaf_rn(h11, y[1][b], h12 * y[2][b]));
          const float z2 = __fmaf_rn(h02, y[0][b], __fmaf_rn(h12, y[1][b], h22 * y[2][b]));
#pragma unroll
          for (int a = 0; a < 4; ++a)
            acc[a][b] = __fmaf_rn(x[0][a], z0, __fmaf_rn(x[1][a], z1, __fmaf_rn(x[2][a], z2,
                                                                                acc[a][b])));
        }
      }
      if (R == 1) {
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const int rr = cj + a, cc = ck + b;
            if (cc <= rr) L[rr * MS + cc] = Mm[rr * MS + cc] + acc[a][b];
          }
      } else {
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) scr[(grp * nbl + blk) * 16 + 4 * a + b] = acc[a][b];
      }
    }
    if (R > 1) {
      __syncthreads();
#pragma unroll 1
      for (int w = S.tid; w < nbl * 16; w += kCtaThreads) {
        const int blk = w >> 4, e = w & 15;
        int bj = 0;
        while ((bj + 1) * (bj + 2) / 2 <= blk) ++bj;
        const int bk = blk - bj * (bj + 1) / 2;
        const int rr = 4 * bj + (e >> 2), cc = 4 * bk + (e & 3);
        float t = 0.f;
        for (int gq = 0; gq < R; ++gq) t += scr[(gq * nbl + blk) * 16 + e];
        if (cc <= rr) L[rr * MS + cc] = Mm[rr * MS + cc] + t;
      }
    }
    __syncthreads();
    return S.factor();
  }

  // ------------------------------------------------------- line search
  // alpha > 0 minimising phi(alpha) = L(a + alpha p) (Eq. 10), p in C_P: as
  // the warp kernel, safeguarded Newton on the increasing
  //   phi'(alpha) = p^T r + alpha p^T M p
  //                 + sum_c (grad_c(u_c + alpha v_c) - grad_c(u_c)) . v_c,
  // v = J p, with p^T r compensated and the gradient differences taken at the
  // same high part of u; the quadratic model's alpha when alpha v is tiny
  // against u.  *dfmax is the largest change of a contact force component.
  __device__ __forceinline__ float line_search(float* dfmax) {
    const int tid = S.tid, nv = S.nv;
    const float* vp = S.V(C_P);
    float vr[MTC], vc[MTC];
    S.rows_dot(vp, vp, false, vr, vc);
#pragma unroll
    for (int u = 0; u < MTC; ++u)
      if (S.row_valid(u)) Xh()[S.row(u)] = vr[u];
    float pMp = 0.f, prh = 0.f, prl = 0.f;
    if (tid < nv) {
      const float* Mr = S.Ms() + tid * S.geo.MS;
      float mp = 0.f;
#pragma unroll 4
      for (int k = 0; k < nv; ++k) mp = __fmaf_rn(Mr[k], vp[k], mp);
      pMp = vp[tid] * mp;
      two_prod(vp[tid], S.V(C_R)[tid], prh, prl);
      prl = __fmaf_rn(vp[tid], S.V(CE_RLO)[tid], prl);
    }
    S.block_sum2(prh, prl);  // also makes Xh visible
    const float pr = prh + prl;
    pMp = S.block_sum(pMp);
    const float* Dm_ = S.Ds();
    float g0[MCTC][3];
    float hv_lin = 0.f, vrel = 0.f, hvmax = 0.f;
#pragma unroll
    for (int u = 0; u < MCTC; ++u) {
      const int c = con(u);
#pragma unroll
      for (int q = 0; q < 3; ++q) g0[u][q] = 0.f;
      if (c < nc) {
        float uh[3], ul[3] = {0.f, 0.f, 0.f}, v[3], un = 0.f, vn = 0.f;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          uh[q] = Uh()[3 * c + q];
          v[q] = Xh()[3 * c + q];
          un = fmaxf(un, fabsf(uh[q]));
          vn = fmaxf(vn, fabsf(v[q]));
        }
        Cone o;
        cone_eval(uh, ul, Dm_[3 * c], Dm_[3 * c + 1], Mu()[c], false, o);
#pragma unroll
        for (int q = 0; q < 3; ++q) g0[u][q] = o.g[q];
        // the quadratic model at u (every contact counts in the smallness
        // test: one outside the cone's force region must not reach it)
        const float hv0 = __fmaf_rn(HB(0)[c], v[0], __fmaf_rn(HB(1)[c], v[1], HB(2)[c] * v[2]));
        const float hv1 = __fmaf_rn(HB(1)[c], v[0], __fmaf_rn(HB(3)[c], v[1], HB(4)[c] * v[2]));
        const float hv2 = __fmaf_rn(HB(2)[c], v[0], __fmaf_rn(HB(4)[c], v[1], HB(5)[c] * v[2]));
        hv_lin = __fmaf_rn(hv0, v[0], __fmaf_rn(hv1, v[1], __fmaf_rn(hv2, v[2], hv_lin)));
        hvmax = fmaxf(hvmax, fmaxf(fabsf(hv0), fmaxf(fabsf(hv1), fabsf(hv2))));
        vrel = fmaxf(vrel, vn / fmaxf(un, 1e-30f));
      }
    }
    const float curv0 = pMp + S.block_sum(hv_lin);
    const float alpha0 = -pr / curv0;
    const float vrel_max = S.block_max(vrel);
    const float hvm = S.block_max(hvmax);
    if (alpha0 > 0.f && alpha0 * vrel_max <= 1e-3f) {
      *dfmax = alpha0 * hvm;
      return alpha0;
    }
    float alpha = 1.f, lo = 0.f, hi = CUDART_INF_F, df = 0.f;
#pragma unroll 1
    for (int it = 0; it < 60; ++it) {
      float d1 = 0.f, d2 = 0.f, dfl = 0.f;
#pragma unroll
      for (int u = 0; u < MCTC; ++u) {
        const int c = con(u);
        if (c < nc) {
          float uh[3], ul[3] = {0.f, 0.f, 0.f}, v[3];
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            v[q] = Xh()[3 * c + q];
            uh[q] = __fmaf_rn(alpha, v[q], Uh()[3 * c + q]);
          }
          Cone o;
          cone_eval(uh, ul, Dm_[3 * c], Dm_[3 * c + 1], Mu()[c], false, o);
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            const float dg = o.g[q] - g0[u][q];
            d1 = __fmaf_rn(dg, v[q], d1);
            dfl = fmaxf(dfl, fabsf(dg));
          }
          const float hv0 = __fmaf_rn(o.h[0], v[0], __fmaf_rn(o.h[1], v[1], o.h[2] * v[2]));
          const float hv1 = __fmaf_rn(o.h[1], v[0], __fmaf_rn(o.h[3], v[1], o.h[4] * v[2]));
          const float hv2 = __fmaf_rn(o.h[2], v[0], __fmaf_rn(o.h[4], v[1], o.h[5] * v[2]));
          d2 = __fmaf_rn(hv0, v[0], __fmaf_rn(hv1, v[1], __fmaf_rn(hv2, v[2], d2)));
        }
      }
      S.block_sum2(d1, d2);
      df = S.block_max(dfl);
      const float d = pr + alpha * pMp + d1;
      const float dd = pMp + d2;
      if (d == 0.f) break;
      if (d < 0.f) lo = alpha; else hi = alpha;
      float an = alpha - d / dd;
      if (!(an > lo && an < hi)) an = (hi == CUDART_INF_F) ? 2.f * alpha : 0.5f * (lo + hi);
      const bool done = fabsf(an - alpha) <= 1e-6f * alpha;
      alpha = an;
      if (done || (hi - lo) <= 1e-7f * hi) break;
    }
    *dfmax = df;
    return alpha;
  }

  // ------------------------------------------------------------ adjoint
  // H w = rhs (+ rhs_lo) with refinement (slots rh, rl < 0: none; result in
  // oh / ol); lambda_c = hess_c (J w)_c (compensated) in Lam / Lamlo per row.
  // `full` refines to the float-pair precision of w (the adjoint: the cone
  // parameters' derivatives carry the small component of J w along a
  // contact's stiff direction); otherwise to FP32 precision.  The stop test
  // is the warp kernel's: the correction taken last and the change of
  // lambda.
  __device__ __forceinline__ void solve_refined(int rh, int rl, int oh, int ol, bool full) {
    const float step_tol = full ? 1e-9f : kStepTol;
    const float force_tol = full ? 1e-7f : kForceTol;
    const int it_max = full ? 2 * kAdjointRefineMax : kAdjointRefineMax;
    const int tid = S.tid, nv = S.nv;
    float* wh = S.V(oh);
    float* wl = S.V(ol);
    for (int j = tid; j < S.geo.nvcap; j += kCtaThreads) {
      wh[j] = S.V(rh)[j];
      wl[j] = 0.f;
    }
    __syncthreads();
    S.chol_solve(oh);
    float* Lm = S.Lam();
    float* Lml = S.Lamlo();
    const float* Jm = S.Js();
    const float* Mm = S.Ms();
    const int* idx = S.Idx();
    const int JS = S.geo.JS, MS = S.geo.MS;
    float lam_prev[3 * MCTC];
#pragma unroll
    for (int k = 0; k < 3 * MCTC; ++k) lam_prev[k] = 0.f;
    float dmax_prev = CUDART_INF_F;
    float dmax_pp = 0.f;  // the correction before dmax_prev (0: w itself)
#pragma unroll 1
    for (int it = 0; it <= it_max; ++it) {
      rows_to_smem(wh, wl, false, Xh(), Xl());
      float lmax = 0.f, dl = 0.f;
#pragma unroll
      for (int u = 0; u < MCTC; ++u) {
        const int c = con(u);
        if (c < nc) {
          const bool on = (zbits >> (2 * u)) & 3u;
          float xh[3], xl[3];
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            xh[q] = Xh()[3 * c + q];
            xl[q] = Xl()[3 * c + q];
          }
          const float hm[3][3] = {{HB(0)[c], HB(1)[c], HB(2)[c]},
                                  {HB(1)[c], HB(3)[c], HB(4)[c]},
                                  {HB(2)[c], HB(4)[c], HB(5)[c]}};
#pragma unroll
          for (int p = 0; p < 3; ++p) {
            float s = 0.f, cc = 0.f;
            if (on) {
#pragma unroll
              for (int q = 0; q < 3; ++q) dot2(s, cc, hm[p][q], xh[q], xl[q]);
            }
            float lh, ll;
            norm_pair(s, cc, lh, ll);
            Lm[3 * c + p] = lh;
            Lml[3 * c + p] = ll;
            lmax = fmaxf(lmax, fabsf(lh));
            dl = fmaxf(dl, fabsf(lh - lam_prev[3 * u + p]));
            lam_prev[3 * u + p] = lh;
          }
        }
      }
      lmax = S.block_max(lmax);
      dl = S.block_max(dl);
      if (it > 0) {
        const float wmax = S.block_max(tid < nv ? fabsf(wh[tid]) : 0.f);
        // or the error left after the correction just applied, predicted
        // from the contraction of two consecutive ones (see the warp
        // solver's refinement), meets both tolerances
        const float q = dmax_prev / (dmax_pp > 0.f ? dmax_pp : wmax);
        const float gq = (dmax_pp > 0.f ? 1.f : kFirstRatioMargin) * q / (1.f - q);
        const bool predicted = q < 0.5f && gq * dmax_prev <= step_tol * wmax &&
                               gq * dl <= force_tol * lmax;
        if ((dmax_prev <= step_tol * wmax && dl <= force_tol * lmax) || predicted ||
            it == it_max)
          break;
        dmax_pp = dmax_prev;
      }
      S.split_dot(nv, S.nact, true,
                  [&](int j, int q, float& a, float& h, float& l) {
                    const int i = idx[q];
                    a = Jm[i * JS + j];
                    h = Lm[i];
                    l = Lml[i];
                  },
                  S.V(CE_S1), S.V(CE_S2));  // J^T lambda (pair)
      S.split_dot(nv, nv, true,
                  [&](int j, int k, float& a, float& h, float& l) {
                    a = Mm[j * MS + k];
                    h = wh[k];
                    l = wl[k];
                  },
                  S.V(C_X), S.V(C_MP));  // M w (pair)
      float* rho = S.V(CE_RHO);
      float dm = 0.f;
      if (tid < nv) {
        float t1, e1, t2, e2;
        two_sum(S.V(rh)[tid], -S.V(C_X)[tid], t1, e1);
        two_sum(t1, -S.V(CE_S1)[tid], t2, e2);
        float lo = __fadd_rn(e1, e2);
        if (rl >= 0) lo = __fadd_rn(lo, S.V(rl)[tid]);
        rho[tid] = __fadd_rn(t2, __fsub_rn(lo, __fadd_rn(S.V(C_MP)[tid], S.V(CE_S2)[tid])));
      }
      for (int j = nv + tid; j < S.geo.nvcap; j += kCtaThreads) rho[j] = 0.f;
      __syncthreads();
      S.chol_solve(CE_RHO);
      if (tid < nv) {
        dm = fabsf(rho[tid]);
        float hh = wh[tid], ll = wl[tid];
        WarpSolver<1, 1>::add_to_pair(hh, ll, rho[tid]);
        wh[tid] = hh;
        wl[tid] = ll;
      }
      dmax_prev = S.block_max(dm);  // also orders the updates of w
    }
    __syncthreads();
  }

  // --------------------------------------------------------- forward
  __device__ __forceinline__ int forward(const Params& P, int* iters) {
    const int tid = S.tid, nv = S.nv;
    *iters = 0;
    if (!S.factor_M()) return CS_ST_CHOLFAIL;
    float* ah = S.V(C_AH);
    float* al = S.V(C_AL);
    float* pv = S.V(C_P);
    for (int j = tid; j < S.geo.nvcap; j += kCtaThreads) {
      ah[j] = S.V(C_QF)[j];
      al[j] = 0.f;
    }
    __syncthreads();
    S.chol_solve(C_AH);
    uint32_t prev_z = 0;
    bool prev_small = false;
    int stall = 0;
    float smax_prev = 0.f;
#pragma unroll 1
    for (int k = 0;; ++k) {
      float scale;
      bool bad;
      const float rmax = residual(&scale, &bad);
      if (bad) return CS_ST_NONFINITE;
      if (rmax <= P.tol * scale) return CS_ST_OK;
      const bool same = !S.block_any(zbits != prev_z);
      if (k > 0 && same && prev_small) return CS_ST_OK;
      // three consecutive steps below the resolution of a with unchanged
      // zones: a has reached its attainable accuracy
      if (stall >= 3) return CS_ST_OK;
      if (k >= P.max_iter) return CS_ST_MAXITER;
      if (!assemble_and_factor()) return CS_ST_CHOLFAIL;
      // Newton direction: one FP32 solve of H p = -r with the factor (the
      // residual is compensated and decides every stop test, as in the warp
      // kernel)
      for (int j = tid; j < S.geo.nvcap; j += kCtaThreads) pv[j] = -S.V(C_R)[j];
      __syncthreads();
      S.chol_solve(C_P);
      const float ptr = S.block_sum(tid < nv ? pv[tid] * S.V(C_R)[tid] : 0.f);
      const float amax = S.block_max(tid < nv ? fabsf(ah[tid]) : 0.f);
      if (!(ptr < 0.f)) {
        const float pm = S.block_max(tid < nv ? fabsf(pv[tid]) : 0.f);
        return (pm <= kStepTol * amax) ? CS_ST_OK : CS_ST_NOPROGRESS;
      }
      float dfm;
      const float alpha = line_search(&dfm);
      float sm = 0.f;
      if (tid < nv) {
        const float dp = alpha * pv[tid];
        float hh = ah[tid], ll = al[tid];
        WarpSolver<1, 1>::add_to_pair(hh, ll, dp);
        ah[tid] = hh;
        al[tid] = ll;
        sm = fabsf(dp);
      }
      *iters = k + 1;
      const float smax = S.block_max(sm);  // also orders the updates of a
      // small, or predicted small (as in the warp kernel)
      const float q = smax / smax_prev;
      const float gq = q / (1.f - q);
      const bool predicted = same && smax_prev > 0.f && q < 0.5f &&
                             gq * smax <= kStepTol * amax && gq * dfm <= kForceTol * S.fmax;
      prev_small = ((smax <= kStepTol * amax) && (dfm <= kForceTol * S.fmax)) || predicted;
      smax_prev = smax;
      stall = (smax <= kStepTol * amax && same) ? stall + 1 : 0;
      prev_z = zbits;
    }
  }

  // dqfrc = w, daref = lambda, dJ = -(grad w^T + lambda a^T), optional dM
  // (symmetric M), dD (D_N on row 3c, D_T on 3c+1, 0 on 3c+2) and dmu (row
  // 3c; other rows 0); w in C_WH / C_WL, lambda in Lam().
  __device__ __forceinline__ void write_grads(const EParams& EP, const cs_inst& e) {
    const Params& P = EP.P;
    const int tid = S.tid, nv = S.nv, m = S.m;
    const float* wh = S.V(C_WH);
    const float* wl = S.V(C_WL);
    const float* ah = S.V(C_AH);
    const float* Lm = S.Lam();
    const float* F = S.Fs();
    for (int j = tid; j < nv; j += kCtaThreads) P.dqfrc[e.off_v + j] = wh[j];
    for (int i = tid; i < m; i += kCtaThreads) P.daref[e.off_r + i] = Lm[i];
    float* dJ = P.dJ + e.off_J;
#pragma unroll 1
    for (int q = tid; q < m * nv; q += kCtaThreads) {
      const int rr = q / nv, cc = q - rr * nv;
      dJ[q] = -__fmaf_rn(F[rr], wh[cc], Lm[rr] * ah[cc]);
    }
    if (P.dM) {
      float* dM = P.dM + e.off_M;
#pragma unroll 1
      for (int q = tid; q < nv * nv; q += kCtaThreads) {
        const int rr = q / nv, cc = q - rr * nv;
        dM[q] = -0.5f * __fmaf_rn(wh[rr], ah[cc], ah[rr] * wh[cc]);
      }
    }
    if (P.dD || EP.dmu) {
      // v = J w (pairs) per row for the contact owners
      rows_to_smem(wh, wl, false, Xh(), Xl());
      const float* Dm_ = S.Ds();
#pragma unroll
      for (int u = 0; u < MCTC; ++u) {
        const int c = con(u);
        if (c >= nc) continue;
        const int z = (zbits >> (2 * u)) & 3u;
        const float DN = Dm_[3 * c], DT = Dm_[3 * c + 1], f = Mu()[c];
        float uh[3], ul[3], vh[3], vl[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          uh[q] = Uh()[3 * c + q];
          ul[q] = Ul()[3 * c + q];
          vh[q] = Xh()[3 * c + q];
          vl[q] = Xl()[3 * c + q];
        }
        // dL/dtheta = -v . d grad / d theta with v = (J w)_c
        float dN = 0.f, dT = 0.f, dmu = 0.f;
        if (z == 2) {
          // grad = (D_N u_N, D_T u_T)
          float s = 0.f, cc = 0.f;
          dot2p(s, cc, uh[0], ul[0], vh[0], vl[0]);
          dN = -__fadd_rn(s, cc);
          s = 0.f;
          cc = 0.f;
          dot2p(s, cc, uh[1], ul[1], vh[1], vl[1]);
          dot2p(s, cc, uh[2], ul[2], vh[2], vl[2]);
          dT = -__fadd_rn(s, cc);
        } else if (z == 1) {
          // grad = Dm phi gv, gv = (-1, mu uhat); every derivative carries
          // gv . v = (mu u_T . v_T - v_N t) / t, formed from the pairs
          float th, tl;
          t_pair(uh, ul, th, tl);
          float s = 0.f, cc = 0.f;
          dot2p(s, cc, uh[1], ul[1], vh[1], vl[1]);
          dot2p(s, cc, uh[2], ul[2], vh[2], vl[2]);
          float uvh, uvl;
          norm_pair(s, cc, uvh, uvl);  // u_T . v_T
          float mh, ml;
          WarpSolver<1, 1>::scale_pair(f, uvh, uvl, mh, ml);
          s = mh;
          cc = ml;
          float nh, nl;
          two_prod(-vh[0], th, nh, nl);
          nl = __fmaf_rn(-vh[0], tl, __fmaf_rn(-vl[0], th, nl));
          add_pair(s, cc, nh, nl);
          const float t = __fadd_rn(th, tl);
          const float gvv = t > 0.f ? __fdiv_rn(__fadd_rn(s, cc), t) : -__fadd_rn(vh[0], vl[0]);
          const float vtu = t > 0.f ? __fdiv_rn(__fadd_rn(uvh, uvl), t) : 0.f;  // v_T . uhat
          const float den = __fmaf_rn(f * f, DN, DT);
          const float Dm = __fdiv_rn(DN * DT, den), phi = Phi()[c];
          const float den2 = den * den;
          const float dDN = __fdiv_rn(DT * DT, den2), dDT = __fdiv_rn(f * f * DN * DN, den2);
          const float dmu_ = __fdiv_rn(-2.f * f * DN * DN * DT, den2);
          dN = -dDN * phi * gvv;
          dT = -dDT * phi * gvv;
          dmu = -__fmaf_rn(__fmaf_rn(dmu_, phi, Dm * t), gvv, Dm * phi * vtu);
        }
        if (P.dD) {
          P.dD[e.off_r + 3 * c] = dN;
          P.dD[e.off_r + 3 * c + 1] = dT;
          P.dD[e.off_r + 3 * c + 2] = 0.f;
        }
        if (EP.dmu) {
          EP.dmu[e.off_r + 3 * c] = dmu;
          EP.dmu[e.off_r + 3 * c + 1] = 0.f;
          EP.dmu[e.off_r + 3 * c + 2] = 0.f;
        }
      }
    }
  }

  __device__ __forceinline__ void zero_grads(const EParams& EP, const cs_inst& e) {
    const Params& P = EP.P;
    const int tid = S.tid, nv = S.nv, m = S.m;
    for (int j = tid; j < nv; j += kCtaThreads) P.dqfrc[e.off_v + j] = 0.f;
    for (int i = tid; i < m; i += kCtaThreads) {
      P.daref[e.off_r + i] = 0.f;
      if (P.dD) P.dD[e.off_r + i] = 0.f;
      if (EP.dmu) EP.dmu[e.off_r + i] = 0.f;
    }
    for (int q = tid; q < m * nv; q += kCtaThreads) P.dJ[e.off_J + q] = 0.f;
    if (P.dM)
      for (int q = tid; q < nv * nv; q += kCtaThreads) P.dM[e.off_M + q] = 0.f;
  }

  __device__ __forceinline__ void run(const EParams& EP, int b) {
    const Params& P = EP.P;
    const cs_inst e = P.inst[b];
    const int tid = S.tid;
    if (!load(EP, e)) {
      if (tid == 0) {
        P.status[b] = CS_ST_BADSHAPE;
        P.iters[b] = 0;
      }
      return;
    }
    const int nv = S.nv;
    for (int j = tid; j < S.geo.nvcap; j += kCtaThreads)
      S.V(C_G)[j] = j < nv ? __ldg(P.g + e.off_v + j) : 0.f;
    int iters = 0;
    const int st = forward(P, &iters);
    for (int j = tid; j < nv; j += kCtaThreads) P.a[e.off_v + j] = S.V(C_AH)[j];
    if (tid == 0) {
      P.status[b] = st;
      P.iters[b] = iters;
    }
    if (st == CS_ST_CHOLFAIL || st == CS_ST_NONFINITE) {
      zero_grads(EP, e);
      return;
    }
    // adjoint at the returned point: H from the Hessian blocks of the last
    // residual evaluation, which was made at that point
    if (!assemble_and_factor()) {
      if (tid == 0) P.status[b] = CS_ST_CHOLFAIL;
      zero_grads(EP, e);
      return;
    }
    solve_refined(C_G, -1, C_WH, C_WL, true);
    write_grads(EP, e);
  }
};

// One CTA per instance; CTAs claim instances dynamically (cost order) or
// round-robin.
template <int MTC>
__global__ void __launch_bounds__(kCtaThreads, MTC == 1 ? 2 : 1)
    cta_elliptic_kernel(const __grid_constant__ EParams EP, const CtaEllGeo eg) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ int claim;
  const Params& P = EP.P;
  CtaElliptic<MTC> X;
  X.S.sm = reinterpret_cast<float*>(smem_raw);
  X.S.geo = eg.g;
  X.eg = eg;
  X.S.tid = threadIdx.x;
  X.S.lane = threadIdx.x & 31;
  X.S.warp = threadIdx.x >> 5;
  int idx = blockIdx.x;
#pragma unroll 1
  for (int guard = 0; guard <= P.n_work; ++guard) {
    if (P.counter) {
      if (X.S.tid == 0) claim = atomicAdd(P.counter, 1);
      __syncthreads();
      idx = claim;
      __syncthreads();
    }
    if (idx >= P.n_work) break;
    const int b = P.order ? P.order[idx] : idx;
    if (b >= 0 && b < P.n) X.run(EP, b);
    __syncthreads();
    if (!P.counter) idx += gridDim.x;
  }
}

}  // namespace csk
