// cs_elliptic.cuh -- the fused solve and IFT adjoint with MuJoCo's round
// Coulomb cone, one warp per instance (device code).
//
// The paper keeps the round cone of Eq. 2; its contact term (Eq. 5) is the
// weighted distance of u = J a - aref to the dual cone K* (Eq. 3).  A contact
// c owns three rows (3c normal, 3c+1 and 3c+2 tangents), with D_N = D[3c],
// D_T = D[3c+1] (one tangential stiffness for both tangent rows; D[3c+2] is
// not read) and mu = mu[3c].  With x = diag(D)^(1/2) u the weighted distance
// becomes the Euclidean distance of x to a second-order cone of slope
// mu sqrt(D_N / D_T), whose projection has three regions (t = |u_T|,
// phi = mu t - u_N, Dm = D_N / (1 + mu^2 D_N / D_T)):
//   zone 0  u_N >= mu t (phi <= 0):  no force;
//   zone 2  mu D_N u_N + D_T t <= 0:  grad s = (D_N u_N, D_T u_T),
//           Hessian diag(D_N, D_T, D_T);
//   zone 1  otherwise:  grad s = Dm phi (-1, mu u_T / t),
//           Hessian Dm g g^T + (Dm phi mu / t) (0 (+) (I - uhat uhat^T)),
//           g = (-1, mu uhat), uhat = u_T / t.
// The residual r = M a - qfrc + J^T grad s (Eq. 6) and the Newton matrix
// H = M + sum_c J_c^T hess_c J_c (Eq. 9) follow; the line search minimises the
// convex phi(alpha) = L(a + alpha p) by safeguarded Newton on phi'.  The
// adjoint (Eq. 17) solves H w = g at the returned a; lambda_c = hess_c (J w)_c
// replaces D_act . (J w), so daref = lambda, dJ = -(grad w^T + lambda a^T),
// and the cone parameters get dL/dtheta_c = -(J w)_c . d grad_c / d theta_c.
//
// Precision: as for the pyramid rows, u is a compensated float pair and the
// cone gradient is formed in float-pair arithmetic (phi = mu t - u_N cancels
// near the zone boundary and is multiplied by stiffnesses up to 1e5), so the
// residual's floor stays below the stopping tolerance.  The Hessian blocks
// are plain FP32: H preconditions a refined solve and sets the Newton step.
#pragma once

#include "cs_warp.cuh"

namespace csk {

struct EParams {
  Params P;          // batch, options, g, outputs (dM may be null), status, iters, claims
  const float* mu;   // friction per row (read on the normal rows 3c)
  float* dmu;        // dL/dmu on the normal rows, or null
};

template <int NV, int MT>
struct EGeo {
  using G = Geo<NV, MT>;
  static constexpr int MCAP = G::MCAP;
  static constexpr int NC = MCAP / 3;          // contacts per instance
  static constexpr int MCT = (NC + 31) / 32;   // contact slots per lane
  static constexpr int NCP = 32 * MCT;
  // extra words after the warp solver's slice
  static constexpr int oUh = G::kWords;        // u = J a - aref per row (pair)
  static constexpr int oUl = oUh + MCAP;
  static constexpr int oXh = oUl + MCAP;       // J x per row (pair): J p, J w
  static constexpr int oXl = oXh + MCAP;
  static constexpr int oMu = oXl + MCAP;       // mu per contact
  static constexpr int oHB = oMu + NCP;        // Hessian blocks, 6 x NCP (SoA)
  static constexpr int oPhi = oHB + 6 * NCP;   // phi = mu t - u_N per contact
  static constexpr int kWords = oPhi + NCP;
  static constexpr int kBytes = ((kWords * 4) + 127) & ~127;
};

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}
// (hi, lo) normalised from s + tail
__device__ __forceinline__ void norm_pair(float s, float tail, float& hi, float& lo) {
  hi = __fadd_rn(s, tail);
  lo = __fsub_rn(tail, __fsub_rn(hi, s));
}

// One contact's cone: zone, gradient as float pairs (precise) or plain, and
// the Hessian block (h00 h01 h02 h11 h12 h22).
struct Cone {
  int zone;
  float g[3], gl[3];
  float h[6];
  float phi;      // phi = mu t - u_N, rounded from its pair
};

// t = |u_T| as a pair, from the pairs of the two tangent components.
__device__ __forceinline__ void t_pair(const float (&uh)[3], const float (&ul)[3], float& th,
                                       float& tl) {
  float p1, e1, p2, e2, s, es;
  two_prod(uh[1], uh[1], p1, e1);
  two_prod(uh[2], uh[2], p2, e2);
  two_sum(p1, p2, s, es);
  float tail = __fadd_rn(es, __fadd_rn(e1, e2));
  tail = __fmaf_rn(2.f * uh[1], ul[1], __fmaf_rn(2.f * uh[2], ul[2], tail));
  float Th, Tl;
  norm_pair(s, tail, Th, Tl);
  th = sqrtf(Th);
  tl = th > 0.f ? __fdiv_rn(__fadd_rn(__fmaf_rn(-th, th, Th), Tl), 2.f * th) : 0.f;
}

// (s, c) += (xh + xl) (yh + yl), compensated.
__device__ __forceinline__ void dot2p(float& s, float& c, float xh, float xl, float yh, float yl) {
  float p, e, t, te;
  two_prod(xh, yh, p, e);
  two_sum(s, p, t, te);
  s = t;
  c = __fadd_rn(c, __fadd_rn(te, __fmaf_rn(xh, yl, __fmaf_rn(xl, yh, e))));
}

__device__ __forceinline__ void cone_eval(const float (&uh)[3], const float (&ul)[3], float DN,
                                          float DT, float mu, bool precise, Cone& o) {
  float th, tl;
  t_pair(uh, ul, th, tl);
  // phi = mu t - u_N (pair)
  float mth, mte;
  two_prod(mu, th, mth, mte);
  mte = __fmaf_rn(mu, tl, mte);
  float ph0, pe0;
  two_sum(mth, -uh[0], ph0, pe0);
  float phih, phil;
  norm_pair(ph0, __fadd_rn(pe0, __fsub_rn(mte, ul[0])), phih, phil);
#pragma unroll
  for (int k = 0; k < 6; ++k) o.h[k] = 0.f;
#pragma unroll
  for (int k = 0; k < 3; ++k) { o.g[k] = 0.f; o.gl[k] = 0.f; }
  o.phi = __fadd_rn(phih, phil);
  if (!(phih > 0.f)) {
    o.zone = 0;
    return;
  }
  if (__fmaf_rn(mu * DN, uh[0], DT * th) <= 0.f) {
    o.zone = 2;
    const float Dr[3] = {DN, DT, DT};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (precise) {
        WarpSolver<1, 1>::scale_pair(Dr[k], uh[k], ul[k], o.g[k], o.gl[k]);
      } else {
        o.g[k] = Dr[k] * uh[k];
      }
    }
    o.h[0] = DN;
    o.h[3] = DT;
    o.h[5] = DT;
    return;
  }
  o.zone = 1;
  const float Dm = __fdiv_rn(DN, __fmaf_rn(mu * mu, __fdiv_rn(DN, DT), 1.f));
  // grad_N = -Dm phi
  if (precise) {
    WarpSolver<1, 1>::scale_pair(-Dm, phih, phil, o.g[0], o.gl[0]);
  } else {
    o.g[0] = -Dm * phih;
  }
  // kappa = Dm mu phi / t; grad_T = kappa u_T
  const float qh = __fdiv_rn(phih, th);
  const float ql = __fdiv_rn(__fsub_rn(__fadd_rn(__fmaf_rn(-qh, th, phih), phil), qh * tl), th);
  float kh, kl;
  WarpSolver<1, 1>::scale_pair(Dm * mu, qh, ql, kh, kl);
#pragma unroll
  for (int k = 1; k < 3; ++k) {
    if (precise) {
      float pp, pe;
      two_prod(kh, uh[k], pp, pe);
      pe = __fmaf_rn(kh, ul[k], __fmaf_rn(kl, uh[k], pe));
      norm_pair(pp, pe, o.g[k], o.gl[k]);
    } else {
      o.g[k] = kh * uh[k];
    }
  }
  const float h1 = __fdiv_rn(uh[1], th), h2 = __fdiv_rn(uh[2], th);
  const float gv1 = mu * h1, gv2 = mu * h2;
  o.h[0] = Dm;
  o.h[1] = -Dm * gv1;
  o.h[2] = -Dm * gv2;
  o.h[3] = __fmaf_rn(Dm * gv1, gv1, kh * (1.f - h1 * h1));
  o.h[4] = __fmaf_rn(Dm * gv1, gv2, -kh * h1 * h2);
  o.h[5] = __fmaf_rn(Dm * gv2, gv2, kh * (1.f - h2 * h2));
}

template <int NV, int MT>
struct EllipticSolver {
  using G = Geo<NV, MT>;
  using E = EGeo<NV, MT>;
  WarpSolver<NV, MT> S;
  int nc;
  uint32_t zbits;       // 2 bits per contact slot: its zone

  __device__ __forceinline__ float* Uh() { return S.sm + E::oUh; }
  __device__ __forceinline__ float* Ul() { return S.sm + E::oUl; }
  __device__ __forceinline__ float* Xh() { return S.sm + E::oXh; }
  __device__ __forceinline__ float* Xl() { return S.sm + E::oXl; }
  __device__ __forceinline__ float* Mu() { return S.sm + E::oMu; }
  __device__ __forceinline__ float* HB(int k) { return S.sm + E::oHB + k * E::NCP; }
  __device__ __forceinline__ float* Phi() { return S.sm + E::oPhi; }

  __device__ __forceinline__ bool load(const EParams& EP, const cs_inst& e) {
    if (!S.load(EP.P, e)) return false;
    if (S.m % 3) return false;
    nc = S.m / 3;
#pragma unroll
    for (int u = 0; u < E::MCT; ++u) {
      const int c = S.lane + 32 * u;
      Mu()[c] = c < nc ? __ldg(EP.mu + e.off_r + 3 * c) : 0.f;
    }
    __syncwarp();
    return true;
  }

  // Per-row pairs x = J (vh + vl) (optionally minus aref) into (Ah, Al).
  __device__ __forceinline__ void rows_to_smem(const float* vh, const float* vl, bool minus_aref,
                                               float* Ah, float* Al) {
    float s[MT], c[MT];
    S.rows_dot2(vh, vl, s, c);
#pragma unroll
    for (int t = 0; t < MT; ++t) {
      if (32 * t < S.m) {
        float u, ue;
        two_sum(s[t], minus_aref ? -S.aref_r[t] : 0.f, u, ue);
        float hi, lo;
        norm_pair(u, __fadd_rn(ue, c[t]), hi, lo);
        if (S.row_valid(t)) {
          Ah[S.lane + 32 * t] = hi;
          Al[S.lane + 32 * t] = lo;
        }
      }
    }
    __syncwarp();
  }

  // ------------------------------------------------------------ residual
  // At a = ah + al: u (pairs) per row, each contact's zone / gradient (F, Flo
  // per row) / Hessian block, the active-row list (rows of contacts not in
  // zone 0), r = M a - qfrc + J^T grad (compensated, r + rlo), maq.
  __device__ __forceinline__ float residual(float* scale, bool* bad) {
    const int lane = S.lane;
    S.put_vec(V_AH, S.ah);
    S.put_vec(V_AL, S.al);
    const float* vh = S.Vec(V_AH);
    const float* vl = S.Vec(V_AL);
    rows_to_smem(vh, vl, true, Uh(), Ul());
    float* F = S.Fs();
    float* Fl = S.Flo();
    int* idx = S.Idx();
    const float* Dm_ = S.Ds();
    int base = 0;
    float fm = 0.f;
    zbits = 0;
#pragma unroll
    for (int u = 0; u < E::MCT; ++u) {
      const int c = lane + 32 * u;
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
      const unsigned bal = __ballot_sync(kFull, on);
      if (on) {
        const int pos = base + 3 * __popc(bal & ((1u << lane) - 1u));
        idx[pos] = 3 * c;
        idx[pos + 1] = 3 * c + 1;
        idx[pos + 2] = 3 * c + 2;
      }
      base += 3 * __popc(bal);
    }
    S.nact = base;
    S.fmax = warp_max(fm);
    __syncwarp();
    float js, jc, ms, mc;
    S.jt_active(F, Fl, js, jc);
    S.m_times(vh, vl, ms, mc);
    float t1, e1, t2, e2;
    two_sum(ms, -S.qf, t1, e1);
    const float lo1 = __fadd_rn(e1, mc);
    S.maq = __fadd_rn(t1, lo1);
    two_sum(t1, js, t2, e2);
    const float lo2 = __fadd_rn(lo1, __fadd_rn(e2, jc));
    S.r = __fadd_rn(t2, lo2);
    S.rlo = __fsub_rn(lo2, __fsub_rn(S.r, t2));
    if (lane >= NV) {
      S.r = 0.f;
      S.rlo = 0.f;
      S.maq = 0.f;
    }
    const float rm = warp_max(fabsf(S.r));
    const float sc =
        fmaxf(fmaxf(1.f, S.qmax), fmaxf(warp_max(fabsf(ms)), warp_max(fabsf(js))));
    *scale = sc;
    *bad = __any_sync(kFull, !(fabsf(S.r) < CUDART_INF_F)) || !(sc < CUDART_INF_F);
    return rm;
  }

  // ----------------------------------------------------- Newton matrix
  // H = M + sum over contacts not in zone 0 of J_c^T hess_c J_c (Eq. 9) into
  // Ls(), then factor.  Lane l < NBLK accumulates one BS x BS block.
  __device__ __forceinline__ bool assemble_and_factor() {
    const float* Mm = S.Ms();
    const float* Jm = S.Js();
    const int* idx = S.Idx();
    float* L = S.Ls();
    const int ncon = S.nact / 3;
    if (S.lane < G::NBLK) {
      int bj = 0;
      while ((bj + 1) * (bj + 2) / 2 <= S.lane) ++bj;
      const int bk = S.lane - bj * (bj + 1) / 2;
      float acc[G::BS][G::BS];
#pragma unroll
      for (int u = 0; u < G::BS; ++u)
#pragma unroll
        for (int v = 0; v < G::BS; ++v) acc[u][v] = 0.f;
      const int cj = bj * G::BS, ck = bk * G::BS;
#pragma unroll 1
      for (int q = 0; q < ncon; ++q) {
        const int r0 = idx[3 * q];
        const int c = r0 / 3;
        const float h00 = HB(0)[c], h01 = HB(1)[c], h02 = HB(2)[c];
        const float h11 = HB(3)[c], h12 = HB(4)[c], h22 = HB(5)[c];
        float x[3][G::BS], y[3][G::BS];
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          const float* Ji = Jm + (r0 + p) * G::JS;
#pragma unroll
          for (int u = 0; u < G::BS; ++u) x[p][u] = Ji[cj + u];
#pragma unroll
          for (int v = 0; v < G::BS; ++v) y[p][v] = Ji[ck + v];
        }
        // z_p = hess_c y (per column v), then acc += x_p z_p^T
#pragma unroll
        for (int v = 0; v < G::BS; ++v) {
          const float z0 = __fmaf_rn(h00, y[0][v], __fmaf_rn(h01, y[1][v], h02 * y[2][v]));
          const float z1 = __fmaf_rn(h01, y[0][v], __fmaf_rn(h11, y[1][v], h12 * y[2][v]));
          const float z2 = __fmaf_rn(h02, y[0][v], __fmaf_rn(h12, y[1][v], h22 * y[2][v]));
#pragma unroll
          for (int u = 0; u < G::BS; ++u)
            acc[u][v] = __fmaf_rn(x[0][u], z0, __fmaf_rn(x[1][u], z1, __fmaf_rn(x[2][u], z2,
                                                                                acc[u][v])));
        }
      }
#pragma unroll
      for (int u = 0; u < G::BS; ++u)
#pragma unroll
        for (int v = 0; v < G::BS; ++v) {
          const int rr = cj + u, cc = ck + v;
          if (rr < NV && cc <= rr) L[rr * G::MS + cc] = Mm[rr * G::MS + cc] + acc[u][v];
        }
    }
    __syncwarp();
    return S.factor();
  }

  // ------------------------------------------------------- line search
  // alpha > 0 minimising phi(alpha) = L(a + alpha p) (Eq. 10): safeguarded
  // Newton on the increasing
  //   phi'(alpha) = p^T r + alpha p^T M p
  //                 + sum_c (grad_c(u_c + alpha v_c) - grad_c(u_c)) . v_c,
  // v = J p, with p^T r from the compensated residual and the gradient
  // differences taken at the same (high-part) u, so that the cancellation of
  // p^T (M a - qfrc) against the contact terms near convergence does not
  // bias alpha.  Stops when the Newton update is below 1e-6 alpha.  *dfmax is
  // the largest change of a contact force component over the step.  Steps
  // that are tiny against u take the quadratic model's alpha (below).
  __device__ __forceinline__ float line_search(float p, float* dfmax) {
    const int lane = S.lane;
    S.put_vec(V_P, p);
    const float* vp = S.Vec(V_P);
    float vr[MT];
    S.rows_dot(vp, vr);
#pragma unroll
    for (int t = 0; t < MT; ++t)
      if (S.row_valid(t)) Xh()[lane + 32 * t] = vr[t];
    const float Mp = S.m_times_plain(vp);
    const float pMp = warp_sum(lane < NV ? p * Mp : 0.f);
    float prh, prl;
    two_prod(p, S.r, prh, prl);
    prl = __fmaf_rn(p, S.rlo, prl);
    const float pr = warp_sum(prh) + warp_sum(prl);
    __syncwarp();
    const float* Dm_ = S.Ds();
    float g0[E::MCT][3];
#pragma unroll
    for (int u = 0; u < E::MCT; ++u) {
      const int c = lane + 32 * u;
#pragma unroll
      for (int q = 0; q < 3; ++q) g0[u][q] = 0.f;
      if (c < nc) {
        float uh[3], ul[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int q = 0; q < 3; ++q) uh[q] = Uh()[3 * c + q];
        Cone o;
        cone_eval(uh, ul, Dm_[3 * c], Dm_[3 * c + 1], Mu()[c], false, o);
#pragma unroll
        for (int q = 0; q < 3; ++q) g0[u][q] = o.g[q];
      }
    }
    // The quadratic model at u: alpha0 = -p^T r / (p^T M p + sum_c v^T hess_c(u) v).
    // When alpha0 v is tiny against u (near convergence) the gradient
    // differences below are below FP32 resolution of u; the model is then
    // the line search (its neglected remainder is second order in alpha v).
    // (every contact counts in the smallness test: one outside the cone's
    // force region must not reach it within the step either)
    float hv_lin = 0.f, vrel = 0.f, hvmax = 0.f;
#pragma unroll
    for (int u = 0; u < E::MCT; ++u) {
      const int c = lane + 32 * u;
      if (c < nc) {
        float v[3], un = 0.f, vn = 0.f;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          v[q] = Xh()[3 * c + q];
          un = fmaxf(un, fabsf(Uh()[3 * c + q]));
          vn = fmaxf(vn, fabsf(v[q]));
        }
        const float hv0 = __fmaf_rn(HB(0)[c], v[0], __fmaf_rn(HB(1)[c], v[1], HB(2)[c] * v[2]));
        const float hv1 = __fmaf_rn(HB(1)[c], v[0], __fmaf_rn(HB(3)[c], v[1], HB(4)[c] * v[2]));
        const float hv2 = __fmaf_rn(HB(2)[c], v[0], __fmaf_rn(HB(4)[c], v[1], HB(5)[c] * v[2]));
        hv_lin = __fmaf_rn(hv0, v[0], __fmaf_rn(hv1, v[1], __fmaf_rn(hv2, v[2], hv_lin)));
        hvmax = fmaxf(hvmax, fmaxf(fabsf(hv0), fmaxf(fabsf(hv1), fabsf(hv2))));
        vrel = fmaxf(vrel, vn / fmaxf(un, 1e-30f));
      }
    }
    const float curv0 = pMp + warp_sum(hv_lin);
    const float alpha0 = -pr / curv0;
    if (alpha0 > 0.f && alpha0 * warp_max(vrel) <= 1e-3f) {
      *dfmax = alpha0 * warp_max(hvmax);
      __syncwarp();
      return alpha0;
    }
    float alpha = 1.f, lo = 0.f, hi = CUDART_INF_F, df = 0.f;
#pragma unroll 1
    for (int it = 0; it < 60; ++it) {
      float d1 = 0.f, d2 = 0.f, dfl = 0.f;
#pragma unroll
      for (int u = 0; u < E::MCT; ++u) {
        const int c = lane + 32 * u;
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
      const float d = pr + alpha * pMp + warp_sum(d1);
      const float dd = pMp + warp_sum(d2);
      df = warp_max(dfl);
      if (d == 0.f) break;
      if (d < 0.f) lo = alpha; else hi = alpha;
      float an = alpha - d / dd;
      if (!(an > lo && an < hi)) an = (hi == CUDART_INF_F) ? 2.f * alpha : 0.5f * (lo + hi);
      const bool done = fabsf(an - alpha) <= 1e-6f * alpha;
      alpha = an;
      if (done || (hi - lo) <= 1e-7f * hi) break;
    }
    *dfmax = df;
    __syncwarp();
    return alpha;
  }

  // ------------------------------------------------------------ adjoint
  // H w = rhs + rhs_lo with refinement; lambda_c = hess_c (J w)_c
  // (compensated) in Lam / Lamlo per row.  `full` refines beyond FP32 (the
  // adjoint: the cone parameters' derivatives carry the small component of
  // J w along a contact's stiff direction, about 1e-4 of the rest), to a
  // correction of 1e-9 |w| and a change of lambda of 1e-7 |lambda| (1e-12 /
  // 1e-10 cost 5 % of the solve for the same gradients); otherwise to FP32
  // precision.
  __device__ __forceinline__ void solve_refined(float rhs, float rhs_lo, float& wh, float& wl,
                                                bool full = false) {
    const float step_tol = full ? 1e-9f : kStepTol;
    const float force_tol = full ? 1e-7f : kForceTol;
    const int it_max = full ? 2 * kAdjointRefineMax : kAdjointRefineMax;
    const int lane = S.lane;
    wh = S.chol_solve(rhs);
    wl = 0.f;
    float* Lm = S.Lam();
    float* Lml = S.Lamlo();
    float lam_prev[3 * E::MCT];
#pragma unroll
    for (int k = 0; k < 3 * E::MCT; ++k) lam_prev[k] = 0.f;
    float dmax_prev = CUDART_INF_F;
    float dmax_pp = 0.f;  // the correction before dmax_prev (0: w itself)
#pragma unroll 1
    for (int it = 0; it <= it_max; ++it) {
      S.put_vec(V_WH, wh);
      S.put_vec(V_WL, wl);
      const float* vh = S.Vec(V_WH);
      const float* vl = S.Vec(V_WL);
      rows_to_smem(vh, vl, false, Xh(), Xl());
      float lmax = 0.f, dl = 0.f;
#pragma unroll
      for (int u = 0; u < E::MCT; ++u) {
        const int c = lane + 32 * u;
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
      lmax = warp_max(lmax);
      dl = warp_max(dl);
      __syncwarp();
      if (it > 0) {
        const float wmax = warp_max(fabsf(wh));
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
      float js, jc, ms, mc;
      S.jt_active(Lm, Lml, js, jc);
      S.m_times(vh, vl, ms, mc);
      float t1, e1, t2, e2;
      two_sum(rhs, -ms, t1, e1);
      two_sum(t1, -js, t2, e2);
      float rho = __fadd_rn(t2, __fsub_rn(__fadd_rn(__fadd_rn(e1, e2), rhs_lo), __fadd_rn(mc, jc)));
      if (lane >= NV) rho = 0.f;
      const float dw = S.chol_solve(rho);
      dmax_prev = warp_max(fabsf(dw));
      WarpSolver<NV, MT>::add_to_pair(wh, wl, dw);
    }
    __syncwarp();
  }

  // --------------------------------------------------------- forward
  __device__ __forceinline__ int forward(const Params& P, int* iters) {
    *iters = 0;
    if (!S.factor_M()) return CS_ST_CHOLFAIL;
    S.ah = S.chol_solve(S.qf);
    S.al = 0.f;
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
      const bool same = !__any_sync(kFull, zbits != prev_z);
      if (k > 0 && same && prev_small) return CS_ST_OK;
      // three consecutive steps below the resolution of a with unchanged
      // zones: a has reached its attainable accuracy (stiff contacts keep
      // the forces moving at that level, so the force test alone may not
      // settle)
      if (stall >= 3) return CS_ST_OK;
      if (k >= P.max_iter) return CS_ST_MAXITER;
      if (!assemble_and_factor()) return CS_ST_CHOLFAIL;
      // Newton direction: one FP32 solve with the factor of H.  The residual
      // it solves is compensated and every stop test and returned quantity
      // comes from that residual, so the direction only has to be a good
      // Newton direction; refining it to FP32 resolution (as an earlier
      // version did, when the residual was plain) cost 45 % of the solve and
      // left the Newton steps unchanged (12.26 against 12.28 per solve on
      // the quadruped batch)
      const float p = S.chol_solve(-S.r);
      const float ptr = warp_sum(p * S.r);
      const float amax = warp_max(fabsf(S.ah));
      if (!(ptr < 0.f)) {
        const float pm = warp_max(fabsf(p));
        return (pm <= kStepTol * amax) ? CS_ST_OK : CS_ST_NOPROGRESS;
      }
      float dfm;
      const float alpha = line_search(p, &dfm);
      const float dp = alpha * p;
      WarpSolver<NV, MT>::add_to_pair(S.ah, S.al, dp);
      *iters = k + 1;
      const float smax = warp_max(fabsf(dp));
      // the step is small, or (two consecutive steps in the same zones) the
      // error it leaves, predicted from their contraction ratio q as q / (1 -
      // q) |dp| (conservative where Newton converges quadratically), is; the
      // residual at the new point is still evaluated before returning
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
  // 3c; other rows 0).
  __device__ __forceinline__ void write_grads(const EParams& EP, const cs_inst& e, float wh,
                                              float wl) {
    const Params& P = EP.P;
    const int lane = S.lane, nv = S.nv, m = S.m;
    if (lane < nv) P.dqfrc[e.off_v + lane] = wh;
    const float* Lm = S.Lam();
    const float* F = S.Fs();
#pragma unroll 1
    for (int i = lane; i < m; i += 32) P.daref[e.off_r + i] = Lm[i];
    S.put_vec(V_WH, wh);
    S.put_vec(V_X, S.ah);
    const float* vw = S.Vec(V_WH);
    const float* va = S.Vec(V_X);
    float* dJ = P.dJ + e.off_J;
#pragma unroll 1
    for (int q = lane; q < m * nv; q += 32) {
      const int rr = q / nv, cc = q - rr * nv;
      dJ[q] = -__fmaf_rn(F[rr], vw[cc], Lm[rr] * va[cc]);
    }
    if (P.dM) {
      float* dM = P.dM + e.off_M;
#pragma unroll 1
      for (int q = lane; q < nv * nv; q += 32) {
        const int rr = q / nv, cc = q - rr * nv;
        dM[q] = -0.5f * __fmaf_rn(vw[rr], va[cc], va[rr] * vw[cc]);
      }
    }
    if (P.dD || EP.dmu) {
      // v = J w (hi parts) per row for the contact owners
      S.put_vec(V_WL, wl);
      rows_to_smem(vw, S.Vec(V_WL), false, Xh(), Xl());
      const float* Dm_ = S.Ds();
#pragma unroll
      for (int u = 0; u < E::MCT; ++u) {
        const int c = lane + 32 * u;
        if (c < nc) {
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
            // gv . v = (mu u_T . v_T - v_N t) / t, which cancels when w moves
            // along the cone's surface: formed from the pairs
            float th, tl;
            t_pair(uh, ul, th, tl);
            float s = 0.f, cc = 0.f;
            dot2p(s, cc, uh[1], ul[1], vh[1], vl[1]);
            dot2p(s, cc, uh[2], ul[2], vh[2], vl[2]);
            float uvh, uvl;
            norm_pair(s, cc, uvh, uvl);          // u_T . v_T
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
  }

  __device__ __forceinline__ void zero_grads(const EParams& EP, const cs_inst& e) {
    const Params& P = EP.P;
    const int lane = S.lane, nv = S.nv, m = S.m;
    if (lane < nv) P.dqfrc[e.off_v + lane] = 0.f;
#pragma unroll 1
    for (int i = lane; i < m; i += 32) {
      P.daref[e.off_r + i] = 0.f;
      if (P.dD) P.dD[e.off_r + i] = 0.f;
      if (EP.dmu) EP.dmu[e.off_r + i] = 0.f;
    }
#pragma unroll 1
    for (int q = lane; q < m * nv; q += 32) P.dJ[e.off_J + q] = 0.f;
    if (P.dM)
#pragma unroll 1
      for (int q = lane; q < nv * nv; q += 32) P.dM[e.off_M + q] = 0.f;
  }

  __device__ __forceinline__ void run(const EParams& EP, int b) {
    const Params& P = EP.P;
    const cs_inst e = P.inst[b];
    if (!load(EP, e)) {
      if (S.lane == 0) {
        P.status[b] = CS_ST_BADSHAPE;
        P.iters[b] = 0;
      }
      return;
    }
    S.gj = (S.lane < S.nv) ? __ldg(P.g + e.off_v + S.lane) : 0.f;
    int iters = 0;
    const int st = forward(P, &iters);
    if (S.lane < S.nv) P.a[e.off_v + S.lane] = S.ah;
    if (S.lane == 0) {
      P.status[b] = st;
      P.iters[b] = iters;
    }
    if (st == CS_ST_CHOLFAIL || st == CS_ST_NONFINITE) {
      zero_grads(EP, e);
      return;
    }
    // adjoint at the returned point: H is rebuilt from the Hessian blocks of
    // the last residual evaluation (they vary with a inside zone 1)
    if (!assemble_and_factor()) {
      if (S.lane == 0) P.status[b] = CS_ST_CHOLFAIL;
      zero_grads(EP, e);
      return;
    }
    float wh, wl;
    solve_refined(S.gj, 0.f, wh, wl, true);
    write_grads(EP, e, wh, wl);
  }
};

template <int NV, int MT>
__global__ void __launch_bounds__(256) warp_elliptic_kernel(const __grid_constant__ EParams EP) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  using E = EGeo<NV, MT>;
  const Params& P = EP.P;
  const int warp = threadIdx.x >> 5;
  EllipticSolver<NV, MT> X;
  X.S.sm = reinterpret_cast<float*>(smem_raw + (size_t)warp * E::kBytes);
  X.S.lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  int idx = blockIdx.x * wpb + warp;
  const int stride = gridDim.x * wpb;
#pragma unroll 1
  for (int guard = 0; guard <= P.n_work; ++guard) {
    if (P.counter) {
      int v = 0;
      if (X.S.lane == 0) v = atomicAdd(P.counter, 1);
      idx = __shfl_sync(kFull, v, 0);
    }
    if (idx >= P.n_work) break;
    const int b = P.order ? P.order[idx] : idx;
    if (b >= 0 && b < P.n) X.run(EP, b);
    __syncwarp();
    if (!P.counter) idx += stride;
  }
}

}  // namespace csk
