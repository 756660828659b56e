// cs_unrolled.cuh -- unrolled reverse-mode differentiation of the Newton
// solve, one warp per instance (device code).
//
// This is the comparison path of Section III-E: instead of the IFT adjoint
// (Eq. 17), which keeps only the converged point, the forward pass records
// the executed trace of at most K Newton steps and the backward pass
// propagates the cotangent g = dL/da_K back through every step.  The trace
// grows linearly with K (per step: the factor of H_k, a_k as a float pair,
// p_k, alpha_k, c1_k and the masks S_k, T_k), which is what the paper
// measures against the constant IFT state.
//
// Each step applies the smooth map (masks held fixed)
//   jar = J a - aref,  S = {jar < 0},  f = D_S jar,  r = M a - qfrc + J^T f,
//   H = M + J_S^T D_S J_S,  p = -H^-1 r,  s = J p,
//   alpha = -c0 / c1 on the line-search segment T = {jar + alpha s < 0}:
//     c0 = p^T (M a - qfrc) + sum_T D s jar,  c1 = p^T M p + sum_T D s^2,
//   a' = a + alpha p.
// Its reverse (cotangents xb; H_T p = M p + J^T (D_T . s) and
// e_T = M (a + p) - qfrc + J^T (D_T . (jar + s)), the residual of the
// segment's rows after a full step; z = H_S^-1 pb):
//   alpha_b = ab . p,  c0b = -alpha_b / c1,  c1b = -alpha_b alpha / c1,
//   pb  = alpha ab + c0b e_T + (2 c1b - c0b) H_T p,
//   a_b = (1 - alpha) (ab - 2 alpha_b / c1 H_T p) - c0b e_T
//   (the grouping in which nothing cancels as alpha -> 1),
//   sb  = T . (c0b D jar + 2 c1b D s),
//   Mb += p (c0b a + c1b p)^T - z (p + a)^T,  qfrcb += z - c0b p,
//   Jb += u p^T + v z^T + w a^T  with  u = sb - S . D (J z),
//         v = -S . D (jar + s),  w = T . c0b D s - S . D (J z),
//   Db += T . (c0b s jar + c1b s^2) - S . (J z) (jar + s),  arefb -= w
// (jar + s, the row after a full step, nearly vanishes on stiff rows of S
// and is formed from compensated pairs).
// A step that crosses no breakpoint is the exact Newton step on S (alpha = 1,
// T = S): its output a' = H_S^-1 (qfrc + J_S^T D_S aref) does not depend on
// a, so a_b = 0 and its reverse is the IFT adjoint at a' (w = H_S^-1 ab:
// qfrcb += w, arefb += D_S J w, Jb -= f' w^T + (D_S J w) a'^T, Mb -= w a'^T,
// Db -= (J w) jar').  The general formulas reach the same values only through
// cancellation, which FP32 cannot resolve.  Finally a_0 = M^-1 qfrc:
// y = M^-1 ab, qfrcb += y, Mb -= y a_0^T; the gradient for a symmetric M is
// (Mb + Mb^T) / 2.
//
// Precision: a_k and p_k are float pairs; r (right-hand side of the Newton
// solve), jar, jar + s, e_T and J z are compensated; every solve with H_k or M is
// refined with compensated residuals, so the FP32 trace follows the FP64 one
// closely enough to differentiate it.
#pragma once

#include "cs_warp.cuh"

namespace csk {

struct UParams {
  Params P;          // batch, options (max_iter = K, tol), a, g, outputs, status, iters
  float* trace;      // K slots of `slot` floats (layout below)
  uint8_t* tmask;    // K slots of total_r bytes: bit 0 = S_k, bit 1 = T_k
  int64_t slot;      // floats per slot: total_M + 4 total_v + 2 n
};
// Slot k of instance b: factor of H_k (packed lower rows) at off_M, then the
// nv-vectors a_k (high part), a_k (low part), p_k (high), p_k (low) at
// total_M + {0, 1, 2, 3} total_v + off_v, and (alpha_k, c1_k) at
// total_M + 4 total_v + 2 b.

template <int NV, int MT>
__device__ __forceinline__ void set_active(WarpSolver<NV, MT>& S, uint32_t bits) {
  int* idx = S.Idx();
  int base = 0;
#pragma unroll
  for (int t = 0; t < MT; ++t) {
    if (32 * t < S.m) {
      const bool on = ((bits >> t) & 1u) && S.row_valid(t);
      const unsigned bal = __ballot_sync(kFull, on);
      if (on) idx[base + __popc(bal & ((1u << S.lane) - 1u))] = S.lane + 32 * t;
      base += __popc(bal);
    }
  }
  S.nact = base;
  S.act_bits = bits;
  __syncwarp();
}

// Sum over all rows i of J_ij x_i (x in shared memory, zero off the rows
// that contribute), for lane j.
template <int NV, int MT>
__device__ __forceinline__ float jt_rows(WarpSolver<NV, MT>& S, const float* x) {
  using G = Geo<NV, MT>;
  const float* Jm = S.Js();
  float s0 = 0.f, s1 = 0.f;
  if (S.lane < NV) {
    int i = 0;
#pragma unroll 1
    for (; i + 1 < S.m; i += 2) {
      s0 = __fmaf_rn(Jm[i * G::JS + S.lane], x[i], s0);
      s1 = __fmaf_rn(Jm[(i + 1) * G::JS + S.lane], x[i + 1], s1);
    }
    if (i < S.m) s0 = __fmaf_rn(Jm[i * G::JS + S.lane], x[i], s0);
  }
  return s0 + s1;
}

template <int NV, int MT>
__device__ __forceinline__ void unrolled_fwd(WarpSolver<NV, MT>& S, const UParams& U, int b) {
  const Params& P = U.P;
  const cs_inst e = P.inst[b];
  const int lane = S.lane;
  if (!S.load(P, e)) {
    if (lane == 0) {
      P.status[b] = CS_ST_BADSHAPE;
      P.iters[b] = 0;
    }
    return;
  }
  const int64_t tv = P.total_v;
  int steps = 0, st = CS_ST_MAXITER;
  if (!S.factor_M()) {
    st = CS_ST_CHOLFAIL;
    S.ah = 0.f;
  } else {
    // a_0 = M^-1 qfrc (Eq. 1), refined
    set_active(S, 0u);
    S.fmask_bits = 0u;
    S.fmask_valid = true;
    S.solve_refined(S.qf, 0.f, S.ah, S.al);
#pragma unroll 1
    for (int k = 0;; ++k) {
      float scale;
      bool bad;
      const float rmax = S.residual(&scale, &bad, true);
      if (bad) { st = CS_ST_NONFINITE; break; }
      if (rmax <= P.tol * scale) { st = CS_ST_OK; break; }
      if (k >= P.max_iter) { st = CS_ST_MAXITER; break; }
      if (S.need_refactor())
        if (!S.assemble_and_factor()) { st = CS_ST_CHOLFAIL; break; }
      float ph, pl;
      S.solve_refined(-S.r, -S.rlo, ph, pl);  // p = -H^-1 r, r kept as a pair
      const float p = ph;
      const float ptr = warp_sum(p * S.r);
      if (!(ptr < 0.f)) {
        const float pm = warp_max(fabsf(p)), amax = warp_max(fabsf(S.ah));
        st = (pm <= kStepTol * amax) ? CS_ST_OK : CS_ST_NOPROGRESS;
        break;
      }
      float dfm;
      bool crossed;
      float alpha = S.line_search(p, &dfm, &crossed);  // leaves s_r = J p
      // no breakpoint before alpha: the root lies on the first segment, where
      // the Newton step is exact (alpha = 1, T = S), which ends the solve
      if (!crossed) alpha = 1.f;
      uint32_t tb = 0;
      float cs = 0.f;
#pragma unroll
      for (int t = 0; t < MT; ++t) {
        const bool on_t = crossed ? (S.row_valid(t) && __fmaf_rn(alpha, S.s_r[t], S.jar_r[t]) < 0.f)
                                  : (((S.act_bits >> t) & 1u) != 0u);
        if (on_t) {
          tb |= 1u << t;
          cs = __fmaf_rn(S.D_r[t] * S.s_r[t], S.s_r[t], cs);
        }
      }
      const float Mp = S.m_times_plain(S.Vec(V_P));
      const float c1 = warp_sum(lane < NV ? p * Mp : 0.f) + warp_sum(cs);
      // record step k
      float* sl = U.trace + (int64_t)k * U.slot;
      S.store_factor(sl + e.off_M);
      if (lane < S.nv) {
        float* v = sl + P.total_M + e.off_v + lane;
        v[0] = S.ah;
        v[tv] = S.al;
        v[2 * tv] = ph;
        v[3 * tv] = pl;
      }
      if (lane == 0) {
        sl[P.total_M + 4 * tv + 2 * (int64_t)b] = alpha;
        sl[P.total_M + 4 * tv + 2 * (int64_t)b + 1] = c1;
      }
      uint8_t* tm = U.tmask + (int64_t)k * P.total_r + e.off_r;
#pragma unroll
      for (int t = 0; t < MT; ++t)
        if (S.row_valid(t))
          tm[lane + 32 * t] = (uint8_t)(((S.act_bits >> t) & 1u) | (((tb >> t) & 1u) << 1));
      if (crossed) {
        WarpSolver<NV, MT>::add_to_pair(S.ah, S.al, alpha * p);
      } else {
        WarpSolver<NV, MT>::add_to_pair(S.ah, S.al, ph);
        WarpSolver<NV, MT>::add_to_pair(S.ah, S.al, pl);
      }
      steps = k + 1;
      if (!crossed) { st = CS_ST_OK; break; }
    }
  }
  if (lane < S.nv) P.a[e.off_v + lane] = S.ah;
  if (lane == 0) {
    P.status[b] = st;
    P.iters[b] = steps;
  }
}

template <int NV, int MT>
__device__ __forceinline__ void unrolled_zero(WarpSolver<NV, MT>& S, const Params& P,
                                              const cs_inst& e) {
  const int nv = S.nv, m = S.m;
  if (S.lane < nv) P.dqfrc[e.off_v + S.lane] = 0.f;
#pragma unroll 1
  for (int i = S.lane; i < m; i += 32) {
    P.daref[e.off_r + i] = 0.f;
    P.dD[e.off_r + i] = 0.f;
  }
#pragma unroll 1
  for (int q = S.lane; q < m * nv; q += 32) P.dJ[e.off_J + q] = 0.f;
#pragma unroll 1
  for (int q = S.lane; q < nv * nv; q += 32) P.dM[e.off_M + q] = 0.f;
}

// jar = J (vh + vl) - aref for this lane's rows, compensated (high parts).
template <int NV, int MT>
__device__ __forceinline__ void jar_at(WarpSolver<NV, MT>& S, const float* vh, const float* vl,
                                       float (&jh)[MT], float (&jl)[MT]) {
  float sj[MT], cj[MT];
  S.rows_dot2(vh, vl, sj, cj);
#pragma unroll
  for (int t = 0; t < MT; ++t) {
    float u, ue;
    two_sum(sj[t], -S.aref_r[t], u, ue);
    const float tl = __fadd_rn(ue, cj[t]);
    jh[t] = __fadd_rn(u, tl);
    jl[t] = __fsub_rn(tl, __fsub_rn(jh[t], u));
  }
}

// Rank-3 update of the instance's Jb (rows u, v, w in Fs, Flo, Lam) with the
// broadcast vectors x, y, z: Jb_i += u_i x^T + v_i y^T + w_i z^T.
template <int NV, int MT>
__device__ __forceinline__ void jb_update(WarpSolver<NV, MT>& S, float* dJ, const float* x,
                                          const float* y, const float* z) {
  const int nv = S.nv;
  const float* U1 = S.Fs();
  const float* V1 = S.Flo();
  const float* W1 = S.Lam();
#pragma unroll 1
  for (int q = S.lane; q < S.m * nv; q += 32) {
    const int rr = q / nv, cc = q - rr * nv;
    dJ[q] += __fmaf_rn(U1[rr], x[cc], __fmaf_rn(V1[rr], y[cc], W1[rr] * z[cc]));
  }
}

template <int NV, int MT>
__device__ __forceinline__ void unrolled_bwd(WarpSolver<NV, MT>& S, const UParams& U, int b) {
  const Params& P = U.P;
  const cs_inst e = P.inst[b];
  const int lane = S.lane;
  if (!S.load(P, e)) return;  // the forward pass marked it CS_ST_BADSHAPE
  const int nv = S.nv, m = S.m;
  const int64_t tv = P.total_v;
  const int st0 = P.status[b];
  if (st0 == CS_ST_CHOLFAIL || st0 == CS_ST_NONFINITE || st0 == CS_ST_BADSHAPE) {
    unrolled_zero(S, P, e);
    return;
  }
  int steps = P.iters[b];
  steps = steps < 0 ? 0 : (steps > P.max_iter ? P.max_iter : steps);
  float ab = (lane < nv) ? __ldg(P.g + e.off_v + lane) : 0.f;
  float qb = 0.f;
  float Db[MT], arb[MT];
#pragma unroll
  for (int t = 0; t < MT; ++t) { Db[t] = 0.f; arb[t] = 0.f; }
  float* dJ = P.dJ + e.off_J;
  float* dM = P.dM + e.off_M;
#pragma unroll 1
  for (int q = lane; q < m * nv; q += 32) dJ[q] = 0.f;
#pragma unroll 1
  for (int q = lane; q < nv * nv; q += 32) dM[q] = 0.f;
  __syncwarp();
#pragma unroll 1
  for (int k = steps - 1; k >= 0; --k) {
    const float* sl = U.trace + (int64_t)k * U.slot;
    S.load_factor(sl + e.off_M);
    const float* v = sl + P.total_M + e.off_v + lane;
    S.ah = (lane < nv) ? v[0] : 0.f;
    S.al = (lane < nv) ? v[tv] : 0.f;
    const float p = (lane < nv) ? v[2 * tv] : 0.f;
    const float plo = (lane < nv) ? v[3 * tv] : 0.f;
    const float alpha = sl[P.total_M + 4 * tv + 2 * (int64_t)b];
    const float c1 = sl[P.total_M + 4 * tv + 2 * (int64_t)b + 1];
    const uint8_t* tm = U.tmask + (int64_t)k * P.total_r + e.off_r;
    uint32_t sbits = 0, tbits = 0;
#pragma unroll
    for (int t = 0; t < MT; ++t)
      if (S.row_valid(t)) {
        const uint8_t x = tm[lane + 32 * t];
        sbits |= (uint32_t)(x & 1u) << t;
        tbits |= (uint32_t)((x >> 1) & 1u) << t;
      }
    const bool exact = alpha == 1.f && !__any_sync(kFull, sbits != tbits);
    set_active(S, sbits);
    S.fmask_bits = sbits;
    S.fmask_valid = true;
    if (exact) {
      // a' = a + p, the exact minimiser on S: the reverse is the IFT adjoint
      // at a' and nothing flows to a_k
      float nh = S.ah, nl = S.al;
      WarpSolver<NV, MT>::add_to_pair(nh, nl, p);
      WarpSolver<NV, MT>::add_to_pair(nh, nl, plo);
      S.put_vec(V_AH, nh);
      S.put_vec(V_AL, nl);
      float jh[MT], jl[MT];
      jar_at(S, S.Vec(V_AH), S.Vec(V_AL), jh, jl);
      float wh, wl;
      S.solve_refined(ab, 0.f, wh, wl);  // Lam = D_S . J w
      const float* Lm = S.Lam();
      float lam_r[MT];
#pragma unroll
      for (int t = 0; t < MT; ++t) lam_r[t] = S.row_valid(t) ? Lm[lane + 32 * t] : 0.f;
      __syncwarp();
      float* U1 = S.Fs();
      float* V1 = S.Flo();
      float* W1 = S.Lam();
#pragma unroll
      for (int t = 0; t < MT; ++t) {
        const bool on_s = (sbits >> t) & 1u;
        const float fp = on_s ? S.D_r[t] * jh[t] : 0.f;
        if (on_s) Db[t] -= __fdiv_rn(lam_r[t] * jh[t], S.D_r[t]);
        arb[t] += lam_r[t];
        if (S.row_valid(t)) {
          U1[lane + 32 * t] = 0.f;
          V1[lane + 32 * t] = -fp;
          W1[lane + 32 * t] = -lam_r[t];
        }
      }
      S.put_vec(V_WH, wh);
      __syncwarp();
      const float* vw = S.Vec(V_WH);
      const float* va = S.Vec(V_AH);
      jb_update(S, dJ, vw, vw, va);
#pragma unroll 1
      for (int q = lane; q < nv * nv; q += 32) {
        const int rr = q / nv, cc = q - rr * nv;
        dM[q] -= vw[rr] * va[cc];
      }
      qb += wh;
      ab = 0.f;
      __syncwarp();
      continue;
    }
    // recompute the step's quantities at a_k
    S.put_vec(V_AH, S.ah);
    S.put_vec(V_AL, S.al);
    S.put_vec(V_P, p);
    S.put_vec(V_X, plo);
    const float* va = S.Vec(V_AH);
    const float* vp = S.Vec(V_P);
    float jl[MT];
    jar_at(S, va, S.Vec(V_AL), S.jar_r, jl);
    // s = J p and jar + s (the row's value after a full step, small on stiff
    // rows of S) from the pairs, compensated
    float sjr[MT], sjl[MT];
    {
      float sh[MT], sc[MT];
      S.rows_dot2(vp, S.Vec(V_X), sh, sc);
#pragma unroll
      for (int t = 0; t < MT; ++t) {
        S.s_r[t] = __fadd_rn(sh[t], sc[t]);
        const float slo = __fsub_rn(sc[t], __fsub_rn(S.s_r[t], sh[t]));
        float u, ue;
        two_sum(S.jar_r[t], S.s_r[t], u, ue);
        const float tl = __fadd_rn(ue, __fadd_rn(jl[t], slo));
        sjr[t] = __fadd_rn(u, tl);
        sjl[t] = __fsub_rn(tl, __fsub_rn(sjr[t], u));
      }
    }
    // e_T = r_T + H_T p = M (a + p) - qfrc + J^T (D_T . (jar + s)), the
    // segment's residual after a full step, compensated with the T rows as
    // the active list; H_T p = M p + J^T (D_T . s)
    set_active(S, tbits);
    float* X1 = S.Fs();
    float* X2 = S.Flo();
    float* X3 = S.Lam();
#pragma unroll
    for (int t = 0; t < MT; ++t) {
      const bool on_t = (tbits >> t) & 1u;
      float fh = 0.f, fl = 0.f;
      if (on_t) WarpSolver<NV, MT>::scale_pair(S.D_r[t], sjr[t], sjl[t], fh, fl);
      if (S.row_valid(t)) {
        X1[lane + 32 * t] = fh;
        X2[lane + 32 * t] = fl;
        X3[lane + 32 * t] = on_t ? S.D_r[t] * S.s_r[t] : 0.f;
      }
    }
    float nh = S.ah, nl = S.al;
    WarpSolver<NV, MT>::add_to_pair(nh, nl, p);
    WarpSolver<NV, MT>::add_to_pair(nh, nl, plo);
    S.put_vec(V_WH, nh);
    S.put_vec(V_WL, nl);
    float js, jc, ms, mc;
    S.jt_active(X1, X2, js, jc);
    S.m_times(S.Vec(V_WH), S.Vec(V_WL), ms, mc);
    float t1, e1, t2, e2;
    two_sum(ms, -S.qf, t1, e1);
    two_sum(t1, js, t2, e2);
    float eT = __fadd_rn(t2, __fadd_rn(__fadd_rn(e1, e2), __fadd_rn(mc, jc)));
    const float Mp = S.m_times_plain(vp);
    float gT = Mp + jt_rows(S, X3);
    if (lane >= nv) {
      eT = 0.f;
      gT = 0.f;
    }
    set_active(S, sbits);
    // alpha = -c0 / c1
    const float alpha_b = warp_sum(ab * p);
    const float c0b = -alpha_b / c1, c1b = -alpha_b * alpha / c1;
    float pb = __fmaf_rn(alpha, ab, __fmaf_rn(c0b, eT, (2.f * c1b - c0b) * gT));
    float akb = __fmaf_rn(1.f - alpha, __fmaf_rn(-2.f * alpha_b / c1, gT, ab), -c0b * eT);
    if (lane >= nv) {
      pb = 0.f;
      akb = 0.f;
    }
    float jarb[MT], sbr[MT];
#pragma unroll
    for (int t = 0; t < MT; ++t) {
      const bool on_t = (tbits >> t) & 1u;
      const float Ds = S.D_r[t] * S.s_r[t];
      sbr[t] = on_t ? __fmaf_rn(c0b * S.D_r[t], S.jar_r[t], 2.f * c1b * Ds) : 0.f;
      jarb[t] = on_t ? c0b * Ds : 0.f;
      if (on_t) Db[t] += __fmaf_rn(c0b * S.s_r[t], S.jar_r[t], c1b * S.s_r[t] * S.s_r[t]);
    }
    float zh, zl;
    S.solve_refined(pb, 0.f, zh, zl);  // z = H_S^-1 pb (uses Lam / Lamlo as scratch)
    // J z (compensated) and the row coefficients of the rank-3 update of Jb
    S.put_vec(V_WH, zh);
    S.put_vec(V_WL, zl);
    float sj[MT], cj[MT];
    S.rows_dot2(S.Vec(V_WH), S.Vec(V_WL), sj, cj);
    float* U1 = S.Fs();
    float* V1 = S.Flo();
    float* W1 = S.Lam();
#pragma unroll
    for (int t = 0; t < MT; ++t) {
      const bool on_s = (sbits >> t) & 1u;
      const float jz = __fadd_rn(sj[t], cj[t]);
      const float Djz = on_s ? S.D_r[t] * jz : 0.f;
      const float w = jarb[t] - Djz;
      if (on_s) Db[t] -= jz * sjr[t];
      arb[t] -= w;
      if (S.row_valid(t)) {
        U1[lane + 32 * t] = sbr[t] - Djz;
        V1[lane + 32 * t] = on_s ? -S.D_r[t] * sjr[t] : 0.f;
        W1[lane + 32 * t] = w;
      }
    }
    __syncwarp();
    const float* vz = S.Vec(V_WH);
    jb_update(S, dJ, vp, vz, va);
#pragma unroll 1
    for (int q = lane; q < nv * nv; q += 32) {
      const int rr = q / nv, cc = q - rr * nv;
      dM[q] += __fmaf_rn(vp[rr], __fmaf_rn(c0b, va[cc], c1b * vp[cc]),
                         -vz[rr] * (vp[cc] + va[cc]));
    }
    qb += zh - c0b * p;
    ab = akb;
    __syncwarp();
  }
  // a_0 = M^-1 qfrc
  float a0 = 0.f;
  if (steps > 0) {
    a0 = (lane < nv) ? U.trace[P.total_M + e.off_v + lane] : 0.f;
  } else {
    a0 = (lane < nv) ? P.a[e.off_v + lane] : 0.f;
  }
  if (!S.factor_M()) {
    unrolled_zero(S, P, e);
    if (lane == 0) P.status[b] = CS_ST_CHOLFAIL;
    return;
  }
  set_active(S, 0u);
  float yh, yl;
  S.solve_refined(ab, 0.f, yh, yl);
  qb += yh;
  S.put_vec(V_WH, yh);
  S.put_vec(V_X, a0);
  const float* vy = S.Vec(V_WH);
  const float* v0 = S.Vec(V_X);
#pragma unroll 1
  for (int q = lane; q < nv * nv; q += 32) {
    const int rr = q / nv, cc = q - rr * nv;
    dM[q] -= vy[rr] * v0[cc];
  }
  __syncwarp();
  // gradient for a symmetric M
#pragma unroll 1
  for (int q = lane; q < nv * nv; q += 32) {
    const int rr = q / nv, cc = q - rr * nv;
    if (rr < cc) {
      const float x = 0.5f * (dM[q] + dM[cc * nv + rr]);
      dM[q] = x;
      dM[cc * nv + rr] = x;
    }
  }
  if (lane < nv) P.dqfrc[e.off_v + lane] = qb;
#pragma unroll
  for (int t = 0; t < MT; ++t)
    if (S.row_valid(t)) {
      P.daref[e.off_r + lane + 32 * t] = arb[t];
      P.dD[e.off_r + lane + 32 * t] = Db[t];
    }
}

// DIR 0: forward with trace; DIR 1: reverse sweep.  Static round-robin over
// instances.
template <int NV, int MT, int DIR>
__global__ void __launch_bounds__(256) warp_unrolled_kernel(const __grid_constant__ UParams U) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  using G = Geo<NV, MT>;
  const int warp = threadIdx.x >> 5;
  WarpSolver<NV, MT> S;
  S.sm = reinterpret_cast<float*>(smem_raw + (size_t)warp * G::kBytes);
  S.lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
#pragma unroll 1
  for (int b = blockIdx.x * wpb + warp; b < U.P.n; b += gridDim.x * wpb) {
    if (DIR == 0)
      unrolled_fwd(S, U, b);
    else
      unrolled_bwd(S, U, b);
    __syncwarp();
  }
}

}  // namespace csk
