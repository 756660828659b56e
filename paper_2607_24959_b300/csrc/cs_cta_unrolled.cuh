// cs_cta_unrolled.cuh -- unrolled reverse-mode differentiation of the Newton
// solve for instances beyond one warp (nv up to 128, m up to 1024), one
// 256-thread CTA per instance (device code).
//
// The same comparison path as cs_unrolled.cuh (Section III-E): the forward
// pass records the executed trace of at most K Newton steps (per step the
// factor of H_k, a_k and p_k as float pairs, alpha_k, c1_k and the masks
// S_k, T_k, in the trace layout of UParams), and the reverse sweep
// propagates g = dL/da_K back through it with the formulas stated at the top
// of cs_unrolled.cuh.  Here the rows are spread over the block (thread t
// owns rows t + 256 u), the nv-vectors live in shared-memory slots, and the
// products use CtaSolver's split-K and row routines, so the arithmetic is
// the warp version's in another order.
#pragma once

#include "cs_cta.cuh"
#include "cs_unrolled.cuh"

namespace csk {

// Vector slots beyond the solver's own (CtaVec).
enum CtaUnrollVec {
  CU_RLO = C_PP + 1,  // low part of the residual r
  CU_RH,              // right-hand side of the Newton solve (-r, high)
  CU_RL,              // (-r, low)
  CU_PL,              // low part of p
  CU_S1, CU_S2,       // scratch of the refined solves / J^T pairs
  CU_AB,              // cotangent of a_k
  CU_QB,              // accumulated cotangent of qfrc
  CU_NH, CU_NL,       // a_k + p_k (pair)
  CU_E,               // e_T
  CU_PB,              // cotangent of p_k
  CU_GT,              // H_T p
  CU_NVEC
};

template <int MTC>
__device__ __forceinline__ void cta_unrolled_fwd(CtaSolver<MTC>& S, const UParams& U, int b) {
  const Params& P = U.P;
  const cs_inst e = P.inst[b];
  const int tid = S.tid;
  if (!S.load(P, e)) {
    if (tid == 0) {
      P.status[b] = CS_ST_BADSHAPE;
      P.iters[b] = 0;
    }
    return;
  }
  const int nv = S.nv;
  const int64_t tv = P.total_v;
  int steps = 0, st = CS_ST_MAXITER;
  float* ah = S.V(C_AH);
  float* al = S.V(C_AL);
  float* pv = S.V(C_P);
  float* pl = S.V(CU_PL);
  S.rlo_slot = CU_RLO;
  if (!S.factor_M()) {
    st = CS_ST_CHOLFAIL;
    for (int j = tid; j < S.geo.nvcap; j += kCtaThreads) ah[j] = 0.f;
    __syncthreads();
  } else {
    // a_0 = M^-1 qfrc (Eq. 1), refined
    S.set_active(0u);
    S.fmask_bits = 0u;
    S.fmask_valid = true;
    S.solve_refined(C_QF, -1, C_AH, C_AL, C_X, C_MP, CU_S1, CU_S2, kStepTol, kForceTol);
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
      // p = -H^-1 r with r kept as a pair
      for (int j = tid; j < S.geo.nvcap; j += kCtaThreads) {
        S.V(CU_RH)[j] = -S.V(C_R)[j];
        S.V(CU_RL)[j] = -S.V(CU_RLO)[j];
      }
      __syncthreads();
      S.solve_refined(CU_RH, CU_RL, C_P, CU_PL, C_X, C_MP, CU_S1, CU_S2, kStepTol, kForceTol);
      const float ptr = S.block_sum(tid < nv ? pv[tid] * S.V(C_R)[tid] : 0.f);
      if (!(ptr < 0.f)) {
        const float pm = S.block_max(tid < nv ? fabsf(pv[tid]) : 0.f);
        const float am = S.block_max(tid < nv ? fabsf(ah[tid]) : 0.f);
        st = (pm <= kStepTol * am) ? CS_ST_OK : CS_ST_NOPROGRESS;
        break;
      }
      float dfm;
      bool crossed;
      float alpha = S.line_search(&dfm, &crossed);  // leaves s_r = J p
      // no breakpoint before alpha: the root lies on the first segment, where
      // the Newton step is exact (alpha = 1, T = S), which ends the solve
      if (!crossed) alpha = 1.f;
      uint32_t tb = 0;
      float cs = 0.f;
#pragma unroll
      for (int u = 0; u < MTC; ++u) {
        const bool on_t = crossed
                              ? (S.row_valid(u) && __fmaf_rn(alpha, S.s_r[u], S.jar_r[u]) < 0.f)
                              : (((S.act_bits >> u) & 1u) != 0u);
        if (on_t) {
          tb |= 1u << u;
          cs = __fmaf_rn(S.D_r[u] * S.s_r[u], S.s_r[u], cs);
        }
      }
      // c1 = p^T M p + sum_T D s^2
      float pmp = 0.f;
      if (tid < nv) {
        const float* Mr = S.Ms() + tid * S.geo.MS;
        float mp = 0.f;
#pragma unroll 1
        for (int q = 0; q < nv; ++q) mp = __fmaf_rn(Mr[q], pv[q], mp);
        pmp = pv[tid] * mp;
      }
      S.block_sum2(pmp, cs);
      const float c1 = pmp + cs;
      // record step k
      float* sl = U.trace + (int64_t)k * U.slot;
      S.store_factor(sl + e.off_M);
      for (int j = tid; j < nv; j += kCtaThreads) {
        float* v = sl + P.total_M + e.off_v + j;
        v[0] = ah[j];
        v[tv] = al[j];
        v[2 * tv] = pv[j];
        v[3 * tv] = pl[j];
      }
      if (tid == 0) {
        sl[P.total_M + 4 * tv + 2 * (int64_t)b] = alpha;
        sl[P.total_M + 4 * tv + 2 * (int64_t)b + 1] = c1;
      }
      uint8_t* tm = U.tmask + (int64_t)k * P.total_r + e.off_r;
#pragma unroll
      for (int u = 0; u < MTC; ++u)
        if (S.row_valid(u))
          tm[S.row(u)] = (uint8_t)(((S.act_bits >> u) & 1u) | (((tb >> u) & 1u) << 1));
      __syncthreads();
      if (tid < nv) {
        float hh = ah[tid], ll = al[tid];
        if (crossed) {
          WarpSolver<1, 1>::add_to_pair(hh, ll, alpha * pv[tid]);
        } else {
          WarpSolver<1, 1>::add_to_pair(hh, ll, pv[tid]);
          WarpSolver<1, 1>::add_to_pair(hh, ll, pl[tid]);
        }
        ah[tid] = hh;
        al[tid] = ll;
      }
      __syncthreads();
      steps = k + 1;
      if (!crossed) { st = CS_ST_OK; break; }
    }
  }
  for (int j = tid; j < nv; j += kCtaThreads) P.a[e.off_v + j] = ah[j];
  if (tid == 0) {
    P.status[b] = st;
    P.iters[b] = steps;
  }
}

template <int MTC>
__device__ __forceinline__ void cta_unrolled_zero(CtaSolver<MTC>& S, const Params& P,
                                                  const cs_inst& e) {
  const int nv = S.nv, m = S.m, tid = S.tid;
  for (int j = tid; j < nv; j += kCtaThreads) P.dqfrc[e.off_v + j] = 0.f;
  for (int i = tid; i < m; i += kCtaThreads) {
    P.daref[e.off_r + i] = 0.f;
    P.dD[e.off_r + i] = 0.f;
  }
  for (int q = tid; q < m * nv; q += kCtaThreads) P.dJ[e.off_J + q] = 0.f;
  for (int q = tid; q < nv * nv; q += kCtaThreads) P.dM[e.off_M + q] = 0.f;
}

// jar = J (vh + vl) - aref for this thread's rows, compensated.
template <int MTC>
__device__ __forceinline__ void cta_jar_at(CtaSolver<MTC>& S, const float* vh, const float* vl,
                                           float (&jh)[MTC], float (&jl)[MTC]) {
  float sj[MTC], cj[MTC];
  S.rows_dot(vh, vl, true, sj, cj);
#pragma unroll
  for (int u = 0; u < MTC; ++u) {
    float t, te;
    two_sum(sj[u], -S.aref_r[u], t, te);
    const float tl = __fadd_rn(te, cj[u]);
    jh[u] = __fadd_rn(t, tl);
    jl[u] = __fsub_rn(tl, __fsub_rn(jh[u], t));
  }
}

// dJ_i += U_i x^T + V_i y^T + W_i z^T (U, V, W in Fs(), Flo(), Lam()).  Each
// thread updates the same entries in every call.
template <int MTC>
__device__ __forceinline__ void cta_jb_update(CtaSolver<MTC>& S, float* dJ, const float* x,
                                              const float* y, const float* z) {
  const int nv = S.nv;
  const float* U1 = S.Fs();
  const float* V1 = S.Flo();
  const float* W1 = S.Lam();
#pragma unroll 1
  for (int q = S.tid; q < S.m * nv; q += kCtaThreads) {
    const int rr = q / nv, cc = q - rr * nv;
    dJ[q] += __fmaf_rn(U1[rr], x[cc], __fmaf_rn(V1[rr], y[cc], W1[rr] * z[cc]));
  }
}

template <int MTC>
__device__ __forceinline__ void cta_unrolled_bwd(CtaSolver<MTC>& S, const UParams& U, int b) {
  const Params& P = U.P;
  const cs_inst e = P.inst[b];
  const int tid = S.tid;
  if (!S.load(P, e)) return;  // the forward pass marked it CS_ST_BADSHAPE
  const int nv = S.nv, m = S.m, nc = S.geo.nvcap;
  const int64_t tv = P.total_v;
  const int st0 = P.status[b];
  if (st0 == CS_ST_CHOLFAIL || st0 == CS_ST_NONFINITE || st0 == CS_ST_BADSHAPE) {
    cta_unrolled_zero(S, P, e);
    return;
  }
  int steps = P.iters[b];
  steps = steps < 0 ? 0 : (steps > P.max_iter ? P.max_iter : steps);
  float* ab = S.V(CU_AB);
  float* qb = S.V(CU_QB);
  float* ah = S.V(C_AH);
  float* al = S.V(C_AL);
  float* pv = S.V(C_P);
  float* pl = S.V(CU_PL);
  float* nh = S.V(CU_NH);
  float* nl = S.V(CU_NL);
  float* wh = S.V(C_WH);
  for (int j = tid; j < nc; j += kCtaThreads) {
    ab[j] = (j < nv) ? __ldg(P.g + e.off_v + j) : 0.f;
    qb[j] = 0.f;
  }
  float Db[MTC], arb[MTC];
#pragma unroll
  for (int u = 0; u < MTC; ++u) {
    Db[u] = 0.f;
    arb[u] = 0.f;
  }
  float* dJ = P.dJ + e.off_J;
  float* dM = P.dM + e.off_M;
  for (int q = tid; q < m * nv; q += kCtaThreads) dJ[q] = 0.f;
  for (int q = tid; q < nv * nv; q += kCtaThreads) dM[q] = 0.f;
  __syncthreads();
  float* U1 = S.Fs();
  float* V1 = S.Flo();
  float* W1 = S.Lam();
#pragma unroll 1
  for (int k = steps - 1; k >= 0; --k) {
    const float* sl = U.trace + (int64_t)k * U.slot;
    S.load_factor(sl + e.off_M);
    for (int j = tid; j < nc; j += kCtaThreads) {
      const float* v = sl + P.total_M + e.off_v + j;
      const bool in = j < nv;
      ah[j] = in ? v[0] : 0.f;
      al[j] = in ? v[tv] : 0.f;
      pv[j] = in ? v[2 * tv] : 0.f;
      pl[j] = in ? v[3 * tv] : 0.f;
    }
    const float alpha = sl[P.total_M + 4 * tv + 2 * (int64_t)b];
    const float c1 = sl[P.total_M + 4 * tv + 2 * (int64_t)b + 1];
    const uint8_t* tm = U.tmask + (int64_t)k * P.total_r + e.off_r;
    uint32_t sbits = 0, tbits = 0;
#pragma unroll
    for (int u = 0; u < MTC; ++u)
      if (S.row_valid(u)) {
        const uint8_t x = tm[S.row(u)];
        sbits |= (uint32_t)(x & 1u) << u;
        tbits |= (uint32_t)((x >> 1) & 1u) << u;
      }
    const bool exact = alpha == 1.f && !S.block_any(sbits != tbits);  // block_any syncs
    S.set_active(sbits);
    S.fmask_bits = sbits;
    S.fmask_valid = true;
    // n = a_k + p_k, the point after a full step
    if (tid < nv) {
      float hh = ah[tid], ll = al[tid];
      WarpSolver<1, 1>::add_to_pair(hh, ll, pv[tid]);
      WarpSolver<1, 1>::add_to_pair(hh, ll, pl[tid]);
      nh[tid] = hh;
      nl[tid] = ll;
    }
    for (int j = nv + tid; j < nc; j += kCtaThreads) {
      nh[j] = 0.f;
      nl[j] = 0.f;
    }
    __syncthreads();
    if (exact) {
      // a' = a + p, the exact minimiser on S: the reverse is the IFT adjoint
      // at a' and nothing flows to a_k
      float jh[MTC], jl[MTC];
      cta_jar_at(S, nh, nl, jh, jl);
      S.solve_refined(CU_AB, -1, C_WH, C_WL, C_X, C_MP, CU_S1, CU_S2, kStepTol, kForceTol);
#pragma unroll
      for (int u = 0; u < MTC; ++u) {
        if (!S.row_valid(u)) continue;
        const int i = S.row(u);
        const float lam = W1[i];  // Lam() = D_S . J w
        const bool on_s = (sbits >> u) & 1u;
        const float fp = on_s ? S.D_r[u] * jh[u] : 0.f;
        if (on_s) Db[u] -= __fdiv_rn(lam * jh[u], S.D_r[u]);
        arb[u] += lam;
        U1[i] = 0.f;
        V1[i] = -fp;
        W1[i] = -lam;
      }
      __syncthreads();
      cta_jb_update(S, dJ, wh, wh, nh);
#pragma unroll 1
      for (int q = tid; q < nv * nv; q += kCtaThreads) {
        const int rr = q / nv, cc = q - rr * nv;
        dM[q] -= wh[rr] * nh[cc];
      }
      if (tid < nv) {
        qb[tid] += wh[tid];
        ab[tid] = 0.f;
      }
      __syncthreads();
      continue;
    }
    // recompute the step's quantities at a_k
    float jl[MTC];
    cta_jar_at(S, ah, al, S.jar_r, jl);
    // s = J p and jar + s (the row's value after a full step, small on stiff
    // rows of S) from the pairs, compensated
    float sjr[MTC], sjl[MTC];
    {
      float sh[MTC], sc[MTC];
      S.rows_dot(pv, pl, true, sh, sc);
#pragma unroll
      for (int u = 0; u < MTC; ++u) {
        S.s_r[u] = __fadd_rn(sh[u], sc[u]);
        const float slo = __fsub_rn(sc[u], __fsub_rn(S.s_r[u], sh[u]));
        float t, te;
        two_sum(S.jar_r[u], S.s_r[u], t, te);
        const float tl = __fadd_rn(te, __fadd_rn(jl[u], slo));
        sjr[u] = __fadd_rn(t, tl);
        sjl[u] = __fsub_rn(tl, __fsub_rn(sjr[u], t));
      }
    }
    // e_T = M (a + p) - qfrc + J^T (D_T . (jar + s)), compensated with the T
    // rows as the active list; H_T p = M p + J^T (D_T . s)
    S.set_active(tbits);
#pragma unroll
    for (int u = 0; u < MTC; ++u) {
      if (!S.row_valid(u)) continue;
      const int i = S.row(u);
      const bool on_t = (tbits >> u) & 1u;
      float fh = 0.f, fl = 0.f;
      if (on_t) WarpSolver<1, 1>::scale_pair(S.D_r[u], sjr[u], sjl[u], fh, fl);
      U1[i] = fh;
      V1[i] = fl;
      W1[i] = on_t ? S.D_r[u] * S.s_r[u] : 0.f;
    }
    __syncthreads();
    {
      const float* Jm = S.Js();
      const float* Mm = S.Ms();
      const int* idx = S.Idx();
      const int JS = S.geo.JS, MS = S.geo.MS;
      S.split_dot(nv, S.nact, true,
                  [&](int j, int q, float& a, float& h, float& l) {
                    const int i = idx[q];
                    a = Jm[i * JS + j];
                    h = U1[i];
                    l = V1[i];
                  },
                  S.V(CU_S1), S.V(CU_S2));  // J^T (D_T . (jar + s)) pair
      S.split_dot(nv, nv, true,
                  [&](int j, int q, float& a, float& h, float& l) {
                    a = Mm[j * MS + q];
                    h = nh[q];
                    l = nl[q];
                  },
                  S.V(C_X), S.V(C_MP));  // M (a + p) pair
      if (tid < nv) {
        float t1, e1, t2, e2;
        two_sum(S.V(C_X)[tid], -S.V(C_QF)[tid], t1, e1);
        two_sum(t1, S.V(CU_S1)[tid], t2, e2);
        S.V(CU_E)[tid] = __fadd_rn(
            t2, __fadd_rn(__fadd_rn(e1, e2), __fadd_rn(S.V(C_MP)[tid], S.V(CU_S2)[tid])));
      }
      S.split_dot(nv, nv, false,
                  [&](int j, int q, float& a, float& h, float& l) {
                    a = Mm[j * MS + q];
                    h = pv[q];
                    l = 0.f;
                  },
                  S.V(C_X), S.V(C_MP));  // M p
      S.split_dot(nv, S.nact, false,
                  [&](int j, int q, float& a, float& h, float& l) {
                    const int i = idx[q];
                    a = Jm[i * JS + j];
                    h = W1[i];
                    l = 0.f;
                  },
                  S.V(CU_GT), S.V(C_MP));  // J^T (D_T . s) over the T rows
      if (tid < nv) S.V(CU_GT)[tid] = S.V(C_X)[tid] + S.V(CU_GT)[tid];
    }
    S.set_active(sbits);
    // alpha = -c0 / c1
    const float alpha_b = S.block_sum(tid < nv ? ab[tid] * pv[tid] : 0.f);
    const float c0b = -alpha_b / c1, c1b = -alpha_b * alpha / c1;
    float akb = 0.f;
    if (tid < nv) {
      const float eT = S.V(CU_E)[tid], gT = S.V(CU_GT)[tid];
      S.V(CU_PB)[tid] = __fmaf_rn(alpha, ab[tid], __fmaf_rn(c0b, eT, (2.f * c1b - c0b) * gT));
      akb = __fmaf_rn(1.f - alpha, __fmaf_rn(-2.f * alpha_b / c1, gT, ab[tid]), -c0b * eT);
    }
    for (int j = nv + tid; j < nc; j += kCtaThreads) S.V(CU_PB)[j] = 0.f;
    float jarb[MTC], sbr[MTC];
#pragma unroll
    for (int u = 0; u < MTC; ++u) {
      const bool on_t = (tbits >> u) & 1u;
      const float Ds = S.D_r[u] * S.s_r[u];
      sbr[u] = on_t ? __fmaf_rn(c0b * S.D_r[u], S.jar_r[u], 2.f * c1b * Ds) : 0.f;
      jarb[u] = on_t ? c0b * Ds : 0.f;
      if (on_t) Db[u] += __fmaf_rn(c0b * S.s_r[u], S.jar_r[u], c1b * S.s_r[u] * S.s_r[u]);
    }
    __syncthreads();
    // z = H_S^-1 pb (C_WH / C_WL)
    S.solve_refined(CU_PB, -1, C_WH, C_WL, C_X, C_MP, CU_S1, CU_S2, kStepTol, kForceTol);
    // J z (compensated) and the row coefficients of the rank-3 update of Jb
    float sj[MTC], cj[MTC];
    S.rows_dot(wh, S.V(C_WL), true, sj, cj);
#pragma unroll
    for (int u = 0; u < MTC; ++u) {
      const bool on_s = (sbits >> u) & 1u;
      const float jz = __fadd_rn(sj[u], cj[u]);
      const float Djz = on_s ? S.D_r[u] * jz : 0.f;
      const float w = jarb[u] - Djz;
      if (on_s) Db[u] -= jz * sjr[u];
      arb[u] -= w;
      if (S.row_valid(u)) {
        const int i = S.row(u);
        U1[i] = sbr[u] - Djz;
        V1[i] = on_s ? -S.D_r[u] * sjr[u] : 0.f;
        W1[i] = w;
      }
    }
    __syncthreads();
    cta_jb_update(S, dJ, pv, wh, ah);
#pragma unroll 1
    for (int q = tid; q < nv * nv; q += kCtaThreads) {
      const int rr = q / nv, cc = q - rr * nv;
      dM[q] += __fmaf_rn(pv[rr], __fmaf_rn(c0b, ah[cc], c1b * pv[cc]),
                         -wh[rr] * (pv[cc] + ah[cc]));
    }
    if (tid < nv) {
      qb[tid] += wh[tid] - c0b * pv[tid];
      ab[tid] = akb;
    }
    __syncthreads();
  }
  // a_0 = M^-1 qfrc
  float* a0 = S.V(CU_NH);
  for (int j = tid; j < nc; j += kCtaThreads)
    a0[j] = (j < nv) ? (steps > 0 ? U.trace[P.total_M + e.off_v + j] : P.a[e.off_v + j]) : 0.f;
  __syncthreads();
  if (!S.factor_M()) {
    cta_unrolled_zero(S, P, e);
    if (tid == 0) P.status[b] = CS_ST_CHOLFAIL;
    return;
  }
  S.set_active(0u);
  S.solve_refined(CU_AB, -1, C_WH, C_WL, C_X, C_MP, CU_S1, CU_S2, kStepTol, kForceTol);
  if (tid < nv) qb[tid] += wh[tid];
#pragma unroll 1
  for (int q = tid; q < nv * nv; q += kCtaThreads) {
    const int rr = q / nv, cc = q - rr * nv;
    dM[q] -= wh[rr] * a0[cc];
  }
  __syncthreads();
  // gradient for a symmetric M
#pragma unroll 1
  for (int q = tid; q < nv * nv; q += kCtaThreads) {
    const int rr = q / nv, cc = q - rr * nv;
    if (rr < cc) {
      const float x = 0.5f * (dM[q] + dM[cc * nv + rr]);
      dM[q] = x;
      dM[cc * nv + rr] = x;
    }
  }
  for (int j = tid; j < nv; j += kCtaThreads) P.dqfrc[e.off_v + j] = qb[j];
#pragma unroll
  for (int u = 0; u < MTC; ++u)
    if (S.row_valid(u)) {
      P.daref[e.off_r + S.row(u)] = arb[u];
      P.dD[e.off_r + S.row(u)] = Db[u];
    }
}

// DIR 0: forward with trace; DIR 1: reverse sweep.  Static round-robin over
// instances, one CTA each.
template <int MTC, int DIR>
__global__ void __launch_bounds__(kCtaThreads, 1)
    cta_unrolled_kernel(const __grid_constant__ UParams U, const CtaGeo geo) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  CtaSolver<MTC> S;
  S.sm = reinterpret_cast<float*>(smem_raw);
  S.geo = geo;
  S.tid = threadIdx.x;
  S.lane = threadIdx.x & 31;
  S.warp = threadIdx.x >> 5;
#pragma unroll 1
  for (int b = blockIdx.x; b < U.P.n; b += gridDim.x) {
    if (DIR == 0)
      cta_unrolled_fwd(S, U, b);
    else
      cta_unrolled_bwd(S, U, b);
    __syncthreads();
  }
}

}  // namespace csk
