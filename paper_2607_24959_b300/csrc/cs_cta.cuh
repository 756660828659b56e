// cs_cta.cuh -- one-CTA-per-instance contact solver for instances beyond one
// warp (nv up to 128 DoF, m up to 1024 rows): the same algorithm as
// cs_warp.cuh (Section III: Eqs. 1, 5-10 forward, Eq. 17 adjoint, compensated
// residuals, exact line search), spread over a 256-thread block.
//
// Work split:
//  * row-parallel quantities (jar, J p, line-search sums, lambda): thread t
//    owns rows t + 256 u, u < MTC;
//  * transposed products (J^T f, J^T lambda) and M-products: split-K over
//    (column, row-group) threads, partial float pairs reduced in shared
//    memory;
//  * H = M + J_act^T D J_act: 4x4 register blocks of the lower triangle,
//    split over groups of active rows when there are few blocks;
//  * Cholesky: blocked right-looking in shared memory over 32-column panels
//    (warp 0 factors the diagonal block, all threads solve the panel below
//    it and update the trailing matrix; see factor());
//  * triangular solves: one warp, four unknowns per shuffle round, no block
//    barrier inside (see tri_solve_warp()).
#pragma once

#include "cs_warp.cuh"

namespace csk {

constexpr int kCtaThreads = 256;
constexpr int kCtaWarps = kCtaThreads / 32;
constexpr int kCtaNvMax = 128;

// Shared-memory geometry for given capacities (runtime, identical on host and
// device).
struct CtaGeo {
  int nvcap, mcap;      // capacities (nvcap multiple of 4)
  int MS, JS;           // odd row strides
  int oM, oL, oJ, oD, oF, oLam, oFlo, oLamlo, oIdx, oVec, oScr, oRed, words;
  __host__ __device__ static CtaGeo make(int nv_max, int m_max, int nvec = 13) {
    CtaGeo g;
    g.nvcap = (nv_max + 3) & ~3;
    g.mcap = (m_max + 31) & ~31;
    if (g.mcap < 32) g.mcap = 32;
    g.MS = g.nvcap | 1;
    g.JS = g.nvcap | 1;
    g.oM = 0;
    g.oL = g.oM + g.nvcap * g.MS;
    g.oJ = g.oL + g.nvcap * g.MS;
    g.oD = g.oJ + g.mcap * g.JS;
    g.oF = g.oD + g.mcap;
    g.oLam = g.oF + g.mcap;
    g.oFlo = g.oLam + g.mcap;
    g.oLamlo = g.oFlo + g.mcap;
    g.oIdx = g.oLamlo + g.mcap;
    g.oVec = g.oIdx + g.mcap;
    g.oScr = g.oVec + nvec * g.nvcap;
    // split-K partials: 2 floats per thread for the transposed products, and
    // 16 per (block, row group) for the Newton matrix when it is split
    const int nb = g.nvcap >> 2, nbl = nb * (nb + 1) / 2;
    const int R = nbl >= kCtaThreads ? 1 : (kCtaThreads / nbl < 16 ? kCtaThreads / nbl : 16);
    const int scr = R > 1 && 16 * nbl * R > 2 * kCtaThreads ? 16 * nbl * R : 2 * kCtaThreads;
    g.oRed = g.oScr + scr;
    g.words = g.oRed + 8 * kCtaWarps + 8;  // two reduction buffers [0, 4 warps),
                                            // the factor's pivot flag [4 warps + 7],
                                            // compaction counts [5 warps, 6 warps)
    return g;
  }
  __host__ __device__ size_t bytes() const { return ((size_t)words * 4 + 127) & ~(size_t)127; }
};

enum CtaVec { C_AH = 0, C_AL, C_P, C_WH, C_WL, C_R, C_MAQ, C_QF, C_G, C_DINV, C_X, C_MP, C_PP };

template <int MTC>
struct CtaSolver {
  float* sm;
  CtaGeo geo;
  int tid, lane, warp;
  int nv, m, nact;
  float aref_r[MTC], D_r[MTC], jar_r[MTC], s_r[MTC];
  uint32_t act_bits, fmask_bits;
  bool fmask_valid;
  float fmax, qmax;
  int rb = 0;  // reduction buffer the next block reduction uses
  int rlo_slot = -1;  // if set, residual() also writes r's low part there

  __device__ __forceinline__ float* Ms() { return sm + geo.oM; }
  __device__ __forceinline__ float* Ls() { return sm + geo.oL; }
  __device__ __forceinline__ float* Js() { return sm + geo.oJ; }
  __device__ __forceinline__ float* Ds() { return sm + geo.oD; }
  __device__ __forceinline__ float* Fs() { return sm + geo.oF; }
  __device__ __forceinline__ float* Lam() { return sm + geo.oLam; }
  __device__ __forceinline__ float* Flo() { return sm + geo.oFlo; }
  __device__ __forceinline__ float* Lamlo() { return sm + geo.oLamlo; }
  __device__ __forceinline__ int* Idx() { return reinterpret_cast<int*>(sm + geo.oIdx); }
  __device__ __forceinline__ float* V(int s) { return sm + geo.oVec + s * geo.nvcap; }
  __device__ __forceinline__ float* Scr() { return sm + geo.oScr; }
  __device__ __forceinline__ float* Red() { return sm + geo.oRed; }
  __device__ __forceinline__ int row(int u) const { return tid + kCtaThreads * u; }
  __device__ __forceinline__ bool row_valid(int u) const { return row(u) < m; }

  // ------------------------------------------------------ block reductions
  // All threads call these (uniform control flow).  Consecutive reductions
  // alternate between two slot buffers, so one barrier per reduction
  // suffices: a thread can write a buffer again only after passing the next
  // reduction's barrier, which every thread reaches only after reading this
  // one's partials.
  __device__ __forceinline__ float* red_buffer() {
    float* R = Red() + rb * 2 * kCtaWarps;
    rb ^= 1;
    return R;
  }
  __device__ __forceinline__ float block_sum(float v) {
    v = warp_sum(v);
    float* R = red_buffer();
    if (lane == 0) R[warp] = v;
    __syncthreads();
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < kCtaWarps; ++w) t += R[w];
    return t;
  }
  __device__ __forceinline__ void block_sum2(float& a, float& b) {
    a = warp_sum(a);
    b = warp_sum(b);
    float* R = red_buffer();
    if (lane == 0) {
      R[warp] = a;
      R[kCtaWarps + warp] = b;
    }
    __syncthreads();
    float ta = 0.f, tb = 0.f;
#pragma unroll
    for (int w = 0; w < kCtaWarps; ++w) {
      ta += R[w];
      tb += R[kCtaWarps + w];
    }
    a = ta;
    b = tb;
  }
  __device__ __forceinline__ float block_max(float v) {
    v = warp_max(v);
    float* R = red_buffer();
    if (lane == 0) R[warp] = v;
    __syncthreads();
    float t = R[0];
#pragma unroll
    for (int w = 1; w < kCtaWarps; ++w) t = fmaxf(t, R[w]);
    return t;
  }
  __device__ __forceinline__ bool block_any(bool p) {
    return __syncthreads_or(p ? 1 : 0) != 0;
  }

  // ------------------------------------------------------------- loading
  __device__ __forceinline__ bool load(const Params& P, const cs_inst& e) {
    nv = e.nv;
    m = e.m;
    if (nv < 1 || nv > geo.nvcap || m < 0 || m > geo.mcap || m > kCtaThreads * MTC) return false;
    if (e.off_M < 0 || e.off_J < 0 || e.off_v < 0 || e.off_r < 0) return false;
    if (e.off_M + (int64_t)nv * nv > P.total_M) return false;
    if (e.off_J + (int64_t)m * nv > P.total_J) return false;
    if (e.off_v + nv > P.total_v || e.off_r + m > P.total_r) return false;
    const float* M = P.M + e.off_M;
    const float* J = P.J + e.off_J;
    float* Ms_ = Ms();
    float* Js_ = Js();
    const int nc = geo.nvcap;
#pragma unroll 4
    for (int q = tid; q < nc * nc; q += kCtaThreads) {
      const int rr = q / nc, cc = q - rr * nc;
      Ms_[rr * geo.MS + cc] =
          (rr < nv && cc < nv) ? __ldg(M + rr * nv + cc) : (rr == cc ? 1.f : 0.f);
    }
#pragma unroll 4
    for (int q = tid; q < m * nv; q += kCtaThreads) {
      const int rr = q / nv, cc = q - rr * nv;
      Js_[rr * geo.JS + cc] = __ldg(J + q);
    }
    const int padc = geo.JS - nv;
#pragma unroll 1
    for (int q = tid; q < m * padc; q += kCtaThreads) {
      const int rr = q / padc, cc = nv + (q - rr * padc);
      Js_[rr * geo.JS + cc] = 0.f;
    }
#pragma unroll
    for (int u = 0; u < MTC; ++u) {
      const int i = row(u);
      const bool v = i < m;
      aref_r[u] = v ? __ldg(P.aref + e.off_r + i) : 0.f;
      D_r[u] = v ? __ldg(P.D + e.off_r + i) : 0.f;
      if (i < geo.mcap) Ds()[i] = D_r[u];
    }
    float* qv = V(C_QF);
    for (int j = tid; j < nc; j += kCtaThreads) qv[j] = (j < nv) ? __ldg(P.qfrc + e.off_v + j) : 0.f;
    __syncthreads();
    float qm = 0.f;
    for (int j = tid; j < nv; j += kCtaThreads) qm = fmaxf(qm, fabsf(qv[j]));
    qmax = block_max(qm);
    return true;
  }

  // ------------------------------------------------------------- Cholesky
  // Blocked right-looking Cholesky, in place on the lower rows of Ls() (the
  // padded rows are identity), panels of 32 columns:
  //  1. the 32 x 32 diagonal block by warp 0 with the block in registers
  //     (lane l holds row kb + l; right-looking over the block's columns, the
  //     pivot broadcast by a shuffle and each column's entries by shuffles,
  //     the next pivot's update taken off the shuffle chain), as the warp
  //     solver factors its whole matrix; a narrower last panel is padded
  //     with identity rows and columns inside the registers;
  //  2. the rows below it by all warps, four rows at a time per warp with a
  //     row's panel entries spread over the lanes: forward substitution
  //     against the diagonal block column by column (L_ic = x_c / L_cc,
  //     broadcast by a shuffle, then x_j -= L_ic L_jc on the lanes j > c);
  //  3. the trailing matrix updated by all threads in 2x2 register blocks.
  // Three barriers per panel.  Returns false on a non-positive pivot.
  //
  // Measured on the nv96 workload (clock64 per phase, two CTAs per SM): the
  // left-looking diagonal block with four-column rounds took about 9.6 k
  // cycles per block, the register one 5.7 k; the panel solve with four
  // threads per row and a warp barrier per column about 12.5 k per panel,
  // one thread per row (two warps busy) 14.8 k.
  //
  // Both helpers are static (every operand passed explicitly): a non-inlined
  // member function would take the solver object by address and move it to
  // local memory for the whole kernel.
  __device__ static __noinline__ bool factor_diag_block(float* L, float* dv, int MS, int lane,
                                                        int kb, int bs) {
    float* Lr = L + (kb + min(lane, bs - 1)) * MS + kb;
    float h[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) {
      const bool real = lane < bs && c <= lane;
      h[c] = real ? Lr[c] : (c == lane ? 1.f : 0.f);
    }
    float diag = 1.f, piv = h[0];
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      const float d = __shfl_sync(kFull, piv, k);
      const float rs = rsqrtf(d);
      const float lkk = d * rs;
      const float l = (lane == k) ? lkk : h[k] * rs;
      h[k] = l;
      diag = (lane == k) ? lkk : diag;
      if (k + 1 < 32) piv = __fmaf_rn(-l, l, h[k + 1]);
#pragma unroll
      for (int c = k + 1; c < 32; ++c) h[c] = __fmaf_rn(-l, __shfl_sync(kFull, l, c), h[c]);
    }
    if (lane < bs) {
#pragma unroll
      for (int c = 0; c < 32; ++c)
        if (c <= lane) Lr[c] = h[c];
      dv[kb + lane] = 1.0f / diag;
    }
    return !__any_sync(kFull, lane < bs && !(diag > 0.f && diag < CUDART_INF_F));
  }

  // Rows [r0, nc) of the full panel kb (32 columns): L_i = H_i L_kk^-T.  Each
  // warp takes every eighth row, four rows at a time, with a row's 32 panel
  // entries spread over the lanes (lane c holds column c); column by column
  // the lane that owns column c scales it by the reciprocal pivot and
  // broadcasts it, and the lanes after it subtract its multiple of the
  // diagonal block's column c, which each lane reads once per column for
  // all four rows.
  __device__ static __noinline__ void panel_solve(float* L, const float* dv, int MS, int lane,
                                                  int warp, int kb, int r0, int nc) {
    const float dl = dv[kb + lane];
    const float* Lk = L + kb * MS + kb + lane * MS;  // row kb + lane of the block
#pragma unroll 1
    for (int i0 = r0 + 4 * warp; i0 < nc; i0 += 4 * kCtaWarps) {
      float x[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) x[u] = (i0 + u < nc) ? L[(i0 + u) * MS + kb + lane] : 0.f;
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const float lj = (lane > c) ? Lk[c] : 0.f;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float y = __shfl_sync(kFull, x[u] * dl, c);
          x[u] = (lane == c) ? y : __fmaf_rn(-y, lj, x[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (i0 + u < nc) L[(i0 + u) * MS + kb + lane] = x[u];
    }
  }

  __device__ __forceinline__ bool factor() {
    float* L = Ls();
    const int nc = geo.nvcap, MS = geo.MS;
    bool ok = true;
#pragma unroll 1
    for (int kb = 0; kb < nc; kb += 32) {
      const int bs = min(32, nc - kb);
      if (warp == 0) {
        ok = factor_diag_block(L, V(C_DINV), MS, lane, kb, bs) && ok;
        if (lane == 0) Red()[4 * kCtaWarps + 7] = ok ? 1.f : 0.f;
      }
      __syncthreads();
      const int r0 = kb + bs, nrows = nc - r0;
      if (nrows > 0) panel_solve(L, V(C_DINV), MS, lane, warp, kb, r0, nc);
      __syncthreads();
      if (nrows > 0) {
        const int nb2 = (nrows + 1) >> 1;
        const int nblk = nb2 * (nb2 + 1) / 2;
#pragma unroll 1
        for (int w = tid; w < nblk; w += kCtaThreads) {
          int bi = (int)((sqrtf(8.f * (float)w + 1.f) - 1.f) * 0.5f);
          while (bi * (bi + 1) / 2 > w) --bi;
          while ((bi + 1) * (bi + 2) / 2 <= w) ++bi;
          const int bj = w - bi * (bi + 1) / 2;
          const int i0 = r0 + 2 * bi, j0 = r0 + 2 * bj;
          const int i1 = min(i0 + 1, nc - 1), j1 = min(j0 + 1, nc - 1);
          const float* A0 = L + i0 * MS + kb;
          const float* A1 = L + i1 * MS + kb;
          const float* B0 = L + j0 * MS + kb;
          const float* B1 = L + j1 * MS + kb;
          float c00 = 0.f, c01 = 0.f, c10 = 0.f, c11 = 0.f;
#pragma unroll 4
          for (int pp = 0; pp < bs; ++pp) {
            const float a0 = A0[pp], a1 = A1[pp], b0 = B0[pp], b1 = B1[pp];
            c00 = __fmaf_rn(a0, b0, c00);
            c01 = __fmaf_rn(a0, b1, c01);
            c10 = __fmaf_rn(a1, b0, c10);
            c11 = __fmaf_rn(a1, b1, c11);
          }
          L[i0 * MS + j0] -= c00;
          if (j0 + 1 <= i0 && j0 + 1 < nc) L[i0 * MS + j0 + 1] -= c01;
          if (i0 + 1 < nc) {
            L[(i0 + 1) * MS + j0] -= c10;
            if (j0 + 1 <= i0 + 1 && j0 + 1 < nc) L[(i0 + 1) * MS + j0 + 1] -= c11;
          }
        }
      }
      __syncthreads();
    }
    const bool all_ok = Red()[4 * kCtaWarps + 7] != 0.f;  // warp 0's running flag
    __syncthreads();
    return all_ok;
  }

  // x <- (L L^T)^-1 x by one warp, with no block barrier inside: lane l
  // holds x at rows l, l + 32, l + 64, l + 96.  Forward substitution takes
  // the unknowns four at a time: the four are gathered by shuffles, each lane
  // solves their 4 x 4 diagonal block itself (the same operations in the same
  // order as column-at-a-time substitution), and every lane subtracts their
  // contributions from its own rows below them, one column after the other.
  // The backward substitution with L^T does the same from the last four
  // unknowns up, reading L's rows (the transposed entries of each column).
  // The register index of a lane's rows is fixed in each unrolled copy of
  // the outer loop, so x stays in registers.
  //
  // Measured on the nv96 workload: the blocked version (warp 0 on the
  // diagonal blocks, all warps on the coupling products, a block barrier
  // between) took 17 k cycles per solve; one warp alone takes a few thousand.
  __device__ static __noinline__ void tri_solve_warp(const float* L, const float* dv, float* X,
                                                     int MS, int nc, int lane) {
    float xr[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = lane + 32 * j;
      xr[j] = (r < nc) ? X[r] : 0.f;
    }
    // forward: L y = x
#pragma unroll
    for (int jb = 0; jb < 4; ++jb) {
      if (32 * jb >= nc) break;
      const int cend = min(32, nc - 32 * jb);
#pragma unroll 2
      for (int c0 = 0; c0 < cend; c0 += 4) {
        const int cb = 32 * jb + c0;
        float y[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) y[u] = __shfl_sync(kFull, xr[jb], c0 + u);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float* Lu = L + (cb + u) * MS + cb;
#pragma unroll
          for (int w = 0; w < u; ++w) y[u] = __fmaf_rn(-Lu[w], y[w], y[u]);
          y[u] = y[u] * dv[cb + u];
        }
#pragma unroll
        for (int j = jb; j < 4; ++j) {
          const int r = lane + 32 * j;
          if (r > cb + 3 && r < nc) {
            const float* Lr = L + r * MS + cb;
#pragma unroll
            for (int u = 0; u < 4; ++u) xr[j] = __fmaf_rn(-Lr[u], y[u], xr[j]);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (lane == c0 + u) xr[jb] = y[u];
      }
    }
    // backward: L^T x = y
#pragma unroll
    for (int jb = 3; jb >= 0; --jb) {
      if (32 * jb >= nc) continue;
      const int cend = min(32, nc - 32 * jb);
#pragma unroll 2
      for (int c0 = cend - 4; c0 >= 0; c0 -= 4) {
        const int ct = 32 * jb + c0;
        float z[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) z[u] = __shfl_sync(kFull, xr[jb], c0 + u);
#pragma unroll
        for (int u = 3; u >= 0; --u) {
#pragma unroll
          for (int w = 3; w > u; --w) z[u] = __fmaf_rn(-L[(ct + w) * MS + ct + u], z[w], z[u]);
          z[u] = z[u] * dv[ct + u];
        }
#pragma unroll
        for (int j = 0; j <= jb; ++j) {
          const int r = lane + 32 * j;
          if (r < ct) {
#pragma unroll
            for (int w = 3; w >= 0; --w) xr[j] = __fmaf_rn(-L[(ct + w) * MS + r], z[w], xr[j]);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (lane == c0 + u) xr[jb] = z[u];
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = lane + 32 * j;
      if (r < nc) X[r] = xr[j];
    }
  }

  // x (shared vector slot `slot`, nvcap entries) <- (L L^T)^-1 x.  The other
  // warps wait at the barrier.
  __device__ __forceinline__ void chol_solve(int slot) {
    if (warp == 0) tri_solve_warp(Ls(), V(C_DINV), V(slot), geo.MS, geo.nvcap, lane);
    __syncthreads();
  }

  __device__ __forceinline__ bool factor_M() {
    const float* Mm = Ms();
    float* L = Ls();
    const int nc = geo.nvcap, MS = geo.MS;
    for (int q = tid; q < nc * nc; q += kCtaThreads) {
      const int rr = q / nc, cc = q - rr * nc;
      if (cc <= rr) L[rr * MS + cc] = Mm[rr * MS + cc];
    }
    __syncthreads();
    return factor();
  }

  // H = M + sum_{active} D_i J_i^T J_i (Eq. 9) into Ls(), then factor.  4x4
  // register blocks of the lower triangle, split over groups of active rows
  // when there are few blocks.
  __device__ __forceinline__ bool assemble_and_factor() {
    const float* Mm = Ms();
    const float* Jm = Js();
    const float* Dm = Ds();
    const int* idx = Idx();
    float* L = Ls();
    float* scr = Scr();
    const int nc = geo.nvcap, MS = geo.MS, JS = geo.JS;
    const int nb = nc >> 2;                 // 4x4 blocks per edge
    const int nbl = nb * (nb + 1) / 2;      // lower blocks
    const int R = max(1, min(kCtaThreads / nbl, 16));  // row groups (split-K)
    const int items = nbl * R;
#pragma unroll 1
    for (int w = tid; w < items; w += kCtaThreads) {
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
      for (int q = grp; q < nact; q += R) {
        const int i = idx[q];
        const float d = Dm[i];
        const float* Ji = Jm + i * JS;
        float x[4], y[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) x[a] = Ji[cj + a] * d;
#pragma unroll
        for (int b = 0; b < 4; ++b) y[b] = Ji[ck + b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = __fmaf_rn(x[a], y[b], acc[a][b]);
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
      for (int w = tid; w < nbl * 16; w += kCtaThreads) {
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
    const bool ok = factor();
    fmask_bits = act_bits;
    fmask_valid = true;
    return ok;
  }

  __device__ __forceinline__ bool need_refactor() {
    return block_any(!fmask_valid || act_bits != fmask_bits);
  }

  // ---------------------------------------------------- split-K products
  // out (compensated pair per column j < ncols) of sum_q A(j, q) v_q where the
  // q range is split over R = 256 / ncols groups.  get(j, q, &a, &vh, &vl).
  template <class Get>
  __device__ __forceinline__ void split_dot(int ncols, int nq, bool precise, Get get,
                                            float* out_s, float* out_c) {
    const int R = max(1, kCtaThreads / max(ncols, 1));
    float* scr = Scr();
    const int col = tid % max(ncols, 1), grp = tid / max(ncols, 1);
    float s = 0.f, c = 0.f;
    if (grp < R && col < ncols) {
#pragma unroll 4
      for (int q = grp; q < nq; q += R) {
        float a, vh, vl;
        get(col, q, a, vh, vl);
        if (precise) dot2(s, c, a, vh, vl);
        else s = __fmaf_rn(a, vh, s);
      }
      scr[2 * (grp * ncols + col)] = s;
      scr[2 * (grp * ncols + col) + 1] = c;
    }
    __syncthreads();
    if (tid < ncols) {
      float ts = scr[2 * tid], tc = scr[2 * tid + 1];
      for (int gq = 1; gq < R; ++gq) add_pair(ts, tc, scr[2 * (gq * ncols + tid)], scr[2 * (gq * ncols + tid) + 1]);
      out_s[tid] = ts;
      out_c[tid] = tc;
    }
    __syncthreads();
  }

  // jar-like row products: s[u] + c[u] = J_i . (vh + vl) for own rows.
  __device__ __forceinline__ void rows_dot(const float* vh, const float* vl, bool precise,
                                           float (&s)[MTC], float (&c)[MTC]) {
    const float* Jm = Js();
    const int JS = geo.JS;
#pragma unroll
    for (int u = 0; u < MTC; ++u) {
      s[u] = 0.f;
      c[u] = 0.f;
    }
    if (32 * warp >= m) return;  // no row of this warp is valid
#pragma unroll 4
    for (int k = 0; k < nv; ++k) {
      const float xh = vh[k], xl = vl[k];
#pragma unroll
      for (int u = 0; u < MTC; ++u) {
        if (kCtaThreads * u + 32 * warp < m) {
          const float a = Jm[min(row(u), m - 1) * JS + k];
          if (precise) dot2(s[u], c[u], a, xh, xl);
          else s[u] = __fmaf_rn(a, xh, s[u]);
        }
      }
    }
  }

  // ------------------------------------------------------------ residual
  // At a = (C_AH + C_AL): jar, active set + list, f, r (C_R), Ma - qfrc
  // (C_MAQ).  Returns max|r|, *scale, *bad.
  __device__ __forceinline__ float residual(float* scale, bool* bad, bool precise) {
    const float* vh = V(C_AH);
    const float* vl = V(C_AL);
    float s[MTC], c[MTC];
    rows_dot(vh, vl, precise, s, c);
    act_bits = 0;
    float* F = Fs();
    int* idx = Idx();
    float* Rd = Red() + 5 * kCtaWarps;  // compaction counts (own slots)
    float fm = 0.f;
    int base = 0;
#pragma unroll
    for (int u = 0; u < MTC; ++u) {
      if (kCtaThreads * u < m) {
        float t, te;
        two_sum(s[u], -aref_r[u], t, te);
        const float tl = __fadd_rn(te, c[u]);
        jar_r[u] = __fadd_rn(t, tl);
        const float jlo = __fsub_rn(tl, __fsub_rn(jar_r[u], t));
        const bool on = row_valid(u) && jar_r[u] < 0.f;
        float f = 0.f, flo = 0.f;
        if (on) WarpSolver<1, 1>::scale_pair(D_r[u], jar_r[u], jlo, f, flo);
        if (row_valid(u)) {
          F[row(u)] = f;
          Flo()[row(u)] = flo;
        }
        fm = fmaxf(fm, fabsf(f));
        // block-wide compaction in row order
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
          act_bits |= 1u << u;
          idx[before + __popc(bal & ((1u << lane) - 1u))] = row(u);
        }
        base = total;
        __syncthreads();
      }
    }
    nact = base;
    fmax = block_max(fm);
    // J^T f over active rows and M a, split-K
    const float* Jm = Js();
    const float* Mm = Ms();
    const int JS = geo.JS, MS = geo.MS;
    float* x = V(C_X);
    float* mp = V(C_MP);
    const float* Fl = Flo();
    split_dot(nv, nact, precise,
              [&](int j, int q, float& a, float& h, float& l) {
                const int i = idx[q];
                a = Jm[i * JS + j];
                h = F[i];
                l = Fl[i];
              },
              x, mp);  // x = (J^T f)_hi, mp = lo
    float* ms_s = V(C_R);
    float* ms_c = V(C_MAQ);
    split_dot(nv, nv, precise,
              [&](int j, int k, float& a, float& h, float& l) {
                a = Mm[j * MS + k];
                h = vh[k];
                l = vl[k];
              },
              ms_s, ms_c);
    float rloc = 0.f, msm = 0.f, jsm = 0.f;
    bool nonfinite = false;
    if (tid < nv) {
      const float ms = ms_s[tid], mc = ms_c[tid], js = x[tid], jc = mp[tid];
      const float qf = V(C_QF)[tid];
      float t1, e1, t2, e2;
      two_sum(ms, -qf, t1, e1);
      const float lo1 = __fadd_rn(e1, mc);
      const float maq = __fadd_rn(t1, lo1);
      two_sum(t1, js, t2, e2);
      const float tl = __fadd_rn(lo1, __fadd_rn(e2, jc));
      const float r = __fadd_rn(t2, tl);
      // thread tid reads and overwrites only entry tid of these slots
      V(C_R)[tid] = r;
      V(C_MAQ)[tid] = maq;
      if (rlo_slot >= 0) V(rlo_slot)[tid] = __fsub_rn(tl, __fsub_rn(r, t2));
      rloc = fabsf(r);
      msm = fabsf(ms);
      jsm = fabsf(js);
      nonfinite = !(rloc < CUDART_INF_F);
    }
    for (int j = nv + tid; j < geo.nvcap; j += kCtaThreads) {
      V(C_R)[j] = 0.f;
      V(C_MAQ)[j] = 0.f;
      if (rlo_slot >= 0) V(rlo_slot)[j] = 0.f;
    }
    const float rm = block_max(rloc);
    const float sc = fmaxf(fmaxf(1.f, qmax), fmaxf(block_max(msm), block_max(jsm)));
    *scale = sc;
    *bad = block_any(nonfinite) || !(sc < CUDART_INF_F);
    return rm;
  }

  // --------------------------------------------------------- line search
  // p in C_P (already -H^-1 r).  Same algorithm as the warp solver.
  __device__ __forceinline__ float line_search(float* dfmax, bool* crossed) {
    const float* vp = V(C_P);
    const float* Jm = Js();
    const float* Mm = Ms();
    const int JS = geo.JS, MS = geo.MS;
#pragma unroll
    for (int u = 0; u < MTC; ++u) s_r[u] = 0.f;
    if (32 * warp < m) {  // warps without a valid row skip J p
#pragma unroll 4
      for (int k = 0; k < nv; ++k) {
        const float pk = vp[k];
#pragma unroll
        for (int u = 0; u < MTC; ++u)
          if (kCtaThreads * u + 32 * warp < m)
            s_r[u] = __fmaf_rn(Jm[min(row(u), m - 1) * JS + k], pk, s_r[u]);
      }
    }
    float pMp = 0.f, c0 = 0.f;
    if (tid < nv) {
      float mp = 0.f;
      const float* Mr = Mm + tid * MS;
#pragma unroll 4
      for (int k = 0; k < nv; ++k) mp = __fmaf_rn(Mr[k], vp[k], mp);
      pMp = vp[tid] * mp;
      c0 = vp[tid] * V(C_MAQ)[tid];
    }
    block_sum2(pMp, c0);
    float bp[MTC];
#pragma unroll
    for (int u = 0; u < MTC; ++u)
      bp[u] = (row_valid(u) && s_r[u] != 0.f) ? __fdividef(-jar_r[u], s_r[u]) : CUDART_INF_F;
    float alpha = 1.f, lo = 0.f, hi = CUDART_INF_F;
#pragma unroll 1
    for (int it = 0; it < kLineSearchMax; ++it) {
      float sum = 0.f, cs = 0.f;
#pragma unroll
      for (int u = 0; u < MTC; ++u) {
        if (row_valid(u)) {
          const float uu = __fmaf_rn(alpha, s_r[u], jar_r[u]);
          const float ds = D_r[u] * s_r[u];
          if (uu < 0.f) {
            sum = __fmaf_rn(ds, uu, sum);
            cs = __fmaf_rn(ds, s_r[u], cs);
          }
        }
      }
      block_sum2(sum, cs);
      const float d = c0 + alpha * pMp + sum;
      if (d == 0.f) break;
      float an = alpha - __fdividef(d, pMp + cs), x0, x1;
      if (d < 0.f) {
        lo = alpha;
        x0 = alpha;
        x1 = an;
      } else {
        hi = alpha;
        x0 = an;
        x1 = alpha;
      }
      bool inside = false;
#pragma unroll
      for (int u = 0; u < MTC; ++u) inside = inside || (bp[u] > x0 && bp[u] < x1);
      const bool any_in = block_any(inside);
      if (!any_in && an > 0.f) {
        alpha = an;
        break;
      }
      if (!(an > lo && an < hi)) an = (hi == CUDART_INF_F) ? 2.f * alpha : 0.5f * (lo + hi);
      alpha = an;
      if (it == kLineSearchMax - 1) alpha = (lo > 0.f) ? lo : alpha;
    }
    float df = 0.f;
    bool cr = false;
#pragma unroll
    for (int u = 0; u < MTC; ++u) {
      if ((act_bits >> u) & 1u) df = fmaxf(df, fabsf(D_r[u] * alpha * s_r[u]));
      cr = cr || (bp[u] > 0.f && bp[u] < alpha);
    }
    *dfmax = block_max(df);
    *crossed = block_any(cr);
    return alpha;
  }

  // ------------------------------------------------------------- forward
  // Whether the correction z (shared slot, nvcap entries) would move a by at
  // most kStepTol max|a| and every active force D_i (J z)_i by at most
  // kForceTol fmax (fmax from the last compensated residual).  All threads.
  __device__ __forceinline__ bool small_correction(const float* z) {
    float zm = 0.f, am = 0.f;
    if (tid < nv) {
      zm = fabsf(z[tid]);
      am = fabsf(V(C_AH)[tid]);
    }
    const float zmax = block_max(zm);
    const float amax = block_max(am);
    if (!(zmax <= kStepTol * amax)) return false;
    float s[MTC], c[MTC];
    rows_dot(z, z, false, s, c);
    float df = 0.f;
#pragma unroll
    for (int u = 0; u < MTC; ++u)
      if ((act_bits >> u) & 1u) df = fmaxf(df, fabsf(D_r[u] * s[u]));
    return block_max(df) <= kForceTol * fmax;
  }

  // After a step a += alpha p that crossed no breakpoint: jar and the active
  // forces f (pair) advanced by alpha J p from the line search's products;
  // the active set and its row list are unchanged (as in the warp solver).
  __device__ __forceinline__ void advance_forces(float alpha) {
    float* F = Fs();
    float* Fl = Flo();
#pragma unroll
    for (int u = 0; u < MTC; ++u) {
      if (row_valid(u)) {
        const float ds = alpha * s_r[u];
        jar_r[u] = __fadd_rn(jar_r[u], ds);
        if ((act_bits >> u) & 1u) {
          float fh = F[row(u)], fl = Fl[row(u)];
          WarpSolver<1, 1>::add_to_pair(fh, fl, D_r[u] * ds);
          F[row(u)] = fh;
          Fl[row(u)] = fl;
        }
      }
    }
    __syncthreads();
  }

  __device__ __forceinline__ int forward(const Params& P, int* iters) {
    *iters = 0;
    if (!factor_M()) return CS_ST_CHOLFAIL;
    fmask_bits = 0;
    fmask_valid = true;
    float* ah = V(C_AH);
    float* al = V(C_AL);
    for (int j = tid; j < geo.nvcap; j += kCtaThreads) {
      ah[j] = V(C_QF)[j];
      al[j] = 0.f;
    }
    __syncthreads();
    chol_solve(C_AH);
    uint32_t prev_bits = 0;
    bool prev_small = false, precise = false;
    bool cg = false;  // conjugate settled-set steps (see the warp solver)
    float zr_prev = 1.f, smax_prev = 0.f;
    float* pp = V(C_PP);
#pragma unroll 1
    for (int k = 0;; ++k) {
      float scale;
      bool bad;
      const float rmax = residual(&scale, &bad, precise);
      if (bad) return CS_ST_NONFINITE;
      if (!precise && (k >= P.max_iter || rmax <= P.tol * scale)) {
        precise = true;
        --k;
        continue;
      }
      if (rmax <= P.tol * scale) return CS_ST_OK;
      const bool same = !block_any(act_bits != prev_bits);
      if (k >= P.max_iter) return CS_ST_MAXITER;
      cg = cg && same;
      if (need_refactor()) {
        if (!assemble_and_factor()) return CS_ST_CHOLFAIL;
        cg = false;
      }
      float* p = V(C_P);  // first z = H^-1 r, then the step
      for (int j = tid; j < geo.nvcap; j += kCtaThreads) p[j] = V(C_R)[j];
      __syncthreads();
      chol_solve(C_P);
      // Once the active set has settled (compensated phase, the same set as
      // at the previous point), the FP32 Newton correction z estimates the
      // remaining error of a: a is returned as it is when z would move it by
      // <= kStepTol |a| and every active force by <= kForceTol |f|, or when
      // the step just taken was that small (as in the warp solver)
      if (precise && k > 0 && same && (prev_small || small_correction(p))) return CS_ST_OK;
      float zr = 0.f, ptr = 0.f;
      if (tid < nv) zr = p[tid] * V(C_R)[tid];
      float d0 = 0.f;
      block_sum2(zr, d0);
      const float beta = (cg && zr_prev > 0.f) ? fmaxf(zr / zr_prev, 0.f) : 0.f;
      float am = 0.f, pm = 0.f, pz = 0.f;
      if (tid < nv) {
        pz = -p[tid];
        const float pv = __fmaf_rn(beta, pp[tid], pz);
        ptr = pv * V(C_R)[tid];
        am = fabsf(ah[tid]);
      }
      block_sum2(ptr, d0);
      const bool restart = !(ptr < 0.f) && beta != 0.f;
      if (tid < nv) {
        const float pv = restart ? pz : __fmaf_rn(beta, pp[tid], pz);
        p[tid] = pv;
        pm = fabsf(pv);
      }
      if (restart) ptr = -zr;
      const float amax = block_max(am);
      if (!(ptr < 0.f)) {
        const float pmax = block_max(pm);
        return (pmax <= kStepTol * amax) ? CS_ST_OK : CS_ST_NOPROGRESS;
      }
      float dfm;
      bool crossed;
      const float alpha = line_search(&dfm, &crossed);
      float sm = 0.f;
      if (tid < nv) {
        const float dp = alpha * p[tid];
        float hh = ah[tid], ll = al[tid];
        WarpSolver<1, 1>::add_to_pair(hh, ll, dp);
        ah[tid] = hh;
        al[tid] = ll;
        sm = fabsf(dp);
      }
      *iters = k + 1;
      const float smax = block_max(sm);
      // predicted-error stop of the refinement steps (see the warp solver)
      if (precise && same && !crossed) {
        const float q = smax / (cg ? smax_prev : amax);
        const float gq = (cg ? 1.f : kFirstRatioMargin) * q / (1.f - q);
        if (q < 0.5f && gq * smax <= kStepTol * amax && gq * dfm <= kForceTol * fmax) {
          advance_forces(alpha);
          return CS_ST_OK;
        }
      }
      smax_prev = smax;
      prev_small = precise && (smax <= kStepTol * amax) && (dfm <= kForceTol * fmax);
      prev_bits = act_bits;
      cg = precise && !crossed;
      zr_prev = zr;
      if (tid < nv) pp[tid] = p[tid];
      precise = precise || !crossed;
    }
  }

  // ------------------------------------------------------------- adjoint
  // w = H^-1 (rhs + rhs_lo) for the factored H and the active list: a first
  // solve, then refinement with compensated residuals rhs - M w - J^T lambda
  // (lambda = D_act . (J w), compensated); stops when the untaken correction
  // moves w by <= step_tol |w| and the active lambda by <= force_tol |lambda|,
  // or (kPredict) once the correction just applied leaves a predicted error
  // within them (geometric contraction, as in the warp solver; lambda is then
  // advanced by D_act (J dw)).
  // Slots: rh / rl the right-hand side's parts (rl < 0: none), oh / ol the
  // result pair; jh / jl and mh / mr scratch (J^T lambda and M w pairs, mr
  // also the correction).  Leaves lambda (pair) in Lam() / Lamlo().
  template <bool kPredict = false>
  __device__ __forceinline__ void solve_refined(int rh, int rl, int oh, int ol, int jh, int jl,
                                                int mh, int mr, float step_tol, float force_tol) {
    float prev = 0.f;  // max |last correction| (0: w itself is the last one)
    float* wh = V(oh);
    float* wl = V(ol);
    for (int j = tid; j < geo.nvcap; j += kCtaThreads) {
      wh[j] = V(rh)[j];
      wl[j] = 0.f;
    }
    __syncthreads();
    chol_solve(oh);
    float* Lm = Lam();
    const float* Jm = Js();
    const float* Mm = Ms();
    const int* idx = Idx();
    const int JS = geo.JS, MS = geo.MS;
#pragma unroll 1
    for (int it = 0; it <= kAdjointRefineMax; ++it) {
      float s[MTC], c[MTC];
      rows_dot(wh, wl, true, s, c);
      float lmax = 0.f;
#pragma unroll
      for (int u = 0; u < MTC; ++u) {
        if (kCtaThreads * u < m) {
          const bool on = (act_bits >> u) & 1u;
          const float uh = __fadd_rn(s[u], c[u]);
          const float ul = __fsub_rn(c[u], __fsub_rn(uh, s[u]));
          float lam = 0.f, lamlo = 0.f;
          if (on) WarpSolver<1, 1>::scale_pair(D_r[u], uh, ul, lam, lamlo);
          if (row_valid(u)) {
            Lm[row(u)] = lam;
            Lamlo()[row(u)] = lamlo;
          }
          lmax = fmaxf(lmax, fabsf(lam));
        }
      }
      lmax = block_max(lmax);
      if (it == kAdjointRefineMax) break;
      float* js_s = V(jh);
      float* js_c = V(jl);
      const float* Lml = Lamlo();
      split_dot(nv, nact, true,
                [&](int j, int q, float& a, float& h, float& l) {
                  const int i = idx[q];
                  a = Jm[i * JS + j];
                  h = Lm[i];
                  l = Lml[i];
                },
                js_s, js_c);
      float* ms_s = V(mh);
      float* ms_c = V(mr);
      split_dot(nv, nv, true,
                [&](int j, int k, float& a, float& h, float& l) {
                  a = Mm[j * MS + k];
                  h = wh[k];
                  l = wl[k];
                },
                ms_s, ms_c);
      float* rho = V(mr);
      float rv = 0.f;
      if (tid < nv) {
        float t1, e1, t2, e2;
        two_sum(V(rh)[tid], -ms_s[tid], t1, e1);
        two_sum(t1, -js_s[tid], t2, e2);
        float lo = __fadd_rn(e1, e2);
        if (rl >= 0) lo = __fadd_rn(lo, V(rl)[tid]);
        rv = __fadd_rn(t2, __fsub_rn(lo, __fadd_rn(ms_c[tid], js_c[tid])));
      }
      __syncthreads();
      for (int j = tid; j < geo.nvcap; j += kCtaThreads) rho[j] = (j < nv) ? rv : 0.f;
      __syncthreads();
      chol_solve(mr);
      // the correction's size, in w and in the active lambda = D (J dw)
      float dm = 0.f, wm = 0.f;
      if (tid < nv) {
        dm = fabsf(rho[tid]);
        wm = fabsf(wh[tid]);
      }
      const float dmax = block_max(dm);
      const float wmax = block_max(wm);
      const float q = dmax / (prev > 0.f ? prev : wmax);
      const float gq = (prev > 0.f ? 1.f : kFirstRatioMargin) * q / (1.f - q);
      const bool predict = kPredict && q < 0.5f && gq * dmax <= step_tol * wmax;
      bool done = false;
      if (dmax <= step_tol * wmax || predict) {
        float sd[MTC], cd[MTC];
        rows_dot(rho, rho, false, sd, cd);
        float dl = 0.f;
#pragma unroll
        for (int u = 0; u < MTC; ++u)
          if ((act_bits >> u) & 1u) dl = fmaxf(dl, fabsf(D_r[u] * sd[u]));
        dl = block_max(dl);
        if (dmax <= step_tol * wmax && dl <= force_tol * lmax) break;
        if (predict && gq * dl <= force_tol * lmax) {
          // apply dw and advance lambda by D_act (J dw) (own rows only)
#pragma unroll
          for (int u = 0; u < MTC; ++u)
            if ((act_bits >> u) & 1u) {
              float lh = Lm[row(u)], ll = Lamlo()[row(u)];
              WarpSolver<1, 1>::add_to_pair(lh, ll, D_r[u] * sd[u]);
              Lm[row(u)] = lh;
              Lamlo()[row(u)] = ll;
            }
          done = true;
        }
      }
      if (tid < nv) {
        float hh = wh[tid], ll = wl[tid];
        WarpSolver<1, 1>::add_to_pair(hh, ll, rho[tid]);
        wh[tid] = hh;
        wl[tid] = ll;
      }
      __syncthreads();
      if (done) break;
      prev = dmax;
    }
    __syncthreads();
  }

  // The IFT adjoint (Eq. 17): w = H^-1 g in C_WH / C_WL, lambda in Lam(),
  // refined to the adjoint's resolution (kAdjStepTol, kAdjForceTol, as in
  // the warp solver).
  __device__ __forceinline__ void adjoint() {
    solve_refined<true>(C_G, -1, C_WH, C_WL, C_X, C_MP, C_P, C_R, kAdjStepTol, kAdjForceTol);
  }

  // Active list and bits from a given row mask (rows in order).
  __device__ __forceinline__ void set_active(uint32_t bits) {
    int* idx = Idx();
    float* Rd = Red() + 5 * kCtaWarps;
    int base = 0;
#pragma unroll
    for (int u = 0; u < MTC; ++u) {
      if (kCtaThreads * u < m) {
        const bool on = row_valid(u) && ((bits >> u) & 1u);
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
        if (on) idx[before + __popc(bal & ((1u << lane) - 1u))] = row(u);
        base = total;
        __syncthreads();
      }
    }
    nact = base;
    act_bits = bits;
  }

  __device__ __forceinline__ void write_grads(const Params& P, const cs_inst& e) {
    const float* wh = V(C_WH);
    const float* ah = V(C_AH);
    const float* Lm = Lam();
    const float* F = Fs();
    for (int j = tid; j < nv; j += kCtaThreads) P.dqfrc[e.off_v + j] = wh[j];
    for (int i = tid; i < m; i += kCtaThreads) P.daref[e.off_r + i] = Lm[i];
    float* dJ = P.dJ + e.off_J;
#pragma unroll 1
    for (int q = tid; q < m * nv; q += kCtaThreads) {
      const int rr = q / nv, cc = q - rr * nv;
      dJ[q] = -__fmaf_rn(F[rr], wh[cc], Lm[rr] * ah[cc]);
    }
    if (P.dD) {
#pragma unroll
      for (int u = 0; u < MTC; ++u)
        if (row_valid(u)) {
          const int i = row(u);
          P.dD[e.off_r + i] = jar_r[u] < 0.f ? -__fdiv_rn(Lm[i] * jar_r[u], D_r[u]) : 0.f;
        }
    }
    if (P.dM) {
      float* dM = P.dM + e.off_M;
#pragma unroll 1
      for (int q = tid; q < nv * nv; q += kCtaThreads) {
        const int rr = q / nv, cc = q - rr * nv;
        dM[q] = -0.5f * __fmaf_rn(wh[rr], ah[cc], ah[rr] * wh[cc]);
      }
    }
  }

  __device__ __forceinline__ void zero_grads(const Params& P, const cs_inst& e) {
    for (int j = tid; j < nv; j += kCtaThreads) P.dqfrc[e.off_v + j] = 0.f;
    for (int i = tid; i < m; i += kCtaThreads) P.daref[e.off_r + i] = 0.f;
    for (int q = tid; q < m * nv; q += kCtaThreads) P.dJ[e.off_J + q] = 0.f;
    if (P.dD)
      for (int i = tid; i < m; i += kCtaThreads) P.dD[e.off_r + i] = 0.f;
    if (P.dM)
      for (int q = tid; q < nv * nv; q += kCtaThreads) P.dM[e.off_M + q] = 0.f;
  }

  __device__ __forceinline__ void load_factor(const float* Lp) {
    float* L = Ls();
    const int nc = geo.nvcap, MS = geo.MS;
    for (int q = tid; q < nc * nc; q += kCtaThreads) {
      const int rr = q / nc, cc = q - rr * nc;
      if (cc <= rr) {
        float v;
        if (rr < nv) v = __ldg(Lp + rr * (rr + 1) / 2 + cc);
        else v = (rr == cc) ? 1.f : 0.f;
        L[rr * MS + cc] = v;
      }
    }
    __syncthreads();
    for (int j = tid; j < nc; j += kCtaThreads) V(C_DINV)[j] = 1.0f / L[j * MS + j];
    __syncthreads();
  }

  __device__ __forceinline__ void store_factor(float* Lp) {
    const float* L = Ls();
    for (int q = tid; q < nv * nv; q += kCtaThreads) {
      const int rr = q / nv, cc = q - rr * nv;
      if (cc <= rr) Lp[rr * (rr + 1) / 2 + cc] = L[rr * geo.MS + cc];
    }
  }

  // ------------------------------------------------------------- driver
  template <int MODE>
  __device__ __forceinline__ void run(const Params& P, int b) {
    const cs_inst e = P.inst[b];
    const bool ok_load = load(P, e);  // every thread takes the same branch
    if (!ok_load) {
      if (tid == 0) {
        P.status[b] = CS_ST_BADSHAPE;
        P.iters[b] = 0;
      }
      __syncthreads();
      return;
    }
    float* gv = V(C_G);
    for (int j = tid; j < geo.nvcap; j += kCtaThreads)
      gv[j] = (MODE != MODE_FWD && j < nv) ? __ldg(P.g + e.off_v + j) : 0.f;
    if (MODE == MODE_FWD || MODE == MODE_FUSED) {
      int iters = 0;
      const int st = forward(P, &iters);
      for (int j = tid; j < nv; j += kCtaThreads) P.a[e.off_v + j] = V(C_AH)[j];
      if (tid == 0) {
        P.status[b] = st;
        P.iters[b] = iters;
      }
      if (st == CS_ST_CHOLFAIL || st == CS_ST_NONFINITE) {
        if (MODE == MODE_FUSED) zero_grads(P, e);
        __syncthreads();
        return;
      }
      if (MODE == MODE_FWD) {
        for (int j = tid; j < nv; j += kCtaThreads) P.a_lo[e.off_v + j] = V(C_AL)[j];
#pragma unroll
        for (int u = 0; u < MTC; ++u)
          if (row_valid(u)) P.act[e.off_r + row(u)] = (act_bits >> u) & 1u;
        if (P.keep_factor && P.Lst) {
          if (need_refactor())
            if (!assemble_and_factor()) {
              if (tid == 0) P.status[b] = CS_ST_CHOLFAIL;
              __syncthreads();
              return;
            }
          store_factor(P.Lst + e.off_M);
        }
        __syncthreads();
        return;
      }
      if (need_refactor())
        if (!assemble_and_factor()) {
          if (tid == 0) P.status[b] = CS_ST_CHOLFAIL;
          zero_grads(P, e);
          __syncthreads();
          return;
        }
      adjoint();
      write_grads(P, e);
    } else {  // MODE_ADJ
      const int st0 = P.status[b];
      if (st0 == CS_ST_CHOLFAIL || st0 == CS_ST_NONFINITE || st0 == CS_ST_BADSHAPE) {
        zero_grads(P, e);
        __syncthreads();
        return;
      }
      for (int j = tid; j < geo.nvcap; j += kCtaThreads) {
        V(C_AH)[j] = (j < nv) ? __ldg(P.a + e.off_v + j) : 0.f;
        V(C_AL)[j] = (j < nv) ? __ldg(P.a_lo + e.off_v + j) : 0.f;
      }
      __syncthreads();
      float scale;
      bool bad;
      residual(&scale, &bad, true);
      uint32_t kept = 0;
#pragma unroll
      for (int u = 0; u < MTC; ++u)
        if (row_valid(u) && P.act[e.off_r + row(u)]) kept |= 1u << u;
      if (P.keep_factor && P.Lst) {
        load_factor(P.Lst + e.off_M);
        fmask_bits = kept;
        fmask_valid = true;
      } else {
        fmask_valid = false;
      }
      if (need_refactor())
        if (!assemble_and_factor()) {
          if (tid == 0) P.status[b] = CS_ST_CHOLFAIL;
          zero_grads(P, e);
          __syncthreads();
          return;
        }
      adjoint();
      write_grads(P, e);
    }
    __syncthreads();
  }
};

// One CTA per instance; CTAs claim instances dynamically or round-robin.
template <int MTC, int MODE>
__global__ void __launch_bounds__(kCtaThreads, MTC == 1 ? 2 : 1) cta_solve_kernel(const __grid_constant__ Params P,
                                                                 const CtaGeo geo) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ int claim;
  CtaSolver<MTC> S;
  S.sm = reinterpret_cast<float*>(smem_raw);
  S.geo = geo;
  S.tid = threadIdx.x;
  S.lane = threadIdx.x & 31;
  S.warp = threadIdx.x >> 5;
  int idx = blockIdx.x;
#pragma unroll 1
  for (int guard = 0; guard <= P.n_work; ++guard) {
    if (P.counter) {
      if (S.tid == 0) claim = atomicAdd(P.counter, 1);
      __syncthreads();
      idx = claim;
      __syncthreads();
    }
    if (idx >= P.n_work) break;
    const int b = P.order ? P.order[idx] : idx;
    if (b >= 0 && b < P.n) S.template run<MODE>(P, b);
    __syncthreads();
    if (!P.counter) idx += gridDim.x;
  }
}

}  // namespace csk
