// cs_warp.cuh -- one-warp-per-instance contact solver (device code).
//
// A warp owns one instance at a time.  Its M, J, D and the Newton matrix /
// Cholesky factor sit in the warp's slice of shared memory; every per-row
// quantity (jar, J p, D, aref) is spread over the lanes as "row i = lane + 32
// t, t < MT"; every nv-vector is spread as "element j on lane j" and broadcast
// through a small shared buffer.
//
// Arithmetic (Section III of the paper):
//  * residual r = M a - qfrc + J^T f, f = D . min(J a - aref, 0) (Eqs. 6, 8).
//    a is carried as an unevaluated float pair (hi + lo) and r, jar are
//    accumulated with error-free transformations (TwoSum / TwoProd), so the
//    contact forces f keep their accuracy when a stiff row has |jar| << |J a|;
//  * H = M + sum_{i active} D_i J_i^T J_i (Eq. 9), a left-looking Cholesky in
//    shared memory (lane j computes row j), blocked triangular solves with
//    shuffles;
//  * p = -H^-1 r and an exact line search on the piecewise-linear derivative
//    of phi(alpha) = L(a + alpha p) (Eq. 10): safeguarded Newton on phi' that
//    stops when no breakpoint separates the trial point from its Newton
//    point, which makes the returned alpha the exact root;
//  * the IFT adjoint H w = g (Eq. 17), refined with compensated residuals so
//    that D_act . (J w) keeps its accuracy for stiff rows.
//
// Code size matters as much as instruction count here: a fully unrolled
// solver overflows the instruction cache (measured: "no instruction" was the
// dominant stall), so loops over nv and over rows stay rolled and only the
// short per-lane row loops (t < MT) are unrolled.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include <type_traits>

#include "contact_solve.h"

namespace csk {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kLineSearchMax = 64;  // exact line-search trial points
constexpr int kAdjointRefineMax = 8;
// Step test: a step that moves a by <= kStepTol |a| and the active forces by
// <= kForceTol |f| with an unchanged active set means the fp32 Newton /
// refinement iteration has reached its attainable accuracy.
constexpr float kStepTol = 1.0e-7f;
constexpr float kForceTol = 1.0e-6f;
// Margin on the predicted-error stop of the refinement steps when the
// contraction ratio comes from the first correction alone (measured against
// the solution itself, which tracks the true ratio only loosely at large
// cond(H)); a ratio of two consecutive corrections is used as it is.
constexpr float kFirstRatioMargin = 16.0f;
// The adjoint's refinement stops once the next correction would move w by
// <= kAdjStepTol |w| and the active lambda = D_act . J w by <= kAdjForceTol
// |lambda|: that bounds the remaining error of every gradient well below the
// 1e-3 relative tolerance they are held to (measured worst against the FP64
// oracle: 3.4e-5 over the quadruped, Franka and nv = 96 batches) without the
// passes that only chase FP32 resolution; 1e-6 / 1e-5 gave 7e-6 for 5 % more
// time per fused solve.  (The forward keeps the tighter pair above: a decides
// the active set, whose rows are compared one by one.)
constexpr float kAdjStepTol = 1.0e-5f;
constexpr float kAdjForceTol = 3.0e-5f;

// ---------------------------------------------------------------- EFT helpers
// __f*_rn intrinsics are never contracted into FMAs, which keeps the
// error-free transformations exact.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float z = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}
// (s, c) += x * (yh + yl)
__device__ __forceinline__ void dot2(float& s, float& c, float x, float yh, float yl) {
  float p = __fmul_rn(x, yh);
  float pe = __fmaf_rn(x, yh, -p);
  float t, te;
  two_sum(s, p, t, te);
  s = t;
  c = __fadd_rn(c, __fadd_rn(te, __fmaf_rn(x, yl, pe)));
}
// (s, c) += x * y
__device__ __forceinline__ void dot2s(float& s, float& c, float x, float y) {
  float p = __fmul_rn(x, y);
  float pe = __fmaf_rn(x, y, -p);
  float t, te;
  two_sum(s, p, t, te);
  s = t;
  c = __fadd_rn(c, __fadd_rn(te, pe));
}
// (s, c) += (s2, c2) for unnormalised float pairs.
__device__ __forceinline__ void add_pair(float& s, float& c, float s2, float c2) {
  float t, e;
  two_sum(s, s2, t, e);
  s = t;
  c = __fadd_rn(__fadd_rn(c, c2), e);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
// One warp-wide reduction instruction (redux.sync .f32, sm_100 family):
// exact, and like fmaxf it ignores NaN inputs; five dependent shuffle / max
// rounds before.
__device__ __forceinline__ float warp_max(float v) {
  float r;
  asm volatile("redux.sync.max.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
  return r;
}

// ------------------------------------------------------------------ geometry
// kShare: lambda and its low part reuse the words of D and of f's low part,
// which are dead while the adjoint runs (D in shared memory is read only by
// the assembly, which precedes the adjoint; f's low part only by the
// compensated residual; f itself stays, the gradient writer reads it).  The
// warp kernel's own modes use it; callers that keep f, its low part and
// lambda live together (the unrolled reverse sweep, the round cone) do not.
// Number of RA x 4 blocks (RA rows, an aligned quad of columns) that cover
// the lower triangle of an NV x NV matrix.
__host__ __device__ constexpr int quad_blocks(int NV, int RA) {
  int n = 0;
  for (int r0 = 0; r0 < NV; r0 += RA) n += ((r0 + RA < NV ? r0 + RA : NV) + 3) / 4;
  return n;
}
// Rows per assembly block: the smallest of 1, 2, 4, 8 whose blocks fit 32 lanes.
__host__ __device__ constexpr int quad_rows(int NV) {
  return quad_blocks(NV, 1) <= 32 ? 1 : quad_blocks(NV, 2) <= 32 ? 2
       : quad_blocks(NV, 4) <= 32 ? 4 : 8;
}

template <int NV, int MT, bool kShare = false>
struct Geo {
  static_assert(NV >= 1 && NV <= 32, "one lane per row of H");
  static constexpr int MCAP = 32 * MT;               // rows per instance
  static constexpr int BS = (NV + 6) / 7;            // block edge of the round-cone assembly
  static constexpr int NB = (NV + BS - 1) / BS;      // blocks per edge (<= 7)
  static constexpr int NBLK = NB * (NB + 1) / 2;     // lower blocks (<= 28)
  // J rows hold NP pairs of columns; the row stride is twice an odd number,
  // so that the 8-byte loads of sixteen consecutive lanes' rows (one
  // shared-memory wavefront) fall in sixteen distinct bank pairs, and columns
  // walked by consecutive lanes are consecutive words.
  static constexpr int NP = (NV + 1) / 2;            // column pairs
  static constexpr int JS = 2 * (NP | 1);            // J row stride
  static constexpr int RA = quad_rows(NV);           // rows per assembly block
  static constexpr int NABLK = quad_blocks(NV, RA);  // assembly blocks (<= 32)
  static_assert(NABLK <= 32, "one lane per assembly block");
  static constexpr int MS = NV | 1;                  // M/L row stride (odd)
  // shared-memory slice of one warp, in 4-byte words
  static constexpr int oM = 0;                       // M   NV x MS
  static constexpr int oL = oM + NV * MS;            // H/L NV x MS
  static constexpr int oJ = (oL + NV * MS + 3) & ~3; // J   MCAP x JS (16-byte aligned)
  static constexpr int oD = oJ + MCAP * JS;          // D   MCAP
  static constexpr int oF = oD + MCAP;               // f   MCAP
  static constexpr int oLam = kShare ? oD : oF + MCAP;              // lambda = D_act J w
  static constexpr int oFlo = kShare ? oF + MCAP : oLam + MCAP;     // low parts of f ...
  static constexpr int oLamlo = kShare ? oFlo : oFlo + MCAP;        // ... and of lambda
  static constexpr int oIdx = oLamlo + MCAP;         // active rows (bytes if kShare, else int)
  static constexpr int oVec = oIdx + (kShare ? MCAP / 4 : MCAP);  // broadcast vectors
  static constexpr int kVec = kShare ? 4 : 7;        // broadcast slots (below)
  // kShare (the warp kernel's modes): the assembled Newton matrix of the
  // factored active set is kept, so that the next one is formed from the
  // rows that entered or left the set (below), with a list of those rows
  static constexpr int kChg = 32;                    // changed rows per update
  static constexpr int oH = oVec + kVec * 32;        // H   NV x MS (kShare)
  static constexpr int oChg = oH + (kShare ? NV * MS : 0);
  static constexpr int kWords = oChg + (kShare ? kChg : 0);
  static constexpr int kBytes = ((kWords * 4) + 127) & ~127;
};

enum VecSlot { V_AH = 0, V_AL = 1, V_P = 2, V_WH = 3, V_WL = 4, V_X = 5, V_DINV = 6 };

// Kernel parameters (one struct, passed by value).
struct Params {
  int32_t n;                // instances in the batch (bound for indices)
  int32_t n_work;           // claimable entries (order length, or n)
  const cs_inst* inst;
  const float *M, *J, *qfrc, *aref, *D, *g;
  int64_t total_M, total_J, total_v, total_r;
  float* a;                 // out (fwd, fused) / in (adjoint)
  float *dqfrc, *daref, *dJ;
  float *dM, *dD;           // optional parameter gradients for M and D, or null
  float* a_lo;              // state
  uint8_t* act;             // state
  float* Lst;               // state factor (packed lower rows) or null
  int32_t *status, *iters;
  float tol;
  int32_t max_iter;
  int32_t keep_factor;
  int32_t* counter;         // dynamic claim counter (fused) or null
  const int32_t* order;     // claim order or null
};

enum Mode { MODE_FWD = 0, MODE_ADJ = 1, MODE_FUSED = 2, MODE_FUSED_NCG = 3 };

template <int NV, int MT, bool kShare = false>
struct WarpSolver {
  using G = Geo<NV, MT, kShare>;
  float* sm;   // warp slice
  int lane;

  // problem sizes of the current instance
  int nv, m;
  // row registers: row i = lane + 32 t
  float aref_r[MT], D_r[MT], jar_r[MT], s_r[MT];
  uint32_t act_bits;    // bit t: row lane+32t active at the current point
  uint32_t fmask_bits;  // active set the factor in Ls() belongs to
  bool fmask_valid;
  uint32_t hmask_bits;  // active set the matrix in Hs() belongs to (kShare)
  bool hmask_valid;
  int nact;
  // element registers (lane j < NV)
  float ah, al;          // a = ah + al
  float qf, gj;          // qfrc_j, g_j
  float r, maq;          // r_j, (M a - qfrc)_j
  float rlo;             // low part of the compensated r (r + rlo)
  float fmax;            // max |f| at the current point
  float qmax;            // max |qfrc|

  __device__ __forceinline__ float* Ms() { return sm + G::oM; }
  __device__ __forceinline__ float* Ls() { return sm + G::oL; }
  __device__ __forceinline__ float* Hs() { return sm + G::oH; }
  __device__ __forceinline__ int* Chg() { return reinterpret_cast<int*>(sm + G::oChg); }
  __device__ __forceinline__ float* Js() { return sm + G::oJ; }
  __device__ __forceinline__ float* Ds() { return sm + G::oD; }
  __device__ __forceinline__ float* Fs() { return sm + G::oF; }
  __device__ __forceinline__ float* Lam() { return sm + G::oLam; }
  __device__ __forceinline__ float* Flo() { return sm + G::oFlo; }
  __device__ __forceinline__ float* Lamlo() { return sm + G::oLamlo; }
  // Active-row list: row numbers < MCAP <= 256 fit a byte in the warp
  // kernel's layout; the round cone and the unrolled sweep keep ints.
  using idx_t = typename std::conditional<kShare, uint8_t, int>::type;
  __device__ __forceinline__ idx_t* Idx() { return reinterpret_cast<idx_t*>(sm + G::oIdx); }
  // Broadcast slot of vector s.  kShare: w's pair takes the slots of p and of
  // a's low part, and the gradient writer's copy of a the slot of a's high
  // part (it holds the same value): in the warp kernel's modes the adjoint
  // runs after the last line search and evaluates no residual.
  __host__ __device__ static constexpr int slot(int s) {
    return !kShare ? s
                   : (s == V_WH ? V_P : s == V_WL ? V_AL : s == V_X ? V_AH : s == V_DINV ? 3 : s);
  }
  __device__ __forceinline__ float* Vec(int s) { return sm + G::oVec + 32 * slot(s); }

  __device__ __forceinline__ bool row_valid(int t) const { return lane + 32 * t < m; }

  // Broadcast the lane-distributed vector v into slot s (lanes >= NV write 0).
  __device__ __forceinline__ void put_vec(int s, float v) {
    Vec(s)[lane] = (lane < NV) ? v : 0.f;
    __syncwarp();
  }

  // ------------------------------------------------------------- loading
  // Whether an instance record fits this kernel and its blocks lie inside
  // the batch arrays.
  __device__ __forceinline__ static bool in_bounds(const Params& P, const cs_inst& e) {
    const int nv_ = e.nv, m_ = e.m;
    if (nv_ < 1 || nv_ > NV || m_ < 0 || m_ > G::MCAP) return false;
    if (e.off_M < 0 || e.off_J < 0 || e.off_v < 0 || e.off_r < 0) return false;
    if (e.off_M + (int64_t)nv_ * nv_ > P.total_M) return false;
    if (e.off_J + (int64_t)m_ * nv_ > P.total_J) return false;
    if (e.off_v + nv_ > P.total_v || e.off_r + m_ > P.total_r) return false;
    return true;
  }

  // Bulk prefetch of [p, p + bytes) into L2, shrunk to whole 16-byte units
  // (the start rounded up, the end down), so that it never leaves the range.
  __device__ __forceinline__ static void l2_prefetch(const float* p, int64_t bytes) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    const uintptr_t lo = (a + 15) & ~uintptr_t(15);
    const uintptr_t hi = (a + (uintptr_t)bytes) & ~uintptr_t(15);
    if (hi > lo)
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo),
                   "r"((unsigned)(hi - lo))
                   : "memory");
  }

  // Warm L2 with the inputs of an instance that will be staged soon (one
  // lane, no registers held across the solve; the record is checked exactly
  // as load() checks it before any address is formed).
  __device__ __forceinline__ void prefetch(const Params& P, const cs_inst& e) {
    if (lane != 0 || !in_bounds(P, e)) return;
    l2_prefetch(P.J + e.off_J, 4LL * e.m * e.nv);
    l2_prefetch(P.M + e.off_M, 4LL * e.nv * e.nv);
    l2_prefetch(P.aref + e.off_r, 4LL * e.m);
    l2_prefetch(P.D + e.off_r, 4LL * e.m);
    l2_prefetch(P.qfrc + e.off_v, 4LL * e.nv);
    if (P.g) l2_prefetch(P.g + e.off_v, 4LL * e.nv);
  }

  // 4-byte asynchronous global -> shared copy: nothing is held in registers,
  // so a lane issues its whole share of an instance back to back and the
  // warp waits for the memory system once.
  __device__ __forceinline__ static void cp_async4(float* dst, const float* src) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
  }

  // Stage one instance into shared memory.  Instances with nv < NV are padded
  // with identity rows of M and zero columns of J (the padded unknowns stay
  // exactly zero and do not touch the real ones).  Measured: asynchronous
  // copies pay off where J is large (nv = 18, m up to 128: staging 15 % -> 6 %
  // of a warp's time, 2.16 -> 2.09 ms per quadruped step); at nv = 9, m = 64
  // the fewer instructions of 16-byte loads through registers win (0.233 vs
  // 0.242 ms per franka step).
  __device__ __forceinline__ bool load(const Params& P, const cs_inst& e) {
    nv = e.nv;
    m = e.m;
    hmask_valid = false;
    if (!in_bounds(P, e)) return false;
    if constexpr (NV >= 16 || MT >= 3) {
      load_async(P, e);
    } else {
      load_sync(P, e);
    }
    return true;
  }

  __device__ __forceinline__ void load_async(const Params& P, const cs_inst& e) {
    const float* M = P.M + e.off_M;
    const float* J = P.J + e.off_J;
    float* Ms_ = Ms();
    float* Js_ = Js();
    // J (row stride JS) and the real block of M (row stride MS), copied
    // asynchronously; the padding is written by plain stores to disjoint words
    const int mnv = m * nv;
    if (nv == NV) {
#pragma unroll 4
      for (int q = lane; q < mnv; q += 32) {
        const int rr = q / NV, cc = q - rr * NV;
        cp_async4(Js_ + rr * G::JS + cc, J + q);
      }
#pragma unroll 4
      for (int q = lane; q < NV * NV; q += 32) {
        const int rr = q / NV, cc = q - rr * NV;
        cp_async4(Ms_ + rr * G::MS + cc, M + q);
      }
    } else {
#pragma unroll 1
      for (int q = lane; q < mnv; q += 32) {
        const int rr = q / nv, cc = q - rr * nv;
        cp_async4(Js_ + rr * G::JS + cc, J + q);
      }
#pragma unroll 1
      for (int q = lane; q < NV * NV; q += 32) {
        const int rr = q / NV, cc = q - rr * NV;
        if (rr < nv && cc < nv)
          cp_async4(Ms_ + rr * G::MS + cc, M + rr * nv + cc);
        else
          Ms_[rr * G::MS + cc] = (rr == cc) ? 1.f : 0.f;
      }
    }
    // per-row and per-element data, loaded while the copies are in flight
    const int mpad = min(G::MCAP, (m + 31) & ~31);
#pragma unroll
    for (int t = 0; t < MT; ++t) {
      const int i = lane + 32 * t;
      const bool v = i < m;
      aref_r[t] = v ? __ldg(P.aref + e.off_r + i) : 0.f;
      D_r[t] = v ? __ldg(P.D + e.off_r + i) : 0.f;
    }
    qf = (lane < nv) ? __ldg(P.qfrc + e.off_v + lane) : 0.f;
    // zero padded columns of real rows, and whole rows up to the next
    // multiple of 32 (read by the row loops but never active)
    const int padc = G::JS - nv;
#pragma unroll 1
    for (int q = lane; q < m * padc; q += 32) {
      int rr = q / padc, cc = nv + (q - rr * padc);
      Js_[rr * G::JS + cc] = 0.f;
    }
#pragma unroll 1
    for (int q = m * G::JS + lane; q < mpad * G::JS; q += 32) Js_[q] = 0.f;
#pragma unroll
    for (int t = 0; t < MT; ++t) {
      const int i = lane + 32 * t;
      if (i < mpad) Ds()[i] = D_r[t];
    }
    qmax = warp_max(fabsf(qf));
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncwarp();
  }

  __device__ __forceinline__ void load_sync(const Params& P, const cs_inst& e) {
    const float* M = P.M + e.off_M;
    const float* J = P.J + e.off_J;
    float* Ms_ = Ms();
    float* Js_ = Js();
#pragma unroll 1
    for (int q = lane; q < NV * NV; q += 32) {
      int rr = q / NV, cc = q - rr * NV;
      float v = (rr < nv && cc < nv) ? __ldg(M + rr * nv + cc) : (rr == cc ? 1.f : 0.f);
      Ms_[rr * G::MS + cc] = v;
    }
    const int mnv = m * nv;
    if (nv == NV && (reinterpret_cast<uintptr_t>(J) & 15) == 0) {
      const float4* J4 = reinterpret_cast<const float4*>(J);
#pragma unroll 1
      for (int q = lane; q < (mnv >> 2); q += 32) {
        float4 v = __ldg(J4 + q);
        int b = 4 * q;
        int rr = b / NV, cc = b - rr * NV;
        float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          Js_[rr * G::JS + cc] = vv[u];
          if (++cc == NV) { cc = 0; ++rr; }
        }
      }
#pragma unroll 1
      for (int q = (mnv & ~3) + lane; q < mnv; q += 32) {
        int rr = q / NV, cc = q - rr * NV;
        Js_[rr * G::JS + cc] = __ldg(J + q);
      }
    } else {
#pragma unroll 1
      for (int q = lane; q < mnv; q += 32) {
        int rr = q / nv, cc = q - rr * nv;
        Js_[rr * G::JS + cc] = __ldg(J + q);
      }
    }
    // zero padded columns of real rows, and whole rows up to the next
    // multiple of 32 (read by the row loops but never active)
    const int mpad = min(G::MCAP, (m + 31) & ~31);
    const int padc = G::JS - nv;
#pragma unroll 1
    for (int q = lane; q < m * padc; q += 32) {
      int rr = q / padc, cc = nv + (q - rr * padc);
      Js_[rr * G::JS + cc] = 0.f;
    }
#pragma unroll 1
    for (int q = m * G::JS + lane; q < mpad * G::JS; q += 32) Js_[q] = 0.f;
#pragma unroll
    for (int t = 0; t < MT; ++t) {
      int i = lane + 32 * t;
      bool v = i < m;
      aref_r[t] = v ? __ldg(P.aref + e.off_r + i) : 0.f;
      D_r[t] = v ? __ldg(P.D + e.off_r + i) : 0.f;
      if (i < mpad) Ds()[i] = D_r[t];
    }
    qf = (lane < nv) ? __ldg(P.qfrc + e.off_v + lane) : 0.f;
    qmax = warp_max(fabsf(qf));
    __syncwarp();
  }


  // ------------------------------------------------------------- Cholesky
  // Cholesky of the lower rows in Ls(), in place, with the matrix in
  // registers: lane j loads row j of H, and for every column k (right-
  // looking, unrolled) the pivot H_kk is broadcast from lane k, lane j forms
  // L_jk = H_jk / L_kk, and the trailing entries of its row are updated,
  // H_jc -= L_jk L_ck for c > k, with L_ck shuffled from lane c.  Every
  // entry sees the same fused multiply-adds in the same order as the
  // left-looking recurrence L_jc = (H_jc - sum_{i<c} L_ji L_ci) / L_cc, so the
  // factor does not depend on the loop order.  Entries above the diagonal
  // are carried along (loaded, updated and stored back) but never read by
  // anything else, which saves a predicate per entry.  The reciprocal
  // pivots go to the V_DINV slot.  Returns false on a non-positive or
  // non-finite pivot: such a pivot makes its L_kk NaN (rsqrt of a negative
  // number or of zero, times the pivot), so one test of the diagonal at the
  // end finds it.  The fp32 factor only preconditions a compensated
  // iteration, so the reciprocal square root is the MUFU one.
  //
  // The matrix is read from src (rows of stride MS: Ls() itself, M, or the
  // kept Newton matrix) and the factor written to Ls().
  //
  // Not inlined: the unrolled body is NV (NV - 1) / 2 shuffle / fma pairs,
  // and a copy per call site would crowd the instruction cache.
  __device__ __noinline__ bool factor(const float* src = nullptr) {
    float* Lj = Ls() + min(lane, NV - 1) * G::MS;
    const float* Sj = (src ? src : Ls()) + min(lane, NV - 1) * G::MS;
    float h[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) h[c] = Sj[c];
    float diag = 1.f;
    // next pivot, H_kk after every update: lane k forms its own
    // H_kk - L_k,k-1^2 without waiting for the shuffle that carries L_k,k-1
    // to the other lanes (the same fma, so the same value), which keeps one
    // shuffle and the MUFU off each column's critical path
    float piv = h[0];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const float d = __shfl_sync(kFull, piv, k);
      const float rs = rsqrtf(d);
      const float lkk = d * rs;
      const float l = (lane == k) ? lkk : h[k] * rs;
      h[k] = l;
      diag = (lane == k) ? lkk : diag;
      if (k + 1 < NV) piv = __fmaf_rn(-l, l, h[k + 1]);
#pragma unroll
      for (int c = k + 1; c < NV; ++c) h[c] = __fmaf_rn(-l, __shfl_sync(kFull, l, c), h[c]);
    }
    __syncwarp();
    if (lane < NV) {
#pragma unroll
      for (int c = 0; c < NV; ++c) Lj[c] = h[c];
      // the reciprocal pivot is derived from the stored diagonal, exactly as
      // load_factor() does, so a kept factor solves bit-identically
      Vec(V_DINV)[lane] = 1.0f / diag;
    }
    __syncwarp();
    return !__any_sync(kFull, lane < NV && !(diag > 0.f && diag < CUDART_INF_F));
  }

  // z = (L L^T)^-1 x, vectors spread one element per lane.
  //
  // Blocked substitution: per block of kSB unknowns, the partially reduced
  // right-hand sides are gathered from their lanes with independent
  // shuffles, every lane solves the kSB x kSB diagonal block itself (L and
  // the reciprocal pivots are shared-memory broadcasts), and each lane below
  // (forward) or above (backward) the block subtracts the block's part.
  // Every unknown sees the same fused multiply-adds in the same order as in
  // column-at-a-time substitution, so the result is identical bit for bit;
  // the dependency chain has one shuffle per block instead of per column.
  static constexpr int kSB = (NV % 4 == 0) ? 4 : (NV % 3 == 0) ? 3 : (NV % 2 == 0) ? 2 : 1;
  // Block rounds unrolled in full only for small NV: at NV = 9 that took the
  // Franka step from 0.176 to 0.171 ms; at NV = 18 the unrolled copies (one
  // per call site) made the quadruped step 12 % slower.
  static constexpr int kSubUnroll = (NV <= 9) ? NV / kSB : 1;
  __device__ __forceinline__ float chol_solve(float x) { return chol_backward(chol_forward(x)); }

  // L y = x (forward substitution, blocked as above).
  __device__ __forceinline__ float chol_forward(float x) {
    const float* L = Ls();
    const float* dinv = Vec(V_DINV);
    const float* Lrow = L + min(lane, NV - 1) * G::MS;
#pragma unroll (kSubUnroll)
    for (int kb = 0; kb < NV; kb += kSB) {
      float y[kSB];
#pragma unroll
      for (int u = 0; u < kSB; ++u) y[u] = __shfl_sync(kFull, x, kb + u);
#pragma unroll
      for (int u = 0; u < kSB; ++u) {
        const float* Lu = L + (kb + u) * G::MS + kb;
#pragma unroll
        for (int w = 0; w < u; ++w) y[u] = __fmaf_rn(-Lu[w], y[w], y[u]);
        y[u] *= dinv[kb + u];
      }
      if (lane >= kb + kSB && lane < NV) {
#pragma unroll
        for (int u = 0; u < kSB; ++u) x = __fmaf_rn(-Lrow[kb + u], y[u], x);
      }
#pragma unroll
      for (int u = 0; u < kSB; ++u)
        if (lane == kb + u) x = y[u];
    }
    return x;
  }

  // L^T z = y (backward substitution, blocked as above).
  __device__ __forceinline__ float chol_backward(float x) {
    const float* L = Ls();
    const float* dinv = Vec(V_DINV);
#pragma unroll (kSubUnroll)
    for (int kt = NV - kSB; kt >= 0; kt -= kSB) {
      float z[kSB];
#pragma unroll
      for (int u = 0; u < kSB; ++u) z[u] = __shfl_sync(kFull, x, kt + u);
#pragma unroll
      for (int u = kSB - 1; u >= 0; --u) {
#pragma unroll
        for (int w = kSB - 1; w > u; --w)
          z[u] = __fmaf_rn(-L[(kt + w) * G::MS + kt + u], z[w], z[u]);
        z[u] *= dinv[kt + u];
      }
      if (lane < kt) {
#pragma unroll
        for (int w = kSB - 1; w >= 0; --w) x = __fmaf_rn(-L[(kt + w) * G::MS + lane], z[w], x);
      }
#pragma unroll
      for (int u = 0; u < kSB; ++u)
        if (lane == kt + u) x = z[u];
    }
    return (lane < NV) ? x : 0.f;
  }

  // Cholesky of M (the factor for the empty active set).
  __device__ __forceinline__ bool factor_M() {
    hmask_valid = false;
    return factor(Ms());
  }

  // H = M + sum_{active} D_i J_i^T J_i (Eq. 9), then its Cholesky factor in
  // Ls().  Lane l < NABLK owns one RA x 4 block of the lower triangle (RA
  // rows from RA*g, an aligned quad of columns) and reads a row's quad with
  // one 16-byte load; every entry sums its terms in row-list order.
  //
  // kShare: H is kept in Hs() with the active set it belongs to, and the next
  // one is formed from the rows that changed side, H += D_i J_i^T J_i for a
  // row that entered and -= for one that left, when there are at most kChg
  // of them and at most a quarter of the active count (else H is rebuilt
  // from M).  A Newton step changes a few rows of the set (a median of four
  // on the benchmark batch), so this replaces most of the assembly.  The
  // rounding of such an update is that of adding or removing one row's
  // terms, the same order as the rounding of a full assembly of the set, so
  // the factor stays an equally good preconditioner; a factor that fails
  // after an update is retried from a full assembly.
  __device__ __forceinline__ int assembly_block(int& r0, int& c0) const {
    int g = 0, qd = lane;
#pragma unroll 1
    while (true) {
      const int nq = (min(G::RA * (g + 1), NV) + 3) / 4;
      if (qd < nq) break;
      qd -= nq;
      ++g;
    }
    r0 = G::RA * g;
    c0 = 4 * qd;
    return g;
  }

  // acc += sum over list entries of s_i D_i J_i[r0..] J_i[c0..c0+3]^T, with
  // s_i = -1 for entries marked by the top bit.
  template <bool kSigned, typename T>
  __device__ __forceinline__ void accumulate_rows(const T* list, int n, int r0, int c0,
                                                  float (&acc)[G::RA][4]) {
    constexpr int RA = G::RA;
    const float* Jm = Js();
    const float* Dm = Ds();
    int q = 0;
    // two rows per pass: their loads issue back to back
#pragma unroll 1
    for (; q + 2 <= n; q += 2) {
      float x[2][RA];
      float4 y[2];
#pragma unroll
      for (int r2 = 0; r2 < 2; ++r2) {
        const int e = list[q + r2];
        const int i = kSigned ? (e & 0x7fffffff) : e;
        const float d = (kSigned && e < 0) ? -Dm[i] : Dm[i];
        const float* Ji = Jm + i * G::JS;
#pragma unroll
        for (int u = 0; u < RA; ++u) x[r2][u] = Ji[r0 + u] * d;
        const float2 ya = *reinterpret_cast<const float2*>(Ji + c0);
        const float2 yb = *reinterpret_cast<const float2*>(Ji + c0 + 2);
        y[r2] = make_float4(ya.x, ya.y, yb.x, yb.y);
      }
#pragma unroll
      for (int r2 = 0; r2 < 2; ++r2)
#pragma unroll
        for (int u = 0; u < RA; ++u) {
          acc[u][0] = __fmaf_rn(x[r2][u], y[r2].x, acc[u][0]);
          acc[u][1] = __fmaf_rn(x[r2][u], y[r2].y, acc[u][1]);
          acc[u][2] = __fmaf_rn(x[r2][u], y[r2].z, acc[u][2]);
          acc[u][3] = __fmaf_rn(x[r2][u], y[r2].w, acc[u][3]);
        }
    }
    if (q < n) {
      const int e = list[q];
      const int i = kSigned ? (e & 0x7fffffff) : e;
      const float d = (kSigned && e < 0) ? -Dm[i] : Dm[i];
      const float* Ji = Jm + i * G::JS;
      const float2 ya = *reinterpret_cast<const float2*>(Ji + c0);
      const float2 yb = *reinterpret_cast<const float2*>(Ji + c0 + 2);
      const float4 y = make_float4(ya.x, ya.y, yb.x, yb.y);
#pragma unroll
      for (int u = 0; u < RA; ++u) {
        const float x = Ji[r0 + u] * d;
        acc[u][0] = __fmaf_rn(x, y.x, acc[u][0]);
        acc[u][1] = __fmaf_rn(x, y.y, acc[u][1]);
        acc[u][2] = __fmaf_rn(x, y.z, acc[u][2]);
        acc[u][3] = __fmaf_rn(x, y.w, acc[u][3]);
      }
    }
  }

  // Full assembly H = M + sum over the active list into dst (rows of stride MS).
  __device__ __forceinline__ void assemble_full(float* dst) {
    const float* Mm = Ms();
    if (lane < G::NABLK) {
      int r0, c0;
      assembly_block(r0, c0);
      float acc[G::RA][4];
#pragma unroll
      for (int u = 0; u < G::RA; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
      accumulate_rows<false>(Idx(), nact, r0, c0, acc);
#pragma unroll
      for (int u = 0; u < G::RA; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int rr = r0 + u, cc = c0 + v;
          if (rr < NV && cc <= rr) dst[rr * G::MS + cc] = Mm[rr * G::MS + cc] + acc[u][v];
        }
    }
    __syncwarp();
  }

  // Rows whose side differs between act_bits and hmask_bits, into Chg() (the
  // top bit marks a row that left the set).  Returns their number (the list
  // holds the first kChg).
  __device__ __forceinline__ int changed_rows() {
    int* chg = Chg();
    int base = 0;
#pragma unroll
    for (int t = 0; t < MT; ++t) {
      if (32 * t < m) {
        const bool on = (act_bits >> t) & 1u;
        const bool diff = row_valid(t) && (((act_bits ^ hmask_bits) >> t) & 1u);
        const unsigned bal = __ballot_sync(kFull, diff);
        const int pos = base + __popc(bal & ((1u << lane) - 1u));
        if (diff && pos < G::kChg) chg[pos] = (lane + 32 * t) | (on ? 0 : (int)0x80000000);
        base += __popc(bal);
      }
    }
    __syncwarp();
    return base;
  }

  __device__ __forceinline__ bool assemble_and_factor() {
    if constexpr (kShare) {
      int nchg = G::kChg + 1;
      if (__all_sync(kFull, hmask_valid)) nchg = changed_rows();
      const bool update = nchg <= G::kChg && 4 * nchg <= nact;
      float* H = Hs();
      if (update) {
        if (nchg > 0 && lane < G::NABLK) {
          int r0, c0;
          assembly_block(r0, c0);
          float acc[G::RA][4];
#pragma unroll
          for (int u = 0; u < G::RA; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
          accumulate_rows<true>(Chg(), nchg, r0, c0, acc);
#pragma unroll
          for (int u = 0; u < G::RA; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
              const int rr = r0 + u, cc = c0 + v;
              if (rr < NV && cc <= rr) H[rr * G::MS + cc] += acc[u][v];
            }
        }
        __syncwarp();
      } else {
        assemble_full(H);
      }
      hmask_bits = act_bits;
      hmask_valid = true;
      bool ok = factor(H);
      if (!ok && update) {
        assemble_full(H);
        ok = factor(H);
      }
      fmask_bits = act_bits;
      fmask_valid = true;
      return ok;
    } else {
      assemble_full(Ls());
      const bool ok = factor();
      fmask_bits = act_bits;
      fmask_valid = true;
      return ok;
    }
  }

  // True when the active set differs from the factored one on any lane.
  __device__ __forceinline__ bool need_refactor() {
    return __any_sync(kFull, !fmask_valid || (act_bits != fmask_bits));
  }

  // ------------------------------------------------- compensated products
  // s[t] + c[t] = J_i . (vh + vl) for the rows of this lane.  The vectors are
  // broadcast slots (16-byte aligned, zero beyond NV); J rows and vectors are
  // read a pair of columns at a time, and the terms are accumulated in column
  // order.
  __device__ __forceinline__ void rows_dot2(const float* vh, const float* vl, float (&s)[MT],
                                            float (&c)[MT]) {
    const float2* Jm = reinterpret_cast<const float2*>(Js() + lane * G::JS);
    const float2* vh2 = reinterpret_cast<const float2*>(vh);
    const float2* vl2 = reinterpret_cast<const float2*>(vl);
#pragma unroll
    for (int t = 0; t < MT; ++t) { s[t] = 0.f; c[t] = 0.f; }
#pragma unroll 1
    for (int q = 0; q < G::NP; ++q) {
      const float2 xh = vh2[q], xl = vl2[q];
#pragma unroll
      for (int t = 0; t < MT; ++t)
        if (32 * t < m) {
          const float2 j = Jm[16 * t * G::JS + q];
          dot2(s[t], c[t], j.x, xh.x, xl.x);
          dot2(s[t], c[t], j.y, xh.y, xl.y);
        }
    }
  }

  // Transposed products over the active rows.  From NV = 8 on the lanes
  // take (column pair, row group): lane l reads columns 2 (l % NP) and
  // 2 (l % NP) + 1 of J with one 8-byte load, for every kTG-th active row
  // from l / NP on (kTG = 32 / NP groups: 6 at NV = 9, 3 at NV = 18, 2 at
  // NV = 32); the groups' partial sums meet in the lanes of group 0 by
  // shuffles, and lane j then takes column j from lane j / 2.  Below NV = 8
  // (16 groups and their 15 shuffles for a handful of rows) lane j walks
  // column j over every active row.
  static constexpr int kTG = 32 / G::NP;

  // Group 0's lanes gather the partial sums of the other groups (shuffled
  // from copies, so that no lane reads a sum another lane already added to).
  __device__ __forceinline__ static void gather_groups(float& x, int lane) {
    const float o = x;
#pragma unroll
    for (int g = 1; g < kTG; ++g) x += __shfl_sync(kFull, o, lane + g * G::NP);
  }
  __device__ __forceinline__ static void gather_groups(float& s, float& c, int lane) {
    const float os = s, oc = c;
#pragma unroll
    for (int g = 1; g < kTG; ++g)
      add_pair(s, c, __shfl_sync(kFull, os, lane + g * G::NP),
               __shfl_sync(kFull, oc, lane + g * G::NP));
  }
  // Column j of a pair-spread result, for lane j (0 beyond NV).
  __device__ __forceinline__ float column_of_pairs(float x, float y) const {
    const float ex = __shfl_sync(kFull, x, lane >> 1);
    const float ey = __shfl_sync(kFull, y, lane >> 1);
    return (lane < NV) ? ((lane & 1) ? ey : ex) : 0.f;
  }

  // (s, c) = sum over active rows i of J_ij (v_i + vlo_i), for lane j
  // (compensated; v carried as a float pair so that a force computed from a
  // rounded jar does not put a floor under the residual).
  __device__ __forceinline__ void jt_active(const float* v, const float* vlo, float& s,
                                            float& c) {
    const float* Jm = Js();
    const idx_t* idx = Idx();
    if constexpr (NV >= 8) {
      constexpr int RS = G::JS / 2;  // J row stride in float2
      const int gg = lane / G::NP;
      const float2* Jp = reinterpret_cast<const float2*>(Jm) + lane % G::NP;
      // one row per pass: the two compensated chains already hide each
      // other's latency, and a second pair of them measured slower (register
      // pressure)
      float sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f;
      if (gg < kTG) {
#pragma unroll 1
        for (int q = gg; q < nact; q += kTG) {
          const int i0 = idx[q];
          const float2 a = Jp[i0 * RS];
          const float h0 = v[i0], l0 = vlo[i0];
          dot2(sx, cx, a.x, h0, l0);
          dot2(sy, cy, a.y, h0, l0);
        }
      }
      gather_groups(sx, cx, lane);
      gather_groups(sy, cy, lane);
      s = column_of_pairs(sx, sy);
      c = column_of_pairs(cx, cy);
      return;
    }
    float s2 = 0.f, c2 = 0.f;
    s = 0.f;
    c = 0.f;
    if (lane < NV) {
      int q = 0;
      // four rows per pass, their loads issued before the arithmetic; rows
      // q, q+2 go to one accumulator pair and q+1, q+3 to the other, as in
      // a two-row pass
#pragma unroll 1
      for (; q + 3 < nact; q += 4) {
        int i[4];
        float x[4], y[4], z[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) i[u] = idx[q + u];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          x[u] = Jm[i[u] * G::JS + lane];
          y[u] = v[i[u]];
          z[u] = vlo[i[u]];
        }
        dot2(s, c, x[0], y[0], z[0]);
        dot2(s2, c2, x[1], y[1], z[1]);
        dot2(s, c, x[2], y[2], z[2]);
        dot2(s2, c2, x[3], y[3], z[3]);
      }
#pragma unroll 1
      for (; q + 1 < nact; q += 2) {
        const int i0 = idx[q], i1 = idx[q + 1];
        dot2(s, c, Jm[i0 * G::JS + lane], v[i0], vlo[i0]);
        dot2(s2, c2, Jm[i1 * G::JS + lane], v[i1], vlo[i1]);
      }
      if (q < nact) {
        const int i0 = idx[q];
        dot2(s, c, Jm[i0 * G::JS + lane], v[i0], vlo[i0]);
      }
      add_pair(s, c, s2, c2);
    }
  }

  // hi + lo = D * (xh + xl), as a float pair.
  __device__ __forceinline__ static void scale_pair(float d, float xh, float xl, float& hi,
                                                    float& lo) {
    hi = __fmul_rn(d, xh);
    lo = __fmaf_rn(d, xl, __fmaf_rn(d, xh, -hi));
  }

  // M products.  For 8 <= NV <= 16 the lanes take (row, column group): lane
  // l sums row l % NV over the columns k = l / NV (mod kMG) (kMG = 32 / NV
  // groups: 3 at NV = 9), and the groups' partial sums meet in lane l of
  // group 0 by shuffles; otherwise lane j walks row j.
  static constexpr int kMG = (NV >= 8 && NV <= 16) ? 32 / NV : 1;
  __device__ __forceinline__ void gather_rows(float& x) const {
    const float o = x;
#pragma unroll
    for (int g = 1; g < kMG; ++g) x += __shfl_sync(kFull, o, lane + g * NV);
  }
  __device__ __forceinline__ void gather_rows(float& s, float& c) const {
    const float os = s, oc = c;
#pragma unroll
    for (int g = 1; g < kMG; ++g)
      add_pair(s, c, __shfl_sync(kFull, os, lane + g * NV), __shfl_sync(kFull, oc, lane + g * NV));
  }

  // (s, c) = (M (vh + vl))_j for lane j (compensated).
  __device__ __forceinline__ void m_times(const float* vh, const float* vl, float& s, float& c) {
    s = 0.f;
    c = 0.f;
    if constexpr (kMG > 1) {
      const int gg = lane / NV;
      if (gg < kMG) {
        const float* Mr = Ms() + (lane - gg * NV) * G::MS;
#pragma unroll
        for (int k = gg; k < NV; k += kMG) dot2(s, c, Mr[k], vh[k], vl[k]);
      }
      gather_rows(s, c);
      if (lane >= NV) s = c = 0.f;
      return;
    }
    if (lane < NV) {
      const float* Mr = Ms() + lane * G::MS;
#pragma unroll (kSB)
      for (int k = 0; k < NV; ++k) dot2(s, c, Mr[k], vh[k], vl[k]);
    }
  }

  // Plain FP32 counterparts, used while the active set is still changing.
  __device__ __forceinline__ void rows_dot(const float* vh, float (&s)[MT]) {
    const float2* Jm = reinterpret_cast<const float2*>(Js() + lane * G::JS);
    const float2* v2 = reinterpret_cast<const float2*>(vh);
#pragma unroll
    for (int t = 0; t < MT; ++t) s[t] = 0.f;
#pragma unroll
    for (int q = 0; q < G::NP; ++q) {
      const float2 x = v2[q];
#pragma unroll
      for (int t = 0; t < MT; ++t)
        if (32 * t < m) {
          const float2 j = Jm[16 * t * G::JS + q];
          s[t] = __fmaf_rn(j.x, x.x, s[t]);
          s[t] = __fmaf_rn(j.y, x.y, s[t]);
        }
    }
  }
  __device__ __forceinline__ float jt_active_plain(const float* v) {
    const float* Jm = Js();
    const idx_t* idx = Idx();
    if constexpr (NV >= 8) {
      constexpr int RS = G::JS / 2;
      const int gg = lane / G::NP;
      const float2* Jp = reinterpret_cast<const float2*>(Jm) + lane % G::NP;
      float sx = 0.f, sy = 0.f, tx = 0.f, ty = 0.f;
      if (gg < kTG) {
        int q = gg;
#pragma unroll 1
        for (; q + kTG < nact; q += 2 * kTG) {
          const int i0 = idx[q], i1 = idx[q + kTG];
          const float2 a = Jp[i0 * RS], b = Jp[i1 * RS];
          const float v0 = v[i0], v1 = v[i1];
          sx = __fmaf_rn(a.x, v0, sx);
          sy = __fmaf_rn(a.y, v0, sy);
          tx = __fmaf_rn(b.x, v1, tx);
          ty = __fmaf_rn(b.y, v1, ty);
        }
        if (q < nact) {
          const int i0 = idx[q];
          const float2 a = Jp[i0 * RS];
          sx = __fmaf_rn(a.x, v[i0], sx);
          sy = __fmaf_rn(a.y, v[i0], sy);
        }
      }
      sx += tx;
      sy += ty;
      gather_groups(sx, lane);
      gather_groups(sy, lane);
      return column_of_pairs(sx, sy);
    }
    float s = 0.f, s2 = 0.f;
    if (lane < NV) {
      int q = 0;
#pragma unroll 1
      for (; q + 3 < nact; q += 4) {
        int i[4];
        float x[4], y[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) i[u] = idx[q + u];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          x[u] = Jm[i[u] * G::JS + lane];
          y[u] = v[i[u]];
        }
        s = __fmaf_rn(x[0], y[0], s);
        s2 = __fmaf_rn(x[1], y[1], s2);
        s = __fmaf_rn(x[2], y[2], s);
        s2 = __fmaf_rn(x[3], y[3], s2);
      }
#pragma unroll 1
      for (; q + 1 < nact; q += 2) {
        const int i0 = idx[q], i1 = idx[q + 1];
        s = __fmaf_rn(Jm[i0 * G::JS + lane], v[i0], s);
        s2 = __fmaf_rn(Jm[i1 * G::JS + lane], v[i1], s2);
      }
      if (q < nact) s = __fmaf_rn(Jm[idx[q] * G::JS + lane], v[idx[q]], s);
    }
    return s + s2;
  }
  __device__ __forceinline__ float m_times_plain(const float* vh) {
    float s = 0.f;
    if constexpr (kMG > 1) {
      const int gg = lane / NV;
      if (gg < kMG) {
        const float* Mr = Ms() + (lane - gg * NV) * G::MS;
#pragma unroll
        for (int k = gg; k < NV; k += kMG) s = __fmaf_rn(Mr[k], vh[k], s);
      }
      gather_rows(s);
      return (lane < NV) ? s : 0.f;
    }
    if (lane < NV) {
      const float* Mr = Ms() + lane * G::MS;
#pragma unroll (kSB)
      for (int k = 0; k < NV; ++k) s = __fmaf_rn(Mr[k], vh[k], s);
    }
    return s;
  }

  // --------------------------------------------------------- residual
  // At a = ah + al: jar (compensated), active set, f, active row list,
  // r = M a - qfrc + J^T f (compensated), maq = M a - qfrc.
  // Returns max|r|; *scale = max(1, |qfrc|, |Ma|, |J^T f|); *bad = non-finite.
  //
  // precise = false evaluates the same quantities in plain FP32 (used while
  // the active set is still changing, where only the direction matters).
  __device__ __forceinline__ float residual(float* scale, bool* bad, bool precise = true) {
    put_vec(V_AH, ah);
    put_vec(V_AL, al);
    const float* vh = Vec(V_AH);
    const float* vl = Vec(V_AL);
    float s[MT], c[MT];
    if (precise) {
      rows_dot2(vh, vl, s, c);
    } else {
      rows_dot(vh, s);
#pragma unroll
      for (int t = 0; t < MT; ++t) c[t] = 0.f;
    }
    act_bits = 0;
    float* F = Fs();
    float* Fl = Flo();
    idx_t* idx = Idx();
    int base = 0;
    float fm = 0.f;
#pragma unroll
    for (int t = 0; t < MT; ++t) {
      if (32 * t < m) {
        // plain: jar = fl(s - aref) and f = fl(D jar), the high parts of the
        // compensated forms; f's low part is read only after a compensated
        // residual has rewritten it
        float jlo = 0.f;
        if (precise) {
          float u, ue;
          two_sum(s[t], -aref_r[t], u, ue);
          const float tl = __fadd_rn(ue, c[t]);
          jar_r[t] = __fadd_rn(u, tl);
          jlo = __fsub_rn(tl, __fsub_rn(jar_r[t], u));
        } else {
          jar_r[t] = __fsub_rn(s[t], aref_r[t]);
        }
        const bool on = row_valid(t) && jar_r[t] < 0.f;
        float f = 0.f, flo = 0.f;
        if (on) {
          if (precise) scale_pair(D_r[t], jar_r[t], jlo, f, flo);
          else f = __fmul_rn(D_r[t], jar_r[t]);
        }
        if (row_valid(t)) {
          F[lane + 32 * t] = f;
          if (precise) Fl[lane + 32 * t] = flo;
        }
        fm = fmaxf(fm, fabsf(f));
        const unsigned bal = __ballot_sync(kFull, on);
        if (on) {
          act_bits |= 1u << t;
          idx[base + __popc(bal & ((1u << lane) - 1u))] = lane + 32 * t;
        }
        base += __popc(bal);
      }
    }
    nact = base;
    if (precise) fmax = warp_max(fm);  // read only by the compensated phase's step test
    __syncwarp();
    float js, jc, ms, mc;
    if (precise) {
      jt_active(F, Fl, js, jc);
      m_times(vh, vl, ms, mc);
    } else {
      js = jt_active_plain(F);
      ms = m_times_plain(vh);
      jc = 0.f;
      mc = 0.f;
    }
    float t1, e1, t2, e2;
    two_sum(ms, -qf, t1, e1);
    const float lo1 = __fadd_rn(e1, mc);
    maq = __fadd_rn(t1, lo1);
    two_sum(t1, js, t2, e2);
    const float lo2 = __fadd_rn(lo1, __fadd_rn(e2, jc));
    r = __fadd_rn(t2, lo2);
    rlo = __fsub_rn(lo2, __fsub_rn(r, t2));
    if (lane >= NV) {
      r = 0.f;
      rlo = 0.f;
      maq = 0.f;
    }
    const float rm = warp_max(fabsf(r));
    const float sc = fmaxf(fmaxf(1.f, qmax), warp_max(fmaxf(fabsf(ms), fabsf(js))));
    *scale = sc;
    *bad = __any_sync(kFull, !(fabsf(r) < CUDART_INF_F)) || !(sc < CUDART_INF_F);
    return rm;
  }

  // -------------------------------------------------------- line search
  // alpha > 0 minimising phi(alpha) = L(a + alpha p) (Eq. 10), p spread per
  // lane.  phi'(alpha) = c0 + alpha p^T M p + sum_i D_i s_i min(jar_i + alpha s_i, 0)
  // with c0 = p^T (M a - qfrc) and s = J p; phi' is continuous, piecewise
  // linear and strictly increasing.  Also leaves s_r = J p.
  //
  // kDiff evaluates the same phi' in difference form,
  //   phi'(alpha) = p^T r + alpha (p^T M p + sum_{active at alpha} D s^2)
  //                 - sum_{leaving} D s jar + sum_{entering} D s jar,
  // with p^T r compensated: nothing cancels, so a directional derivative far
  // below the size of p^T (M a - qfrc) and of the contact terms (conjugate
  // gradients near a*) is still resolved.  Newton steps have their root near
  // alpha = 1 and use the plain form.
  template <bool kDiff = false>
  __device__ __forceinline__ float line_search(float p, float* dfmax, bool* crossed) {
    put_vec(V_P, p);
    const float* vp = Vec(V_P);
    rows_dot(vp, s_r);
    const float Mp = m_times_plain(vp);
    const float pMp = warp_sum(lane < NV ? p * Mp : 0.f);
    float c0;
    if (kDiff) {
      const float prh = __fmul_rn(p, r);
      const float prl = __fmaf_rn(p, rlo, __fmaf_rn(p, r, -prh));
      c0 = warp_sum(prh) + warp_sum(prl);
    } else {
      c0 = warp_sum(p * maq);
    }
    float bp[MT];
#pragma unroll
    for (int t = 0; t < MT; ++t)
      bp[t] = (row_valid(t) && s_r[t] != 0.f) ? __fdividef(-jar_r[t], s_r[t]) : CUDART_INF_F;
    // The slope uses the rows strictly active at alpha; a row exactly at its
    // breakpoint (u == 0) is a measure-zero event whose only effect would be
    // one more trial.
    float alpha = 1.f, lo = 0.f, hi = CUDART_INF_F;
#pragma unroll 1
    for (int it = 0; it < kLineSearchMax; ++it) {
      float sum = 0.f, cs = 0.f;
#pragma unroll
      for (int t = 0; t < MT; ++t) {
        if (row_valid(t)) {
          const float u = __fmaf_rn(alpha, s_r[t], jar_r[t]);
          const float ds = D_r[t] * s_r[t];
          if (kDiff) {
            const bool on0 = (act_bits >> t) & 1u;
            if (u < 0.f) cs = __fmaf_rn(ds, s_r[t], cs);
            if (on0 && !(u < 0.f)) sum = __fmaf_rn(-ds, jar_r[t], sum);
            if (!on0 && u < 0.f) sum = __fmaf_rn(ds, jar_r[t], sum);
          } else if (u < 0.f) {
            sum = __fmaf_rn(ds, u, sum);
            cs = __fmaf_rn(ds, s_r[t], cs);
          }
        }
      }
      sum = warp_sum(sum);
      cs = warp_sum(cs);
      const float d = kDiff ? c0 + alpha * (pMp + cs) + sum : c0 + alpha * pMp + sum;
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
      // any breakpoint strictly between the trial and its Newton point
      bool inside = false;
#pragma unroll
      for (int t = 0; t < MT; ++t) inside = inside || (bp[t] > x0 && bp[t] < x1);
      if (!__any_sync(kFull, inside) && an > 0.f) {
        alpha = an;
        break;
      }
      if (!(an > lo && an < hi)) an = (hi == CUDART_INF_F) ? 2.f * alpha : 0.5f * (lo + hi);
      alpha = an;
      if (it == kLineSearchMax - 1) alpha = (lo > 0.f) ? lo : alpha;
    }
    // largest change of an active force over the step, and whether any row
    // changes side of its breakpoint within (0, alpha)
    float df = 0.f;
    int cr = 0;
#pragma unroll
    for (int t = 0; t < MT; ++t) {
      if ((act_bits >> t) & 1u) df = fmaxf(df, fabsf(D_r[t] * alpha * s_r[t]));
      cr |= (bp[t] > 0.f && bp[t] < alpha) ? 1 : 0;
    }
    *dfmax = warp_max(df);
    *crossed = __any_sync(kFull, cr);
    return alpha;
  }

  // v += dv, kept as a normalised float pair (vh, vl).
  __device__ __forceinline__ static void add_to_pair(float& vh, float& vl, float dv) {
    float s, e;
    two_sum(vh, dv, s, e);
    const float lo = __fadd_rn(vl, e);
    vh = __fadd_rn(s, lo);
    vl = __fsub_rn(lo, __fsub_rn(vh, s));
  }

  // Whether the correction z (spread per lane) would move a by at most
  // kStepTol amax and every active force D_i (J z)_i by at most kForceTol
  // fmax (fmax from the last compensated residual).  Uses the V_X slot.
  __device__ __forceinline__ bool small_correction(float z, float amax) {
    const float zm = warp_max(fabsf(z));
    if (!(zm <= kStepTol * amax)) return false;
    put_vec(V_X, z);
    float sz[MT];
    rows_dot(Vec(V_X), sz);
    float df = 0.f;
#pragma unroll
    for (int t = 0; t < MT; ++t)
      if ((act_bits >> t) & 1u) df = fmaxf(df, fabsf(D_r[t] * sz[t]));
    return warp_max(df) <= kForceTol * fmax;
  }

  // After a step a += alpha p that crossed no breakpoint: the residual
  // quantities the adjoint and the outputs read (jar, the active forces f as
  // a pair) advanced by alpha J p from the line search's products s_r = J p;
  // the active set and its row list are unchanged.
  __device__ __forceinline__ void advance_forces(float alpha) {
    float* F = Fs();
    float* Fl = Flo();
#pragma unroll
    for (int t = 0; t < MT; ++t) {
      if (row_valid(t)) {
        const float ds = alpha * s_r[t];
        jar_r[t] = __fadd_rn(jar_r[t], ds);
        if ((act_bits >> t) & 1u) {
          float fh = F[lane + 32 * t], fl = Fl[lane + 32 * t];
          add_to_pair(fh, fl, D_r[t] * ds);
          F[lane + 32 * t] = fh;
          Fl[lane + 32 * t] = fl;
        }
      }
    }
    __syncwarp();
  }

  // --------------------------------------------------------- forward solve
  // Newton iteration (Eqs. 9-10) from a0 = M^-1 qfrc (Eq. 1).  Returns the
  // status; *iters = Newton steps.  On return the residual quantities (jar,
  // act_bits, f, active list) belong to the returned a.
  __device__ __forceinline__ int forward(const Params& P, int* iters) {
    *iters = 0;
    if (!factor_M()) return CS_ST_CHOLFAIL;
    fmask_bits = 0;
    fmask_valid = true;
    ah = chol_solve(qf);
    al = 0.f;
    uint32_t prev_bits = 0;
    bool prev_small = false;
    // Plain FP32 residuals while the active set changes; compensated ones
    // from the first step that crosses no breakpoint on (every stop test and
    // every returned quantity is taken in the compensated phase).
    bool precise = false;
    // Once the active set has settled the problem is a fixed quadratic and
    // the FP32 factor only preconditions it: consecutive such steps are
    // conjugated (preconditioned CG, Fletcher-Reeves beta), restarted
    // whenever the active set or the factor changes.
    bool cg = false;
    float p_prev = 0.f, zr_prev = 1.f, dpm_prev = 0.f;
#pragma unroll 1
    for (int k = 0;; ++k) {
      float scale;
      bool bad;
      const float rmax = residual(&scale, &bad, precise);
      if (bad) return CS_ST_NONFINITE;
      if (!precise && (k >= P.max_iter || rmax <= P.tol * scale)) {
        precise = true;  // re-evaluate this point accurately before stopping
        --k;
        continue;
      }
      if (rmax <= P.tol * scale) return CS_ST_OK;
      const bool same = !__any_sync(kFull, act_bits != prev_bits);
      if (k >= P.max_iter) return CS_ST_MAXITER;
      cg = cg && same;
      if (need_refactor()) {
        if (!assemble_and_factor()) return CS_ST_CHOLFAIL;
        cg = false;
      }
      const float z = chol_solve(r);
      const float amax = warp_max(fabsf(ah));
      // Once the active set has settled (compensated phase, the same set as
      // at the previous point), the FP32 Newton correction z = H^-1 r
      // estimates the remaining error of a: when it would move a by <=
      // kStepTol |a| and every active force by <= kForceTol |f|, a is at the
      // attainable FP32 accuracy and is returned as it is (its residual
      // quantities are the ones just evaluated).
      // A step just taken that was itself that small (a conjugated or
      // stagnating direction whose line search found only a tiny alpha) ends
      // the solve the same way.
      if (precise && k > 0 && same && (prev_small || small_correction(z, amax)))
        return CS_ST_OK;
      const float zr = warp_sum(z * r);
      const float beta = (cg && zr_prev > 0.f) ? fmaxf(zr / zr_prev, 0.f) : 0.f;
      float p = __fmaf_rn(beta, p_prev, -z);
      float ptr = warp_sum(p * r);
      if (!(ptr < 0.f) && beta != 0.f) {  // lost descent: restart from -z
        p = -z;
        ptr = -zr;
      }
      if (!(ptr < 0.f)) {
        const float pm = warp_max(fabsf(p));
        return (pm <= kStepTol * amax) ? CS_ST_OK : CS_ST_NOPROGRESS;
      }
      float dfm;
      bool crossed;
      const float alpha = line_search(p, &dfm, &crossed);
      const float dp = alpha * p;
      add_to_pair(ah, al, dp);
      *iters = k + 1;
      const float dpm = warp_max(fabsf(dp));
      // A step at the settled set that crossed no breakpoint is a step of an
      // iterative refinement (conjugated after the first): its steps shrink
      // geometrically, by a ratio q estimated from two consecutive ones (the
      // first against a itself; Demmel et al., ACM TOMS 32(2), 2006), so the
      // error it leaves is about q / (1 - q) |dp|.  When that meets both
      // stop tolerances the solve ends here, with f and jar advanced along
      // the step instead of re-evaluated by another compensated residual.
      if (precise && same && !crossed) {
        const float q = dpm / (cg ? dpm_prev : amax);
        const float gq = (cg ? 1.f : kFirstRatioMargin) * q / (1.f - q);
        if (q < 0.5f && gq * dpm <= kStepTol * amax && gq * dfm <= kForceTol * fmax) {
          advance_forces(alpha);
          return CS_ST_OK;
        }
      }
      dpm_prev = dpm;
      prev_small = precise && (dpm <= kStepTol * amax) && (dfm <= kForceTol * fmax);
      prev_bits = act_bits;
      cg = precise && !crossed;
      p_prev = p;
      zr_prev = zr;
      precise = precise || !crossed;
    }
  }

  // ------------------------------------------- nonlinear conjugate gradients
  // The other forward solver MJX offers: conjugate directions on the same
  // objective (Eq. 5), preconditioned by M^-1 (the factor of M stays in
  // Ls()), the Polak-Ribiere+ beta (which resets itself when the gradient
  // turns; a non-descent direction restarts from -M^-1 r), and the exact line
  // search of Eq. 10.  Residuals are compensated throughout (CG steps keep
  // crossing breakpoints, so the plain phase of forward() would never end).
  // It stops on the residual test, or once the residual has not halved over
  // 4 nv + 20 steps while below 1e-5 of its scale (FP32 conjugacy is lost at
  // cond(M^-1 H) ~ 1e6 and the iteration only creeps); a short CG step alone
  // says nothing about the distance to a*.  The adjoint does not depend on
  // how a* was reached (Eq. 14): run<MODE_FUSED_NCG> rebuilds H(a*).
  __device__ __forceinline__ int forward_ncg(const Params& P, int* iters) {
    *iters = 0;
    if (!factor_M()) return CS_ST_CHOLFAIL;
    fmask_valid = false;  // Ls() holds chol(M), not a factor of H
    ah = chol_solve(qf);
    al = 0.f;
    bool have_prev = false;
    float d_prev = 0.f, r_prev = 0.f, zr_prev = 1.f, best = CUDART_INF_F;
    int since_best = 0;
#pragma unroll 1
    for (int k = 0;; ++k) {
      float scale;
      bool bad;
      const float rmax = residual(&scale, &bad, true);
      if (bad) return CS_ST_NONFINITE;
      if (rmax <= P.tol * scale) return CS_ST_OK;
      if (rmax < 0.5f * best) {
        best = rmax;
        since_best = 0;
      } else if (++since_best > 4 * nv + 20 && rmax <= 1e-5f * scale) {
        return CS_ST_OK;
      }
      if (k >= P.max_iter) return CS_ST_MAXITER;
      const float z = chol_solve(r);
      const float zr = warp_sum(z * r);
      float beta = 0.f;
      if (have_prev && zr_prev > 0.f) beta = fmaxf(warp_sum(z * (r - r_prev)) / zr_prev, 0.f);
      float d = __fmaf_rn(beta, d_prev, -z);
      float dtr = warp_sum(d * r);
      if (!(dtr < 0.f) && beta != 0.f) {
        d = -z;
        dtr = -zr;
      }
      const float amax = warp_max(fabsf(ah));
      if (!(dtr < 0.f)) {
        const float dm = warp_max(fabsf(d));
        return (dm <= kStepTol * amax) ? CS_ST_OK : CS_ST_NOPROGRESS;
      }
      float dfm;
      bool crossed;
      const float alpha = line_search<true>(d, &dfm, &crossed);
      add_to_pair(ah, al, alpha * d);
      *iters = k + 1;
      d_prev = d;
      r_prev = r;
      zr_prev = zr;
      have_prev = true;
    }
  }

  // ---------------------------------------------------------- adjoint
  // Solve H w = g at the current point (Eq. 17) by iterative refinement with
  // compensated residuals.  Leaves w in (wh, wl), lambda = D_act . J w in
  // Lam() for every row < m.
  __device__ __forceinline__ void adjoint(float& wh, float& wl) {
    solve_refined<true>(gj, 0.f, wh, wl, kAdjStepTol, kAdjForceTol);
  }

  // H w = rhs + rhs_lo (spread per lane) with H = M + sum over the active
  // list of D_i J_i^T J_i factored in Ls(): FP32 factor as preconditioner,
  // residuals rhs - M w - J^T (D_act . J w) accumulated with error-free
  // transformations.
  //
  // Each pass forms lambda = D_act . J w (compensated) at the current w, then
  // the residual rho and the correction dw = H^-1 rho; when dw would move w
  // by <= step_tol |w| and every active lambda by <= force_tol |lambda|, w is
  // kept as it is (its error is bounded by the untaken correction) and lambda
  // already belongs to it, so no pass is spent re-evaluating lambda at a
  // point that differs from w only beyond that resolution.  The default pair
  // is the forward's (FP32 resolution), which the unrolled reverse sweep
  // needs; the IFT adjoint passes the looser kAdjStepTol / kAdjForceTol.
  //
  // kPredict also ends the refinement one pass earlier: the corrections of
  // an iterative refinement shrink geometrically, by a ratio q estimated from
  // two consecutive ones (the first solve counting as the correction from
  // w = 0; Demmel, Hida, Kahan, Li, Mukherjee and Riedy, "Error bounds from
  // extra-precise iterative refinement", ACM TOMS 32(2), 2006), so the error
  // left after applying dw is about q / (1 - q) |dw|.  When that meets both
  // tolerances dw is applied, lambda advanced by D_act (J dw) from the
  // products the test already formed, and no pass is spent confirming it.
  template <bool kPredict = false>
  __device__ __forceinline__ void solve_refined(float rhs, float rhs_lo, float& wh, float& wl,
                                                float step_tol = kStepTol,
                                                float force_tol = kForceTol) {
    wh = chol_solve(rhs);
    wl = 0.f;
    float* Lm = Lam();
    float* Lml = Lamlo();
    float prev = 0.f;  // max |last correction| (0: w itself is the last one)
#pragma unroll 1
    for (int it = 0;; ++it) {
      put_vec(V_WH, wh);
      put_vec(V_WL, wl);
      const float* vh = Vec(V_WH);
      const float* vl = Vec(V_WL);
      float s[MT], c[MT];
      rows_dot2(vh, vl, s, c);
      float lmax = 0.f;
#pragma unroll
      for (int t = 0; t < MT; ++t) {
        if (32 * t < m) {
          const bool on = (act_bits >> t) & 1u;
          const float uh = __fadd_rn(s[t], c[t]);
          const float ul = __fsub_rn(c[t], __fsub_rn(uh, s[t]));
          float lam = 0.f, lamlo = 0.f;
          if (on) scale_pair(D_r[t], uh, ul, lam, lamlo);
          if (row_valid(t)) {
            Lm[lane + 32 * t] = lam;
            Lml[lane + 32 * t] = lamlo;
          }
          lmax = fmaxf(lmax, fabsf(lam));
        }
      }
      lmax = warp_max(lmax);
      __syncwarp();
      if (it == kAdjointRefineMax) break;
      // rho = g - M w - J^T lambda (compensated)
      float js, jc, ms, mc;
      jt_active(Lm, Lml, js, jc);
      m_times(vh, vl, ms, mc);
      float t1, e1, t2, e2;
      two_sum(rhs, -ms, t1, e1);
      two_sum(t1, -js, t2, e2);
      float rho = __fadd_rn(t2, __fsub_rn(__fadd_rn(__fadd_rn(e1, e2), rhs_lo), __fadd_rn(mc, jc)));
      if (lane >= NV) rho = 0.f;
      const float dw = chol_solve(rho);
      // the correction's size, in w and in the active lambda = D (J dw)
      put_vec(V_X, dw);
      float sd[MT];
      rows_dot(Vec(V_X), sd);
      float dl = 0.f;
#pragma unroll
      for (int t = 0; t < MT; ++t)
        if ((act_bits >> t) & 1u) dl = fmaxf(dl, fabsf(D_r[t] * sd[t]));
      const float dmax = warp_max(fabsf(dw));
      const float wmax = warp_max(fabsf(wh));
      dl = warp_max(dl);
      if (dmax <= step_tol * wmax && dl <= force_tol * lmax) break;
      add_to_pair(wh, wl, dw);
      if (kPredict) {
        const float q = dmax / (prev > 0.f ? prev : wmax);
        const float gq = (prev > 0.f ? 1.f : kFirstRatioMargin) * q / (1.f - q);
        if (q < 0.5f && gq * dmax <= step_tol * wmax && gq * dl <= force_tol * lmax) {
#pragma unroll
          for (int t = 0; t < MT; ++t)
            if ((act_bits >> t) & 1u) {
              float lh = Lm[lane + 32 * t], ll = Lml[lane + 32 * t];
              add_to_pair(lh, ll, D_r[t] * sd[t]);
              Lm[lane + 32 * t] = lh;
              Lml[lane + 32 * t] = ll;
            }
          break;
        }
        prev = dmax;
      }
    }
    __syncwarp();
  }

  // Write dqfrc = w, daref = lambda, dJ = -(f w^T + lambda a^T), and when
  // asked for, dM = -(w a^T + a w^T) / 2 (M symmetric) and
  // dD_i = -(J w)_i min(jar_i, 0) = -lambda_i jar_i / D_i on active rows.
  __device__ __forceinline__ void write_grads(const Params& P, const cs_inst& e, float wh) {
    if (lane < nv) P.dqfrc[e.off_v + lane] = wh;
    const float* Lm = Lam();
    const float* F = Fs();
#pragma unroll
    for (int t = 0; t < MT; ++t)
      if (row_valid(t)) P.daref[e.off_r + lane + 32 * t] = Lm[lane + 32 * t];
    put_vec(V_WH, wh);
    put_vec(V_X, ah);
    const float* vw = Vec(V_WH);
    const float* va = Vec(V_X);
    float* dJ = P.dJ + e.off_J;
    const int mnv = m * nv;
    int q0 = 0;
    if (nv == NV && NV >= 4 && (reinterpret_cast<uintptr_t>(dJ) & 15) == 0) {
      // four consecutive entries per lane and one 16-byte store; the four
      // span at most two rows of J
      const int n4 = mnv >> 2;
#pragma unroll 1
      for (int q4 = lane; q4 < n4; q4 += 32) {
        const int q = 4 * q4;
        const int rr = q / NV, cc = q - rr * NV;
        const float f0 = F[rr], l0 = Lm[rr], f1 = F[rr + 1], l1 = Lm[rr + 1];
        float o[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const bool next = cc + u >= NV;
          const int c = next ? cc + u - NV : cc + u;
          o[u] = -__fmaf_rn(next ? f1 : f0, vw[c], (next ? l1 : l0) * va[c]);
        }
        *reinterpret_cast<float4*>(dJ + q) = make_float4(o[0], o[1], o[2], o[3]);
      }
      q0 = 4 * n4;
    }
#pragma unroll 1
    for (int q = q0 + lane; q < mnv; q += 32) {
      int rr, cc;
      if (nv == NV) {
        rr = q / NV;
        cc = q - rr * NV;
      } else {
        rr = q / nv;
        cc = q - rr * nv;
      }
      dJ[q] = -__fmaf_rn(F[rr], vw[cc], Lm[rr] * va[cc]);
    }
    if (P.dD) {
#pragma unroll
      for (int t = 0; t < MT; ++t)
        if (row_valid(t)) {
          const bool on = (act_bits >> t) & 1u;
          P.dD[e.off_r + lane + 32 * t] =
              on ? -__fdiv_rn(Lm[lane + 32 * t] * jar_r[t], D_r[t]) : 0.f;
        }
    }
    if (P.dM) {
      float* dM = P.dM + e.off_M;
      const int nn = nv * nv;
#pragma unroll 1
      for (int q = lane; q < nn; q += 32) {
        const int rr = q / nv, cc = q - rr * nv;
        dM[q] = -0.5f * __fmaf_rn(vw[rr], va[cc], va[rr] * vw[cc]);
      }
    }
  }

  // Load the factor kept by the forward pass (packed lower rows of the real
  // nv x nv block; padded rows are the identity).
  __device__ __forceinline__ void load_factor(const float* Lp) {
    float* L = Ls();
    if (lane < NV) {
#pragma unroll 1
      for (int k = 0; k <= lane; ++k) {
        float v;
        if (lane < nv) v = __ldg(Lp + lane * (lane + 1) / 2 + k);
        else v = (k == lane) ? 1.f : 0.f;
        L[lane * G::MS + k] = v;
      }
    }
    __syncwarp();
    if (lane < NV) Vec(V_DINV)[lane] = 1.0f / L[lane * G::MS + lane];
    __syncwarp();
  }

  __device__ __forceinline__ void store_factor(float* Lp) {
    const float* L = Ls();
    if (lane < nv) {
#pragma unroll 1
      for (int k = 0; k <= lane; ++k) Lp[lane * (lane + 1) / 2 + k] = L[lane * G::MS + k];
    }
  }

  __device__ __forceinline__ void zero_grads(const Params& P, const cs_inst& e) {
    if (lane < nv) P.dqfrc[e.off_v + lane] = 0.f;
#pragma unroll 1
    for (int i = lane; i < m; i += 32) P.daref[e.off_r + i] = 0.f;
#pragma unroll 1
    for (int q = lane; q < m * nv; q += 32) P.dJ[e.off_J + q] = 0.f;
    if (P.dD)
#pragma unroll 1
      for (int i = lane; i < m; i += 32) P.dD[e.off_r + i] = 0.f;
    if (P.dM)
#pragma unroll 1
      for (int q = lane; q < nv * nv; q += 32) P.dM[e.off_M + q] = 0.f;
  }

  // ------------------------------------------------------------ drivers
  template <int MODE>
  __device__ __forceinline__ void run(const Params& P, int b, const cs_inst& e) {
    if (!load(P, e)) {
      if (lane == 0) {
        P.status[b] = CS_ST_BADSHAPE;
        P.iters[b] = 0;
      }
      return;
    }
    if (MODE == MODE_FWD || MODE == MODE_FUSED || MODE == MODE_FUSED_NCG) {
      gj = (MODE != MODE_FWD && lane < nv) ? __ldg(P.g + e.off_v + lane) : 0.f;
      int iters = 0;
      const int st = (MODE == MODE_FUSED_NCG) ? forward_ncg(P, &iters) : forward(P, &iters);
      if (lane < nv) P.a[e.off_v + lane] = ah;
      if (lane == 0) {
        P.status[b] = st;
        P.iters[b] = iters;
      }
      if (st == CS_ST_CHOLFAIL || st == CS_ST_NONFINITE) {
        if (MODE != MODE_FWD) zero_grads(P, e);
        return;
      }
      if (MODE == MODE_FWD) {
        if (lane < nv) P.a_lo[e.off_v + lane] = al;
#pragma unroll
        for (int t = 0; t < MT; ++t)
          if (row_valid(t)) P.act[e.off_r + lane + 32 * t] = (act_bits >> t) & 1u;
        if (P.keep_factor && P.Lst) {
          if (need_refactor())
            if (!assemble_and_factor()) {
              if (lane == 0) P.status[b] = CS_ST_CHOLFAIL;
              return;
            }
          store_factor(P.Lst + e.off_M);
        }
        return;
      }
      // fused: adjoint at the returned point
      if (need_refactor())
        if (!assemble_and_factor()) {
          if (lane == 0) P.status[b] = CS_ST_CHOLFAIL;
          zero_grads(P, e);
          return;
        }
      float wh, wl;
      adjoint(wh, wl);
      write_grads(P, e, wh);
    } else {  // MODE_ADJ
      gj = (lane < nv) ? __ldg(P.g + e.off_v + lane) : 0.f;
      const int st0 = P.status[b];
      if (st0 == CS_ST_CHOLFAIL || st0 == CS_ST_NONFINITE || st0 == CS_ST_BADSHAPE) {
        zero_grads(P, e);
        return;
      }
      ah = (lane < nv) ? __ldg(P.a + e.off_v + lane) : 0.f;
      al = (lane < nv) ? __ldg(P.a_lo + e.off_v + lane) : 0.f;
      float scale;
      bool bad;
      residual(&scale, &bad);  // jar, f, active list at a*
      uint32_t kept = 0;
#pragma unroll
      for (int t = 0; t < MT; ++t)
        if (row_valid(t) && P.act[e.off_r + lane + 32 * t]) kept |= 1u << t;
      if (P.keep_factor && P.Lst) {
        load_factor(P.Lst + e.off_M);
        fmask_bits = kept;
        fmask_valid = true;
      } else {
        fmask_valid = false;
      }
      if (need_refactor())
        if (!assemble_and_factor()) {
          if (lane == 0) P.status[b] = CS_ST_CHOLFAIL;
          zero_grads(P, e);
          return;
        }
      float wh, wl;
      adjoint(wh, wl);
      write_grads(P, e, wh);
    }
  }
};

// One warp per instance; warps claim instances dynamically (counter) or in a
// static round-robin.
// Register budget per thread by rows per lane, measured on the quadruped
// batch (nv 18): each bucket's time alone at budgets 80 / 96 / 112 / 128 was
// best at 80 for m <= 32 (whose small shared-memory slice lets the most
// warps in), 96 for m <= 64 and 112 beyond.  The nv 32 kernels, whose
// shared-memory slices already hold fewer warps per SM, get 32 more so that
// the 32-wide factor does not spill.  Launches use at most 256 threads.
__host__ __device__ constexpr int warp_kernel_regs(int NV, int MT) {
  return (MT <= 1 ? 80 : MT <= 2 ? 96 : MT <= 4 ? 112 : 128) + (NV > 18 ? 32 : 0);
}

template <int NV, int MT, int MODE>
__global__ void __maxnreg__(warp_kernel_regs(NV, MT))
    warp_solve_kernel(const __grid_constant__ Params P) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  using G = Geo<NV, MT, true>;
  const int warp = threadIdx.x >> 5;
  WarpSolver<NV, MT, true> S;
  S.sm = reinterpret_cast<float*>(smem_raw + (size_t)warp * G::kBytes);
  S.lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  int idx = blockIdx.x * wpb + warp;
  const int stride = gridDim.x * wpb;
#pragma unroll 1
  for (int guard = 0; guard <= P.n_work; ++guard) {
    if (P.counter) {
      int v = 0;
      if (S.lane == 0) v = atomicAdd(P.counter, 1);
      idx = __shfl_sync(kFull, v, 0);
    }
    if (idx >= P.n_work) break;
    // the entry one grid of warps further on is claimed about one solve
    // later (by this warp under static striding, by whichever warp is free
    // under the claim counter): its inputs are prefetched into L2 now
    const int ipf = idx + stride;
    const int b = P.order ? P.order[idx] : idx;
    int pf = (ipf < P.n_work) ? (P.order ? P.order[ipf] : ipf) : -1;
    if (pf >= P.n) pf = -1;
    if (b >= 0 && b < P.n) {
      const cs_inst e = P.inst[b];
      if (pf >= 0) {
        const cs_inst epf = P.inst[pf];
        S.prefetch(P, epf);
      }
      S.template run<MODE>(P, b, e);
    }
    __syncwarp();
    if (!P.counter) idx += stride;
  }
}

}  // namespace csk
