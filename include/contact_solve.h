/*
 * contact_solve.h -- C ABI of the B300 batched regularised smooth-contact solve
 * and its implicit-function-theorem (IFT) adjoint.
 *
 * The operation (Section III of "Amortising Trajectory Optimisation for
 * Residual MPC via Implicit Contact Differentiation"), per instance b:
 *
 *   a0  = M^-1 qfrc                                            (Eq. 1)
 *   a*  = argmin_a 1/2 (a-a0)^T M (a-a0) + 1/2 sum_i D_i min(jar_i, 0)^2,
 *         jar = J a - aref                                     (Eq. 5, with the
 *         cone term read as four one-sided pyramid rows per contact and
 *         D = R^-1 of Eq. 4)
 *   found by Newton steps on the stationarity residual
 *         r(a) = M a - qfrc + J^T f,  f = D . min(jar, 0)      (Eqs. 6, 8)
 *   with H = M + J^T diag(D . [jar < 0]) J                     (Eq. 9)
 *   and an exact line search on the piecewise-quadratic cost   (Eq. 10).
 *   Adjoint at the returned a, with F_a = H (symmetric)        (Eq. 17):
 *         H w = g,  dL/dqfrc = w,  dL/daref = D_act . (J w),
 *         dL/dJ = -(f w^T + (D_act . J w) a^T),
 *   and, from the *_theta entry points, dL/dM = -(w a^T + a w^T)/2 and
 *         dL/dD = -(J w) . min(jar, 0).
 *
 * Conventions shared by every entry point:
 *  - All float data are IEEE binary32, row-major, packed per instance at the
 *    element offsets of the instance table (cs_inst).  M is nv x nv and must be
 *    symmetric positive definite; J is m x nv (rows grouped four per contact);
 *    nv-vectors (qfrc, a, g, dqfrc, a_lo) sit at off_v; m-vectors (aref, D,
 *    daref, act) at off_r; dJ uses J's layout.  Offsets that are multiples of
 *    4 elements let the kernels use 16-byte loads; any offset is accepted.
 *  - Pointers marked "device" must be CUDA device (or managed) memory on the
 *    current device; the caller owns every buffer it passes and keeps it alive
 *    until the work on `stream` has completed.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *    asynchronous: they validate on the host, enqueue kernels and return;
 *    outputs are valid once the stream has been synchronised.
 *  - Return codes are CS_OK (0) or a negative CS_E* code; nothing is thrown
 *    across the ABI.  cs_last_error() describes the last failure of the
 *    calling thread.  Per-instance numerical outcomes (CS_ST_*) are written to
 *    the status array, never returned.
 *  - Supported sizes: 1 <= nv <= 128 and 0 <= m <= 1024 per instance.  Up to
 *    nv = 32 and m = 256 one warp solves an instance; beyond, one 256-thread
 *    CTA does, and nv_max x m_max must then fit one CTA's shared memory
 *    (about nv_max * (2 nv_max + m_max) * 4 bytes; checked, CS_EUNSUPPORTED
 *    otherwise).  An instance outside the batch's bounds gets
 *    CS_ST_BADSHAPE.
 */
#ifndef CONTACT_SOLVE_H
#define CONTACT_SOLVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes -------------------------------------------------------- */
#define CS_OK 0
#define CS_EINVAL (-1)       /* bad argument, shape or pointer */
#define CS_ECUDA (-2)        /* CUDA runtime error (cs_last_error has text) */
#define CS_ENOMEM (-3)       /* device or host allocation failed */
#define CS_EBUSY (-4)        /* serving: no free slot or arena bytes now */
#define CS_ENOTFOUND (-5)    /* serving: unknown or already collected ticket */
#define CS_EUNSUPPORTED (-6) /* sizes beyond the compiled kernels */
#define CS_PENDING 1         /* serving: result not ready yet */

/* ---- per-instance status (written to the status array) ------------------ */
#define CS_ST_OK 0         /* converged (residual or step test) */
#define CS_ST_MAXITER 1    /* Newton step cap max_iter reached */
#define CS_ST_CHOLFAIL 2   /* non-positive pivot in a Cholesky factor */
#define CS_ST_NONFINITE 3  /* NaN or Inf in the residual */
#define CS_ST_BADSHAPE 4   /* nv/m outside the supported range, or offsets
                              outside the batch totals */
#define CS_ST_NOPROGRESS 5 /* the Newton direction was not a descent one */
#define CS_ST_FAILED 6     /* serving: the request's batch failed to launch
                              or transfer (the error is counted in
                              cs_serve_stats.failed_launches) */
#define CS_ST_TIMEOUT 7    /* serving: the request waited in the queue longer
                              than cs_serve_config.queue_timeout_ms and was
                              not run (counted in cs_serve_stats.timed_out) */

/* One instance of a ragged batch (40 bytes).  Offsets are in elements. */
typedef struct cs_inst {
  int32_t nv;    /* degrees of freedom */
  int32_t m;     /* constraint rows, 4 per contact */
  int64_t off_M; /* M (nv*nv) in cs_batch.M; factor slot in cs_state.L */
  int64_t off_J; /* J (m*nv) in cs_batch.J; dJ in the output */
  int64_t off_v; /* nv-vectors: qfrc, g, a, a_lo, dqfrc */
  int64_t off_r; /* m-vectors: aref, D, daref, act */
} cs_inst;

/* A ragged batch.  inst and the five data arrays are device pointers.  The
 * totals are the element counts of the arrays; every instance's block must
 * lie inside them (checked on the device, CS_ST_BADSHAPE otherwise).
 * nv_max and m_max are host-side bounds over the batch (they pick the
 * kernel); an instance above them is marked CS_ST_BADSHAPE. */
typedef struct cs_batch {
  int32_t n;             /* number of instances (0 is a no-op) */
  int32_t nv_max;        /* max nv over the batch, 1..128 */
  int32_t m_max;         /* max m over the batch, 0..1024 */
  int32_t reserved;
  const cs_inst* inst;   /* device, n entries */
  const float* M;        /* device */
  const float* J;        /* device */
  const float* qfrc;     /* device */
  const float* aref;     /* device */
  const float* D;        /* device, entries > 0 */
  int64_t total_M, total_J, total_v, total_r;
} cs_batch;

/* Solver options. */
typedef struct cs_options {
  float tol;           /* stop when ||r||_inf <= tol * max(1,|qfrc|,|Ma|,|J^T f|) */
  int32_t max_iter;    /* Newton step cap K (>= 0; 0 returns a0) */
  int32_t keep_factor; /* fwd: 1 = store the Cholesky factor of H(a*) for the
                          adjoint; 0 = store only a*, a_lo and the active set
                          and refactor in the adjoint (less memory) */
  int32_t warps_per_block; /* 0 = library choice (autotuned), else 1..8 */
} cs_options;

/* Adjoint state written by cs_solve_fwd and read by cs_solve_adjoint.  All
 * arrays are caller-allocated device memory laid out like the batch.  Its
 * size does not depend on the number of Newton iterations. */
typedef struct cs_state {
  float* a_lo;     /* device, total_v: low part of a* (a* = a + a_lo) */
  uint8_t* act;    /* device, total_r: active set at a* (1 = jar < 0) */
  float* L;        /* device, total_M: packed lower rows of chol(H(a*)),
                      nv(nv+1)/2 per instance at off_M; may be NULL when
                      keep_factor == 0 */
  int32_t* status; /* device, n: CS_ST_* */
  int32_t* iters;  /* device, n: Newton steps taken */
} cs_state;

/* Library version (major*10000 + minor*100 + patch). */
int cs_version(void);

/* Text for a CS_* return code. */
const char* cs_strerror(int code);

/* Text of the calling thread's last failure ("" if none). */
const char* cs_last_error(void);

/* Forward solve (Eqs. 1, 5-10).  Writes a (device, total_v) and the adjoint
 * state.  Returns CS_EINVAL for a NULL/inconsistent argument, CS_ECUDA on a
 * launch failure.
 *
 * Accuracy and stopping (FP32 with compensated residuals): an instance
 * returns CS_ST_OK when ||r|| <= tol * scale, or, once its active set has
 * settled, when the Newton correction it would take next, or the error the
 * refinement step just taken is predicted to leave (from the ratio of
 * consecutive corrections), is within 1e-7 max|a| and moves no active force
 * by more than 1e-6 max|f|.  a then lies within about 1e-6 (relative, max
 * norm) of the exact minimiser; the adjoints refine w to 1e-5 and lambda to
 * 3e-5 the same way.  The forces f behind dJ and dD are the forward's own in
 * cs_solve_fused, re-evaluated at the returned a in cs_solve_adjoint: with
 * keep_factor == 1 the two paths agree bit for bit in a, dqfrc and daref and
 * to rounding in dJ and dD (with keep_factor == 0, a agrees bit for bit and
 * the gradients to the refinement's accuracy). */
int cs_solve_fwd(const cs_batch* batch, const cs_options* opt, float* a,
                 const cs_state* state, void* stream);

/* IFT adjoint (Eq. 17) at the state left by cs_solve_fwd for the same batch
 * and the same a.  g (device, total_v) is dL/da.  Writes dqfrc (total_v),
 * daref (total_r) and dJ (total_J), all device.  With keep_factor == 0 (or
 * state->L == NULL) the factor is rebuilt from the stored active set. */
int cs_solve_adjoint(const cs_batch* batch, const cs_options* opt,
                     const float* a, const cs_state* state, const float* g,
                     float* dqfrc, float* daref, float* dJ, void* stream);

/* ---- library-owned adjoint state --------------------------------------- */

/* The same state, allocated and owned by the library: a cs_state whose five
 * arrays are device memory the library allocated for one batch shape (the
 * batch's totals and n, and keep_factor: the factor array is allocated only
 * when it is 1).  It is used with cs_solve_fwd / cs_solve_adjoint like a
 * caller-built one, and released with cs_state_free.  Creation allocates
 * device memory (cudaMalloc) and synchronises nothing.  Returns CS_EINVAL for
 * a NULL or inconsistent argument (out is then NULL), CS_ENOMEM when the
 * device memory is not available. */
int cs_state_create(const cs_batch* batch, int32_t keep_factor, cs_state** out);

/* Forward solve into a library-owned state: when *st is NULL a state for
 * this batch (and opt->keep_factor) is created first and returned in *st;
 * otherwise *st must be a state from cs_state_create (or from an earlier
 * call) made for a batch of the same totals and n, and with a factor array
 * when opt->keep_factor is 1 (CS_EINVAL otherwise).  Then as cs_solve_fwd.
 * A state this call created is freed again if the launch fails. */
int cs_solve_fwd_alloc(const cs_batch* batch, const cs_options* opt, float* a,
                       cs_state** st, void* stream);

/* Copy the per-instance status (CS_ST_*) and Newton step counts of a
 * library-owned state into caller buffers (device, n entries each; either
 * may be NULL), asynchronously on `stream`.  They are valid once the forward
 * that wrote the state and this copy have completed.  CS_EINVAL for a state
 * that cs_state_create did not make. */
int cs_state_status(const cs_state* st, int32_t* status, int32_t* iters,
                    void* stream);

/* Free a library-owned state (after the work that uses it has completed).
 * NULL, and a pointer that cs_state_create did not return, are ignored. */
void cs_state_free(cs_state* st);

/* ---- the remaining parameters of Eq. 17: M and D ---------------------- */

/* cs_solve_adjoint that also writes the gradients with respect to M and D
 * (Eq. 17 with theta = M, D: F_M = (delta-row) a^T, F_D,i = J_i^T min(jar_i,0)):
 *   dM (device, total_M, M's layout): -(w a^T + a w^T) / 2, the gradient with
 *      respect to a symmetric M (the kernels read only M's lower triangle, so
 *      M is a symmetric parameter; the symmetric part of -w a^T is its
 *      gradient);
 *   dD (device, total_r): -(J w)_i min(jar_i, 0), zero on inactive rows.
 * Either may be NULL to skip it; with both NULL this is cs_solve_adjoint.
 * Errors as for cs_solve_adjoint. */
int cs_solve_adjoint_theta(const cs_batch* batch, const cs_options* opt,
                           const float* a, const cs_state* state,
                           const float* g, float* dqfrc, float* daref,
                           float* dJ, float* dM, float* dD, void* stream);

/* Bytes of device workspace cs_solve_fused needs for n instances. */
size_t cs_fused_workspace_bytes(int32_t n);

/* Fused forward + adjoint for a known cotangent g: one persistent launch
 * whose warps claim instances from a work counter kept in `workspace`
 * (device, >= cs_fused_workspace_bytes(n) bytes, 16-byte aligned; the call
 * resets the counter on `stream` first).  `order` (device, n entries, or
 * NULL for 0..n-1) is the claim order.  Writes a, dqfrc, daref, dJ (device)
 * and status, iters (device, n).  Nothing is kept between the two halves in
 * global memory. */
int cs_solve_fused(const cs_batch* batch, const cs_options* opt,
                   const float* g, const int32_t* order, float* a,
                   float* dqfrc, float* daref, float* dJ, int32_t* status,
                   int32_t* iters, void* workspace, size_t workspace_bytes,
                   void* stream);

/* cs_solve_fused with the nonlinear conjugate-gradient forward solver, the
 * other iteration MJX offers for the same objective (Section III-B): search
 * directions preconditioned by M^-1 with the Polak-Ribiere+ beta (clipped
 * at zero, and restarted from the preconditioned residual whenever the
 * conjugated direction is not a descent direction) and the exact line search
 * of Eq. 10; opt->max_iter caps the CG steps (many more than Newton needs).
 * The adjoint is the same IFT rule at the returned point (Eq. 17): it does
 * not depend on the path taken to a* (Eq. 14).  One warp per instance only
 * (nv_max <= 32, m_max <= 256), CS_EUNSUPPORTED otherwise; arguments and
 * errors as for cs_solve_fused. */
int cs_solve_fused_ncg(const cs_batch* batch, const cs_options* opt,
                       const float* g, const int32_t* order, float* a,
                       float* dqfrc, float* daref, float* dJ, int32_t* status,
                       int32_t* iters, void* workspace, size_t workspace_bytes,
                       void* stream);

/* cs_solve_fused that also writes dM and dD as cs_solve_adjoint_theta does
 * (either may be NULL). */
int cs_solve_fused_theta(const cs_batch* batch, const cs_options* opt,
                         const float* g, const int32_t* order, float* a,
                         float* dqfrc, float* daref, float* dJ, float* dM,
                         float* dD, int32_t* status, int32_t* iters,
                         void* workspace, size_t workspace_bytes,
                         void* stream);

/* ---- fused solve without any allocation ------------------------------- */

/* Instances cs_solve_fused_static can take in one call. */
#define CS_STATIC_MAX_INSTANCES (1 << 20)

/* cs_solve_fused for callers that cannot allocate device memory: processes
 * that may not call cudaMalloc (a host framework owns a fixed pool, or
 * allocation is forbidden where the call is made) and so cannot provide the
 * scratch workspace cs_solve_fused takes.  The paper has no counterpart; this
 * is a deployment variant of the same fused kernel.
 *
 * Scratch (the claim counter and the claim order) lives in a static device
 * array inside the library: about 4 MiB, held on every GPU that loads the
 * library until the process exits.  The call allocates nothing (no cudaMalloc,
 * cudaFree or allocating library routine).  The caller still passes every
 * input and output, as for cs_solve_fused.  inst_host (a host copy of the
 * instance table, or NULL) orders the claims by decreasing cost; with NULL
 * the instances are claimed in index order.
 *
 * Limits and sharing: n above CS_STATIC_MAX_INSTANCES returns
 * CS_EUNSUPPORTED.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) and caches it for the life of the process;
 * make that first call before any stream capture, and do not reset the
 * device (cudaDeviceReset) after it, which would leave the cached address
 * stale.  With inst_host != NULL the call uploads the claim order from a
 * host array that lives only for the call, so it returns CS_EUNSUPPORTED on
 * a stream that is being captured (index-order claims, inst_host = NULL, do
 * not upload anything).  Every call shares the one array and resets the
 * counter itself; calls whose work overlaps on the GPU (different streams,
 * or different host threads) race on it and must be serialised by the
 * caller. */
int cs_solve_fused_static(const cs_batch* batch, const cs_options* opt,
                          const float* g, const cs_inst* inst_host, float* a,
                          float* dqfrc, float* daref, float* dJ,
                          int32_t* status, int32_t* iters, void* stream);

/* ---- execution plans (fused path) ------------------------------------- */

/* Plan flags. */
#define CS_PLAN_AUTOTUNE 1 /* time warps-per-block candidates per bucket */
#define CS_PLAN_GRAPH 2    /* capture the launch as one CUDA graph */

typedef struct cs_plan cs_plan; /* opaque, owned by the library */

/* What a plan launches. */
typedef struct cs_plan_info {
  int32_t n_kernels;          /* one kernel per (nv bucket, rows per lane) */
  int32_t graph;              /* 1 if launched as a CUDA graph */
  int32_t nv_bucket[8];
  int32_t rows_per_lane[8];   /* m <= 32 * rows_per_lane */
  int32_t instances[8];
  int32_t warps_per_block[8];
  float tuned_ms[8];          /* autotuned time of the bucket alone (0 if not) */
  int32_t cta[8];             /* 1: one CTA per instance (nv_bucket = its max nv,
                                 rows_per_lane = rows per thread) */
} cs_plan_info;

/* Make a plan for the fused forward + adjoint (the work of cs_solve_fused)
 * on one batch and one set of output buffers, all of which must outlive the
 * plan.  inst_host is a host copy of batch->inst (read during the call only)
 * used to bucket instances by (nv, m) and to order each bucket's claims by
 * decreasing cost.  flags: CS_PLAN_AUTOTUNE times warps-per-block candidates
 * on this data (this runs the solve; outputs are overwritten) unless
 * opt->warps_per_block is set; CS_PLAN_GRAPH captures the bucket kernels as
 * parallel branches of one CUDA graph.  The plan allocates its own device
 * buffers (claim orders and counters).  Synchronises `stream` once.
 * Returns CS_EINVAL, CS_ENOMEM, CS_ECUDA or CS_EUNSUPPORTED on failure (then
 * *out is NULL). */
int cs_plan_create_fused(const cs_batch* batch, const cs_options* opt,
                         const cs_inst* inst_host, const float* g, float* a,
                         float* dqfrc, float* daref, float* dJ, int32_t* status,
                         int32_t* iters, int32_t flags, void* stream,
                         cs_plan** out);

/* cs_plan_create_fused whose launches also write dM and dD as
 * cs_solve_adjoint_theta does (either may be NULL). */
int cs_plan_create_fused_theta(const cs_batch* batch, const cs_options* opt,
                               const cs_inst* inst_host, const float* g,
                               float* a, float* dqfrc, float* daref, float* dJ,
                               float* dM, float* dD, int32_t* status,
                               int32_t* iters, int32_t flags, void* stream,
                               cs_plan** out);

/* Enqueue the plan's work on `stream` (one graph launch, or the bucket
 * kernels in order).  Launches of one plan on different streams must not
 * overlap in time: they share the claim counters. */
int cs_plan_launch(cs_plan* plan, void* stream);

/* Describe the plan's kernels. */
int cs_plan_describe(const cs_plan* plan, cs_plan_info* info);

/* Free the plan (after its last launch has completed). */
void cs_plan_destroy(cs_plan* plan);

/* Autotuner cache, one line per (device, nv bucket, rows per lane):
 * "device nv_bucket rows_per_lane warps_per_block ms".  dump writes at most
 * len-1 characters (NUL-terminated) and returns the full length; load parses
 * such text and returns the number of entries taken. */
int cs_autotune_cache_dump(char* buf, size_t len);
int cs_autotune_cache_load(const char* text);

/* ---- MuJoCo's round Coulomb cone --------------------------------------- */

/* cs_solve_fused with the round cone the paper keeps (Eq. 2) instead of
 * pyramid rows.  Each contact c owns three rows of J, aref and D: 3c (normal)
 * and 3c+1, 3c+2 (tangents); every instance's m must be a multiple of 3
 * (CS_ST_BADSHAPE otherwise).  Its cost is the weighted distance of
 * u = J a - aref to the dual cone (Eqs. 3-5),
 *   s_c(u) = min over z_N >= mu_c |z_T| of 1/2 (u - z)^T diag(D_N, D_T, D_T) (u - z),
 * with D_N = D[3c], D_T = D[3c+1] (one tangential stiffness; D[3c+2] is not
 * read) and mu_c = mu[3c] (mu: device, total_r floats laid out like D; only
 * the normal rows are read).  The solve is Newton on r = M a - qfrc +
 * J^T grad s with H = M + sum_c J_c^T hess_c J_c and an exact line search on
 * the convex phi(alpha); the adjoint (Eq. 17) at the returned a writes
 * dqfrc = w, daref = hess (J w) per contact, dJ = -(grad s w^T + daref a^T)
 * and, where non-NULL, dM (symmetric M, as cs_solve_fused_theta), dD
 * (dL/dD_N on row 3c, dL/dD_T on row 3c+1, 0 on 3c+2) and dmu (dL/dmu_c on
 * row 3c, 0 on the tangent rows).  Sizes: nv_max <= 128 and m_max <= 1024,
 * one warp per instance up to nv_max = 32 and m_max = 256 and one 256-thread
 * CTA per instance beyond (CS_EUNSUPPORTED when one CTA's shared memory cannot
 * hold an instance).  Workspace, order and errors as for cs_solve_fused. */
int cs_solve_fused_elliptic(const cs_batch* batch, const cs_options* opt,
                            const float* mu, const float* g,
                            const int32_t* order, float* a, float* dqfrc,
                            float* daref, float* dJ, float* dM, float* dD,
                            float* dmu, int32_t* status, int32_t* iters,
                            void* workspace, size_t workspace_bytes,
                            void* stream);

/* ---- unrolled differentiation (the paper's comparison) ---------------- */

/* The sensitivity the paper sets against the IFT adjoint (Section III-E):
 * reverse-mode differentiation of the executed trace of at most K Newton
 * steps.  cs_unrolled_fwd runs the solve from a0 = M^-1 qfrc (Eq. 1) for at
 * most K = opt->max_iter steps (Eqs. 6-10; stopping early on the residual
 * test, a non-descent direction, or an exact step that crosses no
 * breakpoint) and records each step in `trace` and `tmask`;
 * cs_unrolled_bwd propagates g = dL/da_K back through the recorded steps and
 * writes dL/dqfrc, dL/daref, dL/dJ, dL/dM (symmetric M, as the *_theta entry
 * points) and dL/dD.  Run to convergence this equals the IFT adjoint; for a
 * truncated solve it is the derivative of the truncated map.
 *
 * Memory: the trace holds, per step, the factor of H_k, a_k and p_k (float
 * pairs), alpha_k and c1_k (cs_unrolled_trace_floats(batch, K) floats: K x
 * (total_M + 4 total_v + 2 n)) and the masks S_k, T_k
 * (cs_unrolled_mask_bytes(batch, K) bytes: K x total_r), so it grows
 * linearly with K, unlike cs_state.
 *
 * Sizes: nv_max <= 128 and m_max <= 1024, one warp per instance up to
 * nv_max = 32 and m_max = 256 and one 256-thread CTA per instance beyond
 * (CS_EUNSUPPORTED when one CTA's shared memory cannot hold an instance and
 * its slots: M, the factor, J and 26 nv-vectors).  All pointers are device
 * memory; `a`,
 * `status` and `iters` are written by the forward and read by the
 * backward (same batch, same options).  cs_unrolled_bwd uses dJ and dM as
 * accumulators; every output must be non-NULL (daref, dJ, dD may be NULL
 * only when m_max == 0).  Errors as for cs_solve_fwd. */
size_t cs_unrolled_trace_floats(const cs_batch* batch, int32_t K);
size_t cs_unrolled_mask_bytes(const cs_batch* batch, int32_t K);
int cs_unrolled_fwd(const cs_batch* batch, const cs_options* opt, float* a,
                    float* trace, uint8_t* tmask, int32_t* status,
                    int32_t* iters, void* stream);
int cs_unrolled_bwd(const cs_batch* batch, const cs_options* opt,
                    const float* a, const float* trace, const uint8_t* tmask,
                    int32_t* status, const int32_t* iters, const float* g,
                    float* dqfrc, float* daref, float* dJ, float* dM,
                    float* dD, void* stream);

/* ---- serving: continuous batching ------------------------------------ */

#define CS_SERVE_CONTINUOUS 0 /* admit queued requests whenever a slot frees */
#define CS_SERVE_FIXED 1      /* launch only batches of fixed_batch requests */

/* Server configuration.  The device arena (arena_bytes) is split evenly over
 * `streams` slots; each slot holds one batch in flight (inputs, outputs,
 * tables), so a batch admits requests while they fit its slot's bytes
 * (admission by device memory) and up to max_batch of them.  Several slots
 * in flight on their own streams let later batches overlap earlier ones on
 * the device.  Under CS_SERVE_CONTINUOUS a batch holds one kernel kind
 * (instances one warp solves, or instances one CTA solves), taken in arrival
 * order within the kind.  tol / max_iter as in cs_options.  max_queue bounds the host
 * queue (0 = 2^20). */
typedef struct cs_serve_config {
  size_t arena_bytes;  /* >= 1 MiB per stream */
  int32_t streams;     /* 1..16 */
  int32_t max_batch;   /* >= 1 */
  int32_t policy;      /* CS_SERVE_CONTINUOUS or CS_SERVE_FIXED */
  int32_t fixed_batch; /* batch size of CS_SERVE_FIXED */
  float tol;
  int32_t max_iter;
  int32_t max_queue;
  int32_t queue_timeout_ms; /* > 0: a request still queued (not yet admitted
                               to a batch) this long after its submission is
                               completed with CS_ST_TIMEOUT; 0 = no limit */
} cs_serve_config;

/* One request: a forward solve followed by the IFT adjoint for g.  All
 * pointers are HOST memory, read during cs_serve_submit only (the data are
 * copied).  Layouts as for one instance of a batch (row-major M, J). */
typedef struct cs_request {
  int32_t nv, m;
  const float *M, *J, *qfrc, *aref, *D, *g;
} cs_request;

/* Result of a request.  The caller provides the host output buffers (nv,
 * nv, m, m*nv floats; any may be NULL to skip it).  Times are seconds of one
 * steady clock: submission, launch of its batch, completion seen by the
 * server. */
typedef struct cs_result {
  float *a, *dqfrc, *daref, *dJ;
  int32_t status, iters;
  double t_submit, t_start, t_done;
} cs_result;

typedef struct cs_serve_stats {
  int64_t submitted, completed, batches, batched_requests, queued;
  int32_t max_inflight;    /* most batches on the GPU at once */
  int32_t failed_launches; /* batches whose copy, launch or completion failed */
  int64_t timed_out;       /* requests completed with CS_ST_TIMEOUT */
} cs_serve_stats;

typedef struct cs_server cs_server; /* opaque, owned by the library */

/* Create a server on the current device: allocates the arena and pinned
 * staging, starts the scheduler thread.  CS_EINVAL / CS_ENOMEM on failure. */
int cs_serve_create(const cs_serve_config* cfg, cs_server** out);

/* Queue a request (its data are copied); *ticket identifies it.  Returns
 * CS_EUNSUPPORTED for sizes no kernel or slot can take, CS_EBUSY when the
 * queue is full.  Never blocks on the GPU. */
int cs_serve_submit(cs_server* srv, const cs_request* req, uint64_t* ticket);

/* CS_PENDING while the request is queued or on the GPU; CS_OK once done
 * (outputs copied to res, the ticket is then retired); CS_ENOTFOUND for an
 * unknown or retired ticket.  Never blocks. */
int cs_serve_poll(cs_server* srv, uint64_t ticket, cs_result* res);

/* Bulk forms for high-rate clients.  submit_batch queues reqs[0..n) in
 * order and returns how many were queued (n, or fewer if one failed; a
 * negative code if the first failed).  poll_batch polls each ticket whose
 * done[i] is not already 1 (done is in/out, start it at 0) and sets done[i] =
 * 1 (result in res[i], ticket retired), 0 (pending) or -1 (unknown); it
 * returns the number completed in this call. */
int cs_serve_submit_batch(cs_server* srv, int32_t n, const cs_request* reqs,
                          uint64_t* tickets);
int cs_serve_poll_batch(cs_server* srv, int32_t n, const uint64_t* tickets,
                        cs_result* res, int32_t* done);

/* The server's clock (seconds, steady; the clock of cs_result's t_submit,
 * t_start and t_done). */
double cs_serve_clock(void);

/* A load generator for measurements, run in the calling thread: reqs[i]
 * (host data, copied at submission as by cs_serve_submit) is submitted once
 * cs_serve_clock() reaches t0 + t_arrival[i] (seconds, ascending), the ones
 * due together in one bulk call; tickets[i] receives its ticket.  The thread
 * sleeps while the next arrival is more than 150 us away and yields closer
 * to it, so the submission lags the schedule by microseconds rather than by
 * an interpreter's scheduling.  A full queue (CS_EBUSY) is retried; any
 * other failure ends the replay.  Returns the number queued (n unless a
 * submission failed), or the first failure's code if none was queued;
 * CS_EINVAL for NULL arrays with n > 0. */
int cs_serve_replay(cs_server* srv, int32_t n, const cs_request* reqs,
                    const double* t_arrival, double t0, uint64_t* tickets);

/* Tickets whose requests completed since the previous call, in completion
 * order (at most max of them, written to tickets); returns their number.
 * A client that holds many outstanding tickets collects exactly these with
 * cs_serve_poll_batch instead of scanning every outstanding one.  Each
 * completion is reported once. */
int cs_serve_completed(cs_server* srv, int32_t max, uint64_t* tickets);

/* Drop a request that is still queued (CS_EBUSY once it is on the GPU). */
int cs_serve_cancel(cs_server* srv, uint64_t ticket);

/* CS_SERVE_FIXED: release the queued requests as a partial batch. */
int cs_serve_flush(cs_server* srv);

int cs_serve_get_stats(cs_server* srv, cs_serve_stats* stats);

/* Stop admitting, wait for the batches in flight, free everything. */
void cs_serve_destroy(cs_server* srv);

/* Host-side fault injection, for testing how a server handles failures
 * without making the device fail.  Before each step of a batch the
 * scheduler calls hook(stage, batch, user), batch numbering the batches in
 * the order they are launched from 0; a nonzero return makes that step fail
 * as if the runtime call had failed (the step is not issued), so the batch's
 * requests complete with CS_ST_FAILED, cs_serve_stats.failed_launches counts
 * it, and its slot is reused.  Stages: */
#define CS_SERVE_FAULT_H2D 0      /* the batch's input copy */
#define CS_SERVE_FAULT_LAUNCH 1   /* each bucket kernel launch */
#define CS_SERVE_FAULT_D2H 2      /* the batch's output copy */
#define CS_SERVE_FAULT_COMPLETE 3 /* the completion the event reports */
typedef int (*cs_serve_fault_fn)(int stage, int64_t batch, void* user);

/* Install (or, with NULL, remove) the hook.  It is called from the
 * scheduler's thread and must not call back into the server. */
int cs_serve_set_fault_hook(cs_server* srv, cs_serve_fault_fn hook, void* user);

#ifdef __cplusplus
}
#endif

#endif /* CONTACT_SOLVE_H */
