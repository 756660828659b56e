/*
 * cs_oracle.c -- plain FP64 CPU oracle for the regularised smooth-contact solve
 * and its implicit-function-theorem adjoint.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA path; the two meet only in the seeded
 * input generators.
 *
 * What it computes (per instance, Section III of the paper):
 *   a0   = M^-1 qfrc                                  (Eq. 1, qfrc = tau - c)
 *   L(a) = 1/2 (a-a0)^T M (a-a0) + 1/2 sum_i D_i min(jar_i,0)^2,
 *          jar = J a - aref                           (Eq. 5, pyramidal rows,
 *                                                      D = R^-1 of Eq. 4)
 *   r(a) = M a - qfrc + J^T f,  f = D . min(jar,0)    (Eqs. 6 and 8)
 *   H(a) = M + J^T diag(D . [jar<0]) J                (Eq. 9)
 *   Newton: p = -H^-1 r, a <- a + alpha p             (Eq. 10), alpha from an
 *   exact search of the convex piecewise-quadratic phi(alpha) = L(a+alpha p).
 *   Adjoint at the returned a (Eq. 17 with F_a = H symmetric):
 *     H w = g;  dL/dqfrc = w;  dL/daref = D_act . (J w);
 *     dL/dJ = -(f w^T + (D_act . J w) a^T).
 *
 * Everything is written out plainly in double precision: dense unblocked
 * Cholesky, explicit loops, qsort for the line-search breakpoints.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum {
  OR_OK = 0,          /* ||r||_inf <= tol * scale, or exact termination */
  OR_MAXITER = 1,     /* Newton step cap reached */
  OR_CHOLFAIL = 2,    /* non-positive pivot */
  OR_NONFINITE = 3,   /* NaN/Inf met */
  OR_BADSHAPE = 4,    /* nv < 1 or m < 0 */
  OR_NOPROGRESS = 5   /* p^T r >= 0: no descent direction */
};

/* ---- dense helpers ------------------------------------------------------ */

/* In-place Cholesky of the n x n row-major SPD matrix A (lower triangle used
 * and overwritten by L, upper triangle zeroed).  Returns 0, or -1 on a
 * non-positive pivot. */
static int chol(int n, double *A) {
  for (int j = 0; j < n; ++j) {
    double d = A[j * n + j];
    for (int k = 0; k < j; ++k) d -= A[j * n + k] * A[j * n + k];
    if (!(d > 0.0)) return -1;
    double ljj = sqrt(d);
    A[j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double s = A[i * n + j];
      for (int k = 0; k < j; ++k) s -= A[i * n + k] * A[j * n + k];
      A[i * n + j] = s / ljj;
    }
    for (int k = j + 1; k < n; ++k) A[j * n + k] = 0.0;
  }
  return 0;
}

/* x <- (L L^T)^-1 x. */
static void chol_solve(int n, const double *L, double *x) {
  for (int i = 0; i < n; ++i) {
    double s = x[i];
    for (int k = 0; k < i; ++k) s -= L[i * n + k] * x[k];
    x[i] = s / L[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = x[i];
    for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * x[k];
    x[i] = s / L[i * n + i];
  }
}

static double inf_norm(int n, const double *x) {
  double v = 0.0;
  for (int i = 0; i < n; ++i) {
    double a = fabs(x[i]);
    if (a > v || a != a) v = a;
  }
  return v;
}

/* ---- problem pieces ----------------------------------------------------- */

typedef struct {
  int nv, m;
  const double *M, *J, *qfrc, *aref, *D;
} problem;

/* jar = J a - aref, act = [jar < 0], f = D . min(jar, 0),
 * Ma = M a, Jtf = J^T f, r = Ma - qfrc + Jtf (Eqs. 6 and 8).
 * Returns the scale max(1, |qfrc|, |Ma|, |Jtf|) used by the stopping test. */
static double residual(const problem *P, const double *a, double *jar,
                       uint8_t *act, double *f, double *Ma, double *Jtf,
                       double *r) {
  const int nv = P->nv, m = P->m;
  for (int i = 0; i < m; ++i) {
    double s = 0.0;
    for (int k = 0; k < nv; ++k) s += P->J[i * nv + k] * a[k];
    jar[i] = s - P->aref[i];
    act[i] = jar[i] < 0.0;
    f[i] = act[i] ? P->D[i] * jar[i] : 0.0;
  }
  for (int j = 0; j < nv; ++j) {
    double s = 0.0;
    for (int k = 0; k < nv; ++k) s += P->M[j * nv + k] * a[k];
    Ma[j] = s;
    double t = 0.0;
    for (int i = 0; i < m; ++i) t += P->J[i * nv + j] * f[i];
    Jtf[j] = t;
    r[j] = Ma[j] - P->qfrc[j] + Jtf[j];
  }
  double scale = 1.0, v;
  if ((v = inf_norm(nv, P->qfrc)) > scale) scale = v;
  if ((v = inf_norm(nv, Ma)) > scale) scale = v;
  if ((v = inf_norm(nv, Jtf)) > scale) scale = v;
  return scale;
}

/* H = M + sum_{i active} D_i J_i^T J_i (Eq. 9), full symmetric. */
static void newton_matrix(const problem *P, const uint8_t *act, double *H) {
  const int nv = P->nv, m = P->m;
  memcpy(H, P->M, sizeof(double) * nv * nv);
  for (int i = 0; i < m; ++i) {
    if (!act[i]) continue;
    const double *Ji = P->J + (size_t)i * nv;
    for (int j = 0; j < nv; ++j)
      for (int k = 0; k < nv; ++k) H[j * nv + k] += P->D[i] * Ji[j] * Ji[k];
  }
}

typedef struct {
  double alpha;
  int row;
} breakpoint;

static int bp_cmp(const void *x, const void *y) {
  double a = ((const breakpoint *)x)->alpha, b = ((const breakpoint *)y)->alpha;
  return (a > b) - (a < b);
}

/* Exact minimiser of phi(alpha) = L(a + alpha p) over alpha > 0.
 *
 * phi'(alpha) = p^T (M (a + alpha p) - qfrc) + sum_i D_i s_i min(jar_i + alpha s_i, 0)
 * with s = J p.  phi' is continuous, piecewise linear and increasing (phi is
 * strongly convex along p because p^T M p > 0).  On each interval between
 * breakpoints alpha_i = -jar_i / s_i it equals c0 + c1 alpha, where the sums
 * run over the rows active on that interval.  The breakpoints are sorted and
 * swept in increasing order; the first interval that contains the root of
 * its line returns it. */
static double line_search(const problem *P, const double *a, const double *p,
                          const double *jar, const double *Ma, double *s,
                          breakpoint *bp) {
  const int nv = P->nv, m = P->m;
  double c0 = 0.0, c1 = 0.0;
  for (int j = 0; j < nv; ++j) {
    double Mp = 0.0;
    for (int k = 0; k < nv; ++k) Mp += P->M[j * nv + k] * p[k];
    c0 += p[j] * (Ma[j] - P->qfrc[j]);
    c1 += p[j] * Mp;
  }
  int nb = 0;
  for (int i = 0; i < m; ++i) {
    double si = 0.0;
    for (int k = 0; k < nv; ++k) si += P->J[i * nv + k] * p[k];
    s[i] = si;
    /* active just to the right of alpha = 0 */
    int on = jar[i] < 0.0 || (jar[i] == 0.0 && si < 0.0);
    if (on) {
      c0 += P->D[i] * si * jar[i];
      c1 += P->D[i] * si * si;
    }
    if (si != 0.0) {
      double al = -jar[i] / si;
      if (al > 0.0) {
        bp[nb].alpha = al;
        bp[nb].row = i;
        ++nb;
      }
    }
  }
  qsort(bp, nb, sizeof(breakpoint), bp_cmp);
  for (int q = 0; q < nb; ++q) {
    double root = -c0 / c1;
    if (root <= bp[q].alpha) return root;
    /* cross the breakpoint: row toggles */
    int i = bp[q].row;
    double sgn = (jar[i] < 0.0) ? -1.0 : 1.0; /* leaves if it was active */
    c0 += sgn * P->D[i] * s[i] * jar[i];
    c1 += sgn * P->D[i] * s[i] * s[i];
  }
  return -c0 / c1;
}

/* ---- public entry points ------------------------------------------------ */

/* Solve one instance.  a (out, nv) holds the returned acceleration; act (out,
 * m) its active set; *iters the Newton steps taken.  a_init may be NULL
 * (start at a0 = M^-1 qfrc) or a warm start.  Returns a status code. */
int oracle_solve(int nv, int m, const double *M, const double *J,
                 const double *qfrc, const double *aref, const double *D,
                 const double *a_init, double tol, int max_iter, double *a,
                 uint8_t *act, int *iters) {
  *iters = 0;
  if (nv < 1 || m < 0) return OR_BADSHAPE;
  problem P = {nv, m, M, J, qfrc, aref, D};
  size_t wd = (size_t)(6 * m + 6 * nv + 2 * nv * nv + 8);
  double *w = (double *)calloc(wd, sizeof(double));
  breakpoint *bp = (breakpoint *)calloc((size_t)m + 1, sizeof(breakpoint));
  uint8_t *act2 = (uint8_t *)calloc((size_t)m + 1, 1);
  double *jar = w, *f = jar + m, *s = f + m, *jar2 = s + m, *Ma = jar2 + m;
  double *Jtf = Ma + nv, *r = Jtf + nv, *p = r + nv, *an = p + nv;
  double *H = an + nv;
  int status = OR_MAXITER;

  if (a_init) {
    memcpy(a, a_init, sizeof(double) * nv);
  } else { /* a0 = M^-1 qfrc (Eq. 1) */
    memcpy(H, M, sizeof(double) * nv * nv);
    if (chol(nv, H)) { status = OR_CHOLFAIL; goto done; }
    memcpy(a, qfrc, sizeof(double) * nv);
    chol_solve(nv, H, a);
  }

  for (int k = 0;; ++k) {
    double scale = residual(&P, a, jar, act, f, Ma, Jtf, r);
    double rn = inf_norm(nv, r);
    if (!isfinite(rn) || !isfinite(scale)) { status = OR_NONFINITE; break; }
    if (rn <= tol * scale) { status = OR_OK; break; }
    if (k >= max_iter) { status = OR_MAXITER; break; }
    newton_matrix(&P, act, H);
    if (chol(nv, H)) { status = OR_CHOLFAIL; break; }
    for (int j = 0; j < nv; ++j) p[j] = -r[j];
    chol_solve(nv, H, p);
    double ptr = 0.0;
    for (int j = 0; j < nv; ++j) ptr += p[j] * r[j];
    if (!(ptr < 0.0)) { status = OR_NOPROGRESS; break; }
    /* Exact termination: if the full step keeps the active set, a + p is the
     * minimiser of the quadratic on that set and consistent with it, hence
     * the exact solution. */
    for (int j = 0; j < nv; ++j) an[j] = a[j] + p[j];
    int same = 1;
    for (int i = 0; i < m; ++i) {
      double v = 0.0;
      for (int q = 0; q < nv; ++q) v += J[i * nv + q] * an[q];
      jar2[i] = v - aref[i];
      act2[i] = jar2[i] < 0.0;
      if (act2[i] != act[i]) same = 0;
    }
    if (same) {
      memcpy(a, an, sizeof(double) * nv);
      *iters = k + 1;
      residual(&P, a, jar, act, f, Ma, Jtf, r);
      status = OR_OK;
      break;
    }
    double alpha = line_search(&P, a, p, jar, Ma, s, bp);
    for (int j = 0; j < nv; ++j) a[j] += alpha * p[j];
    *iters = k + 1;
  }
done:
  free(w);
  free(bp);
  free(act2);
  return status;
}

/* Adjoint at the returned a (Eq. 17): H(a) w = g with the active set of a,
 * then dqfrc = w, daref = D_act . (J w), dJ = -(f w^T + daref a^T).
 * act (out, m) receives the active set used.  Returns 0 or OR_CHOLFAIL. */
/* The remaining parameter terms of Eq. 17, for theta = M and theta = D:
 *   dF/dM_kj = delta_kj-row a_j           -> dL/dM = -w a^T, read here as a
 *     derivative with respect to a symmetric M (only the lower triangle is an
 *     input), i.e. its symmetric part -(w a^T + a w^T) / 2;
 *   dF/dD_i  = J_i^T min(jar_i, 0)       -> dL/dD_i = -(J w)_i min(jar_i, 0).
 * dM (nv*nv, row-major) and dD (m) may each be NULL. */
int oracle_adjoint_theta(int nv, int m, const double *M, const double *J,
                         const double *qfrc, const double *aref,
                         const double *D, const double *a, const double *g,
                         double *dqfrc, double *daref, double *dJ, double *dM,
                         double *dD, uint8_t *act) {
  if (nv < 1 || m < 0) return OR_BADSHAPE;
  problem P = {nv, m, M, J, qfrc, aref, D};
  double *w = (double *)calloc((size_t)(3 * m + 3 * nv + nv * nv + 8), sizeof(double));
  double *jar = w, *f = jar + m, *u = f + m, *Ma = u + m, *Jtf = Ma + nv;
  double *r = Jtf + nv, *H = r + nv;
  int status = 0;
  residual(&P, a, jar, act, f, Ma, Jtf, r);
  newton_matrix(&P, act, H);
  if (chol(nv, H)) { status = OR_CHOLFAIL; goto done; }
  memcpy(dqfrc, g, sizeof(double) * nv);
  chol_solve(nv, H, dqfrc);
  for (int i = 0; i < m; ++i) {
    double v = 0.0;
    for (int k = 0; k < nv; ++k) v += J[i * nv + k] * dqfrc[k];
    u[i] = v;
    daref[i] = act[i] ? D[i] * v : 0.0;
  }
  for (int i = 0; i < m; ++i)
    for (int k = 0; k < nv; ++k)
      dJ[i * nv + k] = -(f[i] * dqfrc[k] + daref[i] * a[k]);
  if (dM)
    for (int j = 0; j < nv; ++j)
      for (int k = 0; k < nv; ++k)
        dM[j * nv + k] = -0.5 * (dqfrc[j] * a[k] + a[j] * dqfrc[k]);
  if (dD)
    for (int i = 0; i < m; ++i) dD[i] = jar[i] < 0.0 ? -u[i] * jar[i] : 0.0;
done:
  free(w);
  return status;
}

/* IFT adjoint of Eq. 17 for theta = (qfrc, aref, J) at the point a. */
int oracle_adjoint(int nv, int m, const double *M, const double *J,
                   const double *qfrc, const double *aref, const double *D,
                   const double *a, const double *g, double *dqfrc,
                   double *daref, double *dJ, uint8_t *act) {
  return oracle_adjoint_theta(nv, m, M, J, qfrc, aref, D, a, g, dqfrc, daref,
                              dJ, NULL, NULL, act);
}

/* Residual r(a), forces f and active set at a given a (for invariants). */
double oracle_residual(int nv, int m, const double *M, const double *J,
                       const double *qfrc, const double *aref, const double *D,
                       const double *a, double *r, double *f, uint8_t *act) {
  problem P = {nv, m, M, J, qfrc, aref, D};
  double *w = (double *)calloc((size_t)(m + 2 * nv + 4), sizeof(double));
  double scale = residual(&P, a, w, act, f, w + m, w + m + nv, r);
  free(w);
  return scale;
}

/* Objective L(a) of Eq. 5 (pyramidal rows); a0 = M^-1 qfrc is recomputed. */
double oracle_objective(int nv, int m, const double *M, const double *J,
                        const double *qfrc, const double *aref, const double *D,
                        const double *a) {
  double *w = (double *)calloc((size_t)(nv * nv + 2 * nv + 4), sizeof(double));
  double *H = w, *a0 = H + nv * nv, *d = a0 + nv;
  memcpy(H, M, sizeof(double) * nv * nv);
  if (chol(nv, H)) { free(w); return NAN; }
  memcpy(a0, qfrc, sizeof(double) * nv);
  chol_solve(nv, H, a0);
  for (int j = 0; j < nv; ++j) d[j] = a[j] - a0[j];
  double v = 0.0;
  for (int j = 0; j < nv; ++j)
    for (int k = 0; k < nv; ++k) v += 0.5 * d[j] * M[j * nv + k] * d[k];
  for (int i = 0; i < m; ++i) {
    double s = 0.0;
    for (int k = 0; k < nv; ++k) s += J[i * nv + k] * a[k];
    s -= aref[i];
    if (s < 0.0) v += 0.5 * D[i] * s * s;
  }
  free(w);
  return v;
}

/* Batched forward + adjoint over instances [lo, hi) of a ragged batch laid out
 * like the C ABI (offsets in elements).  Inputs are float32 widened to double
 * by the caller.  Per instance: a, act, status, iters, dqfrc, daref, dJ.
 * g may be NULL (forward only). */
void oracle_batch(int lo, int hi, const int32_t *nv, const int32_t *m,
                  const int64_t *off_M, const int64_t *off_J,
                  const int64_t *off_v, const int64_t *off_r, const double *M,
                  const double *J, const double *qfrc, const double *aref,
                  const double *D, const double *g, double tol, int max_iter,
                  double *a, uint8_t *act, int32_t *status, int32_t *iters,
                  double *dqfrc, double *daref, double *dJ, double *dM,
                  double *dD) {
  for (int b = lo; b < hi; ++b) {
    int it = 0;
    const double *Mb = M + off_M[b], *Jb = J + off_J[b];
    status[b] = oracle_solve(nv[b], m[b], Mb, Jb, qfrc + off_v[b],
                             aref + off_r[b], D + off_r[b], NULL, tol, max_iter,
                             a + off_v[b], act + off_r[b], &it);
    iters[b] = it;
    if (g && status[b] != OR_BADSHAPE && status[b] != OR_CHOLFAIL &&
        status[b] != OR_NONFINITE) {
      int s2 = oracle_adjoint_theta(
          nv[b], m[b], Mb, Jb, qfrc + off_v[b], aref + off_r[b], D + off_r[b],
          a + off_v[b], g + off_v[b], dqfrc + off_v[b], daref + off_r[b],
          dJ + off_J[b], dM ? dM + off_M[b] : NULL, dD ? dD + off_r[b] : NULL,
          act + off_r[b]);
      if (s2) status[b] = s2;
    }
  }
}

/* ---- round (elliptic) Coulomb cone (Eqs. 2-5 as the paper states them) -- */

/* One contact c owns three rows: 3c (normal) and 3c+1, 3c+2 (tangents), with
 * u = J a - aref on those rows, D_N = D[3c], D_T = D[3c+1] (one tangential
 * regularisation for both tangent rows; D[3c+2] is not read) and
 * mu = mu[3c].  Its cost is the weighted distance of Eq. 5,
 *   s(u) = min over z in K* of 1/2 (u - z)^T diag(D_N, D_T, D_T) (u - z),
 *   K* = {z : z_N >= mu |z_T|}  (dual of the cone of Eq. 2, Eq. 3).
 * With x = diag(D)^(1/2) u the weighted distance is the Euclidean distance of
 * x to the second-order cone {x_N >= mu~ |x_T|}, mu~ = mu sqrt(D_N / D_T),
 * whose projection has three regions (t = |u_T|):
 *   zone 0 (u inside K*):          u_N >= mu t                      s = 0
 *   zone 2 (x in the polar cone):  mu D_N u_N + D_T t <= 0          s = 1/2 (D_N u_N^2 + D_T t^2)
 *   zone 1 (between):              phi = mu t - u_N > 0,            s = 1/2 Dm phi^2,
 *                                  Dm = D_N / (1 + mu^2 D_N / D_T).
 * Writes s, the gradient (3) and the Hessian (3x3 row-major) and returns the
 * zone.  In zone 1, grad = Dm phi (-1, mu uhat) with uhat = u_T / t and
 * hess = Dm [(-1, mu uhat)(-1, mu uhat)^T + phi mu / t (0 (+) (I - uhat uhat^T))]. */
static int ell_cone(const double *u, double DN, double DT, double mu, double *s,
                    double *grad, double *hess) {
  const double uN = u[0], u1 = u[1], u2 = u[2];
  const double t = sqrt(u1 * u1 + u2 * u2);
  for (int k = 0; k < 9; ++k) hess[k] = 0.0;
  if (uN >= mu * t) {
    *s = 0.0;
    grad[0] = grad[1] = grad[2] = 0.0;
    return 0;
  }
  if (mu * DN * uN + DT * t <= 0.0) {
    *s = 0.5 * (DN * uN * uN + DT * t * t);
    grad[0] = DN * uN;
    grad[1] = DT * u1;
    grad[2] = DT * u2;
    hess[0] = DN;
    hess[4] = DT;
    hess[8] = DT;
    return 2;
  }
  const double Dm = DN / (1.0 + mu * mu * DN / DT);
  const double phi = mu * t - uN;
  const double h1 = t > 0.0 ? u1 / t : 0.0, h2 = t > 0.0 ? u2 / t : 0.0;
  const double gv[3] = {-1.0, mu * h1, mu * h2};
  *s = 0.5 * Dm * phi * phi;
  for (int k = 0; k < 3; ++k) grad[k] = Dm * phi * gv[k];
  for (int j = 0; j < 3; ++j)
    for (int k = 0; k < 3; ++k) hess[3 * j + k] = Dm * gv[j] * gv[k];
  if (t > 0.0) {
    const double c = Dm * phi * mu / t;
    hess[4] += c * (1.0 - h1 * h1);
    hess[5] += c * (-h1 * h2);
    hess[7] += c * (-h2 * h1);
    hess[8] += c * (1.0 - h2 * h2);
  }
  return 1;
}

/* The cone pieces on their own, for pinning them: s, gradient, Hessian. */
int oracle_ell_cone(const double *u, double DN, double DT, double mu, double *s,
                    double *grad, double *hess) {
  return ell_cone(u, DN, DT, mu, s, grad, hess);
}

/* u = J a - aref, per-contact zone / gradient / Hessian block, Ma, J^T grad,
 * r = Ma - qfrc + J^T grad (Eq. 6 with s of the round cone).  Returns the
 * stopping scale max(1, |qfrc|, |Ma|, |J^T grad|); *cost += sum_c s_c. */
static double ell_residual(const problem *P, const double *mu, const double *a,
                           double *u, uint8_t *zone, double *grad,
                           double *hessb, double *Ma, double *Jtf, double *r,
                           double *cost) {
  const int nv = P->nv, m = P->m, nc = m / 3;
  for (int i = 0; i < m; ++i) {
    double v = 0.0;
    for (int k = 0; k < nv; ++k) v += P->J[i * nv + k] * a[k];
    u[i] = v - P->aref[i];
  }
  double sc = 0.0;
  for (int c = 0; c < nc; ++c) {
    double s;
    const int z = ell_cone(u + 3 * c, P->D[3 * c], P->D[3 * c + 1], mu[3 * c], &s,
                           grad + 3 * c, hessb + 9 * c);
    zone[3 * c] = zone[3 * c + 1] = zone[3 * c + 2] = (uint8_t)z;
    sc += s;
  }
  if (cost) *cost += sc;
  for (int j = 0; j < nv; ++j) {
    double v = 0.0, t = 0.0;
    for (int k = 0; k < nv; ++k) v += P->M[j * nv + k] * a[k];
    for (int i = 0; i < 3 * nc; ++i) t += P->J[i * nv + j] * grad[i];
    Ma[j] = v;
    Jtf[j] = t;
    r[j] = v - P->qfrc[j] + t;
  }
  double scale = 1.0, v;
  if ((v = inf_norm(nv, P->qfrc)) > scale) scale = v;
  if ((v = inf_norm(nv, Ma)) > scale) scale = v;
  if ((v = inf_norm(nv, Jtf)) > scale) scale = v;
  return scale;
}

/* H = M + sum_c J_c^T hess_c J_c (Eq. 9 with the block Hessians). */
static void ell_newton_matrix(const problem *P, const double *hessb, double *H) {
  const int nv = P->nv, nc = P->m / 3;
  memcpy(H, P->M, sizeof(double) * nv * nv);
  for (int c = 0; c < nc; ++c) {
    const double *Jc = P->J + (size_t)3 * c * nv, *Hc = hessb + 9 * c;
    for (int j = 0; j < nv; ++j)
      for (int k = 0; k < nv; ++k) {
        double v = 0.0;
        for (int p = 0; p < 3; ++p)
          for (int q = 0; q < 3; ++q) v += Jc[p * nv + j] * Hc[3 * p + q] * Jc[q * nv + k];
        H[j * nv + k] += v;
      }
  }
}

/* phi'(alpha) for phi(alpha) = L(a + alpha p): p^T (M (a + alpha p) - qfrc)
 * + sum_c grad_c(u_c + alpha v_c) . v_c, with v = J p. */
static double ell_dphi(const problem *P, const double *mu, const double *a,
                       const double *p, double alpha) {
  const int nv = P->nv, nc = P->m / 3;
  double d = 0.0;
  for (int j = 0; j < nv; ++j) {
    double v = 0.0;
    for (int k = 0; k < nv; ++k) v += P->M[j * nv + k] * (a[k] + alpha * p[k]);
    d += p[j] * (v - P->qfrc[j]);
  }
  for (int c = 0; c < nc; ++c) {
    double uc[3], vc[3], s, g[3], h[9];
    for (int q = 0; q < 3; ++q) {
      const double *Ji = P->J + (size_t)(3 * c + q) * nv;
      double x = 0.0, y = 0.0;
      for (int k = 0; k < nv; ++k) {
        x += Ji[k] * a[k];
        y += Ji[k] * p[k];
      }
      uc[q] = x - P->aref[3 * c + q] + alpha * y;
      vc[q] = y;
    }
    ell_cone(uc, P->D[3 * c], P->D[3 * c + 1], mu[3 * c], &s, g, h);
    d += g[0] * vc[0] + g[1] * vc[1] + g[2] * vc[2];
  }
  return d;
}

/* Exact line search along p (phi is convex, phi' continuous and increasing):
 * bracket the root of phi' by doubling from alpha = 1, then bisect until the
 * bracket cannot shrink in double precision. */
static double ell_line_search(const problem *P, const double *mu, const double *a,
                              const double *p) {
  double lo = 0.0, hi = 1.0;
  for (int k = 0; k < 200 && ell_dphi(P, mu, a, p, hi) < 0.0; ++k) {
    lo = hi;
    hi *= 2.0;
  }
  for (int k = 0; k < 400; ++k) {
    const double mid = 0.5 * (lo + hi);
    if (!(mid > lo && mid < hi)) break;
    if (ell_dphi(P, mu, a, p, mid) < 0.0) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

double oracle_ell_line_search(int nv, int m, const double *M, const double *J,
                              const double *qfrc, const double *aref,
                              const double *D, const double *mu, const double *a,
                              const double *p) {
  problem P = {nv, m, M, J, qfrc, aref, D};
  return ell_line_search(&P, mu, a, p);
}

/* Objective of Eq. 5 with the round cone at a (a0 = M^-1 qfrc recomputed). */
double oracle_ell_objective(int nv, int m, const double *M, const double *J,
                            const double *qfrc, const double *aref,
                            const double *D, const double *mu, const double *a) {
  problem P = {nv, m, M, J, qfrc, aref, D};
  double *w = (double *)calloc((size_t)(nv * nv + 5 * nv + 14 * m + 8), sizeof(double));
  uint8_t *zone = (uint8_t *)calloc((size_t)m + 1, 1);
  double *H = w, *a0 = H + nv * nv, *d = a0 + nv, *Ma = d + nv, *Jtf = Ma + nv;
  double *r = Jtf + nv, *u = r + nv, *grad = u + m, *hessb = grad + m;
  memcpy(H, M, sizeof(double) * nv * nv);
  double v = NAN;
  if (!chol(nv, H)) {
    memcpy(a0, qfrc, sizeof(double) * nv);
    chol_solve(nv, H, a0);
    v = 0.0;
    for (int j = 0; j < nv; ++j) d[j] = a[j] - a0[j];
    for (int j = 0; j < nv; ++j)
      for (int k = 0; k < nv; ++k) v += 0.5 * d[j] * M[j * nv + k] * d[k];
    ell_residual(&P, mu, a, u, zone, grad, hessb, Ma, Jtf, r, &v);
  }
  free(w);
  free(zone);
  return v;
}

/* Newton on the stationarity residual with the round cone (Eqs. 6-10): from
 * a0 = M^-1 qfrc, p = -H^-1 r with the block Hessians, exact line search,
 * stop at ||r||_inf <= tol * scale or at a step below double-precision
 * resolution of a (64 eps |a|_inf; Newton converges quadratically, so a is
 * then at its double-precision fixed point).  zone (out, m) holds each contact's zone
 * on its three rows at the returned a.  Returns a status code. */
int oracle_ell_solve(int nv, int m, const double *M, const double *J,
                     const double *qfrc, const double *aref, const double *D,
                     const double *mu, double tol, int max_iter, double *a,
                     uint8_t *zone, int *iters) {
  *iters = 0;
  if (nv < 1 || m < 0 || m % 3) return OR_BADSHAPE;
  problem P = {nv, m, M, J, qfrc, aref, D};
  double *w = (double *)calloc((size_t)(nv * nv + 5 * nv + 14 * m + 8), sizeof(double));
  double *H = w, *p = H + nv * nv, *Ma = p + nv, *Jtf = Ma + nv, *r = Jtf + nv;
  double *u = r + nv, *grad = u + m, *hessb = grad + m;
  int status = OR_MAXITER;
  memcpy(H, M, sizeof(double) * nv * nv);
  if (chol(nv, H)) { status = OR_CHOLFAIL; goto done; }
  memcpy(a, qfrc, sizeof(double) * nv);
  chol_solve(nv, H, a);
  for (int k = 0;; ++k) {
    const double scale = ell_residual(&P, mu, a, u, zone, grad, hessb, Ma, Jtf, r, NULL);
    const double rn = inf_norm(nv, r);
    if (!isfinite(rn) || !isfinite(scale)) { status = OR_NONFINITE; break; }
    if (rn <= tol * scale) { status = OR_OK; break; }
    if (k >= max_iter) { status = OR_MAXITER; break; }
    ell_newton_matrix(&P, hessb, H);
    if (chol(nv, H)) { status = OR_CHOLFAIL; break; }
    for (int j = 0; j < nv; ++j) p[j] = -r[j];
    chol_solve(nv, H, p);
    double ptr = 0.0;
    for (int j = 0; j < nv; ++j) ptr += p[j] * r[j];
    if (!(ptr < 0.0)) { status = OR_NOPROGRESS; break; }
    const double alpha = ell_line_search(&P, mu, a, p);
    double step = 0.0;
    for (int j = 0; j < nv; ++j) {
      const double dj = alpha * p[j];
      a[j] += dj;
      if (fabs(dj) > step) step = fabs(dj);
    }
    *iters = k + 1;
    /* a step below double-precision resolution: the residual has reached its
     * rounding floor (the middle zone's gradient cancels large terms) */
    if (step <= 64.0 * 2.220446049250313e-16 * inf_norm(nv, a)) {
      ell_residual(&P, mu, a, u, zone, grad, hessb, Ma, Jtf, r, NULL);
      status = OR_OK;
      break;
    }
  }
done:
  free(w);
  return status;
}

/* IFT adjoint (Eq. 17) with the round cone at the point a: H w = g with
 * H = M + sum_c J_c^T hess_c J_c; dqfrc = w; daref_c = hess_c (J w)_c;
 * dJ = -(grad w^T + daref a^T); dM = -(w a^T + a w^T)/2 (symmetric M);
 * and the cone parameters, dL/dtheta_c = -(J w)_c . d grad_c / d theta_c:
 * dD[3c] for D_N, dD[3c+1] for D_T (dD[3c+2] = 0: not read), dmu[3c] for mu
 * (the other rows 0).  Any output after dJ may be NULL. */
int oracle_ell_adjoint(int nv, int m, const double *M, const double *J,
                       const double *qfrc, const double *aref, const double *D,
                       const double *mu, const double *a, const double *g,
                       double *dqfrc, double *daref, double *dJ, double *dM,
                       double *dD, double *dmu, uint8_t *zone) {
  if (nv < 1 || m < 0 || m % 3) return OR_BADSHAPE;
  problem P = {nv, m, M, J, qfrc, aref, D};
  const int nc = m / 3;
  double *w = (double *)calloc((size_t)(nv * nv + 5 * nv + 14 * m + 8), sizeof(double));
  double *H = w, *Ma = H + nv * nv, *Jtf = Ma + nv, *r = Jtf + nv;
  double *u = r + nv, *grad = u + m, *hessb = grad + m, *v = hessb + 9 * (m / 3) + 3;
  int status = 0;
  ell_residual(&P, mu, a, u, zone, grad, hessb, Ma, Jtf, r, NULL);
  ell_newton_matrix(&P, hessb, H);
  if (chol(nv, H)) { status = OR_CHOLFAIL; goto done; }
  memcpy(dqfrc, g, sizeof(double) * nv);
  chol_solve(nv, H, dqfrc);
  for (int i = 0; i < m; ++i) {
    double x = 0.0;
    for (int k = 0; k < nv; ++k) x += J[i * nv + k] * dqfrc[k];
    v[i] = x;
  }
  for (int c = 0; c < nc; ++c)
    for (int q = 0; q < 3; ++q) {
      double x = 0.0;
      for (int p = 0; p < 3; ++p) x += hessb[9 * c + 3 * q + p] * v[3 * c + p];
      daref[3 * c + q] = x;
    }
  for (int i = 0; i < m; ++i)
    for (int k = 0; k < nv; ++k) dJ[i * nv + k] = -(grad[i] * dqfrc[k] + daref[i] * a[k]);
  if (dM)
    for (int j = 0; j < nv; ++j)
      for (int k = 0; k < nv; ++k)
        dM[j * nv + k] = -0.5 * (dqfrc[j] * a[k] + a[j] * dqfrc[k]);
  if (dD || dmu) {
    for (int c = 0; c < nc; ++c) {
      const double DN = D[3 * c], DT = D[3 * c + 1], f = mu[3 * c];
      const double *uc = u + 3 * c, *vc = v + 3 * c;
      double gN[3] = {0, 0, 0}, gT[3] = {0, 0, 0}, gm[3] = {0, 0, 0};
      const double t = sqrt(uc[1] * uc[1] + uc[2] * uc[2]);
      if (zone[3 * c] == 2) {
        gN[0] = uc[0];
        gT[1] = uc[1];
        gT[2] = uc[2];
      } else if (zone[3 * c] == 1) {
        const double den = DT + f * f * DN;
        const double Dm = DN * DT / den, phi = f * t - uc[0];
        const double h1 = t > 0.0 ? uc[1] / t : 0.0, h2 = t > 0.0 ? uc[2] / t : 0.0;
        const double gv[3] = {-1.0, f * h1, f * h2};
        const double dDN = DT * DT / (den * den), dDT = f * f * DN * DN / (den * den);
        const double dmu_ = -2.0 * f * DN * DN * DT / (den * den);
        for (int q = 0; q < 3; ++q) {
          gN[q] = dDN * phi * gv[q];
          gT[q] = dDT * phi * gv[q];
          gm[q] = dmu_ * phi * gv[q] + Dm * t * gv[q];
        }
        gm[1] += Dm * phi * h1;
        gm[2] += Dm * phi * h2;
      }
      if (dD) {
        dD[3 * c] = -(vc[0] * gN[0] + vc[1] * gN[1] + vc[2] * gN[2]);
        dD[3 * c + 1] = -(vc[0] * gT[0] + vc[1] * gT[1] + vc[2] * gT[2]);
        dD[3 * c + 2] = 0.0;
      }
      if (dmu) {
        dmu[3 * c] = -(vc[0] * gm[0] + vc[1] * gm[1] + vc[2] * gm[2]);
        dmu[3 * c + 1] = dmu[3 * c + 2] = 0.0;
      }
    }
  }
done:
  free(w);
  return status;
}

/* ---- unrolled reverse-mode derivative (the paper's comparison) --------- */

/* Derivative of L = g^T a_K through the executed trace of at most K Newton
 * steps (the "unrolled AD" sensitivity of Section III-E, which the paper sets
 * against the IFT adjoint of Eq. 17).
 *
 * Forward, in the order of oracle_solve: a_0 = M^-1 qfrc (Eq. 1); at step k,
 * stop if ||r||_inf <= tol * scale (or k = K, or p^T r >= 0); otherwise
 * S_k = {jar < 0}, H_k (Eq. 9), p_k = -H_k^-1 r_k, then either exact
 * termination (the mask at a_k + p_k equals S_k: alpha_k = 1, T_k = S_k, and
 * the loop ends after this step) or the exact line search (Eq. 10), which
 * returns alpha_k = -c0/c1 on the segment whose rows T_k = {jar + alpha s <
 * 0} are active, with
 *   c0 = p^T (M a - qfrc) + sum_{T} D_i s_i jar_i,  c1 = p^T M p + sum_{T} D_i s_i^2,
 *   s = J p.  Then a_{k+1} = a_k + alpha_k p_k.
 * The trace keeps a_k, p_k, alpha_k, S_k and T_k; the masks are locally
 * constant, so the derivative is that of the smooth map each step applies.
 *
 * Reverse (cotangents written xb), per step from the last:
 *   alpha_b = ab . p,  pb = alpha ab,  a_k's cotangent starts at ab;
 *   alpha = -c0/c1:   c0b = -alpha_b / c1,  c1b = -alpha_b alpha / c1;
 *   c0, c1:  pb += c0b (M a - qfrc) + 2 c1b M p,  a_kb += c0b M p,
 *            Mb += c0b p a^T + c1b p p^T,  qfrcb -= c0b p,
 *            rows of T:  Db += c0b s jar + c1b s^2,  sb = c0b D jar + 2 c1b D s,
 *                        jarb += c0b D s;
 *   s = J p:          pb += J^T sb,  Jb += sb p^T;
 *   p = -H^-1 r:      z = H^-1 pb,  rb = -z,  Hb = -z p^T;
 *   H = M + J_S^T D_S J_S:  Mb += Hb,  rows of S: Jb_i -= D_i (s_i z + (J z)_i p),
 *                        Db_i -= (J z)_i s_i;
 *   r = M a - qfrc + J^T f:  a_kb -= M z,  Mb -= z a^T,  qfrcb += z,
 *                        Jb_i -= f_i z,  fb = -J z;
 *   f = D_S jar:      rows of S: Db += fb jar,  jarb += fb D;
 *   jar = J a - aref: a_kb += J^T jarb,  Jb += jarb a^T,  arefb -= jarb.
 * Finally a_0 = M^-1 qfrc: y = M^-1 ab, qfrcb += y, Mb -= y a_0^T.  M is a
 * symmetric parameter (as in oracle_adjoint_theta): dM = (Mb + Mb^T) / 2.
 *
 * Outputs a (the returned a_K), *steps, and dqfrc, daref, dJ, dM, dD (any of
 * the last five may be NULL).  Returns a status code as oracle_solve. */
int oracle_unrolled(int nv, int m, const double *M, const double *J,
                    const double *qfrc, const double *aref, const double *D,
                    const double *g, int K, double tol, double *a, int *steps,
                    double *dqfrc, double *daref, double *dJ, double *dM,
                    double *dD) {
  *steps = 0;
  if (nv < 1 || m < 0 || K < 0) return OR_BADSHAPE;
  problem P = {nv, m, M, J, qfrc, aref, D};
  const size_t km = (size_t)(K > 0 ? K : 1) * (size_t)(m > 0 ? m : 1);
  double *A = (double *)calloc((size_t)(K + 1) * nv, sizeof(double));
  double *Pk = (double *)calloc((size_t)(K > 0 ? K : 1) * nv, sizeof(double));
  double *alph = (double *)calloc((size_t)(K > 0 ? K : 1), sizeof(double));
  uint8_t *Sk = (uint8_t *)calloc(km, 1), *Tk = (uint8_t *)calloc(km, 1);
  size_t wd = (size_t)(10 * m + 12 * nv + 4 * nv * nv + 8);
  double *w = (double *)calloc(wd, sizeof(double));
  breakpoint *bp = (breakpoint *)calloc((size_t)m + 1, sizeof(breakpoint));
  uint8_t *act = (uint8_t *)calloc((size_t)m + 1, 1);
  double *jar = w, *f = jar + m, *s = f + m, *jar2 = s + m, *sb = jar2 + m;
  double *jarb = sb + m, *Jz = jarb + m, *Db = Jz + m, *arb = Db + m;
  double *Ma = arb + m, *Jtf = Ma + nv, *r = Jtf + nv, *p = r + nv;
  double *Mp = p + nv, *ab = Mp + nv, *akb = ab + nv, *pb = akb + nv, *z = pb + nv;
  double *qb = z + nv, *Maq = qb + nv, *y = Maq + nv;
  double *H = y + nv, *Mb = H + nv * nv, *Jb = NULL;
  int status = OR_MAXITER, n = 0;

  /* ---- forward: a_0 = M^-1 qfrc, then at most K recorded Newton steps */
  memcpy(H, M, sizeof(double) * nv * nv);
  if (chol(nv, H)) { status = OR_CHOLFAIL; goto done; }
  memcpy(A, qfrc, sizeof(double) * nv);
  chol_solve(nv, H, A);
  for (int k = 0;; ++k) {
    double *ak = A + (size_t)k * nv;
    double scale = residual(&P, ak, jar, act, f, Ma, Jtf, r);
    double rn = inf_norm(nv, r);
    if (!isfinite(rn) || !isfinite(scale)) { status = OR_NONFINITE; break; }
    if (rn <= tol * scale) { status = OR_OK; break; }
    if (k >= K) { status = OR_MAXITER; break; }
    newton_matrix(&P, act, H);
    if (chol(nv, H)) { status = OR_CHOLFAIL; break; }
    for (int j = 0; j < nv; ++j) p[j] = -r[j];
    chol_solve(nv, H, p);
    double ptr = 0.0;
    for (int j = 0; j < nv; ++j) ptr += p[j] * r[j];
    if (!(ptr < 0.0)) { status = OR_NOPROGRESS; break; }
    int same = 1;
    for (int i = 0; i < m; ++i) {
      double v = 0.0;
      for (int q = 0; q < nv; ++q) v += J[i * nv + q] * (ak[q] + p[q]);
      if ((v - aref[i] < 0.0) != (act[i] != 0)) same = 0;
    }
    double alpha = same ? 1.0 : line_search(&P, ak, p, jar, Ma, s, bp);
    for (int i = 0; i < m; ++i) {
      double si = 0.0;
      for (int q = 0; q < nv; ++q) si += J[i * nv + q] * p[q];
      Sk[(size_t)k * m + i] = act[i];
      Tk[(size_t)k * m + i] = same ? act[i] : (jar[i] + alpha * si < 0.0);
    }
    memcpy(Pk + (size_t)k * nv, p, sizeof(double) * nv);
    alph[k] = alpha;
    for (int j = 0; j < nv; ++j) ak[nv + j] = ak[j] + alpha * p[j];
    n = k + 1;
    if (same) { status = OR_OK; break; }
  }
  *steps = n;
  memcpy(a, A + (size_t)n * nv, sizeof(double) * nv);
  if (status == OR_CHOLFAIL || status == OR_NONFINITE) goto done;

  /* ---- reverse sweep over the recorded steps */
  Jb = (double *)calloc((size_t)(m > 0 ? m : 1) * nv, sizeof(double));
  memcpy(ab, g, sizeof(double) * nv);
  for (int k = n - 1; k >= 0; --k) {
    const double *ak = A + (size_t)k * nv, *pk = Pk + (size_t)k * nv;
    const uint8_t *S = Sk + (size_t)k * m, *T = Tk + (size_t)k * m;
    const double alpha = alph[k];
    for (int i = 0; i < m; ++i) {
      double u = 0.0, v = 0.0;
      for (int q = 0; q < nv; ++q) {
        u += J[i * nv + q] * ak[q];
        v += J[i * nv + q] * pk[q];
      }
      jar[i] = u - aref[i];
      s[i] = v;
      f[i] = S[i] ? D[i] * jar[i] : 0.0;
      sb[i] = 0.0;
      jarb[i] = 0.0;
    }
    double c1 = 0.0, alpha_b = 0.0;
    for (int j = 0; j < nv; ++j) {
      double u = 0.0, v = 0.0;
      for (int q = 0; q < nv; ++q) {
        u += M[j * nv + q] * pk[q];
        v += M[j * nv + q] * ak[q];
      }
      Mp[j] = u;
      Maq[j] = v - qfrc[j];
      c1 += pk[j] * u;
      alpha_b += ab[j] * pk[j];
    }
    for (int i = 0; i < m; ++i)
      if (T[i]) c1 += D[i] * s[i] * s[i];
    const double c0b = -alpha_b / c1, c1b = -alpha_b * alpha / c1;
    for (int j = 0; j < nv; ++j) {
      pb[j] = alpha * ab[j] + c0b * Maq[j] + 2.0 * c1b * Mp[j];
      akb[j] = ab[j] + c0b * Mp[j];
      qb[j] -= c0b * pk[j];
      for (int q = 0; q < nv; ++q)
        Mb[j * nv + q] += c0b * pk[j] * ak[q] + c1b * pk[j] * pk[q];
    }
    for (int i = 0; i < m; ++i) {
      if (!T[i]) continue;
      Db[i] += c0b * s[i] * jar[i] + c1b * s[i] * s[i];
      sb[i] = c0b * D[i] * jar[i] + 2.0 * c1b * D[i] * s[i];
      jarb[i] += c0b * D[i] * s[i];
    }
    for (int i = 0; i < m; ++i)
      for (int q = 0; q < nv; ++q) {
        pb[q] += J[i * nv + q] * sb[i];
        Jb[i * nv + q] += sb[i] * pk[q];
      }
    newton_matrix(&P, S, H);
    if (chol(nv, H)) { status = OR_CHOLFAIL; goto done; }
    memcpy(z, pb, sizeof(double) * nv);
    chol_solve(nv, H, z);
    for (int i = 0; i < m; ++i) {
      double v = 0.0;
      for (int q = 0; q < nv; ++q) v += J[i * nv + q] * z[q];
      Jz[i] = v;
    }
    for (int j = 0; j < nv; ++j) {
      double v = 0.0;
      for (int q = 0; q < nv; ++q) v += M[j * nv + q] * z[q];
      akb[j] -= v;
      qb[j] += z[j];
      for (int q = 0; q < nv; ++q) Mb[j * nv + q] -= z[j] * pk[q] + z[j] * ak[q];
    }
    for (int i = 0; i < m; ++i) {
      for (int q = 0; q < nv; ++q) Jb[i * nv + q] -= f[i] * z[q];
      if (!S[i]) continue;
      for (int q = 0; q < nv; ++q)
        Jb[i * nv + q] -= D[i] * (s[i] * z[q] + Jz[i] * pk[q]);
      Db[i] -= Jz[i] * s[i];
      const double fb = -Jz[i];
      Db[i] += fb * jar[i];
      jarb[i] += fb * D[i];
    }
    for (int i = 0; i < m; ++i) {
      for (int q = 0; q < nv; ++q) {
        akb[q] += J[i * nv + q] * jarb[i];
        Jb[i * nv + q] += jarb[i] * ak[q];
      }
      arb[i] -= jarb[i];
    }
    memcpy(ab, akb, sizeof(double) * nv);
  }
  /* a_0 = M^-1 qfrc */
  memcpy(H, M, sizeof(double) * nv * nv);
  if (chol(nv, H)) { status = OR_CHOLFAIL; goto done; }
  memcpy(y, ab, sizeof(double) * nv);
  chol_solve(nv, H, y);
  for (int j = 0; j < nv; ++j) {
    qb[j] += y[j];
    for (int q = 0; q < nv; ++q) Mb[j * nv + q] -= y[j] * A[q];
  }
  if (dqfrc) memcpy(dqfrc, qb, sizeof(double) * nv);
  if (daref) memcpy(daref, arb, sizeof(double) * m);
  if (dD) memcpy(dD, Db, sizeof(double) * m);
  if (dJ) memcpy(dJ, Jb, sizeof(double) * m * nv);
  if (dM)
    for (int j = 0; j < nv; ++j)
      for (int q = 0; q < nv; ++q)
        dM[j * nv + q] = 0.5 * (Mb[j * nv + q] + Mb[q * nv + j]);
done:
  free(A);
  free(Pk);
  free(alph);
  free(Sk);
  free(Tk);
  free(w);
  free(bp);
  free(act);
  free(Jb);
  return status;
}

/* The exact line search on its own, for pinning it: returns the minimiser of
 * phi(alpha) = L(a + alpha p) over alpha > 0. */
double oracle_line_search(int nv, int m, const double *M, const double *J,
                          const double *qfrc, const double *aref,
                          const double *D, const double *a, const double *p) {
  problem P = {nv, m, M, J, qfrc, aref, D};
  double *w = (double *)calloc((size_t)(4 * m + 4 * nv + 4), sizeof(double));
  breakpoint *bp = (breakpoint *)calloc((size_t)m + 1, sizeof(breakpoint));
  uint8_t *act = (uint8_t *)calloc((size_t)m + 1, 1);
  double *jar = w, *f = jar + m, *s = f + m, *Ma = s + m, *Jtf = Ma + nv;
  double *r = Jtf + nv;
  residual(&P, a, jar, act, f, Ma, Jtf, r);
  double alpha = line_search(&P, a, p, jar, Ma, s, bp);
  free(w);
  free(bp);
  free(act);
  return alpha;
}
