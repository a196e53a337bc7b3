/*
 * Plain FP64 CPU oracle for distributed bundle adjustment by consensus ADMM
 * (arXiv 1708.07954).  TEST INFRASTRUCTURE ONLY: loaded by the tests, the
 * package smoke check and the benchmark's CPU-baseline leg, never by the
 * product path.  No blocking, fusion or reordering beyond the paper's steps;
 * every function names the passage it restates.  Built without fast-math and
 * without floating-point contraction so results do not depend on the host.
 */
#include "dba_oracle.h"

/* Levenberg damping factors: lambda is divided by ORA_LM_DECREASE after an accepted step
 * and multiplied by ORA_LM_INCREASE after a rejected one (the textbook factor 10).  They
 * are macros only so that the tests can build deliberately wrong oracles and check that
 * the step-wise pins reject them; the product path never builds this file. */
#ifndef ORA_LM_DECREASE
#define ORA_LM_DECREASE 10.0
#endif
#ifndef ORA_LM_INCREASE
#define ORA_LM_INCREASE 10.0
#endif

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ Sec. 2.1 */

static void mat3_mul(const double A[9], const double B[9], double C[9]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double acc = 0.0;
      for (int k = 0; k < 3; ++k) acc += A[3 * i + k] * B[3 * k + j];
      C[3 * i + j] = acc;
    }
}

static void mat3_vec(const double A[9], const double x[3], double y[3]) {
  for (int i = 0; i < 3; ++i) y[i] = A[3 * i] * x[0] + A[3 * i + 1] * x[1] + A[3 * i + 2] * x[2];
}

/* R1(a): rotation by a about the first axis, and its derivative d/da. */
static void rot1(double a, double R[9], double dR[9]) {
  double c = cos(a), s = sin(a);
  double r[9] = {1, 0, 0, 0, c, -s, 0, s, c};
  double d[9] = {0, 0, 0, 0, -s, -c, 0, c, -s};
  memcpy(R, r, sizeof r);
  memcpy(dR, d, sizeof d);
}
/* R2(b): rotation about the second axis. */
static void rot2(double b, double R[9], double dR[9]) {
  double c = cos(b), s = sin(b);
  double r[9] = {c, 0, s, 0, 1, 0, -s, 0, c};
  double d[9] = {-s, 0, c, 0, 0, 0, -c, 0, -s};
  memcpy(R, r, sizeof r);
  memcpy(dR, d, sizeof d);
}
/* R3(g): rotation about the third axis. */
static void rot3(double g, double R[9], double dR[9]) {
  double c = cos(g), s = sin(g);
  double r[9] = {c, -s, 0, s, c, 0, 0, 0, 1};
  double d[9] = {-s, -c, 0, c, -s, 0, 0, 0, 0};
  memcpy(R, r, sizeof r);
  memcpy(dR, d, sizeof d);
}

/* R = R3(gamma) R2(beta) R1(alpha), Sec. 2.1. */
void ora_rotation(const double y[6], double R[9]) {
  double R1[9], R2[9], R3[9], d[9], T[9];
  rot1(y[0], R1, d);
  rot2(y[1], R2, d);
  rot3(y[2], R3, d);
  mat3_mul(R2, R1, T);
  mat3_mul(R3, T, R);
}

/* z~ = R x + t; z = f z~_{1,2} / z~_3 + (cx, cy)  (Sec. 2.1, Eq. 1). */
double ora_project(const ora_config* c, const double x[3], const double y[6], double zout[2]) {
  double R[9], p[3];
  ora_rotation(y, R);
  mat3_vec(R, x, p);
  p[0] += y[3];
  p[1] += y[4];
  p[2] += y[5];
  zout[0] = c->focal * p[0] / p[2] + c->cx;
  zout[1] = c->focal * p[1] / p[2] + c->cy;
  return p[2];
}

/* J = dz/dz~ * dz~/d(x, alpha, beta, gamma, t): chain rule on Eq. 1 and Sec. 2.1. */
void ora_jacobian(const ora_config* c, const double x[3], const double y[6], double J[18]) {
  double R1[9], R2[9], R3[9], d1[9], d2[9], d3[9], R[9], T[9], D[3][9];
  rot1(y[0], R1, d1);
  rot2(y[1], R2, d2);
  rot3(y[2], R3, d3);
  mat3_mul(R2, R1, T);
  mat3_mul(R3, T, R); /* R */
  mat3_mul(R2, d1, T);
  mat3_mul(R3, T, D[0]); /* dR/dalpha = R3 R2 R1' */
  mat3_mul(d2, R1, T);
  mat3_mul(R3, T, D[1]); /* dR/dbeta  = R3 R2' R1 */
  mat3_mul(d3, R2, T);
  mat3_mul(T, R1, D[2]); /* dR/dgamma = R3' R2 R1 */

  double p[3];
  mat3_vec(R, x, p);
  p[0] += y[3];
  p[1] += y[4];
  p[2] += y[5];
  /* dz/dz~ (2x3) */
  double P[6] = {c->focal / p[2], 0.0, -c->focal * p[0] / (p[2] * p[2]),
                 0.0, c->focal / p[2], -c->focal * p[1] / (p[2] * p[2])};
  /* dz~/dv (3x9): [R | dR/da x, dR/db x, dR/dg x | I] */
  double G[27];
  memset(G, 0, sizeof G);
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) G[9 * i + k] = R[3 * i + k];
  for (int a = 0; a < 3; ++a) {
    double col[3];
    mat3_vec(D[a], x, col);
    for (int i = 0; i < 3; ++i) G[9 * i + 3 + a] = col[i];
  }
  for (int i = 0; i < 3; ++i) G[9 * i + 6 + i] = 1.0;
  for (int r = 0; r < 2; ++r)
    for (int k = 0; k < 9; ++k) {
      double acc = 0.0;
      for (int i = 0; i < 3; ++i) acc += P[3 * r + i] * G[9 * i + k];
      J[9 * r + k] = acc;
    }
}

/* ------------------------------------------------- misfit losses, Sec. 3.1 */

/* phi_m as a function of s = |e|^2 (squared l2, Huber, Student's t). */
double ora_loss(int kind, double param, double s) {
  if (kind == ORA_LOSS_HUBER) {
    double d = param;
    return s <= d * d ? s : 2.0 * d * sqrt(s) - d * d;
  }
  if (kind == ORA_LOSS_STUDENT_T) {
    double nu = param;
    return nu * log1p(s / nu);
  }
  return s;
}

/* d phi_m / d s: the iteratively reweighted least-squares weight. */
double ora_weight(int kind, double param, double s) {
  if (kind == ORA_LOSS_HUBER) {
    double d = param;
    return s <= d * d ? 1.0 : d / sqrt(s);
  }
  if (kind == ORA_LOSS_STUDENT_T) {
    double nu = param;
    return nu / (nu + s);
  }
  return 1.0;
}

/* ------------------------------------------------ local subproblem, Eq. (9) */

/* Penalty of coordinate k of (x, alpha, beta, gamma, t).  phi_a is the squared
 * Euclidean distance (Sec. 3.1); the camera block may weight its angles
 * (radians) apart from its translation (lengths), rho_angle <= 0 keeping the
 * paper's single rho_y. */
static double rho_of(const ora_config* c, int k) {
  if (k < 3) return c->rho_x;
  if (k < 6 && c->rho_angle > 0.0) return c->rho_angle;
  return c->rho_y;
}

/* phi_m(z - f(v)) + r^T (x - xbar) + s^T (y - ybar) + rho_x/2 |x - xbar|^2 + rho_y/2 |y - ybar|^2 */
double ora_local_objective(const ora_config* c, const double z[2], const double xbar[3],
                           const double ybar[6], const double dual[9], const double v[9]) {
  double zp[2];
  double depth = ora_project(c, v, v + 3, zp);
  if (!(depth > c->eps_depth)) return INFINITY;
  double e0 = z[0] - zp[0], e1 = z[1] - zp[1];
  double L = ora_loss(c->loss, c->loss_param, e0 * e0 + e1 * e1);
  for (int k = 0; k < 9; ++k) {
    double d = v[k] - (k < 3 ? xbar[k] : ybar[k - 3]);
    L += dual[k] * d + 0.5 * rho_of(c, k) * d * d;
  }
  return L;
}

int ora_chol_solve(int n, const double* A, const double* b, double* x) {
  double* L = (double*)calloc((size_t)n * n, sizeof(double));
  if (!L) return -1;
  for (int j = 0; j < n; ++j) {
    double d = A[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) d -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
    if (!(d > 0.0)) {
      free(L);
      return -1;
    }
    double ljj = sqrt(d);
    L[(size_t)j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double acc = A[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) acc -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
      L[(size_t)i * n + j] = acc / ljj;
    }
  }
  /* L y = b, then L^T x = y */
  for (int i = 0; i < n; ++i) {
    double acc = b[i];
    for (int k = 0; k < i; ++k) acc -= L[(size_t)i * n + k] * x[k];
    x[i] = acc / L[(size_t)i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double acc = x[i];
    for (int k = i + 1; k < n; ++k) acc -= L[(size_t)k * n + i] * x[k];
    x[i] = acc / L[(size_t)i * n + i];
  }
  free(L);
  return 0;
}

/*
 * Eq. (9) solved by damped Gauss-Newton (Levenberg) steps with IRLS weights,
 * the paper's Gauss-Newton for the squared loss (Sec. 3.1) extended to the
 * robust losses.  Each of the inner_steps steps:
 *   e = z - f(v), s = |e|^2, w = phi'(s), J = df/dv
 *   g = -2 w J^T e + (r, s) + diag(rho) (v - vbar)        gradient of Eq. (9)
 *   H = 2 w J^T J + diag(rho)                              Gauss-Newton Hessian
 *   (H + lambda I) d = -g;  accept v + d iff it is in front of the camera and
 *   lowers Eq. (9): lambda /= 10 (clamped), else lambda *= 10.
 * lambda starts at lm_lambda0 * mean(diag H) at the first step.  A linearisation
 * point behind the camera contributes no misfit term (the proximal step).  A
 * step whose predicted decrease is below the objective's rounding noise is
 * accepted without the comparison (lm_model_tol); like every accepted step it
 * then re-evaluates Eq. (9) at the new point.
 */
void ora_local_solve(const ora_config* c, const double z[2], const double xbar[3],
                     const double ybar[6], const double dual[9], double v[9]) {
  double lambda = -1.0;
  double L_old = ora_local_objective(c, z, xbar, ybar, dual, v);
  for (int step = 0; step < c->inner_steps; ++step) {
    double H[81], g[9], d[9], vt[9], J[18] = {0};
    double zp[2], e[2] = {0.0, 0.0}, w = 0.0;
    double depth = ora_project(c, v, v + 3, zp);
    if (depth > c->eps_depth) {
      e[0] = z[0] - zp[0];
      e[1] = z[1] - zp[1];
      w = ora_weight(c->loss, c->loss_param, e[0] * e[0] + e[1] * e[1]);
      ora_jacobian(c, v, v + 3, J);
    }
    for (int a = 0; a < 9; ++a) {
      double vbar_a = a < 3 ? xbar[a] : ybar[a - 3];
      g[a] = -2.0 * w * (J[a] * e[0] + J[9 + a] * e[1]) + dual[a] + rho_of(c, a) * (v[a] - vbar_a);
      for (int b = 0; b < 9; ++b)
        H[9 * a + b] = 2.0 * w * (J[a] * J[b] + J[9 + a] * J[9 + b]) + (a == b ? rho_of(c, a) : 0.0);
    }
    if (lambda < 0.0) {
      double tr = 0.0;
      for (int a = 0; a < 9; ++a) tr += H[9 * a + a];
      lambda = c->lm_lambda0 * tr / 9.0;
    }
    double neg_g[9];
    for (int a = 0; a < 9; ++a) {
      H[9 * a + a] += lambda;
      neg_g[a] = -g[a];
    }
    if (ora_chol_solve(9, H, neg_g, d) != 0) {
      lambda *= ORA_LM_INCREASE;
      continue;
    }
    /* Decrease of the Gauss-Newton model -g.d - d^T H d / 2 (undamped H); since
       (H + lambda I) d = -g it equals (lambda |d|^2 - g.d) / 2. */
    double gd = 0.0, dd = 0.0;
    for (int a = 0; a < 9; ++a) {
      gd += g[a] * d[a];
      dd += d[a] * d[a];
    }
    double pred = 0.5 * (lambda * dd - gd);
    /* Below the rounding noise of the objective (residuals carry ~u |z| each), comparing
       objective values cannot tell a better point from a worse one, so the model's step
       is trusted: accepted if the trial point is in front of the camera. */
    int trust = 0;
    if (isfinite(L_old) && c->lm_model_tol > 0.0) {
      double noise = c->lm_model_tol * 0x1p-53 *
                     (fabs(L_old) + 2.0 * w * sqrt(e[0] * e[0] + e[1] * e[1]) * (fabs(z[0]) + fabs(z[1])));
      trust = pred <= noise;
    }
    for (int a = 0; a < 9; ++a) vt[a] = v[a] + d[a];
    double L_new = ora_local_objective(c, z, xbar, ybar, dual, vt); /* +inf behind the camera */
    if (isfinite(L_new) && (trust || L_new < L_old)) {
      memcpy(v, vt, sizeof vt);
      L_old = L_new;
      lambda = fmax(lambda / ORA_LM_DECREASE, c->lm_lambda_min);
    } else {
      lambda *= ORA_LM_INCREASE;
    }
  }
}

/* Gradient of Eq. (9) at v: -2 w J^T e + dual + diag(rho) (v - vbar); a point behind the
 * camera contributes no misfit term.  Also returns the noise scale 2 w |e| (|z1| + |z2|). */
static void local_gradient(const ora_config* c, const double z[2], const double xbar[3],
                           const double ybar[6], const double dual[9], const double v[9], double g[9],
                           double* noise) {
  double zp[2], J[18] = {0}, e[2] = {0.0, 0.0}, w = 0.0;
  if (ora_project(c, v, v + 3, zp) > c->eps_depth) {
    e[0] = z[0] - zp[0];
    e[1] = z[1] - zp[1];
    w = ora_weight(c->loss, c->loss_param, e[0] * e[0] + e[1] * e[1]);
    ora_jacobian(c, v, v + 3, J);
  }
  for (int a = 0; a < 9; ++a) {
    double vbar_a = a < 3 ? xbar[a] : ybar[a - 3];
    g[a] = -2.0 * w * (J[a] * e[0] + J[9 + a] * e[1]) + dual[a] + rho_of(c, a) * (v[a] - vbar_a);
  }
  *noise = 2.0 * w * sqrt(e[0] * e[0] + e[1] * e[1]) * (fabs(z[0]) + fabs(z[1]));
}

/*
 * L-BFGS (Nocedal and Wright, Numerical Optimization, Ch. 7) on Eq. (9) in the scaled
 * coordinates u_a = sqrt(rho_a) (v_a - vbar_a), where the penalty has unit curvature:
 *   p = -H g_u by the two-loop recursion over the last ORA_LBFGS_MEMORY pairs (s, y),
 *       H0 = (s^T y / y^T y) I of the newest pair (I before the first);
 *   step t = 1, 1/2, 1/4, ... until v + t p (unscaled) is in front of the camera and
 *       L(trial) <= L + c1 t g_u.p, or the decrease -t g_u.p is below the objective's
 *       rounding noise (the local solve's noise rule); no acceptable step ends the solve;
 *   a pair is kept only when s^T y > 0.
 */
void ora_local_solve_lbfgs(const ora_config* c, const double z[2], const double xbar[3],
                           const double ybar[6], const double dual[9], double v[9]) {
  enum { M = ORA_LBFGS_MEMORY };
  double r[9];
  for (int a = 0; a < 9; ++a) r[a] = sqrt(rho_of(c, a));
  double S[M][9], Y[M][9], rho_h[M];
  int n_hist = 0, newest = -1;
  double L = ora_local_objective(c, z, xbar, ybar, dual, v);
  double g[9], gu[9], noise;
  local_gradient(c, z, xbar, ybar, dual, v, g, &noise);
  for (int a = 0; a < 9; ++a) gu[a] = g[a] / r[a];
  for (int it = 0; it < c->inner_steps; ++it) {
    /* two-loop recursion: q = g_u, newest to oldest, then H0, then oldest to newest */
    double q[9], alpha[M];
    for (int a = 0; a < 9; ++a) q[a] = gu[a];
    for (int h = 0; h < n_hist; ++h) {
      int k = (newest - h + M) % M;
      double sq = 0.0;
      for (int a = 0; a < 9; ++a) sq += S[k][a] * q[a];
      alpha[k] = rho_h[k] * sq;
      for (int a = 0; a < 9; ++a) q[a] -= alpha[k] * Y[k][a];
    }
    double gamma = 1.0;
    if (n_hist > 0) {
      double sy = 0.0, yy = 0.0;
      for (int a = 0; a < 9; ++a) {
        sy += S[newest][a] * Y[newest][a];
        yy += Y[newest][a] * Y[newest][a];
      }
      gamma = sy / yy;
    }
    for (int a = 0; a < 9; ++a) q[a] *= gamma;
    for (int h = n_hist - 1; h >= 0; --h) {
      int k = (newest - h + M) % M;
      double yq = 0.0;
      for (int a = 0; a < 9; ++a) yq += Y[k][a] * q[a];
      double beta = rho_h[k] * yq;
      for (int a = 0; a < 9; ++a) q[a] += S[k][a] * (alpha[k] - beta);
    }
    double p[9], gp = 0.0;
    for (int a = 0; a < 9; ++a) {
      p[a] = -q[a];
      gp += gu[a] * p[a];
    }
    if (!(gp < 0.0)) { /* not a descent direction: steepest descent */
      gp = 0.0;
      for (int a = 0; a < 9; ++a) {
        p[a] = -gu[a];
        gp -= gu[a] * gu[a];
      }
    }
    /* backtracking line search */
    double t = 1.0, vt[9], Lt = INFINITY;
    int accepted = 0;
    for (int hv = 0; hv <= ORA_LBFGS_HALVINGS; ++hv, t *= 0.5) {
      for (int a = 0; a < 9; ++a) vt[a] = v[a] + t * p[a] / r[a];
      Lt = ora_local_objective(c, z, xbar, ybar, dual, vt);
      if (!isfinite(Lt)) continue;
      int trust = isfinite(L) && c->lm_model_tol > 0.0 &&
                  -t * gp <= c->lm_model_tol * 0x1p-53 * (fabs(L) + noise);
      if (trust || Lt <= L + ORA_LBFGS_ARMIJO * t * gp) {
        accepted = 1;
        break;
      }
    }
    if (!accepted) break;
    double gt[9], gut[9], noise_t;
    local_gradient(c, z, xbar, ybar, dual, vt, gt, &noise_t);
    double sy = 0.0, sv[9], yv[9];
    for (int a = 0; a < 9; ++a) {
      gut[a] = gt[a] / r[a];
      sv[a] = t * p[a];
      yv[a] = gut[a] - gu[a];
      sy += sv[a] * yv[a];
    }
    if (sy > 0.0) {
      newest = (newest + 1) % M;
      memcpy(S[newest], sv, sizeof sv);
      memcpy(Y[newest], yv, sizeof yv);
      rho_h[newest] = 1.0 / sy;
      if (n_hist < M) n_hist += 1;
    }
    memcpy(v, vt, sizeof vt);
    memcpy(gu, gut, sizeof gut);
    L = Lt;
    noise = noise_t;
  }
}

/* ------------------------------------------- ADMM iteration, Eqs. (9)-(13) */

void ora_admm_init(int n_cams, int n_pts, long n_obs, const int* pt_idx, const int* cam_idx,
                   const double* cams, const double* pts, double* copies, double* duals) {
  (void)n_cams;
  (void)n_pts;
  for (long o = 0; o < n_obs; ++o) {
    for (int k = 0; k < 3; ++k) copies[9 * o + k] = pts[3 * (long)pt_idx[o] + k];
    for (int k = 0; k < 6; ++k) copies[9 * o + 3 + k] = cams[6 * (long)cam_idx[o] + k];
    for (int k = 0; k < 9; ++k) duals[9 * o + k] = 0.0;
  }
}

static int check_indices(int n_cams, int n_pts, long n_obs, const int* pt_idx, const int* cam_idx) {
  for (long o = 0; o < n_obs; ++o)
    if (pt_idx[o] < 0 || pt_idx[o] >= n_pts || cam_idx[o] < 0 || cam_idx[o] >= n_cams) return -1;
  return 0;
}

int ora_admm_iterate(const ora_config* c, int n_cams, int n_pts, long n_obs, const int* pt_idx,
                     const int* cam_idx, const double* z, const double* z_true, double* copies,
                     double* duals, double* cams, double* pts, int iters, int nthreads,
                     ora_metrics* metrics) {
  if (n_cams < 0 || n_pts < 0 || n_obs < 0 || iters < 0) return -1;
  if (check_indices(n_cams, n_pts, n_obs, pt_idx, cam_idx) != 0) return -1;
#ifdef _OPENMP
  omp_set_num_threads(nthreads > 0 ? nthreads : omp_get_num_procs());
#else
  (void)nthreads;
#endif
  double* sum_x = (double*)calloc((size_t)n_pts * 3 + 1, sizeof(double));
  double* sum_y = (double*)calloc((size_t)n_cams * 6 + 1, sizeof(double));
  long* cnt_x = (long*)calloc((size_t)n_pts + 1, sizeof(long));
  long* cnt_y = (long*)calloc((size_t)n_cams + 1, sizeof(long));
  double* pts_prev = (double*)malloc(((size_t)n_pts * 3 + 1) * sizeof(double));
  double* cams_prev = (double*)malloc(((size_t)n_cams * 6 + 1) * sizeof(double));
  if (!sum_x || !sum_y || !cnt_x || !cnt_y || !pts_prev || !cams_prev) {
    free(sum_x); free(sum_y); free(cnt_x); free(cnt_y); free(pts_prev); free(cams_prev);
    return -1;
  }
  for (int it = 0; it < iters; ++it) {
    memcpy(pts_prev, pts, (size_t)n_pts * 3 * sizeof(double));
    memcpy(cams_prev, cams, (size_t)n_cams * 6 * sizeof(double));

    /* Eq. (9): every observation's local subproblem, warm-started at its copy. */
#pragma omp parallel for schedule(dynamic, 256)
    for (long o = 0; o < n_obs; ++o) {
      if (c->local_solver == ORA_SOLVER_LBFGS)
        ora_local_solve_lbfgs(c, z + 2 * o, pts + 3 * (long)pt_idx[o], cams + 6 * (long)cam_idx[o],
                              duals + 9 * o, copies + 9 * o);
      else
        ora_local_solve(c, z + 2 * o, pts + 3 * (long)pt_idx[o], cams + 6 * (long)cam_idx[o],
                        duals + 9 * o, copies + 9 * o);
    }

    /* Eq. (10): x_i = mean over its copies of (x_i^j + r_i^j / rho_x), old duals. */
    memset(sum_x, 0, (size_t)n_pts * 3 * sizeof(double));
    memset(cnt_x, 0, (size_t)n_pts * sizeof(long));
    for (long o = 0; o < n_obs; ++o) {
      long i = pt_idx[o];
      for (int k = 0; k < 3; ++k) sum_x[3 * i + k] += copies[9 * o + k] + duals[9 * o + k] / c->rho_x;
      cnt_x[i] += 1;
    }
    for (long i = 0; i < n_pts; ++i)
      if (cnt_x[i] > 0)
        for (int k = 0; k < 3; ++k) pts[3 * i + k] = sum_x[3 * i + k] / (double)cnt_x[i];

    /* Eq. (11): y_j = mean over its copies of (y_j^i + s_j^i / rho_y), old duals. */
    memset(sum_y, 0, (size_t)n_cams * 6 * sizeof(double));
    memset(cnt_y, 0, (size_t)n_cams * sizeof(long));
    for (long o = 0; o < n_obs; ++o) {
      long j = cam_idx[o];
      for (int k = 0; k < 6; ++k)
        sum_y[6 * j + k] += copies[9 * o + 3 + k] + duals[9 * o + 3 + k] / rho_of(c, 3 + k);
      cnt_y[j] += 1;
    }
    for (long j = 0; j < n_cams; ++j)
      if (cnt_y[j] > 0)
        for (int k = 0; k < 6; ++k) cams[6 * j + k] = sum_y[6 * j + k] / (double)cnt_y[j];

    /* Eqs. (12), (13): dual ascent with the new consensus. */
#pragma omp parallel for schedule(static)
    for (long o = 0; o < n_obs; ++o) {
      long i = pt_idx[o], j = cam_idx[o];
      for (int k = 0; k < 3; ++k) duals[9 * o + k] += c->rho_x * (copies[9 * o + k] - pts[3 * i + k]);
      for (int k = 0; k < 6; ++k)
        duals[9 * o + 3 + k] += rho_of(c, 3 + k) * (copies[9 * o + 3 + k] - cams[6 * j + k]);
    }
  }
  if (metrics)
    ora_eval(c, n_cams, n_pts, n_obs, pt_idx, cam_idx, z, z_true, copies, cams, pts,
             iters > 0 ? cams_prev : NULL, iters > 0 ? pts_prev : NULL, metrics);
  free(sum_x); free(sum_y); free(cnt_x); free(cnt_y); free(pts_prev); free(cams_prev);
  return 0;
}

void ora_eval(const ora_config* c, int n_cams, int n_pts, long n_obs, const int* pt_idx,
              const int* cam_idx, const double* z, const double* z_true, const double* copies,
              const double* cams, const double* pts, const double* cams_prev,
              const double* pts_prev, ora_metrics* out) {
  (void)n_cams;
  (void)n_pts;
  double se = 0.0, sg = 0.0, obj = 0.0, pr = 0.0, dr = 0.0;
  long valid = 0, invalid = 0;
  for (long o = 0; o < n_obs; ++o) {
    const double* x = pts + 3 * (long)pt_idx[o];
    const double* y = cams + 6 * (long)cam_idx[o];
    double zp[2];
    double depth = ora_project(c, x, y, zp);
    if (depth > c->eps_depth) {
      double e0 = z[2 * o] - zp[0], e1 = z[2 * o + 1] - zp[1];
      se += e0 * e0 + e1 * e1;
      obj += ora_loss(c->loss, c->loss_param, e0 * e0 + e1 * e1);
      if (z_true) {
        double g0 = zp[0] - z_true[2 * o], g1 = zp[1] - z_true[2 * o + 1];
        sg += g0 * g0 + g1 * g1;
      }
      valid += 1;
    } else {
      invalid += 1;
    }
    if (copies)
      for (int k = 0; k < 9; ++k) {
        double d = copies[9 * o + k] - (k < 3 ? x[k] : y[k - 3]);
        pr += d * d;
      }
    if (cams_prev && pts_prev) {
      for (int k = 0; k < 3; ++k) {
        double d = c->rho_x * (x[k] - pts_prev[3 * (long)pt_idx[o] + k]);
        dr += d * d;
      }
      for (int k = 0; k < 6; ++k) {
        double d = rho_of(c, 3 + k) * (y[k] - cams_prev[6 * (long)cam_idx[o] + k]);
        dr += d * d;
      }
    }
  }
  out->rmse_obs = valid > 0 ? sqrt(se / (double)valid) : 0.0;
  out->rmse_gt = (valid > 0 && z_true) ? sqrt(sg / (double)valid) : 0.0;
  out->objective = obj;
  out->primal_res = sqrt(pr);
  out->dual_res = sqrt(dr);
  out->n_invalid = invalid;
}

/* -------------------------------------- centralized LM (Sec. 2.2, Sec. 4) */

static double total_objective(const ora_config* c, long n_obs, const int* pt_idx,
                              const int* cam_idx, const double* z, const double* cams,
                              const double* pts) {
  double obj = 0.0;
  for (long o = 0; o < n_obs; ++o) {
    double zp[2];
    double depth = ora_project(c, pts + 3 * (long)pt_idx[o], cams + 6 * (long)cam_idx[o], zp);
    if (!(depth > c->eps_depth)) return INFINITY;
    double e0 = z[2 * o] - zp[0], e1 = z[2 * o + 1] - zp[1];
    obj += ora_loss(c->loss, c->loss_param, e0 * e0 + e1 * e1);
  }
  return obj;
}

int ora_dense_lm(const ora_config* c, int n_cams, int n_pts, long n_obs, const int* pt_idx,
                 const int* cam_idx, const double* z, double* cams, double* pts, int max_iters,
                 double* final_objective) {
  if (check_indices(n_cams, n_pts, n_obs, pt_idx, cam_idx) != 0) return -1;
  int N = 6 * n_cams + 3 * n_pts; /* unknowns: cameras first, then points */
  double* H = (double*)malloc((size_t)N * N * sizeof(double));
  double* g = (double*)malloc((size_t)N * sizeof(double));
  double* neg_g = (double*)malloc((size_t)N * sizeof(double));
  double* d = (double*)malloc((size_t)N * sizeof(double));
  double* cams_t = (double*)malloc((size_t)n_cams * 6 * sizeof(double));
  double* pts_t = (double*)malloc((size_t)n_pts * 3 * sizeof(double));
  if (!H || !g || !neg_g || !d || !cams_t || !pts_t) {
    free(H); free(g); free(neg_g); free(d); free(cams_t); free(pts_t);
    return -1;
  }
  double obj = total_objective(c, n_obs, pt_idx, cam_idx, z, cams, pts);
  double lambda = 1e-3;
  int it = 0;
  for (; it < max_iters; ++it) {
    if (obj < 1e-14 || lambda > 1e16) break;
    memset(H, 0, (size_t)N * N * sizeof(double));
    memset(g, 0, (size_t)N * sizeof(double));
    for (long o = 0; o < n_obs; ++o) {
      const double* x = pts + 3 * (long)pt_idx[o];
      const double* y = cams + 6 * (long)cam_idx[o];
      double zp[2], J[18];
      ora_project(c, x, y, zp);
      ora_jacobian(c, x, y, J);
      double e0 = z[2 * o] - zp[0], e1 = z[2 * o + 1] - zp[1];
      double w = ora_weight(c->loss, c->loss_param, e0 * e0 + e1 * e1);
      int col[9];
      for (int k = 0; k < 3; ++k) col[k] = 6 * n_cams + 3 * pt_idx[o] + k;
      for (int k = 0; k < 6; ++k) col[3 + k] = 6 * cam_idx[o] + k;
      for (int a = 0; a < 9; ++a) {
        g[col[a]] += -2.0 * w * (J[a] * e0 + J[9 + a] * e1);
        for (int b = 0; b < 9; ++b)
          H[(size_t)col[a] * N + col[b]] += 2.0 * w * (J[a] * J[b] + J[9 + a] * J[9 + b]);
      }
    }
    for (int a = 0; a < N; ++a) {
      H[(size_t)a * N + a] += lambda;
      neg_g[a] = -g[a];
    }
    if (ora_chol_solve(N, H, neg_g, d) != 0) {
      lambda *= 10.0;
      continue;
    }
    for (int j = 0; j < n_cams; ++j)
      for (int k = 0; k < 6; ++k) cams_t[6 * j + k] = cams[6 * j + k] + d[6 * j + k];
    for (int i = 0; i < n_pts; ++i)
      for (int k = 0; k < 3; ++k) pts_t[3 * i + k] = pts[3 * i + k] + d[6 * n_cams + 3 * i + k];
    double obj_t = total_objective(c, n_obs, pt_idx, cam_idx, z, cams_t, pts_t);
    if (obj_t < obj) {
      memcpy(cams, cams_t, (size_t)n_cams * 6 * sizeof(double));
      memcpy(pts, pts_t, (size_t)n_pts * 3 * sizeof(double));
      obj = obj_t;
      lambda /= 10.0;
    } else {
      lambda *= 10.0;
    }
  }
  if (final_objective) *final_objective = obj;
  free(H); free(g); free(neg_g); free(d); free(cams_t); free(pts_t);
  return it;
}

/* ------------------------------------------ generalized block step, Eq. (14) */

/* Eq. (14) for one block: misfits of its observations + dual terms + rho/2 penalties
 * of its copies.  Unknown order: point copies (3 each), then camera copies (6 each). */
double ora_block_objective(const ora_config* c, int np, int nc, int no, const int* opl, const int* ocl,
                           const double* z, const double* xbar, const double* ybar, const double* rx,
                           const double* sy, const double* X, const double* Y) {
  double L = 0.0;
  for (int k = 0; k < no; ++k) {
    double zp[2];
    double depth = ora_project(c, X + 3 * opl[k], Y + 6 * ocl[k], zp);
    if (!(depth > c->eps_depth)) return INFINITY;
    double e0 = z[2 * k] - zp[0], e1 = z[2 * k + 1] - zp[1];
    L += ora_loss(c->loss, c->loss_param, e0 * e0 + e1 * e1);
  }
  for (int p = 0; p < np; ++p)
    for (int a = 0; a < 3; ++a) {
      double d = X[3 * p + a] - xbar[3 * p + a];
      L += rx[3 * p + a] * d + 0.5 * rho_of(c, a) * d * d;
    }
  for (int q = 0; q < nc; ++q)
    for (int a = 0; a < 6; ++a) {
      double d = Y[6 * q + a] - ybar[6 * q + a];
      L += sy[6 * q + a] * d + 0.5 * rho_of(c, 3 + a) * d * d;
    }
  return L;
}

/* The local solve of Eq. (9) carried over to the block: each step linearises every
 * observation of the block, assembles the dense Gauss-Newton system of Eq. (14)
 *   g = sum_k -2 w_k J_k^T e_k + duals + diag(rho) (v - vbar),
 *   H = sum_k 2 w_k J_k^T J_k + diag(rho),
 * solves (H + lambda I) d = -g by Cholesky and accepts or rejects as the local
 * solve does (lambda starts at lm_lambda0 * mean diag H; noise bound summed over
 * the block's observations). */
void ora_block_solve(const ora_config* c, int np, int nc, int no, const int* opl, const int* ocl,
                     const double* z, const double* xbar, const double* ybar, const double* rx,
                     const double* sy, double* X, double* Y) {
  const int n = 3 * np + 6 * nc;
  double* H = (double*)malloc((size_t)n * n * sizeof(double));
  double* g = (double*)malloc((size_t)n * sizeof(double));
  double* neg_g = (double*)malloc((size_t)n * sizeof(double));
  double* d = (double*)malloc((size_t)n * sizeof(double));
  double* Xt = (double*)malloc((size_t)(3 * np + 1) * sizeof(double));
  double* Yt = (double*)malloc((size_t)(6 * nc + 1) * sizeof(double));
  if (!H || !g || !neg_g || !d || !Xt || !Yt) {
    free(H); free(g); free(neg_g); free(d); free(Xt); free(Yt);
    return;
  }
  double lambda = -1.0;
  double L_old = ora_block_objective(c, np, nc, no, opl, ocl, z, xbar, ybar, rx, sy, X, Y);
  for (int step = 0; step < c->inner_steps; ++step) {
    memset(H, 0, (size_t)n * n * sizeof(double));
    memset(g, 0, (size_t)n * sizeof(double));
    double noise_terms = 0.0;
    for (int k = 0; k < no; ++k) {
      const double* x = X + 3 * opl[k];
      const double* y = Y + 6 * ocl[k];
      double zp[2], J[18];
      double depth = ora_project(c, x, y, zp);
      if (!(depth > c->eps_depth)) continue; /* no misfit term at this linearisation point */
      double e0 = z[2 * k] - zp[0], e1 = z[2 * k + 1] - zp[1];
      double w = ora_weight(c->loss, c->loss_param, e0 * e0 + e1 * e1);
      ora_jacobian(c, x, y, J);
      int col[9];
      for (int a = 0; a < 3; ++a) col[a] = 3 * opl[k] + a;
      for (int a = 0; a < 6; ++a) col[3 + a] = 3 * np + 6 * ocl[k] + a;
      for (int a = 0; a < 9; ++a) {
        g[col[a]] += -2.0 * w * (J[a] * e0 + J[9 + a] * e1);
        for (int b = 0; b < 9; ++b)
          H[(size_t)col[a] * n + col[b]] += 2.0 * w * (J[a] * J[b] + J[9 + a] * J[9 + b]);
      }
      noise_terms += 2.0 * w * sqrt(e0 * e0 + e1 * e1) * (fabs(z[2 * k]) + fabs(z[2 * k + 1]));
    }
    for (int p = 0; p < np; ++p)
      for (int a = 0; a < 3; ++a) {
        int u = 3 * p + a;
        g[u] += rx[u] + rho_of(c, a) * (X[u] - xbar[u]);
        H[(size_t)u * n + u] += rho_of(c, a);
      }
    for (int q = 0; q < nc; ++q)
      for (int a = 0; a < 6; ++a) {
        int u = 3 * np + 6 * q + a;
        g[u] += sy[6 * q + a] + rho_of(c, 3 + a) * (Y[6 * q + a] - ybar[6 * q + a]);
        H[(size_t)u * n + u] += rho_of(c, 3 + a);
      }
    if (lambda < 0.0) {
      double tr = 0.0;
      for (int u = 0; u < n; ++u) tr += H[(size_t)u * n + u];
      lambda = c->lm_lambda0 * tr / (double)n;
    }
    for (int u = 0; u < n; ++u) {
      H[(size_t)u * n + u] += lambda;
      neg_g[u] = -g[u];
    }
    if (ora_chol_solve(n, H, neg_g, d) != 0) {
      lambda *= ORA_LM_INCREASE;
      continue;
    }
    double gd = 0.0, dd = 0.0;
    for (int u = 0; u < n; ++u) {
      gd += g[u] * d[u];
      dd += d[u] * d[u];
    }
    double pred = 0.5 * (lambda * dd - gd);
    int trust = 0;
    if (isfinite(L_old) && c->lm_model_tol > 0.0)
      trust = pred <= c->lm_model_tol * 0x1p-53 * (fabs(L_old) + noise_terms);
    for (int u = 0; u < 3 * np; ++u) Xt[u] = X[u] + d[u];
    for (int u = 0; u < 6 * nc; ++u) Yt[u] = Y[u] + d[3 * np + u];
    /* +inf when an observation of the block is behind its camera */
    double L_new = ora_block_objective(c, np, nc, no, opl, ocl, z, xbar, ybar, rx, sy, Xt, Yt);
    if (isfinite(L_new) && (trust || L_new < L_old)) {
      memcpy(X, Xt, (size_t)3 * np * sizeof(double));
      memcpy(Y, Yt, (size_t)6 * nc * sizeof(double));
      L_old = L_new;
      lambda = fmax(lambda / ORA_LM_DECREASE, c->lm_lambda_min);
    } else {
      lambda *= ORA_LM_INCREASE;
    }
  }
  free(H); free(g); free(neg_g); free(d); free(Xt); free(Yt);
}

int ora_block_iterate(const ora_config* c, int n_cams, int n_pts, long n_obs, const int* pt_idx,
                      const int* cam_idx, const double* z, const double* z_true, long n_blocks,
                      const long* obs_off, const long* blk_obs, const int* obs_lp, const int* obs_lc,
                      const long* pc_off, const int* pc_pt, const long* cc_off, const int* cc_cam,
                      double* pcopies, double* pduals, double* ccopies, double* cduals, double* cams,
                      double* pts, int iters, int nthreads, ora_metrics* metrics) {
  if (n_cams < 0 || n_pts < 0 || n_obs < 0 || n_blocks < 0 || iters < 0) return -1;
  if (check_indices(n_cams, n_pts, n_obs, pt_idx, cam_idx) != 0) return -1;
  const long n_pc = pc_off[n_blocks], n_cc = cc_off[n_blocks];
  for (long k = 0; k < n_pc; ++k)
    if (pc_pt[k] < 0 || pc_pt[k] >= n_pts) return -1;
  for (long k = 0; k < n_cc; ++k)
    if (cc_cam[k] < 0 || cc_cam[k] >= n_cams) return -1;
  if (obs_off[n_blocks] != n_obs) return -1;
#ifdef _OPENMP
  omp_set_num_threads(nthreads > 0 ? nthreads : omp_get_num_procs());
#else
  (void)nthreads;
#endif
  double* sum_x = (double*)calloc((size_t)n_pts * 3 + 1, sizeof(double));
  double* sum_y = (double*)calloc((size_t)n_cams * 6 + 1, sizeof(double));
  long* cnt_x = (long*)calloc((size_t)n_pts + 1, sizeof(long));
  long* cnt_y = (long*)calloc((size_t)n_cams + 1, sizeof(long));
  double* pts_prev = (double*)malloc(((size_t)n_pts * 3 + 1) * sizeof(double));
  double* cams_prev = (double*)malloc(((size_t)n_cams * 6 + 1) * sizeof(double));
  if (!sum_x || !sum_y || !cnt_x || !cnt_y || !pts_prev || !cams_prev) {
    free(sum_x); free(sum_y); free(cnt_x); free(cnt_y); free(pts_prev); free(cams_prev);
    return -1;
  }
  int status = 0;
  for (int it = 0; it < iters && status == 0; ++it) {
    memcpy(pts_prev, pts, (size_t)n_pts * 3 * sizeof(double));
    memcpy(cams_prev, cams, (size_t)n_cams * 6 * sizeof(double));

    /* Eq. (14): every block's subproblem, warm-started at its copies. */
#pragma omp parallel for schedule(dynamic, 16)
    for (long b = 0; b < n_blocks; ++b) {
      const int np = (int)(pc_off[b + 1] - pc_off[b]), nc = (int)(cc_off[b + 1] - cc_off[b]);
      const int no = (int)(obs_off[b + 1] - obs_off[b]);
      double* xbar = (double*)malloc((size_t)(3 * np + 1) * sizeof(double));
      double* ybar = (double*)malloc((size_t)(6 * nc + 1) * sizeof(double));
      double* zb = (double*)malloc((size_t)(2 * no + 1) * sizeof(double));
      if (!xbar || !ybar || !zb) {
        free(xbar); free(ybar); free(zb);
        continue;
      }
      for (int p = 0; p < np; ++p)
        for (int a = 0; a < 3; ++a) xbar[3 * p + a] = pts[3 * (long)pc_pt[pc_off[b] + p] + a];
      for (int q = 0; q < nc; ++q)
        for (int a = 0; a < 6; ++a) ybar[6 * q + a] = cams[6 * (long)cc_cam[cc_off[b] + q] + a];
      for (int k = 0; k < no; ++k) {
        zb[2 * k] = z[2 * blk_obs[obs_off[b] + k]];
        zb[2 * k + 1] = z[2 * blk_obs[obs_off[b] + k] + 1];
      }
      ora_block_solve(c, np, nc, no, obs_lp + obs_off[b], obs_lc + obs_off[b], zb, xbar, ybar,
                      pduals + 3 * pc_off[b], cduals + 6 * cc_off[b], pcopies + 3 * pc_off[b],
                      ccopies + 6 * cc_off[b]);
      free(xbar); free(ybar); free(zb);
    }

    /* Eqs. (10)-(11) over copies: x_i = mean over the copies of point i of (copy + r / rho_x),
       y_j likewise, with the old duals. */
    memset(sum_x, 0, (size_t)n_pts * 3 * sizeof(double));
    memset(cnt_x, 0, (size_t)n_pts * sizeof(long));
    for (long k = 0; k < n_pc; ++k) {
      long i = pc_pt[k];
      for (int a = 0; a < 3; ++a) sum_x[3 * i + a] += pcopies[3 * k + a] + pduals[3 * k + a] / rho_of(c, a);
      cnt_x[i] += 1;
    }
    for (long i = 0; i < n_pts; ++i)
      if (cnt_x[i] > 0)
        for (int a = 0; a < 3; ++a) pts[3 * i + a] = sum_x[3 * i + a] / (double)cnt_x[i];
    memset(sum_y, 0, (size_t)n_cams * 6 * sizeof(double));
    memset(cnt_y, 0, (size_t)n_cams * sizeof(long));
    for (long k = 0; k < n_cc; ++k) {
      long j = cc_cam[k];
      for (int a = 0; a < 6; ++a) sum_y[6 * j + a] += ccopies[6 * k + a] + cduals[6 * k + a] / rho_of(c, 3 + a);
      cnt_y[j] += 1;
    }
    for (long j = 0; j < n_cams; ++j)
      if (cnt_y[j] > 0)
        for (int a = 0; a < 6; ++a) cams[6 * j + a] = sum_y[6 * j + a] / (double)cnt_y[j];

    /* Eqs. (12)-(13) per copy, with the new consensus. */
    for (long k = 0; k < n_pc; ++k)
      for (int a = 0; a < 3; ++a)
        pduals[3 * k + a] += rho_of(c, a) * (pcopies[3 * k + a] - pts[3 * (long)pc_pt[k] + a]);
    for (long k = 0; k < n_cc; ++k)
      for (int a = 0; a < 6; ++a)
        cduals[6 * k + a] += rho_of(c, 3 + a) * (ccopies[6 * k + a] - cams[6 * (long)cc_cam[k] + a]);
  }
  if (metrics && status == 0) {
    /* reprojection terms at consensus as ora_eval; residuals over the copies */
    ora_eval(c, n_cams, n_pts, n_obs, pt_idx, cam_idx, z, z_true, NULL, cams, pts, NULL, NULL, metrics);
    double pr = 0.0, dr = 0.0;
    for (long k = 0; k < n_pc; ++k)
      for (int a = 0; a < 3; ++a) {
        long u = 3 * (long)pc_pt[k] + a;
        double d = pcopies[3 * k + a] - pts[u];
        pr += d * d;
        if (iters > 0) {
          double q = rho_of(c, a) * (pts[u] - pts_prev[u]);
          dr += q * q;
        }
      }
    for (long k = 0; k < n_cc; ++k)
      for (int a = 0; a < 6; ++a) {
        long u = 6 * (long)cc_cam[k] + a;
        double d = ccopies[6 * k + a] - cams[u];
        pr += d * d;
        if (iters > 0) {
          double q = rho_of(c, 3 + a) * (cams[u] - cams_prev[u]);
          dr += q * q;
        }
      }
    metrics->primal_res = sqrt(pr);
    metrics->dual_res = sqrt(dr);
  }
  free(sum_x); free(sum_y); free(cnt_x); free(cnt_y); free(pts_prev); free(cams_prev);
  return status;
}
