/*
 * Plain FP64 CPU oracle for distributed bundle adjustment by consensus ADMM
 * (Ramamurthy et al., "Distributed Bundle Adjustment", arXiv 1708.07954).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA path; it is deliberately slow and
 * written to be checked against the paper by eye.
 *
 * Conventions (readings of the paper, each also listed in the design notes):
 *  - camera y = (alpha, beta, gamma, tx, ty, tz), R = Rz(gamma) Ry(beta) Rx(alpha)
 *    (Sec. 2.1), active right-handed rotations, z~ = R x + t (world to camera);
 *  - pixel z = f * z~_{1,2} / z~_3 + (cx, cy)  (Eq. 1 with K = diag(f,f,1)
 *    applied and a known principal point);
 *  - equation numbers follow the paper's LaTeX order: (1) projection, (2) BA,
 *    (5)-(7) split problem, (8) augmented Lagrangian, (9) local subproblem,
 *    (10)/(11) point/camera consensus, (12)/(13) dual updates, (14) blocks;
 *  - misfit phi_m(e) = rho(s), s = |e|^2:  l2: s;  Huber(d): s if s <= d^2 else
 *    2 d sqrt(s) - d^2;  Student's t(nu): nu log(1 + s/nu);  phi_a = |.|^2;
 *  - observation vectors are 9 values: point part x (3) then camera part y (6);
 *    duals likewise: r (3) then s (6).
 */
#ifndef DBA_ORACLE_H
#define DBA_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORA_LOSS_L2 = 0, ORA_LOSS_HUBER = 1, ORA_LOSS_STUDENT_T = 2 };

typedef struct {
  double focal, cx, cy;
  int loss;             /* ORA_LOSS_* */
  double loss_param;    /* Huber delta (px) or Student's t nu */
  double rho_x, rho_y;  /* consensus penalties, Eq. (8): points; camera translations */
  double rho_angle;     /* camera Euler angles; <= 0: rho_y (the paper's single camera penalty) */
  int inner_steps;      /* damped Gauss-Newton steps per local solve */
  double lm_lambda0;    /* initial damping = lm_lambda0 * mean diag of H */
  double lm_lambda_min; /* lower clamp of the damping */
  double eps_depth;     /* a copy with z~_3 <= eps_depth is rejected (Thm. 1 proof, A4) */
  double lm_model_tol;  /* kappa: a step whose predicted decrease is <= kappa u (|L| + 2 w |e| (|z1|+|z2|)),
                           the rounding noise of the objective (u = 2^-53), is accepted without
                           the objective comparison; 0 disables */
  int local_solver;     /* ORA_SOLVER_GN: damped Gauss-Newton; ORA_SOLVER_LBFGS: L-BFGS (Sec. 3.1) */
} ora_config;

enum { ORA_SOLVER_GN = 0, ORA_SOLVER_LBFGS = 1 };
/* L-BFGS constants; macros only so that the tests can build deliberately wrong oracles
 * and check that the step-wise pins reject them. */
#ifndef ORA_LBFGS_MEMORY
#define ORA_LBFGS_MEMORY 4
#endif
#ifndef ORA_LBFGS_HALVINGS
#define ORA_LBFGS_HALVINGS 10
#endif
#ifndef ORA_LBFGS_ARMIJO
#define ORA_LBFGS_ARMIJO 1e-4
#endif

typedef struct {
  double rmse_obs;   /* sqrt(mean |z - f(x_i, y_j)|^2) at consensus */
  double rmse_gt;    /* sqrt(mean |f(x_i, y_j) - z_true|^2) at consensus (if z_true given) */
  double objective;  /* sum phi_m(z - f(x_i, y_j)) at consensus, Eq. (BA) with phi_m */
  double primal_res; /* sqrt(sum |copy - consensus|^2) */
  double dual_res;   /* sqrt(sum over copies of rho^2 |consensus - previous consensus|^2) */
  long n_invalid;    /* observations whose consensus depth is <= eps_depth (excluded) */
} ora_metrics;

/* Sec. 2.1 forward model. */
void ora_rotation(const double y[6], double R[9]);
/* Returns z~_3 (depth); writes the pixel into zout. */
double ora_project(const ora_config* c, const double x[3], const double y[6], double zout[2]);
/* 2x9 Jacobian of the pixel with respect to (x, y), row-major. */
void ora_jacobian(const ora_config* c, const double x[3], const double y[6], double J[18]);

double ora_loss(int kind, double param, double s);
double ora_weight(int kind, double param, double s);

/* Local objective of Eq. (9) at v = (x, y); +INFINITY when z~_3 <= eps_depth. */
double ora_local_objective(const ora_config* c, const double z[2], const double xbar[3],
                           const double ybar[6], const double dual[9], const double v[9]);
/* Local solve of Eq. (9): inner_steps damped Gauss-Newton steps from v (in/out). */
void ora_local_solve(const ora_config* c, const double z[2], const double xbar[3],
                     const double ybar[6], const double dual[9], double v[9]);

/* Local solve of Eq. (9) by L-BFGS (Sec. 3.1 names it for the Huber loss): inner_steps
 * iterations in the coordinates u = sqrt(rho) (v - vbar), memory ORA_LBFGS_MEMORY, two-loop
 * recursion with H0 = (s^T y / y^T y) I (I before the first pair), backtracking Armijo line
 * search from step 1 (constant ORA_LBFGS_ARMIJO, at most ORA_LBFGS_HALVINGS halvings).  v in/out. */
void ora_local_solve_lbfgs(const ora_config* c, const double z[2], const double xbar[3],
                           const double ybar[6], const double dual[9], double v[9]);

/* Solves A x = b for symmetric positive definite A (n x n, row-major, copied). 0 on success. */
int ora_chol_solve(int n, const double* A, const double* b, double* x);

/* copies[9l] = broadcast of (pts, cams); duals[9l] = 0. */
void ora_admm_init(int n_cams, int n_pts, long n_obs, const int* pt_idx, const int* cam_idx,
                   const double* cams, const double* pts, double* copies, double* duals);
/* Runs `iters` ADMM iterations, Eqs. (9)-(13), in place.  Observations in caller order.
 * z_true may be NULL.  metrics (nullable) receives the state after the last iteration.
 * nthreads <= 0 uses every processor.  Returns 0, or -1 on bad input. */
int ora_admm_iterate(const ora_config* c, int n_cams, int n_pts, long n_obs, const int* pt_idx,
                     const int* cam_idx, const double* z, const double* z_true, double* copies,
                     double* duals, double* cams, double* pts, int iters, int nthreads,
                     ora_metrics* metrics);
/* Metrics at consensus; cams_prev/pts_prev may be NULL (dual_res = 0), copies may be
 * NULL (primal_res = 0). */
void ora_eval(const ora_config* c, int n_cams, int n_pts, long n_obs, const int* pt_idx,
              const int* cam_idx, const double* z, const double* z_true, const double* copies,
              const double* cams, const double* pts, const double* cams_prev,
              const double* pts_prev, ora_metrics* out);

/* Centralized robust Levenberg-Marquardt over all 6m+3n unknowns with dense normal
 * equations (tiny scenes only).  Stops when the objective < 1e-14 or the damping
 * exceeds 1e16 (Sec. 4), or after max_iters.  Returns iterations done, -1 on error. */
int ora_dense_lm(const ora_config* c, int n_cams, int n_pts, long n_obs, const int* pt_idx,
                 const int* cam_idx, const double* z, double* cams, double* pts, int max_iters,
                 double* final_objective);

/* ------------------------------------------ generalized block step, Eq. (14) */
/* A block holds np point copies, nc camera copies and no observations; observation k
 * links local point opl[k] and local camera ocl[k] with pixel z[2k..2k+1].  Arrays per
 * copy: xbar/rx/X 3 values per point copy, ybar/sy/Y 6 per camera copy (consensus,
 * unscaled dual, copy).  The block objective is Eq. (14): the sum of the misfits of
 * the block's observations plus, per copy, the dual term and the rho/2 penalty;
 * +INFINITY when an observation is behind its camera. */
double ora_block_objective(const ora_config* c, int np, int nc, int no, const int* opl, const int* ocl,
                           const double* z, const double* xbar, const double* ybar, const double* rx,
                           const double* sy, const double* X, const double* Y);
/* inner_steps damped Gauss-Newton steps on Eq. (14) over all 3 np + 6 nc unknowns of
 * the block (dense normal matrix, Cholesky), with the local solve's damping, acceptance
 * and noise rules; X, Y in/out. */
void ora_block_solve(const ora_config* c, int np, int nc, int no, const int* opl, const int* ocl,
                     const double* z, const double* xbar, const double* ybar, const double* rx,
                     const double* sy, double* X, double* Y);
/* ADMM with block subproblems.  Block b owns observations blk_obs[obs_off[b] .. obs_off[b+1])
 * (ids into the caller's arrays; obs_lp/obs_lc give their local point/camera index, aligned
 * with blk_obs), point copies pc_off[b] .. pc_off[b+1] of points pc_pt[.], camera copies
 * cc_off[b] .. cc_off[b+1] of cameras cc_cam[.].  pcopies/pduals: 3 per point copy,
 * ccopies/cduals: 6 per camera copy.  Each iteration: block solves (Eq. 14), consensus as
 * the mean over copies of copy + dual / rho (Eqs. 10-11 over copies, old duals), dual
 * ascent (Eqs. 12-13).  metrics (nullable): as ora_eval, with the primal residual over the
 * copies and the dual residual summed over the copies.  Returns 0, or -1 on bad input. */
int ora_block_iterate(const ora_config* c, int n_cams, int n_pts, long n_obs, const int* pt_idx,
                      const int* cam_idx, const double* z, const double* z_true, long n_blocks,
                      const long* obs_off, const long* blk_obs, const int* obs_lp, const int* obs_lc,
                      const long* pc_off, const int* pc_pt, const long* cc_off, const int* cc_cam,
                      double* pcopies, double* pduals, double* ccopies, double* cduals, double* cams,
                      double* pts, int iters, int nthreads, ora_metrics* metrics);

#ifdef __cplusplus
}
#endif
#endif
