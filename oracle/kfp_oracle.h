/*
 * kfp_oracle.h -- plain FP64 CPU oracle for Schwarz waveform relaxation (SWR)
 * applied to the Kolmogorov equation  u_t + v u_x - u_vv = f.
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists so that the tests, the smoke
 * check and the CPU-baseline leg of the benchmark can check the CUDA path
 * against an obviously correct implementation.  The product path never links,
 * loads or calls it, and it shares no code with the CUDA path.
 *
 * What it computes (paper: Section 2 for the problem and the two transmission
 * conditions; Section 6.3 for the interface variables lambda_1, lambda_2, the
 * operators Q_1, Q_2, the iteration SWR1-SWR4 and the stopping criterion; the
 * Remark after the criterion for the parallel (Jacobi) form used here).
 *
 * Discretisation (the paper leaves it open for the general case; its own test
 * scheme in Section 6.2 is not used):
 *   grid        x_m = x0 + m hx (m = 0..nx), v_i = v0 + i hv (i = 0..nv),
 *               t^n = n dt (n = 0..nt); nx, nv count intervals.
 *   transport   explicit first-order upwind by the sign of v_i, at t^n.
 *   diffusion   implicit Euler, centred second difference in v:
 *               (1+2r) u_i - r u_{i-1} - r u_{i+1} = T_i + dt f_i, r = dt/hv^2.
 *   x boundary  inflow Dirichlet data (m = 0 where v_i > 0, m = nx where v_i < 0),
 *               or periodic (periodic_x).
 *   v boundary  Dirichlet data at v0 and v1, or homogeneous Neumann half-cell rows
 *               (1+2r) u_0 - 2r u_1 = R_0 and (1+2r) u_nv - 2r u_{nv-1} = R_nv (neumann_v).
 *   Robin rows  half-cell finite-volume rows for (p + d/dv) u = lambda_1 at the
 *               lower strip's top node and (q - d/dv) u = lambda_2 at the upper
 *               strip's bottom node.
 * Scheme 1 (Section 6.2, Lie splitting with P1 finite elements in v):
 *   step 1      (M/dt + S) w = M (u^n/dt + f^{n+1}) per column, M and S the P1 mass and
 *               stiffness matrices (exact integrals; zero flux is the natural condition
 *               at v0 and v1); Robin ends add p (top) or q (bottom) to the end row's
 *               diagonal and lambda to its right-hand side; Dirichlet ends set w = lambda.
 *   step 2      u^{n+1} = w - c_i (w_m - w_{m-1}) for v_i > 0 and w - c_i (w_{m+1} - w_m) for
 *               v_i < 0, c_i = |v_i| dt / hx (periodic in x).
 *   traces      from w: Dirichlet w; Robin without overlap (p+q) w - lambda_in; Robin with
 *               overlap, p w (resp. q w) minus the half-row residual of the strip that
 *               holds the node inside it (the discrete flux that makes the converged
 *               iterate the single-domain solution).
 * Every call runs on the calling thread, allocates with malloc and frees before
 * returning.  Return value 0 = success, negative = invalid input (see below).
 */
#ifndef KFP_ORACLE_H
#define KFP_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double x0, x1, v0, v1, dt;
  int nx, nv, nt;      /* numbers of intervals in x, v and time steps */
  int nstrips;         /* S >= 1 strips in v; S divides nv */
  int overlap;         /* overlap in cells, 0 <= overlap < nv/S */
  int robin;           /* 0: classical (Dirichlet) transmission, 1: optimized (Robin) */
  const double* p;     /* [S-1] Robin p_j of interface j (lower strip's top, p + d/dv) */
  const double* q;     /* [S-1] Robin q_j of interface j (upper strip's bottom, q - d/dv) */
  int gauss_seidel;    /* 0: parallel form (every strip uses iterate k-1, Remark of Section
                          6.3); 1: serial form SWR1-SWR4 -- strips in increasing order, each
                          taking lambda_2 from the strip below of the same iteration */
  int neumann_v;       /* 1: homogeneous Neumann rows at v0 and v1 (the model problem of
                          Section 6.1) instead of Dirichlet data; bc_v is ignored */
  int periodic_x;      /* 1: x periodic (Section 6.1): nodes m = 0..nx-1 are the unknowns,
                          node nx repeats node 0; bc_xin is ignored */
  int scheme;          /* 0: implicit Euler in v with upwind transport at t^n (finite volumes,
                          the default); 1: the Lie splitting of Section 6.2 -- implicit Euler
                          with P1 finite elements in v over dt, then explicit upwind transport
                          over dt (model problem only: needs periodic_x and neumann_v) */
} kfo_desc;

typedef struct {
  const double* u0;      /* [nv+1][nx+1] initial data */
  int nforce;            /* number of separable terms of f */
  const double* f_time;  /* [nforce][nt+1]   a_r(t^n) */
  const double* f_space; /* [nforce][nv+1][nx+1]  F_r(x_m, v_i); f = sum_r a_r F_r */
  const double* bc_xin;  /* [nt+1][2][nv+1] inflow data at x0 (0) and x1 (1); NULL = 0 */
  const double* bc_v;    /* [nt+1][2][nx+1] data at v0 (0) and v1 (1); NULL = 0 */
} kfo_problem;

/* Error codes. */
#define KFO_OK 0
#define KFO_EINVAL (-1)
#define KFO_ECFL (-2)
#define KFO_ENOMEM (-3)

/* Validate a descriptor (grid, strip layout, CFL, Robin parameters). */
int kfo_validate(const kfo_desc* d);

/* Node range [lo_s, hi_s] of every strip (arrays of length S). */
int kfo_strip_layout(const kfo_desc* d, int* lo, int* hi);

/*
 * One parallel SWR iteration.  Trace arrays have shape [S-1][2][nt][nx+1]:
 * [j][0][n-1][m] = lambda_1 of interface j at t^n (data at the lower strip's
 * top node beta_j), [j][1][n-1][m] = lambda_2 (data at the upper strip's
 * bottom node alpha_j).  lam_in holds iterate k-1, lam_out receives iterate k.
 * bands (may be NULL) receives [S-1][2][nt][overlap+1][nx+1]: the lower (0)
 * and upper (1) strip's values on nodes alpha_j..beta_j.  u_T (may be NULL)
 * receives the assembled solution at t = T, [nv+1][nx+1], node i taken from
 * the lower strip of interface j when i <= I_j and from the upper one otherwise.
 */
int kfo_swr_iteration(const kfo_desc* d, const kfo_problem* pb, const double* lam_in,
                      double* lam_out, double* bands, double* u_T);

/* Interface norms of one iterate: e_mis = max |u_j - u_{j+1}| over the bands,
 * e_chg = max |lam_new - lam_old|, j_l2 = dt hx sum (u_j - u_{j+1})^2. */
int kfo_interface_norms(const kfo_desc* d, const double* bands, const double* lam_new,
                        const double* lam_old, double* e_mis, double* e_chg, double* j_l2);

/*
 * Iterate until the chosen norm (tol_kind 0: e_chg, 1: e_mis) is below tol or
 * max_iters iterations ran.  lam holds lambda^0 on entry and the last iterate
 * on exit.  hist (may be NULL) receives max_iters rows of (e_mis, e_chg, j_l2).
 * *iters receives the number of iterations run.  u_T as above (last iterate).
 * With periodic_x, column nx of lam is set to column 0 on entry (node nx repeats node 0).
 */
int kfo_swr_solve(const kfo_desc* d, const kfo_problem* pb, double* lam, int max_iters,
                  double tol, int tol_kind, int* iters, double* hist, double* u_T);

/* Single-domain solve (the same scheme with one strip): u_T [nv+1][nx+1];
 * u_all (may be NULL) receives every time level, [nt+1][nv+1][nx+1]. */
int kfo_monolithic(const kfo_desc* d, const kfo_problem* pb, double* u_T, double* u_all);

/*
 * Discrete adjoint (gradient) of K parallel SWR iterations with Robin transmission
 * and no overlap.  Objective: J = dt hx sum_j sum_{n=1..nt} sum_m (u_j - u_{j+1})^2,
 * the squared L2 mismatch on the interface nodes of the K-th iterate (u_j is the
 * lower strip of interface j).  lam0 (may be NULL = 0) is lambda^0.  Outputs J and
 * dJ/dp_j, dJ/dq_j for j = 0..S-2 (grad_p, grad_q of length S-1).  The forward run
 * keeps the interface-node values of every iterate; the adjoint solves the
 * transposed implicit-Euler systems backward in time and the transposed exchange
 * backward over the iterations.  Returns KFO_EINVAL unless robin and overlap == 0.
 */
int kfo_swr_adjoint(const kfo_desc* d, const kfo_problem* pb, const double* lam0, int K, double* J,
                    double* grad_p, double* grad_q);

/* Plain Thomas algorithm for a tridiagonal system of size n (exported for the
 * oracle's own unit tests): a = sub-diagonal (a[0] unused), b = diagonal,
 * c = super-diagonal (c[n-1] unused), d = right-hand side, x = solution. */
int kfo_thomas(int n, const double* a, const double* b, const double* c, const double* d,
               double* x);

#ifdef __cplusplus
}
#endif
#endif
