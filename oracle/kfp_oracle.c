/*
 * kfp_oracle.c -- plain FP64 CPU oracle for Schwarz waveform relaxation on the
 * Kolmogorov equation.  TEST INFRASTRUCTURE ONLY (tests, smoke check and the
 * benchmark's CPU-baseline leg); the product path never uses it.
 *
 * It is written to be read against the paper, not to be fast: every strip is
 * solved on its own over the whole time window (Section 6.3, SWR1 and SWR3),
 * the interface variables lambda_1 = Q_1 u_2 and lambda_2 = Q_2 u_1 are formed
 * from the new iterates (SWR2 and SWR4) in the parallel form of the Remark in
 * Section 6.3 (every strip uses iterate k-1), and convergence is measured by
 * the L-infinity mismatch of neighbouring strips on the overlap (criterion
 * "error" of Section 6.3).  Each time step of a strip assembles, for every
 * x-column, the tridiagonal implicit-Euler system in v and solves it by the
 * plain Thomas algorithm, with no prefactoring or reuse between columns.
 *
 * Readings of the paper used here (Section 2 and Section 6.3):
 *  - Each subdomain takes its transmission data at its own interface end: the
 *    lower strip of interface j at beta_j, the upper one at alpha_j.
 *  - Q_1 = p + d/dv at the lower strip's top, Q_2 = q - d/dv at the upper
 *    strip's bottom (classical: both the identity).
 *  - A Robin end row is the half-cell finite-volume row
 *      top:    (1 + 2r + 2 p dt/hv) u_b - 2r u_{b-1} = R_b + (2 dt/hv) lambda_1
 *      bottom: (1 + 2r + 2 q dt/hv) u_a - 2r u_{a+1} = R_a + (2 dt/hv) lambda_2
 *    with R = transport + dt f at the same node.
 *  - The outgoing Robin trace uses the centred difference for d/dv where the
 *    node is interior to the strip (overlap >= 1) and, where the node is the
 *    strip's own Robin row (overlap 0), the derivative implied by that row's
 *    condition, which gives lambda_out = (p + q) u - lambda_in.
 *  - Row precedence: v boundary, then x inflow, then interface, then interior.
 */
#include "kfp_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Geometry of the decomposition (Section 2: Omega_1, Omega_2 split in v;    */
/* Section 6.3: Omega_1 = [.., beta], Omega_2 = [alpha, ..], L = beta-alpha). */
/* ------------------------------------------------------------------------ */

static int cells_per_strip(const kfo_desc* d) { return d->nv / d->nstrips; }
/* centre node I_j of interface j = 0..S-2 */
static int centre_node(const kfo_desc* d, int j) { return (j + 1) * cells_per_strip(d); }
static int alpha_node(const kfo_desc* d, int j) { return centre_node(d, j) - d->overlap / 2; }
static int beta_node(const kfo_desc* d, int j) { return alpha_node(d, j) + d->overlap; }
static int strip_lo(const kfo_desc* d, int s) { return s == 0 ? 0 : alpha_node(d, s - 1); }
static int strip_hi(const kfo_desc* d, int s) {
  return s == d->nstrips - 1 ? d->nv : beta_node(d, s);
}

static double hx_of(const kfo_desc* d) { return (d->x1 - d->x0) / d->nx; }
static double hv_of(const kfo_desc* d) { return (d->v1 - d->v0) / d->nv; }
static double v_node(const kfo_desc* d, int i) { return d->v0 + i * hv_of(d); }

int kfo_validate(const kfo_desc* d) {
  if (!d) return KFO_EINVAL;
  if (d->nx < 1 || d->nv < 2 || d->nt < 1 || d->nstrips < 1) return KFO_EINVAL;
  if (!(d->x1 > d->x0) || !(d->v1 > d->v0) || !(d->dt > 0)) return KFO_EINVAL;
  if (d->nv % d->nstrips != 0) return KFO_EINVAL;
  if (d->periodic_x && d->nx < 2) return KFO_EINVAL;
  if (d->scheme != 0 && !(d->scheme == 1 && d->periodic_x && d->neumann_v)) return KFO_EINVAL;
  if (d->nstrips > 1) {
    int w = cells_per_strip(d);
    if (w < 2 || d->overlap < 0 || d->overlap >= w) return KFO_EINVAL;
    if (d->robin) {
      if (!d->p || !d->q) return KFO_EINVAL;
      for (int j = 0; j < d->nstrips - 1; ++j)
        if (!(d->p[j] > 0) || !(d->q[j] > 0)) return KFO_EINVAL;
    }
  }
  /* CFL of the explicit upwind step: |v_i| dt / hx <= 1 at every node. */
  for (int i = 0; i <= d->nv; ++i)
    if (fabs(v_node(d, i)) * d->dt / hx_of(d) > 1.0) return KFO_ECFL;
  return KFO_OK;
}

int kfo_strip_layout(const kfo_desc* d, int* lo, int* hi) {
  int rc = kfo_validate(d);
  if (rc) return rc;
  for (int s = 0; s < d->nstrips; ++s) {
    lo[s] = strip_lo(d, s);
    hi[s] = strip_hi(d, s);
  }
  return KFO_OK;
}

int kfo_thomas(int n, const double* a, const double* b, const double* c, const double* d,
               double* x) {
  double* cp = (double*)malloc(sizeof(double) * (size_t)n);
  double* dp = (double*)malloc(sizeof(double) * (size_t)n);
  if (!cp || !dp) {
    free(cp);
    free(dp);
    return KFO_ENOMEM;
  }
  cp[0] = c[0] / b[0];
  dp[0] = d[0] / b[0];
  for (int i = 1; i < n; ++i) {
    double den = b[i] - a[i] * cp[i - 1];
    cp[i] = c[i] / den;
    dp[i] = (d[i] - a[i] * dp[i - 1]) / den;
  }
  x[n - 1] = dp[n - 1];
  for (int i = n - 2; i >= 0; --i) x[i] = dp[i] - cp[i] * x[i + 1];
  free(cp);
  free(dp);
  return KFO_OK;
}

/* ------------------------------------------------------------------------ */
/* One strip over the whole window (SWR1 / SWR3 of Section 6.3).            */
/* ------------------------------------------------------------------------ */

typedef struct {
  const double* lam_bot; /* lambda_2 of interface s-1 at this strip's bottom, [nt][nx+1] */
  const double* lam_top; /* lambda_1 of interface s at this strip's top, [nt][nx+1] */
  double* out_bot;       /* lambda_1 of interface s-1 = Q_1 u_s at beta_{s-1} */
  double* out_top;       /* lambda_2 of interface s   = Q_2 u_s at alpha_s */
  double* band_bot;      /* u_s on alpha_{s-1}..beta_{s-1}, [nt][ov+1][nx+1] */
  double* band_top;      /* u_s on alpha_s..beta_s */
  double* u_all;         /* optional: every time level of the strip [nt+1][L][nx+1] */
} strip_io;

/* Right-hand side of the explicit part at node (i, m) for time level n+1:
 * upwind transport of u^n plus dt times the forcing at t^{n+1}. */
static double explicit_part(const kfo_desc* d, const kfo_problem* pb, const double* un, int lo,
                            int i, int m, int n) {
  const int nxp = d->nx + 1;
  const double* row = un + (size_t)(i - lo) * nxp;
  const double vi = v_node(d, i);
  const double cfl = vi * d->dt / hx_of(d);
  /* upwind neighbours; periodic x wraps the unknowns m = 0..nx-1 */
  const int mm = d->periodic_x ? (m - 1 + d->nx) % d->nx : m - 1;
  const int mp = d->periodic_x ? (m + 1) % d->nx : m + 1;
  double T;
  if (vi > 0)
    T = row[m] - cfl * (row[m] - row[mm]);
  else if (vi < 0)
    T = row[m] - cfl * (row[mp] - row[m]);
  else
    T = row[m];
  double f = 0.0;
  for (int r = 0; r < pb->nforce; ++r)
    f += pb->f_time[(size_t)r * (d->nt + 1) + (n + 1)] *
         pb->f_space[((size_t)r * (d->nv + 1) + i) * nxp + m];
  return T + d->dt * f;
}

static int solve_strip(const kfo_desc* d, const kfo_problem* pb, int s, const strip_io* io,
                       double* u_T_strip) {
  const int S = d->nstrips, nx = d->nx, nxp = d->nx + 1, nt = d->nt, ov = d->overlap;
  const int lo = strip_lo(d, s), hi = strip_hi(d, s), L = hi - lo + 1;
  const double hv = hv_of(d), r = d->dt / (hv * hv);
  const int has_bot = s > 0, has_top = s < S - 1;
  const double p_top = (has_top && d->robin) ? d->p[s] : 0.0;
  const double q_bot = (has_bot && d->robin) ? d->q[s - 1] : 0.0;

  double* un = (double*)malloc(sizeof(double) * (size_t)L * nxp);
  double* unew = (double*)malloc(sizeof(double) * (size_t)L * nxp);
  double* a = (double*)malloc(sizeof(double) * (size_t)L);
  double* b = (double*)malloc(sizeof(double) * (size_t)L);
  double* c = (double*)malloc(sizeof(double) * (size_t)L);
  double* R = (double*)malloc(sizeof(double) * (size_t)L);
  double* x = (double*)malloc(sizeof(double) * (size_t)L);
  if (!un || !unew || !a || !b || !c || !R || !x) {
    free(un); free(unew); free(a); free(b); free(c); free(R); free(x);
    return KFO_ENOMEM;
  }
  for (int l = 0; l < L; ++l)
    memcpy(un + (size_t)l * nxp, pb->u0 + (size_t)(lo + l) * nxp, sizeof(double) * nxp);

  if (d->periodic_x) /* node nx repeats node 0 */
    for (int l = 0; l < L; ++l) un[(size_t)l * nxp + nx] = un[(size_t)l * nxp + 0];
  if (io->u_all) memcpy(io->u_all, un, sizeof(double) * (size_t)L * nxp);
  const int mlast = d->periodic_x ? nx - 1 : nx;
  for (int n = 0; n < nt; ++n) {
    for (int m = 0; m <= mlast; ++m) {
      for (int l = 0; l < L; ++l) {
        const int i = lo + l;
        const double vi = v_node(d, i);
        a[l] = 0.0; b[l] = 1.0; c[l] = 0.0;
        if (i == 0 && !d->neumann_v) { /* v boundary at v0 */
          R[l] = pb->bc_v ? pb->bc_v[((size_t)(n + 1) * 2 + 0) * nxp + m] : 0.0;
        } else if (i == d->nv && !d->neumann_v) { /* v boundary at v1 */
          R[l] = pb->bc_v ? pb->bc_v[((size_t)(n + 1) * 2 + 1) * nxp + m] : 0.0;
        } else if (!d->periodic_x && m == 0 && vi > 0) { /* inflow at x0 */
          R[l] = pb->bc_xin ? pb->bc_xin[((size_t)(n + 1) * 2 + 0) * (d->nv + 1) + i] : 0.0;
        } else if (!d->periodic_x && m == nx && vi < 0) { /* inflow at x1 */
          R[l] = pb->bc_xin ? pb->bc_xin[((size_t)(n + 1) * 2 + 1) * (d->nv + 1) + i] : 0.0;
        } else if (i == 0) { /* zero-flux half cell at v0 */
          b[l] = 1.0 + 2.0 * r;
          c[l] = -2.0 * r;
          R[l] = explicit_part(d, pb, un, lo, i, m, n);
        } else if (i == d->nv) { /* zero-flux half cell at v1 */
          a[l] = -2.0 * r;
          b[l] = 1.0 + 2.0 * r;
          R[l] = explicit_part(d, pb, un, lo, i, m, n);
        } else if (has_top && i == hi) { /* Q_1 u_s = lambda_1 at beta_s */
          const double lam = io->lam_top ? io->lam_top[(size_t)n * nxp + m] : 0.0;
          if (d->robin) {
            a[l] = -2.0 * r;
            b[l] = 1.0 + 2.0 * r + 2.0 * p_top * d->dt / hv;
            R[l] = explicit_part(d, pb, un, lo, i, m, n) + (2.0 * d->dt / hv) * lam;
          } else {
            R[l] = lam;
          }
        } else if (has_bot && i == lo) { /* Q_2 u_s = lambda_2 at alpha_{s-1} */
          const double lam = io->lam_bot ? io->lam_bot[(size_t)n * nxp + m] : 0.0;
          if (d->robin) {
            b[l] = 1.0 + 2.0 * r + 2.0 * q_bot * d->dt / hv;
            c[l] = -2.0 * r;
            R[l] = explicit_part(d, pb, un, lo, i, m, n) + (2.0 * d->dt / hv) * lam;
          } else {
            R[l] = lam;
          }
        } else { /* interior implicit-Euler row */
          a[l] = -r;
          b[l] = 1.0 + 2.0 * r;
          c[l] = -r;
          R[l] = explicit_part(d, pb, un, lo, i, m, n);
        }
      }
      int rc = kfo_thomas(L, a, b, c, R, x);
      if (rc) {
        free(un); free(unew); free(a); free(b); free(c); free(R); free(x);
        return rc;
      }
      for (int l = 0; l < L; ++l) unew[(size_t)l * nxp + m] = x[l];
    }
    if (d->periodic_x)
      for (int l = 0; l < L; ++l) unew[(size_t)l * nxp + nx] = unew[(size_t)l * nxp + 0];

    /* SWR2 / SWR4: interface variables of the new iterate at t^{n+1}.  With periodic x
       the incoming data of column nx is never used: column nx repeats column 0. */
    for (int m = 0; m <= nx; ++m) {
      const int mi = (d->periodic_x && m == nx) ? 0 : m;
#define U(i) unew[(size_t)((i) - lo) * nxp + m]
      if (has_top && io->out_top) { /* lambda_2 of interface s = Q_2 u_s at alpha_s */
        const int al = alpha_node(d, s);
        double lam;
        if (!d->robin)
          lam = U(al);
        else if (ov >= 1)
          lam = d->q[s] * U(al) - (U(al + 1) - U(al - 1)) / (2.0 * hv);
        else
          lam = (d->p[s] + d->q[s]) * U(al) -
                (io->lam_top ? io->lam_top[(size_t)n * nxp + mi] : 0.0);
        io->out_top[(size_t)n * nxp + m] = lam;
      }
      if (has_bot && io->out_bot) { /* lambda_1 of interface s-1 = Q_1 u_s at beta_{s-1} */
        const int be = beta_node(d, s - 1);
        double lam;
        if (!d->robin)
          lam = U(be);
        else if (ov >= 1)
          lam = d->p[s - 1] * U(be) + (U(be + 1) - U(be - 1)) / (2.0 * hv);
        else
          lam = (d->p[s - 1] + d->q[s - 1]) * U(be) -
                (io->lam_bot ? io->lam_bot[(size_t)n * nxp + mi] : 0.0);
        io->out_bot[(size_t)n * nxp + m] = lam;
      }
      for (int k = 0; k <= ov; ++k) {
        if (has_top && io->band_top)
          io->band_top[((size_t)n * (ov + 1) + k) * nxp + m] = U(alpha_node(d, s) + k);
        if (has_bot && io->band_bot)
          io->band_bot[((size_t)n * (ov + 1) + k) * nxp + m] = U(alpha_node(d, s - 1) + k);
      }
#undef U
    }
    if (io->u_all)
      memcpy(io->u_all + (size_t)(n + 1) * L * nxp, unew, sizeof(double) * (size_t)L * nxp);
    double* t = un;
    un = unew;
    unew = t;
  }
  if (u_T_strip) memcpy(u_T_strip, un, sizeof(double) * (size_t)L * nxp);
  free(un); free(unew); free(a); free(b); free(c); free(R); free(x);
  return KFO_OK;
}

/* ------------------------------------------------------------------------ */
/* Scheme 1: the Lie splitting of Section 6.2 (P1 elements in v, implicit     */
/* Euler over dt, then explicit upwind transport over dt), periodic x and     */
/* zero flux in v, on one strip over the whole window.                      */
/* ------------------------------------------------------------------------ */

static double forcing_at(const kfo_desc* d, const kfo_problem* pb, int i, int m, int n) {
  const int nxp = d->nx + 1;
  double f = 0.0;
  for (int r = 0; r < pb->nforce; ++r)
    f += pb->f_time[(size_t)r * (d->nt + 1) + n] * pb->f_space[((size_t)r * (d->nv + 1) + i) * nxp + m];
  return f;
}

static int solve_strip_fe(const kfo_desc* d, const kfo_problem* pb, int s, const strip_io* io,
                          double* u_T_strip) {
  const int S = d->nstrips, nx = d->nx, nxp = d->nx + 1, nt = d->nt, ov = d->overlap;
  const int lo = strip_lo(d, s), hi = strip_hi(d, s), L = hi - lo + 1;
  const double h = hv_of(d), dt = d->dt, hx = hx_of(d);
  const int has_bot = s > 0, has_top = s < S - 1;
  /* entries of M/dt + S (full row, half row at an end node, off-diagonal) and of M */
  const double k_full = 2.0 * h / (3.0 * dt) + 2.0 / h;
  const double k_half = h / (3.0 * dt) + 1.0 / h;
  const double k_off = h / (6.0 * dt) - 1.0 / h;
  const double m_full = 2.0 * h / 3.0, m_half = h / 3.0, m_off = h / 6.0;

  double* un = (double*)malloc(sizeof(double) * (size_t)L * nxp);
  double* w = (double*)malloc(sizeof(double) * (size_t)L * nxp);
  double* z = (double*)malloc(sizeof(double) * (size_t)L * nxp);
  double* a = (double*)malloc(sizeof(double) * (size_t)L);
  double* b = (double*)malloc(sizeof(double) * (size_t)L);
  double* c = (double*)malloc(sizeof(double) * (size_t)L);
  double* R = (double*)malloc(sizeof(double) * (size_t)L);
  double* x = (double*)malloc(sizeof(double) * (size_t)L);
  if (!un || !w || !z || !a || !b || !c || !R || !x) {
    free(un); free(w); free(z); free(a); free(b); free(c); free(R); free(x);
    return KFO_ENOMEM;
  }
  for (int l = 0; l < L; ++l) {
    memcpy(un + (size_t)l * nxp, pb->u0 + (size_t)(lo + l) * nxp, sizeof(double) * nxp);
    un[(size_t)l * nxp + nx] = un[(size_t)l * nxp + 0]; /* node nx repeats node 0 */
  }
  if (io->u_all) memcpy(io->u_all, un, sizeof(double) * (size_t)L * nxp);
#define Z(l, m) z[(size_t)(l) * nxp + (m)]
#define W(l, m) w[(size_t)(l) * nxp + (m)]
  for (int n = 0; n < nt; ++n) {
    /* step 1: (M/dt + S) w = M z, z = u^n / dt + f^{n+1}, column by column */
    for (int l = 0; l < L; ++l)
      for (int m = 0; m < nx; ++m) Z(l, m) = un[(size_t)l * nxp + m] / dt + forcing_at(d, pb, lo + l, m, n + 1);
    for (int m = 0; m < nx; ++m) {
      for (int l = 0; l < L; ++l) {
        a[l] = k_off; b[l] = k_full; c[l] = k_off;
        if (l == 0) a[l] = 0.0;
        if (l == L - 1) c[l] = 0.0;
        if (l == 0 && l == L - 1) R[l] = m_half * Z(l, m);
        else if (l == 0) R[l] = m_half * Z(l, m) + m_off * Z(l + 1, m);
        else if (l == L - 1) R[l] = m_half * Z(l, m) + m_off * Z(l - 1, m);
        else R[l] = m_off * Z(l - 1, m) + m_full * Z(l, m) + m_off * Z(l + 1, m);
        if (l == 0 || l == L - 1) b[l] = k_half; /* end node: one element only */
      }
      /* transmission rows (SWR1 / SWR3): Robin adds p or q to the end row, lambda to its
       * right-hand side; Dirichlet sets the end value */
      if (has_top) {
        const double lam = io->lam_top ? io->lam_top[(size_t)n * nxp + m] : 0.0;
        if (d->robin) { b[L - 1] += d->p[s]; R[L - 1] += lam; }
        else { a[L - 1] = 0.0; b[L - 1] = 1.0; R[L - 1] = lam; }
      }
      if (has_bot) {
        const double lam = io->lam_bot ? io->lam_bot[(size_t)n * nxp + m] : 0.0;
        if (d->robin) { b[0] += d->q[s - 1]; R[0] += lam; }
        else { c[0] = 0.0; b[0] = 1.0; R[0] = lam; }
      }
      int rc = kfo_thomas(L, a, b, c, R, x);
      if (rc) {
        free(un); free(w); free(z); free(a); free(b); free(c); free(R); free(x);
        return rc;
      }
      for (int l = 0; l < L; ++l) W(l, m) = x[l];
    }
    for (int l = 0; l < L; ++l) { W(l, nx) = W(l, 0); Z(l, nx) = Z(l, 0); }

    /* SWR2 / SWR4 from the diffusion step's solution w */
    for (int m = 0; m <= nx; ++m) {
      const int mi = m == nx ? 0 : m;
      if (has_top && io->out_top) { /* lambda_2 of interface s at alpha_s */
        const int al = alpha_node(d, s) - lo;
        double lam;
        if (!d->robin)
          lam = W(al, m);
        else if (ov >= 1) /* q w minus the residual of the lower half of row alpha */
          lam = d->q[s] * W(al, m) -
                (k_half * W(al, m) + k_off * W(al - 1, m) - m_half * Z(al, m) - m_off * Z(al - 1, m));
        else
          lam = (d->p[s] + d->q[s]) * W(al, m) - (io->lam_top ? io->lam_top[(size_t)n * nxp + mi] : 0.0);
        io->out_top[(size_t)n * nxp + m] = lam;
      }
      if (has_bot && io->out_bot) { /* lambda_1 of interface s-1 at beta_{s-1} */
        const int be = beta_node(d, s - 1) - lo;
        double lam;
        if (!d->robin)
          lam = W(be, m);
        else if (ov >= 1) /* p w minus the residual of the upper half of row beta */
          lam = d->p[s - 1] * W(be, m) -
                (k_half * W(be, m) + k_off * W(be + 1, m) - m_half * Z(be, m) - m_off * Z(be + 1, m));
        else
          lam = (d->p[s - 1] + d->q[s - 1]) * W(be, m) -
                (io->lam_bot ? io->lam_bot[(size_t)n * nxp + mi] : 0.0);
        io->out_bot[(size_t)n * nxp + m] = lam;
      }
    }

    /* step 2: explicit upwind transport of w over dt, periodic in x:
       w_t + v w_x = 0 with the difference taken on the side the flow comes from */
    for (int l = 0; l < L; ++l) {
      const double vi = v_node(d, lo + l), cfl = vi * dt / hx;
      for (int m = 0; m < nx; ++m) {
        double u;
        if (vi > 0) u = W(l, m) - cfl * (W(l, m) - W(l, (m - 1 + nx) % nx));
        else if (vi < 0) u = W(l, m) - cfl * (W(l, (m + 1) % nx) - W(l, m));
        else u = W(l, m);
        un[(size_t)l * nxp + m] = u;
      }
      un[(size_t)l * nxp + nx] = un[(size_t)l * nxp + 0];
    }
    for (int m = 0; m <= nx; ++m)
      for (int k = 0; k <= ov; ++k) {
        if (has_top && io->band_top)
          io->band_top[((size_t)n * (ov + 1) + k) * nxp + m] = un[(size_t)(alpha_node(d, s) + k - lo) * nxp + m];
        if (has_bot && io->band_bot)
          io->band_bot[((size_t)n * (ov + 1) + k) * nxp + m] =
              un[(size_t)(alpha_node(d, s - 1) + k - lo) * nxp + m];
      }
    if (io->u_all) memcpy(io->u_all + (size_t)(n + 1) * L * nxp, un, sizeof(double) * (size_t)L * nxp);
  }
#undef Z
#undef W
  if (u_T_strip) memcpy(u_T_strip, un, sizeof(double) * (size_t)L * nxp);
  free(un); free(w); free(z); free(a); free(b); free(c); free(R); free(x);
  return KFO_OK;
}

/* Owner of node i at t = T: the lower strip of interface j for i <= I_j. */
static int owner_strip(const kfo_desc* d, int i) {
  int s = 0;
  while (s < d->nstrips - 1 && i > centre_node(d, s)) ++s;
  return s;
}

int kfo_swr_iteration(const kfo_desc* d, const kfo_problem* pb, const double* lam_in,
                      double* lam_out, double* bands, double* u_T) {
  int rc = kfo_validate(d);
  if (rc) return rc;
  const int S = d->nstrips, nxp = d->nx + 1, nt = d->nt, ov = d->overlap;
  const size_t tr = (size_t)nt * nxp;          /* one trace array */
  const size_t bd = (size_t)nt * (ov + 1) * nxp; /* one band array */
  double** uT = (double**)calloc((size_t)S, sizeof(double*));
  if (!uT) return KFO_ENOMEM;
  for (int s = 0; s < S && rc == KFO_OK; ++s) {
    const int L = strip_hi(d, s) - strip_lo(d, s) + 1;
    strip_io io;
    memset(&io, 0, sizeof io);
    if (s > 0) {
      /* serial form (SWR3 uses lambda_2^k just produced by the strip below) or the
       * parallel form of the Remark (lambda_2^{k-1}) */
      if (d->gauss_seidel && lam_out)
        io.lam_bot = lam_out + ((size_t)(s - 1) * 2 + 1) * tr;
      else
        io.lam_bot = lam_in ? lam_in + ((size_t)(s - 1) * 2 + 1) * tr : NULL;
      io.out_bot = lam_out ? lam_out + ((size_t)(s - 1) * 2 + 0) * tr : NULL;
      io.band_bot = bands ? bands + ((size_t)(s - 1) * 2 + 1) * bd : NULL;
    }
    if (s < S - 1) {
      io.lam_top = lam_in ? lam_in + ((size_t)s * 2 + 0) * tr : NULL;
      io.out_top = lam_out ? lam_out + ((size_t)s * 2 + 1) * tr : NULL;
      io.band_top = bands ? bands + ((size_t)s * 2 + 0) * bd : NULL;
    }
    if (u_T) {
      uT[s] = (double*)malloc(sizeof(double) * (size_t)L * nxp);
      if (!uT[s]) { rc = KFO_ENOMEM; break; }
    }
    rc = d->scheme == 1 ? solve_strip_fe(d, pb, s, &io, uT[s]) : solve_strip(d, pb, s, &io, uT[s]);
  }
  if (rc == KFO_OK && u_T) {
    for (int i = 0; i <= d->nv; ++i) {
      const int s = owner_strip(d, i);
      memcpy(u_T + (size_t)i * nxp, uT[s] + (size_t)(i - strip_lo(d, s)) * nxp,
             sizeof(double) * nxp);
    }
  }
  for (int s = 0; s < S; ++s) free(uT[s]);
  free(uT);
  return rc;
}

int kfo_interface_norms(const kfo_desc* d, const double* bands, const double* lam_new,
                        const double* lam_old, double* e_mis, double* e_chg, double* j_l2) {
  const int S = d->nstrips, nxp = d->nx + 1, nt = d->nt, ov = d->overlap;
  const size_t bd = (size_t)nt * (ov + 1) * nxp, tr = (size_t)nt * nxp;
  double mis = 0.0, chg = 0.0, sq = 0.0;
  for (int j = 0; j < S - 1; ++j) {
    const double* lower = bands + ((size_t)j * 2 + 0) * bd;
    const double* upper = bands + ((size_t)j * 2 + 1) * bd;
    for (size_t e = 0; e < bd; ++e) {
      const double diff = lower[e] - upper[e];
      if (fabs(diff) > mis) mis = fabs(diff);
      if (!(d->periodic_x && (int)(e % nxp) == d->nx)) sq += diff * diff; /* node nx repeats node 0 */
    }
  }
  if (lam_new && lam_old)
    for (size_t e = 0; e < (size_t)(S - 1) * 2 * tr; ++e) {
      const double diff = fabs(lam_new[e] - lam_old[e]);
      if (diff > chg) chg = diff;
    }
  if (e_mis) *e_mis = mis;
  if (e_chg) *e_chg = chg;
  if (j_l2) *j_l2 = d->dt * hx_of(d) * sq;
  return KFO_OK;
}

int kfo_swr_solve(const kfo_desc* d, const kfo_problem* pb, double* lam, int max_iters,
                  double tol, int tol_kind, int* iters, double* hist, double* u_T) {
  int rc = kfo_validate(d);
  if (rc) return rc;
  const int S = d->nstrips, nxp = d->nx + 1, nt = d->nt, ov = d->overlap;
  const size_t ntr = (size_t)(S - 1) * 2 * nt * nxp;
  const size_t nbd = (size_t)(S - 1) * 2 * nt * (ov + 1) * nxp;
  double* lam_new = (double*)malloc(sizeof(double) * (ntr ? ntr : 1));
  double* bands = (double*)malloc(sizeof(double) * (nbd ? nbd : 1));
  if (!lam_new || !bands) {
    free(lam_new); free(bands);
    return KFO_ENOMEM;
  }
  if (d->periodic_x) /* periodic x: column nx of the interface data repeats column 0 */
    for (size_t line = 0; line < ntr / nxp; ++line) lam[line * nxp + d->nx] = lam[line * nxp];
  int k = 0;
  while (k < max_iters) {
    rc = kfo_swr_iteration(d, pb, lam, lam_new, bands, u_T);
    if (rc) break;
    double mis, chg, jl2;
    kfo_interface_norms(d, bands, lam_new, lam, &mis, &chg, &jl2);
    if (hist) {
      hist[3 * k + 0] = mis;
      hist[3 * k + 1] = chg;
      hist[3 * k + 2] = jl2;
    }
    memcpy(lam, lam_new, sizeof(double) * ntr);
    ++k;
    if ((tol_kind == 0 ? chg : mis) < tol) break;
  }
  if (iters) *iters = k;
  free(lam_new);
  free(bands);
  return rc;
}

int kfo_monolithic(const kfo_desc* d, const kfo_problem* pb, double* u_T, double* u_all) {
  kfo_desc one = *d;
  one.nstrips = 1;
  one.overlap = 0;
  int rc = kfo_validate(&one);
  if (rc) return rc;
  strip_io io;
  memset(&io, 0, sizeof io);
  io.u_all = u_all;
  return one.scheme == 1 ? solve_strip_fe(&one, pb, 0, &io, u_T) : solve_strip(&one, pb, 0, &io, u_T);
}

/* ------------------------------------------------------------------------ */
/* Discrete adjoint of K parallel SWR iterations (Robin, no overlap).        */
/*                                                                          */
/* Per strip and time step the forward scheme is A u^{n+1} = E u^n + rhs,    */
/* where A (tridiagonal, per column) holds the Robin coefficient             */
/* 1 + 2r + 2 p dt/hv on the strip's top row and 1 + 2r + 2 q dt/hv on its   */
/* bottom row, E is the explicit upwind transport, and the Robin rows carry  */
/* + (2 dt/hv) lambda_in.  Without overlap the outgoing data are             */
/* lambda_out = (p + q) u_node - lambda_in (Section 6.3, SWR2 / SWR4).       */
/* The adjoint solves A^T w^{n+1} = dJ/du^{n+1} + (p + q) lambda_out_bar     */
/* + E^T w^{n+2} backward in time; lambda_in_bar = (2 dt/hv) w_node -        */
/* lambda_out_bar; dJ/dp gets -(2 dt/hv) w_node u_node (through A) and       */
/* lambda_out_bar u_node (through the outgoing data), dJ/dq likewise.        */
/* The lambda_in_bar of iterate k is the lambda_out_bar of iterate k-1.      */
/* ------------------------------------------------------------------------ */

/* Row type of node i, column m in strip s (same precedence as solve_strip):
 * 0 interior, 1 identity (v boundary, x inflow, Dirichlet interface),
 * 2 Robin top (p + d/dv), 3 Robin bottom (q - d/dv). */
static int row_kind(const kfo_desc* d, int s, int i, int m) {
  const double vi = v_node(d, i);
  if (i == 0 || i == d->nv) return 1;
  if ((m == 0 && vi > 0) || (m == d->nx && vi < 0)) return 1;
  if (s < d->nstrips - 1 && i == strip_hi(d, s)) return d->robin ? 2 : 1;
  if (s > 0 && i == strip_lo(d, s)) return d->robin ? 3 : 1;
  return 0;
}

static void row_matrix(const kfo_desc* d, int s, int kind, double* a, double* b, double* c) {
  const double hv = hv_of(d), r = d->dt / (hv * hv);
  *a = 0.0; *b = 1.0; *c = 0.0;
  if (kind == 0) { *a = -r; *b = 1.0 + 2.0 * r; *c = -r; }
  if (kind == 2) { *a = -2.0 * r; *b = 1.0 + 2.0 * r + 2.0 * d->p[s] * d->dt / hv; }
  if (kind == 3) { *b = 1.0 + 2.0 * r + 2.0 * d->q[s - 1] * d->dt / hv; *c = -2.0 * r; }
}

/* Adjoint of strip s over one iterate.  bands: that iterate's interface-node values
 * [S-1][2][nt][1][nx+1]; lbar_out: adjoint of the data the strip produced (trace
 * layout); lbar_in (accumulated): adjoint of the data the strip consumed. */
static int adjoint_strip(const kfo_desc* d, int s, int last, const double* bands, const double* lbar_out,
                         double* lbar_in, double* gp, double* gq) {
  const int S = d->nstrips, nx = d->nx, nxp = d->nx + 1, nt = d->nt;
  const int lo = strip_lo(d, s), hi = strip_hi(d, s), L = hi - lo + 1;
  const double hv = hv_of(d), dthx = d->dt * hx_of(d), two_dt_hv = 2.0 * d->dt / hv;
  const int has_top = s < S - 1, has_bot = s > 0;
  const size_t tr = (size_t)nt * nxp;  /* one trace / one band (overlap 0) array */
  double* w_next = (double*)calloc((size_t)L * nxp, sizeof(double));
  double* w_cur = (double*)calloc((size_t)L * nxp, sizeof(double));
  double* a = (double*)malloc(sizeof(double) * (size_t)L);
  double* b = (double*)malloc(sizeof(double) * (size_t)L);
  double* c = (double*)malloc(sizeof(double) * (size_t)L);
  double* at = (double*)malloc(sizeof(double) * (size_t)L);
  double* ct = (double*)malloc(sizeof(double) * (size_t)L);
  double* mu = (double*)malloc(sizeof(double) * (size_t)L);
  double* x = (double*)malloc(sizeof(double) * (size_t)L);
  if (!w_next || !w_cur || !a || !b || !c || !at || !ct || !mu || !x) {
    free(w_next); free(w_cur); free(a); free(b); free(c); free(at); free(ct); free(mu); free(x);
    return KFO_ENOMEM;
  }
  for (int n = nt - 1; n >= 0; --n) { /* time level n+1 */
    const int have_next = (n + 1 < nt);
    for (int m = 0; m <= nx; ++m) {
      for (int l = 0; l < L; ++l) {
        const int i = lo + l;
        double e = 0.0; /* (E^T w^{n+2})_{i,m} */
        if (have_next) {
          const double vi = v_node(d, i);
          const double cabs = fabs(vi * d->dt / hx_of(d));
          if (row_kind(d, s, i, m) != 1) e += (1.0 - cabs) * w_next[(size_t)l * nxp + m];
          if (vi > 0 && m + 1 <= nx && row_kind(d, s, i, m + 1) != 1) e += cabs * w_next[(size_t)l * nxp + m + 1];
          if (vi < 0 && m - 1 >= 0 && row_kind(d, s, i, m - 1) != 1) e += cabs * w_next[(size_t)l * nxp + m - 1];
        }
        mu[l] = e;
        int k = row_kind(d, s, i, m);
        row_matrix(d, s, k, &a[l], &b[l], &c[l]);
      }
      if (has_top) {
        const double uh = bands[(((size_t)s * 2 + 0) * tr) + (size_t)n * nxp + m];
        const double uo = bands[(((size_t)s * 2 + 1) * tr) + (size_t)n * nxp + m];
        if (last) mu[L - 1] += 2.0 * dthx * (uh - uo);
        mu[L - 1] += (d->p[s] + d->q[s]) * lbar_out[(((size_t)s * 2 + 1) * tr) + (size_t)n * nxp + m];
      }
      if (has_bot) {
        const double ul = bands[((((size_t)s - 1) * 2 + 1) * tr) + (size_t)n * nxp + m];
        const double uo = bands[((((size_t)s - 1) * 2 + 0) * tr) + (size_t)n * nxp + m];
        if (last) mu[0] += -2.0 * dthx * (uo - ul);
        mu[0] += (d->p[s - 1] + d->q[s - 1]) * lbar_out[((((size_t)s - 1) * 2 + 0) * tr) + (size_t)n * nxp + m];
      }
      /* transposed system: sub-diagonal c_{l-1}, super-diagonal a_{l+1} */
      for (int l = 0; l < L; ++l) {
        at[l] = l > 0 ? c[l - 1] : 0.0;
        ct[l] = l < L - 1 ? a[l + 1] : 0.0;
      }
      int rc = kfo_thomas(L, at, b, ct, mu, x);
      if (rc) {
        free(w_next); free(w_cur); free(a); free(b); free(c); free(at); free(ct); free(mu); free(x);
        return rc;
      }
      for (int l = 0; l < L; ++l) w_cur[(size_t)l * nxp + m] = x[l];
      if (has_top) {
        const int k = row_kind(d, s, hi, m);
        const double uh = bands[(((size_t)s * 2 + 0) * tr) + (size_t)n * nxp + m];
        const double lo_bar = lbar_out[(((size_t)s * 2 + 1) * tr) + (size_t)n * nxp + m];
        const double wr = (k == 2) ? x[L - 1] : 0.0;
        lbar_in[(((size_t)s * 2 + 0) * tr) + (size_t)n * nxp + m] += two_dt_hv * wr - lo_bar;
        gp[s] += -two_dt_hv * wr * uh + lo_bar * uh;
        gq[s] += lo_bar * uh;
      }
      if (has_bot) {
        const int k = row_kind(d, s, lo, m);
        const double ul = bands[((((size_t)s - 1) * 2 + 1) * tr) + (size_t)n * nxp + m];
        const double lo_bar = lbar_out[((((size_t)s - 1) * 2 + 0) * tr) + (size_t)n * nxp + m];
        const double wr = (k == 3) ? x[0] : 0.0;
        lbar_in[((((size_t)s - 1) * 2 + 1) * tr) + (size_t)n * nxp + m] += two_dt_hv * wr - lo_bar;
        gq[s - 1] += -two_dt_hv * wr * ul + lo_bar * ul;
        gp[s - 1] += lo_bar * ul;
      }
    }
    double* t = w_next;
    w_next = w_cur;
    w_cur = t;
  }
  free(w_next); free(w_cur); free(a); free(b); free(c); free(at); free(ct); free(mu); free(x);
  return KFO_OK;
}

int kfo_swr_adjoint(const kfo_desc* d, const kfo_problem* pb, const double* lam0, int K, double* J,
                    double* grad_p, double* grad_q) {
  int rc = kfo_validate(d);
  if (rc) return rc;
  if (!d->robin || d->overlap != 0 || d->nstrips < 2 || K < 1 || d->gauss_seidel || d->neumann_v || d->scheme ||
      d->periodic_x)
    return KFO_EINVAL;
  const int S = d->nstrips, nxp = d->nx + 1, nt = d->nt;
  const size_t ntr = (size_t)(S - 1) * 2 * nt * nxp; /* traces = bands (overlap 0) */
  double* lam = (double*)calloc(ntr, sizeof(double));
  double* lam_new = (double*)calloc(ntr, sizeof(double));
  double* bands = (double*)calloc(ntr * (size_t)K, sizeof(double));
  double* lbar_out = (double*)calloc(ntr, sizeof(double));
  double* lbar_in = (double*)calloc(ntr, sizeof(double));
  if (!lam || !lam_new || !bands || !lbar_out || !lbar_in) {
    free(lam); free(lam_new); free(bands); free(lbar_out); free(lbar_in);
    return KFO_ENOMEM;
  }
  if (lam0) memcpy(lam, lam0, sizeof(double) * ntr);
  for (int k = 0; k < K && rc == KFO_OK; ++k) {
    rc = kfo_swr_iteration(d, pb, lam, lam_new, bands + (size_t)k * ntr, NULL);
    double* t = lam; lam = lam_new; lam_new = t;
  }
  if (rc == KFO_OK) {
    double jl2 = 0.0;
    kfo_interface_norms(d, bands + (size_t)(K - 1) * ntr, NULL, NULL, NULL, NULL, &jl2);
    if (J) *J = jl2;
    for (int j = 0; j < S - 1; ++j) { grad_p[j] = 0.0; grad_q[j] = 0.0; }
    for (int k = K; k >= 1 && rc == KFO_OK; --k) {
      memset(lbar_in, 0, sizeof(double) * ntr);
      for (int s = 0; s < S && rc == KFO_OK; ++s)
        rc = adjoint_strip(d, s, k == K, bands + (size_t)(k - 1) * ntr, lbar_out, lbar_in, grad_p, grad_q);
      /* the data iterate k consumed were produced by iterate k-1 in the same slots */
      double* t = lbar_out; lbar_out = lbar_in; lbar_in = t;
    }
  }
  free(lam); free(lam_new); free(bands); free(lbar_out); free(lbar_in);
  return rc;
}
