// kfp_adjoint.cuh -- discrete adjoint of K parallel SWR iterations (sm_103a, FP64).
//
// Objective: J = dt hx sum_j sum_{n=1..nt} sum_m (u_j - u_{j+1})^2 on the interface
// nodes of the K-th iterate (Robin transmission without overlap), gradient with
// respect to the Robin parameters p_j, q_j of every interface.
//
// Per strip and step the forward scheme is A u^{n+1} = E u^n + rhs, with the Robin
// coefficient 1 + 2r + 2p dt/hv (top row) or 1 + 2r + 2q dt/hv (bottom row) in A,
// + (2dt/hv) lambda_in on the Robin rows, and outgoing data
// lambda_out = (p + q) u_node - lambda_in (Section 6.3, SWR2/SWR4, no overlap).
// Backward in time the adjoint solves
//     A^T w^l = E^T w^{l+1} + dJ/du^l + (p + q) lambda_out_bar^l   (on the node rows)
// and yields lambda_in_bar^l = (2dt/hv) w_node - lambda_out_bar^l and the gradient
// terms -(2dt/hv) w_node u_node (through A) and lambda_out_bar u_node (through the
// outgoing data).  Backward over iterations, the lambda_in_bar of iterate k is the
// lambda_out_bar of iterate k-1 (same slots).  Only interface-node values of the
// forward iterates enter, so no forward state is stored or recomputed.
//
// One thread owns one (strip, column) and solves its transposed tridiagonal system
// with host-factored coefficients; the elimination residue goes to a scratch array.
#pragma once
#include <cuda_runtime.h>

#include "kfp_kernels.cuh"

namespace kfp {

struct AdjArgs {
  int nx, nv, nt, S, Lmax;
  double two_dt_hv, dthx;
  const StripInfo* strips;
  const double* fac;        // [S][3 classes][3 fields][Lmax]: 1/pivot, sub-diagonal, back-substitution coef
  const double* cabs;       // [nv+1] |v_i| dt / hx
  const signed char* sgn;   // [nv+1]
  const double* bands;      // [S-1][2][nt][nx+1] interface-node values of this iterate
  const double* lbar_out;   // [S-1][2][nt][nx+1] adjoint of the data this iterate produced
  double* lbar_in;          // same layout: adjoint of the data this iterate consumed
  double* contrib;          // [S-1][4][nt][nx+1]: dJ/dp from the lower strip, dJ/dq from the lower strip,
                            //                      dJ/dp from the upper strip, dJ/dq from the upper strip
  double* w0;               // [rows][nx+1] adjoint state, even levels
  double* w1;               // odd levels
  double* scratch;          // [rows][nx+1] elimination residue
  int rows;
};

// Row type at node i, column m of strip s: 0 interior, 1 identity, 2 Robin top, 3 Robin bottom.
__device__ __forceinline__ int adj_row_kind(const AdjArgs& A, const StripInfo& st, int i, int m) {
  if (i == 0 || i == A.nv) return 1;
  const int sg = A.sgn[i];
  if ((m == 0 && sg > 0) || (m == A.nx && sg < 0)) return 1;
  if (st.has_top && i == st.hi) return 2;
  if (st.has_bot && i == st.lo) return 3;
  return 0;
}

// Level l (1..nt) of the adjoint of one iterate, all strips and columns.
__global__ void __launch_bounds__(128)
adjoint_level_kernel(const AdjArgs A, const int l, const int last_iterate) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = blockIdx.y;
  if (m > A.nx) return;
  const StripInfo st = A.strips[s];
  const int L = st.L, lo = st.lo, nxp = A.nx + 1, nt = A.nt;
  const int cls = m == 0 ? 0 : (m == A.nx ? 2 : 1);
  const double* g = A.fac + ((size_t)(s * 3 + cls) * 3 + 0) * A.Lmax;
  const double* sub = A.fac + ((size_t)(s * 3 + cls) * 3 + 1) * A.Lmax;
  const double* cp = A.fac + ((size_t)(s * 3 + cls) * 3 + 2) * A.Lmax;
  const double* wn = (l + 1) & 1 ? A.w1 : A.w0;  // w^{l+1} (zero beyond nt)
  double* wc = l & 1 ? A.w1 : A.w0;               // w^l
  const bool have_next = l < nt;
  const size_t tr = (size_t)nt * nxp;
  const size_t at = (size_t)(l - 1) * nxp + m;    // time level l in trace layout

  // node values and outgoing-data adjoints at this level
  double u_hi = 0, u_hi_other = 0, lbo_top = 0, u_lo = 0, u_lo_other = 0, lbo_bot = 0;
  if (st.has_top) {
    u_hi = A.bands[((size_t)s * 2 + 0) * tr + at];
    u_hi_other = A.bands[((size_t)s * 2 + 1) * tr + at];
    lbo_top = A.lbar_out[((size_t)s * 2 + 1) * tr + at];
  }
  if (st.has_bot) {
    u_lo = A.bands[((size_t)(s - 1) * 2 + 1) * tr + at];
    u_lo_other = A.bands[((size_t)(s - 1) * 2 + 0) * tr + at];
    lbo_bot = A.lbar_out[((size_t)(s - 1) * 2 + 0) * tr + at];
  }

  // ascending elimination of A^T w = mu
  double y_prev = 0.0;
  for (int r = 0; r < L; ++r) {
    const int i = lo + r;
    const size_t e = (size_t)(st.rowoff + r) * nxp + m;
    double mu = 0.0;
    if (have_next) {  // (E^T w^{l+1})_{i,m}
      const double c = A.cabs[i];
      const int sg = A.sgn[i];
      if (adj_row_kind(A, st, i, m) != 1) mu += (1.0 - c) * wn[e];
      if (sg > 0 && m + 1 <= A.nx && adj_row_kind(A, st, i, m + 1) != 1) mu += c * wn[e + 1];
      if (sg < 0 && m - 1 >= 0 && adj_row_kind(A, st, i, m - 1) != 1) mu += c * wn[e - 1];
    }
    if (r == L - 1 && st.has_top) {
      if (last_iterate) mu += 2.0 * A.dthx * (u_hi - u_hi_other);
      mu += (st.p_top + st.q_top) * lbo_top;
    }
    if (r == 0 && st.has_bot) {
      if (last_iterate) mu += -2.0 * A.dthx * (u_lo_other - u_lo);
      mu += (st.p_bot + st.q_bot) * lbo_bot;
    }
    const double y = g[r] * (mu - sub[r] * y_prev);
    A.scratch[e] = y;
    y_prev = y;
  }
  // descending back-substitution
  double w_next = 0.0, w_top = 0.0, w_bot = 0.0;
  for (int r = L - 1; r >= 0; --r) {
    const size_t e = (size_t)(st.rowoff + r) * nxp + m;
    const double w = A.scratch[e] - cp[r] * w_next;
    wc[e] = w;
    w_next = w;
    if (r == L - 1) w_top = w;
    if (r == 0) w_bot = w;
  }
  // adjoint of the consumed data and gradient contributions
  if (st.has_top) {
    const double wr = adj_row_kind(A, st, st.hi, m) == 2 ? w_top : 0.0;
    A.lbar_in[((size_t)s * 2 + 0) * tr + at] = A.two_dt_hv * wr - lbo_top;
    A.contrib[((size_t)s * 4 + 0) * tr + at] += -A.two_dt_hv * wr * u_hi + lbo_top * u_hi;
    A.contrib[((size_t)s * 4 + 1) * tr + at] += lbo_top * u_hi;
  }
  if (st.has_bot) {
    const double wr = adj_row_kind(A, st, st.lo, m) == 3 ? w_bot : 0.0;
    A.lbar_in[((size_t)(s - 1) * 2 + 1) * tr + at] = A.two_dt_hv * wr - lbo_bot;
    A.contrib[((size_t)(s - 1) * 4 + 3) * tr + at] += -A.two_dt_hv * wr * u_lo + lbo_bot * u_lo;
    A.contrib[((size_t)(s - 1) * 4 + 2) * tr + at] += lbo_bot * u_lo;
  }
}

// grad_p[j] = sum of contrib[j][0] + contrib[j][2]; grad_q[j] = contrib[j][1] + contrib[j][3].
// One block per (interface, parameter); fixed summation order (reproducible).
__global__ void __launch_bounds__(kReduceThreads)
gradient_reduce_kernel(const double* __restrict__ contrib, size_t per, double* __restrict__ grad) {
  const int j = blockIdx.x >> 1, which = blockIdx.x & 1;  // which: 0 = p, 1 = q
  const double* a = contrib + ((size_t)j * 4 + which) * per;
  const double* b = contrib + ((size_t)j * 4 + 2 + which) * per;
  double mx = 0.0, sm = 0.0;
  for (size_t e = threadIdx.x; e < per; e += blockDim.x) sm += a[e] + b[e];
  block_reduce(mx, sm);
  if (threadIdx.x == 0) grad[blockIdx.x] = sm;  // [j][p, q]
}

}  // namespace kfp
