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
#pragma once
#include <cuda_runtime.h>

#include "kfp_kernels.cuh"

namespace kfp {

// ---------------------------------------------------------------------------
// One launch per time level, lanes = x-columns.
//
// The adjoint of one iterate runs the forward schedule backward: pass j
// back-substitutes level nt-j+1 (its system was eliminated by pass j-1 in the other
// row order) and, in the same row order, eliminates level nt-j.  The transposed
// upwind term E^T w^{l+1} of a row needs w^{l+1} of the downstream column, which
// comes from a warp shuffle (lane + sign of v); lanes 0 and 31 are halo columns
// that recompute their neighbour's back-substitution, as in the forward sweep.
// Only the elimination residue is stored (Y[2][rows][P], column m at m+1).
// ---------------------------------------------------------------------------

struct AdjPassArgs {
  int nx, nv, nt, P, W, Lmax;
  double two_dt_hv, dthx;
  const StripInfo* strips;
  const double* coef;       // [S][3][2][3][Lmax] LU of A^T per class and direction: 1/pivot, coupling, cp
  const double* cabs;       // [nv+1] |v_i| dt / hx
  const signed char* sgn;   // [nv+1]
  const double* bands;      // [S-1][2][nt][nx+1] interface-node values of this iterate
  const double* lbar_out;   // [S-1][2][nt][nx+1]
  double* lbar_in;
  double* contrib;          // [S-1][4][nt][nx+1]
  double* Y0;               // [rows][P] elimination residue, even passes
  double* Y1;               // odd passes
};

// row (i, m) of the forward system is an identity row (v boundary or x inflow);
// sg = sign of v_i
__device__ __forceinline__ bool adj_identity(const AdjPassArgs& A, int i, int m, int sg) {
  if (i == 0 || i == A.nv) return true;
  return (m == 0 && sg > 0) || (m == A.nx && sg < 0);
}

// MODE 0: eliminate level nt (no back-substitution); 1: back-substitute level
// nt-j+1 and eliminate level nt-j; 2: back-substitute level 1 only.
template <bool UP, int MODE>
__device__ __forceinline__ void adjoint_pass(const AdjPassArgs& A, const int j, const int last_iterate) {
  const int lane = threadIdx.x & 31;
  const int w = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (w >= A.W) return;  // whole warp leaves together
  const int s = blockIdx.y;
  const StripInfo st = A.strips[s];
  const int m = w * kOutCols - 1 + lane;
  const int col = m + 1;
  const bool in_dom = (m >= 0) && (m <= A.nx);
  const bool out_lane = in_dom && lane >= 1 && lane <= kOutCols;
  const int cls = (m <= 0) ? 0 : (m >= A.nx ? 2 : 1);
  const int L = st.L, lo = st.lo, P = A.P, nxp = A.nx + 1, nt = A.nt;
  const int dirE = UP ? 0 : 1, dirB = UP ? 1 : 0;
  const double* __restrict__ gE = A.coef + ((size_t)((s * 3 + cls) * 2 + dirE) * 3 + 0) * A.Lmax;
  const double* __restrict__ aE = A.coef + ((size_t)((s * 3 + cls) * 2 + dirE) * 3 + 1) * A.Lmax;
  const double* __restrict__ cpB = A.coef + ((size_t)((s * 3 + cls) * 2 + dirB) * 3 + 2) * A.Lmax;
  const double* __restrict__ Ycur = (j & 1) ? A.Y0 : A.Y1;   // written by pass j-1
  double* __restrict__ Ynext = (j & 1) ? A.Y1 : A.Y0;
  const int le = nt - j;        // level eliminated by this pass (MODE 0, 1)
  const int lb = nt - j + 1;    // level back-substituted (MODE 1, 2)
  const size_t tr = (size_t)nt * nxp;

  // interface-node data of both levels, one value per lane
  double ue_top = 0, ue_top_o = 0, lbo_e_top = 0, ue_bot = 0, ue_bot_o = 0, lbo_e_bot = 0;
  double ub_top = 0, lbo_b_top = 0, ub_bot = 0, lbo_b_bot = 0;
  if (in_dom) {
    if (st.has_top) {
      const double* bl = A.bands + ((size_t)s * 2 + 0) * tr + m;
      const double* bu = A.bands + ((size_t)s * 2 + 1) * tr + m;
      const double* lo_ = A.lbar_out + ((size_t)s * 2 + 1) * tr + m;
      if (MODE != 2) { ue_top = bl[(size_t)(le - 1) * nxp]; ue_top_o = bu[(size_t)(le - 1) * nxp]; lbo_e_top = lo_[(size_t)(le - 1) * nxp]; }
      if (MODE != 0) { ub_top = bl[(size_t)(lb - 1) * nxp]; lbo_b_top = lo_[(size_t)(lb - 1) * nxp]; }
    }
    if (st.has_bot) {
      const double* bu = A.bands + ((size_t)(s - 1) * 2 + 1) * tr + m;
      const double* bl = A.bands + ((size_t)(s - 1) * 2 + 0) * tr + m;
      const double* lo_ = A.lbar_out + ((size_t)(s - 1) * 2 + 0) * tr + m;
      if (MODE != 2) { ue_bot = bu[(size_t)(le - 1) * nxp]; ue_bot_o = bl[(size_t)(le - 1) * nxp]; lbo_e_bot = lo_[(size_t)(le - 1) * nxp]; }
      if (MODE != 0) { ub_bot = bu[(size_t)(lb - 1) * nxp]; lbo_b_bot = lo_[(size_t)(lb - 1) * nxp]; }
    }
  }

  double w_prev = 0.0, y_prev = 0.0;
  // Row l(t) = t (UP) or L-1-t of the pass; its table entries and residue rows are
  // addressed from the row of t = 0 in steps of dl or dP.
  constexpr int dl = UP ? 1 : -1;
  const int l_first = UP ? 0 : L - 1;
  const ptrdiff_t dP = (ptrdiff_t)dl * P;
  const double* __restrict__ gEt = gE + l_first;
  const double* __restrict__ aEt = aE + l_first;
  const double* __restrict__ cpt = cpB + l_first;
  const double* __restrict__ cabt = A.cabs + lo + l_first;
  const signed char* __restrict__ sgt = A.sgn + lo + l_first;
  const double* __restrict__ yt = Ycur + (size_t)(st.rowoff + l_first) * P + col;
  double* __restrict__ ynt = Ynext + (size_t)(st.rowoff + l_first) * P + col;
  // Away from v = v0, v1 a row (i, m) is an identity row only at an inflow column, so
  // whether the transposed upwind term takes w of this column (a) and of the
  // downstream column m + sg (b) depends on the lane and the sign of v alone.
  const bool a_pos = m != 0, a_neg = m != A.nx;
  const bool b_pos = m >= 0 && m <= A.nx - 1, b_neg = m >= 1 && m <= A.nx;

  // rows go in groups of kPrefetch whose inputs are loaded together, so that the
  // loads of a group are in flight at once instead of one latency per row
  // (the inputs of the next group are loaded while the current one is computed)
  constexpr int kPrefetch = 4;
  double ynx[kPrefetch], cnx[kPrefetch], gnx[kPrefetch], anx[kPrefetch], cabnx[kPrefetch];
  int sgnx[kPrefetch];
  auto load_group = [&](int tb) {
    if (tb + kPrefetch <= L) {  // uniform: a whole group inside the strip
#pragma unroll
      for (int u = 0; u < kPrefetch; ++u) {
        const int t = tb + u;
        ynx[u] = MODE != 0 ? yt[dP * t] : 0.0;
        cnx[u] = cpt[dl * t];
        gnx[u] = gEt[dl * t];
        anx[u] = aEt[dl * t];
        cabnx[u] = cabt[dl * t];
        sgnx[u] = sgt[dl * t];
      }
    } else {
#pragma unroll
      for (int u = 0; u < kPrefetch; ++u) {
        const int t = tb + u;
        const bool ok = t < L;
        ynx[u] = (MODE != 0 && ok) ? yt[dP * t] : 0.0;
        cnx[u] = ok ? cpt[dl * t] : 0.0;
        gnx[u] = ok ? gEt[dl * t] : 0.0;
        anx[u] = ok ? aEt[dl * t] : 0.0;
        cabnx[u] = ok ? cabt[dl * t] : 0.0;
        sgnx[u] = ok ? sgt[dl * t] : 0;
      }
    }
  };

  double ypre[kPrefetch], cpre[kPrefetch], gpre[kPrefetch], apre[kPrefetch], cabpre[kPrefetch];
  int sgpre[kPrefetch];
  // Groups of rows 1 .. L-2 only (no interface row, no v boundary) take the plain
  // path: no interface terms and no identity-row tests per row.
  auto run_group = [&](auto plain_tag, const int t0) {
    constexpr bool PLAIN = decltype(plain_tag)::value;
#pragma unroll
    for (int u = 0; u < kPrefetch; ++u) {
      const int t = t0 + u;
      if (!PLAIN && t >= L) break;  // uniform across the warp
      const int l = UP ? t : (L - 1 - t);
      const int i = lo + l;
      double wv = 0.0;  // w^{le+1} (zero beyond nt)
      if (MODE != 0) {
        wv = ypre[u] - cpre[u] * w_prev;
        w_prev = wv;
        // ---- adjoint of the consumed data and the gradient terms at level lb ----
        if (!PLAIN && out_lane) {
          if (st.has_top && l == L - 1) {
            const double wr = adj_identity(A, i, m, sgpre[u]) ? 0.0 : wv;
            const size_t at = (size_t)(lb - 1) * nxp + m;
            A.lbar_in[((size_t)s * 2 + 0) * tr + at] = A.two_dt_hv * wr - lbo_b_top;
            A.contrib[((size_t)s * 4 + 0) * tr + at] += -A.two_dt_hv * wr * ub_top + lbo_b_top * ub_top;
            A.contrib[((size_t)s * 4 + 1) * tr + at] += lbo_b_top * ub_top;
          }
          if (st.has_bot && l == 0) {
            const double wr = adj_identity(A, i, m, sgpre[u]) ? 0.0 : wv;
            const size_t at = (size_t)(lb - 1) * nxp + m;
            A.lbar_in[((size_t)(s - 1) * 2 + 1) * tr + at] = A.two_dt_hv * wr - lbo_b_bot;
            A.contrib[((size_t)(s - 1) * 4 + 3) * tr + at] += -A.two_dt_hv * wr * ub_bot + lbo_b_bot * ub_bot;
            A.contrib[((size_t)(s - 1) * 4 + 2) * tr + at] += lbo_b_bot * ub_bot;
          }
        }
        if (MODE == 2) continue;
      }
      // ---- right-hand side of level le: E^T w^{le+1} + sources, then elimination ----
      const int sg = sgpre[u];
      const double wdn = shfl_val(wv, lane + sg);  // w^{le+1} of the downstream column
      const double c = cabpre[u];
      double mu = 0.0;
      if (PLAIN) {
        if (MODE != 0) {  // (1 - c) a + c b as a + c (b - a)
          const double a = (sg > 0 ? a_pos : (sg < 0 ? a_neg : true)) ? wv : 0.0;
          const double b = (sg > 0 ? b_pos : (sg < 0 ? b_neg : false)) ? wdn : 0.0;
          mu = a + c * (b - a);
        }
      } else {
        if (MODE != 0) {
          if (!adj_identity(A, i, m, sg)) mu += (1.0 - c) * wv;
          const int md = m + sg;
          if (sg != 0 && md >= 0 && md <= A.nx && !adj_identity(A, i, md, sg)) mu += c * wdn;
        }
        if (st.has_top && l == L - 1) {
          if (last_iterate) mu += 2.0 * A.dthx * (ue_top - ue_top_o);
          mu += (st.p_top + st.q_top) * lbo_e_top;
        }
        if (st.has_bot && l == 0) {
          if (last_iterate) mu += -2.0 * A.dthx * (ue_bot_o - ue_bot);
          mu += (st.p_bot + st.q_bot) * lbo_e_bot;
        }
      }
      const double y = gpre[u] * (mu - apre[u] * y_prev);
      if (out_lane) ynt[dP * t] = y;
      y_prev = y;
    }
  };

  load_group(0);
  for (int t0 = 0; t0 < L; t0 += kPrefetch) {
#pragma unroll
    for (int u = 0; u < kPrefetch; ++u) {
      ypre[u] = ynx[u]; cpre[u] = cnx[u]; gpre[u] = gnx[u]; apre[u] = anx[u]; cabpre[u] = cabnx[u]; sgpre[u] = sgnx[u];
    }
    if (t0 + kPrefetch < L) load_group(t0 + kPrefetch);
    if (t0 >= 1 && t0 + kPrefetch <= L - 1) run_group(BoolTag<true>{}, t0);
    else run_group(BoolTag<false>{}, t0);
  }
}

// ---------------------------------------------------------------------------
// One launch runs, for each iterate z = blockIdx.z of a group of pipelined adjoint
// iterates (one iterate at a time: a group of one), its pass j[z].  Going backward over the iterates, the
// adjoint of iterate k-1 reads in pass j the lambda_out_bar of levels nt-j and
// nt-j+1, which the adjoint of iterate k writes in its passes j+1 and j; with pass
// j of the group's q-th iterate in slot j + 2q, every launch only reads what earlier
// launches wrote, each iterate has its own residue buffers and lambda_bar slots,
// and the iterates of one launch add their gradient terms at different levels, in
// the order of one iterate at a time (bitwise the same sums).
// ---------------------------------------------------------------------------

constexpr int kAdjGroupMax = 16;  // 16 x 120 B of arguments: well inside the parameter space
struct AdjGroup {
  AdjPassArgs A[kAdjGroupMax];
  int j[kAdjGroupMax];
  int last[kAdjGroupMax];
};

template <bool UP, int MODE>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
adjoint_group_kernel(const __grid_constant__ AdjGroup G) {
  const int z = blockIdx.z;
  adjoint_pass<UP, MODE>(G.A[z], G.j[z], G.last[z]);
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
