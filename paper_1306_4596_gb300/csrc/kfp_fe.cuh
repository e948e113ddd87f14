// kfp_fe.cuh -- sweep pass of the Lie splitting of Section 6.2 (sm_103a).
//
// One time step of the paper's own scheme for the model problem (periodic in x,
// zero flux in v):
//   step 1  (M + dt S) w = M z,  z = u^n + dt f^{n+1}     (P1 elements in v, implicit
//           Euler over dt; both sides scaled by dt), per x-column; a Robin end adds
//           dt p (top) or dt q (bottom) to the end row and dt lambda to its right-hand
//           side, a Dirichlet end sets w = lambda;
//   step 2  u^{n+1} = w - c_i (w - w_upstream), c_i = |v_i| dt / hx  (upwind transport).
// As in the unsplit sweep, one launch per time step fuses the back-substitution of
// step k (it produces w^k row by row) with the elimination of step k+1; lanes are
// x-columns and the upstream value of a row comes from a warp shuffle.  Two
// differences: the transport now follows the solve (u^k = T w^k), and the
// right-hand side M z of a row needs z of both neighbouring rows, so the
// elimination runs one row behind the back-substitution.
//
// Outgoing interface data come from w^k: Dirichlet w; Robin without overlap
// (p + q) w - lambda_in; Robin with overlap p w (q w) minus the half-row residual of
// this strip at the node, which needs z^k of the node and its neighbour: those two
// values per end are kept from the previous pass in a small buffer Zrec.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>

#include "kfp_kernels.cuh"

namespace kfp {

struct FeArgs {
  double m_half, m_off;          // P1 mass matrix entries: h/3 (end node), h/6 (interior: 4 m_off)
  double k_half, k_off;          // (M + dt S) entries of an end row: h/3 + dt/h, h/6 - dt/h
  double dt, inv_dt;
  double dt_mo, inv_mo;          // dt / m_off, 1 / m_off
  double* zrec;                  // [2 parities][S][2 ends][2 rows][nx+1] z^k at the trace rows
  const void* tab;               // [S][2 directions][2][Lmax] of T: g m_off, g a (elimination
                                 // of a right-hand side in units of m_off)
};

template <typename T, bool UP, int MODE>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
fe_pass_kernel(const PassArgs<T> A, const FeArgs E, const int k) {
  const int lane = threadIdx.x & 31;
  const int w = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (w >= A.W) return;  // whole warp leaves together
  const int s = blockIdx.y + A.strip0;
  const StripInfo st = A.strips[s];
  const int m = w * kOutCols - 1 + lane;
  const int col = m + 1;
  const bool in_dom = (m >= 0) && (m <= A.nx);
  const bool out_lane = in_dom && lane >= 1 && lane <= kOutCols;
  const int L = st.L, lo = st.lo, P = A.P, nxp = A.nx + 1, nt = A.nt;
  const int dirE = UP ? 0 : 1;
  const int dirB = UP ? 1 : 0;
  // periodic x: every column has the same factors (class 1); the elimination takes
  // g m_off and g a, with right-hand sides M z / m_off = z_{l-1} + 4 z_l + z_{l+1}
  // (an end row: 2 z_l + z_neighbour)
  const T* __restrict__ gE = (const T*)E.tab + ((size_t)s * 2 + dirE) * 2 * A.Lmax;
  const T* __restrict__ aE = gE + A.Lmax;
  const T* __restrict__ cpB = A.coef + ((size_t)((s * 3 + 1) * 2 + dirB) * 3 + 2) * A.Lmax;
  const T* __restrict__ Ycur = (k & 1) ? A.Y1 : A.Y0;
  T* __restrict__ Ynext = ((k + 1) & 1) ? A.Y1 : A.Y0;
  const int k1 = k + 1;
  const int ov = A.ov;
  const bool robin_ov = A.robin && ov >= 1;
  const size_t zslab = (size_t)2 * 2 * nxp;  // one strip's Zrec entries
  const double* zcur = E.zrec + ((size_t)(k & 1) * A.S + s) * zslab;
  double* znext = E.zrec + ((size_t)(k1 & 1) * A.S + s) * zslab;

  // local rows of the outgoing data: top = alpha_s (data for the strip above),
  // bottom = beta_{s-1} (data for the strip below); the half-row residual of the top
  // node uses the row below it, that of the bottom node the row above it
  const int aT = st.has_top ? st.alpha_top - lo : -10;
  const int bB = st.has_bot ? st.alpha_bot - lo + ov : -10;
  const int aB = st.alpha_bot - lo;

  // interface data of this strip for the system being eliminated (t^{k+1})
  double lam_rhs_top = 0.0, lam_rhs_bot = 0.0;
  if (MODE != 2 && in_dom) {
    if (st.has_top) lam_rhs_top = A.lam_in[(((size_t)s * 2 + 0) * nt + k) * nxp + m];
    if (st.has_bot) lam_rhs_bot = A.lam_bot_src[((((size_t)s - 1) * 2 + 1) * nt + k) * nxp + m];
  }

  T w_prev = T(0), y_prev = T(0), zm1 = T(0), zm2 = T(0);
  T g_last = T(0), a_last = T(0);  // factors of the previous row in pass order
  T w_last = T(0);                 // w of the previous row in pass order
  // elimination of local row l from the right-hand side rhs = (M z)_l / m_off, with
  // gl = g_l m_off and al = g_l a_l (end rows take the interface data: a Robin row adds
  // dt lambda to M z, a Dirichlet row is w = lambda)
  auto eliminate = [&](int l, T rhs, T gl, T al) {
    const bool top_end = l == L - 1, bot_end = l == 0;
    T R = rhs;
    if (top_end && st.has_top)
      R = A.robin ? (T)((double)R + E.dt_mo * lam_rhs_top) : (T)(lam_rhs_top * E.inv_mo);
    if (bot_end && st.has_bot)
      R = A.robin ? (T)((double)R + E.dt_mo * lam_rhs_bot) : (T)(lam_rhs_bot * E.inv_mo);
    const T y = fma(-al, y_prev, gl * R);
    if (out_lane) Ynext[(size_t)(st.rowoff + l) * P + col] = y;
    y_prev = y;
  };

  // Element t of the pass is local row l(t) = t (UP) or L-1-t; the per-row tables
  // and grid rows of l(t) are addressed from the row of t = 0 in steps of dl or dP.
  constexpr int dl = UP ? 1 : -1;
  const int l_first = UP ? 0 : L - 1;
  const ptrdiff_t dP = (ptrdiff_t)dl * P;
  const T* __restrict__ gEt = gE + l_first;
  const T* __restrict__ aEt = aE + l_first;
  const T* __restrict__ cpt = cpB + l_first;
  const T* __restrict__ cabt = A.cabs + lo + l_first;
  const signed char* __restrict__ sgt = A.sgn + lo + l_first;
  const T* __restrict__ yt =
      (MODE == 0 ? A.U0 + (size_t)(lo + l_first) * P : Ycur + (size_t)(st.rowoff + l_first) * P) + col;
  const T* __restrict__ ft = A.F + (size_t)(lo + l_first) * P + col;
  T* __restrict__ ynt = Ynext + (size_t)(st.rowoff + l_first) * P + col;

  // Rows go in groups of kGroup.  The inputs of the next group are loaded while the
  // current one is computed (two register buffers), then per group: (A) the
  // back-substitution chain, (B) the transport, z and the overlap values of every row
  // of the group (independent of each other), (C) the elimination chain of the rows
  // whose right-hand side is complete.
  constexpr int kGroup = 4;
  T ynx[kGroup], f0nx[kGroup], cpnx[kGroup], gnx[kGroup], anx[kGroup], cabnx[kGroup];
  int sgnx[kGroup];
  const bool force0 = MODE != 2 && A.nforce > 0;
  const T dta0 = force0 ? (T)A.dta[(size_t)k1 * A.nforce] : T(0);
  auto load_group = [&](int tb) {
    if (tb + kGroup <= L) {  // uniform: a whole group inside the strip
#pragma unroll
      for (int u = 0; u < kGroup; ++u) {
        const int t = tb + u;
        ynx[u] = yt[dP * t];
        f0nx[u] = force0 ? ft[dP * t] : T(0);
        cpnx[u] = cpt[dl * t];
        gnx[u] = gEt[dl * t];
        anx[u] = aEt[dl * t];
        cabnx[u] = cabt[dl * t];
        sgnx[u] = sgt[dl * t];
      }
    } else {
#pragma unroll
      for (int u = 0; u < kGroup; ++u) {
        const int t = tb + u;
        const bool ok = t < L;
        ynx[u] = ok ? yt[dP * t] : T(0);
        f0nx[u] = (force0 && ok) ? ft[dP * t] : T(0);
        cpnx[u] = ok ? cpt[dl * t] : T(0);
        gnx[u] = ok ? gEt[dl * t] : T(0);
        anx[u] = ok ? aEt[dl * t] : T(0);
        cabnx[u] = ok ? cabt[dl * t] : T(0);
        sgnx[u] = ok ? sgt[dl * t] : 0;
      }
    }
  };

  // Groups whose rows (and the row before them, which they eliminate) are neither a
  // strip end nor a row of the outgoing data (traces, overlap values, z records) take
  // the plain path.  Rows [ls0, ls1] are such rows; a group starting at t0 touches
  // the rows of t0-1 .. t0+kGroup-1.
  int ls0 = 1, ls1 = L - 2;
  if (st.has_bot) ls0 = max(ls0, max(aB + ov, bB + 1) + 1);
  if (st.has_top) ls1 = min(ls1, aT - 2);
  const int t_plain0 = UP ? ls0 + 1 : L - ls1;
  const int t_plain1 = UP ? ls1 - kGroup + 1 : L - kGroup - ls0;

  T ypre[kGroup], fpre[kGroup], cppre[kGroup], gpre[kGroup], apre[kGroup], cabpre[kGroup];
  int sgpre[kGroup];
  auto run_group = [&](auto plain_tag, const int t0, const int n) {
    constexpr bool PLAIN = decltype(plain_tag)::value;
    // (A) back-substitution chain: w^k of the group's rows
    T wv[kGroup];
#pragma unroll
    for (int u = 0; u < kGroup; ++u) {
      if (MODE != 0 && (PLAIN || u < n)) w_prev = ypre[u] - cppre[u] * w_prev;
      wv[u] = w_prev;
    }
    // outgoing interface data of t^k from w^k (rows alpha / alpha-1 and beta / beta+1)
    if (!PLAIN && MODE != 0 && out_lane) {
      T wlast = w_last;  // w of the previous row in pass order
#pragma unroll
      for (int u = 0; u < kGroup; ++u) {
        const int t = t0 + u;
        const int l = u < n ? (UP ? t : (L - 1 - t)) : -100;  // rows beyond the strip match nothing
        const T wcur = wv[u];
        if (st.has_top) {
          const int eT = robin_ov ? (UP ? aT : aT - 1) : aT;  // the later of alpha, alpha-1
          if (l == eT) {
            const double wa = robin_ov && !UP ? (double)wlast : (double)wcur;  // w(alpha)
            double lam;
            if (!A.robin) {
              lam = wa;
            } else if (ov >= 1) {
              const double wb = UP ? (double)wlast : (double)wcur;  // w(alpha - 1)
              const double* zk = zcur + 0 * 2 * nxp;                 // z^k at alpha, alpha-1
              lam = st.q_top * wa - E.inv_dt * (E.k_half * wa + E.k_off * wb - E.m_half * zk[m] - E.m_off * zk[nxp + m]);
            } else {
              lam = (st.p_top + st.q_top) * wa - A.lam_in[(((size_t)s * 2 + 0) * nt + (k - 1)) * nxp + m];
            }
            A.lam_next[(((size_t)s * 2 + 1) * nt + (k - 1)) * nxp + m] = lam;
          }
        }
        if (st.has_bot) {
          const int eB = robin_ov ? (UP ? bB + 1 : bB) : bB;  // the later of beta, beta+1
          if (l == eB) {
            const double wbeta = robin_ov && UP ? (double)wlast : (double)wcur;  // w(beta)
            double lam;
            if (!A.robin) {
              lam = wbeta;
            } else if (ov >= 1) {
              const double wu = UP ? (double)wcur : (double)wlast;  // w(beta + 1)
              const double* zk = zcur + 1 * 2 * nxp;                // z^k at beta, beta+1
              lam = st.p_bot * wbeta - E.inv_dt * (E.k_half * wbeta + E.k_off * wu - E.m_half * zk[m] - E.m_off * zk[nxp + m]);
            } else {
              lam = (st.p_bot + st.q_bot) * wbeta -
                    A.lam_bot_src[((((size_t)s - 1) * 2 + 1) * nt + (k - 1)) * nxp + m];
            }
            A.lam_next[((((size_t)s - 1) * 2 + 0) * nt + (k - 1)) * nxp + m] = lam;
          }
        }
        wlast = wcur;
      }
    }

    // (B) transport over dt, u^k = w^k - c (w^k - w^k upstream), and z^{k+1} = u^k + dt f^{k+1}
    T zv[kGroup];
#pragma unroll
    for (int u = 0; u < kGroup; ++u) {
      const int t = t0 + u;
      const bool ok = PLAIN || u < n;  // uniform
      const int l = ok ? (UP ? t : (L - 1 - t)) : -100;
      T uv;
      if (MODE == 0) {
        uv = ypre[u];
      } else {
        const T wnb = shfl_val(wv[u], lane - sgpre[u]);
        uv = wv[u] - cabpre[u] * (wv[u] - wnb);
        if (!PLAIN && out_lane && ok) {
          if (st.has_top && l >= aT && l <= aT + ov)
            A.bands[((((size_t)s * 2 + 0) * nt + (k - 1)) * (ov + 1) + (l - aT)) * nxp + m] = (double)uv;
          if (st.has_bot && l >= aB && l <= aB + ov)
            A.bands[((((size_t)(s - 1) * 2 + 1) * nt + (k - 1)) * (ov + 1) + (l - aB)) * nxp + m] = (double)uv;
        }
        if (MODE == 2 && out_lane && ok) A.UT[(size_t)(st.rowoff + l) * P + col] = uv;
      }
      // forcing at t^{k+1}: the first term from the prefetched row, further terms directly
      T z = fma(dta0, fpre[u], uv);
      if (MODE != 2 && ok)
        for (int r = 1; r < A.nforce; ++r)
          z += (T)A.dta[(size_t)k1 * A.nforce + r] * A.F[((size_t)r * (A.nv + 1) + lo + l) * P + col];
      zv[u] = z;
      // z^{k+1} at the trace rows, for the next pass (halo lanes hold a wrong u: their
      // upstream lane is missing)
      if (!PLAIN && MODE != 2 && robin_ov && out_lane) {
        if (st.has_top && (l == aT || l == aT - 1)) znext[(size_t)(0 * 2 + (aT - l)) * nxp + m] = (double)zv[u];
        if (st.has_bot && (l == bB || l == bB + 1)) znext[(size_t)(1 * 2 + (l - bB)) * nxp + m] = (double)zv[u];
      }
    }

    // (C) elimination of the previous row of every row of the group (its right-hand
    //     side M z needs z of both neighbours); zm2, zm1, g_last, a_last, w_last follow
    //     the rows in pass order
#pragma unroll
    for (int u = 0; u < kGroup; ++u) {
      const int t = t0 + u;
      if (PLAIN || u < n) {
        if (MODE != 2 && PLAIN) {  // an interior row: three elements, no interface data
          const T y = fma(-a_last, y_prev, g_last * fma(T(4), zm1, zm2 + zv[u]));
          if (out_lane) ynt[dP * (t - 1)] = y;
          y_prev = y;
        } else if (MODE != 2 && t >= 1) {
          const T rhs = (t == 1) ? fma(T(2), zm1, zv[u])  // end row: one element
                                 : fma(T(4), zm1, zm2 + zv[u]);
          eliminate(UP ? t - 1 : L - t, rhs, g_last, a_last);
        }
        zm2 = zm1;
        zm1 = zv[u];
        g_last = gpre[u];
        a_last = apre[u];
        w_last = wv[u];
      }
    }
  };

  load_group(0);
  for (int t0 = 0; t0 < L; t0 += kGroup) {
    const int n = L - t0 < kGroup ? L - t0 : kGroup;  // rows of this group (uniform)
#pragma unroll
    for (int u = 0; u < kGroup; ++u) {
      ypre[u] = ynx[u];
      fpre[u] = f0nx[u];
      cppre[u] = cpnx[u];
      gpre[u] = gnx[u];
      apre[u] = anx[u];
      cabpre[u] = cabnx[u];
      sgpre[u] = sgnx[u];
    }
    if (t0 + kGroup < L) load_group(t0 + kGroup);
    if (t0 >= t_plain0 && t0 <= t_plain1) run_group(BoolTag<true>{}, t0, kGroup);
    else run_group(BoolTag<false>{}, t0, n);
  }
  if (MODE != 2) {
    // the last row in pass order: an end row (one element)
    const T rhs = (L == 1) ? T(2) * zm1 : fma(T(2), zm1, zm2);
    eliminate(UP ? L - 1 : 0, rhs, g_last, a_last);
  }
}

}  // namespace kfp
