// kfp_fe_tma.cuh -- TMA-fed sweep pass of the Lie splitting of Section 6.2 (sm_103a).
//
// The same fused pass as fe_pass_kernel (kfp_fe.cuh): back-substitution of step k
// (it yields w^k), upwind transport u^k = T w^k by warp shuffle, z = u^k + dt f^{k+1},
// and the elimination of step k+1 of (M + dt S) w = M z, one row behind (M z of a row
// needs z of both neighbours).  Its inputs come through the TMA ring of the unsplit
// sweep (producer warp, kfp_sweep_tma.cuh), and it stores a scaled residue:
//
//   the elimination of a pass is y_l = G_l R_l - H_l y_prev with G = g m_off, H = g a
//   (R_l = (M z)_l / m_off); the pass keeps yh_l = y_l / G_l instead, so that
//     yh_l = R_l - rho_l yh_prev,                  rho_l = H_l G_prev / G_l
//   and the next pass back-substitutes the scaled unknown wh = w / G (G of the
//   elimination that produced y) and transports with the scale folded in:
//     wh_l = yh_l - kappa_l wh_prev,               kappa_l = cp_l G_prev / G_l
//     z_l  = A'_l wh_l + B'_l wh_upwind + dt f_l,  A' = G (1 - c_l), B' = G c_l
//   (every column of a row has the same factors: periodic x).  A row costs six FP64
//   operations: one on each chain, two for z, two for R = z_- + 4 z + z_+.  The
//   true w = G wh is formed only where it is recorded (interface data) and the true
//   u = A' wh + B' wh_upwind where it is stored (overlap values, u at t = T).
//
// Coefficient record of one row and pass direction (24 = 3 column classes x 8
// fields, the three classes alike):
//   0: -kappa   1: A'   2: B'   3: -rho   4: G (of the back-substituted step)
//   5: unused   6: sign of v_i (integer bits)   7: unused
// kappa and rho are 0 on the first row in pass order.
#pragma once
#include <cuda_runtime.h>

#include "kfp_fe.cuh"
#include "kfp_slot.cuh"

namespace kfp {

// One unit's pass, consumer warps.  Rows are taken in pass order t = 0..L-1 (local
// row l = t going up, L-1-t going down), in chunks of SH::CH rows from the ring.
// A chunk whose rows, and the rows it eliminates (one behind), are all interior and
// record nothing runs branch-free: (A) the back-substitution chain interleaved with
// the previous chunk's deferred elimination chain, (B) z of every row, (C) the
// right-hand sides of the rows one behind, whose elimination chain is deferred.
// Every other chunk goes row by row (general path).
template <typename T, bool UP, int MODE, int FMODE, class SH>
__device__ __forceinline__ bool consume_fe_unit(const TmaArgs<T>& X, const FeArgs& E, const int k, const int s,
                                                const int bx, TmaSmem<T, SH>& sm, const unsigned cbase) {
  constexpr int CH = SH::CH, NST = SH::NST;
  const PassArgs<T>& A = X.p;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const StripInfo st = A.strips[s];
  const int L = st.L, lo = st.lo;
  const int NC = (L + CH - 1) / CH;
  const int wl = warp;
  const int w = bx * kWarpsPerBlock + wl;
  const bool warp_live = w < A.W;
  const int m = w * kOutCols - 1 + lane;
  const int col = m + 1;
  const bool in_dom = (m >= 0) && (m <= A.nx);
  const bool out_lane = warp_live && in_dom && lane >= 1 && lane <= kOutCols;
  const int cb = wl * kOutCols + lane;  // this lane's column in a tile
  const int P = A.P, nxp = A.nx + 1, nt = A.nt, ov = A.ov;
  const int k1 = k + 1;
  T* __restrict__ Ynext = (k1 & 1) ? A.Y1 : A.Y0;
  const bool robin_ov = A.robin && ov >= 1;
  const size_t zslab = (size_t)2 * 2 * nxp;
  const double* zcur = E.zrec + ((size_t)(k & 1) * A.S + s) * zslab;
  double* znext = E.zrec + ((size_t)(k1 & 1) * A.S + s) * zslab;
  T dtak = T(0);
  if (FMODE == 2 && MODE != 2) dtak = (T)A.dta[(size_t)k1 * A.nforce];

  // local rows of the outgoing data (as in fe_pass_kernel): top = alpha_s, bottom =
  // beta_{s-1}; the Robin data with overlap need the row next to each
  const int aT = st.has_top ? st.alpha_top - lo : -10;
  const int bB = st.has_bot ? st.alpha_bot - lo + ov : -10;
  const int aB = st.alpha_bot - lo;
  // rows the general path must take: the band rows and trace rows with a margin of
  // one on each side (the z records and the w of the neighbouring row)
  int rloB = 1, rhiB = 0, rloT = 1, rhiT = 0;
  if (st.has_bot) { rloB = aB - 1; rhiB = bB + 2; }
  if (st.has_top) { rloT = aT - 2; rhiT = aT + ov + 1; }

  // interface data of this strip: at t^{k+1} for the end rows of the system being
  // eliminated, at t^k for the Robin data without overlap recorded from w^k
  double lam_rhs_top = 0.0, lam_rhs_bot = 0.0, lam_rec_top = 0.0, lam_rec_bot = 0.0;
  if (in_dom) {
    const bool rec_in = MODE != 0 && A.robin && ov == 0;
    if (st.has_top) {
      const double* src = A.lam_in + ((size_t)s * 2 + 0) * nt * nxp + m;
      if (MODE != 2) lam_rhs_top = src[(size_t)k * nxp];
      if (rec_in) lam_rec_top = src[(size_t)(k - 1) * nxp];
    }
    if (st.has_bot) {
      const double* src = A.lam_bot_src + ((size_t)(s - 1) * 2 + 1) * nt * nxp + m;
      if (MODE != 2) lam_rhs_bot = src[(size_t)k * nxp];
      if (rec_in) lam_rec_bot = src[(size_t)(k - 1) * nxp];
    }
  }

  // carried state, all in pass order: wh of the previous row and its true w, z of the
  // two previous rows, the scaled residue of the last eliminated row, -rho of the
  // previous row (its elimination waits for z of this one)
  T wh_prev = T(0), w_last = T(0), zm1 = T(0), zm2 = T(0), yh_prev = T(0), nrho_last = T(0);
  auto yrow = [&](int t) { return Ynext + (size_t)(st.rowoff + (UP ? t : L - 1 - t)) * P + col; };

  // right-hand side of row t (pass order) from z of rows t-1, t, t+1 (zp = z_{t-1},
  // zc = z_t, zn = z_{t+1}; an end row has one neighbour), plus its interface data
  auto end_rhs = [&](int t, T zc, T znb, bool single) -> T {
    const int l = UP ? t : L - 1 - t;
    T R = single ? T(2) * zc : fma(T(2), zc, znb);
    if (l == L - 1 && st.has_top)
      R = A.robin ? (T)((double)R + E.dt_mo * lam_rhs_top) : (T)(lam_rhs_top * E.inv_mo);
    if (l == 0 && st.has_bot)
      R = A.robin ? (T)((double)R + E.dt_mo * lam_rhs_bot) : (T)(lam_rhs_bot * E.inv_mo);
    return R;
  };

  // One row t (pass order) at tile row r of stage q, general path: back-substitution
  // (or u^0 in the first pass), the outgoing data of t^k, the overlap values, u^nt in
  // the last pass, z with its records, and the elimination of row t-1.  The z and
  // right-hand-side arithmetic is the branch-free path's, operation for operation.
  auto general_row = [&](int t, int q, int r) {
    const int l = UP ? t : L - 1 - t;
    const T* rc = &sm.rec[q][r][8];  // the three column classes are alike
    T gterm = T(0);
    if (MODE != 2) {
      if (FMODE == 1) gterm = sm.frc[q][r][cb];
      if (FMODE == 2) gterm = dtak * sm.frc[q][r][cb];
    }
    T z;
    if (MODE == 0) {
      z = sm.tile[q][r][cb] + gterm;
    } else {
      const T wh = fma(rc[0], wh_prev, sm.tile[q][r][cb]);
      const T wcur = rc[4] * wh;  // the true w^k of this row
      if (out_lane) {
        if (st.has_top) {
          const int eT = robin_ov ? (UP ? aT : aT - 1) : aT;  // the later of alpha, alpha-1
          if (l == eT) {
            const double wa = robin_ov && !UP ? (double)w_last : (double)wcur;  // w(alpha)
            double lam;
            if (!A.robin) {
              lam = wa;
            } else if (ov >= 1) {
              const double wb = UP ? (double)w_last : (double)wcur;  // w(alpha - 1)
              const double* zk = zcur;                                // z^k at alpha, alpha-1
              lam = st.q_top * wa -
                    E.inv_dt * (E.k_half * wa + E.k_off * wb - E.m_half * zk[m] - E.m_off * zk[nxp + m]);
            } else {
              lam = (st.p_top + st.q_top) * wa - lam_rec_top;
            }
            const size_t o = (((size_t)s * 2 + 1) * nt + (k - 1)) * nxp + m;
            A.lam_next[o] = A.lam_add ? lam + A.lam_add[o] : lam;
          }
        }
        if (st.has_bot) {
          const int eB = robin_ov ? (UP ? bB + 1 : bB) : bB;  // the later of beta, beta+1
          if (l == eB) {
            const double wbeta = robin_ov && UP ? (double)w_last : (double)wcur;  // w(beta)
            double lam;
            if (!A.robin) {
              lam = wbeta;
            } else if (ov >= 1) {
              const double wu = UP ? (double)wcur : (double)w_last;  // w(beta + 1)
              const double* zk = zcur + 2 * nxp;                      // z^k at beta, beta+1
              lam = st.p_bot * wbeta -
                    E.inv_dt * (E.k_half * wbeta + E.k_off * wu - E.m_half * zk[m] - E.m_off * zk[nxp + m]);
            } else {
              lam = (st.p_bot + st.q_bot) * wbeta - lam_rec_bot;
            }
            const size_t o = ((((size_t)s - 1) * 2 + 0) * nt + (k - 1)) * nxp + m;
            A.lam_next[o] = A.lam_add ? lam + A.lam_add[o] : lam;
          }
        }
      }
      const T whnb = shfl_val(wh, lane - slot_int(rc[6]));
      if (out_lane && ((st.has_top && l >= aT && l <= aT + ov) || (st.has_bot && l >= aB && l <= aB + ov) ||
                       MODE == 2)) {
        const T u = fma(rc[1], wh, rc[2] * whnb);  // the true u^k
        if (st.has_top && l >= aT && l <= aT + ov)
          A.bands[((((size_t)s * 2 + 0) * nt + (k - 1)) * (ov + 1) + (l - aT)) * nxp + m] = (double)u;
        if (st.has_bot && l >= aB && l <= aB + ov)
          A.bands[((((size_t)(s - 1) * 2 + 1) * nt + (k - 1)) * (ov + 1) + (l - aB)) * nxp + m] = (double)u;
        if (MODE == 2) A.UT[(size_t)(st.rowoff + l) * P + col] = u;
      }
      wh_prev = wh;
      w_last = wcur;
      if (MODE == 2) return;
      z = fma(rc[1], wh, fma(rc[2], whnb, gterm));
    }
    // z^{k+1} at the trace rows, for the next pass (halo lanes hold a wrong z: their
    // upstream lane is missing)
    if (robin_ov && out_lane) {
      if (st.has_top && (l == aT || l == aT - 1)) znext[(size_t)(0 * 2 + (aT - l)) * nxp + m] = (double)z;
      if (st.has_bot && (l == bB || l == bB + 1)) znext[(size_t)(1 * 2 + (l - bB)) * nxp + m] = (double)z;
    }
    // elimination of row t-1 (its right-hand side needed z of this row)
    if (t >= 1) {
      const T R = (t == 1) ? end_rhs(0, zm1, z, false) : fma(T(4), zm1, zm2 + z);
      const T yh = fma(nrho_last, yh_prev, R);
      if (out_lane) *yrow(t - 1) = yh;
      yh_prev = yh;
    }
    zm2 = zm1;
    zm1 = z;
    nrho_last = rc[3];
  };

  // The deferred elimination chain of the last branch-free chunk: -rho and the
  // right-hand sides of its rows one behind, and where their residues go.
  bool pend = false;
  T nr[CH], Rd[CH];
  T* pout = nullptr;
  const ptrdiff_t step = UP ? (ptrdiff_t)P : -(ptrdiff_t)P;
  auto drain = [&]() {
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      yh_prev = fma(nr[u], yh_prev, Rd[u]);
      if (out_lane) *pout = yh_prev;
      pout += step;
    }
    pend = false;
  };

  for (int c = 0; c < NC; ++c) {
    const unsigned g = cbase + (unsigned)c;
    const int q = (int)(g % NST);
    if (!mbar_wait(&sm.full[q], (g / NST) & 1)) {
      atomicExch(X.flag, 1);
      return false;
    }
    const int t0 = c * CH;
    // local rows of the chunk and of the row before it (the first row it eliminates)
    const int la = UP ? t0 - 1 : L - t0, lb = UP ? t0 + CH - 1 : L - 1 - (t0 + CH - 1);
    const int lmin = la < lb ? la : lb, lmax = la < lb ? lb : la;
    const bool touches = (rloB <= rhiB && !(lmax < rloB || lmin > rhiB)) ||
                         (rloT <= rhiT && !(lmax < rloT || lmin > rhiT));
    const int sg_first = slot_int(sm.rec[q][0][8 + 6]);
    const int sg_last = slot_int(sm.rec[q][CH - 1][8 + 6]);
    const bool fast = MODE != 2 && t0 >= 2 && t0 + CH <= L && !touches && sg_first * sg_last >= 0;
    if (fast) {
      const int src = lane - (sg_first != 0 ? sg_first : sg_last);  // upwind lane of the chunk
      // (A) back-substitution chain, interleaved with the deferred elimination chain
      T wv[CH];
      if (MODE == 0) {
        if (pend) drain();
#pragma unroll
        for (int u = 0; u < CH; ++u) wv[u] = sm.tile[q][UP ? u : CH - 1 - u][cb];
      } else if (pend) {
#pragma unroll
        for (int u = 0; u < CH; ++u) {
          const int r = UP ? u : CH - 1 - u;
          wh_prev = fma(sm.rec[q][r][8 + 0], wh_prev, sm.tile[q][r][cb]);
          wv[u] = wh_prev;
          yh_prev = fma(nr[u], yh_prev, Rd[u]);
          if (out_lane) *pout = yh_prev;
          pout += step;
        }
        pend = false;
      } else {
#pragma unroll
        for (int u = 0; u < CH; ++u) {
          const int r = UP ? u : CH - 1 - u;
          wh_prev = fma(sm.rec[q][r][8 + 0], wh_prev, sm.tile[q][r][cb]);
          wv[u] = wh_prev;
        }
      }
      // (B) z of every row (independent of one another)
      T zv[CH];
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const int r = UP ? u : CH - 1 - u;
        T gterm = T(0);
        if (FMODE == 1) gterm = sm.frc[q][r][cb];
        if (FMODE == 2) gterm = dtak * sm.frc[q][r][cb];
        if (MODE == 0) {
          zv[u] = wv[u] + gterm;
        } else {
          const T whnb = shfl_val(wv[u], src);
          zv[u] = fma(sm.rec[q][r][8 + 1], wv[u], fma(sm.rec[q][r][8 + 2], whnb, gterm));
        }
      }
      if (MODE != 0) w_last = sm.rec[q][UP ? CH - 1 : 0][8 + 4] * wv[CH - 1];
      // (C) right-hand sides of rows t0-1 .. t0+CH-2 and their -rho; their
      //     elimination chain runs with the next chunk's back-substitution
      Rd[0] = fma(T(4), zm1, zm2 + zv[0]);
      nr[0] = nrho_last;
      Rd[1] = fma(T(4), zv[0], zm1 + zv[1]);
#pragma unroll
      for (int u = 2; u < CH; ++u) Rd[u] = fma(T(4), zv[u - 1], zv[u - 2] + zv[u]);
#pragma unroll
      for (int u = 1; u < CH; ++u) nr[u] = sm.rec[q][UP ? u - 1 : CH - u][8 + 3];
      nrho_last = sm.rec[q][UP ? CH - 1 : 0][8 + 3];
      zm2 = zv[CH - 2];
      zm1 = zv[CH - 1];
      pout = yrow(t0 - 1);
      pend = true;
    } else {
      if (pend) drain();
#pragma unroll 1
      for (int u = 0; u < CH; ++u) {
        const int t = t0 + u;
        if (t >= L) break;  // rows beyond the strip (uniform)
        general_row(t, q, UP ? u : CH - 1 - u);
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&sm.empty[q]);
  }
  if (pend) drain();
  if (MODE != 2) {
    // the last row in pass order: an end row (one element)
    const T R = end_rhs(L - 1, zm1, zm2, L == 1);
    const T yh = fma(nrho_last, yh_prev, R);
    if (out_lane) *yrow(L - 1) = yh;
  }
  return true;
}

// Passes of the split scheme, one launch per slot of pipelined iterates (as
// sweep_slot_kernel; one iterate at a time is a slot of one): every unit of the grid
// (blockIdx.x: column block, blockIdx.y: strip from X.p.strip0, blockIdx.z: iterate);
// the producer warp streams the scaled residue (or u^0), the pre-scaled forcing and
// the records through the ring.
template <typename T>
struct FeSlotArgs {
  TmaMaps maps[kSlotMax];
  TmaArgs<T> X[kSlotMax];
  FeArgs E[kSlotMax];
  int k[kSlotMax];
};

template <typename T, bool UP, int MODE, int FMODE, class SH>
__global__ void __launch_bounds__((kWarpsPerBlock + 1) * 32, SH::MINB)
fe_slot_kernel(const __grid_constant__ FeSlotArgs<T> G) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  TmaSmem<T, SH>& sm = *reinterpret_cast<TmaSmem<T, SH>*>(smem_raw);
  init_ring(sm);
  const int z = blockIdx.z;
  const TmaArgs<T>& X = G.X[z];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.y + X.p.strip0, bx = blockIdx.x;
  if (warp == kWarpsPerBlock) {
    if (lane != 0) return;
    const StripInfo st = X.p.strips[s];
    (void)produce_unit<T, UP, MODE, FMODE, SH>(G.maps[z], X, G.k[z], s, bx, st, sm, 0u, nullptr);
    return;
  }
  (void)consume_fe_unit<T, UP, MODE, FMODE, SH>(X, G.E[z], G.k[z], s, bx, sm, 0u);
}

}  // namespace kfp
