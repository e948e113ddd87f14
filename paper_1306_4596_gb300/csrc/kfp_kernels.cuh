// kfp_kernels.cuh -- sm_103a kernels of the SWR sweep for the Kolmogorov equation.
//
// Sweep (one kernel launch per time step, all strips at once).
//   The implicit-Euler system of step k in every (strip, column) is tridiagonal in v
//   with constant coefficients per strip and column class (m = 0, interior, m = nx),
//   so its LU factors are computed once on the host.  A time step needs an
//   elimination sweep and a back-substitution sweep in opposite row orders.  This
//   kernel fuses the back-substitution of step k with the elimination of step k+1:
//   each pass walks the rows of every column once, in the order in which step k's
//   back-substitution produces u^k, and immediately builds the right-hand side of
//   step k+1 from it (upwind transport + forcing + interface data) and eliminates
//   it.  Consecutive passes therefore alternate between ascending and descending
//   row order (step k+1 is factored "upward" when k+1 is odd and "downward" when it
//   is even), and the only state kept between passes is the elimination residue
//   y^{k+1} of every node: one read and one write per node and step.
//
//   Lanes of a warp own 32 consecutive x-columns and walk the rows in lockstep; the
//   upwind neighbour u^k_{i,m-1} or u^k_{i,m+1} of the same row comes from a warp
//   shuffle.  Lanes 1..30 produce output; lanes 0 and 31 are halo columns that
//   recompute their neighbour's back-substitution (their y^k is complete in memory)
//   so that no warp waits for another inside a pass.
//
//   Interface rows (Section 6.3, SWR1/SWR3): Dirichlet u = lambda, or the half-cell
//   Robin rows; the outgoing interface data (SWR2/SWR4: lambda_2 = Q_2 u at alpha,
//   lambda_1 = Q_1 u at beta) and the overlap values are recorded during the pass
//   that produces u^k.
//
// The warp and block reductions used by the exchange and error kernels (grid-stride,
// warp shuffles, deterministic last-block final reduction) live here; the kernels
// themselves are in kfp_reduce.cuh.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace kfp {

constexpr int kOutCols = 30;   // output columns per warp (lanes 1..30)
constexpr int kWarpsPerBlock = 4;
constexpr int kReduceThreads = 256;

struct StripInfo {
  int lo, hi, L, rowoff;       // global node range [lo, hi], L = hi-lo+1, first row in Y
  int has_bot, has_top;        // interface below / above
  int alpha_bot, alpha_top;    // alpha node of interface s-1 / s (global)
  double p_top, q_top;         // Robin parameters of interface s
  double p_bot, q_bot;         // Robin parameters of interface s-1
};

template <typename T>
struct PassArgs {
  int nx, nv, nt, S, ov, P, W, Lmax, nforce, robin;
  int neumann_v, periodic_x;   // model-problem boundary conditions (Section 6.1)
  double two_dt_hv;            // 2 dt / hv (Robin row)
  double inv_2hv;              // 1 / (2 hv) (centred difference of the Robin trace)
  const StripInfo* strips;     // [S]
  const T* coef;               // [S][3 classes][2 directions][3 fields][Lmax]: g, coupling, cp
  const T* cabs;               // [nv+1] |v_i| dt / hx
  const signed char* sgn;      // [nv+1] sign of v_i
  const T* U0;                 // [nv+1][P] initial data, column m stored at m+1
  const T* F;                  // [nforce][nv+1][P]
  const double* dta;           // [nt+1][nforce] dt * a_r(t^n)
  const double* bc_xin;        // [nt+1][2][nv+1] or nullptr
  const double* bc_v;          // [nt+1][2][nx+1] or nullptr
  const double* lam_in;        // [S-1][2][nt][nx+1] interface data of the previous iterate
  const double* lam_bot_src;   // where a strip reads its lower interface data: lam_in (parallel
                               // form) or lam_next (serial form: the strip below, this iterate)
  int strip0;                  // strip of blockIdx.y = 0 (the serial form launches one strip at a time)
  double* lam_next;            // same shape, written by the sweep
  const double* lam_add;       // NULL, or added to every value written to lam_next (the
                               // right-hand side d of a correction solve delta = M delta + d,
                               // TMA-fed sweep only)
  double* bands;               // [S-1][2][nt][ov+1][nx+1]
  T* Y0;                       // [rows][P] elimination residue, even steps
  T* Y1;                       // odd steps
  T* UT;                       // [rows][P] state at t = T
};

// compile-time flag for a generic lambda instantiated on two code paths
template <bool B>
struct BoolTag {
  static constexpr bool value = B;
};

__device__ __forceinline__ double shfl_val(double v, int src) {
  return __shfl_sync(0xffffffffu, v, src);
}
__device__ __forceinline__ float shfl_val(float v, int src) {
  return __shfl_sync(0xffffffffu, v, src);
}

// MODE 0: first pass (eliminate step 1 from u^0); 1: back-substitute step k and
// eliminate step k+1; 2: back-substitute the last step and store u^nt.
// UP: rows in ascending order.
template <typename T, bool UP, int MODE>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
sweep_pass_kernel(const PassArgs<T> A, const int k) {
  const int lane = threadIdx.x & 31;
  const int w = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (w >= A.W) return;  // whole warp leaves together
  const int s = blockIdx.y + A.strip0;
  const StripInfo st = A.strips[s];
  const int m = w * kOutCols - 1 + lane;
  const int col = m + 1;
  const bool in_dom = (m >= 0) && (m <= A.nx);
  const bool out_lane = in_dom && lane >= 1 && lane <= kOutCols;
  const int kappa = (m <= 0) ? 0 : (m >= A.nx ? 2 : 1);
  const int inflow_side = (m == 0) ? 0 : (m == A.nx ? 1 : -1);
  const int L = st.L, lo = st.lo, P = A.P, nxp = A.nx + 1, nt = A.nt;
  const int dirE = UP ? 0 : 1;  // elimination direction of step k+1 = this pass's direction
  const int dirB = UP ? 1 : 0;  // step k was eliminated the other way
  const T* __restrict__ gE = A.coef + ((size_t)((s * 3 + kappa) * 2 + dirE) * 3 + 0) * A.Lmax;
  const T* __restrict__ aE = A.coef + ((size_t)((s * 3 + kappa) * 2 + dirE) * 3 + 1) * A.Lmax;
  const T* __restrict__ cpB = A.coef + ((size_t)((s * 3 + kappa) * 2 + dirB) * 3 + 2) * A.Lmax;
  const T* __restrict__ Ycur = (k & 1) ? A.Y1 : A.Y0;
  T* __restrict__ Ynext = ((k + 1) & 1) ? A.Y1 : A.Y0;
  const int k1 = k + 1;  // time level of the system being eliminated

  // recording geometry (local rows)
  const int ov = A.ov;
  const int aT = st.alpha_top - lo;        // top overlap starts at alpha_s
  const int aB = st.alpha_bot - lo;        // bottom overlap starts at alpha_{s-1} (= 0)
  const bool robin_in = A.robin && ov >= 1;
  const int eT = robin_in ? (UP ? aT + 1 : aT - 1) : aT;           // row that emits lambda_2
  const int eB = robin_in ? (UP ? aB + ov + 1 : aB + ov - 1) : aB + ov;  // row that emits lambda_1

  T u_prev = T(0), u_m1 = T(0), u_m2 = T(0), y_prev = T(0);
  for (int t = 0; t < L; ++t) {
    const int l = UP ? t : (L - 1 - t);
    const int i = lo + l;
    const size_t e = (size_t)(st.rowoff + l) * P + col;
    T u;
    if (MODE == 0) {
      u = A.U0[(size_t)i * P + col];
    } else {
      const T y = Ycur[e];
      u = y - cpB[l] * u_prev;
      u_prev = u;
      // ---- record u^k on the overlaps and the outgoing interface data ----
      if (st.has_top) {
        if (l >= aT && l <= aT + ov && out_lane)
          A.bands[((((size_t)s * 2 + 0) * nt + (k - 1)) * (ov + 1) + (l - aT)) * nxp + m] = (double)u;
        if (l == eT && out_lane) {
          double lam;
          if (!A.robin) {
            lam = (double)u;
          } else if (ov >= 1) {
            const double d = UP ? ((double)u - (double)u_m2) : ((double)u_m2 - (double)u);
            lam = st.q_top * (double)u_m1 - d * A.inv_2hv;
          } else {
            lam = (st.p_top + st.q_top) * (double)u -
                  A.lam_in[(((size_t)s * 2 + 0) * nt + (k - 1)) * nxp + m];
          }
          A.lam_next[(((size_t)s * 2 + 1) * nt + (k - 1)) * nxp + m] = lam;
        }
      }
      if (st.has_bot) {
        if (l >= aB && l <= aB + ov && out_lane)
          A.bands[((((size_t)(s - 1) * 2 + 1) * nt + (k - 1)) * (ov + 1) + (l - aB)) * nxp + m] = (double)u;
        if (l == eB && out_lane) {
          double lam;
          if (!A.robin) {
            lam = (double)u;
          } else if (ov >= 1) {
            const double d = UP ? ((double)u - (double)u_m2) : ((double)u_m2 - (double)u);
            lam = st.p_bot * (double)u_m1 + d * A.inv_2hv;
          } else {
            lam = (st.p_bot + st.q_bot) * (double)u -
                  A.lam_bot_src[((((size_t)s - 1) * 2 + 1) * nt + (k - 1)) * nxp + m];
          }
          A.lam_next[((((size_t)s - 1) * 2 + 0) * nt + (k - 1)) * nxp + m] = lam;
        }
      }
      u_m2 = u_m1;
      u_m1 = u;
      if (MODE == 2) {
        if (out_lane) A.UT[e] = u;
        continue;
      }
    }

    // ---- right-hand side of step k+1 at row i, then elimination ----
    const int sg = A.sgn[i];
    const T unb = shfl_val(u, lane - sg);  // upwind neighbour of the same row
    T R;
    if (!A.neumann_v && (i == 0 || i == A.nv)) {
      R = (A.bc_v && in_dom) ? (T)A.bc_v[((size_t)k1 * 2 + (i == 0 ? 0 : 1)) * nxp + m] : T(0);
    } else if (!A.periodic_x && ((inflow_side == 0 && sg > 0) || (inflow_side == 1 && sg < 0))) {
      R = A.bc_xin ? (T)A.bc_xin[((size_t)k1 * 2 + inflow_side) * (A.nv + 1) + i] : T(0);
    } else {
      R = u - A.cabs[i] * (u - unb);
      for (int r = 0; r < A.nforce; ++r)
        R += (T)A.dta[(size_t)k1 * A.nforce + r] * A.F[((size_t)r * (A.nv + 1) + i) * P + col];
      if (l == L - 1 && st.has_top) {
        const double lam = in_dom ? A.lam_in[(((size_t)s * 2 + 0) * nt + k) * nxp + m] : 0.0;
        R = A.robin ? (T)((double)R + A.two_dt_hv * lam) : (T)lam;
      } else if (l == 0 && st.has_bot) {
        const double lam = in_dom ? A.lam_bot_src[((((size_t)s - 1) * 2 + 1) * nt + k) * nxp + m] : 0.0;
        R = A.robin ? (T)((double)R + A.two_dt_hv * lam) : (T)lam;
      }
    }
    const T y = gE[l] * (R - aE[l] * y_prev);
    if (out_lane) Ynext[e] = y;
    y_prev = y;
  }
}

// ---------------------------------------------------------------------------
// Reductions
// ---------------------------------------------------------------------------

// max that keeps a NaN (fmax would drop it), so that a blown-up iterate is reported
__device__ __forceinline__ double nan_max(double a, double b) {
  return (a != a || b != b) ? __longlong_as_double(0x7ff8000000000000LL) : fmax(a, b);
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = nan_max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide reduction of (max, sum); result valid in thread 0.
__device__ __forceinline__ void block_reduce(double& mx, double& sm) {
  __shared__ double smax[kReduceThreads / 32], ssum[kReduceThreads / 32];
  mx = warp_max(mx);
  sm = warp_sum(sm);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { smax[wid] = mx; ssum[wid] = sm; }
  __syncthreads();
  if (wid == 0) {
    mx = lane < (int)(blockDim.x >> 5) ? smax[lane] : 0.0;
    sm = lane < (int)(blockDim.x >> 5) ? ssum[lane] : 0.0;
    mx = warp_max(mx);
    sm = warp_sum(sm);
  }
}

// Final step shared by both reductions: the last block to finish combines the
// per-block partials into result[0..1] in a fixed order -- thread t takes blocks t,
// t + blockDim, ... in turn, then the fixed shuffle tree of block_reduce -- so that the
// result does not depend on which block finished last (reproducible bit for bit).
// out_sum may be NULL (no sum wanted).
__device__ __forceinline__ bool last_block_combine(double* partial, unsigned* ticket, double mx,
                                                   double sm, double* out_max, double* out_sum) {
  __shared__ bool is_last;
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x + 0] = mx;
    partial[2 * blockIdx.x + 1] = sm;
    __threadfence();
    const unsigned done = atomicAdd(ticket, 1u);
    is_last = (done == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  double m2 = 0.0, s2 = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
    m2 = nan_max(m2, ((volatile double*)partial)[2 * b + 0]);
    if (out_sum) s2 += ((volatile double*)partial)[2 * b + 1];
  }
  block_reduce(m2, s2);
  if (threadIdx.x == 0) {
    *out_max = m2;
    if (out_sum) *out_sum = s2;
    *ticket = 0u;
  }
  return true;
}

// Periodic x on a padded [nrows][P] array (column m at m+1): column nx repeats
// column 0, and the ghost columns -1 and nx+1 hold columns nx-1 and 1, so that the
// halo lanes of the next pass see the wrapped upwind neighbours.  Needs nx >= 2.
template <typename T>
__device__ __forceinline__ void periodic_wrap_rows(T* __restrict__ a, int nrows, int P, int nx) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nrows; r += gridDim.x * blockDim.x) {
    T* row = a + (size_t)r * P;
    const T c0 = row[1], c1 = row[2], clast = row[nx];
    row[0] = clast;
    row[nx + 1] = c0;
    row[nx + 2] = c1;
  }
}
template <typename T>
__global__ void periodic_wrap_kernel(T* __restrict__ a, int nrows, int P, int nx) {
  periodic_wrap_rows(a, nrows, P, nx);
}
// The same for up to four arrays at once (blockIdx.y selects one): the pipelined
// iterates of one slot.
template <typename T>
struct WrapGroup {
  T* a[4];
};
template <typename T>
__global__ void periodic_wrap_group_kernel(const WrapGroup<T> g, int nrows, int P, int nx) {
  periodic_wrap_rows(g.a[blockIdx.y], nrows, P, nx);
}

// u(T) assembled from the strips: row i taken from row_of[i] of UT.
template <typename T>
__global__ void gather_solution_kernel(const T* __restrict__ UT, const int* __restrict__ row_of,
                                       int nv, int nx, int P, double* __restrict__ dst) {
  const size_t n = (size_t)(nv + 1) * (nx + 1);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / (nx + 1)), m = (int)(e - (size_t)i * (nx + 1));
    dst[e] = (double)UT[(size_t)row_of[i] * P + m + 1];
  }
}

// Copy [rows][nx+1] FP64 into the padded [rows][P] layout (column m at m+1), as T.
template <typename T>
__global__ void pad_rows_kernel(const double* __restrict__ src, int rows, int nx, int P,
                                T* __restrict__ dst) {
  const size_t n = (size_t)rows * (nx + 1);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / (nx + 1)), m = (int)(e - (size_t)i * (nx + 1));
    dst[(size_t)i * P + m + 1] = (T)src[e];
  }
}

}  // namespace kfp
