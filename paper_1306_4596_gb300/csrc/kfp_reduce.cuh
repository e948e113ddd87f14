// kfp_reduce.cuh -- the exchange and interface-error reductions of an SWR iteration
// and the mixed-precision defect-correction kernels (sm_103a); included by the host
// driver only (non-template kernels: one definition in the library).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "kfp_kernels.cuh"

namespace kfp {

// |d| as an integer whose order is that of |d|: the bit pattern without the sign
// (non-negative doubles order as their bits, and every NaN pattern lies above
// infinity, so a maximum over these keeps a NaN).  The maxima below run on the
// integer units; GB300's FP64 pipe is left the subtractions and squares.
__device__ __forceinline__ unsigned long long abs_key(double d) {
  return (unsigned long long)__double_as_longlong(d) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ double key_value(unsigned long long k) { return __longlong_as_double((long long)k); }

// Exchange: e_chg = max |lam_next - lam_prev| (trace change) into *chg, and
// lam_dst <- lam_next unless lam_dst is NULL.  lam_dst may be lam_prev (each element
// is read before it is written, by the same thread).  n is even (the data come in
// pairs of sides), so the arrays are read as 16-byte pairs; four pairs per thread
// and round are in flight at once.
__global__ void __launch_bounds__(kReduceThreads)
exchange_kernel(const double* __restrict__ lam_next, const double* lam_prev, double* lam_dst, size_t n,
                double* partial, unsigned* ticket, double* chg) {
  unsigned long long mk = 0;
  const double2* __restrict__ nx2 = reinterpret_cast<const double2*>(lam_next);
  const double2* pv2 = reinterpret_cast<const double2*>(lam_prev);
  double2* ds2 = reinterpret_cast<double2*>(lam_dst);
  const size_t n2 = n / 2, stride = (size_t)gridDim.x * blockDim.x;
  size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; e + 3 * stride < n2; e += 4 * stride) {
    double2 a[4], b[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) { a[r] = nx2[e + r * stride]; b[r] = pv2[e + r * stride]; }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      mk = max(mk, max(abs_key(a[r].x - b[r].x), abs_key(a[r].y - b[r].y)));
      if (ds2) ds2[e + r * stride] = a[r];
    }
  }
  for (; e < n2; e += stride) {
    const double2 a = nx2[e], b = pv2[e];
    mk = max(mk, max(abs_key(a.x - b.x), abs_key(a.y - b.y)));
    if (ds2) ds2[e] = a;
  }
  double mx = key_value(mk), sm = 0.0;
  block_reduce(mx, sm);
  last_block_combine(partial, ticket, mx, sm, chg, nullptr);
}

// Defect correction on the interface problem (mixed precision).  With G the map of
// one FP64 iteration, the residual of the current interface data lam is
// d = G(lam) - lam; the correction delta solves delta = M delta + d, where M is the
// linear part of G, by FP32 iterations of the homogeneous problem; then lam += delta.

// d = lam_next - lam_in (lam_in unchanged), scal[1] = max |d|.
__global__ void __launch_bounds__(kReduceThreads)
residual_kernel(const double* __restrict__ lam_next, const double* __restrict__ lam_in,
                double* __restrict__ d, size_t n, double* partial, unsigned* ticket, double* scal) {
  double mx = 0.0, sm = 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    const double r = lam_next[e] - lam_in[e];
    d[e] = r;
    mx = nan_max(mx, fabs(r));
  }
  block_reduce(mx, sm);
  last_block_combine(partial, ticket, mx, sm, &scal[1], nullptr);
}

// delta <- M delta + d, where lam_next holds M delta from the homogeneous sweep;
// scal[1] = max |new delta - old delta|.
__global__ void __launch_bounds__(kReduceThreads)
inner_exchange_kernel(const double* __restrict__ lam_next, const double* __restrict__ d,
                      double* __restrict__ delta, size_t n, double* partial, unsigned* ticket, double* scal) {
  double mx = 0.0, sm = 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    const double v = lam_next[e] + d[e];
    mx = nan_max(mx, fabs(v - delta[e]));
    delta[e] = v;
  }
  block_reduce(mx, sm);
  last_block_combine(partial, ticket, mx, sm, &scal[1], nullptr);
}

// lam_in += delta
__global__ void correct_kernel(double* __restrict__ lam_in, const double* __restrict__ delta, size_t n) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    lam_in[e] += delta[e];
}

// Error: e_mis = max |lower - upper| over the overlaps, j_l2 = dt hx sum (lower-upper)^2.
// Also appends (e_mis, e_chg, j_l2) to the device history, e_chg read from *chg and
// copied to scal[1].  Interface by interface, bands[j][0][r] is paired with
// bands[j][1][r] over the grid stride; when per_side is even both sides start on a
// 16-byte boundary and the values are read in pairs, four pairs per thread and round
// in flight at once.
__global__ void __launch_bounds__(kReduceThreads)
error_kernel(const double* __restrict__ bands, int nif, size_t per_side, double dthx,
             double* partial, unsigned* ticket, const double* chg, double* scal, double* hist, int* iter,
             int hist_cap, int wrap_nxp) {
  // wrap_nxp = nx + 1 with periodic x (column nx repeats column 0 and is left out of
  // the L2 sum), 0 otherwise; per_side is a multiple of nx + 1, so the column of
  // value r of a side is r mod (nx + 1)
  unsigned long long mk = 0;
  double sm = 0.0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t nxp = (size_t)wrap_nxp;
  // one value pair d of column m: max and (unless m is the repeated column) sum
  auto take = [&](double d, size_t m) {
    mk = max(mk, abs_key(d));
    if (nxp == 0 || m != nxp - 1) sm += d * d;
  };
  if ((per_side & 1) == 0) {
    const size_t n2 = per_side / 2;
    const size_t m_step = nxp ? (2 * stride) % nxp : 0;
    for (int j = 0; j < nif; ++j) {
      const double2* __restrict__ lo = reinterpret_cast<const double2*>(bands + (size_t)2 * j * per_side);
      const double2* __restrict__ up = reinterpret_cast<const double2*>(bands + ((size_t)2 * j + 1) * per_side);
      size_t m = nxp ? (2 * t0) % nxp : 0;  // column of the first value of pair e
      auto next = [&]() {
        if (nxp) {
          m += m_step;
          if (m >= nxp) m -= nxp;
        }
      };
      size_t e = t0;
      for (; e + 3 * stride < n2; e += 4 * stride) {
        double2 a[4], b[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) { a[k] = lo[e + k * stride]; b[k] = up[e + k * stride]; }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          take(a[k].x - b[k].x, m);
          take(a[k].y - b[k].y, nxp && m + 1 == nxp ? 0 : m + 1);
          next();
        }
      }
      for (; e < n2; e += stride) {
        const double2 a = lo[e], b = up[e];
        take(a.x - b.x, m);
        take(a.y - b.y, nxp && m + 1 == nxp ? 0 : m + 1);
        next();
      }
    }
  } else {
    const size_t m_step = nxp ? stride % nxp : 0;
    for (int j = 0; j < nif; ++j) {
      const double* __restrict__ lo = bands + (size_t)2 * j * per_side;
      const double* __restrict__ up = lo + per_side;
      size_t m = nxp ? t0 % nxp : 0;
      for (size_t e = t0; e < per_side; e += stride) {
        take(lo[e] - up[e], m);
        if (nxp) {
          m += m_step;
          if (m >= nxp) m -= nxp;
        }
      }
    }
  }
  double mx = key_value(mk);
  block_reduce(mx, sm);
  double emis = 0.0, ssum = 0.0;
  if (last_block_combine(partial, ticket, mx, sm, &emis, &ssum) && threadIdx.x == 0) {
    scal[0] = emis;
    scal[1] = *chg;
    scal[2] = dthx * ssum;
    const int it = *iter;
    const int slot = it < hist_cap ? it : hist_cap - 1;
    hist[3 * slot + 0] = scal[0];
    hist[3 * slot + 1] = scal[1];
    hist[3 * slot + 2] = scal[2];
    *iter = it + 1;
  }
}

// Periodic x on interface data [lines][nx+1]: column nx repeats column 0.
__global__ void periodic_trace_kernel(double* __restrict__ lam, size_t lines, int nx) {
  for (size_t l = (size_t)blockIdx.x * blockDim.x + threadIdx.x; l < lines; l += (size_t)gridDim.x * blockDim.x)
    lam[l * (nx + 1) + nx] = lam[l * (nx + 1)];
}

}  // namespace kfp
