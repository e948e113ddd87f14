// kfp_reduce.cuh -- the exchange and interface-error reductions of an SWR iteration
// and the mixed-precision defect-correction kernels (sm_103a); included by the host
// driver only (non-template kernels: one definition in the library).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "kfp_kernels.cuh"

namespace kfp {

// Exchange: e_chg = max |lam_next - lam_prev| (trace change) into *chg, and
// lam_dst <- lam_next unless lam_dst is NULL.  lam_dst may be lam_prev (each element
// is read before it is written, by the same thread).  n is even (the data come in
// pairs of sides), so the arrays are read as 16-byte pairs; four pairs per thread
// and round are in flight at once.
__global__ void __launch_bounds__(kReduceThreads)
exchange_kernel(const double* __restrict__ lam_next, const double* lam_prev, double* lam_dst, size_t n,
                double* partial, unsigned* ticket, double* chg) {
  double mx = 0.0, sm = 0.0;
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
      mx = nan_max(mx, nan_max(fabs(a[r].x - b[r].x), fabs(a[r].y - b[r].y)));
      if (ds2) ds2[e + r * stride] = a[r];
    }
  }
  for (; e < n2; e += stride) {
    const double2 a = nx2[e], b = pv2[e];
    mx = nan_max(mx, nan_max(fabs(a.x - b.x), fabs(a.y - b.y)));
    if (ds2) ds2[e] = a;
  }
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
// copied to scal[1].  Element e = j per_side + r
// of the flat range pairs bands[j][0][r] with bands[j][1][r]; the thread's position
// is advanced by the grid stride instead of being divided out per element, and four
// elements per thread and round are in flight at once.
__global__ void __launch_bounds__(kReduceThreads)
error_kernel(const double* __restrict__ bands, int nif, size_t per_side, double dthx,
             double* partial, unsigned* ticket, const double* chg, double* scal, double* hist, int* iter,
             int hist_cap, int wrap_nxp) {
  // wrap_nxp = nx + 1 with periodic x (column nx repeats column 0 and is left out of
  // the L2 sum), 0 otherwise
  double mx = 0.0, sm = 0.0;
  const size_t n = (size_t)nif * per_side, stride = (size_t)gridDim.x * blockDim.x;
  const size_t e0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  // per_side is a multiple of the row length, so the column of e is e mod (nx + 1)
  const size_t sj = stride / per_side, sr = stride - sj * per_side;
  const int scol = wrap_nxp ? (int)(stride % (size_t)wrap_nxp) : 0;
  struct Pos {
    size_t lo;  // index of bands[j][0][r]; bands[j][1][r] is lo + per_side
    size_t r;
    int m;
  };
  auto advance = [&](Pos p) {
    const size_t r2 = p.r + sr;
    const size_t wrap = r2 >= per_side ? 1 : 0;
    p.lo += (2 * (sj + wrap)) * per_side + sr - wrap * per_side;
    p.r = r2 - wrap * per_side;
    if (wrap_nxp) {
      p.m += scol;
      if (p.m >= wrap_nxp) p.m -= wrap_nxp;
    }
    return p;
  };
  Pos p;
  {
    const size_t j = e0 / per_side;
    p.r = e0 - j * per_side;
    p.lo = 2 * j * per_side + p.r;
    p.m = wrap_nxp ? (int)(e0 % (size_t)wrap_nxp) : 0;
  }
  size_t e = e0;
  for (; e + 3 * stride < n; e += 4 * stride) {
    Pos q[4];
    q[0] = p;
#pragma unroll
    for (int k = 1; k < 4; ++k) q[k] = advance(q[k - 1]);
    double lo[4], up[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) { lo[k] = bands[q[k].lo]; up[k] = bands[q[k].lo + per_side]; }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const double d = lo[k] - up[k];
      mx = nan_max(mx, fabs(d));
      if (wrap_nxp == 0 || q[k].m != wrap_nxp - 1) sm += d * d;
    }
    p = advance(q[3]);
  }
  for (; e < n; e += stride) {
    const double d = bands[p.lo] - bands[p.lo + per_side];
    mx = nan_max(mx, fabs(d));
    if (wrap_nxp == 0 || p.m != wrap_nxp - 1) sm += d * d;
    p = advance(p);
  }
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
