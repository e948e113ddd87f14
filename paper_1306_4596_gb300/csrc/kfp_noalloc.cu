// kfp_noalloc.cu -- interface norms computed without allocating any memory.
//
// kfp_iface_norms_noalloc reduces overlap values that the caller already holds in
// device memory to the same norms as kfp_swr_error (e_mis and j_l2; with periodic
// x the repeated column nx is counted once, as there), plus the same two norms per
// interface.  It is for callers that must not allocate: for
// example a plugin that a host application hands only its input and output
// buffers under a fixed device-memory budget, or a latency-critical loop that
// cannot afford cudaMalloc, which may synchronise the device and takes the
// allocator's lock.  Its only scratch memory is the file-scope array below,
// which every GPU that loads this library keeps until the process exits.
#include "../../include/kfp_swr.h"

#include <cuda_runtime.h>

#include <mutex>

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double keep_nan_max(double a, double b) {
  return (a != a || b != b) ? __longlong_as_double(0x7ff8000000000000LL) : fmax(a, b);
}

// (max, sum) over the block; valid in thread 0.
__device__ __forceinline__ void reduce_block(double& mx, double& sm) {
  __shared__ double smax[kThreads / 32], ssum[kThreads / 32];
  for (int o = 16; o > 0; o >>= 1) {
    mx = keep_nan_max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    sm += __shfl_xor_sync(0xffffffffu, sm, o);
  }
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { smax[wid] = mx; ssum[wid] = sm; }
  __syncthreads();
  if (wid == 0) {
    mx = lane < kThreads / 32 ? smax[lane] : 0.0;
    sm = lane < kThreads / 32 ? ssum[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      mx = keep_nan_max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      sm += __shfl_xor_sync(0xffffffffu, sm, o);
    }
  }
}

constexpr int kMaxIfaces = KFP_NOALLOC_MAX_INTERFACES;  // 64 interfaces
constexpr int kBlocksPerIface = 32;

// Per-(interface, block) partial results (max, sum of squares), one completion
// ticket per call and nothing else: 64 x 32 x 2 doubles = 32 KiB.
struct NoallocScratch {
  double partial[kMaxIfaces][kBlocksPerIface][2];
  unsigned ticket;
};
static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
NoallocScratch* g_scratch_ptr[kMaxDevices] = {};

// Set-up, once per device and with that device current: the device address of
// the scratch array (the host-side name is only a stand-in) and a zeroed ticket.
kfp_status scratch_for_current_device(NoallocScratch** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return KFP_ECUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return KFP_ECUDA;
    }
    if (cudaMemset(&static_cast<NoallocScratch*>(p)->ticket, 0, sizeof(unsigned)) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
      cudaGetLastError();
      return KFP_ECUDA;
    }
    g_scratch_ptr[dev] = static_cast<NoallocScratch*>(p);
  }
  *out = g_scratch_ptr[dev];
  return KFP_OK;
}

// grid (kBlocksPerIface, nif): block (b, j) reduces its share of interface j -- the
// rows (n, overlap node) b, b + kBlocksPerIface, ... of both sides, the first ncols
// columns of each (ncols = nx with periodic x, whose column nx repeats column 0 and
// is counted once, nx + 1 otherwise); the last block to finish combines all
// partials in a fixed order and re-arms the ticket.
__global__ void __launch_bounds__(kThreads)
iface_norms_noalloc_kernel(const double* __restrict__ bands, int nif, size_t nrows, int nxp, int ncols,
                           double dthx, NoallocScratch* scratch, double* __restrict__ out) {
  const int j = blockIdx.y;
  const size_t per_side = nrows * (size_t)nxp;
  const double* lower = bands + ((size_t)j * 2 + 0) * per_side;
  const double* upper = bands + ((size_t)j * 2 + 1) * per_side;
  double mx = 0.0, sm = 0.0;
  for (size_t row = blockIdx.x; row < nrows; row += gridDim.x) {
    const double* lo = lower + row * nxp;
    const double* up = upper + row * nxp;
    for (int m = threadIdx.x; m < ncols; m += blockDim.x) {
      const double d = lo[m] - up[m];
      mx = keep_nan_max(mx, fabs(d));
      sm += d * d;
    }
  }
  reduce_block(mx, sm);
  __shared__ bool is_last;
  if (threadIdx.x == 0) {
    scratch->partial[j][blockIdx.x][0] = mx;
    scratch->partial[j][blockIdx.x][1] = sm;
    __threadfence();
    const unsigned done = atomicAdd(&scratch->ticket, 1u);
    is_last = (done == gridDim.x * gridDim.y - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  if (threadIdx.x == 0) {
    const volatile double* part = &scratch->partial[0][0][0];
    double tmax = 0.0, tsum = 0.0;
    for (int jj = 0; jj < nif; ++jj) {
      double imax = 0.0, isum = 0.0;
      for (int b = 0; b < (int)gridDim.x; ++b) {
        imax = keep_nan_max(imax, part[((size_t)jj * kBlocksPerIface + b) * 2 + 0]);
        isum += part[((size_t)jj * kBlocksPerIface + b) * 2 + 1];
      }
      out[2 + 2 * jj + 0] = imax;
      out[2 + 2 * jj + 1] = dthx * isum;
      tmax = keep_nan_max(tmax, imax);
      tsum += isum;
    }
    out[0] = tmax;
    out[1] = dthx * tsum;
    scratch->ticket = 0u;  // ready for the next call
  }
}

}  // namespace

extern "C" kfp_status kfp_iface_norms_noalloc(const double* bands, int nif, int nt, int overlap_cells, int nx,
                                              int periodic_x, double dt, double hx, double* out,
                                              void* cuda_stream) {
  if (!bands || !out || nif < 1 || nt < 1 || overlap_cells < 0 || nx < 1 || !(dt > 0) || !(hx > 0))
    return KFP_EINVAL;
  if (periodic_x && nx < 2) return KFP_EINVAL;  // the periodic grid has at least two columns
  if (nif > kMaxIfaces) return KFP_EINVAL;       // more interfaces than the scratch array holds
  NoallocScratch* scratch = nullptr;
  kfp_status rc = scratch_for_current_device(&scratch);
  if (rc) return rc;
  const size_t nrows = (size_t)nt * (overlap_cells + 1);
  const dim3 grid(kBlocksPerIface, nif);
  iface_norms_noalloc_kernel<<<grid, kThreads, 0, (cudaStream_t)cuda_stream>>>(
      bands, nif, nrows, nx + 1, periodic_x ? nx : nx + 1, dt * hx, scratch, out);
  if (cudaGetLastError() != cudaSuccess) return KFP_ECUDA;
  return KFP_OK;
}
