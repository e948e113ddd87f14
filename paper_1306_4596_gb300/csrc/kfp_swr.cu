// kfp_swr.cu -- C ABI (include/kfp_swr.h) and host driver of the GB300 SWR sweep.
//
// One handle = one problem resident in HBM.  Per SWR iteration (Section 6.3,
// SWR1-SWR4 in the parallel form of the Remark) the driver enqueues
//   nt+1 sweep passes (kfp_kernels.cuh: back-substitution of step k fused with the
//   elimination of step k+1, all strips and columns at once),
//   the exchange kernel (new interface data -> current, trace change), and
//   the error kernel (overlap mismatch e_mis and its squared L2 norm),
// either as direct launches or as one replayed CUDA graph.
#include "../../include/kfp_swr.h"
#include "kfp_kernels.cuh"
#include "kfp_reduce.cuh"
#include "kfp_sweep_tma.cuh"
#include "kfp_launch.h"
#include "kfp_adjoint.cuh"
#include "kfp_fe.cuh"

#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

namespace {

thread_local std::string g_create_error;

// NVTX range for the host timeline of a profiler (kfp.iteration, kfp.sweep,
// kfp.exchange, kfp.error): it marks where the host enqueues (or captures) the
// work; device times come from CUDA events or the profiler's kernel list.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Runtime choice of the tile shape of the TMA-fed sweep (kfp_launch.h).
template <typename T>
struct Tma {
  static size_t smem_bytes(int sh) {
    return sh == 0 ? kfp::LaunchSet<T, 0>::smem_bytes()
                   : (sh == 1 ? kfp::LaunchSet<T, 1>::smem_bytes() : kfp::LaunchSet<T, 2>::smem_bytes());
  }
  static cudaError_t set_attrs() {
    cudaError_t e = kfp::LaunchSet<T, 0>::set_attrs();
    if (e == cudaSuccess) e = kfp::LaunchSet<T, 1>::set_attrs();
    if (e == cudaSuccess) e = kfp::LaunchSet<T, 2>::set_attrs();
    return e;
  }
  static int blocks_per_sm(int sh, int fmode) {
    return sh == 0 ? kfp::LaunchSet<T, 0>::blocks_per_sm(fmode)
                   : (sh == 1 ? kfp::LaunchSet<T, 1>::blocks_per_sm(fmode) : kfp::LaunchSet<T, 2>::blocks_per_sm(fmode));
  }
  static void pass(int sh, int fmode, bool up, int mode, dim3 grid, cudaStream_t st, const kfp::TmaMaps& maps,
                   const kfp::TmaArgs<T>& X, int k) {
    if (sh == 0) kfp::LaunchSet<T, 0>::pass(fmode, up, mode, grid, st, maps, X, k);
    else if (sh == 1) kfp::LaunchSet<T, 1>::pass(fmode, up, mode, grid, st, maps, X, k);
    else kfp::LaunchSet<T, 2>::pass(fmode, up, mode, grid, st, maps, X, k);
  }
  static cudaError_t stream(int sh, int fmode, unsigned grid, cudaStream_t st, const kfp::StreamProblem<T>* probs,
                            const kfp::StreamArgs& P) {
    if (sh == 0) return kfp::LaunchSet<T, 0>::stream(fmode, grid, st, probs, P);
    if (sh == 1) return kfp::LaunchSet<T, 1>::stream(fmode, grid, st, probs, P);
    return kfp::LaunchSet<T, 2>::stream(fmode, grid, st, probs, P);
  }
  static void slot(int sh, int fmode, bool up, int mode, dim3 grid, cudaStream_t st, const kfp::SlotArgs<T>& G) {
    if (sh == 0) kfp::LaunchSet<T, 0>::slot(fmode, up, mode, grid, st, G);
    else if (sh == 1) kfp::LaunchSet<T, 1>::slot(fmode, up, mode, grid, st, G);
    else kfp::LaunchSet<T, 2>::slot(fmode, up, mode, grid, st, G);
  }
  static void fe_slot(int sh, int fmode, bool up, int mode, dim3 grid, cudaStream_t st,
                      const kfp::FeSlotArgs<T>& G) {
    if (sh == 0) kfp::LaunchSet<T, 0>::fe_slot(fmode, up, mode, grid, st, G);
    else if (sh == 1) kfp::LaunchSet<T, 1>::fe_slot(fmode, up, mode, grid, st, G);
    else kfp::LaunchSet<T, 2>::fe_slot(fmode, up, mode, grid, st, G);
  }
  static void edge(int sh, int mode, int fmode, unsigned grid, cudaStream_t st, const kfp::StreamProblem<T>* probs,
                   const kfp::StreamUnit* units, int n) {
    if (sh == 0) kfp::LaunchSet<T, 0>::edge(mode, fmode, grid, st, probs, units, n);
    else if (sh == 1) kfp::LaunchSet<T, 1>::edge(mode, fmode, grid, st, probs, units, n);
    else kfp::LaunchSet<T, 2>::edge(mode, fmode, grid, st, probs, units, n);
  }
};

// Tile shape requested through the descriptor flags (-1: choose automatically).
int requested_shape(unsigned flags) {
  const int f = (int)((flags >> KFP_FLAG_SHAPE_SHIFT) & 3u);
  return f == 0 ? -1 : f - 1;
}

// Iterates per pipelined group requested through the flags (-1: choose automatically).
constexpr int kMaxDepth = 8;
int requested_depth(unsigned flags) {
  const int f = (int)((flags >> KFP_FLAG_DEPTH_SHIFT) & 15u);
  return f == 0 ? -1 : std::min(f, kMaxDepth);
}

// Return a status with the CUDA error text; OBJ is the handle whose message is set.
#define KFP_CUDA_TRY_ON(OBJ, call)                                                        \
  do {                                                                                    \
    cudaError_t e__ = (call);                                                             \
    if (e__ != cudaSuccess) {                                                             \
      cudaGetLastError();                                                                 \
      return (OBJ)->fail(e__ == cudaErrorMemoryAllocation ? KFP_ENOMEM : KFP_ECUDA,       \
                         "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e__),         \
                         __FILE__, __LINE__);                                             \
    }                                                                                     \
  } while (0)
#define KFP_CUDA_TRY(call) KFP_CUDA_TRY_ON(this, call)
#define KFP_CUDA_TRY_H(call) KFP_CUDA_TRY_ON(h, call)

struct Geometry {
  double x0, x1, v0, v1, dt, hx, hv, r;
  int nx, nv, nt, S, ov, robin, P, W, Lmax, rows, nforce;
  int neumann, periodic;  // zero flux in v, periodic in x (Section 6.1)
  int split;              // the Lie splitting with P1 elements of Section 6.2
  std::vector<double> p, q;
  std::vector<kfp::StripInfo> strips;
  std::vector<int> row_of;  // [nv+1] row of UT holding node i at t = T
  long long cells_per_iter;
};

// ---------------------------------------------------------------------------
// Validation and strip layout (Section 2 and Section 6.3, eq. "Om1_Om2", for S strips)
// ---------------------------------------------------------------------------

kfp_status build_geometry(const kfp_swr_desc* d, int nforce, Geometry* g, std::string* err) {
  auto bad = [&](kfp_status c, const char* m) {
    *err = m;
    return c;
  };
  if (!d) return bad(KFP_EINVAL, "desc is NULL");
  if (d->nx < 1 || d->nv < 2 || d->nt < 1 || d->nstrips < 1)
    return bad(KFP_EINVAL, "need nx >= 1, nv >= 2, nt >= 1, nstrips >= 1");
  if (!(d->x1 > d->x0) || !(d->v1 > d->v0) || !(d->dt > 0) || !std::isfinite(d->dt))
    return bad(KFP_EINVAL, "need x1 > x0, v1 > v0, dt > 0");
  if (d->nv % d->nstrips != 0) return bad(KFP_EINVAL, "nstrips must divide nv");
  if (d->tc != KFP_DIRICHLET && d->tc != KFP_ROBIN) return bad(KFP_EINVAL, "unknown transmission");
  if (d->prec != KFP_F64 && d->prec != KFP_F32 && d->prec != KFP_MIXED) return bad(KFP_EINVAL, "unknown precision");
  if (nforce < 0) return bad(KFP_EINVAL, "nforce < 0");
  const int S = d->nstrips;
  const int w = d->nv / S;
  const int ov = S > 1 ? d->overlap_cells : 0;
  if (S > 1 && (w < 2 || ov < 0 || ov >= w))
    return bad(KFP_EINVAL, "need nv/nstrips >= 2 and 0 <= overlap_cells < nv/nstrips");
  g->p.assign(std::max(S - 1, 0), 0.0);
  g->q.assign(std::max(S - 1, 0), 0.0);
  if (S > 1 && d->tc == KFP_ROBIN) {
    if (!d->p) return bad(KFP_EINVAL, "Robin transmission needs p");
    for (int j = 0; j < S - 1; ++j) {
      g->p[j] = d->p[j];
      g->q[j] = d->q ? d->q[j] : d->p[j];
      if (!(g->p[j] > 0) || !(g->q[j] > 0) || !std::isfinite(g->p[j]) || !std::isfinite(g->q[j]))
        return bad(KFP_EINVAL, "Robin parameters must be finite and > 0");
    }
  }
  g->x0 = d->x0; g->x1 = d->x1; g->v0 = d->v0; g->v1 = d->v1; g->dt = d->dt;
  g->nx = d->nx; g->nv = d->nv; g->nt = d->nt; g->S = S; g->ov = ov;
  g->robin = (d->tc == KFP_ROBIN) ? 1 : 0;
  g->nforce = nforce;
  g->neumann = (d->flags & KFP_FLAG_NEUMANN_V) ? 1 : 0;
  g->periodic = (d->flags & KFP_FLAG_PERIODIC_X) ? 1 : 0;
  if (g->periodic && d->nx < 2) return bad(KFP_EINVAL, "periodic x needs nx >= 2");
  g->split = (d->flags & KFP_FLAG_SPLIT_SCHEME) ? 1 : 0;
  if (g->split && !(g->neumann && g->periodic))
    return bad(KFP_EINVAL, "the split scheme is built for the model problem: zero flux in v, periodic x");
  g->hx = (d->x1 - d->x0) / d->nx;
  g->hv = (d->v1 - d->v0) / d->nv;
  g->r = d->dt / (g->hv * g->hv);
  for (int i = 0; i <= d->nv; ++i) {
    const double vi = d->v0 + i * g->hv;
    if (std::fabs(vi) * d->dt / g->hx > 1.0) return bad(KFP_ECFL, "CFL |v| dt / hx > 1");
  }
  auto alpha = [&](int j) { return (j + 1) * w - ov / 2; };
  g->strips.resize(S);
  int rowoff = 0, Lmax = 0;
  long long nodes = 0;
  for (int s = 0; s < S; ++s) {
    kfp::StripInfo& st = g->strips[s];
    std::memset(&st, 0, sizeof st);
    st.lo = s == 0 ? 0 : alpha(s - 1);
    st.hi = s == S - 1 ? d->nv : alpha(s) + ov;
    st.L = st.hi - st.lo + 1;
    st.rowoff = rowoff;
    st.has_bot = s > 0;
    st.has_top = s < S - 1;
    st.alpha_bot = s > 0 ? alpha(s - 1) : 0;
    st.alpha_top = s < S - 1 ? alpha(s) : 0;
    if (s < S - 1) { st.p_top = g->p[s]; st.q_top = g->q[s]; }
    if (s > 0) { st.p_bot = g->p[s - 1]; st.q_bot = g->q[s - 1]; }
    rowoff += st.L;
    Lmax = std::max(Lmax, st.L);
    nodes += st.L;
  }
  g->rows = rowoff;
  g->Lmax = Lmax;
  g->W = (d->nx + 1 + kfp::kOutCols - 1) / kfp::kOutCols;
  g->P = ((kfp::kOutCols * g->W + 2) + 31) / 32 * 32;
  g->cells_per_iter = (long long)(d->nx + 1) * nodes * d->nt;
  g->row_of.resize(d->nv + 1);
  for (int i = 0; i <= d->nv; ++i) {
    int s = 0;
    while (s < S - 1 && i > (s + 1) * w) ++s;  // lower strip owns i <= I_s
    g->row_of[i] = g->strips[s].rowoff + (i - g->strips[s].lo);
  }
  return KFP_OK;
}

// Rows of the split scheme's system (M + dt S) w (Section 6.2, P1 elements in v):
// interior (h/6 - dt/h, 2h/3 + 2dt/h, h/6 - dt/h); an end row (strip end or v0, v1)
// has one element, h/3 + dt/h on the diagonal, plus dt p (top) or dt q (bottom) at a
// Robin interface; a Dirichlet interface row is the identity.
void split_rows(const Geometry& g, const kfp::StripInfo& st, double* a, double* b, double* c) {
  const double h = g.hv, dt = g.dt;
  for (int l = 0; l < st.L; ++l) {
    const bool top = l == st.L - 1, bot = l == 0;
    a[l] = bot ? 0.0 : h / 6 - dt / h;
    c[l] = top ? 0.0 : h / 6 - dt / h;
    b[l] = (top || bot) ? h / 3 + dt / h : 2 * h / 3 + 2 * dt / h;
    if (top && st.has_top) {
      if (g.robin) b[l] += dt * st.p_top;
      else { a[l] = 0.0; b[l] = 1.0; }
    }
    if (bot && st.has_bot) {
      if (g.robin) b[l] += dt * st.q_bot;
      else { c[l] = 0.0; b[l] = 1.0; }
    }
  }
}

// Constant-coefficient LU factors of every strip's implicit-Euler system for the
// three column classes (m = 0, interior, m = nx) and both elimination directions.
// Layout [S][3][2][3][Lmax]: field 0 = 1/pivot, 1 = coupling to the previously
// eliminated row, 2 = back-substitution coefficient.
// transposed: the factors of A^T (sub-diagonal c_{l-1}, super-diagonal a_{l+1}) for
// the fused adjoint pass.
std::vector<double> build_factors(const Geometry& g, bool transposed = false) {
  std::vector<double> coef((size_t)g.S * 3 * 2 * 3 * g.Lmax, 0.0);
  std::vector<double> a(g.Lmax), b(g.Lmax), c(g.Lmax), cp(g.Lmax);
  const double r = g.r;
  for (int s = 0; s < g.S; ++s) {
    const kfp::StripInfo& st = g.strips[s];
    const int L = st.L;
    for (int kappa = 0; kappa < 3; ++kappa) {
      if (g.split) split_rows(g, st, a.data(), b.data(), c.data());
      for (int l = 0; l < L && !g.split; ++l) {
        const int i = st.lo + l;
        const double vi = g.v0 + i * g.hv;
        const bool inflow = !g.periodic && ((kappa == 0 && vi > 0) || (kappa == 2 && vi < 0));
        const bool top = st.has_top && i == st.hi;
        const bool bot = st.has_bot && i == st.lo;
        a[l] = 0.0; b[l] = 1.0; c[l] = 0.0;
        if ((!g.neumann && (i == 0 || i == g.nv)) || inflow) continue;  // identity rows
        if (i == 0) { b[l] = 1 + 2 * r; c[l] = -2 * r; continue; }      // zero-flux half cells
        if (i == g.nv) { a[l] = -2 * r; b[l] = 1 + 2 * r; continue; }
        if (top || bot) {
          if (!g.robin) continue;                               // Dirichlet: identity
          if (top) { a[l] = -2 * r; b[l] = 1 + 2 * r + 2 * st.p_top * g.dt / g.hv; }
          else     { c[l] = -2 * r; b[l] = 1 + 2 * r + 2 * st.q_bot * g.dt / g.hv; }
          continue;
        }
        a[l] = -r; b[l] = 1 + 2 * r; c[l] = -r;
      }
      if (transposed) {
        std::vector<double> at(L), ct(L);
        for (int l = 0; l < L; ++l) {
          at[l] = l > 0 ? c[l - 1] : 0.0;
          ct[l] = l < L - 1 ? a[l + 1] : 0.0;
        }
        for (int l = 0; l < L; ++l) { a[l] = at[l]; c[l] = ct[l]; }
      }
      double* up = &coef[(((size_t)s * 3 + kappa) * 2 + 0) * 3 * g.Lmax];
      double* dn = &coef[(((size_t)s * 3 + kappa) * 2 + 1) * 3 * g.Lmax];
      // ascending elimination: y_l = g_l (R_l - a_l y_{l-1}); back: u_l = y_l - cp_l u_{l+1}
      for (int l = 0; l < L; ++l) {
        const double piv = b[l] - (l > 0 ? a[l] * cp[l - 1] : 0.0);
        const double gi = 1.0 / piv;
        cp[l] = c[l] * gi;
        up[0 * g.Lmax + l] = gi;
        up[1 * g.Lmax + l] = a[l];
        up[2 * g.Lmax + l] = cp[l];
      }
      // descending elimination: y_l = g_l (R_l - c_l y_{l+1}); back: u_l = y_l - cp_l u_{l-1}
      for (int l = L - 1; l >= 0; --l) {
        const double piv = b[l] - (l < L - 1 ? c[l] * cp[l + 1] : 0.0);
        const double gi = 1.0 / piv;
        cp[l] = a[l] * gi;
        dn[0 * g.Lmax + l] = gi;
        dn[1 * g.Lmax + l] = c[l];
        dn[2 * g.Lmax + l] = cp[l];
      }
    }
  }
  return coef;
}

}  // namespace

// ---------------------------------------------------------------------------
// Handle
// ---------------------------------------------------------------------------

struct kfp_swr {
  Geometry g;
  kfp_precision prec = KFP_F64;
  unsigned flags = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  std::string last_error;

  // device memory
  void* Ybuf = nullptr;        // [2][rows][P]: Y0 = first half, Y1 = second half
  void* Y0 = nullptr;
  void* Y1 = nullptr;
  void* GF = nullptr;          // [2][rows][P] pre-scaled forcing per pass direction (FMODE 1)
  void* rec = nullptr;         // [S][2][Lpad][24] coefficient records
  int* flag = nullptr;         // device error flag (bounded waits)
  int use_tma = 0, fmode = 0, Lpad = 0;
  // persistent (streamed) sweep: the interior passes of an iteration in one co-resident
  // launch (one per strip in the serial form)
  int persist = 0, persist_grid = 0, nbx = 0;
  int shape = 0;               // tile shape of the TMA-fed sweep (kfp_launch.h)
  int use_fe_tma = 0;          // split scheme on the TMA-fed pass (kfp_fe_tma.cuh)
  kfp::TmaMaps maps8;          // tensor maps with 8-row boxes (shapes 1 and 2)
  unsigned* done = nullptr;    // [S * nbx] per-unit completion counters, then [S] tickets
  void* sprob = nullptr;       // device StreamProblem<T> of this handle
  kfp::StreamUnit* sunits = nullptr;  // [S * nbx], strip-major
  int* spass = nullptr;        // [nt] first ticket of each interior pass (per group)
  int stall_unit = -1;         // self-test only
  unsigned long long wait_ns = 4000000000ull;
  // pipelined iterates: groups of `depth` consecutive iterates in one streamed launch
  // (kfp_sweep_tma.cuh); iterates 0..depth-2 of a group write the extra buffers below
  // (slot d), the last one the handle's own
  int depth = 1;               // iterates per group (1: every iterate on its own)
  int pipe_shape = 1, pipe_grid = 0, pipe_ready = 0;
  int pipe_slots = 0;          // 1: one launch per slot of the wavefront (periodic x, split
                               // scheme), 0: one streamed launch per group
  double* pipe_zrec = nullptr; // split scheme: [depth-1][2][S][2][2][nx+1] z^k of the slots
  void* pipe_Y = nullptr;      // [depth-1][2][rows][P] T
  void* pipe_UT = nullptr;     // [depth-1][rows][P] T
  double* pipe_lam = nullptr;  // [depth-1][n_trace] interface data passed between iterates
  double* pipe_bands = nullptr;  // [depth-1][n_band]
  std::vector<kfp::TmaMaps> pipe_maps, pipe_maps8;  // [depth-1] maps of the slots' residue buffers
  unsigned* pipe_done = nullptr;   // [depth * S * nbx] completion counters, then the ticket
  kfp::StreamUnit* pipe_units = nullptr;  // [depth * S * nbx], iterate-major, strip-major
  int* pipe_tab = nullptr;     // per group size D = 2..depth: pass_start[nt], unit_first[nt-1]
  void* pipe_prob = nullptr;   // per group size D = 2..depth: StreamProblem<T>[D]
  double* grp_chg = nullptr;   // [kMaxDepth] trace change of each iterate of the last group
  double* grp_host = nullptr;  // pinned [3 * kMaxDepth]
  cudaGraph_t grp_graph[kMaxDepth + 1] = {};
  cudaGraphExec_t grp_exec[kMaxDepth + 1] = {};
  long long stream_launches = 0, stream_cells = 0;  // streamed launches of the groups (profile)
  long long kernel_launches = 0;  // kernels launched by iterations and groups so far
  double t_stream = 0;
  kfp::TmaMaps maps;
  void* UT = nullptr;
  void* U0 = nullptr;
  void* F = nullptr;
  void* coef = nullptr;
  void* cabs = nullptr;
  signed char* sgn = nullptr;
  kfp::StripInfo* strips = nullptr;
  int* row_of = nullptr;
  double* dta = nullptr;
  double* bc_xin = nullptr;
  double* bc_v = nullptr;
  double* lam_in = nullptr;
  double* lam_next = nullptr;
  double* bands = nullptr;
  double* zrec = nullptr;      // split scheme: z^k at the trace rows, [2][S][2][2][nx+1]
  void* fe_tab = nullptr;      // split scheme: [S][2 directions][2][Lmax] g m_off, g a (T)
  double* partial = nullptr;   // 2 doubles per reduction block
  unsigned* tickets = nullptr; // [2]
  double* scal = nullptr;      // [3] e_mis, e_chg, j_l2
  double* hist = nullptr;      // [hist_cap][3]
  int* iter = nullptr;         // device iteration counter (history slot)
  double* stage = nullptr;     // [nv+1][nx+1] solution staging
  double* host_scal = nullptr; // pinned [3]
  int hist_cap = 0;
  int reduce_blocks = 0;

  size_t n_trace = 0, n_band = 0, band_per_side = 0;
  long long iterations = 0;
  std::vector<double> history;  // host copy, 3 per iteration

  cudaGraph_t graph[3] = {nullptr, nullptr, nullptr};
  cudaGraphExec_t graph_exec[3] = {nullptr, nullptr, nullptr};
  // mixed precision: the homogeneous FP32 solver of the corrections, the residual
  // d = G(lam) - lam of the outer (FP64) handle, and the inner handle's view of it
  kfp_swr* inner = nullptr;
  double* d_res = nullptr;
  const double* d_ext = nullptr;
  long long inner_iterations = 0;
  int inner_max = 4000;
  // Tightest relative change an inner solve is asked for.  Its last iterations below
  // the FP32 residual floor of one correction (about 1e-5 |d|) still shrink the
  // slowest error mode, which the next correction would otherwise have to remove.
  double inner_rtol = 1e-7;
  // kept for kfp_swr_set_robin: the constant-in-time forcing (FMODE 1) and its factor
  std::vector<double> Fh_keep;
  double a0_keep = 0.0;
  // adjoint buffers (allocated by the first kfp_swr_gradient)
  double* adj_bands = nullptr;   // [K][S-1][2][nt][nx+1]
  double* adj_lbar = nullptr;    // [adj_DA + 1][S-1][2][nt][nx+1] lambda_bar slots
  double* adj_contrib = nullptr; // [S-1][4][nt][nx+1]
  double* adj_w = nullptr;       // [adj_DA][2][rows][P] elimination residue of the adjoint passes
  double* adj_fac = nullptr;     // [S][3][2][3][Lmax] LU factors of A^T
  double* adj_grad = nullptr;    // [S-1][2]
  int adj_K = 0;
  int adj_DA = 0;                // adjoint iterates in flight the buffers hold
  cudaStream_t cap_stream = nullptr;
  cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  double t_sweep = 0, t_exchange = 0, t_error = 0;

  kfp_status fail(kfp_status c, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    last_error = buf;
    return c;
  }

  size_t elem() const { return prec == KFP_F64 ? sizeof(double) : sizeof(float); }
  int nbx_tma() const { return (g.W + kfp::kWarpsPerBlock - 1) / kfp::kWarpsPerBlock; }  // column blocks per strip
  int launches_per_iter() const {
    if (depth > 1) return (group_launches(depth) + depth - 1) / depth;
    return single_launches(kStandard);
  }
  // kernel launches of one iteration on its own (the exchange and, outside a
  // correction solve, the error reduction only with interfaces)
  int single_launches(int kind) const {
    const int groups = (flags & KFP_FLAG_GAUSS_SEIDEL) ? g.S : 1;
    const int passes = persist ? groups * (g.nt > 1 ? 3 : 2) : (g.nt + 1 + (g.periodic ? g.nt : 0)) * groups;
    return passes + (g.S > 1 ? (kind == 2 ? 1 : 2) : 0);
  }
  // kernel launches of one pipelined group of D iterates: the passes before and after
  // the streamed launch (D (D + 1) / 2 each), the streamed launch, D exchanges and D
  // error reductions (none in a correction solve)
  int group_launches(int D) const {
    return (pipe_slots ? slot_launches(D) : D * (D + 1) + 1) + D + (d_ext ? 0 : D);
  }
  // launches of the passes of a group run one launch per slot: per slot one per pass
  // kind present, and with periodic x one column wrap
  int slot_launches(int D) const {
    int n = 0;
    for (int slot = 0; slot <= g.nt + 2 * (D - 1); ++slot) {
      int has[3] = {0, 0, 0}, wrap = 0;
      for (int d = 0; d < D; ++d) {
        const int k = slot - 2 * d;
        if (k < 0 || k > g.nt) continue;
        has[k == 0 ? 0 : (k == g.nt ? 2 : 1)] = 1;
        if (g.periodic && k < g.nt) wrap = 1;
      }
      n += has[0] + has[1] + has[2] + wrap;
    }
    return n;
  }

  template <typename T>
  kfp::PassArgs<T> pass_args() const {
    kfp::PassArgs<T> A;
    A.nx = g.nx; A.nv = g.nv; A.nt = g.nt; A.S = g.S; A.ov = g.ov; A.P = g.P; A.W = g.W;
    A.Lmax = g.Lmax; A.nforce = g.nforce; A.robin = g.robin;
    A.neumann_v = g.neumann; A.periodic_x = g.periodic;
    A.two_dt_hv = 2.0 * g.dt / g.hv;
    A.inv_2hv = 1.0 / (2.0 * g.hv);
    A.strips = strips;
    A.coef = (const T*)coef;
    A.cabs = (const T*)cabs;
    A.sgn = sgn;
    A.U0 = (const T*)U0;
    A.F = (const T*)F;
    A.dta = dta;
    A.bc_xin = bc_xin;
    A.bc_v = bc_v;
    A.lam_in = lam_in;
    A.lam_bot_src = (flags & KFP_FLAG_GAUSS_SEIDEL) ? lam_next : lam_in;
    A.strip0 = 0;
    A.lam_next = lam_next;
    A.lam_add = nullptr;
    A.bands = bands;
    A.Y0 = (T*)Y0;
    A.Y1 = (T*)Y1;
    A.UT = (T*)UT;
    return A;
  }

  // The split scheme on the TMA-fed pass: one launch per pass, the periodic column
  // wrap after every pass that leaves a residue.
  template <typename T>
  void enqueue_fe_tma(cudaStream_t st) const {
    kfp::TmaArgs<T> X = tma_args<T>();
    const kfp::FeArgs E = fe_args();
    const bool serial = (flags & KFP_FLAG_GAUSS_SEIDEL) != 0;
    const int groups = serial ? g.S : 1;
    const dim3 grid(nbx_tma(), serial ? 1 : g.S);
    const kfp::TmaMaps& mp = shape_maps();
    // the one-iterate slot kernel: the pipelined groups run the same code, so that
    // they give the same bits
    kfp::FeSlotArgs<T> F;
    F.maps[0] = mp;
    F.E[0] = E;
    for (int grp = 0; grp < groups; ++grp) {
      X.p.strip0 = serial ? grp : 0;
      F.X[0] = X;
      for (int k = 0; k <= g.nt; ++k) {
        F.k[0] = k;
        Tma<T>::fe_slot(shape, fmode, !(k & 1), k == 0 ? 0 : (k == g.nt ? 2 : 1), grid, st, F);
        if (k < g.nt) wrap_after_pass<T>(st, k, X.p.strip0, serial ? 1 : g.S);
      }
    }
  }

  template <typename T>
  void enqueue_passes(cudaStream_t st) const {
    if (use_tma) {
      enqueue_passes_tma<T>(st);
      return;
    }
    if (use_fe_tma) {
      enqueue_fe_tma<T>(st);
      return;
    }
    kfp::PassArgs<T> A = pass_args<T>();
    // parallel form: all strips in every launch; serial form: one strip at a time, in
    // increasing order, so that each reads the data the strip below just produced
    const bool serial = (flags & KFP_FLAG_GAUSS_SEIDEL) != 0;
    const int groups = serial ? g.S : 1;
    const dim3 grid((g.W + kfp::kWarpsPerBlock - 1) / kfp::kWarpsPerBlock, serial ? 1 : g.S);
    const dim3 block(kfp::kWarpsPerBlock * 32);
    if (g.split) {
      const kfp::FeArgs E = fe_args();
      for (int grp = 0; grp < groups; ++grp) {
        A.strip0 = serial ? grp : 0;
        kfp::fe_pass_kernel<T, true, 0><<<grid, block, 0, st>>>(A, E, 0);
        wrap_after_pass<T>(st, 0, A.strip0, serial ? 1 : g.S);
        for (int k = 1; k < g.nt; ++k) {
          if (k & 1) kfp::fe_pass_kernel<T, false, 1><<<grid, block, 0, st>>>(A, E, k);
          else       kfp::fe_pass_kernel<T, true, 1><<<grid, block, 0, st>>>(A, E, k);
          wrap_after_pass<T>(st, k, A.strip0, serial ? 1 : g.S);
        }
        if (g.nt & 1) kfp::fe_pass_kernel<T, false, 2><<<grid, block, 0, st>>>(A, E, g.nt);
        else          kfp::fe_pass_kernel<T, true, 2><<<grid, block, 0, st>>>(A, E, g.nt);
      }
      return;
    }
    for (int grp = 0; grp < groups; ++grp) {
      A.strip0 = serial ? grp : 0;
      // pass k runs in ascending row order when k is even (step 1 is factored upward)
      kfp::sweep_pass_kernel<T, true, 0><<<grid, block, 0, st>>>(A, 0);
      wrap_after_pass<T>(st, 0, A.strip0, serial ? 1 : g.S);
      for (int k = 1; k < g.nt; ++k) {
        if (k & 1) kfp::sweep_pass_kernel<T, false, 1><<<grid, block, 0, st>>>(A, k);
        else       kfp::sweep_pass_kernel<T, true, 1><<<grid, block, 0, st>>>(A, k);
        wrap_after_pass<T>(st, k, A.strip0, serial ? 1 : g.S);
      }
      if (g.nt & 1) kfp::sweep_pass_kernel<T, false, 2><<<grid, block, 0, st>>>(A, g.nt);
      else          kfp::sweep_pass_kernel<T, true, 2><<<grid, block, 0, st>>>(A, g.nt);
    }
  }

  // Periodic x: after pass k wrote y^{k+1} of strips [s0, s0 + ns), refresh column nx
  // and the ghost columns of those rows for the halo lanes of pass k+1.
  template <typename T>
  void wrap_after_pass(cudaStream_t st, int k, int s0, int ns) const {
    if (!g.periodic) return;
    T* Yn = (T*)(((k + 1) & 1) ? Y1 : Y0);
    const int r0 = g.strips[s0].rowoff;
    const int r1 = (s0 + ns < g.S) ? g.strips[s0 + ns].rowoff : g.rows;
    kfp::periodic_wrap_kernel<T><<<(r1 - r0 + 255) / 256, 256, 0, st>>>(Yn + (size_t)r0 * g.P, r1 - r0, g.P, g.nx);
  }

  kfp::FeArgs fe_args() const {
    kfp::FeArgs E;
    const double h = g.hv;
    E.m_half = h / 3.0;
    E.m_off = h / 6.0;
    E.k_half = h / 3.0 + g.dt / h;
    E.k_off = h / 6.0 - g.dt / h;
    E.dt = g.dt;
    E.inv_dt = 1.0 / g.dt;
    E.dt_mo = g.dt / E.m_off;
    E.inv_mo = 1.0 / E.m_off;
    E.zrec = zrec;
    E.tab = fe_tab;
    return E;
  }

  // Tensor maps with the box height of this handle's tile shape.
  const kfp::TmaMaps& shape_maps() const { return kfp::shape_rows(shape) == 8 ? maps8 : maps; }

  // The persistent sweep, per group of strips (all strips; one strip at a time in the
  // serial form): the first pass, the nt-1 interior passes in one cooperative launch
  // of the streamed kernel (after the units' counters and tickets are zeroed), the
  // last pass.
  template <typename T>
  void enqueue_persistent(cudaStream_t st, bool interior_only = false) const {
    kfp::TmaArgs<T> X = tma_args<T>();
    const bool serial = (flags & KFP_FLAG_GAUSS_SEIDEL) != 0;
    const int groups = serial ? g.S : 1;
    const dim3 pgrid(nbx_tma(), serial ? 1 : g.S);
    if (g.nt > 1) cudaMemsetAsync(done, 0, sizeof(unsigned) * ((size_t)g.S * nbx + g.S), st);
    for (int grp = 0; grp < groups; ++grp) {
      X.p.strip0 = serial ? grp : 0;
      if (!interior_only) Tma<T>::pass(shape, fmode, true, 0, pgrid, st, shape_maps(), X, 0);
      if (g.nt > 1) enqueue_interior<T>(st, serial ? grp : -1);
      if (interior_only) continue;
      Tma<T>::pass(shape, fmode, !(g.nt & 1), 2, pgrid, st, shape_maps(), X, g.nt);
    }
  }

  // Interior passes of all strips (strip < 0) or of one strip (serial form).
  template <typename T>
  void enqueue_interior(cudaStream_t st, int strip) const {
    const int base = strip < 0 ? 0 : strip * nbx;
    kfp::StreamArgs P;
    P.units = sunits + base;
    P.pass_start = spass;
    P.unit_first = nullptr;
    P.npass = g.nt - 1;
    P.depth = 1;
    P.dynamic = (strip < 0 ? g.S * nbx : nbx) > persist_grid ? 1 : 0;
    P.done = done + base;
    P.ticket = done + (size_t)g.S * nbx + (strip < 0 ? 0 : strip);
    P.flag = flag;
    P.stall_unit = stall_unit;
    P.wait_ns = wait_ns;
    Tma<T>::stream(shape, fmode, (unsigned)persist_grid, st, (const kfp::StreamProblem<T>*)sprob, P);
  }

  template <typename T>
  void enqueue_passes_tma(cudaStream_t st) const {
    if (persist) {
      enqueue_persistent<T>(st);
      return;
    }
    kfp::TmaArgs<T> X = tma_args<T>();
    const bool serial = (flags & KFP_FLAG_GAUSS_SEIDEL) != 0;
    const int groups = serial ? g.S : 1;
    const dim3 grid(nbx_tma(), serial ? 1 : g.S);
    const kfp::TmaMaps& mp = shape_maps();
    for (int grp = 0; grp < groups; ++grp) {
      X.p.strip0 = serial ? grp : 0;
      // pass k runs in ascending row order when k is even (step 1 is factored upward)
      Tma<T>::pass(shape, fmode, true, 0, grid, st, mp, X, 0);
      wrap_after_pass<T>(st, 0, X.p.strip0, serial ? 1 : g.S);
      for (int k = 1; k < g.nt; ++k) {
        Tma<T>::pass(shape, fmode, !(k & 1), 1, grid, st, mp, X, k);
        wrap_after_pass<T>(st, k, X.p.strip0, serial ? 1 : g.S);
      }
      Tma<T>::pass(shape, fmode, !(g.nt & 1), 2, grid, st, mp, X, g.nt);
    }
  }

  // Blocks of the streamed sweep in this handle's shape that fit on the device at
  // once (0 if none).
  template <typename T>
  int persistent_capacity() const {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return Tma<T>::blocks_per_sm(shape, fmode) * sms;
  }

  void record(int idx, cudaStream_t st, bool capturing) const {
    if (!(flags & KFP_FLAG_PROFILE)) return;
    if (capturing) cudaEventRecordWithFlags(ev[idx], st, cudaEventRecordExternal);
    else cudaEventRecord(ev[idx], st);
  }

  // One SWR iteration: the nt+1 sweep passes, then
  //   kStandard: exchange (lam_in <- lam_next, e_chg) and error (e_mis, j_l2);
  //   kResidual: d = lam_next - lam_in (lam_in kept) and error -- the outer FP64 step
  //              of the mixed-precision form;
  //   kInner:    delta <- M delta + d on the homogeneous FP32 problem (no error).
  enum IterKind { kStandard = 0, kResidual = 1, kInner = 2 };

  void enqueue_iteration(cudaStream_t st, bool capturing, int kind) const {
    record(0, st, capturing);
    {
      NvtxRange r("kfp.sweep");
      if (prec == KFP_F64) enqueue_passes<double>(st);
      else enqueue_passes<float>(st);
    }
    record(1, st, capturing);
    if (g.S > 1) {
      NvtxRange r("kfp.exchange");
      if (kind == kStandard)
        kfp::exchange_kernel<<<reduce_blocks, kfp::kReduceThreads, 0, st>>>(
            lam_next, lam_in, lam_in, n_trace, partial, tickets + 0, scal + 1);
      else if (kind == kResidual)
        kfp::residual_kernel<<<reduce_blocks, kfp::kReduceThreads, 0, st>>>(
            lam_next, lam_in, d_res, n_trace, partial, tickets + 0, scal);
      else
        kfp::inner_exchange_kernel<<<reduce_blocks, kfp::kReduceThreads, 0, st>>>(
            lam_next, d_ext, lam_in, n_trace, partial, tickets + 0, scal);
    }
    record(2, st, capturing);
    if (g.S > 1 && kind != kInner) {
      NvtxRange r("kfp.error");
      kfp::error_kernel<<<reduce_blocks, kfp::kReduceThreads, 0, st>>>(
          bands, g.S - 1, band_per_side, g.dt * g.hx, partial + 2 * reduce_blocks, tickets + 1,
          scal + 1, scal, hist, iter, hist_cap, g.periodic ? g.nx + 1 : 0);
    }
    record(3, st, capturing);
  }

  // Exchange + error of one standard iteration (used by the batched form).
  void enqueue_reductions(cudaStream_t st) const {
    if (g.S < 2) return;
    kfp::exchange_kernel<<<reduce_blocks, kfp::kReduceThreads, 0, st>>>(lam_next, lam_in, lam_in, n_trace,
                                                                          partial, tickets + 0, scal + 1);
    kfp::error_kernel<<<reduce_blocks, kfp::kReduceThreads, 0, st>>>(
        bands, g.S - 1, band_per_side, g.dt * g.hx, partial + 2 * reduce_blocks, tickets + 1, scal + 1, scal, hist,
        iter, hist_cap, g.periodic ? g.nx + 1 : 0);
  }

  // ---- pipelined iterates -------------------------------------------------------
  // Iterate d of a group of D reads iter_lam_in(d) and writes iter_lam_next(d, D),
  // which iterate d+1 reads; the last iterate writes the handle's own lam_next, bands,
  // residue and final-state buffers, so that after a full group the handle holds its
  // results exactly as after a lone iteration.
  size_t ystate_bytes() const { return (size_t)g.rows * g.P * elem(); }
  double* iter_lam_in(int d) const { return d == 0 ? lam_in : pipe_lam + (size_t)(d - 1) * n_trace; }
  double* iter_lam_next(int d, int D) const { return d == D - 1 ? lam_next : pipe_lam + (size_t)d * n_trace; }
  double* iter_bands(int d, int D) const { return d == D - 1 ? bands : pipe_bands + (size_t)d * n_band; }
  void* iter_UT(int d, int D) const { return d == D - 1 ? UT : (char*)pipe_UT + (size_t)d * ystate_bytes(); }
  const kfp::TmaMaps& iter_maps(int d, int D, bool rows8) const {
    if (d == D - 1) return rows8 ? maps8 : maps;
    return rows8 ? pipe_maps8[d] : pipe_maps[d];
  }
  template <typename T>
  kfp::TmaArgs<T> iter_args(int d, int D) const {
    kfp::TmaArgs<T> X = tma_args<T>();
    X.p.lam_in = iter_lam_in(d);
    X.p.lam_bot_src = X.p.lam_in;
    X.p.lam_next = iter_lam_next(d, D);
    X.p.lam_add = d_ext;  // a correction solve folds its right-hand side into the new data
    X.p.bands = iter_bands(d, D);
    if (d < D - 1) {
      char* y = (char*)pipe_Y + (size_t)d * 2 * ystate_bytes();
      X.p.Y0 = (T*)y;
      X.p.Y1 = (T*)(y + ystate_bytes());
    }
    X.p.UT = (T*)iter_UT(d, D);
    return X;
  }
  // offsets of group size D's slot tables and problem records
  size_t tab_off(int D) const { return (size_t)(D - 2) * (2 * (size_t)g.nt - 1); }
  int prob_off(int D) const { return (D - 2) * (D + 1) / 2; }
  // cell-updates of the passes a group's streamed launch runs (every iterate runs
  // nt - D of its passes there; a pass advances every node by one step)
  long long stream_cells_of(int D) const { return g.cells_per_iter / g.nt * (long long)D * (g.nt - D); }

  kfp::FeArgs iter_fe(int d, int D) const {
    kfp::FeArgs E = fe_args();
    if (d < D - 1) E.zrec = pipe_zrec + (size_t)d * 2 * g.S * 2 * 2 * (g.nx + 1);
    return E;
  }

  // The same wavefront as enqueue_group_passes with one launch per slot and pass kind
  // (grid.z = the slot's iterates of that kind), for the forms that need a step
  // between passes: periodic x wraps the columns of every residue a slot wrote.
  template <typename T>
  void enqueue_group_slots(cudaStream_t st, int D) const {
    const int nt = g.nt;
    const bool r8 = kfp::shape_rows(pipe_shape) == 8;
    for (int slot = 0; slot <= nt + 2 * (D - 1); ++slot) {
      kfp::WrapGroup<T> wg;
      int nwrap = 0;
      for (int mode = 0; mode < 3; ++mode) {
        kfp::SlotArgs<T> G;
        kfp::FeSlotArgs<T> F;
        int nz = 0;
        for (int d = 0; d < D; ++d) {
          const int k = slot - 2 * d;
          if (k < 0 || k > nt || (k == 0 ? 0 : (k == nt ? 2 : 1)) != mode) continue;
          const kfp::TmaArgs<T> X = iter_args<T>(d, D);
          if (g.split) {
            F.maps[nz] = iter_maps(d, D, r8);
            F.X[nz] = X;
            F.E[nz] = iter_fe(d, D);
            F.k[nz] = k;
          } else {
            G.maps[nz] = iter_maps(d, D, r8);
            G.X[nz] = X;
            G.k[nz] = k;
          }
          ++nz;
          if (g.periodic && k < nt) wg.a[nwrap++] = ((k + 1) & 1) ? X.p.Y1 : X.p.Y0;
        }
        if (nz == 0) continue;
        const dim3 grid(nbx, g.S, nz);
        const bool up = !(slot & 1);  // k = slot - 2d has the parity of the slot
        if (g.split) Tma<T>::fe_slot(pipe_shape, fmode, up, mode, grid, st, F);
        else Tma<T>::slot(pipe_shape, fmode, up, mode, grid, st, G);
      }
      if (nwrap > 0)
        kfp::periodic_wrap_group_kernel<T><<<dim3((g.rows + 255) / 256, nwrap), 256, 0, st>>>(wg, g.rows, g.P, g.nx);
    }
  }

  // The sweeps of D consecutive iterates: pass k of iterate d runs in slot k + 2d, so
  // that iterate d-1 has recorded the interface data at t^k and t^(k+1) (its passes k
  // and k+1) before iterate d reads them.  The passes k <= D-1-d (which include the
  // first passes) run as launches before the streamed launch, the passes k >= nt-d
  // (which include the last passes) after it, each in slot order.
  template <typename T>
  void enqueue_group_passes(cudaStream_t st, bool capturing, int D) const {
    if (pipe_slots) {
      enqueue_group_slots<T>(st, D);
      return;
    }
    const int nt = g.nt, SN = g.S * nbx;
    const dim3 grid(nbx, g.S);
    const bool r8 = kfp::shape_rows(pipe_shape) == 8;
    cudaMemsetAsync(pipe_done, 0, sizeof(unsigned) * ((size_t)D * SN + 1), st);
    for (int slot = 0; slot <= 2 * (D - 1); ++slot)
      for (int d = 0; d < D; ++d) {
        const int k = slot - 2 * d;
        if (k >= 0 && k <= D - 1 - d)
          Tma<T>::pass(pipe_shape, fmode, !(k & 1), k == 0 ? 0 : 1, grid, st, iter_maps(d, D, r8),
                       iter_args<T>(d, D), k);
      }
    kfp::StreamArgs P;
    P.units = pipe_units;
    P.pass_start = pipe_tab + tab_off(D);
    P.unit_first = P.pass_start + nt;
    P.npass = nt - 1;
    P.depth = D;
    P.dynamic = D * SN > pipe_grid ? 1 : 0;
    P.done = pipe_done;
    P.ticket = pipe_done + (size_t)D * SN;
    P.flag = flag;
    P.stall_unit = -1;
    P.wait_ns = wait_ns;
    record(4, st, capturing);
    Tma<T>::stream(pipe_shape, fmode, (unsigned)pipe_grid, st,
                   (const kfp::StreamProblem<T>*)pipe_prob + prob_off(D), P);
    record(5, st, capturing);
    for (int slot = nt; slot <= nt + 2 * (D - 1); ++slot)
      for (int d = 0; d < D; ++d) {
        const int k = slot - 2 * d;
        if (k >= nt - d && k <= nt)
          Tma<T>::pass(pipe_shape, fmode, !(k & 1), k == nt ? 2 : 1, grid, st, iter_maps(d, D, r8),
                       iter_args<T>(d, D), k);
      }
  }

  // One group: the sweeps, then per iterate the trace change (the last iterate's new
  // data become the current ones) and, outside a correction solve, the error.
  void enqueue_group(cudaStream_t st, bool capturing, int D) const {
    record(0, st, capturing);
    {
      NvtxRange r("kfp.sweep");
      if (prec == KFP_F64) enqueue_group_passes<double>(st, capturing, D);
      else enqueue_group_passes<float>(st, capturing, D);
    }
    record(1, st, capturing);
    {
      NvtxRange r("kfp.exchange");
      for (int d = 0; d < D; ++d)
        kfp::exchange_kernel<<<reduce_blocks, kfp::kReduceThreads, 0, st>>>(
            iter_lam_next(d, D), iter_lam_in(d), d == D - 1 ? lam_in : nullptr, n_trace, partial, tickets + 0,
            grp_chg + d);
    }
    record(2, st, capturing);
    if (!d_ext) {
      NvtxRange r("kfp.error");
      for (int d = 0; d < D; ++d)
        kfp::error_kernel<<<reduce_blocks, kfp::kReduceThreads, 0, st>>>(
            iter_bands(d, D), g.S - 1, band_per_side, g.dt * g.hx, partial + 2 * reduce_blocks, tickets + 1,
            grp_chg + d, scal, hist, iter, hist_cap, g.periodic ? g.nx + 1 : 0);
    }
    record(3, st, capturing);
  }

  template <typename T>
  kfp::TmaArgs<T> tma_args() const {
    kfp::TmaArgs<T> X;
    X.p = pass_args<T>();
    X.rows = g.rows;
    X.Lpad = Lpad;
    X.flag = flag;
    X.bc_data = ((bc_xin && !g.periodic) || (bc_v && !g.neumann)) ? 1 : 0;
    return X;
  }

  kfp_status build_graph(int kind) {
    if (graph_exec[kind]) return KFP_OK;
    if (!cap_stream) KFP_CUDA_TRY(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking));
    KFP_CUDA_TRY(cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal));
    enqueue_iteration(cap_stream, true, kind);
    cudaGraph_t gr = nullptr;
    cudaError_t e = cudaStreamEndCapture(cap_stream, &gr);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(KFP_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
    }
    graph[kind] = gr;
    KFP_CUDA_TRY(cudaGraphInstantiate(&graph_exec[kind], graph[kind], 0));
    return KFP_OK;
  }

  void drop_graph() {
    for (int k = 0; k < 3; ++k) {
      if (graph_exec[k]) cudaGraphExecDestroy(graph_exec[k]);
      if (graph[k]) cudaGraphDestroy(graph[k]);
      graph_exec[k] = nullptr;
      graph[k] = nullptr;
    }
    for (int k = 0; k <= kMaxDepth; ++k) {
      if (grp_exec[k]) cudaGraphExecDestroy(grp_exec[k]);
      if (grp_graph[k]) cudaGraphDestroy(grp_graph[k]);
      grp_exec[k] = nullptr;
      grp_graph[k] = nullptr;
    }
  }

  kfp_status ensure_history(int n) {
    if (n <= hist_cap) return KFP_OK;
    int cap = std::max(n, 64);
    double* h = nullptr;
    KFP_CUDA_TRY(cudaStreamSynchronize(stream));
    KFP_CUDA_TRY(cudaMalloc(&h, sizeof(double) * 3 * (size_t)cap));
    if (hist) cudaFree(hist);
    hist = h;
    hist_cap = cap;
    drop_graph();  // the graphs captured the old pointer
    return KFP_OK;
  }

  // Launch one iteration of the given kind (graph replay or direct launches) and,
  // with KFP_FLAG_PROFILE, add its kernel times.
  kfp_status launch_iteration(int kind) {
    NvtxRange r(kind == kInner ? "kfp.iteration.fp32_correction" : "kfp.iteration");
    kernel_launches += single_launches(kind);
    if (!(flags & KFP_FLAG_NO_GRAPH)) {
      kfp_status rc = build_graph(kind);
      if (rc) return rc;
      KFP_CUDA_TRY(cudaGraphLaunch(graph_exec[kind], stream));
    } else {
      enqueue_iteration(stream, false, kind);
      KFP_CUDA_TRY(cudaGetLastError());
    }
    if (flags & KFP_FLAG_PROFILE) {
      KFP_CUDA_TRY(cudaEventSynchronize(ev[3]));
      float a = 0, b = 0, c = 0;
      KFP_CUDA_TRY(cudaEventElapsedTime(&a, ev[0], ev[1]));
      KFP_CUDA_TRY(cudaEventElapsedTime(&b, ev[1], ev[2]));
      KFP_CUDA_TRY(cudaEventElapsedTime(&c, ev[2], ev[3]));
      t_sweep += a; t_exchange += b; t_error += c;
    }
    return KFP_OK;
  }

  // The device records of the groups (unit lists, slot tables, pass arguments of every
  // iterate), written at the first group: a correction solver learns its right-hand
  // side only after create.
  template <typename T>
  kfp_status upload_pipeline() {
    const int SN = g.S * nbx, nt = g.nt;
    std::vector<kfp::StreamUnit> su((size_t)depth * SN);
    for (int d = 0; d < depth; ++d)
      for (int s = 0; s < g.S; ++s)
        for (int bx = 0; bx < nbx; ++bx) {
          kfp::StreamUnit& un = su[(size_t)d * SN + (size_t)s * nbx + bx];
          const int n = d * SN + s * nbx + bx;
          un.inst = d;
          un.strip = s;
          un.bx = bx;
          un.nc = (g.strips[s].L + kfp::kChunkMax - 1) / kfp::kChunkMax;
          un.left = bx > 0 ? n - 1 : -1;
          un.right = bx + 1 < nbx ? n + 1 : -1;
          un.dep_lo = (d > 0 && s > 0) ? n - SN - nbx : -1;
          un.dep_hi = (d > 0 && s + 1 < g.S) ? n - SN + nbx : -1;
        }
    // slot j of a group of D holds the units of iterates max(0, j-(nt-1-D)) ..
    // min(D-1, j), iterate-major
    std::vector<int> tab((size_t)(depth - 1) * (2 * (size_t)nt - 1));
    std::vector<kfp::StreamProblem<T>> sp((size_t)prob_off(depth + 1));
    for (int D = 2; D <= depth; ++D) {
      int* ps = tab.data() + tab_off(D);
      int* uf = ps + nt;
      ps[0] = 0;
      for (int j = 0; j < nt - 1; ++j) {
        const int dlo = std::max(0, j - (nt - 1 - D)), dhi = std::min(D - 1, j);
        uf[j] = dlo * SN;
        ps[j + 1] = ps[j] + (dhi - dlo + 1) * SN;
      }
      for (int d = 0; d < D; ++d) {
        kfp::StreamProblem<T>& p = sp[(size_t)prob_off(D) + d];
        std::memset(&p, 0, sizeof p);
        p.maps = iter_maps(d, D, false);
        p.maps8 = iter_maps(d, D, true);
        p.args = iter_args<T>(d, D);
        p.nt = nt;
        p.fmode = fmode;
        p.lag = d;
      }
    }
    KFP_CUDA_TRY(cudaMemcpy(pipe_units, su.data(), sizeof(kfp::StreamUnit) * su.size(), cudaMemcpyHostToDevice));
    KFP_CUDA_TRY(cudaMemcpy(pipe_tab, tab.data(), sizeof(int) * tab.size(), cudaMemcpyHostToDevice));
    KFP_CUDA_TRY(cudaMemcpy(pipe_prob, sp.data(), sizeof(kfp::StreamProblem<T>) * sp.size(), cudaMemcpyHostToDevice));
    pipe_ready = 1;
    return KFP_OK;
  }

  // Launch one group of D >= 2 iterates (graph replay or direct launches).
  kfp_status launch_group(int D) {
    NvtxRange r(d_ext ? "kfp.group.fp32_correction" : "kfp.group");
    if (!pipe_ready && !pipe_slots) {
      kfp_status rc = prec == KFP_F64 ? upload_pipeline<double>() : upload_pipeline<float>();
      if (rc) return rc;
    }
    if (!(flags & KFP_FLAG_NO_GRAPH)) {
      // the graphs of every group size at once, so that the first group of a sweep
      // builds what its remainder group needs too
      for (int Dg = 2; Dg <= depth; ++Dg) {
        if (grp_exec[Dg]) continue;
        if (!cap_stream) KFP_CUDA_TRY(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking));
        KFP_CUDA_TRY(cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal));
        enqueue_group(cap_stream, true, Dg);
        cudaGraph_t gr = nullptr;
        cudaError_t e = cudaStreamEndCapture(cap_stream, &gr);
        if (e != cudaSuccess) {
          cudaGetLastError();
          return fail(KFP_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
        }
        grp_graph[Dg] = gr;
        KFP_CUDA_TRY(cudaGraphInstantiate(&grp_exec[Dg], gr, 0));
        KFP_CUDA_TRY(cudaGraphUpload(grp_exec[Dg], stream));
      }
      KFP_CUDA_TRY(cudaGraphLaunch(grp_exec[D], stream));
    } else {
      enqueue_group(stream, false, D);
      KFP_CUDA_TRY(cudaGetLastError());
    }
    if (!pipe_slots) {
      stream_launches += 1;
      stream_cells += stream_cells_of(D);
    }
    kernel_launches += group_launches(D);
    if (flags & KFP_FLAG_PROFILE) {
      KFP_CUDA_TRY(cudaEventSynchronize(ev[3]));
      float a = 0, b = 0, c = 0, q = 0;
      KFP_CUDA_TRY(cudaEventElapsedTime(&a, ev[0], ev[1]));
      KFP_CUDA_TRY(cudaEventElapsedTime(&b, ev[1], ev[2]));
      KFP_CUDA_TRY(cudaEventElapsedTime(&c, ev[2], ev[3]));
      if (!pipe_slots) KFP_CUDA_TRY(cudaEventElapsedTime(&q, ev[4], ev[5]));
      t_sweep += a; t_exchange += b; t_error += c; t_stream += q;
    }
    return KFP_OK;
  }

  // Make iterate d of the last group (D iterates) the handle's current one: its new
  // interface data, bands and final state replace those of the group's last iterate.
  kfp_status adopt_iterate(int d, int D) {
    if (d == D - 1) return KFP_OK;
    KFP_CUDA_TRY(cudaMemcpyAsync(lam_in, iter_lam_next(d, D), sizeof(double) * n_trace, cudaMemcpyDeviceToDevice,
                                 stream));
    KFP_CUDA_TRY(cudaMemcpyAsync(lam_next, iter_lam_next(d, D), sizeof(double) * n_trace,
                                 cudaMemcpyDeviceToDevice, stream));
    KFP_CUDA_TRY(cudaMemcpyAsync(bands, iter_bands(d, D), sizeof(double) * n_band, cudaMemcpyDeviceToDevice,
                                 stream));
    KFP_CUDA_TRY(cudaMemcpyAsync(UT, iter_UT(d, D), ystate_bytes(), cudaMemcpyDeviceToDevice, stream));
    return KFP_OK;
  }

  kfp_status read_scalars() {
    KFP_CUDA_TRY(cudaMemcpyAsync(host_scal, scal, sizeof(double) * 3, cudaMemcpyDeviceToHost, stream));
    KFP_CUDA_TRY(cudaStreamSynchronize(stream));
    return KFP_OK;
  }

  kfp_status check_flag() {
    if (!use_tma && !use_fe_tma) return KFP_OK;
    int f = 0;
    KFP_CUDA_TRY(cudaMemcpy(&f, flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (f) return fail(KFP_ETIMEOUT, "a bounded wait in the sweep kernel expired");
    return KFP_OK;
  }

  kfp_status pull_history(int done) {
    if (g.S > 1) {
      std::vector<double> h((size_t)3 * done);
      KFP_CUDA_TRY(cudaMemcpyAsync(h.data(), hist, sizeof(double) * 3 * (size_t)std::min(done, hist_cap),
                                   cudaMemcpyDeviceToHost, stream));
      KFP_CUDA_TRY(cudaStreamSynchronize(stream));
      history.insert(history.end(), h.begin(), h.end());
    } else {
      KFP_CUDA_TRY(cudaStreamSynchronize(stream));
      history.insert(history.end(), (size_t)3 * done, 0.0);
    }
    return KFP_OK;
  }

  kfp_status sweep(int max_iters, double tol, int tol_kind, int* iters_done) {
    if (iters_done) *iters_done = 0;
    if (max_iters < 0 || (tol_kind != 0 && tol_kind != 1))
      return fail(KFP_EINVAL, "need max_iters >= 0 and tol_kind in {0, 1}");
    if (max_iters == 0) return KFP_OK;
    if (inner) return sweep_mixed(max_iters, tol, tol_kind, iters_done);
    kfp_status rc = ensure_history(max_iters);
    if (rc) return rc;
    KFP_CUDA_TRY(cudaMemsetAsync(iter, 0, sizeof(int), stream));
    const bool check = tol > 0;
    int done = 0;
    bool converged = false;
    while (done < max_iters) {
      const int D = std::min(depth, max_iters - done);
      if (D >= 2) {
        // a group of D iterates; with a tolerance, the first iterate that meets it
        // ends the sweep and the later ones are discarded
        rc = launch_group(D);
        if (rc) return rc;
        int stop = -1;
        if (check) {
          KFP_CUDA_TRY(cudaMemcpyAsync(grp_host, hist + 3 * (size_t)done, sizeof(double) * 3 * D,
                                       cudaMemcpyDeviceToHost, stream));
          KFP_CUDA_TRY(cudaStreamSynchronize(stream));
          for (int d = 0; d < D && stop < 0; ++d) {
            const double* r = grp_host + 3 * d;
            if (!std::isfinite(r[0]) || !std::isfinite(r[1]) || !std::isfinite(r[2])) {
              rc = fail(KFP_ENUMERIC, "non-finite interface norm at iteration %lld", iterations + done + d + 1);
              stop = d;
            } else if ((tol_kind == 0 ? r[1] : r[0]) < tol) {
              converged = true;
              stop = d;
            }
          }
        }
        if (stop >= 0) {
          kfp_status ra = adopt_iterate(stop, D);
          if (ra) return ra;
          done += stop + 1;
          break;
        }
        done += D;
        continue;
      }
      rc = launch_iteration(kStandard);
      if (rc) return rc;
      ++done;
      if (check && g.S > 1) {
        rc = read_scalars();
        if (rc) return rc;
        const double v = tol_kind == 0 ? host_scal[1] : host_scal[0];
        if (!std::isfinite(host_scal[0]) || !std::isfinite(host_scal[1]) || !std::isfinite(host_scal[2])) {
          rc = fail(KFP_ENUMERIC, "non-finite interface norm at iteration %lld", iterations + done);
          break;
        }
        if (v < tol) { converged = true; break; }
      }
    }
    kfp_status rh = pull_history(done);
    if (rh) return rh;
    KFP_CUDA_TRY(cudaGetLastError());
    iterations += done;
    if (iters_done) *iters_done = done;
    if (rc) return rc;
    rc = check_flag();
    if (rc) return rc;
    if (g.S > 1) {
      const double* last = &history[history.size() - 3];
      if (!std::isfinite(last[0]) || !std::isfinite(last[1]) || !std::isfinite(last[2]))
        return fail(KFP_ENUMERIC, "non-finite interface norm");
    }
    if (check && g.S > 1 && !converged)
      return fail(KFP_ENOTCONV, "tolerance %g not reached in %d iterations", tol, done);
    return KFP_OK;
  }

  // Mixed precision: defect correction on the interface problem.  Each outer step
  // runs one FP64 iteration from the current interface data lam (its overlap
  // mismatch e_mis and residual d = G(lam) - lam are the reported norms), then
  // solves delta = M delta + d with FP32 iterations of the homogeneous problem
  // (zero data; only the interface data delta drive it) and sets lam += delta in
  // FP64.  The FP32 rounding then sits on the correction, not on lam.  max_iters
  // counts outer (FP64) steps; the inner loop stops when its change falls below
  // eta * |d| -- eta = inner_rtol, or looser when the target tolerance is near --
  // or stops decreasing (FP32 floor), at most inner_max steps.
  kfp_status sweep_mixed(int max_outer, double tol, int tol_kind, int* iters_done) {
    kfp_status rc = ensure_history(max_outer);
    if (rc) return rc;
    KFP_CUDA_TRY(cudaMemsetAsync(iter, 0, sizeof(int), stream));
    KFP_CUDA_TRY(cudaStreamSynchronize(stream));
    int done = 0;
    bool converged = false;
    const int blocks = reduce_blocks;
    for (int outer = 0; outer < max_outer; ++outer) {
      rc = launch_iteration(kResidual);
      if (rc) break;
      ++done;
      rc = read_scalars();
      if (rc) break;
      if (!std::isfinite(host_scal[0]) || !std::isfinite(host_scal[1]) || !std::isfinite(host_scal[2])) {
        rc = fail(KFP_ENUMERIC, "non-finite interface norm at outer step %lld", iterations + done);
        break;
      }
      const double metric = tol_kind == 0 ? host_scal[1] : host_scal[0];
      if (tol > 0 && metric < tol) { converged = true; break; }
      if (outer == max_outer - 1) break;  // the last FP64 step is a measurement
      const double dnorm = host_scal[1];
      if (!(dnorm > 0)) { converged = tol > 0; break; }
      // Solve the correction only as far as the target needs: the remaining error
      // must drop by about tol / metric (with margin), at most to inner_rtol.
      double eta = inner_rtol;
      if (tol > 0) eta = std::min(0.5, std::max(inner_rtol, 0.2 * tol / metric));
      // inner FP32 iterations: delta_0 = d, delta <- M delta + d
      KFP_CUDA_TRY(cudaMemcpyAsync(inner->lam_in, d_res, sizeof(double) * n_trace, cudaMemcpyDeviceToDevice,
                                   stream));
      double best = INFINITY;
      int since_best = 0, j = 0;
      const double* delta = inner->lam_in;  // the correction the loop ends with
      // true when the change chg of an inner iterate ends the loop
      auto ends = [&](double chg) {
        if (chg < eta * dnorm) return true;
        if (chg < 0.5 * best) { best = chg; since_best = 0; }
        else if (++since_best >= 25) return true;  // stalled at FP32 resolution
        return false;
      };
      while (j < inner_max) {
        const int D = std::min(inner->depth, inner_max - j);
        if (D >= 2) {
          // a group of D inner iterates: the first one whose change ends the loop
          // gives the correction
          rc = inner->launch_group(D);
          if (rc) { last_error = inner->last_error; break; }
          KFP_CUDA_TRY(cudaMemcpyAsync(inner->grp_host, inner->grp_chg, sizeof(double) * D, cudaMemcpyDeviceToHost,
                                       stream));
          KFP_CUDA_TRY(cudaStreamSynchronize(stream));
          int stop = -1;
          for (int d = 0; d < D && stop < 0 && !rc; ++d) {
            const double chg = inner->grp_host[d];
            if (!std::isfinite(chg)) rc = fail(KFP_ENUMERIC, "non-finite correction");
            else if (ends(chg)) stop = d;
          }
          if (rc) break;
          if (stop >= 0) {
            j += stop + 1;
            delta = inner->iter_lam_next(stop, D);  // iterate stop's delta (the last one: lam_in)
            if (stop == D - 1) delta = inner->lam_in;
            break;
          }
          j += D;
          continue;
        }
        rc = inner->launch_iteration(kInner);
        if (rc) { last_error = inner->last_error; break; }
        rc = inner->read_scalars();
        if (rc) { last_error = inner->last_error; break; }
        const double chg = inner->host_scal[1];
        ++j;
        if (!std::isfinite(chg)) { rc = fail(KFP_ENUMERIC, "non-finite correction"); break; }
        if (ends(chg)) break;
      }
      if (rc) break;
      inner_iterations += j;
      kfp::correct_kernel<<<blocks, 256, 0, stream>>>(lam_in, delta, n_trace);
      KFP_CUDA_TRY(cudaGetLastError());
    }
    kfp_status rh = pull_history(done);
    if (rh) return rh;
    iterations += done;
    if (iters_done) *iters_done = done;
    if (rc) return rc;
    rc = check_flag();
    if (!rc) rc = inner->check_flag();
    if (rc) return rc;
    if (tol > 0 && !converged)
      return fail(KFP_ENOTCONV, "tolerance %g not reached in %d outer steps", tol, done);
    return KFP_OK;
  }

  void release() {
    if (inner) {
      inner->release();
      delete inner;
      inner = nullptr;
    }
    drop_graph();
    if (cap_stream) cudaStreamDestroy(cap_stream);
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
    void* bufs[] = {Ybuf, GF, rec, flag, done, sprob, sunits, spass, pipe_Y, pipe_UT, pipe_lam, pipe_bands, pipe_zrec,
                    pipe_done,
                    pipe_units, pipe_tab, pipe_prob, grp_chg, UT, U0, F, coef, cabs, sgn, strips, row_of, dta, bc_xin, bc_v,
                    lam_in, lam_next, bands, zrec, fe_tab, partial, tickets, scal, hist, iter, stage, d_res,
                    adj_bands, adj_lbar, adj_contrib, adj_w, adj_fac, adj_grad};
    for (void* b : bufs)
      if (b) cudaFree(b);
    if (host_scal) cudaFreeHost(host_scal);
    if (grp_host) cudaFreeHost(grp_host);
  }
};

namespace {

// Copy a caller FP64 array [rows][nx+1] into a padded device array [rows][P] of T.
kfp_status upload_padded(kfp_swr* h, const double* src, int rows, int on_device, void* dst) {
  const Geometry& g = h->g;
  const size_t n = (size_t)rows * (g.nx + 1);
  double* tmp = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&tmp, sizeof(double) * n, h->stream);
  if (e != cudaSuccess) return h->fail(KFP_ENOMEM, "staging allocation failed");
  e = cudaMemcpyAsync(tmp, src, sizeof(double) * n,
                      on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) {
    const int blocks = (int)std::min<size_t>((n + 255) / 256, 4096);
    if (h->prec == KFP_F64)
      kfp::pad_rows_kernel<double><<<blocks, 256, 0, h->stream>>>(tmp, rows, g.nx, g.P, (double*)dst);
    else
      kfp::pad_rows_kernel<float><<<blocks, 256, 0, h->stream>>>(tmp, rows, g.nx, g.P, (float*)dst);
    e = cudaGetLastError();
  }
  cudaFreeAsync(tmp, h->stream);
  if (e != cudaSuccess) return h->fail(KFP_ECUDA, "upload failed: %s", cudaGetErrorString(e));
  return KFP_OK;
}

// Periodic x: column nx of interface data [.][nx+1] repeats column 0.
kfp_status wrap_traces(kfp_swr* h, double* lam) {
  if (!h->g.periodic || h->n_trace == 0) return KFP_OK;
  const size_t lines = h->n_trace / (h->g.nx + 1);
  kfp::periodic_trace_kernel<<<(int)std::min<size_t>((lines + 255) / 256, 4096), 256, 0, h->stream>>>(lam, lines,
                                                                                                     h->g.nx);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return h->fail(KFP_ECUDA, "periodic trace wrap failed: %s", cudaGetErrorString(e));
  return KFP_OK;
}

kfp_status alloc(kfp_swr* h, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return h->fail(KFP_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
  }
  return KFP_OK;
}

kfp_status copy_in(kfp_swr* h, void* dst, const void* src, size_t bytes, int on_device) {
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  h->stream);
  if (e != cudaSuccess) return h->fail(KFP_ECUDA, "copy failed: %s", cudaGetErrorString(e));
  return KFP_OK;
}


typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// 2D row-major tensor [rows][cols] of T, tile box [box_rows][box_cols].
kfp_status encode_2d(kfp_swr* h, CUtensorMap* map, void* base, size_t rows, size_t cols, int box_rows,
                     int box_cols) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return h->fail(KFP_ECUDA, "cuTensorMapEncodeTiled is not available");
  const size_t es = h->elem();
  cuuint64_t gdim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t gstride[1] = {(cuuint64_t)(cols * es)};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, es == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, gdim,
                  gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return h->fail(KFP_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return KFP_OK;
}

template <typename T>
void put_bits(T* slot, long long v) {
  if (sizeof(T) == 8) std::memcpy(slot, &v, 8);
  else { int x = (int)v; std::memcpy(slot, &x, 4); }
}

// Coefficient records [S][2 pass directions][Lpad][3 classes][8] (field order in kfp_sweep_tma.cuh)
// and, for one constant-in-time forcing term, G = g dt a F per pass direction.
template <typename T>
kfp_status build_records(kfp_swr* h, const std::vector<double>& coef, const std::vector<double>& Fh, double a0,
                         std::vector<T>* rec_out, std::vector<T>* gf_out) {
  const Geometry& g = h->g;
  const int Lpad = h->Lpad, Lm = g.Lmax;
  rec_out->assign((size_t)g.S * 2 * Lpad * kfp::kRecW, T(0));
  const double two_dt_hv = 2.0 * g.dt / g.hv;
  for (int s = 0; s < g.S; ++s) {
    const kfp::StripInfo& st = g.strips[s];
    for (int dir = 0; dir < 2; ++dir) {          // pass direction: 0 ascending, 1 descending
      const int dE = dir, dB = 1 - dir;           // elimination of step k+1 / of step k
      for (int cls = 0; cls < 3; ++cls) {
        const double* cE = &coef[(((size_t)s * 3 + cls) * 2 + dE) * 3 * Lm];
        const double* cB = &coef[(((size_t)s * 3 + cls) * 2 + dB) * 3 * Lm];
        for (int l = 0; l < st.L; ++l) {
          const int i = st.lo + l;
          const double vi = g.v0 + i * g.hv;
          const double cab = std::fabs(vi * g.dt / g.hx);
          const bool inflow = !g.periodic && ((cls == 0 && vi > 0) || (cls == 2 && vi < 0));
          int kind = 0;
          if (!g.neumann && (i == 0 || i == g.nv)) kind = 2;
          else if (inflow) kind = 1;
          else if (st.has_top && i == st.hi) kind = g.robin ? 5 : 3;
          else if (st.has_bot && i == st.lo) kind = g.robin ? 6 : 4;
          const double gE = cE[0 * Lm + l], aE = cE[1 * Lm + l], cpB = cB[2 * Lm + l];
          T* r = &(*rec_out)[(((size_t)s * 2 + dir) * Lpad + kfp::kRecPad + l) * kfp::kRecW + cls * 8];
          const bool ident = kind >= 1 && kind <= 4;
          r[0] = (T)(-cpB);
          r[1] = ident ? T(0) : (T)(gE * (1.0 - cab));
          r[2] = ident ? T(0) : (T)(gE * cab);
          r[3] = ident ? T(0) : (T)(-gE * aE);
          r[4] = ident ? T(0) : (T)gE;
          r[5] = (T)(gE * two_dt_hv);
          put_bits(&r[6], vi > 0 ? 1 : (vi < 0 ? -1 : 0));
          put_bits(&r[7], kind);
        }
      }
    }
  }
  if (gf_out) {
    gf_out->assign((size_t)2 * g.rows * g.P, T(0));
    const size_t nxp = g.nx + 1;
    for (int dir = 0; dir < 2; ++dir)
      for (int s = 0; s < g.S; ++s) {
        const kfp::StripInfo& st = g.strips[s];
        for (int l = 0; l < st.L; ++l) {
          const int i = st.lo + l;
          T* row = &(*gf_out)[((size_t)dir * g.rows + st.rowoff + l) * g.P];
          const double vi = g.v0 + i * g.hv;
          const bool vbnd = !g.neumann && (i == 0 || i == g.nv);
          const bool dir_if = !g.robin && ((st.has_top && i == st.hi) || (st.has_bot && i == st.lo));
          for (int m = 0; m <= g.nx; ++m) {
            const int cls = m == 0 ? 0 : (m == g.nx ? 2 : 1);
            const bool inflow = !g.periodic && ((cls == 0 && vi > 0) || (cls == 2 && vi < 0));
            const double gE = coef[(((size_t)s * 3 + cls) * 2 + dir) * 3 * Lm + l];
            row[m + 1] = (vbnd || inflow || dir_if) ? T(0) : (T)(gE * (g.dt * a0) * Fh[(size_t)i * nxp + m]);
          }
        }
      }
  }
  return KFP_OK;
}

// Forcing mode of the TMA-fed passes: 0 none, 1 one constant-in-time term (pre-scaled;
// its factor a0 and, on the host, F with column nx canonicalised), 2 one
// time-dependent term.
kfp_status forcing_mode(kfp_swr* h, const kfp_swr_problem* pb, double* a0_out, std::vector<double>* Fh_out) {
  const Geometry& g = h->g;
  const size_t nxp = g.nx + 1;
  double a0 = 0.0;
  std::vector<double>& Fh = *Fh_out;
  if (g.nforce == 0) {
    h->fmode = 0;
  } else {
    std::vector<double> ft(g.nt + 1);
    KFP_CUDA_TRY_H(cudaMemcpy(ft.data(), pb->f_time, sizeof(double) * ft.size(),
                              pb->on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost));
    bool constant = true;
    for (int n = 2; n <= g.nt; ++n) constant = constant && (ft[n] == ft[1]);
    h->fmode = constant ? 1 : 2;
    a0 = ft[1];
    if (h->fmode == 1) {
      Fh.resize((size_t)(g.nv + 1) * nxp);
      KFP_CUDA_TRY_H(cudaMemcpy(Fh.data(), pb->f_space, sizeof(double) * Fh.size(),
                                pb->on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost));
      if (g.periodic)  // node nx repeats node 0
        for (int i = 0; i <= g.nv; ++i) Fh[(size_t)i * nxp + g.nx] = Fh[(size_t)i * nxp];
    }
  }
  *a0_out = a0;
  return KFP_OK;
}

// Iterates per pipelined group (parallel form, nt >= 3, interfaces): the flag's value,
// or by default as many as give two blocks per resident slot of the device (streamed)
// or one wave of the grid (one launch per slot: its blocks do not persist, and a
// second, partial wave measured no faster), at most kMaxDepth (kSlotMax) -- none with
// the explicit launch forms KFP_FLAG_PERSISTENT / KFP_FLAG_PER_PASS.
template <typename T>
void choose_depth(kfp_swr* h, int sms, int units_per_pass) {
  const Geometry& g = h->g;
  h->depth = 1;
  h->nbx = h->nbx_tma();
  const int dreq = requested_depth(h->flags);
  if ((h->flags & KFP_FLAG_GAUSS_SEIDEL) || g.S < 2 || g.nt < 3 || dreq == 1) return;
  const int rs = requested_shape(h->flags);
  h->pipe_shape = rs >= 0 ? rs : 1;
  const int pcap = Tma<T>::blocks_per_sm(h->pipe_shape, h->fmode) * sms;
  if (pcap < 1) return;
  const int dmax = h->pipe_slots ? kfp::kSlotMax : kMaxDepth;
  int D = dreq;
  if (D < 0)
    D = (h->flags & (KFP_FLAG_PERSISTENT | KFP_FLAG_PER_PASS))
            ? 1
            : (h->pipe_slots ? 1 : 2) * pcap / std::max(units_per_pass, 1);
  D = std::min(std::min(D, dmax), g.nt - 1);
  if (D >= 2) {
    h->depth = D;
    h->pipe_grid = pcap;
  }
}

template <typename T>
kfp_status setup_tma_t(kfp_swr* h, const kfp_swr_problem* pb) {
  Geometry& g = h->g;
  double a0 = 0.0;
  std::vector<double> Fh;
  kfp_status rc0 = forcing_mode(h, pb, &a0, &Fh);
  if (rc0) return rc0;
  h->Lpad = g.Lmax + 2 * kfp::kRecPad;
  std::vector<double> coef = build_factors(g);
  std::vector<T> rec, gf;
  kfp_status rc = build_records<T>(h, coef, Fh, a0, &rec, h->fmode == 1 ? &gf : nullptr);
  if (rc) return rc;
  h->Fh_keep = Fh;
  h->a0_keep = a0;
  rc = alloc(h, &h->rec, sizeof(T) * rec.size());
  if (rc) return rc;
  KFP_CUDA_TRY_H(cudaMemcpy(h->rec, rec.data(), sizeof(T) * rec.size(), cudaMemcpyHostToDevice));
  if (h->fmode == 1) {
    rc = alloc(h, &h->GF, sizeof(T) * gf.size());
    if (rc) return rc;
    KFP_CUDA_TRY_H(cudaMemcpy(h->GF, gf.data(), sizeof(T) * gf.size(), cudaMemcpyHostToDevice));
  }
  rc = alloc(h, (void**)&h->flag, sizeof(int));
  if (rc) return rc;
  KFP_CUDA_TRY_H(cudaMemset(h->flag, 0, sizeof(int)));
  // tensor maps, with 16-row and 8-row boxes (the rows of a ring stage of each shape)
  for (int box : {16, 8}) {
    kfp::TmaMaps& m = box == 16 ? h->maps : h->maps8;
    rc = encode_2d(h, &m.state, h->Ybuf, (size_t)2 * g.rows, g.P, box, kfp::kBoxW);
    if (!rc) rc = encode_2d(h, &m.init, h->U0, g.nv + 1, g.P, box, kfp::kBoxW);
    if (!rc && h->fmode == 1) rc = encode_2d(h, &m.force, h->GF, (size_t)2 * g.rows, g.P, box, kfp::kBoxW);
    if (!rc && h->fmode == 2) rc = encode_2d(h, &m.force, h->F, g.nv + 1, g.P, box, kfp::kBoxW);
    if (!rc && h->fmode == 0) m.force = m.init;  // never read
    if (!rc) rc = encode_2d(h, &m.rec, h->rec, (size_t)g.S * 2 * h->Lpad, kfp::kRecW, box, kfp::kRecW);
    if (rc) return rc;
  }
  cudaError_t e = Tma<T>::set_attrs();
  if (e != cudaSuccess) return h->fail(KFP_ECUDA, "shared-memory attribute: %s", cudaGetErrorString(e));
  h->use_tma = 1;
  // Tile shape: 16-row stages and one block per SM when a pass has at most one unit
  // per SM, otherwise 8-row stages and two blocks per SM (two consumer warps per
  // sub-partition hide each other's latencies) -- unless the flags fix one.
  // Streamed sweep when forced, or by default when a pass has more units than the
  // device holds blocks at once (then it beats one launch per pass; below that the
  // neighbour wait costs more than the launch it saves).  Periodic x needs its
  // column wrap between passes and keeps one launch per pass.
  KFP_CUDA_TRY_H(cudaGetDevice(&h->device));
  int sms = 0;
  KFP_CUDA_TRY_H(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
  const bool serial = (h->flags & KFP_FLAG_GAUSS_SEIDEL) != 0;
  const int units_per_pass = (serial ? 1 : g.S) * h->nbx_tma();
  h->shape = requested_shape(h->flags);
  if (h->shape < 0) h->shape = units_per_pass > sms ? 1 : 0;
  const int cap = h->persistent_capacity<T>();
  const bool want = (h->flags & KFP_FLAG_PERSISTENT) ||
                    (!(h->flags & KFP_FLAG_PER_PASS) && g.nt > 2 && units_per_pass > cap);
  if (want && !g.periodic) {
    if (cap >= 1) {
      const int nbx = (g.W + kfp::kWarpsPerBlock - 1) / kfp::kWarpsPerBlock;
      h->nbx = nbx;
      const size_t nu = (size_t)g.S * nbx;
      rc = alloc(h, (void**)&h->done, sizeof(unsigned) * (nu + g.S));
      if (!rc) rc = alloc(h, (void**)&h->sunits, sizeof(kfp::StreamUnit) * nu);
      if (!rc) rc = alloc(h, (void**)&h->spass, sizeof(int) * (size_t)std::max(g.nt, 1));
      if (!rc) rc = alloc(h, &h->sprob, sizeof(kfp::StreamProblem<T>));
      if (rc) return rc;
      KFP_CUDA_TRY_H(cudaMemset(h->done, 0, sizeof(unsigned) * (nu + g.S)));
      // units strip-major; neighbour indices relative to the list a launch gets (the
      // whole list, or one strip's part of it in the serial form)
      std::vector<kfp::StreamUnit> su(nu);
      for (int s = 0; s < g.S; ++s)
        for (int bx = 0; bx < nbx; ++bx) {
          kfp::StreamUnit& un = su[(size_t)s * nbx + bx];
          const int rel = serial ? bx : s * nbx + bx;
          un.inst = 0;
          un.strip = s;
          un.bx = bx;
          un.nc = (g.strips[s].L + kfp::kChunkMax - 1) / kfp::kChunkMax;
          un.left = bx > 0 ? rel - 1 : -1;
          un.right = bx + 1 < nbx ? rel + 1 : -1;
          un.dep_lo = un.dep_hi = -1;
        }
      const int per_pass = serial ? nbx : (int)nu;
      std::vector<int> ps((size_t)std::max(g.nt, 1));
      for (size_t j = 0; j < ps.size(); ++j) ps[j] = (int)j * per_pass;
      KFP_CUDA_TRY_H(cudaMemcpy(h->sunits, su.data(), sizeof(kfp::StreamUnit) * nu, cudaMemcpyHostToDevice));
      KFP_CUDA_TRY_H(cudaMemcpy(h->spass, ps.data(), sizeof(int) * ps.size(), cudaMemcpyHostToDevice));
      // h->sprob is written at the end of create, once every buffer it points to exists
      h->persist_grid = cap;
      h->persist = 1;
    }
  }
  // Pipelined iterates: streamed, or one launch per slot with periodic x (its column
  // wrap runs between passes); the buffers are allocated at the end of create
  // (setup_pipeline).
  h->pipe_slots = g.periodic ? 1 : 0;
  choose_depth<T>(h, sms, units_per_pass);
  return KFP_OK;
}

// Buffers of the pipelined iterates: per extra iterate in flight its residue and
// final-state buffers, interface data and bands, and the tensor maps of its residue
// buffers; the counters, unit list, slot tables and problem records of the streamed
// launches.  If the device memory is not there, the handle runs without pipelining.
template <typename T>
kfp_status setup_pipeline(kfp_swr* h) {
  if (h->depth < 2) return KFP_OK;
  const Geometry& g = h->g;
  const int D = h->depth, SN = g.S * h->nbx;
  const size_t ys = h->ystate_bytes();
  const size_t nzr = g.split ? (size_t)2 * g.S * 2 * 2 * (g.nx + 1) : 0;
  kfp_status rc = alloc(h, &h->pipe_Y, (size_t)(D - 1) * 2 * ys);
  if (!rc) rc = alloc(h, &h->pipe_UT, (size_t)(D - 1) * ys);
  if (!rc) rc = alloc(h, (void**)&h->pipe_lam, sizeof(double) * (D - 1) * h->n_trace);
  if (!rc) rc = alloc(h, (void**)&h->pipe_bands, sizeof(double) * (D - 1) * std::max<size_t>(h->n_band, 1));
  if (!rc && nzr) rc = alloc(h, (void**)&h->pipe_zrec, sizeof(double) * (D - 1) * nzr);
  if (!rc && !h->pipe_slots) {  // the streamed launch's counters, units, tables and records
    rc = alloc(h, (void**)&h->pipe_done, sizeof(unsigned) * ((size_t)D * SN + 1));
    if (!rc) rc = alloc(h, (void**)&h->pipe_units, sizeof(kfp::StreamUnit) * (size_t)D * SN);
    if (!rc) rc = alloc(h, (void**)&h->pipe_tab, sizeof(int) * (size_t)(D - 1) * (2 * (size_t)g.nt - 1));
    if (!rc) rc = alloc(h, &h->pipe_prob, sizeof(kfp::StreamProblem<T>) * (size_t)h->prob_off(D + 1));
  }
  if (!rc) rc = alloc(h, (void**)&h->grp_chg, sizeof(double) * kMaxDepth);
  if (rc == KFP_ENOMEM) {
    // run without pipelining
    void* bufs[] = {h->pipe_Y, h->pipe_UT, h->pipe_lam, h->pipe_bands, h->pipe_zrec, h->pipe_done, h->pipe_units,
                    h->pipe_tab, h->pipe_prob, h->grp_chg};
    for (void* b : bufs)
      if (b) cudaFree(b);
    h->pipe_Y = h->pipe_UT = h->pipe_prob = nullptr;
    h->pipe_lam = h->pipe_bands = h->grp_chg = h->pipe_zrec = nullptr;
    h->pipe_done = nullptr;
    h->pipe_units = nullptr;
    h->pipe_tab = nullptr;
    h->depth = 1;
    h->last_error.clear();
    return KFP_OK;
  }
  if (rc) return rc;
  KFP_CUDA_TRY_H(cudaMemsetAsync(h->pipe_Y, 0, (size_t)(D - 1) * 2 * ys, h->stream));
  KFP_CUDA_TRY_H(cudaMemsetAsync(h->pipe_UT, 0, (size_t)(D - 1) * ys, h->stream));
  KFP_CUDA_TRY_H(cudaMemsetAsync(h->pipe_lam, 0, sizeof(double) * (D - 1) * h->n_trace, h->stream));
  KFP_CUDA_TRY_H(cudaMemsetAsync(h->pipe_bands, 0, sizeof(double) * (D - 1) * std::max<size_t>(h->n_band, 1),
                                 h->stream));
  KFP_CUDA_TRY_H(cudaMemsetAsync(h->grp_chg, 0, sizeof(double) * kMaxDepth, h->stream));
  if (nzr) KFP_CUDA_TRY_H(cudaMemsetAsync(h->pipe_zrec, 0, sizeof(double) * (D - 1) * nzr, h->stream));
  KFP_CUDA_TRY_H(cudaMallocHost((void**)&h->grp_host, sizeof(double) * 3 * kMaxDepth));
  h->pipe_maps.assign((size_t)D - 1, h->maps);
  h->pipe_maps8.assign((size_t)D - 1, h->maps8);
  for (int d = 0; d < D - 1; ++d)
    for (int box : {16, 8}) {
      kfp::TmaMaps& m = box == 16 ? h->pipe_maps[d] : h->pipe_maps8[d];
      rc = encode_2d(h, &m.state, (char*)h->pipe_Y + (size_t)d * 2 * ys, (size_t)2 * g.rows, g.P, box, kfp::kBoxW);
      if (rc) return rc;
    }
  return KFP_OK;
}

// The streamed sweep's device copy of this problem's tensor maps and pass arguments.
template <typename T>
kfp_status upload_stream_problem(kfp_swr* h) {
  kfp::StreamProblem<T> sp;
  std::memset(&sp, 0, sizeof sp);
  sp.maps = h->maps;
  sp.maps8 = h->maps8;
  sp.args = h->tma_args<T>();
  sp.nt = h->g.nt;
  sp.fmode = h->fmode;
  KFP_CUDA_TRY_H(cudaMemcpy(h->sprob, &sp, sizeof sp, cudaMemcpyHostToDevice));
  return KFP_OK;
}

kfp_status setup_tma(kfp_swr* h, const kfp_swr_problem* pb) {
  return h->prec == KFP_F64 ? setup_tma_t<double>(h, pb) : setup_tma_t<float>(h, pb);
}

// Split scheme on the TMA-fed pass: the records of the scaled recurrences
// (kfp_fe_tma.cuh), [S][2 pass directions][Lpad][3 classes][8], from the current LU
// factors COEF.  Pass direction d eliminates step k+1 with the factors of direction
// d (G = g m_off, H = g a) and back-substitutes step k, eliminated the other way; the
// previous row in pass order is l-1 going up and l+1 going down.
template <typename T>
void build_fe_records(const kfp_swr* h, const std::vector<double>& coef, std::vector<T>* out) {
  const Geometry& g = h->g;
  const int Lm = g.Lmax, Lpad = h->Lpad;
  const double m_off = g.hv / 6.0;
  out->assign((size_t)g.S * 2 * Lpad * kfp::kRecW, T(0));
  for (int s = 0; s < g.S; ++s) {
    const kfp::StripInfo& st = g.strips[s];
    const int L = st.L;
    for (int d = 0; d < 2; ++d) {
      const double* cE = &coef[(((size_t)s * 3 + 1) * 2 + d) * 3 * Lm];      // g, coupling, cp
      const double* cB = &coef[(((size_t)s * 3 + 1) * 2 + (1 - d)) * 3 * Lm];
      for (int l = 0; l < L; ++l) {
        const bool first = d == 0 ? l == 0 : l == L - 1;
        const int prev = d == 0 ? l - 1 : l + 1;
        const double GB = cB[l] * m_off, GE = cE[l] * m_off;
        const double kappa = first ? 0.0 : cB[2 * Lm + l] * (cB[prev] * m_off) / GB;
        const double rho = first ? 0.0 : (cE[l] * cE[Lm + l]) * (cE[prev] * m_off) / GE;
        const double vi = g.v0 + (st.lo + l) * g.hv;
        const double c = std::fabs(vi * g.dt / g.hx);
        for (int cls = 0; cls < 3; ++cls) {
          T* r = &(*out)[(((size_t)s * 2 + d) * Lpad + kfp::kRecPad + l) * kfp::kRecW + cls * 8];
          r[0] = (T)(-kappa);
          r[1] = (T)(GB * (1.0 - c));
          r[2] = (T)(GB * c);
          r[3] = (T)(-rho);
          r[4] = (T)GB;
          put_bits(&r[6], vi > 0 ? 1 : (vi < 0 ? -1 : 0));
          put_bits(&r[7], 0);
        }
      }
    }
  }
}

// Split scheme on the TMA-fed pass (one forcing term at most): records, the forcing
// pre-scaled by dt a (one constant-in-time term; both pass directions alike), tensor
// maps over the scaled residue, u^0, the forcing and the records, and the tile shape.
template <typename T>
kfp_status setup_fe_tma_t(kfp_swr* h, const kfp_swr_problem* pb) {
  Geometry& g = h->g;
  double a0 = 0.0;
  std::vector<double> Fh;
  kfp_status rc = forcing_mode(h, pb, &a0, &Fh);
  if (rc) return rc;
  h->Lpad = g.Lmax + 2 * kfp::kRecPad;
  h->Fh_keep = Fh;
  h->a0_keep = a0;
  std::vector<T> rec;
  build_fe_records<T>(h, build_factors(g), &rec);
  rc = alloc(h, &h->rec, sizeof(T) * rec.size());
  if (rc) return rc;
  KFP_CUDA_TRY_H(cudaMemcpy(h->rec, rec.data(), sizeof(T) * rec.size(), cudaMemcpyHostToDevice));
  if (h->fmode == 1) {
    const size_t nxp = g.nx + 1;
    std::vector<T> gf((size_t)2 * g.rows * g.P, T(0));
    for (int d = 0; d < 2; ++d)
      for (int s = 0; s < g.S; ++s) {
        const kfp::StripInfo& st = g.strips[s];
        for (int l = 0; l < st.L; ++l) {
          T* row = &gf[((size_t)d * g.rows + st.rowoff + l) * g.P];
          for (int m = 0; m <= g.nx; ++m) row[m + 1] = (T)((g.dt * a0) * Fh[(size_t)(st.lo + l) * nxp + m]);
        }
      }
    rc = alloc(h, &h->GF, sizeof(T) * gf.size());
    if (rc) return rc;
    KFP_CUDA_TRY_H(cudaMemcpy(h->GF, gf.data(), sizeof(T) * gf.size(), cudaMemcpyHostToDevice));
  }
  rc = alloc(h, (void**)&h->flag, sizeof(int));
  if (rc) return rc;
  KFP_CUDA_TRY_H(cudaMemset(h->flag, 0, sizeof(int)));
  for (int box : {16, 8}) {
    kfp::TmaMaps& m = box == 16 ? h->maps : h->maps8;
    rc = encode_2d(h, &m.state, h->Ybuf, (size_t)2 * g.rows, g.P, box, kfp::kBoxW);
    if (!rc) rc = encode_2d(h, &m.init, h->U0, g.nv + 1, g.P, box, kfp::kBoxW);
    if (!rc && h->fmode == 1) rc = encode_2d(h, &m.force, h->GF, (size_t)2 * g.rows, g.P, box, kfp::kBoxW);
    if (!rc && h->fmode == 2) rc = encode_2d(h, &m.force, h->F, g.nv + 1, g.P, box, kfp::kBoxW);
    if (!rc && h->fmode == 0) m.force = m.init;  // never read
    if (!rc) rc = encode_2d(h, &m.rec, h->rec, (size_t)g.S * 2 * h->Lpad, kfp::kRecW, box, kfp::kRecW);
    if (rc) return rc;
  }
  cudaError_t e = Tma<T>::set_attrs();
  if (e != cudaSuccess) return h->fail(KFP_ECUDA, "shared-memory attribute: %s", cudaGetErrorString(e));
  int sms = 0;
  KFP_CUDA_TRY_H(cudaGetDevice(&h->device));
  KFP_CUDA_TRY_H(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
  const bool serial = (h->flags & KFP_FLAG_GAUSS_SEIDEL) != 0;
  const int units_per_pass = (serial ? 1 : g.S) * h->nbx_tma();
  h->shape = requested_shape(h->flags);
  if (h->shape < 0) h->shape = units_per_pass > sms ? 1 : 0;
  h->use_fe_tma = 1;
  // pipelined iterates, one launch per slot (the passes are not streamed)
  h->pipe_slots = 1;
  choose_depth<T>(h, sms, units_per_pass);
  return KFP_OK;
}

// Split scheme: the elimination factors scaled for a right-hand side in units of
// m_off = hv/6, [S][2 directions][2][Lmax]:
//   y_l = (g_l m_off) (M z)_l / m_off - (g_l a_l) y_{l-1}   (periodic x: class 1 only),
// written in the handle's precision.  Built from the current LU factors COEF, so a
// new Robin parameter reaches the elimination as well as the back-substitution.
kfp_status upload_fe_tab(kfp_swr* h, const std::vector<double>& coef) {
  const Geometry& g = h->g;
  std::vector<double> tab((size_t)g.S * 2 * 2 * g.Lmax, 0.0);
  const double m_off = g.hv / 6.0;
  for (int s = 0; s < g.S; ++s)
    for (int d = 0; d < 2; ++d) {
      const double* gf = &coef[((((size_t)s * 3 + 1) * 2 + d) * 3 + 0) * g.Lmax];
      const double* af = &coef[((((size_t)s * 3 + 1) * 2 + d) * 3 + 1) * g.Lmax];
      double* t = &tab[(((size_t)s * 2 + d) * 2) * g.Lmax];
      for (int l = 0; l < g.strips[s].L; ++l) {
        t[l] = gf[l] * m_off;
        t[g.Lmax + l] = gf[l] * af[l];
      }
    }
  if (h->prec == KFP_F64) {
    KFP_CUDA_TRY_H(cudaMemcpy(h->fe_tab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice));
  } else {
    const std::vector<float> t32(tab.begin(), tab.end());
    KFP_CUDA_TRY_H(cudaMemcpy(h->fe_tab, t32.data(), sizeof(float) * t32.size(), cudaMemcpyHostToDevice));
  }
  return KFP_OK;
}

kfp_status create_impl(kfp_swr* h, const kfp_swr_desc* d, const kfp_swr_problem* pb) {
  Geometry& g = h->g;
  const size_t es = h->elem();
  const size_t nxp = g.nx + 1;
  kfp_status rc;
#define TRY(x)            \
  do {                    \
    rc = (x);             \
    if (rc) return rc;    \
  } while (0)
  // state buffers
  const size_t ystate = (size_t)g.rows * g.P * es;
  TRY(alloc(h, &h->Ybuf, 2 * ystate));
  h->Y0 = h->Ybuf;
  h->Y1 = (char*)h->Ybuf + ystate;
  TRY(alloc(h, &h->UT, ystate));
  TRY(alloc(h, &h->U0, (size_t)(g.nv + 1) * g.P * es));
  TRY(alloc(h, &h->F, (size_t)std::max(g.nforce, 1) * (g.nv + 1) * g.P * es));
  KFP_CUDA_TRY_H(cudaMemsetAsync(h->Ybuf, 0, 2 * ystate, h->stream));
  KFP_CUDA_TRY_H(cudaMemsetAsync(h->UT, 0, ystate, h->stream));
  KFP_CUDA_TRY_H(cudaMemsetAsync(h->U0, 0, (size_t)(g.nv + 1) * g.P * es, h->stream));
  KFP_CUDA_TRY_H(cudaMemsetAsync(h->F, 0, (size_t)std::max(g.nforce, 1) * (g.nv + 1) * g.P * es, h->stream));
  TRY(upload_padded(h, pb->u0, g.nv + 1, pb->on_device, h->U0));
  for (int r = 0; r < g.nforce; ++r)
    TRY(upload_padded(h, pb->f_space + (size_t)r * (g.nv + 1) * nxp, g.nv + 1, pb->on_device,
                      (char*)h->F + (size_t)r * (g.nv + 1) * g.P * es));
  if (g.periodic) {  // column nx repeats column 0; ghost columns for the first pass
    const int fr = std::max(g.nforce, 1) * (g.nv + 1);
    if (h->prec == KFP_F64) {
      kfp::periodic_wrap_kernel<double><<<(g.nv + 256) / 256, 256, 0, h->stream>>>((double*)h->U0, g.nv + 1, g.P, g.nx);
      kfp::periodic_wrap_kernel<double><<<(fr + 255) / 256, 256, 0, h->stream>>>((double*)h->F, fr, g.P, g.nx);
    } else {
      kfp::periodic_wrap_kernel<float><<<(g.nv + 256) / 256, 256, 0, h->stream>>>((float*)h->U0, g.nv + 1, g.P, g.nx);
      kfp::periodic_wrap_kernel<float><<<(fr + 255) / 256, 256, 0, h->stream>>>((float*)h->F, fr, g.P, g.nx);
    }
    KFP_CUDA_TRY_H(cudaGetLastError());
  }

  // dt * a_r(t^n), [nt+1][nforce]
  {
    std::vector<double> fa((size_t)std::max(g.nforce, 1) * (g.nt + 1), 0.0);
    if (g.nforce > 0) {
      std::vector<double> ft((size_t)g.nforce * (g.nt + 1));
      if (pb->on_device) {
        if (cudaMemcpy(ft.data(), pb->f_time, sizeof(double) * ft.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
          return h->fail(KFP_ECUDA, "reading f_time failed");
      } else {
        std::memcpy(ft.data(), pb->f_time, sizeof(double) * ft.size());
      }
      for (int n = 0; n <= g.nt; ++n)
        for (int r = 0; r < g.nforce; ++r)
          fa[(size_t)n * g.nforce + r] = g.dt * ft[(size_t)r * (g.nt + 1) + n];
    }
    TRY(alloc(h, (void**)&h->dta, sizeof(double) * fa.size()));
    KFP_CUDA_TRY_H(cudaMemcpy(h->dta, fa.data(), sizeof(double) * fa.size(), cudaMemcpyHostToDevice));
  }

  // per-row tables and factors
  {
    std::vector<double> cabs(g.nv + 1);
    std::vector<signed char> sgn(g.nv + 1);
    for (int i = 0; i <= g.nv; ++i) {
      const double vi = g.v0 + i * g.hv;
      cabs[i] = std::fabs(vi * g.dt / g.hx);
      sgn[i] = vi > 0 ? 1 : (vi < 0 ? -1 : 0);
    }
    std::vector<double> coef = build_factors(g);
    TRY(alloc(h, &h->cabs, (g.nv + 1) * es));
    TRY(alloc(h, &h->coef, coef.size() * es));
    if (h->prec == KFP_F64) {
      KFP_CUDA_TRY_H(cudaMemcpy(h->cabs, cabs.data(), sizeof(double) * cabs.size(), cudaMemcpyHostToDevice));
      KFP_CUDA_TRY_H(cudaMemcpy(h->coef, coef.data(), sizeof(double) * coef.size(), cudaMemcpyHostToDevice));
    } else {
      std::vector<float> c32(cabs.begin(), cabs.end()), f32(coef.begin(), coef.end());
      KFP_CUDA_TRY_H(cudaMemcpy(h->cabs, c32.data(), sizeof(float) * c32.size(), cudaMemcpyHostToDevice));
      KFP_CUDA_TRY_H(cudaMemcpy(h->coef, f32.data(), sizeof(float) * f32.size(), cudaMemcpyHostToDevice));
    }
    TRY(alloc(h, (void**)&h->sgn, sgn.size()));
    KFP_CUDA_TRY_H(cudaMemcpy(h->sgn, sgn.data(), sgn.size(), cudaMemcpyHostToDevice));
    TRY(alloc(h, (void**)&h->strips, sizeof(kfp::StripInfo) * g.S));
    KFP_CUDA_TRY_H(cudaMemcpy(h->strips, g.strips.data(), sizeof(kfp::StripInfo) * g.S, cudaMemcpyHostToDevice));
    TRY(alloc(h, (void**)&h->row_of, sizeof(int) * (g.nv + 1)));
    KFP_CUDA_TRY_H(cudaMemcpy(h->row_of, g.row_of.data(), sizeof(int) * (g.nv + 1), cudaMemcpyHostToDevice));
  }

  // TMA-fed sweep: records, pre-scaled forcing, tensor maps
  if (g.split) {
    const size_t nz = (size_t)2 * g.S * 2 * 2 * nxp;
    TRY(alloc(h, (void**)&h->zrec, sizeof(double) * nz));
    KFP_CUDA_TRY_H(cudaMemsetAsync(h->zrec, 0, sizeof(double) * nz, h->stream));
    TRY(alloc(h, &h->fe_tab, (size_t)g.S * 2 * 2 * g.Lmax * es));
    TRY(upload_fe_tab(h, build_factors(g)));
    if (!(h->flags & KFP_FLAG_GENERIC) && g.nforce <= 1)
      TRY(h->prec == KFP_F64 ? setup_fe_tma_t<double>(h, pb) : setup_fe_tma_t<float>(h, pb));
  } else if (!(h->flags & KFP_FLAG_GENERIC) && g.nforce <= 1) {
    rc = setup_tma(h, pb);
    if (rc) return rc;
  }

  // boundary data
  if (pb->bc_xin) {
    const size_t n = (size_t)(g.nt + 1) * 2 * (g.nv + 1);
    TRY(alloc(h, (void**)&h->bc_xin, sizeof(double) * n));
    TRY(copy_in(h, h->bc_xin, pb->bc_xin, sizeof(double) * n, pb->on_device));
  }
  if (pb->bc_v) {
    const size_t n = (size_t)(g.nt + 1) * 2 * nxp;
    TRY(alloc(h, (void**)&h->bc_v, sizeof(double) * n));
    TRY(copy_in(h, h->bc_v, pb->bc_v, sizeof(double) * n, pb->on_device));
  }

  // interface data, overlaps, reductions
  const int nif = std::max(g.S - 1, 0);
  h->n_trace = (size_t)nif * 2 * g.nt * nxp;
  h->band_per_side = (size_t)g.nt * (g.ov + 1) * nxp;
  h->n_band = (size_t)nif * 2 * h->band_per_side;
  TRY(alloc(h, (void**)&h->lam_in, sizeof(double) * h->n_trace));
  TRY(alloc(h, (void**)&h->lam_next, sizeof(double) * h->n_trace));
  TRY(alloc(h, (void**)&h->bands, sizeof(double) * h->n_band));
  KFP_CUDA_TRY_H(cudaMemsetAsync(h->lam_next, 0, sizeof(double) * h->n_trace, h->stream));
  KFP_CUDA_TRY_H(cudaMemsetAsync(h->bands, 0, sizeof(double) * h->n_band, h->stream));
  if (pb->lambda0) TRY(copy_in(h, h->lam_in, pb->lambda0, sizeof(double) * h->n_trace, pb->on_device));
  else KFP_CUDA_TRY_H(cudaMemsetAsync(h->lam_in, 0, sizeof(double) * h->n_trace, h->stream));
  TRY(wrap_traces(h, h->lam_in));

  int dev = 0, sms = 0;
  KFP_CUDA_TRY_H(cudaGetDevice(&dev));
  KFP_CUDA_TRY_H(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  h->device = dev;
  h->reduce_blocks = std::max(sms, 1) * 4;
  TRY(alloc(h, (void**)&h->partial, sizeof(double) * 4 * h->reduce_blocks));
  TRY(alloc(h, (void**)&h->tickets, sizeof(unsigned) * 2));
  TRY(alloc(h, (void**)&h->scal, sizeof(double) * 3));
  TRY(alloc(h, (void**)&h->iter, sizeof(int)));
  TRY(alloc(h, (void**)&h->stage, sizeof(double) * (g.nv + 1) * nxp));
  KFP_CUDA_TRY_H(cudaMemsetAsync(h->tickets, 0, sizeof(unsigned) * 2, h->stream));
  KFP_CUDA_TRY_H(cudaMemsetAsync(h->scal, 0, sizeof(double) * 3, h->stream));
  KFP_CUDA_TRY_H(cudaMemsetAsync(h->iter, 0, sizeof(int), h->stream));
  KFP_CUDA_TRY_H(cudaMallocHost((void**)&h->host_scal, sizeof(double) * 3));
  if (h->persist) TRY(h->prec == KFP_F64 ? upload_stream_problem<double>(h) : upload_stream_problem<float>(h));
  // (a mixed-precision handle runs single FP64 steps; its correction solver pipelines)
  if (d->prec == KFP_MIXED) h->depth = 1;
  if (h->use_tma || h->use_fe_tma)
    TRY(h->prec == KFP_F64 ? setup_pipeline<double>(h) : setup_pipeline<float>(h));
  for (auto& e : h->ev) KFP_CUDA_TRY_H(cudaEventCreate(&e));
  KFP_CUDA_TRY_H(cudaStreamSynchronize(h->stream));
  KFP_CUDA_TRY_H(cudaGetLastError());
  return KFP_OK;
#undef TRY
}

// Mixed precision: the FP32 solver of the homogeneous problem (zero initial data,
// forcing and boundary data; only its interface data drive it) that computes the
// corrections, sharing the outer handle's stream and reading its residual.
kfp_status create_inner(kfp_swr* h, const kfp_swr_desc* d) {
  const Geometry& g = h->g;
  if (g.S < 2) return KFP_OK;  // one strip: no interface problem, FP64 steps only
  kfp_status rc = alloc(h, (void**)&h->d_res, sizeof(double) * h->n_trace);
  if (rc) return rc;
  KFP_CUDA_TRY_H(cudaMemsetAsync(h->d_res, 0, sizeof(double) * h->n_trace, h->stream));
  double* zeros = nullptr;
  const size_t nu = (size_t)(g.nv + 1) * (g.nx + 1);
  rc = alloc(h, (void**)&zeros, sizeof(double) * nu);
  if (rc) return rc;
  KFP_CUDA_TRY_H(cudaMemsetAsync(zeros, 0, sizeof(double) * nu, h->stream));
  kfp_swr_desc di = *d;
  di.prec = KFP_F32;
  kfp_swr_problem pi;
  std::memset(&pi, 0, sizeof pi);
  pi.on_device = 1;
  pi.u0 = zeros;
  kfp_swr* in = new (std::nothrow) kfp_swr();
  if (!in) {
    cudaFree(zeros);
    return h->fail(KFP_ENOMEM, "host allocation failed");
  }
  std::string err;
  rc = build_geometry(&di, 0, &in->g, &err);
  if (!rc) {
    in->prec = KFP_F32;
    in->flags = d->flags;
    in->stream = h->stream;
    rc = create_impl(in, &di, &pi);
    if (rc) err = in->last_error;
  }
  cudaStreamSynchronize(h->stream);
  cudaFree(zeros);
  if (rc) {
    in->release();
    delete in;
    return h->fail(rc, "inner FP32 solver: %s", err.c_str());
  }
  in->d_ext = h->d_res;
  h->inner = in;
  return KFP_OK;
}

kfp_status gradient_impl(kfp_swr* h, int K, const double* lam0, int lam0_on_device, double* J, double* grad_p,
                         double* grad_q) {
  Geometry& g = h->g;
  if (!g.robin || g.ov != 0 || g.S < 2 || h->prec != KFP_F64 || h->inner || (h->flags & KFP_FLAG_GAUSS_SEIDEL) ||
      g.neumann || g.periodic || g.split)
    return h->fail(KFP_ENOTSUP,
                   "the adjoint needs FP64, Robin transmission, no overlap, >= 2 strips and the parallel form");
  if (K < 1) return h->fail(KFP_EINVAL, "need K >= 1");
  const size_t nxp = g.nx + 1, per = (size_t)g.nt * nxp, ntr = h->n_trace;
  kfp_status rc;
  const size_t ystate = (size_t)g.rows * g.P;
  const size_t nfac = (size_t)g.S * 3 * 2 * 3 * g.Lmax;
  // adjoint iterates in flight at once (pipelined like the forward sweep unless the
  // flags ask for one iterate at a time), in groups of even size: each has its
  // residue buffers, and the lambda_bar data passed between them rotate through DA + 1
  // slots
  const int ngroups = (K + kfp::kAdjGroupMax - 1) / kfp::kAdjGroupMax;
  const int DA = requested_depth(h->flags) == 1 ? 1 : (K + ngroups - 1) / ngroups;
  if (!h->adj_contrib) {
    if ((rc = alloc(h, (void**)&h->adj_contrib, sizeof(double) * (size_t)(g.S - 1) * 4 * per))) return rc;
    if ((rc = alloc(h, (void**)&h->adj_fac, sizeof(double) * nfac))) return rc;
    if ((rc = alloc(h, (void**)&h->adj_grad, sizeof(double) * 2 * (g.S - 1)))) return rc;
  }
  if (DA > h->adj_DA) {
    if (h->adj_lbar) cudaFree(h->adj_lbar);
    if (h->adj_w) cudaFree(h->adj_w);
    h->adj_lbar = nullptr;
    h->adj_w = nullptr;
    h->adj_DA = 0;
    if ((rc = alloc(h, (void**)&h->adj_lbar, sizeof(double) * (DA + 1) * ntr))) return rc;
    if ((rc = alloc(h, (void**)&h->adj_w, sizeof(double) * 2 * (size_t)DA * ystate))) return rc;
    h->adj_DA = DA;
  }
  if (K > h->adj_K) {
    if (h->adj_bands) cudaFree(h->adj_bands);
    h->adj_bands = nullptr;
    if ((rc = alloc(h, (void**)&h->adj_bands, sizeof(double) * (size_t)K * ntr))) return rc;
    h->adj_K = K;
  }
  std::vector<double> fac = build_factors(g, true);
  KFP_CUDA_TRY_H(cudaMemcpy(h->adj_fac, fac.data(), sizeof(double) * fac.size(), cudaMemcpyHostToDevice));
  // forward: K iterations from lambda^0, keeping every iterate's interface-node values
  if (lam0) {
    KFP_CUDA_TRY_H(cudaMemcpyAsync(h->lam_in, lam0, sizeof(double) * ntr,
                                   lam0_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
  } else {
    KFP_CUDA_TRY_H(cudaMemsetAsync(h->lam_in, 0, sizeof(double) * ntr, h->stream));
  }
  if ((rc = h->ensure_history(K))) return rc;
  KFP_CUDA_TRY_H(cudaMemsetAsync(h->iter, 0, sizeof(int), h->stream));
  for (int k = 0; k < K;) {
    const int D = std::min(h->depth, K - k);
    if (D >= 2) {  // a group of pipelined iterates, each leaving its bands in its own buffer
      if ((rc = h->launch_group(D))) return rc;
      for (int d = 0; d < D; ++d)
        KFP_CUDA_TRY_H(cudaMemcpyAsync(h->adj_bands + (size_t)(k + d) * ntr, h->iter_bands(d, D),
                                       sizeof(double) * ntr, cudaMemcpyDeviceToDevice, h->stream));
      k += D;
      continue;
    }
    if ((rc = h->launch_iteration(kfp_swr::kStandard))) return rc;
    KFP_CUDA_TRY_H(cudaMemcpyAsync(h->adj_bands + (size_t)k * ntr, h->bands, sizeof(double) * ntr,
                                   cudaMemcpyDeviceToDevice, h->stream));
    ++k;
  }
  if ((rc = h->pull_history(K))) return rc;
  h->iterations += K;
  if ((rc = h->check_flag())) return rc;
  if (J) *J = h->history[h->history.size() - 1];
  // adjoint, backward over iterates and time levels
  KFP_CUDA_TRY_H(cudaMemsetAsync(h->adj_lbar, 0, sizeof(double) * (DA + 1) * ntr, h->stream));
  KFP_CUDA_TRY_H(cudaMemsetAsync(h->adj_contrib, 0, sizeof(double) * (size_t)(g.S - 1) * 4 * per, h->stream));
  KFP_CUDA_TRY_H(cudaMemsetAsync(h->adj_w, 0, sizeof(double) * 2 * (size_t)DA * ystate, h->stream));
  kfp::AdjPassArgs A;
  A.nx = g.nx; A.nv = g.nv; A.nt = g.nt; A.P = g.P; A.W = g.W; A.Lmax = g.Lmax;
  A.two_dt_hv = 2.0 * g.dt / g.hv;
  A.dthx = g.dt * g.hx;
  A.strips = h->strips;
  A.coef = h->adj_fac;
  A.cabs = (const double*)h->cabs;
  A.sgn = h->sgn;
  A.contrib = h->adj_contrib;
  A.Y0 = h->adj_w;
  A.Y1 = h->adj_w + ystate;
  const dim3 grid((g.W + kfp::kWarpsPerBlock - 1) / kfp::kWarpsPerBlock, g.S);
  const dim3 block(kfp::kWarpsPerBlock * 32);
  // Per iterate, from the last: pass j back-substitutes level nt-j+1 and eliminates
  // level nt-j, in ascending row order when j is even.  Iterates go in groups of up
  // to DA; the group's q-th iterate (k = k_hi - q) runs pass j in slot j + 2q, reads
  // lambda_bar slot (b + q) and writes slot (b + q + 1), modulo DA + 1.
  const int nring = DA + 1;
  int b = 0;
  for (int k_hi = K; k_hi >= 1;) {
    const int G = std::min(DA, k_hi);
    kfp::AdjPassArgs Aq[kfp::kAdjGroupMax];
    for (int q = 0; q < G; ++q) {
      const int k = k_hi - q;
      Aq[q] = A;
      Aq[q].bands = h->adj_bands + (size_t)(k - 1) * ntr;
      Aq[q].lbar_out = h->adj_lbar + (size_t)((b + q) % nring) * ntr;
      Aq[q].lbar_in = h->adj_lbar + (size_t)((b + q + 1) % nring) * ntr;
      Aq[q].Y0 = h->adj_w + (size_t)q * 2 * ystate;
      Aq[q].Y1 = Aq[q].Y0 + ystate;
    }
    for (int slot = 0; slot <= g.nt + 2 * (G - 1); ++slot) {
      // the group's iterates in this slot, by pass kind (first, interior, last)
      for (int mode = 0; mode < 3; ++mode) {
        kfp::AdjGroup grp;
        std::memset(&grp, 0, sizeof grp);
        int nz = 0;
        for (int q = 0; q < G; ++q) {
          const int j = slot - 2 * q;
          if (j < 0 || j > g.nt) continue;
          if ((j == 0 ? 0 : (j == g.nt ? 2 : 1)) != mode) continue;
          grp.A[nz] = Aq[q];
          grp.j[nz] = j;
          grp.last[nz] = (k_hi - q) == K ? 1 : 0;
          ++nz;
        }
        if (nz == 0) continue;
        const dim3 gz(grid.x, grid.y, nz);
        const bool up = !(slot & 1);  // j = slot - 2q has the parity of the slot
        if (mode == 0) kfp::adjoint_group_kernel<true, 0><<<gz, block, 0, h->stream>>>(grp);
        else if (mode == 1 && up) kfp::adjoint_group_kernel<true, 1><<<gz, block, 0, h->stream>>>(grp);
        else if (mode == 1) kfp::adjoint_group_kernel<false, 1><<<gz, block, 0, h->stream>>>(grp);
        else if (up) kfp::adjoint_group_kernel<true, 2><<<gz, block, 0, h->stream>>>(grp);
        else kfp::adjoint_group_kernel<false, 2><<<gz, block, 0, h->stream>>>(grp);
      }
    }
    b = (b + G) % nring;
    k_hi -= G;
  }
  kfp::gradient_reduce_kernel<<<2 * (g.S - 1), kfp::kReduceThreads, 0, h->stream>>>(h->adj_contrib, per,
                                                                                     h->adj_grad);
  KFP_CUDA_TRY_H(cudaGetLastError());
  std::vector<double> gr(2 * (g.S - 1));
  KFP_CUDA_TRY_H(cudaMemcpyAsync(gr.data(), h->adj_grad, sizeof(double) * gr.size(), cudaMemcpyDeviceToHost,
                                 h->stream));
  KFP_CUDA_TRY_H(cudaStreamSynchronize(h->stream));
  for (int j = 0; j < g.S - 1; ++j) {
    if (grad_p) grad_p[j] = gr[2 * j];
    if (grad_q) grad_q[j] = gr[2 * j + 1];
  }
  return KFP_OK;
}

// New Robin parameters: strip table, LU factors, the split scheme's scaled
// elimination factors, coefficient records and the pre-scaled forcing are rebuilt in place (same sizes, so captured graphs stay valid).
template <typename T>
kfp_status refresh_tables(kfp_swr* h) {
  Geometry& g = h->g;
  KFP_CUDA_TRY_H(cudaStreamSynchronize(h->stream));
  KFP_CUDA_TRY_H(cudaMemcpy(h->strips, g.strips.data(), sizeof(kfp::StripInfo) * g.S, cudaMemcpyHostToDevice));
  std::vector<double> coef = build_factors(g);
  if (h->prec == KFP_F64) {
    KFP_CUDA_TRY_H(cudaMemcpy(h->coef, coef.data(), sizeof(double) * coef.size(), cudaMemcpyHostToDevice));
  } else {
    std::vector<float> c32(coef.begin(), coef.end());
    KFP_CUDA_TRY_H(cudaMemcpy(h->coef, c32.data(), sizeof(float) * c32.size(), cudaMemcpyHostToDevice));
  }
  if (g.split) {
    kfp_status rc = upload_fe_tab(h, coef);
    if (rc) return rc;
    if (h->use_fe_tma) {
      std::vector<T> rec;
      build_fe_records<T>(h, coef, &rec);
      KFP_CUDA_TRY_H(cudaMemcpy(h->rec, rec.data(), sizeof(T) * rec.size(), cudaMemcpyHostToDevice));
    }
  }
  if (h->use_tma) {
    std::vector<T> rec, gf;
    kfp_status rc = build_records<T>(h, coef, h->Fh_keep, h->a0_keep, &rec, h->fmode == 1 ? &gf : nullptr);
    if (rc) return rc;
    KFP_CUDA_TRY_H(cudaMemcpy(h->rec, rec.data(), sizeof(T) * rec.size(), cudaMemcpyHostToDevice));
    if (h->fmode == 1)
      KFP_CUDA_TRY_H(cudaMemcpy(h->GF, gf.data(), sizeof(T) * gf.size(), cudaMemcpyHostToDevice));
  }
  return KFP_OK;
}

kfp_status set_robin_impl(kfp_swr* h, const double* p, const double* q) {
  Geometry& g = h->g;
  if (!g.robin || g.S < 2) return h->fail(KFP_EINVAL, "no Robin interfaces");
  if (!p) return h->fail(KFP_EINVAL, "p is NULL");
  for (int j = 0; j < g.S - 1; ++j) {
    const double pj = p[j], qj = q ? q[j] : p[j];
    if (!(pj > 0) || !(qj > 0) || !std::isfinite(pj) || !std::isfinite(qj))
      return h->fail(KFP_EINVAL, "Robin parameters must be finite and > 0");
  }
  for (int j = 0; j < g.S - 1; ++j) {
    g.p[j] = p[j];
    g.q[j] = q ? q[j] : p[j];
  }
  for (int s = 0; s < g.S; ++s) {
    kfp::StripInfo& st = g.strips[s];
    if (s < g.S - 1) { st.p_top = g.p[s]; st.q_top = g.q[s]; }
    if (s > 0) { st.p_bot = g.p[s - 1]; st.q_bot = g.q[s - 1]; }
  }
  kfp_status rc = h->prec == KFP_F64 ? refresh_tables<double>(h) : refresh_tables<float>(h);
  if (rc) return rc;
  if (h->inner) {
    rc = set_robin_impl(h->inner, p, q);
    if (rc) return h->fail(rc, "inner solver: %s", h->inner->last_error.c_str());
  }
  return KFP_OK;
}

kfp_status copy_out(kfp_swr* h, double* dst, const double* src, size_t n, int dst_on_device) {
  cudaError_t e = cudaMemcpyAsync(dst, src, sizeof(double) * n,
                                  dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                  h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return h->fail(KFP_ECUDA, "copy out failed: %s", cudaGetErrorString(e));
  return KFP_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Batched form: independent problems swept together, one launch per time step
// ---------------------------------------------------------------------------

struct kfp_batch {
  std::vector<kfp_swr*> inst;
  kfp_precision prec = KFP_F64;
  cudaStream_t stream = nullptr;
  void* probs_dev = nullptr;             // StreamProblem<T> per problem
  kfp::StreamUnit* units_dev = nullptr;  // all units: grouped by forcing mode, each group in pass order
  int* pass_dev = nullptr;               // per group: first ticket of each interior pass
  unsigned* done = nullptr;              // [units] completion counters, then [3] tickets
  std::vector<kfp::StreamUnit> units;    // host copy, in list order
  int grp_begin[4] = {0, 0, 0, 0};       // forcing mode f: units [grp_begin[f], grp_begin[f+1])
  int grp_npass[3] = {0, 0, 0};          // interior passes of group f (its longest problem's nt - 1)
  int grp_pass_off[3] = {0, 0, 0};       // group f's pass table in pass_dev
  int max_nt = 0, sms = 1, stream_grid = 0;
  int blocks_per_sm = 0;               // first/last passes: 0 = one block per unit; > 0 persistent grid
  int shape = 1;                       // tile shape of the streamed interior passes (kfp_launch.h)
  int unit_order = 0;                  // within a pass: 0 = taller strips first; 1 = problem order
  int* flag = nullptr;                 // error flag of the streamed launches
  long long iterations = 0, cells_per_iter = 0;
  double t_sweep = 0, t_reduce = 0;
  unsigned flags = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  std::string last_error;

  kfp_status fail(kfp_status c, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    last_error = buf;
    return c;
  }


  // List the units: by forcing mode (one streamed launch per mode), then by
  // decreasing nt (the units of interior pass k are then a prefix of the group),
  // then taller strips first or problem order.  Neighbour indices and the pass
  // tables follow from the order.
  void order_units() {
    std::stable_sort(units.begin(), units.end(), [&](const kfp::StreamUnit& a, const kfp::StreamUnit& b) {
      const int fa = inst[a.inst]->fmode, fb = inst[b.inst]->fmode;
      if (fa != fb) return fa < fb;
      const int na = inst[a.inst]->g.nt, nb = inst[b.inst]->g.nt;
      if (na != nb) return na > nb;
      if (unit_order == 0 && a.nc != b.nc) return a.nc > b.nc;
      if (a.inst != b.inst) return a.inst < b.inst;
      if (a.strip != b.strip) return a.strip < b.strip;
      return a.bx < b.bx;
    });
    for (int f = 0; f <= 3; ++f) grp_begin[f] = 0;
    for (const auto& u : units) grp_begin[inst[u.inst]->fmode + 1]++;
    for (int f = 1; f <= 3; ++f) grp_begin[f] += grp_begin[f - 1];
    // neighbour indices, relative to the group's first unit
    std::vector<size_t> first(inst.size() + 1, 0);
    for (size_t i = 0; i < inst.size(); ++i) first[i + 1] = first[i] + (size_t)inst[i]->g.S * inst[i]->nbx_tma();
    std::vector<int> where(first.back(), -1);
    for (size_t n = 0; n < units.size(); ++n) {
      const auto& u = units[n];
      where[first[u.inst] + (size_t)u.strip * inst[u.inst]->nbx_tma() + u.bx] = (int)n;
    }
    for (size_t n = 0; n < units.size(); ++n) {
      auto& u = units[n];
      const int base = grp_begin[inst[u.inst]->fmode], nbx = inst[u.inst]->nbx_tma();
      const size_t row = first[u.inst] + (size_t)u.strip * nbx;
      u.left = u.bx > 0 ? where[row + u.bx - 1] - base : -1;
      u.right = u.bx + 1 < nbx ? where[row + u.bx + 1] - base : -1;
    }
  }

  // Pass tables of the three groups, concatenated: group f's interior pass j holds
  // the units whose problem has nt > j + 1.
  std::vector<int> pass_tables() {
    std::vector<int> all;
    for (int f = 0; f < 3; ++f) {
      int mx = 0;
      for (int n = grp_begin[f]; n < grp_begin[f + 1]; ++n) mx = std::max(mx, inst[units[n].inst]->g.nt);
      grp_npass[f] = std::max(mx - 1, 0);
      grp_pass_off[f] = (int)all.size();
      all.push_back(0);
      for (int j = 0; j < grp_npass[f]; ++j) {
        int active = 0;
        for (int n = grp_begin[f]; n < grp_begin[f + 1]; ++n) active += inst[units[n].inst]->g.nt > j + 1 ? 1 : 0;
        all.push_back(all.back() + active);
      }
    }
    return all;
  }

  // First pass (mode 0) or streamed interior passes (mode 1) of forcing-mode group fm.
  template <typename T>
  void enqueue_group(cudaStream_t st, int fm, int mode) const {
    const auto* probs = (const kfp::StreamProblem<T>*)probs_dev;
    const int n = grp_begin[fm + 1] - grp_begin[fm];
    if (n == 0) return;
    if (mode == 0) {
      const int grid = blocks_per_sm > 0 ? std::min(n, blocks_per_sm * sms) : n;
      Tma<T>::edge(0, 0, fm, (unsigned)grid, st, probs, units_dev + grp_begin[fm], n);
      return;
    }
    if (grp_npass[fm] == 0) return;
    kfp::StreamArgs P;
    P.units = units_dev + grp_begin[fm];
    P.pass_start = pass_dev + grp_pass_off[fm];
    P.unit_first = nullptr;
    P.npass = grp_npass[fm];
    P.depth = 1;
    P.dynamic = n > stream_grid ? 1 : 0;  // the first pass is the largest
    P.done = done + grp_begin[fm];
    P.ticket = done + units.size() + fm;
    P.flag = flag;
    P.stall_unit = -1;
    P.wait_ns = 4000000000ull;
    Tma<T>::stream(shape, fm, (unsigned)stream_grid, st, probs, P);
  }

  // One iteration's passes: the first pass of every unit, the interior passes in one
  // streamed launch per forcing mode, the last pass of every unit.  The first and
  // last passes use 16-row stages; the interior passes the configured shape.
  template <typename T>
  void enqueue_passes(cudaStream_t st) const {
    cudaMemsetAsync(done, 0, sizeof(unsigned) * (units.size() + 3), st);
    for (int fm = 0; fm < 3; ++fm) enqueue_group<T>(st, fm, 0);
    for (int fm = 0; fm < 3; ++fm) enqueue_group<T>(st, fm, 1);
    const int n = (int)units.size();
    const int grid = blocks_per_sm > 0 ? std::min(n, blocks_per_sm * sms) : n;
    Tma<T>::edge(0, 2, 0, (unsigned)grid, st, (const kfp::StreamProblem<T>*)probs_dev, units_dev, n);
  }

  // Blocks of the streamed kernel of the configured shape resident at once.
  template <typename T>
  int stream_capacity() const {
    int per_sm = 0;
    for (int fm = 0; fm < 3; ++fm)
      if (grp_begin[fm + 1] > grp_begin[fm]) {
        const int b = Tma<T>::blocks_per_sm(shape, fm);
        per_sm = per_sm == 0 ? b : std::min(per_sm, b);
      }
    if (per_sm == 0) per_sm = Tma<T>::blocks_per_sm(shape, 1);
    return per_sm * sms;
  }

  void enqueue_iteration(cudaStream_t st, bool capturing) const {
    auto rec = [&](int i) {
      if (!(flags & KFP_FLAG_PROFILE)) return;
      if (capturing) cudaEventRecordWithFlags(ev[i], st, cudaEventRecordExternal);
      else cudaEventRecord(ev[i], st);
    };
    rec(0);
    {
      NvtxRange r("kfp.batch.sweep");
      if (prec == KFP_F64) enqueue_passes<double>(st);
      else enqueue_passes<float>(st);
    }
    rec(1);
    {
      NvtxRange r("kfp.batch.exchange_error");
      for (kfp_swr* h : inst) h->enqueue_reductions(st);
    }
    rec(2);
  }

  void drop_graph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
  }

  kfp_status upload_units() {
    order_units();
    const std::vector<int> tables = pass_tables();
    stream_grid = prec == KFP_F64 ? stream_capacity<double>() : stream_capacity<float>();
    if (stream_grid < 1) return fail(KFP_ECUDA, "the streamed sweep does not fit on an SM in shape %d", shape);
    if (units_dev) cudaFree(units_dev);
    if (pass_dev) cudaFree(pass_dev);
    units_dev = nullptr;
    pass_dev = nullptr;
    KFP_CUDA_TRY(cudaMalloc(&units_dev, sizeof(kfp::StreamUnit) * std::max<size_t>(units.size(), 1)));
    KFP_CUDA_TRY(cudaMemcpy(units_dev, units.data(), sizeof(kfp::StreamUnit) * units.size(), cudaMemcpyHostToDevice));
    KFP_CUDA_TRY(cudaMalloc(&pass_dev, sizeof(int) * tables.size()));
    KFP_CUDA_TRY(cudaMemcpy(pass_dev, tables.data(), sizeof(int) * tables.size(), cudaMemcpyHostToDevice));
    drop_graph();
    return KFP_OK;
  }

  kfp_status sweep(int max_iters, double tol, int tol_kind, int* iters_done) {
    if (iters_done) *iters_done = 0;
    if (max_iters < 0 || (tol_kind != 0 && tol_kind != 1))
      return fail(KFP_EINVAL, "need max_iters >= 0 and tol_kind in {0, 1}");
    if (max_iters == 0) return KFP_OK;
    for (kfp_swr* h : inst) {
      kfp_status rc = h->ensure_history(max_iters);
      if (rc) return fail(rc, "%s", h->last_error.c_str());
      KFP_CUDA_TRY(cudaMemsetAsync(h->iter, 0, sizeof(int), stream));
    }
    if (!(flags & KFP_FLAG_NO_GRAPH) && !exec) {
      if (!cap_stream) KFP_CUDA_TRY(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking));
      KFP_CUDA_TRY(cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal));
      enqueue_iteration(cap_stream, true);
      cudaGraph_t gr = nullptr;
      cudaError_t e = cudaStreamEndCapture(cap_stream, &gr);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(KFP_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
      }
      graph = gr;
      KFP_CUDA_TRY(cudaGraphInstantiate(&exec, graph, 0));
    }
    int done = 0;
    bool converged = false;
    kfp_status rc = KFP_OK;
    for (int it = 0; it < max_iters; ++it) {
      if (exec) {
        KFP_CUDA_TRY(cudaGraphLaunch(exec, stream));
      } else {
        enqueue_iteration(stream, false);
        KFP_CUDA_TRY(cudaGetLastError());
      }
      ++done;
      if (flags & KFP_FLAG_PROFILE) {
        KFP_CUDA_TRY(cudaEventSynchronize(ev[2]));
        float a = 0, b = 0;
        KFP_CUDA_TRY(cudaEventElapsedTime(&a, ev[0], ev[1]));
        KFP_CUDA_TRY(cudaEventElapsedTime(&b, ev[1], ev[2]));
        t_sweep += a;
        t_reduce += b;
      }
      if (tol > 0) {
        double worst = 0.0;
        for (kfp_swr* h : inst) {
          if (h->g.S < 2) continue;
          rc = h->read_scalars();
          if (rc) return fail(rc, "%s", h->last_error.c_str());
          const double v = tol_kind == 0 ? h->host_scal[1] : h->host_scal[0];
          if (!std::isfinite(v)) { rc = fail(KFP_ENUMERIC, "non-finite interface norm"); break; }
          worst = std::max(worst, v);
        }
        if (rc) break;
        if (worst < tol) { converged = true; break; }
      }
    }
    for (kfp_swr* h : inst) {
      kfp_status r2 = h->pull_history(done);
      if (r2) return fail(r2, "%s", h->last_error.c_str());
      h->iterations += done;
      r2 = h->check_flag();
      if (r2) return fail(r2, "%s", h->last_error.c_str());
    }
    int f = 0;
    KFP_CUDA_TRY(cudaMemcpy(&f, flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (f) return fail(KFP_ETIMEOUT, "a bounded wait in the streamed sweep expired");
    iterations += done;
    if (iters_done) *iters_done = done;
    if (rc) return rc;
    if (tol > 0 && !converged) return fail(KFP_ENOTCONV, "tolerance %g not reached in %d iterations", tol, done);
    return KFP_OK;
  }

  void release() {
    drop_graph();
    if (cap_stream) cudaStreamDestroy(cap_stream);
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
    if (probs_dev) cudaFree(probs_dev);
    if (units_dev) cudaFree(units_dev);
    if (pass_dev) cudaFree(pass_dev);
    if (done) cudaFree(done);
    if (flag) cudaFree(flag);
    for (kfp_swr* h : inst) {
      if (!h) continue;
      cudaStreamSynchronize(h->stream);
      h->release();
      delete h;
    }
    inst.clear();
  }
};

namespace {

template <typename T>
kfp_status batch_setup(kfp_batch* b) {
  std::vector<kfp::StreamProblem<T>> host(b->inst.size());
  b->units.clear();
  b->max_nt = 0;
  b->cells_per_iter = 0;
  for (size_t i = 0; i < b->inst.size(); ++i) {
    kfp_swr* h = b->inst[i];
    std::memset(&host[i], 0, sizeof host[i]);
    host[i].maps = h->maps;
    host[i].maps8 = h->maps8;
    host[i].args = h->tma_args<T>();
    host[i].nt = h->g.nt;
    host[i].fmode = h->fmode;
    b->max_nt = std::max(b->max_nt, h->g.nt);
    b->cells_per_iter += h->g.cells_per_iter;
    const int nbx = h->nbx_tma();
    for (int s = 0; s < h->g.S; ++s)
      for (int bx = 0; bx < nbx; ++bx)
        b->units.push_back({(int)i, s, bx, (h->g.strips[s].L + kfp::kChunkMax - 1) / kfp::kChunkMax, -1, -1, -1, -1});
  }
  KFP_CUDA_TRY_ON(b, cudaMalloc(&b->probs_dev, sizeof(kfp::StreamProblem<T>) * host.size()));
  KFP_CUDA_TRY_ON(b, cudaMemcpy(b->probs_dev, host.data(), sizeof(kfp::StreamProblem<T>) * host.size(),
                          cudaMemcpyHostToDevice));
  KFP_CUDA_TRY_ON(b, cudaMalloc(&b->done, sizeof(unsigned) * (b->units.size() + 3)));
  KFP_CUDA_TRY_ON(b, cudaMalloc(&b->flag, sizeof(int)));
  KFP_CUDA_TRY_ON(b, cudaMemset(b->flag, 0, sizeof(int)));
  KFP_CUDA_TRY_ON(b, Tma<T>::set_attrs());
  b->stream_grid = 0;
  return b->upload_units();
}

thread_local std::string g_batch_create_error;

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" {

kfp_status kfp_swr_create(const kfp_swr_desc* desc, const kfp_swr_problem* prob, void* cuda_stream,
                          kfp_swr_t* out) {
  g_create_error.clear();
  if (!out) {
    g_create_error = "out is NULL";
    return KFP_EINVAL;
  }
  *out = nullptr;
  if (!desc || !prob || !prob->u0) {
    g_create_error = "desc, prob and prob->u0 are required";
    return KFP_EINVAL;
  }
  if (prob->nforce > 0 && (!prob->f_time || !prob->f_space)) {
    g_create_error = "nforce > 0 needs f_time and f_space";
    return KFP_EINVAL;
  }
  kfp_swr* h = new (std::nothrow) kfp_swr();
  if (!h) {
    g_create_error = "host allocation failed";
    return KFP_ENOMEM;
  }
  std::string err;
  kfp_status rc = build_geometry(desc, prob->nforce, &h->g, &err);
  if (rc) {
    g_create_error = err;
    delete h;
    return rc;
  }
  h->prec = desc->prec == KFP_MIXED ? KFP_F64 : desc->prec;
  h->flags = desc->flags;
  h->stream = (cudaStream_t)cuda_stream;
  rc = create_impl(h, desc, prob);
  if (!rc && desc->prec == KFP_MIXED) rc = create_inner(h, desc);
  if (rc) {
    g_create_error = h->last_error;
    cudaStreamSynchronize(h->stream);
    h->release();
    delete h;
    return rc;
  }
  *out = h;
  return KFP_OK;
}

kfp_status kfp_swr_sweep(kfp_swr_t h, int max_iters, double tol, int tol_kind, int* iters_done) {
  if (!h) return KFP_EINVAL;
  h->last_error.clear();
  return h->sweep(max_iters, tol, tol_kind, iters_done);
}

kfp_status kfp_swr_traces(kfp_swr_t h, int iface, int side, double* dst, int dst_on_device) {
  if (!h) return KFP_EINVAL;
  if (!dst || iface < 0 || iface >= h->g.S - 1 || side < 0 || side > 1)
    return h->fail(KFP_EINVAL, "need 0 <= iface < nstrips-1, side in {0,1}, dst != NULL");
  const size_t n = (size_t)h->g.nt * (h->g.nx + 1);
  return copy_out(h, dst, h->lam_in + ((size_t)iface * 2 + side) * n, n, dst_on_device);
}

kfp_status kfp_swr_set_traces(kfp_swr_t h, const double* src, int src_on_device) {
  if (!h) return KFP_EINVAL;
  if (!src) return h->fail(KFP_EINVAL, "src is NULL");
  if (h->n_trace == 0) return KFP_OK;
  kfp_status rc = copy_in(h, h->lam_in, src, sizeof(double) * h->n_trace, src_on_device);
  if (!rc) rc = wrap_traces(h, h->lam_in);
  if (rc) return rc;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return h->fail(KFP_ECUDA, "sync failed");
  return KFP_OK;
}

kfp_status kfp_swr_error(kfp_swr_t h, double* e_mis, double* e_chg, double* j_l2, double* history,
                         int hist_cap) {
  if (!h) return KFP_EINVAL;
  if (h->iterations == 0) return h->fail(KFP_EINVAL, "no iteration has run");
  const double* last = &h->history[h->history.size() - 3];
  if (e_mis) *e_mis = last[0];
  if (e_chg) *e_chg = last[1];
  if (j_l2) *j_l2 = last[2];
  if (history && hist_cap > 0) {
    const size_t rows = std::min<size_t>((size_t)hist_cap, h->history.size() / 3);
    std::memcpy(history, h->history.data(), sizeof(double) * 3 * rows);
  }
  return KFP_OK;
}

kfp_status kfp_swr_bands(kfp_swr_t h, int iface, int side, double* dst, int dst_on_device) {
  if (!h) return KFP_EINVAL;
  if (!dst || iface < 0 || iface >= h->g.S - 1 || side < 0 || side > 1)
    return h->fail(KFP_EINVAL, "need 0 <= iface < nstrips-1, side in {0,1}, dst != NULL");
  return copy_out(h, dst, h->bands + ((size_t)iface * 2 + side) * h->band_per_side,
                  h->band_per_side, dst_on_device);
}

kfp_status kfp_swr_solution(kfp_swr_t h, double* dst, int dst_on_device) {
  if (!h) return KFP_EINVAL;
  if (!dst) return h->fail(KFP_EINVAL, "dst is NULL");
  if (h->iterations == 0) return h->fail(KFP_EINVAL, "no iteration has run");
  const Geometry& g = h->g;
  const size_t n = (size_t)(g.nv + 1) * (g.nx + 1);
  const int blocks = (int)std::min<size_t>((n + 255) / 256, 4096);
  if (h->prec == KFP_F64)
    kfp::gather_solution_kernel<double><<<blocks, 256, 0, h->stream>>>((const double*)h->UT, h->row_of,
                                                                      g.nv, g.nx, g.P, h->stage);
  else
    kfp::gather_solution_kernel<float><<<blocks, 256, 0, h->stream>>>((const float*)h->UT, h->row_of,
                                                                     g.nv, g.nx, g.P, h->stage);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return h->fail(KFP_ECUDA, "gather failed: %s", cudaGetErrorString(e));
  return copy_out(h, dst, h->stage, n, dst_on_device);
}

kfp_status kfp_swr_stats(kfp_swr_t h, long long* iterations, long long* cell_updates_per_iter,
                         int* launches_per_iter, double* sweep_ms, double* exchange_ms,
                         double* error_ms) {
  if (!h) return KFP_EINVAL;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return h->fail(KFP_ECUDA, "sync failed");
  if (iterations) *iterations = h->iterations;
  if (cell_updates_per_iter) *cell_updates_per_iter = h->g.cells_per_iter;
  if (launches_per_iter) *launches_per_iter = h->g.S > 1 ? h->launches_per_iter() : h->g.nt + 1;
  if (sweep_ms) *sweep_ms = h->t_sweep;
  if (exchange_ms) *exchange_ms = h->t_exchange;
  if (error_ms) *error_ms = h->t_error;
  return KFP_OK;
}

kfp_status kfp_swr_pipeline_stats(kfp_swr_t h, int* depth, long long* kernel_launches, long long* stream_launches,
                                  long long* stream_cell_updates, double* stream_ms) {
  if (!h) return KFP_EINVAL;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return h->fail(KFP_ECUDA, "sync failed");
  if (depth) *depth = h->depth;
  if (kernel_launches) *kernel_launches = h->kernel_launches + (h->inner ? h->inner->kernel_launches : 0);
  if (stream_launches) *stream_launches = h->stream_launches;
  if (stream_cell_updates) *stream_cell_updates = h->stream_cells;
  if (stream_ms) *stream_ms = h->t_stream;
  return KFP_OK;
}

kfp_status kfp_swr_gradient(kfp_swr_t h, int K, const double* lam0, int lam0_on_device, double* J, double* grad_p,
                            double* grad_q) {
  if (!h) return KFP_EINVAL;
  h->last_error.clear();
  return gradient_impl(h, K, lam0, lam0_on_device, J, grad_p, grad_q);
}

kfp_status kfp_swr_set_robin(kfp_swr_t h, const double* p, const double* q) {
  if (!h) return KFP_EINVAL;
  h->last_error.clear();
  return set_robin_impl(h, p, q);
}

kfp_status kfp_swr_counters(kfp_swr_t h, long long* fp64_iterations, long long* fp32_iterations,
                            double* fp32_sweep_ms) {
  if (!h) return KFP_EINVAL;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return h->fail(KFP_ECUDA, "sync failed");
  const bool f64 = h->prec == KFP_F64;
  if (fp64_iterations) *fp64_iterations = f64 ? h->iterations : 0;
  if (fp32_iterations) *fp32_iterations = f64 ? h->inner_iterations : h->iterations;
  if (fp32_sweep_ms) *fp32_sweep_ms = h->inner ? h->inner->t_sweep : (f64 ? 0.0 : h->t_sweep);
  return KFP_OK;
}

void kfp_swr_destroy(kfp_swr_t h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  h->release();
  delete h;
}

const char* kfp_swr_last_error(kfp_swr_t h) { return h ? h->last_error.c_str() : ""; }

kfp_status kfp_batch_create(const kfp_swr_desc* descs, const kfp_swr_problem* probs, int count, void* cuda_stream,
                            kfp_batch_t* out) {
  g_batch_create_error.clear();
  if (!out) return KFP_EINVAL;
  *out = nullptr;
  if (!descs || !probs || count < 1) {
    g_batch_create_error = "need descs, probs and count >= 1";
    return KFP_EINVAL;
  }
  kfp_batch* b = new (std::nothrow) kfp_batch();
  if (!b) return KFP_ENOMEM;
  b->stream = (cudaStream_t)cuda_stream;
  b->prec = descs[0].prec;
  b->flags = descs[0].flags;
  kfp_status rc = KFP_OK;
  if (b->prec != KFP_F64 && b->prec != KFP_F32) {
    g_batch_create_error = "a batch runs in KFP_F64 or KFP_F32";
    rc = KFP_ENOTSUP;
  }
  for (int i = 0; i < count && !rc; ++i) {
    if (descs[i].prec != b->prec) {
      g_batch_create_error = "all problems of a batch need the same precision";
      rc = KFP_EINVAL;
      break;
    }
    if (descs[i].flags & KFP_FLAG_GAUSS_SEIDEL) {
      g_batch_create_error = "the batched sweep runs the parallel form only";
      rc = KFP_ENOTSUP;
      break;
    }
    if (descs[i].flags & (KFP_FLAG_NEUMANN_V | KFP_FLAG_PERIODIC_X | KFP_FLAG_SPLIT_SCHEME)) {
      g_batch_create_error = "the batched sweep takes Dirichlet data in x and v only";
      rc = KFP_ENOTSUP;
      break;
    }
    kfp_swr_desc d = descs[i];
    d.flags &= ~(unsigned)(KFP_FLAG_GENERIC | KFP_FLAG_PROFILE | KFP_FLAG_DEPTH(15));
    d.flags |= KFP_FLAG_DEPTH(1);  // the batch sweeps its instances one iterate at a time
    kfp_swr_t h = nullptr;
    rc = kfp_swr_create(&d, &probs[i], cuda_stream, &h);
    if (rc) {
      g_batch_create_error = std::string("problem ") + std::to_string(i) + ": " + kfp_swr_create_error();
      break;
    }
    b->inst.push_back(h);
    if (!h->use_tma) {
      g_batch_create_error = "problem " + std::to_string(i) + ": the batched sweep needs at most one forcing term";
      rc = KFP_ENOTSUP;
    }
  }
  if (!rc) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || b->sms < 1) {
      cudaGetLastError();
      rc = b->fail(KFP_ECUDA, "querying the device failed");
    }
    for (auto& e : b->ev)
      if (!rc && cudaEventCreate(&e) != cudaSuccess) rc = b->fail(KFP_ECUDA, "cudaEventCreate failed");
    if (!rc) rc = b->prec == KFP_F64 ? batch_setup<double>(b) : batch_setup<float>(b);
    if (rc) g_batch_create_error = b->last_error;
  }
  if (rc) {
    b->release();
    delete b;
    return rc;
  }
  *out = b;
  return KFP_OK;
}

kfp_status kfp_batch_configure(kfp_batch_t b, int blocks_per_sm, int unit_order, int tile_shape) {
  if (!b) return KFP_EINVAL;
  if (blocks_per_sm < 0 || blocks_per_sm > 64 || unit_order < 0 || unit_order > 1 || tile_shape < 0 ||
      tile_shape >= kfp::kShapes)
    return b->fail(KFP_EINVAL, "need 0 <= blocks_per_sm <= 64, unit_order in {0, 1} and tile_shape in 0..%d",
                   kfp::kShapes - 1);
  b->blocks_per_sm = blocks_per_sm;
  b->unit_order = unit_order;
  b->shape = tile_shape;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return b->fail(KFP_ECUDA, "sync failed");
  return b->upload_units();
}

kfp_status kfp_batch_sweep(kfp_batch_t b, int max_iters, double tol, int tol_kind, int* iters_done) {
  if (!b) return KFP_EINVAL;
  b->last_error.clear();
  return b->sweep(max_iters, tol, tol_kind, iters_done);
}

kfp_status kfp_batch_instance(kfp_batch_t b, int index, kfp_swr_t* h) {
  if (!b || !h) return KFP_EINVAL;
  if (index < 0 || index >= (int)b->inst.size()) return b->fail(KFP_EINVAL, "index out of range");
  *h = b->inst[index];
  return KFP_OK;
}

kfp_status kfp_batch_stats(kfp_batch_t b, long long* iterations, long long* cell_updates_per_iter, double* sweep_ms,
                           double* reduce_ms) {
  if (!b) return KFP_EINVAL;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return b->fail(KFP_ECUDA, "sync failed");
  if (iterations) *iterations = b->iterations;
  if (cell_updates_per_iter) *cell_updates_per_iter = b->cells_per_iter;
  if (sweep_ms) *sweep_ms = b->t_sweep;
  if (reduce_ms) *reduce_ms = b->t_reduce;
  return KFP_OK;
}

void kfp_batch_destroy(kfp_batch_t b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  b->release();
  delete b;
}

const char* kfp_batch_last_error(kfp_batch_t b) { return b ? b->last_error.c_str() : g_batch_create_error.c_str(); }

const char* kfp_swr_create_error(void) { return g_create_error.c_str(); }

}  // extern "C"

// ---------------------------------------------------------------------------
// Check of the bounded device waits (no counterpart in the paper): one block polls
// an mbarrier phase that nothing completes, with the primitives of the sweep ring.
// ---------------------------------------------------------------------------

namespace {

__global__ void bounded_wait_selftest_kernel(int* flag, unsigned limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    kfp::mbar_init(&bar, 1);  // one arrival expected; none comes
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    bool done = false;
    for (unsigned it = 0; it < limit && !done; ++it) done = kfp::mbar_try_wait(&bar, 0);
    *flag = done ? 0 : 1;
  }
}

}  // namespace

extern "C" kfp_status kfp_swr_selftest_stall(kfp_swr_t h, int unit, double limit_s) {
  if (!h) return KFP_EINVAL;
  if (!h->persist) return h->fail(KFP_ENOTSUP, "the handle does not use the persistent sweep");
  const int units = ((h->flags & KFP_FLAG_GAUSS_SEIDEL) ? 1 : h->g.S) * h->nbx;
  if (unit < 0 || unit >= units) return h->fail(KFP_EINVAL, "unit %d outside 0..%d", unit, units - 1);
  if (!(limit_s > 0) || limit_s > 10) return h->fail(KFP_EINVAL, "limit_s must be in (0, 10]");
  if (h->g.nt < 3) return h->fail(KFP_EINVAL, "the check needs nt >= 3 (two interior passes)");
  KFP_CUDA_TRY_ON(h, cudaStreamSynchronize(h->stream));
  const unsigned long long keep = h->wait_ns;
  h->stall_unit = unit;
  h->wait_ns = (unsigned long long)(limit_s * 1e9);
  // the interior sweep passes only: the interface data and the norms stay as they are
  if (h->prec == KFP_F64) h->enqueue_persistent<double>(h->stream, true);
  else h->enqueue_persistent<float>(h->stream, true);
  h->stall_unit = -1;
  h->wait_ns = keep;
  KFP_CUDA_TRY_ON(h, cudaGetLastError());
  KFP_CUDA_TRY_ON(h, cudaStreamSynchronize(h->stream));
  int f = 0;
  KFP_CUDA_TRY_ON(h, cudaMemcpy(&f, h->flag, sizeof(int), cudaMemcpyDeviceToHost));
  KFP_CUDA_TRY_ON(h, cudaMemset(h->flag, 0, sizeof(int)));
  KFP_CUDA_TRY_ON(h, cudaDeviceSynchronize());
  return f ? KFP_ETIMEOUT : KFP_OK;
}

extern "C" kfp_status kfp_selftest_bounded_wait(unsigned limit, void* cuda_stream) {
  if (limit == 0) return KFP_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int* flag = nullptr;
  if (cudaMalloc(&flag, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return KFP_ENOMEM;
  }
  int h = -1;
  cudaError_t e = cudaMemsetAsync(flag, 0xff, sizeof(int), st);
  if (e == cudaSuccess) {
    bounded_wait_selftest_kernel<<<1, 32, 0, st>>>(flag, limit);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(flag);
  if (e != cudaSuccess) return KFP_ECUDA;
  return h == 1 ? KFP_ETIMEOUT : (h == 0 ? KFP_OK : KFP_ECUDA);
}
