/*
 * kfp_swr.h -- C ABI of the GB300 (sm_103a) Schwarz waveform relaxation sweep for
 * the Kolmogorov equation
 *
 *     u_t + v u_x - u_vv = f   on (0,T) x [x0,x1] x [v0,v1]
 *
 * (the problem of Section 2, eq. "Kolmogorovmain", of Gerardo-Giorda & Tran,
 * "Parallelizing the Kolmogorov-Fokker-Planck Equation", arXiv:1306.4596), with the
 * velocity interval split into S strips.  Each iteration solves every strip over
 * the whole time window from the interface data of the previous iterate (the
 * parallel form in the Remark after criterion "error" of Section 6.3), using
 * Dirichlet (classical, eq. "ClassicalSchwarz") or Robin (optimized, eq.
 * "RobinSchwarz") transmission, then exchanges the interface variables
 * lambda_1 = Q_1 u_2, lambda_2 = Q_2 u_1 (eq. "lambda12", SWR2 and SWR4) and
 * measures the mismatch of neighbouring strips on the overlap (eq. "error").
 *
 * Discretisation (the paper leaves it open for this problem):
 *   x_m = x0 + m hx (m = 0..nx), v_i = v0 + i hv (i = 0..nv), t^n = n dt (n = 0..nt);
 *   explicit first-order upwind transport by the sign of v_i (CFL |v_i| dt/hx <= 1);
 *   implicit Euler v-diffusion, centred second difference, one tridiagonal system
 *   per x-column and strip; inflow Dirichlet data at x0 (v_i > 0) and x1 (v_i < 0);
 *   Dirichlet data at v0 and v1; half-cell finite-volume Robin rows.
 * Strips: interface j = 0..S-2 has centre node I_j = (j+1) nv/S, overlap nodes
 * alpha_j = I_j - floor(ov/2) .. beta_j = alpha_j + ov; strip s covers nodes
 * lo_s = (s ? alpha_{s-1} : 0) .. hi_s = (s < S-1 ? beta_s : nv).
 *
 * General conventions
 *   - Every function returns a kfp_status; no function throws or aborts.  On an
 *     error the handle (if any) keeps a message readable with kfp_swr_last_error.
 *   - All GPU work is enqueued on the stream given at create (a cudaStream_t passed
 *     as void*; NULL = the legacy default stream).  Calls that return host data
 *     synchronise that stream.
 *   - The handle owns all device memory it allocates (freed by kfp_swr_destroy).
 *     Input arrays are copied at create; the caller keeps ownership of them.
 *   - A handle is not thread-safe: use it from one host thread at a time.
 *   - Array shapes are row-major, last index fastest, all FP64.
 */
#ifndef KFP_SWR_H
#define KFP_SWR_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kfp_swr* kfp_swr_t; /* opaque handle */

typedef enum {
  KFP_OK = 0,
  KFP_EINVAL = 1,    /* invalid argument or descriptor */
  KFP_ECFL = 2,      /* |v_i| dt / hx > 1 somewhere: the explicit upwind step is unstable */
  KFP_ENOMEM = 3,    /* device or host allocation failed */
  KFP_ECUDA = 4,     /* a CUDA call failed (message holds the CUDA error string) */
  KFP_ENOTCONV = 5,  /* max_iters reached before the requested tolerance */
  KFP_ENUMERIC = 6,  /* a NaN or Inf appeared in the interface norms */
  KFP_ETIMEOUT = 7,  /* a bounded device-side wait expired */
  KFP_ENOTSUP = 8    /* the requested mode is not built into this library */
} kfp_status;

typedef enum { KFP_DIRICHLET = 0, KFP_ROBIN = 1 } kfp_transmission;

/* Arithmetic of the strip solves.  Interface traces, bands, norms and every array
 * crossing the ABI stay FP64 in all modes.
 * KFP_MIXED: defect correction on the interface problem.  Each outer step runs one
 * FP64 iteration from the current interface data lambda (its norms are the ones
 * reported; its residual is d = G(lambda) - lambda with G the map of one iteration),
 * then solves delta = M delta + d (M = the linear part of G) by FP32 iterations of
 * the homogeneous problem and sets lambda += delta in FP64; the FP32 rounding thus
 * falls on the correction only.  kfp_swr_sweep's max_iters counts outer steps. */
typedef enum { KFP_F64 = 0, KFP_F32 = 1, KFP_MIXED = 2 } kfp_precision;

/* Flags of kfp_swr_desc.flags */
#define KFP_FLAG_NO_GRAPH 1u  /* launch every kernel directly instead of replaying a CUDA graph */
#define KFP_FLAG_PROFILE 2u   /* time the sweep, exchange and error kernels with CUDA events */
#define KFP_FLAG_GENERIC 4u   /* use the plain sweep kernel even where the TMA-fed one applies */
#define KFP_FLAG_GAUSS_SEIDEL 8u /* serial form SWR1-SWR4 of Section 6.3: strips in increasing order,
                                  * each taking its lower interface data from the strip below in the
                                  * same iteration (default: the parallel form of the Remark) */
/* Boundary conditions of the model problem of Section 6.1 (default: Dirichlet data). */
#define KFP_FLAG_NEUMANN_V 16u   /* zero flux at v0 and v1: half-cell rows (1+2r) u_0 - 2r u_1 = R_0 and
                                  * (1+2r) u_nv - 2r u_{nv-1} = R_nv; bc_v is ignored */
#define KFP_FLAG_PERIODIC_X 32u  /* periodic in x: the unknowns are m = 0..nx-1 and node nx repeats
                                  * node 0 in every output; bc_xin, column nx of u0 and f_space, and
                                  * column nx of lambda0 / set_traces data are ignored (replaced by
                                  * column 0); needs nx >= 2 */
/* How the nt-1 interior sweep passes of an iteration are launched (TMA-fed sweep
 * without periodic x; results are bitwise the same either way).  By default the
 * library runs them in one co-resident (cooperative) launch -- the streamed sweep --
 * when a pass has more units (strip x block of 120 columns) than the GPU holds
 * blocks at once, and one launch per pass otherwise (measured faster there) -- for a
 * lone iterate; sweeps of several iterations on smaller grids pipeline iterates
 * (KFP_FLAG_DEPTH below).  Either flag also turns pipelining off. */
#define KFP_FLAG_PERSISTENT 128u /* always the streamed sweep */
#define KFP_FLAG_PER_PASS 256u   /* always one launch per pass */
/* Tile shape of the TMA-fed sweep (rows per ring stage, ring stages, blocks per SM);
 * results are bitwise the same for every shape.  By default the library takes shape
 * 0 when a pass has at most one unit per SM and shape 1 otherwise.
 *   KFP_FLAG_SHAPE(0): 16-row stages, 1 block per SM (4 stages FP64, 8 FP32)
 *   KFP_FLAG_SHAPE(1):  8-row stages, 2 blocks per SM (4 stages FP64, 8 FP32)
 *   KFP_FLAG_SHAPE(2):  8-row stages, 2 blocks per SM (6 stages FP64, 12 FP32) */
#define KFP_FLAG_SHAPE_SHIFT 9
#define KFP_FLAG_SHAPE(n) ((unsigned)((n) + 1) << KFP_FLAG_SHAPE_SHIFT)
/* Pipelined iterates (parallel form, TMA-fed sweep, no periodic x, nt >= 3): the
 * sweeps of D consecutive SWR iterates run in one streamed launch as a wavefront
 * over (iterate, time step) -- iterate d solves step k once iterate d-1 has recorded
 * the interface data at t^k and t^(k+1) (Section 6.3: each strip reads its
 * neighbours' previous iterate level by level).  The results of every iterate, the
 * iteration count at a tolerance and the history are bitwise those of lone
 * iterations; kfp_swr_sweep computes up to D-1 iterates beyond the one at which a
 * tolerance is met and discards them.  By default D = 2 x (streamed blocks resident
 * at once) / (units of a pass), at most 8 and at most nt - 1, and 1 (no pipelining)
 * with KFP_FLAG_PERSISTENT or KFP_FLAG_PER_PASS; KFP_FLAG_DEPTH(n), n = 1..8, fixes
 * it (n = 1: none; larger n count as 8).  Each extra iterate in flight holds its own
 * residue buffers, final state, overlap bands and interface data (device memory).
 * kfp_swr_gradient pipelines its forward iterates the same way and its adjoint
 * iterates in groups of up to 16 (one at a time with n = 1). */
#define KFP_FLAG_DEPTH_SHIFT 11
#define KFP_FLAG_DEPTH(n) ((unsigned)(n) << KFP_FLAG_DEPTH_SHIFT)
#define KFP_FLAG_SPLIT_SCHEME 64u /* the paper's own discretisation (Section 6.2): Lie splitting, each
                                  * step (M + dt S) w = M (u^n + dt f^{n+1}) with P1 elements in v
                                  * (mass M, stiffness S; Robin ends add dt p or dt q to the end row
                                  * and dt lambda to its right-hand side), then explicit upwind
                                  * transport u^{n+1} = w - c_i (w - w_upstream), c_i = |v_i| dt / hx;
                                  * needs KFP_FLAG_NEUMANN_V | KFP_FLAG_PERIODIC_X.  The interface data
                                  * come from w: Dirichlet w, Robin without overlap (p+q) w - lambda_in,
                                  * Robin with overlap p w (q w) minus the half-row residual */

typedef struct {
  double x0, x1, v0, v1; /* box [x0,x1] x [v0,v1], x1 > x0, v1 > v0 */
  double dt;             /* time step, T = nt dt */
  int nx, nv, nt;        /* intervals in x (>= 1) and v (>= 2), time steps (>= 1) */
  int nstrips;           /* S >= 1, must divide nv; nv/S >= 2 when S > 1 */
  int overlap_cells;     /* ov, 0 <= ov < nv/S (ignored when S == 1) */
  kfp_transmission tc;   /* transmission condition on every interface */
  const double* p;       /* host [S-1]: Robin p_j > 0 (lower strip's top, p + d/dv); NULL for Dirichlet */
  const double* q;       /* host [S-1]: Robin q_j > 0 (upper strip's bottom, q - d/dv); NULL = p */
  kfp_precision prec;    /* arithmetic of the strip solves */
  unsigned flags;        /* KFP_FLAG_* */
} kfp_swr_desc;

typedef struct {
  int on_device;          /* 1: the pointers below are device memory of the current device; 0: host */
  const double* u0;       /* [nv+1][nx+1] initial data u0(x_m, v_i) (required) */
  int nforce;             /* number of separable forcing terms R >= 0 */
  const double* f_time;   /* [R][nt+1] a_r(t^n)       (NULL allowed only when R == 0) */
  const double* f_space;  /* [R][nv+1][nx+1] F_r(x_m, v_i); f = sum_r a_r(t) F_r(x, v) */
  const double* bc_xin;   /* [nt+1][2][nv+1] inflow data at x0 ([.][0]) and x1 ([.][1]); NULL = 0 */
  const double* bc_v;     /* [nt+1][2][nx+1] Dirichlet data at v0 ([.][0]) and v1 ([.][1]); NULL = 0 */
  const double* lambda0;  /* [S-1][2][nt][nx+1] initial interface data lambda^0; NULL = 0.
                           * [j][0][n-1] = lambda_1 of interface j at t^n (data at the lower
                           * strip's top node beta_j), [j][1][n-1] = lambda_2 (data at the
                           * upper strip's bottom node alpha_j). */
} kfp_swr_problem;

/*
 * Create a solver: validate the descriptor (grid, strip layout, CFL, Robin
 * parameters), build the strip layout and the constant-coefficient tridiagonal
 * factors (Section 6.3, eq. "Om1_Om2" generalised to S strips), allocate device
 * memory and copy the inputs (stream-ordered on `cuda_stream`).
 * Errors: KFP_EINVAL (NULL or inconsistent arguments), KFP_ECFL, KFP_ENOMEM, KFP_ECUDA.
 * On error *out is set to NULL.
 */
kfp_status kfp_swr_create(const kfp_swr_desc* desc, const kfp_swr_problem* prob, void* cuda_stream,
                          kfp_swr_t* out);

/*
 * Run SWR iterations (Section 6.3, SWR1-SWR4 in the parallel form of the Remark):
 * each iteration sweeps every strip over all nt steps from the current interface
 * data, exchanges the new interface data, and reduces the norms
 *   e_mis = max over interfaces, n = 1..nt, overlap nodes, m of |u_j - u_{j+1}|  (eq. "error"),
 *   e_chg = max |lambda^k - lambda^{k-1}|,   j_l2 = dt hx sum (u_j - u_{j+1})^2.
 * Stops after max_iters iterations or as soon as the norm chosen by tol_kind
 * (0: e_chg, 1: e_mis) is below tol.  tol <= 0 runs exactly max_iters iterations
 * without reading anything back in between.  Iterations continue from the current
 * interface data (calls can be chained).  *iters_done (may be NULL) receives the
 * number of iterations run by this call.  With pipelined iterates (KFP_FLAG_DEPTH)
 * the tolerance is read after each group of D iterations and the handle is left at
 * the first iterate that met it: the same count and state as one iterate at a time.
 * Errors: KFP_EINVAL, KFP_ECUDA, KFP_ENOTCONV (tol > 0 not reached), KFP_ENUMERIC,
 * KFP_ETIMEOUT (a bounded wait of the streamed sweep expired).
 */
kfp_status kfp_swr_sweep(kfp_swr_t h, int max_iters, double tol, int tol_kind, int* iters_done);

/* Copy the current interface data lambda^k of interface `iface` (0..S-2), side 0
 * (lambda_1 = Q_1 u of eq. "lambda12", the data that the lower strip takes at its
 * top node beta_j) or 1 (lambda_2 = Q_2 u, the data that the upper strip takes at
 * its bottom node alpha_j): [nt][nx+1], row n-1 at t^n, to dst (host, or device
 * memory when dst_on_device; the caller owns dst).  After an iteration these are
 * the data the next iteration uses (SWR2 and SWR4 of Section 6.3).  Synchronises.
 * Errors: KFP_EINVAL (NULL handle or dst, iface or side out of range), KFP_ECUDA. */
kfp_status kfp_swr_traces(kfp_swr_t h, int iface, int side, double* dst, int dst_on_device);

/* Replace the interface data by src [S-1][2][nt][nx+1] (host or device); used to
 * resume from a checkpoint taken with kfp_swr_traces.  Errors: KFP_EINVAL, KFP_ECUDA. */
kfp_status kfp_swr_set_traces(kfp_swr_t h, const double* src, int src_on_device);

/* Norms of the last iteration and the history of all iterations of this handle:
 * history (may be NULL) receives min(hist_cap, iterations) rows of
 * (e_mis, e_chg, j_l2).  Any scalar pointer may be NULL.  Synchronises.
 * Errors: KFP_EINVAL (no iteration has run), KFP_ECUDA. */
kfp_status kfp_swr_error(kfp_swr_t h, double* e_mis, double* e_chg, double* j_l2, double* history,
                         int hist_cap);

/* Copy the overlap values of the last iteration, interface `iface`, side 0 (lower
 * strip) or 1 (upper strip): [nt][ov+1][nx+1], rows alpha_j..beta_j.  Synchronises. */
kfp_status kfp_swr_bands(kfp_swr_t h, int iface, int side, double* dst, int dst_on_device);

/* Copy the solution at t = T of the last iteration, [nv+1][nx+1], to dst (host, or
 * device memory when dst_on_device; the caller owns dst).  The paper defines the
 * iterate only per subdomain (u_1^k on Omega_1, u_2^k on Omega_2, Section 6.3); on
 * an overlap both strips hold a value, and this library takes node i from the lower
 * strip of interface j when i <= I_j and from the upper strip otherwise (a tie-break
 * of its own; the two values agree once the iteration has converged).
 * Synchronises.  Errors: KFP_EINVAL (NULL handle or dst, no iteration has run),
 * KFP_ECUDA. */
kfp_status kfp_swr_solution(kfp_swr_t h, double* dst, int dst_on_device);

/* Counters of this handle (all may be NULL): iterations run, cell-updates per
 * iteration ((nx+1) * sum_s (hi_s - lo_s + 1) * nt), kernels launched per
 * iteration, and -- when KFP_FLAG_PROFILE is set -- the summed device time in
 * milliseconds of the sweep kernels, the exchange kernel and the error kernel
 * (CUDA events recorded on the handle's stream).  Synchronises. */
kfp_status kfp_swr_stats(kfp_swr_t h, long long* iterations, long long* cell_updates_per_iter,
                         int* launches_per_iter, double* sweep_ms, double* exchange_ms,
                         double* error_ms);

/* Launch counters of this handle (all pointers may be NULL): the group size D of
 * pipelined iterates chosen at create (see KFP_FLAG_DEPTH; 1: no pipelining); the
 * kernels launched by all sweeps so far (a mixed-precision handle adds those of its
 * FP32 correction solver); and, over the groups run so far, the number of streamed
 * launches, the cell-updates those launches computed (the passes of each group's
 * wavefront that run inside it) and -- with KFP_FLAG_PROFILE -- their summed device
 * time in milliseconds (CUDA events around each streamed launch).  Synchronises.
 * Errors: KFP_EINVAL (NULL handle). */
kfp_status kfp_swr_pipeline_stats(kfp_swr_t h, int* depth, long long* kernel_launches, long long* stream_launches,
                                  long long* stream_cell_updates, double* stream_ms);

/*
 * Gradient of the interface mismatch after K iterations with respect to the Robin
 * parameters (discrete adjoint; Robin transmission, no overlap, KFP_F64).
 *   J = dt hx sum_j sum_{n=1..nt} sum_m (u_j - u_{j+1})^2 on the interface nodes of
 *   the K-th iterate from lambda^0 = lam0 (NULL = 0; host or device memory), i.e. the
 *   j_l2 norm of kfp_swr_sweep.  grad_p, grad_q (host, [S-1], may be NULL) receive
 *   dJ/dp_j and dJ/dq_j (for one-sided OSWR(p) with q = p, dJ/dp_j + dJ/dq_j).
 * The forward part runs K iterations on the handle (they count in its history and
 * leave lambda^K as its interface data); the adjoint solves the transposed
 * implicit-Euler systems backward in time and the transposed exchange backward over
 * the iterates, using only the interface-node values of every iterate.  Errors:
 * KFP_ENOTSUP (other transmission, overlap, precision), KFP_EINVAL, KFP_ECUDA. */
kfp_status kfp_swr_gradient(kfp_swr_t h, int K, const double* lam0, int lam0_on_device, double* J, double* grad_p,
                            double* grad_q);

/* Replace the Robin parameters (host arrays [S-1]; q = NULL means q = p) and rebuild
 * the factors in place; the interface data are kept.  Errors: KFP_EINVAL. */
kfp_status kfp_swr_set_robin(kfp_swr_t h, const double* p, const double* q);

/* Largest interface count accepted by kfp_iface_norms_noalloc. */
#define KFP_NOALLOC_MAX_INTERFACES 64

/*
 * Interface norms computed without allocating memory.  The paper has no
 * counterpart: this entry point serves callers that may not allocate device memory
 * themselves or let a library do so -- for example code running inside a host
 * application that owns every device allocation and hands a plugin only its input
 * and output buffers, or a latency-critical loop that cannot afford cudaMalloc
 * (which can synchronise the device and takes the allocator's lock).
 *
 * bands: device memory, [nif][2][nt][overlap_cells+1][nx+1] FP64, the layout of
 *   kfp_swr_bands ([j][0] = lower strip, [j][1] = upper strip of interface j).
 * periodic_x: nonzero for a problem created with KFP_FLAG_PERIODIC_X.  Column nx
 *   then repeats column 0 and is left out of both sums, as kfp_swr_error does, so
 *   that each node counts once; needs nx >= 2.
 * out:   device memory, 2 + 2*nif doubles, written by the kernel:
 *   out[0] = e_mis = max |lower - upper|, out[1] = j_l2 = dt hx sum (lower - upper)^2,
 *   out[2+2j], out[3+2j] = the same two norms of interface j alone.
 * The work is enqueued on cuda_stream (NULL = legacy default stream); nothing is
 * synchronised except during the set-up below.
 *
 * Scratch: a file-scope device array of 64 x 32 x 2 doubles plus a counter
 * (32 KiB) that every GPU which loads this library keeps until the process exits.
 * The first call on a device does a one-time set-up with that device current (it
 * looks up the array's device address and zeroes the counter, then synchronises
 * the device), so make that first call before any stream capture.  Every call
 * shares the array: calls whose kernels can overlap on the GPU (other streams,
 * other host threads) race and must be serialised by the caller.
 * Errors: KFP_EINVAL for NULL pointers, non-positive sizes, periodic_x with
 * nx < 2 or nif > KFP_NOALLOC_MAX_INTERFACES; KFP_ECUDA if the set-up or the launch fails.
 * Allocates nothing: no cudaMalloc, no cudaFree, no allocating library call.
 */
kfp_status kfp_iface_norms_noalloc(const double* bands, int nif, int nt, int overlap_cells, int nx,
                                   int periodic_x, double dt, double hx, double* out, void* cuda_stream);

/*
 * Check of the bounded device waits; the paper has no counterpart.  Every wait of
 * the sweep kernels on an mbarrier phase gives up after a limit, raises a flag and
 * returns, and the host then reports KFP_ETIMEOUT with the context still usable.
 * This runs that path on purpose without faulting anything: one block polls, at most
 * `limit` times, an mbarrier phase that nothing completes.  Enqueued on cuda_stream
 * and synchronised.  Returns KFP_ETIMEOUT when the wait gave up as designed (KFP_OK
 * would mean the phase completed, which cannot happen); KFP_EINVAL for limit == 0;
 * KFP_ENOMEM, KFP_ECUDA.
 */
kfp_status kfp_selftest_bounded_wait(unsigned limit, void* cuda_stream);

/*
 * Check of the bounded waits between the units of the persistent sweep; the paper
 * has no counterpart.  The streamed sweep (see KFP_FLAG_PERSISTENT) runs the interior
 * passes of an iteration in one launch, and before a unit (strip, block of 120
 * columns) starts pass k it waits until its column neighbours have finished pass k-1.  This
 * runs the sweep passes of one iteration once with unit `unit` never reporting
 * completion, so that its neighbours' waits give up after `limit_s` seconds, raise
 * the error flag and every block leaves; the interface data, history and counters
 * of the handle are not touched, the flag is cleared afterwards, and the next
 * kfp_swr_sweep runs as if this call had not happened.  Synchronises.
 * Returns KFP_ETIMEOUT when the waits gave up as designed (KFP_OK would mean the
 * stalled unit went unnoticed); KFP_ENOTSUP when the handle does not use the
 * streamed sweep; KFP_EINVAL for a unit outside 0..units-1 or limit_s outside
 * (0, 10] or nt < 3 (fewer than two interior passes); KFP_ECUDA.
 */
kfp_status kfp_swr_selftest_stall(kfp_swr_t h, int unit, double limit_s);

/*
 * FP64 fused multiply-add rate of the current device, for the roofline of the FP64
 * sweep (which the FP64 pipe, not HBM, bounds); the paper has no counterpart.  One
 * block of 32 * warps_per_sm threads per SM, each thread running `chains` (1, 2, 4
 * or 8) independent recurrences x <- x a + b for 8 * steps dependent steps, timed
 * with CUDA events on cuda_stream after a short warm-up launch.  *dfma_per_s
 * receives the lane-level DFMA operations per second (2 flops each); *sm_mhz (may
 * be NULL) the SM clock seen during the run (cycle counter over nanosecond timer of
 * block 0).  Many warps with several chains give the pipe's throughput; one warp per
 * sub-partition with one chain gives 1 / (dependent DFMA latency).  Allocates and
 * frees its own small buffers; synchronises.  Errors: KFP_EINVAL (chains not in
 * {1,2,4,8}, warps_per_sm outside 1..32, steps < 1, NULL dfma_per_s), KFP_ENOMEM,
 * KFP_ECUDA.
 */
kfp_status kfp_probe_fp64_rate(int chains, int warps_per_sm, int steps, double* dfma_per_s, double* sm_mhz,
                               void* cuda_stream);

/* Iteration counters (any pointer may be NULL): iterations whose strip solves ran
 * in FP64 and in FP32 (for KFP_MIXED: outer FP64 steps and inner FP32 correction
 * iterations), and -- with KFP_FLAG_PROFILE -- the summed device time of the FP32
 * sweep kernels in milliseconds.  Synchronises.  Errors: KFP_EINVAL, KFP_ECUDA. */
kfp_status kfp_swr_counters(kfp_swr_t h, long long* fp64_iterations, long long* fp32_iterations,
                            double* fp32_sweep_ms);

/* ---------------------------------------------------------------------------
 * Batched form: many independent problems (uneven grids, strip counts, Robin
 * parameters and step counts) swept together.  Every time step of every problem is
 * one work unit per (strip, block of 120 columns).  Per iteration: one launch runs the
 * first pass of every unit; one persistent (cooperative) launch per forcing mode runs
 * all interior passes of all problems, units taking work in pass order and waiting
 * (bounded) on their column neighbours; one launch runs the last pass of every unit;
 * then the per-problem exchange and error reductions.  The iteration replays as one
 * CUDA graph.  The method per problem is exactly that of kfp_swr_sweep (Section 6.3,
 * parallel form), and every problem's results equal its single-problem run bit for bit.
 * ------------------------------------------------------------------------- */
typedef struct kfp_batch* kfp_batch_t;

/* Create count problems (descs[i], probs[i] as for kfp_swr_create) on one stream.
 * All problems use the same precision, KFP_F64 or KFP_F32, and at most one forcing
 * term.  Errors: KFP_EINVAL, KFP_ECFL, KFP_ENOMEM, KFP_ECUDA, KFP_ENOTSUP (mixed
 * precision or two or more forcing terms); the message is kfp_batch_last_error(NULL). */
kfp_status kfp_batch_create(const kfp_swr_desc* descs, const kfp_swr_problem* probs, int count, void* cuda_stream,
                            kfp_batch_t* out);

/* Launch shape.  blocks_per_sm (first and last passes): 0 runs one block per work
 * unit, > 0 a grid of blocks_per_sm x (number of SMs) blocks that walk the unit list.
 * unit_order: 0 lists the units of each step count taller strips first, 1 keeps
 * problem order.  tile_shape (interior passes): the shapes of KFP_FLAG_SHAPE, 0..2
 * (default 1).  Results do not depend on any choice.  Synchronises.  Errors:
 * KFP_EINVAL, KFP_ECUDA. */
kfp_status kfp_batch_configure(kfp_batch_t b, int blocks_per_sm, int unit_order, int tile_shape);

/* Run iterations of every problem, as kfp_swr_sweep; with tol > 0 stop when every
 * problem's chosen norm is below tol. */
kfp_status kfp_batch_sweep(kfp_batch_t b, int max_iters, double tol, int tol_kind, int* iters_done);

/* Handle of problem `index`, for kfp_swr_traces / error / bands / solution / stats.
 * It stays owned by the batch: do not destroy it. */
kfp_status kfp_batch_instance(kfp_batch_t b, int index, kfp_swr_t* h);

/* Iterations run, cell-updates per iteration summed over the problems, and (with
 * KFP_FLAG_PROFILE in descs[0].flags) the summed device time of the sweep launches
 * and of the reductions, in milliseconds.  Synchronises. */
kfp_status kfp_batch_stats(kfp_batch_t b, long long* iterations, long long* cell_updates_per_iter, double* sweep_ms,
                           double* reduce_ms);

/* Free the batch and all its problems (NULL is ignored). */
void kfp_batch_destroy(kfp_batch_t b);

/* Message of the last error on b, or of the last failed kfp_batch_create (b = NULL). */
const char* kfp_batch_last_error(kfp_batch_t b);

/* Free every resource of the handle: the device copies of the problem, the strip
 * states, the interface data and overlap values, graphs and events.  This ends the
 * iteration of Section 6.3; the paper has no further counterpart.  NULL is ignored;
 * the handle must not be used afterwards.  Synchronises its stream; cannot fail. */
void kfp_swr_destroy(kfp_swr_t h);

/* Message of the last error on this handle ("" if none); valid until the next call. */
const char* kfp_swr_last_error(kfp_swr_t h);

/* Message of the last error of a failed kfp_swr_create on this thread. */
const char* kfp_swr_create_error(void);

#ifdef __cplusplus
}
#endif
#endif /* KFP_SWR_H */
