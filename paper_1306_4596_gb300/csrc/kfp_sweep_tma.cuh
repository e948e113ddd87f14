// kfp_sweep_tma.cuh -- TMA-fed sweep pass (sm_103a).
//
// Same pass as sweep_pass_kernel (back-substitution of step k fused with the
// elimination of step k+1 in the same row order, lanes = x-columns, warp-shuffle
// upwind neighbour, halo lanes), but every per-row input is streamed into shared
// memory by the tensor-memory accelerator ahead of use:
//
//   warp 4 (producer, one elected lane) issues, per chunk of CH rows,
//     cp.async.bulk.tensor.2d loads of the block's [CH x kBoxW] tile of the
//     elimination residue y^k (or u^0 in the first pass), the same tile of the
//     forcing term, and the [CH x 24] tile of per-row coefficient records,
//   into a ring of NST stages guarded by full/empty mbarriers;
//   warps 0..3 (consumers) wait on the stage, run the row recurrences from shared
//     memory and store y^{k+1} straight to global memory (coalesced).
//
// Coefficient record of one row, one column class and one pass direction (24 = 3
// classes x 8 fields):
//   0: -cp   back-substitution coefficient of step k (eliminated the other way)
//   1: A  = g (1 - c_i)     2: B = g c_i        (upwind transport, c_i = |v_i| dt/hx)
//   3: -g a (coupling to the previously eliminated row)
//   4: g     5: g * 2dt/hv (Robin interface data)
//   6: sign of v_i (integer bits)
//   7: row kind (integer bits: 0 interior, 1 x inflow, 2 v boundary,
//      3/4 Dirichlet top/bottom, 5/6 Robin top/bottom)
// Fields 0-3 are read as one 16-byte vector (FP32) or two (FP64).
// Identity rows (kinds 1-4) carry A = B = -g a = g = 0 (and G = 0), so that with zero
// boundary data they need no branch; their data, the interface rows and rows whose
// u^k is recorded are handled in the first and last chunk of a pass (general path).
// An interior row costs four fused multiply-adds:
//   u = y^k - cp u_prev;  y^{k+1} = (A u + B u_nb + G) - g a y_prev
// with G = g dt a F pre-scaled once (FMODE 1, constant-in-time forcing), G = 0
// (FMODE 0) or G = (g dt a(t^{k+1})) F (FMODE 2, one time-dependent term).
//
// Every wait on an mbarrier is bounded; on expiry the kernel raises a flag that
// the host reports as KFP_ETIMEOUT, and the producer drains the copies it issued.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "kfp_kernels.cuh"

namespace kfp {

constexpr int kChunkMax = 16;                                // most rows per stage (record padding)

// Tile shape of the TMA-fed sweep: CH rows per ring stage (8 or 16), NST ring stages,
// MINB blocks resident per SM (the launch bound).  16-row stages and one block per
// SM suit a pass with about one unit per SM; 8-row stages need fewer registers and
// less shared memory, so that two blocks -- two consumer warps per SM sub-partition
// -- hide each other's latencies when a pass has several units per SM.
template <int CH_, int NST_, int MINB_>
struct Shape {
  static constexpr int CH = CH_, NST = NST_, MINB = MINB_;
  static_assert(CH == 8 || CH == 16, "tensor maps exist for 8- and 16-row boxes");
};
constexpr int kBoxW = kWarpsPerBlock * kOutCols + 4;         // 124 columns per tile
constexpr int kRecW = 24;                                    // record row: 3 classes x 8
constexpr int kRecPad = kChunkMax;                           // zero rows before/after each record table
constexpr unsigned kSpinLimit = 1u << 26;                    // bounded mbarrier waits

struct TmaMaps {
  CUtensorMap state;   // Y0/Y1 stacked as [2 * rows][P] (buffer b at row offset b*rows)
  CUtensorMap init;    // U0 [nv+1][P]
  CUtensorMap force;   // FMODE 1: GF [2 * rows][P] (pass direction d at row offset d*rows);
                       // FMODE 2: F [nv+1][P]
  CUtensorMap rec;     // records [S * 2 * (Lmax + 2 kRecPad)][24]
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Integer stored bit-for-bit in a record slot (no floating-point conversion).
__device__ __forceinline__ int slot_int(double v) { return (int)__double_as_longlong(v); }
__device__ __forceinline__ int slot_int(float v) { return __float_as_int(v); }

// Bounded wait: false if the limit was reached.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  for (unsigned it = 0; it < kSpinLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

template <typename T>
struct TmaArgs {
  PassArgs<T> p;       // geometry, strips, boundary data, traces, outputs
  int rows;            // total strip rows (sum L_s)
  int Lpad;            // Lmax + 2 kRecPad
  int* flag;           // error flag (1 = a wait timed out)
  int bc_data;         // caller gave x-inflow or v-boundary data (rows of kind 1/2 need it)
};

// Work description the producer of the streamed sweep writes into the stage of a
// unit's first chunk (k < 0: no more work).  The pass arguments travel with it: read
// from shared memory they cannot alias the consumers' global stores, so the
// compiler need not reload them after each store (as it must from global memory).
struct StreamTail {
  StripInfo st;                // the unit's strip
  int k, inst, strip, bx, nc, unit, new_args;
};
template <typename T>
struct StreamHeader {
  TmaArgs<T> args;             // the unit's problem (written only when it changes: new_args)
  StreamTail tail;
};

// Copy n 32-bit words from src to dst, lane `lane` of `lanes` copying every lanes-th.
__device__ __forceinline__ void copy_words(void* dst, const void* src, int n, int lane, int lanes) {
  const int* s = reinterpret_cast<const int*>(src);
  int* d = reinterpret_cast<int*>(dst);
  for (int i = lane; i < n; i += lanes) d[i] = s[i];
}

template <typename T, class SH>
struct TmaSmem {
  T tile[SH::NST][SH::CH][kBoxW];
  T frc[SH::NST][SH::CH][kBoxW];
  T rec[SH::NST][SH::CH][kRecW];
  uint64_t full[SH::NST];
  uint64_t empty[SH::NST];
  StreamHeader<T> hdr[SH::NST];
  // each consumer warp's copy of the header of the unit it is running: once the
  // unit's first stage is released, a later unit's header may land in that stage
  StreamHeader<T> cur[kWarpsPerBlock];
  int abort;  // set by the producer before it completes a stage without data
};

// Fields 0..3 of a record (ncp, A, B, -g a) as vector loads.
__device__ __forceinline__ void load_coef4(const double* rc, double& ncp, double& a, double& b, double& hn) {
  const double2 v0 = *reinterpret_cast<const double2*>(rc);
  const double2 v1 = *reinterpret_cast<const double2*>(rc + 2);
  ncp = v0.x; a = v0.y; b = v1.x; hn = v1.y;
}
__device__ __forceinline__ void load_coef4(const float* rc, float& ncp, float& a, float& b, float& hn) {
  const float4 v = *reinterpret_cast<const float4*>(rc);
  ncp = v.x; a = v.y; b = v.z; hn = v.w;
}

// Record the outgoing interface data and the overlap values of u^k at row l.
// lam_top / lam_bot: the incoming data of this strip at t^k (used by the Robin
// trace without overlap), loaded once per pass.
template <typename T, bool UP>
__device__ __forceinline__ void record_row(const PassArgs<T>& A, const StripInfo& st, int s, int k, int l,
                                           int m, bool out_lane, T u, T u_m1, T u_m2, double lam_top,
                                           double lam_bot) {
  const int ov = A.ov, nt = A.nt, nxp = A.nx + 1, lo = st.lo;
  const bool robin_in = A.robin && ov >= 1;
  if (st.has_top) {
    const int aT = st.alpha_top - lo;
    const int eT = robin_in ? (UP ? aT + 1 : aT - 1) : aT;
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
        lam = (st.p_top + st.q_top) * (double)u - lam_top;
      }
      const size_t o = (((size_t)s * 2 + 1) * nt + (k - 1)) * nxp + m;
      A.lam_next[o] = A.lam_add ? lam + A.lam_add[o] : lam;
    }
  }
  if (st.has_bot) {
    const int aB = st.alpha_bot - lo;
    const int eB = robin_in ? (UP ? aB + ov + 1 : aB + ov - 1) : aB + ov;
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
        lam = (st.p_bot + st.q_bot) * (double)u - lam_bot;
      }
      const size_t o = ((((size_t)s - 1) * 2 + 0) * nt + (k - 1)) * nxp + m;
      A.lam_next[o] = A.lam_add ? lam + A.lam_add[o] : lam;
    }
  }
}

// Right-hand side override of a non-interior row (kinds 1..6), given the regular value.
// lam_top / lam_bot: this strip's incoming data at t^{k1} (0 outside the domain).
template <typename T>
__device__ __forceinline__ T special_row(const PassArgs<T>& A, int kind, int k1, int i, int m, bool in_dom,
                                         int inflow_side, T regular, T glam, double lam_top, double lam_bot) {
  const int nxp = A.nx + 1;
  switch (kind) {
    case 1:
      return (A.bc_xin && inflow_side >= 0) ? (T)A.bc_xin[((size_t)k1 * 2 + inflow_side) * (A.nv + 1) + i] : T(0);
    case 2:
      return (A.bc_v && in_dom) ? (T)A.bc_v[((size_t)k1 * 2 + (i == 0 ? 0 : 1)) * nxp + m] : T(0);
    case 3:
      return (T)lam_top;
    case 4:
      return (T)lam_bot;
    case 5:
      return (T)((double)regular + (double)glam * lam_top);
    case 6:
      return (T)((double)regular + (double)glam * lam_bot);
    default:
      return regular;
  }
}

// MODE 0: eliminate step 1 from u^0; 1: back-substitute step k, eliminate step k+1;
// 2: back-substitute the last step and store u^nt.  FMODE: 0 no forcing, 1 folded
// constant forcing, 2 one time-dependent term.
template <typename T, class SH>
__device__ __forceinline__ void init_ring(TmaSmem<T, SH>& sm) {
  if (threadIdx.x == 0) {
    for (int q = 0; q < SH::NST; ++q) {
      mbar_init(&sm.full[q], 1);
      mbar_init(&sm.empty[q], kWarpsPerBlock);
    }
    sm.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
}

// Producer half of one unit's pass (one elected lane): issue the TMA loads of its
// NC chunks into the ring, from chunk number cbase on; with TAIL, write the unit's
// header (and, when tail->new_args, a copy of X) into the stage of the first chunk
// before that stage is released.  Returns false if a
// bounded wait expired (the copies already issued are drained first).
template <typename T, bool UP, int MODE, int FMODE, class SH>
__device__ __forceinline__ bool produce_unit(const TmaMaps& maps, const TmaArgs<T>& X, const int k, const int s,
                                             const int bx, const StripInfo& st, TmaSmem<T, SH>& sm,
                                             const unsigned cbase, const StreamTail* tail) {
  const int L = st.L;
  const int NC = (L + SH::CH - 1) / SH::CH;
  constexpr bool kUseForce = (MODE != 2) && (FMODE != 0);
  const int dir = UP ? 0 : 1;
  const int x0 = bx * (kWarpsPerBlock * kOutCols);
  const unsigned bytes = (unsigned)(sizeof(T) * (SH::CH * kBoxW * (kUseForce ? 2 : 1) + SH::CH * kRecW));
  const int cur = k & 1;
  bool ok = true;
  int issued = 0;
  for (int c = 0; c < NC; ++c) {
    const unsigned g = cbase + (unsigned)c;
    const int q = (int)(g % SH::NST);
    const unsigned use = g / SH::NST;
    if (use > 0 && !mbar_wait(&sm.empty[q], (use - 1) & 1)) { ok = false; break; }
    const int l0 = UP ? c * SH::CH : L - (c + 1) * SH::CH;
    if (c == 0 && tail) {  // the unit's header, released to the consumers with the stage
      static_assert(sizeof(TmaArgs<T>) % 4 == 0, "arguments are copied as 32-bit words");
      sm.hdr[q].tail = *tail;
      if (tail->new_args) copy_words(&sm.hdr[q].args, &X, (int)(sizeof(TmaArgs<T>) / 4), 0, 1);
    }
    mbar_expect_tx(&sm.full[q], bytes);
    if (MODE == 0) tma_load_2d(&sm.tile[q][0][0], &maps.init, x0, st.lo + l0, &sm.full[q]);
    else tma_load_2d(&sm.tile[q][0][0], &maps.state, x0, cur * X.rows + st.rowoff + l0, &sm.full[q]);
    if (kUseForce) {
      if (FMODE == 1) tma_load_2d(&sm.frc[q][0][0], &maps.force, x0, dir * X.rows + st.rowoff + l0, &sm.full[q]);
      else tma_load_2d(&sm.frc[q][0][0], &maps.force, x0, st.lo + l0, &sm.full[q]);
    }
    tma_load_2d(&sm.rec[q][0][0], &maps.rec, 0, (s * 2 + dir) * X.Lpad + kRecPad + l0, &sm.full[q]);
    ++issued;
  }
  if (!ok) {
    atomicExch(X.flag, 1);
    // drain: wait (bounded) for every stage that still has copies in flight
    for (int c = (issued > SH::NST ? issued - SH::NST : 0); c < issued; ++c) {
      const unsigned g = cbase + (unsigned)c;
      (void)mbar_wait(&sm.full[g % SH::NST], (g / SH::NST) & 1);
    }
    return false;
  }
  return true;
}

// Consumer half of one unit's pass (the kWarpsPerBlock consumer warps).  ST: the
// unit's strip from the stage header, or nullptr to read it from global memory.
template <typename T, bool UP, int MODE, int FMODE, class SH>
__device__ __forceinline__ bool consume_unit(const TmaArgs<T>& X, const int k, const int s, const int bx,
                                             TmaSmem<T, SH>& sm, const unsigned cbase, const StripInfo* st_hdr) {
  const PassArgs<T>& A = X.p;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const StripInfo st = st_hdr ? *st_hdr : A.strips[s];
  const int L = st.L;
  const int NC = (L + SH::CH - 1) / SH::CH;
  auto chunk_l0 = [&](int c) { return UP ? c * SH::CH : L - (c + 1) * SH::CH; };

  // ------------------------------ consumers ------------------------------
  const int wl = warp;
  const int w = bx * kWarpsPerBlock + wl;
  const bool warp_live = w < A.W;
  const int m = w * kOutCols - 1 + lane;
  const int col = m + 1;
  const bool in_dom = (m >= 0) && (m <= A.nx);
  const bool out_lane = warp_live && in_dom && lane >= 1 && lane <= kOutCols;
  const int cls = (m <= 0) ? 0 : (m >= A.nx ? 2 : 1);
  const int inflow_side = (m == 0) ? 0 : (m == A.nx ? 1 : -1);
  const int P = A.P;
  T* __restrict__ Ynext = ((k + 1) & 1) ? A.Y1 : A.Y0;
  const int k1 = k + 1;
  T dtak = T(0);
  if (FMODE == 2 && MODE != 2) dtak = (T)A.dta[(size_t)k1 * A.nforce];

  // rows whose u^k is recorded (overlap and trace stencil), local indices: one window
  // at the bottom interface and one at the top interface (empty windows: lo > hi)
  int rloB = 1, rhiB = 0, rloT = 1, rhiT = 0;
  if (MODE != 0) {
    if (st.has_bot) { rloB = st.alpha_bot - st.lo - 1; rhiB = st.alpha_bot - st.lo + A.ov + 1; }
    if (st.has_top) { rloT = st.alpha_top - st.lo - 1; rhiT = st.alpha_top - st.lo + A.ov + 1; }
  }

  // this strip's incoming interface data, one value per lane, loaded once per pass:
  // at t^{k+1} for the end rows of the system being eliminated, at t^k for the Robin
  // trace without overlap recorded from u^k
  double lam_rhs_top = 0.0, lam_rhs_bot = 0.0, lam_rec_top = 0.0, lam_rec_bot = 0.0;
  if (in_dom) {
    const size_t nxp = (size_t)A.nx + 1, nt = (size_t)A.nt;
    const bool rec_in = MODE != 0 && A.robin && A.ov == 0;
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

  T u_prev = T(0), u_m1 = T(0), u_m2 = T(0), y_prev = T(0);
  const int step = UP ? P : -P;
  // Elimination chain of the previous interior chunk, deferred so that it runs
  // interleaved with the back-substitution chain of the next one: two independent
  // FMA chains keep the FP64 pipe busy.  Its inputs live in registers, so its
  // shared-memory stage is already released.
  bool pend = false;
  T xx[SH::CH], hn[SH::CH];
  T* pout = nullptr;
  auto drain = [&]() {
    T y_last = T(0);
#pragma unroll
    for (int t = 0; t < SH::CH; ++t) {
      if (t > 0 && out_lane) *pout = y_last;
      if (t > 0) pout += step;
      y_prev = fma(hn[t], y_prev, xx[t]);
      y_last = y_prev;
    }
    if (out_lane) *pout = y_last;
    pout += step;
    pend = false;
  };
  for (int c = 0; c < NC; ++c) {
    const unsigned g = cbase + (unsigned)c;
    const int q = (int)(g % SH::NST);
    if (!mbar_wait(&sm.full[q], (g / SH::NST) & 1)) {
      atomicExch(X.flag, 1);
      return false;
    }
    const int l0 = chunk_l0(c);
    const int l1 = l0 + SH::CH - 1;
    const bool rec_chunk = (MODE != 0) && ((rloB <= rhiB && !(l1 < rloB || l0 > rhiB)) ||
                                           (rloT <= rhiT && !(l1 < rloT || l0 > rhiT)));
    // Chunks that reach outside the strip, caller boundary data, and chunks in which
    // the upwind side changes (v changes sign inside) go through the general path.
    // Every other chunk is a run of 16 rows with no per-row branch: its recorded rows
    // are written after the back-substitution chain, and the strip's end rows
    // (interface data) are folded into the chain's first or last term.  A v = 0 row at
    // either end of a chunk has no transport (its upwind coefficient is 0), so it takes
    // the chunk's neighbour lane like the other rows.
    const int sg_first = slot_int(sm.rec[q][0][cls * 8 + 6]);
    const int sg_last = slot_int(sm.rec[q][SH::CH - 1][cls * 8 + 6]);
    const bool general = X.bc_data || l0 < 0 || l1 >= L || sg_first * sg_last < 0;
    if (!general) {
      // upwind neighbour lane for the whole chunk
      const int src = lane - (sg_first != 0 ? sg_first : sg_last);
      const int lf = UP ? l0 : l0 + SH::CH - 1;  // first row in pass order
      const int cbase = wl * kOutCols + lane;
      // (A) back-substitution chain of this chunk, interleaved with the deferred
      //     elimination chain of the previous chunk
      T uu[SH::CH];
      constexpr bool kLateStore = sizeof(T) == 4;  // measured: helps FP32, not FP64
      if (pend && !kLateStore) {
#pragma unroll
        for (int t = 0; t < SH::CH; ++t) {
          const int r = UP ? t : (SH::CH - 1 - t);
          const T tile = sm.tile[q][r][cbase];
          if (MODE == 0) uu[t] = tile;
          else { u_prev = fma(sm.rec[q][r][cls * 8 + 0], u_prev, tile); uu[t] = u_prev; }
          y_prev = fma(hn[t], y_prev, xx[t]);
          if (out_lane) *pout = y_prev;
          pout += step;
        }
        pend = false;
      } else if (pend) {
        // each y is stored one row late, so that no store waits on the FMA just issued
        T y_last = T(0);
#pragma unroll
        for (int t = 0; t < SH::CH; ++t) {
          const int r = UP ? t : (SH::CH - 1 - t);
          const T tile = sm.tile[q][r][cbase];
          if (MODE == 0) uu[t] = tile;
          else { u_prev = fma(sm.rec[q][r][cls * 8 + 0], u_prev, tile); uu[t] = u_prev; }
          if (t > 0 && out_lane) *pout = y_last;
          if (t > 0) pout += step;
          y_prev = fma(hn[t], y_prev, xx[t]);
          y_last = y_prev;
        }
        if (out_lane) *pout = y_last;
        pout += step;
        pend = false;
      } else {
#pragma unroll
        for (int t = 0; t < SH::CH; ++t) {
          const int r = UP ? t : (SH::CH - 1 - t);
          const T tile = sm.tile[q][r][cbase];
          if (MODE == 0) uu[t] = tile;
          else { u_prev = fma(sm.rec[q][r][cls * 8 + 0], u_prev, tile); uu[t] = u_prev; }
        }
      }
      if (MODE != 0) {
        if (rec_chunk) {
#pragma unroll
          for (int t = 0; t < SH::CH; ++t) {
            const int l = UP ? l0 + t : l0 + SH::CH - 1 - t;
            const T um1 = t >= 1 ? uu[t - 1] : u_m1;
            const T um2 = t >= 2 ? uu[t - 2] : (t == 1 ? u_m1 : u_m2);
            if ((l >= rloB && l <= rhiB) || (l >= rloT && l <= rhiT))
              record_row<T, UP>(A, st, s, k, l, m, out_lane, uu[t], um1, um2, lam_rec_top, lam_rec_bot);
          }
        }
        u_m2 = uu[SH::CH - 2];
        u_m1 = uu[SH::CH - 1];
      }
      if (MODE == 2) {
        T* outT = A.UT + (size_t)(st.rowoff + lf) * P + col;
#pragma unroll
        for (int t = 0; t < SH::CH; ++t) {
          if (out_lane) *outT = uu[t];
          outT += step;
        }
      } else {
        // (B) shuffles (all issued before their first use) and the terms that do not
        //     depend on the previous row
        T nb[SH::CH];
        if (kLateStore) {
#pragma unroll
          for (int t = 0; t < SH::CH; ++t) nb[t] = shfl_val(uu[t], src);
        }
#pragma unroll
        for (int t = 0; t < SH::CH; ++t) {
          const int r = UP ? t : (SH::CH - 1 - t);
          const T* rc = &sm.rec[q][r][cls * 8];
          T ncp_unused, ca, cb, chn;
          load_coef4(rc, ncp_unused, ca, cb, chn);
          const T unb = kLateStore ? nb[t] : shfl_val(uu[t], src);
          T gterm;
          if (FMODE == 0) gterm = T(0);
          else if (FMODE == 1) gterm = sm.frc[q][r][cbase];
          else gterm = (rc[4] * dtak) * sm.frc[q][r][cbase];
          xx[t] = fma(ca, uu[t], fma(cb, unb, gterm));
          hn[t] = chn;
        }
        // the strip's first and last rows in pass order carry the interface data
        // (Dirichlet: the value itself; Robin: g 2dt/hv lambda on top of the regular
        // right-hand side); v-boundary and x-inflow rows without caller data are zero
        // rows already
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          if (e == 0 ? c != 0 : c != NC - 1) continue;
          const int te = e == 0 ? 0 : SH::CH - 1;
          const int re = UP ? te : (SH::CH - 1 - te);
          const int kind = slot_int(sm.rec[q][re][cls * 8 + 7]);
          if (kind >= 3) {
            const double lam = (kind == 3 || kind == 5) ? lam_rhs_top : lam_rhs_bot;
            xx[te] = kind <= 4 ? (T)lam : (T)((double)xx[te] + (double)sm.rec[q][re][cls * 8 + 5] * lam);
          }
        }
        pout = Ynext + (size_t)(st.rowoff + lf) * P + col;
        pend = true;
      }
    } else {
      if (pend) drain();
#pragma unroll 1
      for (int t = 0; t < SH::CH; ++t) {
        const int r = UP ? t : (SH::CH - 1 - t);
        const int l = l0 + r;
        if (l < 0 || l >= L) continue;  // rows outside the strip (uniform)
        const T* rc = &sm.rec[q][r][cls * 8];
        T u;
        if (MODE == 0) {
          u = sm.tile[q][r][wl * kOutCols + lane];
        } else {
          u = fma(rc[0], u_prev, sm.tile[q][r][wl * kOutCols + lane]);
          u_prev = u;
          if (rec_chunk) record_row<T, UP>(A, st, s, k, l, m, out_lane, u, u_m1, u_m2, lam_rec_top, lam_rec_bot);
          u_m2 = u_m1;
          u_m1 = u;
          if (MODE == 2) {
            if (out_lane) A.UT[(size_t)(st.rowoff + l) * P + col] = u;
            continue;
          }
        }
        const T unb = shfl_val(u, lane - slot_int(rc[6]));
        T gterm = T(0);
        if (FMODE == 1) gterm = sm.frc[q][r][wl * kOutCols + lane];
        if (FMODE == 2) gterm = (rc[4] * dtak) * sm.frc[q][r][wl * kOutCols + lane];
        T y = fma(rc[3], y_prev, fma(rc[1], u, fma(rc[2], unb, gterm)));
        const int kind = slot_int(rc[7]);
        if (kind != 0)
          y = special_row<T>(A, kind, k1, st.lo + l, m, in_dom, inflow_side, y, rc[5], lam_rhs_top, lam_rhs_bot);
        if (out_lane) Ynext[(size_t)(st.rowoff + l) * P + col] = y;
        y_prev = y;
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&sm.empty[q]);
  }
  if (pend) drain();
  return true;
}

// One work unit: strip s, column block bx (4 warps = 120 output columns) of one
// problem, for pass k.  Ring slots continue from chunk number cbase (so a block can
// run several units back to back).  Returns false if a bounded wait expired.
template <typename T, bool UP, int MODE, int FMODE, class SH>
__device__ __forceinline__ bool pass_unit(const TmaMaps& maps, const TmaArgs<T>& X, const int k, const int s,
                                          const int bx, TmaSmem<T, SH>& sm, const unsigned cbase) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == kWarpsPerBlock) {
    if (lane != 0) return true;
    const StripInfo st = X.p.strips[s];
    return produce_unit<T, UP, MODE, FMODE, SH>(maps, X, k, s, bx, st, sm, cbase, nullptr);
  }
  return consume_unit<T, UP, MODE, FMODE, SH>(X, k, s, bx, sm, cbase, nullptr);
}

// The dynamic shared-memory base is at least 16-byte aligned, which is what an
// unswizzled TMA destination needs; using it directly (no integer round trip) keeps
// every tile access a shared-memory load.
template <typename T, bool UP, int MODE, int FMODE, class SH>
__global__ void __launch_bounds__((kWarpsPerBlock + 1) * 32, SH::MINB)
sweep_pass_tma_kernel(const __grid_constant__ TmaMaps maps, const TmaArgs<T> X, const int k) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  TmaSmem<T, SH>& sm = *reinterpret_cast<TmaSmem<T, SH>*>(smem_raw);
  init_ring(sm);
  (void)pass_unit<T, UP, MODE, FMODE, SH>(maps, X, k, blockIdx.y + X.p.strip0, blockIdx.x, sm, 0u);
}

// ---------------------------------------------------------------------------
// Streamed form: the interior passes of an iteration in one persistent launch.
// ---------------------------------------------------------------------------
//
// The interior passes (1 <= k < nt: back-substitution of step k fused with the
// elimination of step k+1) of one or many problems are a list of tickets in pass
// order: ticket t is unit t - pass_start[j] of pass k = 1 + j, where the units
// (problem, strip s, column block bx) active in pass j are a prefix of the unit list
// (problems sorted by decreasing nt).  A co-resident grid (cooperative launch)
// draws tickets from one counter; each block's producer lane takes a ticket, waits
// until the unit and its two column neighbours have finished the previous pass,
// writes the unit's header into the stage of its first chunk and streams its
// chunks; the consumer warps follow the stream of stages, reading each unit from
// its header.  Pass k of a unit reads the residue of its own columns and of one
// halo column on each side, written by the unit and its neighbours in pass k-1,
// and overwrites the buffer they read in pass k-1; the wait covers both, and keeps
// neighbours within one pass of each other, which the two residue buffers allow.
// Tickets are taken in pass order, so every ticket a block waits on is held by a
// running block: no cycle of waits.  The blocks' rings stay full across unit and
// pass boundaries, so a unit's start-up latency hides behind the previous unit.
//
// Pipelined iterates.  Consecutive SWR iterates of one problem can run in the same
// launch as a wavefront over (iterate, time step): iterate d of a group reads, in
// pass k, the interface data at t^k and t^(k+1) that iterate d-1 records in passes k
// and k+1 (Section 6.3: each strip's data come from its neighbours' previous
// iterate, time level by time level).  Its unit of slot j runs pass k = j + depth -
// 2d, so a unit depends only on units of slot j-1: its own strip's (iterate d, pass
// k-1) and the neighbour strips' (iterate d-1, pass k+1).  The units active in a slot
// are a contiguous range of the list (iterate-major), and the arithmetic of every
// iterate is that of a lone iteration, so the results are the same bits.
//
// Completion of a unit's pass is a per-unit counter to which every consumer warp
// adds one after its stores and a proxy fence (no barrier inside the block, so a
// warp that leaves on an error cannot strand the others).  Every counter wait is
// bounded by wall time (globaltimer); on expiry, or when another block has raised
// the error flag, the producer marks the ring aborted and completes the next stage
// without data, so that the consumers leave as well.

struct StreamUnit {
  int inst, strip, bx, nc;  // problem, strip, column block, 16-row chunks of the strip (work)
  int left, right;          // list indices of the column neighbours (-1: none)
  int dep_lo, dep_hi;       // pipelined iterates: the previous iterate's units of strips s-1
                            // and s+1, same column block (-1: none)
};

template <typename T>
struct StreamProblem {
  TmaMaps maps;    // 64-byte aligned tensor maps of this problem (global memory), 16-row boxes
  TmaMaps maps8;   // the same with 8-row boxes
  TmaArgs<T> args;
  int nt, fmode;
  int lag;         // pipelined iterates: position d of this iterate in its group (0 otherwise)
};

template <class SH, typename T>
__device__ __forceinline__ const TmaMaps& maps_for(const StreamProblem<T>& pr) {
  return SH::CH == 8 ? pr.maps8 : pr.maps;
}

struct StreamArgs {
  const StreamUnit* units;       // sorted by decreasing nt of their problem
  const int* pass_start;         // [npass + 1] first ticket of each interior pass
  const int* unit_first;         // [npass] list index of the first unit of each pass (NULL: 0)
  int npass;                     // interior passes of the longest problem (max nt - 1)
  int depth;                     // iterates per pipelined group (1: none); the unit of iterate
                                 // d in slot j runs pass k = j + depth - 2 d
  int dynamic;                   // 1: tickets from the counter; 0: block b runs unit b of every
                                 // pass (the grid holds the largest pass)
  unsigned* done;                // [units] consumer warps x passes completed (zeroed before)
  unsigned* ticket;              // next ticket (zeroed before)
  int* flag;                     // error flag (1 = a bounded wait expired)
  int stall_unit;                // self-test: this unit never reports completion (-1: none)
  unsigned long long wait_ns;    // limit of one counter wait
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add_u32(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Order this thread's generic-proxy global accesses with later async-proxy (TMA)
// accesses, and the other way round.
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Bounded wait until done[a], done[b], done[c] (b, c may be -1) all reach target.
// False on time-out (the error flag is raised) or when the error flag is already set.
__device__ __forceinline__ bool wait_done(const StreamArgs& P, int a, int b, int c, unsigned target) {
  const unsigned long long t0 = global_ns();
  for (unsigned it = 0;; ++it) {
    bool ok = ld_acquire_u32(P.done + a) >= target;
    if (b >= 0) ok = ok && ld_acquire_u32(P.done + b) >= target;
    if (c >= 0) ok = ok && ld_acquire_u32(P.done + c) >= target;
    if (ok) return true;
    if ((it & 15) == 15) {
      if (*(volatile const int*)P.flag) return false;
      if (global_ns() - t0 > P.wait_ns) {
        atomicExch(P.flag, 1);
        return false;
      }
    }
  }
}

template <typename T, int FMODE, class SH>
__global__ void __launch_bounds__((kWarpsPerBlock + 1) * 32, SH::MINB)
sweep_stream_kernel(const StreamProblem<T>* __restrict__ probs, const StreamArgs P) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  TmaSmem<T, SH>& sm = *reinterpret_cast<TmaSmem<T, SH>*>(smem_raw);
  init_ring(sm);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned cbase = 0;
  if (warp == kWarpsPerBlock) {
    // ------------------------------ producer ------------------------------
    if (lane != 0) return;
    const unsigned total = (unsigned)P.pass_start[P.npass];
    // next ticket: from the counter, or (static) unit blockIdx.x of the next pass
    int j = 0, sj = -1;
    auto next_ticket = [&]() -> unsigned {
      if (P.dynamic) return atomicAdd(P.ticket, 1u);
      // the next pass that has a unit for this block (pass sizes grow at the start
      // of a pipelined group and shrink at its end)
      for (++sj; sj < P.npass; ++sj) {
        const unsigned t = (unsigned)P.pass_start[sj] + blockIdx.x;
        if (t < (unsigned)P.pass_start[sj + 1]) return t;
      }
      return total;
    };
    unsigned t = next_ticket();
    int last_inst = -1;
    for (;;) {
      StreamTail h;
      bool ok = true;
      if (t >= total) {
        h.k = -1;  // no more work
      } else {
        while ((unsigned)P.pass_start[j + 1] <= t) ++j;
        const int u = (P.unit_first ? P.unit_first[j] : 0) + (int)(t - (unsigned)P.pass_start[j]);
        const StreamUnit un = P.units[u];
        const int lag = probs[un.inst].lag;
        h.k = j + P.depth - 2 * lag;
        h.inst = un.inst;
        h.strip = un.strip;
        h.bx = un.bx;
        h.unit = u;
        h.new_args = un.inst != last_inst;
        last_inst = un.inst;
        const StreamProblem<T>& pr = probs[un.inst];
        h.st = pr.args.p.strips[un.strip];
        h.nc = (h.st.L + SH::CH - 1) / SH::CH;
        // passes of this unit in the launch before this one (a pipelined iterate d
        // starts in slot d; the passes before its first one ran before the launch)
        const int jr = j - lag;
        if (jr > 0) ok = wait_done(P, u, un.left, un.right, (unsigned)(jr * kWarpsPerBlock));
        // the previous iterate's neighbour strips have finished pass k + 1
        if (ok && (un.dep_lo >= 0 || un.dep_hi >= 0))
          ok = wait_done(P, un.dep_lo >= 0 ? un.dep_lo : un.dep_hi, un.dep_lo >= 0 ? un.dep_hi : -1, -1,
                         (unsigned)((jr + 1) * kWarpsPerBlock));
        if (ok) {
          fence_proxy_async_global();
          const TmaMaps& mp = maps_for<SH>(pr);
          ok = (h.k & 1) ? produce_unit<T, false, 1, FMODE, SH>(mp, pr.args, h.k, h.strip, h.bx, h.st, sm, cbase, &h)
                         : produce_unit<T, true, 1, FMODE, SH>(mp, pr.args, h.k, h.strip, h.bx, h.st, sm, cbase, &h);
          if (!ok) return;  // a ring wait expired; the consumers time out on their own
          cbase += (unsigned)h.nc;
          // the next ticket only now: a block that held two would sit on the second
          // (possibly a pass ahead) while others run short of work
          t = next_ticket();
          continue;
        }
      }
      // no more work, or a counter wait gave up: complete the next stage without
      // data (after the consumers released it) so that the consumers leave
      if (!ok) sm.abort = 1;
      const int q = (int)(cbase % SH::NST);
      const unsigned use = cbase / SH::NST;
      if (use == 0 || mbar_wait(&sm.empty[q], (use - 1) & 1)) {
        sm.hdr[q].tail.k = -1;
        mbar_arrive(&sm.full[q]);
      }
      return;
    }
  }
  // ------------------------------ consumers ------------------------------
  for (;;) {
    const int q = (int)(cbase % SH::NST);
    if (!mbar_wait(&sm.full[q], (cbase / SH::NST) & 1)) {
      atomicExch(P.flag, 1);
      return;
    }
    // the producer gives up only before a unit (then this stage holds no data), so
    // this is the one place the consumers look at the abort word
    if (*(volatile int*)&sm.abort) return;
    if (sm.hdr[q].tail.k < 0) return;
    // copy the header while the stage is held (its first chunk is not released yet);
    // the pass arguments only when the problem changed (units come in the same order
    // to every consumer warp, so the warp's copy holds the producer's last ones)
    StreamHeader<T>& h = sm.cur[warp];
    if (sm.hdr[q].tail.new_args) copy_words(&h.args, &sm.hdr[q].args, (int)(sizeof(TmaArgs<T>) / 4), lane, 32);
    copy_words(&h.tail, &sm.hdr[q].tail, (int)(sizeof(StreamTail) / 4), lane, 32);
    __syncwarp();
    const int k = h.tail.k, s = h.tail.strip, bx = h.tail.bx, nc = h.tail.nc, u = h.tail.unit;
    const bool ok = (k & 1) ? consume_unit<T, false, 1, FMODE, SH>(h.args, k, s, bx, sm, cbase, &h.tail.st)
                            : consume_unit<T, true, 1, FMODE, SH>(h.args, k, s, bx, sm, cbase, &h.tail.st);
    if (!ok) return;
    // this warp's stores of the pass are visible (to loads and to TMA) before the
    // unit's counter moves
    __threadfence();
    fence_proxy_async_global();
    __syncwarp();
    if (lane == 0 && u != P.stall_unit) red_release_add_u32(P.done + u, 1u);
    cbase += (unsigned)nc;
  }
}

// ---------------------------------------------------------------------------
// First and last passes of many units (one or many problems) in one launch.
// ---------------------------------------------------------------------------

// MODE 0: pass 0 (elimination of step 1 from u^0) of every listed unit; MODE 2: the
// last pass (back-substitution of step nt, u^nt stored) of every listed unit, each
// at its own problem's nt.  Units u = blockIdx.x, blockIdx.x + gridDim.x, ...: one
// block per unit when the grid is as large as the list, persistent blocks otherwise.
template <typename T, int MODE, int FMODE, class SH>
__global__ void __launch_bounds__((kWarpsPerBlock + 1) * 32, SH::MINB)
edge_pass_kernel(const StreamProblem<T>* __restrict__ probs, const StreamUnit* __restrict__ units, const int nunits) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  TmaSmem<T, SH>& sm = *reinterpret_cast<TmaSmem<T, SH>*>(smem_raw);
  init_ring(sm);
  unsigned cbase = 0;
  for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
    const StreamUnit un = units[u];
    const StreamProblem<T>& pr = probs[un.inst];
    const int k = MODE == 0 ? 0 : pr.nt;
    const TmaMaps& mp = maps_for<SH>(pr);
    bool ok;
    if (MODE == 0 || !(k & 1)) ok = pass_unit<T, true, MODE, FMODE, SH>(mp, pr.args, k, un.strip, un.bx, sm, cbase);
    else ok = pass_unit<T, false, MODE, FMODE, SH>(mp, pr.args, k, un.strip, un.bx, sm, cbase);
    if (!ok) return;
    cbase += (unsigned)((pr.args.p.strips[un.strip].L + SH::CH - 1) / SH::CH);
  }
}

}  // namespace kfp
