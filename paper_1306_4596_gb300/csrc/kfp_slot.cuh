// kfp_slot.cuh -- one launch per slot of pipelined iterates for the TMA-fed sweep
// (sm_103a): the forms that cannot stream their passes (periodic x).
#pragma once
#include "kfp_sweep_tma.cuh"

namespace kfp {

// ---------------------------------------------------------------------------
// Pipelined iterates in one launch per slot (the forms whose passes need a step
// between them, such as the periodic column wrap, and cannot stream): the slot's
// launch runs pass k[z] of the z-th iterate of the slot, z = blockIdx.z, each with
// its own tensor maps and pass arguments.  The iterates of one launch do not depend
// on one another (see the streamed form below for the wavefront).
// ---------------------------------------------------------------------------

constexpr int kSlotMax = 4;
template <typename T>
struct SlotArgs {
  TmaMaps maps[kSlotMax];
  TmaArgs<T> X[kSlotMax];
  int k[kSlotMax];
};

template <typename T, bool UP, int MODE, int FMODE, class SH>
__global__ void __launch_bounds__((kWarpsPerBlock + 1) * 32, SH::MINB)
sweep_slot_kernel(const __grid_constant__ SlotArgs<T> G) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  TmaSmem<T, SH>& sm = *reinterpret_cast<TmaSmem<T, SH>*>(smem_raw);
  init_ring(sm);
  const int z = blockIdx.z;
  (void)pass_unit<T, UP, MODE, FMODE, SH>(G.maps[z], G.X[z], G.k[z], blockIdx.y + G.X[z].p.strip0, blockIdx.x, sm,
                                          0u);
}

}  // namespace kfp
