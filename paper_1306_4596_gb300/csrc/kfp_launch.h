// kfp_launch.h -- host entry points of the TMA-fed sweep kernels, per precision and
// tile shape.
//
// The kernels of kfp_sweep_tma.cuh, kfp_slot.cuh and kfp_fe_tma.cuh are instantiated,
// one (precision, shape) pair per translation unit (kfp_launch_<precision>_s<shape>.cu),
// so that they compile in parallel; host code calls them only through
// LaunchSet<T, SHAPE> and the runtime choice of shape in kfp_swr.cu (Tma<T>).  Shapes
// (rows per ring stage CH, ring stages NST, blocks per SM):
//   0: CH 16, NST 4 (FP64) / 8 (FP32), 1 block per SM  -- about one unit per SM
//   1: CH  8, NST 4 (FP64) / 8 (FP32), 2 blocks per SM -- several units per SM
//   2: CH  8, NST 6 (FP64) / 12 (FP32), 2 blocks per SM -- the same, deeper ring
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "kfp_fe_tma.cuh"
#include "kfp_slot.cuh"
#include "kfp_sweep_tma.cuh"

namespace kfp {

constexpr int kShapes = 3;

template <typename T, int SHAPE>
struct ShapeOf;
template <typename T>
struct ShapeOf<T, 0> {
  using type = Shape<16, sizeof(T) == 8 ? 4 : 8, 1>;
};
template <typename T>
struct ShapeOf<T, 1> {
  using type = Shape<8, sizeof(T) == 8 ? 4 : 8, 2>;
};
template <typename T>
struct ShapeOf<T, 2> {
  using type = Shape<8, sizeof(T) == 8 ? 6 : 12, 2>;
};

template <typename T, int SHAPE>
struct LaunchSet {
  // dynamic shared memory of every kernel of this shape (bytes)
  static size_t smem_bytes();
  // raise the dynamic shared-memory limit of every kernel of this shape
  static cudaError_t set_attrs();
  // blocks of the streamed kernel (forcing mode fmode) resident on one SM (0 if none)
  static int blocks_per_sm(int fmode);
  // one sweep pass of all (or, serial form, one strip's) units: pass k, direction UP,
  // MODE 0 (first pass), 1 (interior) or 2 (last pass)
  static void pass(int fmode, bool up, int mode, dim3 grid, cudaStream_t st, const TmaMaps& maps,
                   const TmaArgs<T>& X, int k);
  // the interior passes of one or many problems in one cooperative launch
  static cudaError_t stream(int fmode, unsigned grid, cudaStream_t st, const StreamProblem<T>* probs,
                            const StreamArgs& P);
  // the first (mode 0) or last (mode 2) pass of every listed unit
  static void edge(int mode, int fmode, unsigned grid, cudaStream_t st, const StreamProblem<T>* probs,
                   const StreamUnit* units, int n);
  // one slot of pipelined iterates (grid.z = iterates of the slot, all in pass kind
  // MODE and direction UP), the sweep or the split P1 scheme of Section 6.2
  // (kfp_fe_tma.cuh; its passes always run here, one iterate at a time as a slot of one)
  static void slot(int fmode, bool up, int mode, dim3 grid, cudaStream_t st, const SlotArgs<T>& G);
  static void fe_slot(int fmode, bool up, int mode, dim3 grid, cudaStream_t st, const FeSlotArgs<T>& G);
};

// Rows per ring stage of a shape.
inline int shape_rows(int shape) { return shape == 0 ? 16 : 8; }

}  // namespace kfp
