// kfp_launch.cuh -- definitions of LaunchSet<T, SHAPE> (kfp_launch.h); included only
// by the translation units that instantiate one (precision, shape) pair each.
#pragma once
#include "kfp_launch.h"

namespace kfp {

template <typename T, int SHAPE>
size_t LaunchSet<T, SHAPE>::smem_bytes() {
  return sizeof(TmaSmem<T, typename ShapeOf<T, SHAPE>::type>) + 128;
}

template <typename T, int SHAPE>
cudaError_t LaunchSet<T, SHAPE>::set_attrs() {
  using SH = typename ShapeOf<T, SHAPE>::type;
  const int sm = (int)smem_bytes();
  cudaError_t e = cudaSuccess;
  auto set = [&](const void* fn) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  };
#define KFP_SET_FM(FM)                                                    \
  set((const void*)sweep_pass_tma_kernel<T, true, 0, FM, SH>);            \
  set((const void*)sweep_pass_tma_kernel<T, true, 1, FM, SH>);            \
  set((const void*)sweep_pass_tma_kernel<T, false, 1, FM, SH>);           \
  set((const void*)sweep_stream_kernel<T, FM, SH>);                       \
  set((const void*)edge_pass_kernel<T, 0, FM, SH>);
  KFP_SET_FM(0)
  KFP_SET_FM(1)
  KFP_SET_FM(2)
#undef KFP_SET_FM
  set((const void*)sweep_pass_tma_kernel<T, true, 2, 0, SH>);
  set((const void*)sweep_pass_tma_kernel<T, false, 2, 0, SH>);
  set((const void*)edge_pass_kernel<T, 2, 0, SH>);
#define KFP_SET_SLOT(FM)                                                  \
  set((const void*)sweep_slot_kernel<T, true, 0, FM, SH>);                \
  set((const void*)sweep_slot_kernel<T, true, 1, FM, SH>);                \
  set((const void*)sweep_slot_kernel<T, false, 1, FM, SH>);               \
  set((const void*)fe_slot_kernel<T, true, 0, FM, SH>);                   \
  set((const void*)fe_slot_kernel<T, true, 1, FM, SH>);                   \
  set((const void*)fe_slot_kernel<T, false, 1, FM, SH>);
  KFP_SET_SLOT(0)
  KFP_SET_SLOT(1)
  KFP_SET_SLOT(2)
#undef KFP_SET_SLOT
  set((const void*)sweep_slot_kernel<T, true, 2, 0, SH>);
  set((const void*)sweep_slot_kernel<T, false, 2, 0, SH>);
  set((const void*)fe_slot_kernel<T, true, 2, 0, SH>);
  set((const void*)fe_slot_kernel<T, false, 2, 0, SH>);
  return e;
}

template <typename T, int SHAPE>
void LaunchSet<T, SHAPE>::slot(int fmode, bool up, int mode, dim3 grid, cudaStream_t st, const SlotArgs<T>& G) {
  using SH = typename ShapeOf<T, SHAPE>::type;
  const dim3 block((kWarpsPerBlock + 1) * 32);
  const size_t sm = smem_bytes();
#define KFP_SLOT(UP, MODE, FM) sweep_slot_kernel<T, UP, MODE, FM, SH><<<grid, block, sm, st>>>(G)
  if (mode == 2) {
    if (up) KFP_SLOT(true, 2, 0);
    else KFP_SLOT(false, 2, 0);
  } else if (mode == 0) {
    if (fmode == 0) KFP_SLOT(true, 0, 0);
    else if (fmode == 1) KFP_SLOT(true, 0, 1);
    else KFP_SLOT(true, 0, 2);
  } else if (up) {
    if (fmode == 0) KFP_SLOT(true, 1, 0);
    else if (fmode == 1) KFP_SLOT(true, 1, 1);
    else KFP_SLOT(true, 1, 2);
  } else {
    if (fmode == 0) KFP_SLOT(false, 1, 0);
    else if (fmode == 1) KFP_SLOT(false, 1, 1);
    else KFP_SLOT(false, 1, 2);
  }
#undef KFP_SLOT
}

template <typename T, int SHAPE>
void LaunchSet<T, SHAPE>::fe_slot(int fmode, bool up, int mode, dim3 grid, cudaStream_t st,
                                  const FeSlotArgs<T>& G) {
  using SH = typename ShapeOf<T, SHAPE>::type;
  const dim3 block((kWarpsPerBlock + 1) * 32);
  const size_t sm = smem_bytes();
#define KFP_FESLOT(UP, MODE, FM) fe_slot_kernel<T, UP, MODE, FM, SH><<<grid, block, sm, st>>>(G)
  if (mode == 2) {
    if (up) KFP_FESLOT(true, 2, 0);
    else KFP_FESLOT(false, 2, 0);
  } else if (mode == 0) {
    if (fmode == 0) KFP_FESLOT(true, 0, 0);
    else if (fmode == 1) KFP_FESLOT(true, 0, 1);
    else KFP_FESLOT(true, 0, 2);
  } else if (up) {
    if (fmode == 0) KFP_FESLOT(true, 1, 0);
    else if (fmode == 1) KFP_FESLOT(true, 1, 1);
    else KFP_FESLOT(true, 1, 2);
  } else {
    if (fmode == 0) KFP_FESLOT(false, 1, 0);
    else if (fmode == 1) KFP_FESLOT(false, 1, 1);
    else KFP_FESLOT(false, 1, 2);
  }
#undef KFP_FESLOT
}

template <typename T, int SHAPE>
int LaunchSet<T, SHAPE>::blocks_per_sm(int fmode) {
  using SH = typename ShapeOf<T, SHAPE>::type;
  int n = 0;
  const void* fn = fmode == 0 ? (const void*)sweep_stream_kernel<T, 0, SH>
                              : (fmode == 1 ? (const void*)sweep_stream_kernel<T, 1, SH>
                                            : (const void*)sweep_stream_kernel<T, 2, SH>);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, (kWarpsPerBlock + 1) * 32, smem_bytes()) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

template <typename T, int SHAPE>
void LaunchSet<T, SHAPE>::pass(int fmode, bool up, int mode, dim3 grid, cudaStream_t st, const TmaMaps& maps,
                               const TmaArgs<T>& X, int k) {
  using SH = typename ShapeOf<T, SHAPE>::type;
  const dim3 block((kWarpsPerBlock + 1) * 32);
  const size_t sm = smem_bytes();
  // the last pass reads no forcing, so it has one instantiation per direction
#define KFP_PASS(UP, MODE, FM) sweep_pass_tma_kernel<T, UP, MODE, FM, SH><<<grid, block, sm, st>>>(maps, X, k)
  if (mode == 2) {
    if (up) KFP_PASS(true, 2, 0);
    else KFP_PASS(false, 2, 0);
    return;
  }
  if (mode == 0) {
    if (fmode == 0) KFP_PASS(true, 0, 0);
    else if (fmode == 1) KFP_PASS(true, 0, 1);
    else KFP_PASS(true, 0, 2);
    return;
  }
  if (up) {
    if (fmode == 0) KFP_PASS(true, 1, 0);
    else if (fmode == 1) KFP_PASS(true, 1, 1);
    else KFP_PASS(true, 1, 2);
  } else {
    if (fmode == 0) KFP_PASS(false, 1, 0);
    else if (fmode == 1) KFP_PASS(false, 1, 1);
    else KFP_PASS(false, 1, 2);
  }
#undef KFP_PASS
}

template <typename T, int SHAPE>
cudaError_t LaunchSet<T, SHAPE>::stream(int fmode, unsigned grid, cudaStream_t st, const StreamProblem<T>* probs,
                                        const StreamArgs& P) {
  using SH = typename ShapeOf<T, SHAPE>::type;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3((kWarpsPerBlock + 1) * 32);
  cfg.dynamicSmemBytes = smem_bytes();
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // every block resident: they wait on one another
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (fmode == 0) return cudaLaunchKernelEx(&cfg, sweep_stream_kernel<T, 0, SH>, probs, P);
  if (fmode == 1) return cudaLaunchKernelEx(&cfg, sweep_stream_kernel<T, 1, SH>, probs, P);
  return cudaLaunchKernelEx(&cfg, sweep_stream_kernel<T, 2, SH>, probs, P);
}

template <typename T, int SHAPE>
void LaunchSet<T, SHAPE>::edge(int mode, int fmode, unsigned grid, cudaStream_t st, const StreamProblem<T>* probs,
                               const StreamUnit* units, int n) {
  using SH = typename ShapeOf<T, SHAPE>::type;
  const dim3 block((kWarpsPerBlock + 1) * 32);
  const size_t sm = smem_bytes();
  if (mode == 2) edge_pass_kernel<T, 2, 0, SH><<<grid, block, sm, st>>>(probs, units, n);
  else if (fmode == 0) edge_pass_kernel<T, 0, 0, SH><<<grid, block, sm, st>>>(probs, units, n);
  else if (fmode == 1) edge_pass_kernel<T, 0, 1, SH><<<grid, block, sm, st>>>(probs, units, n);
  else edge_pass_kernel<T, 0, 2, SH><<<grid, block, sm, st>>>(probs, units, n);
}

}  // namespace kfp

#define KFP_INSTANTIATE_LAUNCH(T, SHAPE) template struct kfp::LaunchSet<T, SHAPE>;
