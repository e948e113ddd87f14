"""GB300-native (sm_103a) Schwarz waveform relaxation for the Kolmogorov equation.

u_t + v u_x - u_vv = f is solved on a box split into v-strips; each iteration
solves every strip over the whole time window from the previous iterate's
interface data (Dirichlet or Robin transmission) and exchanges the new data
(Gerardo-Giorda & Tran, arXiv:1306.4596, Sections 2 and 6.3).

Layout:
  include/kfp_swr.h         the C ABI (repository root)
  csrc/kfp_kernels.cuh      sweep / exchange / error kernels
  csrc/kfp_swr.cu           host driver and the C entry points
  build.py                  nvcc build of _build/libkfp_swr.so
  swr.py                    ctypes binding with the C names, plus the ``SWR`` wrapper
  inputs.py                 seeded synthetic problems (data only)
"""
from . import inputs  # noqa: F401

__all__ = ["inputs", "swr", "build"]
