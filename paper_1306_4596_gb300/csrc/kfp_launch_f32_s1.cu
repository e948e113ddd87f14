// Sweep kernels of one precision and tile shape (see kfp_launch.h): float, shape 1.
#include "kfp_launch.cuh"

KFP_INSTANTIATE_LAUNCH(float, 1)
