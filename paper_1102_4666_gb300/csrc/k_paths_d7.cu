// k_paths_d7.cu -- instantiation of the path kernel for d = 7 assets, FP32 (mixed precision) paths.
#include "k_paths.cuh"
BSDE_PATHS_INSTANTIATE(7, float, f32)
