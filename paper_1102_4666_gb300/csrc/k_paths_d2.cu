// k_paths_d2.cu -- instantiation of the path kernel for d = 2 assets, FP32 (mixed precision) paths.
#include "k_paths.cuh"
BSDE_PATHS_INSTANTIATE(2, float, f32)
