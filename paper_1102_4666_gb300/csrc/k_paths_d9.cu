// k_paths_d9.cu -- instantiation of the path kernel for d = 9 assets, FP32 (mixed precision) paths.
#include "k_paths.cuh"
BSDE_PATHS_INSTANTIATE(9, float, f32)
