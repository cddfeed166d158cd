// k_paths_d4.cu -- instantiation of the path kernel for d = 4 assets, FP32 (mixed precision) paths.
#include "k_paths.cuh"
BSDE_PATHS_INSTANTIATE(4, float, f32)
