// k_paths_d5.cu -- instantiation of the path kernel for d = 5 assets, FP32 (mixed precision) paths.
#include "k_paths.cuh"
BSDE_PATHS_INSTANTIATE(5, float, f32)
