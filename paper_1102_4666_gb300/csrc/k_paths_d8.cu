// k_paths_d8.cu -- instantiation of the path kernel for d = 8 assets, FP32 (mixed precision) paths.
#include "k_paths.cuh"
BSDE_PATHS_INSTANTIATE(8, float, f32)
