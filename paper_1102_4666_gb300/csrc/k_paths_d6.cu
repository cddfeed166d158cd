// k_paths_d6.cu -- instantiation of the path kernel for d = 6 assets, FP32 (mixed precision) paths.
#include "k_paths.cuh"
BSDE_PATHS_INSTANTIATE(6, float, f32)
