// k_paths_d10.cu -- instantiation of the path kernel for d = 10 assets, FP32 (mixed precision) paths.
#include "k_paths.cuh"
BSDE_PATHS_INSTANTIATE(10, float, f32)
