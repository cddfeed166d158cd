// k_paths_d3.cu -- instantiation of the path kernel for d = 3 assets, FP32 (mixed precision) paths.
#include "k_paths.cuh"
BSDE_PATHS_INSTANTIATE(3, float, f32)
