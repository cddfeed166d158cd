// k_paths_d1.cu -- instantiation of the path kernel for d = 1 asset, FP32 (mixed precision) paths.
#include "k_paths.cuh"
BSDE_PATHS_INSTANTIATE(1, float, f32)
