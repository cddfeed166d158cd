// k_paths_d1_f64.cu -- instantiation of the path kernel for d = 1 asset, FP64 paths.
#include "k_paths.cuh"
BSDE_PATHS_INSTANTIATE(1, double, f64)
