// k_paths_d4_f64.cu -- instantiation of the path kernel for d = 4 assets, FP64 paths.
#include "k_paths.cuh"
BSDE_PATHS_INSTANTIATE(4, double, f64)
