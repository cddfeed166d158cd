// k_paths_d2_f64.cu -- instantiation of the path kernel for d = 2 assets, FP64 paths.
#include "k_paths.cuh"
BSDE_PATHS_INSTANTIATE(2, double, f64)
