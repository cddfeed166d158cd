// k_paths_d9_f64.cu -- instantiation of the path kernel for d = 9 assets, FP64 paths.
#include "k_paths.cuh"
BSDE_PATHS_INSTANTIATE(9, double, f64)
