// k_paths_d5_f64.cu -- instantiation of the path kernel for d = 5 assets, FP64 paths.
#include "k_paths.cuh"
BSDE_PATHS_INSTANTIATE(5, double, f64)
