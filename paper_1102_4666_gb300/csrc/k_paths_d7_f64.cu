// k_paths_d7_f64.cu -- instantiation of the path kernel for d = 7 assets, FP64 paths.
#include "k_paths.cuh"
BSDE_PATHS_INSTANTIATE(7, double, f64)
