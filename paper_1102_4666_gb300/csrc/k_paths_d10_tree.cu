// k_paths_d10_tree.cu -- prefix-tree (dense, degree 4..6) evaluation kernels of the path kernel
// for d = 10 assets.
#include "k_paths.cuh"
BSDE_PATHS_INSTANTIATE_TREE(10)
