// k_paths_dispatch.cu -- choose the compiled path kernel for the number of
// assets d (the per-asset state is held in registers, so d is a template
// parameter of the kernel).
#include "k_paths.cuh"

#define DECL(DV)                                                                            \
  cudaError_t launch_paths_d##DV(const ModelHost&, const GridHost&, const ProblemDev&, int, \
                                 int, uint32_t, bool, int, int, cudaStream_t);
DECL(1) DECL(2) DECL(3) DECL(4) DECL(5) DECL(6) DECL(7) DECL(8) DECL(9) DECL(10)
#undef DECL

int paths_supported_d(int d) { return d >= 1 && d <= 10; }

size_t paths_smem_bytes(int d, int p, int eta, int N, int tpb, bool mixed, bool dense) {
  // the tanh families tabulate two coefficients per asset and step
  return paths::smem_bytes(d, p, eta < 1 ? 1 : eta, N, tpb, mixed ? sizeof(float) : sizeof(double),
                           dense, 2 * (d < 3 ? 3 : d));
}

cudaError_t launch_paths(const ModelHost& m, const GridHost& g, const ProblemDev& P, int M, int N,
                         uint32_t k, bool mixed, int tpb, int ppt, cudaStream_t st) {
  switch (m.d) {
    case 1: return launch_paths_d1(m, g, P, M, N, k, mixed, tpb, ppt, st);
    case 2: return launch_paths_d2(m, g, P, M, N, k, mixed, tpb, ppt, st);
    case 3: return launch_paths_d3(m, g, P, M, N, k, mixed, tpb, ppt, st);
    case 4: return launch_paths_d4(m, g, P, M, N, k, mixed, tpb, ppt, st);
    case 5: return launch_paths_d5(m, g, P, M, N, k, mixed, tpb, ppt, st);
    case 6: return launch_paths_d6(m, g, P, M, N, k, mixed, tpb, ppt, st);
    case 7: return launch_paths_d7(m, g, P, M, N, k, mixed, tpb, ppt, st);
    case 8: return launch_paths_d8(m, g, P, M, N, k, mixed, tpb, ppt, st);
    case 9: return launch_paths_d9(m, g, P, M, N, k, mixed, tpb, ppt, st);
    case 10: return launch_paths_d10(m, g, P, M, N, k, mixed, tpb, ppt, st);
    default: return cudaErrorInvalidValue;
  }
}
