// Instantiation of the neighborhood pass kernel for PASS_LJ (see pass_impl.cuh).
#include "pass_impl.cuh"

namespace nlg {
cudaError_t launch_pass_lj(const PassArgs &a, int M, int per, int grid, int threads,
                          cudaStream_t s)
{
    return launch_k<PASS_LJ>(a, M, per, grid, threads, s);
}
}  // namespace nlg
