// Instantiation of the neighborhood pass kernel for PASS_LJC, Lennard-Jones
// plus Coulomb at an interaction cutoff inside the list radius (see pass_impl.cuh).
#include "pass_impl.cuh"

namespace nlg {
cudaError_t launch_pass_ljc(const PassArgs &a, int M, int per, int grid, int threads,
                          cudaStream_t s)
{
    return launch_k<PASS_LJC>(a, M, per, grid, threads, s);
}
}  // namespace nlg
