// Instantiation of the neighborhood pass kernel for PASS_MIN, the distance to
// the nearest gather neighbor (a minimum reduction; see pass_impl.cuh).
#include "pass_impl.cuh"

namespace nlg {
cudaError_t launch_pass_min(const PassArgs &a, int M, int per, int grid, int threads,
                          cudaStream_t s)
{
    return launch_k<PASS_MIN>(a, M, per, grid, threads, s);
}
}  // namespace nlg
