// Dispatch of the neighborhood passes (kernels in pass_impl.cuh, one
// translation unit per pass kind) and the gather of pass inputs.
#include "nl_internal.cuh"

namespace nlg {

constexpr int kPassBlocksPerSM = 4;
cudaError_t launch_pass_density(const PassArgs &a, int M, int per, int grid, int threads,
                          cudaStream_t s);
cudaError_t launch_pass_count(const PassArgs &a, int M, int per, int grid, int threads,
                          cudaStream_t s);
cudaError_t launch_pass_sph(const PassArgs &a, int M, int per, int grid, int threads,
                          cudaStream_t s);
cudaError_t launch_pass_lj(const PassArgs &a, int M, int per, int grid, int threads,
                          cudaStream_t s);

cudaError_t launch_pass(const PassArgs &a, int kind, int M, int any_periodic, int num_sms,
                        cudaStream_t s, int threads, int blocks_per_sm)
{
    cudaError_t e = cudaMemsetAsync(&a.st->pass_ticket, 0, 4, s);
    if (e != cudaSuccess) return e;
    const int tpb = threads ? threads : 256;
    const int grid = num_sms * (blocks_per_sm ? blocks_per_sm : kPassBlocksPerSM);
    switch (kind) {
    case PASS_DENSITY: return launch_pass_density(a, M, any_periodic, grid, tpb, s);
    case PASS_COUNT: return launch_pass_count(a, M, any_periodic, grid, tpb, s);
    case PASS_SPH: return launch_pass_sph(a, M, any_periodic, grid, tpb, s);
    case PASS_LJ: return launch_pass_lj(a, M, any_periodic, grid, tpb, s);
    default: return cudaErrorInvalidValue;
    }
}

// Gather per-particle pass inputs into SFC order.
// mode 0: aux = (a, 0); mode 1: aux = (a, b / (c*c)) (SPH: m, P / rho^2).
__global__ void k_gather_aux(uint32_t npad, const uint32_t *__restrict__ perm_pad,
                             const float *__restrict__ a, const float *__restrict__ b,
                             const float *__restrict__ c, int mode, float2 *__restrict__ aux)
{
    uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= npad) return;
    float2 v = make_float2(0.f, 0.f);
    const uint32_t o = perm_pad[k];
    if (o != 0xffffffffu) {
        v.x = a[o];
        if (mode == 1) {
            float rho = c[o];
            v.y = b[o] / (rho * rho);
        }
    }
    aux[k] = v;
}

cudaError_t launch_gather_aux(uint32_t npad, const uint32_t *perm_pad, const float *a,
                              const float *b, const float *c, int mode, float2 *aux,
                              cudaStream_t s)
{
    k_gather_aux<<<(npad + 255) / 256, 256, 0, s>>>(npad, perm_pad, a, b, c, mode, aux);
    return cudaGetLastError();
}

}  // namespace nlg
