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
cudaError_t launch_pass_ljc(const PassArgs &a, int M, int per, int grid, int threads,
                          cudaStream_t s);
cudaError_t launch_pass_min(const PassArgs &a, int M, int per, int grid, int threads,
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
    case PASS_LJC: return launch_pass_ljc(a, M, any_periodic, grid, tpb, s);
    case PASS_MIN: return launch_pass_min(a, M, any_periodic, grid, tpb, s);
    default: return cudaErrorInvalidValue;
    }
}

// Gather per-particle pass inputs into SFC order.
// mode 0: aux = (a, 0); mode 1: aux = (a, b / (c*c)) (SPH: m, P / rho^2).
__global__ void __launch_bounds__(256) k_gather_aux(uint32_t npad, const uint32_t *__restrict__ perm_pad,
                                                    const float *__restrict__ a, const float *__restrict__ b,
                                                    const float *__restrict__ c, int mode,
                                                    float2 *__restrict__ aux, unsigned int *amax)
{
    __shared__ unsigned int wmax[8];
    uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    float2 v = make_float2(0.f, 0.f);
    if (k < npad) {
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
    if (!amax) return;  // uniform over the grid
    // largest |a| of the block, one atomic per block (non-negative floats
    // order like their bit patterns)
    unsigned int m = __reduce_max_sync(0xffffffffu, __float_as_uint(fabsf(v.x)));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? wmax[threadIdx.x] : 0u;
        m = __reduce_max_sync(0xffffffffu, m);
        if (threadIdx.x == 0 && m) atomicMax(amax, m);
    }
}

// Outputs of a half-list pass: density = (sum in fixed point) * 2^-scale *
// W's normalisation 1/(pi h^3), in the same FP32 form as the full-list pass;
// counts as summed; forces rounded from their FP64 sums.  Real slots only,
// written at perm[k] (or k).
__global__ void __launch_bounds__(256) k_half_finish(PassArgs a, int kind, uint32_t npad)
{
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= npad) return;
    const uint32_t pc = a.perm[k];
    if (pc == 0xffffffffu) return;
    const uint32_t o = a.sorted_out ? k : pc;
    if (kind == PASS_COUNT) {
        a.outc[o] = a.hcnt[k];
        return;
    }
    if (kind == PASS_MIN) {  // +inf bits when no neighbor was found
        a.out0[o] = sqrtf(__uint_as_float(a.hcnt[k]));
        return;
    }
    if (kind != PASS_DENSITY) {  // forces: the FP64 sums rounded once to FP32
        a.out0[o] = (float)a.hf[3 * (size_t)k + 0];
        a.out1[o] = (float)a.hf[3 * (size_t)k + 1];
        a.out2[o] = (float)a.hf[3 * (size_t)k + 2];
        return;
    }
    const int ex = half_scale_exp(a.st->m_absmax);
    const double unit = __longlong_as_double((long long)(1023 - ex) << 52);  // 2^-ex
    const float v = (float)((double)(long long)a.hsum[k] * unit);
    const float hinv = 1.f / a.pos[k].w;
    a.out0[o] = v * (0.318309886183790672f * hinv * hinv * hinv);
}

cudaError_t launch_half_finish(const PassArgs &a, int kind, uint32_t npad, cudaStream_t s)
{
    if (kind < PASS_DENSITY || kind > PASS_MIN) return cudaErrorInvalidValue;
    k_half_finish<<<(npad + 255) / 256, 256, 0, s>>>(a, kind, npad);
    return cudaGetLastError();
}

// New positions for a list kept across steps (Verlet buffer): every real
// padded slot takes its particle's caller-order position and keeps its h;
// optionally the largest displacement from the positions the list was built
// on (minimum image on periodic axes), as a float held in an unsigned word
// (non-negative floats order like their bit patterns).
__global__ void __launch_bounds__(256) k_refresh(uint32_t npad, const uint32_t *__restrict__ perm_pad,
                                                 SysTables t, const float *__restrict__ x,
                                                 const float *__restrict__ y,
                                                 const float *__restrict__ z, float4 *__restrict__ pos,
                                                 const float4 *__restrict__ pos_ref,
                                                 unsigned *__restrict__ max_disp)
{
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    float d = 0.f;
    if (k < npad) {
        const uint32_t o = perm_pad[k];
        if (o != 0xffffffffu) {
            const float4 old = pos[k];
            const float4 p = make_float4(x[o], y[o], z[o], old.w);
            pos[k] = p;
            if (max_disp) {
                const PerLen L = per_len(t.box[sys_of(t.pad_off, t.nsys, k)]);
                const float3 dv = pair_dx_acc<true>(pos_ref[k], p, L);
                d = sqrtf(dv.x * dv.x + dv.y * dv.y + dv.z * dv.z);
            }
        }
    }
    if (!max_disp) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d = fmaxf(d, __shfl_xor_sync(0xffffffffu, d, o));
    if ((threadIdx.x & 31) == 0 && d > 0.f) atomicMax(max_disp, __float_as_uint(d));
}

cudaError_t launch_refresh(uint32_t npad, const uint32_t *perm_pad, const SysTables &t,
                           const float *x, const float *y, const float *z, float4 *pos,
                           const float4 *pos_ref, float *max_disp, cudaStream_t s)
{
    if (max_disp) {
        cudaError_t e = cudaMemsetAsync(max_disp, 0, sizeof(float), s);
        if (e != cudaSuccess) return e;
    }
    k_refresh<<<(npad + 255) / 256, 256, 0, s>>>(npad, perm_pad, t, x, y, z, pos, pos_ref,
                                                reinterpret_cast<unsigned *>(max_disp));
    return cudaGetLastError();
}

cudaError_t launch_gather_aux(uint32_t npad, const uint32_t *perm_pad, const float *a,
                              const float *b, const float *c, int mode, float2 *aux,
                              cudaStream_t s, unsigned int *amax)
{
    k_gather_aux<<<(npad + 255) / 256, 256, 0, s>>>(npad, perm_pad, a, b, c, mode, aux, amax);
    return cudaGetLastError();
}

}  // namespace nlg
