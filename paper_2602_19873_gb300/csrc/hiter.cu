// Per-particle smoothing-length iteration to a target neighbor count.
//
// Valid set for particle i: { h : |#{j != i : d2_ij < (support*h)^2} - n_t| <= tol },
// where d2 is the canonical FP32 distance.  The count is a step function of
// h, so the update brackets the window: a count below the window raises the
// lower bracket, above lowers the upper one; while only one side is known
// the step is h * (n_t / count)^(1/3) clamped to [1/2, 2], afterwards the
// new h bisects the bracket in h^3 (the enclosed volume).  Counts come from
// the neighbor list built at a search radius (1 + margin) * h; the list is
// rebuilt only when some h outgrows its search radius.  All state lives in
// SFC-sorted order.
#include "nl_internal.cuh"

namespace nlg {

__global__ void k_fill(float *a, uint32_t n, float v)
{
    uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) a[k] = v;
}

cudaError_t launch_fill(float *a, uint32_t n, float v, cudaStream_t s)
{
    k_fill<<<(n + 255) / 256, 256, 0, s>>>(a, n, v);
    return cudaGetLastError();
}

// (dummy slots carry h = 0 in both directions)
__global__ void k_pos_h(uint32_t npad, const float *__restrict__ hs, float4 *__restrict__ pos)
{
    uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < npad) pos[k].w = hs[k];
}

cudaError_t launch_pos_h(uint32_t npad, const float *hs, float4 *pos, cudaStream_t s)
{
    k_pos_h<<<(npad + 255) / 256, 256, 0, s>>>(npad, hs, pos);
    return cudaGetLastError();
}

__global__ void k_pos_h_to(uint32_t npad, const float4 *__restrict__ pos, float *__restrict__ hq)
{
    uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < npad) hq[k] = pos[k].w;
}

cudaError_t launch_pos_h_to(uint32_t npad, const float4 *pos, float *hq, cudaStream_t s)
{
    k_pos_h_to<<<(npad + 255) / 256, 256, 0, s>>>(npad, pos, hq);
    return cudaGetLastError();
}

// Cluster boxes from the sorted positions (dummies are NaN and ignored).
template <int M>
__global__ void __launch_bounds__(256) k_cluster_boxes(uint32_t npad, const float4 *__restrict__ pos,
                                                       float support, float4 *__restrict__ clo,
                                                       float4 *__restrict__ chi, int MJ,
                                                       float4 *__restrict__ jlo,
                                                       float4 *__restrict__ jhi)
{
    uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;  // npad is a multiple of 32
    if (k >= npad) return;
    float4 p = pos[k];
    bool real = p.x == p.x;
    float r = real ? __fmul_rn(support, p.w) : 0.f;
    cluster_box_reduce<M>(k, real, p, r, MJ, clo, chi, jlo, jhi);
}

cudaError_t launch_cluster_boxes(uint32_t npad, int M, int MJ, const float4 *pos, float support,
                                 float4 *clo, float4 *chi, float4 *jlo, float4 *jhi,
                                 cudaStream_t s)
{
    unsigned grid = (npad + 255) / 256;
    if (MJ == M) jlo = jhi = nullptr;
    else if (!jlo || !jhi || MJ < 1 || M % MJ) return cudaErrorInvalidValue;
    switch (M) {
    case 4: k_cluster_boxes<4><<<grid, 256, 0, s>>>(npad, pos, support, clo, chi, MJ, jlo, jhi); break;
    case 8: k_cluster_boxes<8><<<grid, 256, 0, s>>>(npad, pos, support, clo, chi, MJ, jlo, jhi); break;
    case 16: k_cluster_boxes<16><<<grid, 256, 0, s>>>(npad, pos, support, clo, chi, MJ, jlo, jhi); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Plain start: the 8*M particles of a super-cluster fill (about) its box,
// so the number density there is count / volume and the sphere of radius
// 2h holds n_t particles for h = 0.5 * (3 n_t V / (4 pi count))^(1/3).
__global__ void k_plain_h0(uint32_t nsc, int M, const uint32_t *__restrict__ perm_pad,
                           const float4 *__restrict__ clo, const float4 *__restrict__ chi,
                           float n_target, float *__restrict__ hq)
{
    uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsc) return;
    float lx = INFINITY, ly = INFINITY, lz = INFINITY, hx = -INFINITY, hy = -INFINITY, hz = -INFINITY;
    for (int k = 0; k < kSC; ++k) {
        float4 a = clo[s * kSC + k], b = chi[s * kSC + k];
        lx = fminf(lx, a.x); ly = fminf(ly, a.y); lz = fminf(lz, a.z);
        hx = fmaxf(hx, b.x); hy = fmaxf(hy, b.y); hz = fmaxf(hz, b.z);
    }
    const uint32_t first = s * kSC * M, last = first + kSC * M;
    uint32_t real = 0;
    for (uint32_t k = first; k < last; ++k) real += perm_pad[k] != 0xffffffffu;
    float cnt = (float)real;
    float ex = fmaxf(hx - lx, 0.f), ey = fmaxf(hy - ly, 0.f), ez = fmaxf(hz - lz, 0.f);
    float emax = fmaxf(ex, fmaxf(ey, ez));
    float floor_e = fmaxf(emax * 1e-2f, 1e-30f);  // flat or collinear groups
    float vol = fmaxf(ex, floor_e) * fmaxf(ey, floor_e) * fmaxf(ez, floor_e);
    float h = 0.5f * cbrtf(3.f * n_target * vol / (4.f * 3.14159265f * fmaxf(cnt, 1.f)));
    if (!(h > 0.f) || !isfinite(h)) h = 1e-6f;
    for (uint32_t k = first; k < last; ++k) hq[k] = perm_pad[k] != 0xffffffffu ? h : 0.f;
}

cudaError_t launch_plain_h0(uint32_t nsc, int M, const uint32_t *perm_pad, const float4 *clo,
                            const float4 *chi, float n_target, float *hq, cudaStream_t s)
{
    k_plain_h0<<<(nsc + 127) / 128, 128, 0, s>>>(nsc, M, perm_pad, clo, chi, n_target, hq);
    return cudaGetLastError();
}

// Search h of each particle for a rebuild: h (1 + margin), except that a
// converged particle keeps its h (the gather count of a particle depends on
// its own h only, so it will not change) and a particle whose bisection
// bracket is closed above needs no more than the bracket's upper end (its
// next h stays below it).  Every value is >= the particle's current h.
__global__ void k_hsearch(uint32_t npad, const float *__restrict__ hq,
                          const float *__restrict__ hhi, const uint8_t *__restrict__ conv,
                          float margin, const float *__restrict__ hcap_sys, SysTables t,
                          float *__restrict__ hs)
{
    uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= npad) return;
    const float h = hq[k], hi = hhi[k];
    const float want = conv[k] ? h : fmaxf(fminf(hi, h * (1.f + margin)), h);
    hs[k] = fminf(want, hcap_sys[sys_of(t.pad_off, t.nsys, k)]);
}

cudaError_t launch_hsearch(uint32_t npad, const float *hq, const float *hhi, const uint8_t *conv,
                           float margin, const float *hcap_sys, const SysTables &t, float *hs,
                           cudaStream_t s)
{
    k_hsearch<<<(npad + 255) / 256, 256, 0, s>>>(npad, hq, hhi, conv, margin, hcap_sys, t, hs);
    return cudaGetLastError();
}

// hcap_sys[s] is the largest h whose radius stays below half a periodic box
// length of system s; it bounds both the iterated h and the search h.
__global__ void k_hupdate(uint32_t npad, int M, float n_target, float tol, SysTables t,
                          HIterState h)
{
    uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    bool act = false, reb = false;
    if (k < npad && h.perm_pad[k] != 0xffffffffu && !h.conv[k]) {
        const float hcap = h.hcap_sys[sys_of(t.pad_off, t.nsys, k)];
        float c = (float)h.counts[k];
        float hv = h.hq[k];
        if (fabsf(c - n_target) <= tol) {
            h.conv[k] = 1;
        } else {
            float lo = h.hlo[k], hi = h.hhi[k];
            if (c < n_target) lo = hv; else hi = hv;
            float hn;
            if (lo > 0.f && hi < INFINITY) {
                hn = cbrtf(0.5f * (lo * lo * lo + hi * hi * hi));
            } else {
                float f = cbrtf(n_target / fmaxf(c, 1.f));
                hn = hv * fminf(fmaxf(f, 0.5f), 2.f);
            }
            hn = fminf(hn, hcap);
            h.hlo[k] = lo;
            h.hhi[k] = hi;
            h.hq[k] = hn;
            act = true;
            reb = hn > h.hs[k];
            h.active_flag[k / (kSC * M)] = 1u;
        }
    }
    unsigned na = __popc(__ballot_sync(0xffffffffu, act));
    bool rb = __any_sync(0xffffffffu, reb);
    if (lane_id() == 0) {
        if (na) atomicAdd(&h.words[0], na);
        if (rb) atomicOr(&h.words[1], 1u);
    }
}

cudaError_t launch_hupdate(uint32_t npad, int M, float n_target, float tol, const SysTables &t,
                           const HIterState &h, cudaStream_t s)
{
    k_hupdate<<<(npad + 255) / 256, 256, 0, s>>>(npad, M, n_target, tol, t, h);
    return cudaGetLastError();
}

__global__ void k_active_list(uint32_t nsc, HIterState h)
{
    uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    bool a = s < nsc && h.active_flag[s];
    unsigned b = __ballot_sync(0xffffffffu, a);
    unsigned base = 0;
    if (lane_id() == 0 && b) base = atomicAdd(&h.words[2], __popc(b));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (a) {
        h.active_list[base + __popc(b & lanemask_lt())] = s;
        h.active_flag[s] = 0u;
    }
}

cudaError_t launch_active_list(uint32_t nsc, const HIterState &h, cudaStream_t s)
{
    k_active_list<<<(nsc + 255) / 256, 256, 0, s>>>(nsc, h);
    return cudaGetLastError();
}

__global__ void k_scatter_h(uint32_t npad, const uint32_t *__restrict__ perm_pad,
                            const float *__restrict__ hq, const uint8_t *__restrict__ conv,
                            float *__restrict__ h_out, uint8_t *__restrict__ conv_out)
{
    uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= npad) return;
    const uint32_t o = perm_pad[k];
    if (o == 0xffffffffu) return;
    h_out[o] = hq[k];
    if (conv_out) conv_out[o] = conv[k];
}

cudaError_t launch_scatter_h(uint32_t npad, const uint32_t *perm_pad, const float *hq,
                             const uint8_t *conv, float *h_out, uint8_t *conv_out, cudaStream_t s)
{
    k_scatter_h<<<(npad + 255) / 256, 256, 0, s>>>(npad, perm_pad, hq, conv, h_out, conv_out);
    return cudaGetLastError();
}

}  // namespace nlg
