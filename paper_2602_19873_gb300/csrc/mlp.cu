// Learned smoothing-length start (not in the paper): a small MLP maps
// per-cluster SFC density features to log(h / e64), trained on h values of
// the exact iteration.  8 inputs -> 64 -> 64 -> 64 (SiLU) -> 1, BF16 operands
// on the tensor cores (mma.sync m16n8k16, FP32 accumulate), FP32 master
// weights and Adam.
//
// Features of cluster c (padded SFC order; e(B) = largest side of box B,
// e8 = its cluster box, e64 = its super-cluster box, e512 / e4096 = boxes of
// the 8 / 64 super-clusters around it inside its system, L = largest side
// of the system box, N_s = particles of the system):
//   log(e8/e64), log(e512/e64), log(e4096/e64), log(ex/e8), log(ey/e8),
//   log(ez/e8), log(count/M), log(e64/L) + log(N_s)/3.
// Target: log(mean h of the cluster / e64); the start h of a particle is
// e64 * exp(prediction of its cluster).
#include <cstdint>

#include <cuda_bf16.h>

#include "nl_internal.cuh"
#include "mlp.cuh"

namespace nlg {

__host__ __device__ __forceinline__ int64_t min_i64(int64_t a, int64_t b) { return a < b ? a : b; }

// ---------------------------------------------------------------------------
// Features and targets
// ---------------------------------------------------------------------------
__device__ __forceinline__ float box_extent(const float4 &lo, const float4 &hi)
{
    return fmaxf(fmaxf(hi.x - lo.x, hi.y - lo.y), hi.z - lo.z);
}

__global__ void k_sc_boxes(uint32_t nsc, const float4 *__restrict__ clo, const float4 *__restrict__ chi,
                           float4 *__restrict__ slo, float4 *__restrict__ shi)
{
    uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsc) return;
    float4 lo = make_float4(INFINITY, INFINITY, INFINITY, 0.f);
    float4 hi = make_float4(-INFINITY, -INFINITY, -INFINITY, 0.f);
    for (int k = 0; k < kSC; ++k) {
        float4 a = clo[s * kSC + k], b = chi[s * kSC + k];
        lo.x = fminf(lo.x, a.x); lo.y = fminf(lo.y, a.y); lo.z = fminf(lo.z, a.z);
        hi.x = fmaxf(hi.x, b.x); hi.y = fmaxf(hi.y, b.y); hi.z = fmaxf(hi.z, b.z);
    }
    slo[s] = lo;
    shi[s] = hi;
}

__device__ __forceinline__ float region_extent(const float4 *slo, const float4 *shi, int64_t a,
                                               int64_t b)
{
    float4 lo = make_float4(INFINITY, INFINITY, INFINITY, 0.f);
    float4 hi = make_float4(-INFINITY, -INFINITY, -INFINITY, 0.f);
    for (int64_t s = a; s < b; ++s) {
        float4 p = slo[s], q = shi[s];
        lo.x = fminf(lo.x, p.x); lo.y = fminf(lo.y, p.y); lo.z = fminf(lo.z, p.z);
        hi.x = fmaxf(hi.x, q.x); hi.y = fmaxf(hi.y, q.y); hi.z = fmaxf(hi.z, q.z);
    }
    return box_extent(lo, hi);
}

// one thread per super-cluster: features of its 8 clusters and e64
__global__ void k_features(uint32_t nsc, int M, SysTables t, const float4 *__restrict__ clo,
                           const float4 *__restrict__ chi, const float4 *__restrict__ slo,
                           const float4 *__restrict__ shi, const uint32_t *__restrict__ perm_pad,
                           float *__restrict__ X, float *__restrict__ e64out)
{
    uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsc) return;
    const uint32_t scp = kSC * M;
    const uint32_t sy = sys_of(t.pad_off, t.nsys, s * scp);
    const int64_t s0 = t.pad_off[sy] / scp, s1 = t.pad_off[sy + 1] / scp;
    const DevBox &b = t.box[sy];
    const float L = fmaxf(fmaxf(b.len[0], b.len[1]), b.len[2]);
    const float ns = (float)(t.off[sy + 1] - t.off[sy]);
    const float fl = 1e-7f * L;  // floor of every length
    const float e64 = fmaxf(box_extent(slo[s], shi[s]), fl);
    const float e512 = fmaxf(region_extent(slo, shi, max(s0, (int64_t)s - 3), min(s1, (int64_t)s + 5)), fl);
    const float e4k = fmaxf(region_extent(slo, shi, max(s0, (int64_t)s - 31), min(s1, (int64_t)s + 33)), fl);
    e64out[s] = e64;
    const float dens = logf(e64 / L) + logf(ns) * (1.f / 3.f);
    for (int k = 0; k < kSC; ++k) {
        const uint32_t c = s * kSC + k;
        uint32_t cnt = 0;
        for (int q = 0; q < M; ++q) cnt += perm_pad[c * M + q] != 0xffffffffu;
        float *x = X + (size_t)c * kMlpF;
        if (cnt == 0) {
            for (int f = 0; f < kMlpF; ++f) x[f] = 0.f;
            continue;
        }
        const float4 lo = clo[c], hi = chi[c];
        const float ex = fmaxf(hi.x - lo.x, fl), ey = fmaxf(hi.y - lo.y, fl), ez = fmaxf(hi.z - lo.z, fl);
        const float e8 = fmaxf(fmaxf(ex, ey), ez);
        x[0] = logf(e8 / e64);
        x[1] = logf(e512 / e64);
        x[2] = logf(e4k / e64);
        x[3] = logf(ex / e8);
        x[4] = logf(ey / e8);
        x[5] = logf(ez / e8);
        x[6] = logf((float)cnt / (float)M);
        x[7] = dens;
    }
}

// target of cluster c: log(mean h of its real particles / e64); w = 0 for
// empty clusters
__global__ void k_targets(uint32_t ncl, int M, const uint32_t *__restrict__ perm_pad,
                          const float *__restrict__ h, const float *__restrict__ e64,
                          float *__restrict__ y, float *__restrict__ w)
{
    uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncl) return;
    float s = 0.f;
    int cnt = 0;
    for (int q = 0; q < M; ++q) {
        uint32_t o = perm_pad[c * M + q];
        if (o != 0xffffffffu) {
            s += h[o];
            ++cnt;
        }
    }
    y[c] = cnt ? logf(s / cnt / e64[c / kSC]) : 0.f;
    w[c] = cnt ? 1.f : 0.f;
}

// start h of every real particle from its cluster's prediction
__global__ void k_apply_h0(uint32_t npad, int M, const uint32_t *__restrict__ perm_pad,
                           const float *__restrict__ pred, const float *__restrict__ e64,
                           float *__restrict__ hq)
{
    uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= npad) return;
    const uint32_t c = k / M;
    float h = 0.f;
    if (perm_pad[k] != 0xffffffffu) {
        float p = fminf(fmaxf(pred[c], -20.f), 20.f);
        h = e64[c / kSC] * expf(p);
        if (!(h > 0.f) || !isfinite(h)) h = e64[c / kSC];
    }
    hq[k] = h;
}

cudaError_t mlp_features(uint32_t nsc, int M, const SysTables &t, const float4 *clo,
                         const float4 *chi, const uint32_t *perm_pad, float4 *slo, float4 *shi,
                         float *X, float *e64, cudaStream_t s)
{
    k_sc_boxes<<<(nsc + 255) / 256, 256, 0, s>>>(nsc, clo, chi, slo, shi);
    k_features<<<(nsc + 127) / 128, 128, 0, s>>>(nsc, M, t, clo, chi, slo, shi, perm_pad, X, e64);
    return cudaGetLastError();
}

cudaError_t mlp_targets(uint32_t ncl, int M, const uint32_t *perm_pad, const float *h,
                        const float *e64, float *y, float *w, cudaStream_t s)
{
    k_targets<<<(ncl + 255) / 256, 256, 0, s>>>(ncl, M, perm_pad, h, e64, y, w);
    return cudaGetLastError();
}

cudaError_t mlp_apply_h0(uint32_t npad, int M, const uint32_t *perm_pad, const float *pred,
                         const float *e64, float *hq, cudaStream_t s)
{
    k_apply_h0<<<(npad + 255) / 256, 256, 0, s>>>(npad, M, perm_pad, pred, e64, hq);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Tensor-core building blocks
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ uint32_t pack_raw(__nv_bfloat16 lo, __nv_bfloat16 hi)
{
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// D += A (16x16, row) * B (16x8, col); BF16 operands, FP32 accumulators
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float silu_f(float z) { return z / (1.f + expf(-z)); }

__device__ __forceinline__ float dsilu_f(float z)
{
    float s = 1.f / (1.f + expf(-z));
    return s * (1.f + z * (1.f - s));
}

// Shared-memory copy of the network: BF16 weights row-major (out x in) and
// transposed, FP32 biases and output row.
struct MlpSmem {
    __nv_bfloat16 w1[kMlpH][16];          // inputs padded 8 -> 16 with zeros
    __nv_bfloat16 w2[kMlpH][kMlpH], w3[kMlpH][kMlpH];
    __nv_bfloat16 w2t[kMlpH][kMlpH], w3t[kMlpH][kMlpH];
    __nv_bfloat16 w1t[16][kMlpH];
    float b1[kMlpH], b2[kMlpH], b3[kMlpH], w4[kMlpH];
    float b4;
};

__device__ void load_net(MlpSmem &S, const float *__restrict__ P)
{
    const float *W1 = P, *B1 = W1 + kMlpH * kMlpF, *W2 = B1 + kMlpH, *B2 = W2 + kMlpH * kMlpH;
    const float *W3 = B2 + kMlpH, *B3 = W3 + kMlpH * kMlpH, *W4 = B3 + kMlpH, *B4 = W4 + kMlpH;
    for (int t = threadIdx.x; t < kMlpH * kMlpH; t += blockDim.x) {
        int o = t / kMlpH, i = t % kMlpH;
        __nv_bfloat16 a = __float2bfloat16_rn(W2[t]), b = __float2bfloat16_rn(W3[t]);
        S.w2[o][i] = a;
        S.w2t[i][o] = a;
        S.w3[o][i] = b;
        S.w3t[i][o] = b;
    }
    for (int t = threadIdx.x; t < kMlpH * 16; t += blockDim.x) {
        int o = t / 16, i = t % 16;
        __nv_bfloat16 v = __float2bfloat16_rn(i < kMlpF ? W1[o * kMlpF + i] : 0.f);
        S.w1[o][i] = v;
        S.w1t[i][o] = v;
    }
    for (int t = threadIdx.x; t < kMlpH; t += blockDim.x) {
        S.b1[t] = B1[t];
        S.b2[t] = B2[t];
        S.b3[t] = B3[t];
        S.w4[t] = __bfloat162float(__float2bfloat16_rn(W4[t]));
    }
    if (threadIdx.x == 0) S.b4 = B4[0];
}

// C tiles (16 rows x 64) -> A fragments (4 k-blocks of 16) after activation
__device__ __forceinline__ void to_afrag(const float (&h)[8][4], uint32_t (&A)[4][4])
{
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        A[kk][0] = pack_bf16(h[2 * kk][0], h[2 * kk][1]);
        A[kk][1] = pack_bf16(h[2 * kk][2], h[2 * kk][3]);
        A[kk][2] = pack_bf16(h[2 * kk + 1][0], h[2 * kk + 1][1]);
        A[kk][3] = pack_bf16(h[2 * kk + 1][2], h[2 * kk + 1][3]);
    }
}

// z = A(16x64) * W^T + b, W row-major [64][64] in shared memory
__device__ __forceinline__ void dense64(const uint32_t (&A)[4][4], const __nv_bfloat16 (&W)[kMlpH][kMlpH],
                                       const float *b, float (&z)[8][4])
{
    const unsigned lane = lane_id(), g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        z[j][0] = b[8 * j + 2 * t];
        z[j][1] = b[8 * j + 2 * t + 1];
        z[j][2] = z[j][0];
        z[j][3] = z[j][1];
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const uint32_t b0 = *reinterpret_cast<const uint32_t *>(&W[8 * j + g][16 * kk + 2 * t]);
            const uint32_t b1 = *reinterpret_cast<const uint32_t *>(&W[8 * j + g][16 * kk + 8 + 2 * t]);
            mma16816(z[j], A[kk], b0, b1);
        }
    }
}

// Forward of 16 rows (x: 16 x 8, row r at x + r*8, rows >= nrows are zero).
// Keeps pre-activations z1..z3 when asked (training).
__device__ __forceinline__ void forward16(const MlpSmem &S, const float *x, int ld, int nrows,
                                          float (&z1)[8][4], float (&z2)[8][4], float (&z3)[8][4],
                                          float (&pred)[2])
{
    const unsigned lane = lane_id(), g = lane >> 2, t = lane & 3;
    uint32_t A[4][4];
    {
        float x0 = g < (unsigned)nrows ? x[g * ld + 2 * t] : 0.f;
        float x1 = g < (unsigned)nrows ? x[g * ld + 2 * t + 1] : 0.f;
        float x2 = g + 8 < (unsigned)nrows ? x[(g + 8) * ld + 2 * t] : 0.f;
        float x3 = g + 8 < (unsigned)nrows ? x[(g + 8) * ld + 2 * t + 1] : 0.f;
        uint32_t a0[4] = {pack_bf16(x0, x1), pack_bf16(x2, x3), 0u, 0u};
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            z1[j][0] = S.b1[8 * j + 2 * t];
            z1[j][1] = S.b1[8 * j + 2 * t + 1];
            z1[j][2] = z1[j][0];
            z1[j][3] = z1[j][1];
            const uint32_t b0 = *reinterpret_cast<const uint32_t *>(&S.w1[8 * j + g][2 * t]);
            const uint32_t b1 = *reinterpret_cast<const uint32_t *>(&S.w1[8 * j + g][8 + 2 * t]);
            mma16816(z1[j], a0, b0, b1);
        }
    }
    float h[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) h[j][q] = silu_f(z1[j][q]);
    to_afrag(h, A);
    dense64(A, S.w2, S.b2, z2);
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) h[j][q] = silu_f(z2[j][q]);
    to_afrag(h, A);
    dense64(A, S.w3, S.b3, z3);
    // output: y = b4 + sum_k w4[k] h3[k]; h3 rounded to BF16 like every operand
    float p0 = 0.f, p1 = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float w0 = S.w4[8 * j + 2 * t], w1 = S.w4[8 * j + 2 * t + 1];
        p0 += w0 * __bfloat162float(__float2bfloat16_rn(silu_f(z3[j][0]))) +
              w1 * __bfloat162float(__float2bfloat16_rn(silu_f(z3[j][1])));
        p1 += w0 * __bfloat162float(__float2bfloat16_rn(silu_f(z3[j][2]))) +
              w1 * __bfloat162float(__float2bfloat16_rn(silu_f(z3[j][3])));
    }
    p0 += __shfl_xor_sync(0xffffffffu, p0, 1);
    p0 += __shfl_xor_sync(0xffffffffu, p0, 2);
    p1 += __shfl_xor_sync(0xffffffffu, p1, 1);
    p1 += __shfl_xor_sync(0xffffffffu, p1, 2);
    pred[0] = p0 + S.b4;
    pred[1] = p1 + S.b4;
}

// ---------------------------------------------------------------------------
// Inference: one warp per 16 samples
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_mlp_predict(int64_t n, const float *__restrict__ X,
                                                     const float *__restrict__ P,
                                                     float *__restrict__ out)
{
    extern __shared__ __align__(16) unsigned char mlp_smem[];
    MlpSmem &S = *reinterpret_cast<MlpSmem *>(mlp_smem);
    load_net(S, P);
    __syncthreads();
    const unsigned lane = lane_id(), g = lane >> 2, t = lane & 3;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t tile = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); tile * 16 < n;
         tile += warps) {
        const int64_t r0 = tile * 16;
        const int nrows = (int)min_i64(16, n - r0);
        float z1[8][4], z2[8][4], z3[8][4], pred[2];
        forward16(S, X + r0 * kMlpF, kMlpF, nrows, z1, z2, z3, pred);
        if (t == 0) {
            if ((int)g < nrows) out[r0 + g] = pred[0];
            if ((int)g + 8 < nrows) out[r0 + g + 8] = pred[1];
        }
    }
}

// ---------------------------------------------------------------------------
// Training: each CTA (4 warps) takes 64-sample tiles of the minibatch and
// accumulates its gradient in registers (warp w owns output rows 16w..16w+15
// of every weight matrix); the CTA's gradient goes to its own slot of
// `partial`, and k_mlp_adam reduces the slots in a fixed order.
// ---------------------------------------------------------------------------
struct TrainSmem {
    MlpSmem net;
    float z[3][64][kMlpH];                // pre-activations of the tile
    __nv_bfloat16 h[2][64][kMlpH];        // h1, h2 (BF16, as the forward used them)
    __nv_bfloat16 d[2][64][kMlpH];        // dZ of the current and next layer
    __nv_bfloat16 x[64][16];              // inputs, padded
    float dy[64];
    float loss[4];
};

size_t mlp_train_smem() { return sizeof(TrainSmem); }
size_t mlp_predict_smem() { return sizeof(MlpSmem); }

// stripe gradient: G[o in 16w..16w+15][i] += sum_r D[r][o] * Hin[r][i], i over
// nt n-tiles of 8 (K = 64 samples)
template <int NT, int LD>
__device__ __forceinline__ void grad_stripe(const __nv_bfloat16 (*D)[kMlpH],
                                            const __nv_bfloat16 (*Hin)[LD], float (&G)[NT][4])
{
    const unsigned lane = lane_id(), g = lane >> 2, t = lane & 3, w = threadIdx.x >> 5;
    const int o0 = 16 * w;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const int r = 16 * kk + 2 * t;
        uint32_t A[4];
        A[0] = pack_raw(D[r][o0 + g], D[r + 1][o0 + g]);
        A[1] = pack_raw(D[r][o0 + g + 8], D[r + 1][o0 + g + 8]);
        A[2] = pack_raw(D[r + 8][o0 + g], D[r + 9][o0 + g]);
        A[3] = pack_raw(D[r + 8][o0 + g + 8], D[r + 9][o0 + g + 8]);
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            const uint32_t b0 = pack_raw(Hin[r][8 * j + g], Hin[r + 1][8 * j + g]);
            const uint32_t b1 = pack_raw(Hin[r + 8][8 * j + g], Hin[r + 9][8 * j + g]);
            mma16816(G[j], A, b0, b1);
        }
    }
}

// dH (16 rows of this warp) = dZ (rows) * W, with W^T row-major in shared memory
__device__ __forceinline__ void back64(const __nv_bfloat16 (*D)[kMlpH], int row0,
                                      const __nv_bfloat16 (&WT)[kMlpH][kMlpH], float (&dh)[8][4])
{
    const unsigned lane = lane_id(), g = lane >> 2, t = lane & 3;
    uint32_t A[4][4];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        A[kk][0] = *reinterpret_cast<const uint32_t *>(&D[row0 + g][16 * kk + 2 * t]);
        A[kk][1] = *reinterpret_cast<const uint32_t *>(&D[row0 + g + 8][16 * kk + 2 * t]);
        A[kk][2] = *reinterpret_cast<const uint32_t *>(&D[row0 + g][16 * kk + 8 + 2 * t]);
        A[kk][3] = *reinterpret_cast<const uint32_t *>(&D[row0 + g + 8][16 * kk + 8 + 2 * t]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        dh[j][0] = dh[j][1] = dh[j][2] = dh[j][3] = 0.f;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const uint32_t b0 = *reinterpret_cast<const uint32_t *>(&WT[8 * j + g][16 * kk + 2 * t]);
            const uint32_t b1 = *reinterpret_cast<const uint32_t *>(&WT[8 * j + g][16 * kk + 8 + 2 * t]);
            mma16816(dh[j], A[kk], b0, b1);
        }
    }
}

__global__ void __launch_bounds__(128) k_mlp_train(int64_t nb, const int64_t *__restrict__ idx,
                                                   const float *__restrict__ X,
                                                   const float *__restrict__ Y,
                                                   const float *__restrict__ Wt,
                                                   const float *__restrict__ P, float inv_n,
                                                   float *__restrict__ partial,
                                                   float *__restrict__ loss_out)
{
    extern __shared__ __align__(16) unsigned char mlp_smem[];
    TrainSmem &S = *reinterpret_cast<TrainSmem *>(mlp_smem);
    load_net(S.net, P);
    const unsigned lane = lane_id(), g = lane >> 2, t = lane & 3, w = threadIdx.x >> 5;
    const int row0 = 16 * w;
    float gW1[2][4] = {}, gW2[8][4] = {}, gW3[8][4] = {}, gW4[8][2] = {};
    float gb1 = 0.f, gb2 = 0.f, gb3 = 0.f, gb4 = 0.f, lsum = 0.f;
    __syncthreads();
    for (int64_t tile = blockIdx.x; tile * 64 < nb; tile += gridDim.x) {
        const int64_t base = tile * 64;
        const int nrows = (int)min_i64(64, nb - base);
        // inputs to shared memory (padded, BF16) and, FP32, to a staging buffer
        for (int q = threadIdx.x; q < 64 * 16; q += blockDim.x) {
            const int r = q / 16, i = q % 16;
            float v = 0.f;
            if (r < nrows && i < kMlpF) v = X[idx[base + r] * kMlpF + i];
            S.x[r][i] = __float2bfloat16_rn(v);
            if (i < kMlpF) S.z[0][r][i] = v;  // raw inputs, FP32, read by forward16
        }
        __syncthreads();
        float z1[8][4], z2[8][4], z3[8][4], pred[2];
        forward16(S.net, &S.z[0][row0][0], kMlpH, max(0, min(16, nrows - row0)), z1, z2, z3, pred);
        __syncthreads();  // S.z[0] is reused for z1 below
        // keep pre-activations and BF16 activations of the tile
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = 8 * j + 2 * t;
            S.z[0][row0 + g][c] = z1[j][0];
            S.z[0][row0 + g][c + 1] = z1[j][1];
            S.z[0][row0 + g + 8][c] = z1[j][2];
            S.z[0][row0 + g + 8][c + 1] = z1[j][3];
            S.z[1][row0 + g][c] = z2[j][0];
            S.z[1][row0 + g][c + 1] = z2[j][1];
            S.z[1][row0 + g + 8][c] = z2[j][2];
            S.z[1][row0 + g + 8][c + 1] = z2[j][3];
            S.z[2][row0 + g][c] = z3[j][0];
            S.z[2][row0 + g][c + 1] = z3[j][1];
            S.z[2][row0 + g + 8][c] = z3[j][2];
            S.z[2][row0 + g + 8][c + 1] = z3[j][3];
            S.h[0][row0 + g][c] = __float2bfloat16_rn(silu_f(z1[j][0]));
            S.h[0][row0 + g][c + 1] = __float2bfloat16_rn(silu_f(z1[j][1]));
            S.h[0][row0 + g + 8][c] = __float2bfloat16_rn(silu_f(z1[j][2]));
            S.h[0][row0 + g + 8][c + 1] = __float2bfloat16_rn(silu_f(z1[j][3]));
            S.h[1][row0 + g][c] = __float2bfloat16_rn(silu_f(z2[j][0]));
            S.h[1][row0 + g][c + 1] = __float2bfloat16_rn(silu_f(z2[j][1]));
            S.h[1][row0 + g + 8][c] = __float2bfloat16_rn(silu_f(z2[j][2]));
            S.h[1][row0 + g + 8][c + 1] = __float2bfloat16_rn(silu_f(z2[j][3]));
        }
        if (t == 0) {
            const int ra = row0 + g, rb = row0 + g + 8;
            const float ea = ra < nrows ? (pred[0] - Y[idx[base + ra]]) * Wt[idx[base + ra]] : 0.f;
            const float eb = rb < nrows ? (pred[1] - Y[idx[base + rb]]) * Wt[idx[base + rb]] : 0.f;
            S.dy[ra] = 2.f * ea * inv_n;
            S.dy[rb] = 2.f * eb * inv_n;
            lsum += ea * ea + eb * eb;
        }
        __syncthreads();
        // layer 4 and dZ3 of this warp's rows
#pragma unroll
        for (int j = 0; j < 8; ++j) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int r = row0 + g + (q >= 2 ? 8 : 0), c = 8 * j + 2 * t + (q & 1);
                const float z = S.z[2][r][c];
                const float h3 = __bfloat162float(__float2bfloat16_rn(silu_f(z)));
                gW4[j][q & 1] += S.dy[r] * h3;
                S.d[0][r][c] = __float2bfloat16_rn(S.dy[r] * S.net.w4[c] * dsilu_f(z));
            }
        }
        if (lane == 0)
            for (int r = row0; r < row0 + 16; ++r) gb4 += S.dy[r];
        __syncthreads();
        // layer 3: weights (stripe) and dZ2 of this warp's rows
        grad_stripe<8, kMlpH>(S.d[0], S.h[1], gW3);
        {
            const int o = row0 + (lane & 15);
            float sb = 0.f;
            for (int r = (lane >> 4); r < 64; r += 2) sb += __bfloat162float(S.d[0][r][o]);
            gb3 += sb;
        }
        float dh[8][4];
        back64(S.d[0], row0, S.net.w3t, dh);
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int r = row0 + g + (q >= 2 ? 8 : 0), c = 8 * j + 2 * t + (q & 1);
                S.d[1][r][c] = __float2bfloat16_rn(dh[j][q] * dsilu_f(S.z[1][r][c]));
            }
        __syncthreads();
        // layer 2
        grad_stripe<8, kMlpH>(S.d[1], S.h[0], gW2);
        {
            const int o = row0 + (lane & 15);
            float sb = 0.f;
            for (int r = (lane >> 4); r < 64; r += 2) sb += __bfloat162float(S.d[1][r][o]);
            gb2 += sb;
        }
        back64(S.d[1], row0, S.net.w2t, dh);
        __syncthreads();  // every warp has read d[0] (layer 3) and d[1]
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int r = row0 + g + (q >= 2 ? 8 : 0), c = 8 * j + 2 * t + (q & 1);
                S.d[0][r][c] = __float2bfloat16_rn(dh[j][q] * dsilu_f(S.z[0][r][c]));
            }
        __syncthreads();
        // layer 1 (inputs padded to 16; only i < 8 are real)
        grad_stripe<2, 16>(S.d[0], S.x, gW1);
        {
            const int o = row0 + (lane & 15);
            float sb = 0.f;
            for (int r = (lane >> 4); r < 64; r += 2) sb += __bfloat162float(S.d[0][r][o]);
            gb1 += sb;
        }
        __syncthreads();
    }
    // write this CTA's gradient slot (packing of the parameter vector)
    float *G = partial + (size_t)blockIdx.x * kMlpParams;
    float *gw1 = G, *gbb1 = gw1 + kMlpH * kMlpF, *gw2 = gbb1 + kMlpH, *gbb2 = gw2 + kMlpH * kMlpH;
    float *gw3 = gbb2 + kMlpH, *gbb3 = gw3 + kMlpH * kMlpH, *gw4 = gbb3 + kMlpH, *gbb4 = gw4 + kMlpH;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int i = 8 * j + 2 * t;
        gw2[(row0 + g) * kMlpH + i] = gW2[j][0];
        gw2[(row0 + g) * kMlpH + i + 1] = gW2[j][1];
        gw2[(row0 + g + 8) * kMlpH + i] = gW2[j][2];
        gw2[(row0 + g + 8) * kMlpH + i + 1] = gW2[j][3];
        gw3[(row0 + g) * kMlpH + i] = gW3[j][0];
        gw3[(row0 + g) * kMlpH + i + 1] = gW3[j][1];
        gw3[(row0 + g + 8) * kMlpH + i] = gW3[j][2];
        gw3[(row0 + g + 8) * kMlpH + i + 1] = gW3[j][3];
    }
    if (t < 4) {  // n-tile 0 of layer 1 holds inputs 0..7
        const int i = 2 * t;
        gw1[(row0 + g) * kMlpF + i] = gW1[0][0];
        gw1[(row0 + g) * kMlpF + i + 1] = gW1[0][1];
        gw1[(row0 + g + 8) * kMlpF + i] = gW1[0][2];
        gw1[(row0 + g + 8) * kMlpF + i + 1] = gW1[0][3];
    }
    // biases: lanes l and l+16 hold halves of the same output
    gb1 += __shfl_xor_sync(0xffffffffu, gb1, 16);
    gb2 += __shfl_xor_sync(0xffffffffu, gb2, 16);
    gb3 += __shfl_xor_sync(0xffffffffu, gb3, 16);
    if (lane < 16) {
        gbb1[row0 + lane] = gb1;
        gbb2[row0 + lane] = gb2;
        gbb3[row0 + lane] = gb3;
    }
    // output row: every warp summed its own rows for all 64 inputs
#pragma unroll
    for (int j = 0; j < 8; ++j) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            float v = gW4[j][q];
            v += __shfl_xor_sync(0xffffffffu, v, 4);
            v += __shfl_xor_sync(0xffffffffu, v, 8);
            v += __shfl_xor_sync(0xffffffffu, v, 16);
            gW4[j][q] = v;
        }
    }
    __shared__ float w4acc[4][kMlpH];
    __shared__ float b4acc[4], lacc[4];
    if (g == 0) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            w4acc[w][8 * j + 2 * t] = gW4[j][0];
            w4acc[w][8 * j + 2 * t + 1] = gW4[j][1];
        }
    }
    lsum += __shfl_xor_sync(0xffffffffu, lsum, 4);
    lsum += __shfl_xor_sync(0xffffffffu, lsum, 8);
    lsum += __shfl_xor_sync(0xffffffffu, lsum, 16);
    if (lane == 0) {
        b4acc[w] = gb4;
        lacc[w] = lsum;
    }
    __syncthreads();
    if (threadIdx.x < kMlpH)
        gw4[threadIdx.x] = w4acc[0][threadIdx.x] + w4acc[1][threadIdx.x] + w4acc[2][threadIdx.x] +
                           w4acc[3][threadIdx.x];
    if (threadIdx.x == 0) {
        gbb4[0] = b4acc[0] + b4acc[1] + b4acc[2] + b4acc[3];
        loss_out[blockIdx.x] = lacc[0] + lacc[1] + lacc[2] + lacc[3];
    }
}

// Sum the CTA slots in order; optionally apply Adam to the master weights.
__global__ void k_mlp_reduce_adam(int nslots, const float *__restrict__ partial, float *__restrict__ grad,
                                  float *__restrict__ P, float *__restrict__ m, float *__restrict__ v,
                                  int adam, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= kMlpParams) return;
    float s = 0.f;
    for (int q = 0; q < nslots; ++q) s += partial[(size_t)q * kMlpParams + k];
    if (grad) grad[k] = s;
    if (!adam) return;
    const float mk = b1 * m[k] + (1.f - b1) * s;
    const float vk = b2 * v[k] + (1.f - b2) * s * s;
    m[k] = mk;
    v[k] = vk;
    P[k] -= lr * (mk * c1) / (sqrtf(vk * c2) + eps);
}

cudaError_t mlp_predict(int64_t n, const float *X, const float *P, float *out, int num_sms,
                        cudaStream_t s)
{
    cudaError_t e = set_max_dynamic_smem((const void *)k_mlp_predict, mlp_predict_smem());
    if (e != cudaSuccess) return e;
    const int64_t tiles = (n + 15) / 16;
    const int grid = (int)min_i64((tiles + 3) / 4, (int64_t)num_sms * 8);
    if (grid > 0) k_mlp_predict<<<grid, 128, mlp_predict_smem(), s>>>(n, X, P, out);
    return cudaGetLastError();
}

cudaError_t mlp_train_step(int64_t nb, const int64_t *idx, const float *X, const float *Y,
                           const float *W, float *P, float *m, float *v, float *partial,
                           int slots, float *grad, float *loss, int adam, float lr, int step,
                           float inv_n, cudaStream_t s)
{
    cudaError_t e = set_max_dynamic_smem((const void *)k_mlp_train, mlp_train_smem());
    if (e != cudaSuccess) return e;
    const int grid = (int)min_i64((nb + 63) / 64, slots);
    if (grid <= 0) return cudaSuccess;
    k_mlp_train<<<grid, 128, mlp_train_smem(), s>>>(nb, idx, X, Y, W, P, inv_n, partial, loss);
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f / (1.f - powf(b1, (float)step)), c2 = 1.f / (1.f - powf(b2, (float)step));
    k_mlp_reduce_adam<<<(kMlpParams + 255) / 256, 256, 0, s>>>(grid, partial, grad, P, m, v, adam, lr,
                                                               b1, b2, 1e-8f, c1, c2);
    return cudaGetLastError();
}

}  // namespace nlg
