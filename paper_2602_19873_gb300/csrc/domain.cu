// SFC domain decomposition: the per-rank device steps (Sec. I: the domain is
// split into contiguous key ranges of the space-filling curve, as in the
// Cornerstone octree library the method builds on; Sec. IV: each rank builds
// its list over its own particles plus the halo it receives from the others).
//
// A decomposition step on P ranks (the exchange itself is done by the
// caller, e.g. over torch.distributed):
//   1. nl_sfc_keys: 63-bit keys of the local particles in the global box;
//   2. nl_key_histogram: counts per key bucket, summed over ranks, twice
//      (16 bits, then 16 more bits inside the buckets that hold a splitter),
//      give P-1 splitters that balance the particle counts;
//   3. nl_domain_owner_mask + nl_domain_count / nl_domain_group: the local
//      particles grouped by owner rank (one all-to-all moves them);
//   4. nl_domain_box: box and largest radius of the owned particles (one
//      all-gather shares them);
//   5. nl_domain_halo_mask + count / group: the owned particles that may be a
//      symmetric neighbor of a particle inside another rank's box (the node
//      test of the search, with the same monotone rounding, so no pair can be
//      missed); one more all-to-all moves them;
//   6. nl_build over owned + halo particles and any pass: the owned
//      particles' neighbor sets are complete.
#include <cstdio>

#include "nl_internal.cuh"

namespace nlg {
nl_status report_error(nl_status st, const char *msg);
}

using namespace nlg;

namespace {

constexpr int kMaxRanks = 64;   // destinations are bits of a 64-bit mask
constexpr int kGroupThreads = 256;
constexpr int kGroupItems = 4;  // particles per thread in the grouping kernels
constexpr int kGroupTile = kGroupThreads * kGroupItems;

DevBox to_devbox(const nl_box &b)
{
    DevBox d{};
    for (int a = 0; a < 3; ++a) {
        volatile float lo = b.lo[a], hi = b.hi[a];
        float len = hi - lo;
        volatile float num = 2097152.0f;
        d.lo[a] = lo;
        d.hi[a] = hi;
        d.len[a] = len;
        d.half[a] = 0.5f * len;
        d.qs[a] = num / len;
        d.per[a] = b.periodic[a] ? 1 : 0;
    }
    return d;
}

bool box_ok(const nl_box *b)
{
    for (int a = 0; a < 3; ++a) {
        volatile float lo = b->lo[a], hi = b->hi[a];
        if (!(lo < hi) || !(hi - lo < 3.0e38f) || !(lo > -3.0e38f)) return false;
    }
    return true;
}

nl_status cuda_fail(cudaError_t e, const char *what)
{
    (void)cudaGetLastError();
    static thread_local char msg[256];
    snprintf(msg, sizeof(msg), "%s: %s", what, cudaGetErrorString(e));
    return report_error(NL_ERR_CUDA, msg);
}

// Bucket counts of sorted-or-not keys; lanes of a warp that hit the same
// bucket add once (dense cores put many keys in few buckets).
__global__ void __launch_bounds__(256) k_key_hist(const uint64_t *__restrict__ keys, int64_t n,
                                                  uint64_t lo, int shift, uint32_t nbins,
                                                  unsigned long long *__restrict__ hist)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < n; i0 += stride) {
        const int64_t i = i0 + threadIdx.x;
        uint32_t bin = 0xffffffffu;
        if (i < n) {
            const uint64_t k = keys[i];
            if (k >= lo) {
                const uint64_t b = (k - lo) >> shift;
                if (b < nbins) bin = (uint32_t)b;
            }
        }
        const uint32_t peers = __match_any_sync(0xffffffffu, bin);
        if (bin != 0xffffffffu && lane_id() == (uint32_t)(__ffs(peers) - 1))
            atomicAdd(&hist[bin], (unsigned long long)__popc(peers));
    }
}

// owner = number of splitters <= key (splitters ascending)
__global__ void __launch_bounds__(256) k_owner_mask(const uint64_t *__restrict__ keys, int64_t n,
                                                    const uint64_t *__restrict__ split, int nsplit,
                                                    unsigned long long *__restrict__ mask)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t k = keys[i];
    int lo = 0, hi = nsplit;  // first splitter > k
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (split[mid] <= k) lo = mid + 1; else hi = mid;
    }
    mask[i] = 1ull << lo;
}

// Box and largest radius of the particles: float bits mapped to an order-
// preserving unsigned code so that integer atomics give the min and max.
__device__ __forceinline__ unsigned ordered_bits(float f)
{
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float from_ordered_bits(unsigned u)
{
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

__global__ void k_box_init(unsigned *acc)
{
    if (threadIdx.x < 3) acc[threadIdx.x] = 0xffffffffu;      // min codes
    else if (threadIdx.x < 6) acc[threadIdx.x] = 0u;          // max codes
    else if (threadIdx.x == 6) acc[6] = ordered_bits(0.f);    // max radius
}

__global__ void __launch_bounds__(256) k_box_reduce(const float *__restrict__ x,
                                                    const float *__restrict__ y,
                                                    const float *__restrict__ z,
                                                    const float *__restrict__ h, int64_t n,
                                                    float support, unsigned *acc)
{
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    float r = 0.f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float p[3] = {x[i], y[i], z[i]};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = fminf(lo[a], p[a]);
            hi[a] = fmaxf(hi[a], p[a]);
        }
        r = fmaxf(r, __fmul_rn(support, h[i]));
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
        r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, o));
    }
    if (lane_id() == 0) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            atomicMin(&acc[a], ordered_bits(lo[a]));
            atomicMax(&acc[3 + a], ordered_bits(hi[a]));
        }
        atomicMax(&acc[6], ordered_bits(r));
    }
}

__global__ void k_box_finish(const unsigned *acc, int64_t n, float *out)
{
    if (threadIdx.x != 0) return;
    for (int a = 0; a < 3; ++a) {
        out[a] = n > 0 ? from_ordered_bits(acc[a]) : INFINITY;
        out[4 + a] = n > 0 ? from_ordered_bits(acc[3 + a]) : -INFINITY;
    }
    out[3] = n > 0 ? from_ordered_bits(acc[6]) : 0.f;
    out[7] = 0.f;
}

// Halo destinations: bit q set when the particle (radius r = support * h)
// could be a symmetric neighbor of a particle inside rank q's box, whose
// largest radius is dom[q].w (the search's conservative node test).
__global__ void __launch_bounds__(256) k_halo_mask(const float *__restrict__ x,
                                                   const float *__restrict__ y,
                                                   const float *__restrict__ z,
                                                   const float *__restrict__ h, int64_t n,
                                                   PerLen L, float support,
                                                   const float4 *__restrict__ dom, int P, int self,
                                                   unsigned long long *__restrict__ mask)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 p = make_float4(x[i], y[i], z[i], 0.f);
    const float r = __fmul_rn(support, h[i]);
    unsigned long long m = 0;
    for (int q = 0; q < P; ++q) {
        if (q == self) continue;
        const float4 lo = dom[2 * q], hi = dom[2 * q + 1];
        if (!(lo.x <= hi.x)) continue;  // a rank without particles
        const bool near = (L.x < INFINITY || L.y < INFINITY || L.z < INFINITY)
                              ? point_near<true>(p, r, lo, hi, L)
                              : point_near<false>(p, r, lo, hi, L);
        if (near) m |= 1ull << q;
    }
    mask[i] = m;
}

__global__ void __launch_bounds__(256) k_mask_count(const unsigned long long *__restrict__ mask,
                                                    int64_t n, int P,
                                                    unsigned long long *__restrict__ counts)
{
    __shared__ unsigned sc[kMaxRanks];
    for (int q = threadIdx.x; q < P; q += blockDim.x) sc[q] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < n; i0 += stride) {
        const int64_t i = i0 + threadIdx.x;
        const unsigned long long m = i < n ? mask[i] : 0ull;
        for (int q = 0; q < P; ++q) {
            const unsigned b = __ballot_sync(0xffffffffu, (m >> q) & 1ull);
            if (lane_id() == 0 && b) atomicAdd(&sc[q], (unsigned)__popc(b));
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < P; q += blockDim.x)
        if (sc[q]) atomicAdd(&counts[q], (unsigned long long)sc[q]);
}

// Stable multi-split by destination bit: per tile of kGroupTile particles
// (thread t holds particles 4t..4t+3 of the tile), the count of each bit ...
__global__ void __launch_bounds__(kGroupThreads) k_group_tiles(const unsigned long long *__restrict__ mask,
                                                               int64_t n, int P,
                                                               unsigned *__restrict__ tile_cnt,
                                                               uint32_t ntiles)
{
    __shared__ unsigned sc[kMaxRanks];
    for (int q = threadIdx.x; q < P; q += blockDim.x) sc[q] = 0;
    __syncthreads();
    const int64_t i0 = (int64_t)blockIdx.x * kGroupTile + (int64_t)threadIdx.x * kGroupItems;
    unsigned long long m[kGroupItems];
#pragma unroll
    for (int k = 0; k < kGroupItems; ++k) m[k] = i0 + k < n ? mask[i0 + k] : 0ull;
    for (int q = 0; q < P; ++q) {
        unsigned c = 0;
#pragma unroll
        for (int k = 0; k < kGroupItems; ++k) c += (unsigned)((m[k] >> q) & 1ull);
        c = warp_sum(c);
        if (lane_id() == 0 && c) atomicAdd(&sc[q], c);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < P; q += blockDim.x) tile_cnt[(size_t)q * ntiles + blockIdx.x] = sc[q];
}

// ... an exclusive scan of those counts over the tiles of each destination
// (one block per destination) ...
__global__ void __launch_bounds__(1024) k_group_scan(unsigned *__restrict__ tile_cnt, uint32_t ntiles)
{
    __shared__ unsigned wsum[32];
    __shared__ unsigned carry;
    unsigned *row = tile_cnt + (size_t)blockIdx.x * ntiles;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t b0 = 0; b0 < ntiles; b0 += blockDim.x) {
        const uint32_t t = b0 + threadIdx.x;
        const unsigned v = t < ntiles ? row[t] : 0u;
        const unsigned incl = warp_incl_scan(v);
        if (lane_id() == 31) wsum[threadIdx.x >> 5] = incl;
        __syncthreads();
        if (threadIdx.x < 32) {
            const unsigned w = threadIdx.x < (blockDim.x >> 5) ? wsum[threadIdx.x] : 0u;
            wsum[threadIdx.x] = warp_incl_scan(w);
        }
        __syncthreads();
        const unsigned before = (threadIdx.x >= 32 ? wsum[(threadIdx.x >> 5) - 1] : 0u) + carry;
        if (t < ntiles) row[t] = before + incl - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = before + incl;
        __syncthreads();
    }
}

// ... and the scatter: particle i goes to offsets[q] + (tile base) + (rank of
// i among the tile's particles with bit q), for every bit q of its mask.
__global__ void __launch_bounds__(kGroupThreads) k_group_scatter(const unsigned long long *__restrict__ mask,
                                                                 int64_t n, int P,
                                                                 const unsigned *__restrict__ tile_base,
                                                                 uint32_t ntiles,
                                                                 const long long *__restrict__ offsets,
                                                                 uint32_t *__restrict__ idx)
{
    __shared__ unsigned wsum[kGroupThreads / 32];
    const int64_t i0 = (int64_t)blockIdx.x * kGroupTile + (int64_t)threadIdx.x * kGroupItems;
    unsigned long long m[kGroupItems];
#pragma unroll
    for (int k = 0; k < kGroupItems; ++k) m[k] = i0 + k < n ? mask[i0 + k] : 0ull;
    const unsigned warp = threadIdx.x >> 5;
    for (int q = 0; q < P; ++q) {
        unsigned c = 0;
#pragma unroll
        for (int k = 0; k < kGroupItems; ++k) c += (unsigned)((m[k] >> q) & 1ull);
        const unsigned incl = warp_incl_scan(c);
        __syncthreads();  // wsum of the previous destination has been read
        if (lane_id() == 31) wsum[warp] = incl;
        __syncthreads();
        unsigned before = 0;
        for (unsigned w = 0; w < warp; ++w) before += wsum[w];
        if (c) {
            unsigned long long pos = (unsigned long long)offsets[q] +
                                     tile_base[(size_t)q * ntiles + blockIdx.x] + before + incl - c;
#pragma unroll
            for (int k = 0; k < kGroupItems; ++k)
                if ((m[k] >> q) & 1ull) idx[pos++] = (uint32_t)(i0 + k);
        }
    }
}

unsigned grid_for(int64_t n, int per_block)
{
    const int64_t g = (n + per_block - 1) / per_block;
    return (unsigned)(g < 1 ? 1 : (g > 65535 * 16 ? 65535 * 16 : g));
}

}  // namespace

extern "C" nl_status nl_sfc_keys(const float *x, const float *y, const float *z, const float *h,
                                 int64_t n, const nl_box *box, int32_t key, float support,
                                 uint64_t *keys, void *stream)
{
    if (!x || !y || !z || !h || !box || !keys) return report_error(NL_ERR_ARG, "nl_sfc_keys: NULL argument");
    if (n < 0 || n > ((int64_t)1 << 31)) return report_error(NL_ERR_ARG, "nl_sfc_keys: need 0 <= n <= 2^31");
    if (key != NL_KEY_MORTON && key != NL_KEY_HILBERT)
        return report_error(NL_ERR_ARG, "nl_sfc_keys: unknown key kind");
    if (!(support > 0.f) || !(support < 3.0e38f))
        return report_error(NL_ERR_ARG, "nl_sfc_keys: support must be finite and > 0");
    if (!box_ok(box)) return report_error(NL_ERR_ARG, "nl_sfc_keys: need finite box lo < hi");
    if (n == 0) return NL_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const DevBox b = to_devbox(*box);
    Status *st = nullptr;
    uint32_t *vals = nullptr;
    cudaError_t e = cudaMallocAsync(&st, sizeof(Status), s);
    if (e == cudaSuccess) e = cudaMallocAsync(&vals, (size_t)n * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(st, 0, sizeof(Status), s);
    if (e == cudaSuccess) e = launch_keys(n, x, y, z, h, b, support, key, keys, vals, st, s);
    Status hs{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, st, sizeof(Status), cudaMemcpyDeviceToHost, s);
    if (vals) cudaFreeAsync(vals, s);
    if (st) cudaFreeAsync(st, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "nl_sfc_keys");
    if (hs.bad_input)
        return report_error(NL_ERR_ARG, "nl_sfc_keys: invalid particle input "
                                        "(non-finite or out-of-box coordinate, or h <= 0)");
    const float rmax = __builtin_bit_cast(float, hs.rmax_bits);
    for (int a = 0; a < 3; ++a)
        if (b.per[a] && !(rmax < b.half[a]))
            return report_error(NL_ERR_RADIUS, "nl_sfc_keys: support*max(h) >= L/2 on a periodic axis");
    return NL_OK;
}

extern "C" nl_status nl_key_histogram(const uint64_t *keys, int64_t n, uint64_t lo, int32_t shift,
                                      int32_t nbins, uint64_t *hist, void *stream)
{
    if (!hist || (n > 0 && !keys)) return report_error(NL_ERR_ARG, "nl_key_histogram: NULL argument");
    if (n < 0 || shift < 0 || shift > 63 || nbins < 1 || nbins > (1 << 24))
        return report_error(NL_ERR_ARG, "nl_key_histogram: need n >= 0, 0 <= shift <= 63, "
                                        "1 <= nbins <= 2^24");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(hist, 0, (size_t)nbins * 8, s);
    if (e == cudaSuccess && n > 0) {
        k_key_hist<<<grid_for(n, 256 * 8), 256, 0, s>>>(keys, n, lo, shift, (uint32_t)nbins,
                                                        reinterpret_cast<unsigned long long *>(hist));
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? NL_OK : cuda_fail(e, "nl_key_histogram");
}

extern "C" nl_status nl_domain_owner_mask(const uint64_t *keys, int64_t n, const uint64_t *splitters,
                                          int32_t P, uint64_t *mask, void *stream)
{
    if (P < 1 || P > kMaxRanks) return report_error(NL_ERR_ARG, "nl_domain_owner_mask: need 1 <= P <= 64");
    if (n < 0 || (n > 0 && (!keys || !mask)) || (P > 1 && !splitters))
        return report_error(NL_ERR_ARG, "nl_domain_owner_mask: bad argument");
    if (n == 0) return NL_OK;
    cudaStream_t s = (cudaStream_t)stream;
    k_owner_mask<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
        keys, n, splitters, P - 1, reinterpret_cast<unsigned long long *>(mask));
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? NL_OK : cuda_fail(e, "nl_domain_owner_mask");
}

extern "C" nl_status nl_domain_box(const float *x, const float *y, const float *z, const float *h,
                                   int64_t n, float support, float *out, void *stream)
{
    if (!out || n < 0 || (n > 0 && (!x || !y || !z || !h)))
        return report_error(NL_ERR_ARG, "nl_domain_box: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned *acc = nullptr;
    cudaError_t e = cudaMallocAsync(&acc, 8 * sizeof(unsigned), s);
    if (e == cudaSuccess) {
        k_box_init<<<1, 32, 0, s>>>(acc);
        if (n > 0) k_box_reduce<<<grid_for(n, 256 * 16), 256, 0, s>>>(x, y, z, h, n, support, acc);
        k_box_finish<<<1, 32, 0, s>>>(acc, n, out);
        e = cudaGetLastError();
        cudaFreeAsync(acc, s);
    }
    return e == cudaSuccess ? NL_OK : cuda_fail(e, "nl_domain_box");
}

extern "C" nl_status nl_domain_halo_mask(const float *x, const float *y, const float *z,
                                         const float *h, int64_t n, const nl_box *box, float support,
                                         const float *dom, int32_t P, int32_t self, uint64_t *mask,
                                         void *stream)
{
    if (!box || !dom || P < 1 || P > kMaxRanks || self < 0 || self >= P || n < 0 ||
        (n > 0 && (!x || !y || !z || !h || !mask)))
        return report_error(NL_ERR_ARG, "nl_domain_halo_mask: bad argument");
    if (!box_ok(box)) return report_error(NL_ERR_ARG, "nl_domain_halo_mask: need finite box lo < hi");
    if (reinterpret_cast<uintptr_t>(dom) % 16)
        return report_error(NL_ERR_ARG, "nl_domain_halo_mask: dom must be 16-byte aligned");
    if (n == 0) return NL_OK;
    const DevBox b = to_devbox(*box);
    cudaStream_t s = (cudaStream_t)stream;
    k_halo_mask<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
        x, y, z, h, n,
        PerLen{b.per[0] ? b.len[0] : INFINITY, b.per[1] ? b.len[1] : INFINITY,
               b.per[2] ? b.len[2] : INFINITY},
        support, reinterpret_cast<const float4 *>(dom), P, self,
        reinterpret_cast<unsigned long long *>(mask));
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? NL_OK : cuda_fail(e, "nl_domain_halo_mask");
}

extern "C" nl_status nl_domain_count(const uint64_t *mask, int64_t n, int32_t P, int64_t *counts,
                                     void *stream)
{
    if (!counts || P < 1 || P > kMaxRanks || n < 0 || (n > 0 && !mask))
        return report_error(NL_ERR_ARG, "nl_domain_count: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(counts, 0, (size_t)P * 8, s);
    if (e == cudaSuccess && n > 0) {
        k_mask_count<<<grid_for(n, 256 * 16), 256, 0, s>>>(
            reinterpret_cast<const unsigned long long *>(mask), n, P,
            reinterpret_cast<unsigned long long *>(counts));
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? NL_OK : cuda_fail(e, "nl_domain_count");
}

extern "C" nl_status nl_domain_group(const uint64_t *mask, int64_t n, int32_t P,
                                     const int64_t *offsets, uint32_t *idx, void *stream)
{
    if (!offsets || P < 1 || P > kMaxRanks || n < 0 || n > ((int64_t)1 << 32) ||
        (n > 0 && (!mask || !idx)))
        return report_error(NL_ERR_ARG, "nl_domain_group: bad argument");
    if (n == 0) return NL_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t ntiles = (uint32_t)((n + kGroupTile - 1) / kGroupTile);
    unsigned *tile = nullptr;
    cudaError_t e = cudaMallocAsync(&tile, (size_t)P * ntiles * sizeof(unsigned), s);
    if (e == cudaSuccess) {
        const auto *m = reinterpret_cast<const unsigned long long *>(mask);
        k_group_tiles<<<ntiles, kGroupThreads, 0, s>>>(m, n, P, tile, ntiles);
        k_group_scan<<<P, 1024, 0, s>>>(tile, ntiles);
        k_group_scatter<<<ntiles, kGroupThreads, 0, s>>>(
            m, n, P, tile, ntiles, reinterpret_cast<const long long *>(offsets), idx);
        e = cudaGetLastError();
        cudaFreeAsync(tile, s);
    }
    return e == cudaSuccess ? NL_OK : cuda_fail(e, "nl_domain_group");
}
