// SFC key generation with input validation, and a stable LSD radix sort of
// (key, index) pairs (Sec. II-A: particles in SFC order; stability makes
// equal keys keep their original order).
//
// Sort design (reduce-then-scan, no inter-CTA waiting): for each 8-bit
// digit, (1) every 4096-key tile counts its digits, (2) one CTA per digit
// scans the per-tile counts, (3) every tile ranks its keys stably with
// warp match + per-warp counters, reorders them in shared memory and writes
// each digit's run contiguously (coalesced).
#include "nl_internal.cuh"

namespace nlg {

// ---------------------------------------------------------------------------
// Keys + validation
// ---------------------------------------------------------------------------
template <int KIND>
__global__ void __launch_bounds__(256) k_keys(int64_t n, const float *__restrict__ x,
                                              const float *__restrict__ y,
                                              const float *__restrict__ z,
                                              const float *__restrict__ h, DevBox b, float support,
                                              uint64_t *__restrict__ keys,
                                              uint32_t *__restrict__ vals, Status *st)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned bad = 0;
    float r = 0.f;
    if (i < n) {
        float px = x[i], py = y[i], pz = z[i], ph = h[i];
        if (!isfinite(px) || !isfinite(py) || !isfinite(pz)) bad |= 1u;
        if (!(px >= b.lo[0] && px <= b.hi[0] && py >= b.lo[1] && py <= b.hi[1] &&
              pz >= b.lo[2] && pz <= b.hi[2]))
            bad |= 2u;
        if (!(ph > 0.f) || !isfinite(ph)) bad |= 4u;
        r = __fmul_rn(support, ph);
        if (!(r >= 0.f) || !isfinite(r)) r = 0.f;
        uint32_t qx = quantize21(px, b.lo[0], b.qs[0]);
        uint32_t qy = quantize21(py, b.lo[1], b.qs[1]);
        uint32_t qz = quantize21(pz, b.lo[2], b.qs[2]);
        keys[i] = KIND == NL_KEY_MORTON ? morton_key(qx, qy, qz) : hilbert_key(qx, qy, qz);
        vals[i] = (uint32_t)i;
    }
    // block reductions: OR of flags, max radius
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
        r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, o));
    }
    __shared__ unsigned sb[8];
    __shared__ float sr[8];
    if (lane_id() == 0) {
        sb[threadIdx.x >> 5] = bad;
        sr[threadIdx.x >> 5] = r;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            bad |= sb[w];
            r = fmaxf(r, sr[w]);
        }
        if (bad) atomicOr(&st->bad_input, bad);
        atomicMax(&st->rmax_bits, __float_as_uint(r));
    }
}

cudaError_t launch_keys(int64_t n, const float *x, const float *y, const float *z, const float *h,
                        const DevBox &box, float support, int kind, uint64_t *keys, uint32_t *vals,
                        Status *st, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    unsigned grid = (unsigned)((n + 255) / 256);
    if (kind == NL_KEY_MORTON)
        k_keys<NL_KEY_MORTON><<<grid, 256, 0, s>>>(n, x, y, z, h, box, support, keys, vals, st);
    else
        k_keys<NL_KEY_HILBERT><<<grid, 256, 0, s>>>(n, x, y, z, h, box, support, keys, vals, st);
    return cudaGetLastError();
}

template <int KIND>
__global__ void __launch_bounds__(256) k_keys_batch(int64_t n, const float *__restrict__ x,
                                                    const float *__restrict__ y,
                                                    const float *__restrict__ z,
                                                    const float *__restrict__ h, SysTables t,
                                                    float support, uint64_t *__restrict__ keys,
                                                    uint32_t *__restrict__ vals, Status *st)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned bad = 0;
    if (i < n) {
        const DevBox &b = t.box[sys_of(t.off, t.nsys, (uint32_t)i)];
        float px = x[i], py = y[i], pz = z[i], ph = h[i];
        if (!isfinite(px) || !isfinite(py) || !isfinite(pz)) bad |= 1u;
        if (!(px >= b.lo[0] && px <= b.hi[0] && py >= b.lo[1] && py <= b.hi[1] &&
              pz >= b.lo[2] && pz <= b.hi[2]))
            bad |= 2u;
        if (!(ph > 0.f) || !isfinite(ph)) bad |= 4u;
        // a search radius reaching half a periodic box length is reported
        float r = __fmul_rn(support, ph);
        for (int a = 0; a < 3; ++a)
            if (b.per[a] && !(r < b.half[a])) bad |= 8u;
        uint32_t qx = quantize21(px, b.lo[0], b.qs[0]);
        uint32_t qy = quantize21(py, b.lo[1], b.qs[1]);
        uint32_t qz = quantize21(pz, b.lo[2], b.qs[2]);
        keys[i] = KIND == NL_KEY_MORTON ? morton_key(qx, qy, qz) : hilbert_key(qx, qy, qz);
        vals[i] = (uint32_t)i;
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    if (lane_id() == 0 && bad) atomicOr(&st->bad_input, bad);
}

cudaError_t launch_keys_batch(int64_t n, const float *x, const float *y, const float *z,
                              const float *h, const SysTables &t, float support, int kind,
                              uint64_t *keys, uint32_t *vals, Status *st, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    unsigned grid = (unsigned)((n + 255) / 256);
    if (kind == NL_KEY_MORTON)
        k_keys_batch<NL_KEY_MORTON><<<grid, 256, 0, s>>>(n, x, y, z, h, t, support, keys, vals, st);
    else
        k_keys_batch<NL_KEY_HILBERT><<<grid, 256, 0, s>>>(n, x, y, z, h, t, support, keys, vals, st);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Radix sort
// ---------------------------------------------------------------------------
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;  // 4096 keys
constexpr int RS_WARP_SPAN = 32 * RS_ITEMS;     // 512 consecutive keys per warp

static uint32_t rs_tiles(uint32_t n) { return (n + RS_TILE - 1) / RS_TILE; }

size_t radix_hist_words(uint32_t n) { return (size_t)256 * rs_tiles(n) + 256; }

// Digit of an element: 8 key bits, or 8 bits of the system owning the value
// (a caller index) for the final by-system passes.
struct DigitSrc {
    const uint32_t *sys_off;  // NULL: key digits
    uint32_t nsys;
    __device__ __forceinline__ uint32_t operator()(uint64_t key, uint32_t val, int shift) const
    {
        if (!sys_off) return (unsigned)(key >> shift) & 0xffu;
        return (sys_of(sys_off, nsys, val) >> shift) & 0xffu;
    }
};

// Per-tile digit counts, digit-major: hist[d * ntiles + tile].
__global__ void __launch_bounds__(RS_THREADS) k_rs_upsweep_sys(const uint32_t *__restrict__ vals,
                                                               uint32_t n, int shift, DigitSrc dg,
                                                               uint32_t *__restrict__ hist,
                                                               uint32_t ntiles)
{
    __shared__ uint32_t cnt[RS_WARPS][256];
    for (int t = threadIdx.x; t < RS_WARPS * 256; t += RS_THREADS) (&cnt[0][0])[t] = 0;
    __syncthreads();
    const uint32_t base = blockIdx.x * RS_TILE;
    const int warp = threadIdx.x >> 5;
    for (int it = 0; it < RS_ITEMS; ++it) {
        uint32_t k = base + it * RS_THREADS + threadIdx.x;
        if (k < n) atomicAdd(&cnt[warp][dg(0ull, vals[k], shift)], 1u);
    }
    __syncthreads();
    const int d = threadIdx.x;
    uint32_t sum = 0;
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) sum += cnt[w][d];
    hist[(size_t)d * ntiles + blockIdx.x] = sum;
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_upsweep(const uint64_t *__restrict__ keys,
                                                           uint32_t n, int shift,
                                                           uint32_t *__restrict__ hist,
                                                           uint32_t ntiles)
{
    __shared__ uint32_t cnt[RS_WARPS][256];
    for (int t = threadIdx.x; t < RS_WARPS * 256; t += RS_THREADS) (&cnt[0][0])[t] = 0;
    __syncthreads();
    const uint32_t base = blockIdx.x * RS_TILE;
    const int warp = threadIdx.x >> 5;
#pragma unroll 4
    for (int it = 0; it < RS_ITEMS; ++it) {
        uint32_t k = base + it * RS_THREADS + threadIdx.x;
        if (k < n) atomicAdd(&cnt[warp][(unsigned)(keys[k] >> shift) & 0xffu], 1u);
    }
    __syncthreads();
    const int d = threadIdx.x;
    uint32_t sum = 0;
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) sum += cnt[w][d];
    hist[(size_t)d * ntiles + blockIdx.x] = sum;
}

// One CTA per digit: exclusive scan over tiles in place; the digit total
// goes to tot[d].
__global__ void __launch_bounds__(1024) k_rs_scan(uint32_t *__restrict__ hist, uint32_t ntiles,
                                                  uint32_t *__restrict__ tot)
{
    __shared__ uint32_t sh[33];
    uint32_t *row = hist + (size_t)blockIdx.x * ntiles;
    uint32_t carry = 0;
    for (uint32_t b = 0; b < ntiles; b += 1024) {
        uint32_t i = b + threadIdx.x;
        uint32_t v = i < ntiles ? row[i] : 0u;
        uint32_t t;
        uint32_t e = block_excl_scan(v, sh, &t);
        if (i < ntiles) row[i] = carry + e;
        carry += t;
    }
    if (threadIdx.x == 0) tot[blockIdx.x] = carry;
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_downsweep(
    const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint64_t *__restrict__ kout,
    uint32_t *__restrict__ vout, uint32_t n, int shift, const uint32_t *__restrict__ hist,
    const uint32_t *__restrict__ tot, uint32_t ntiles, DigitSrc dg)
{
    extern __shared__ __align__(16) unsigned char rs_smem[];
    uint64_t *skeys = reinterpret_cast<uint64_t *>(rs_smem);
    uint32_t *svals = reinterpret_cast<uint32_t *>(skeys + RS_TILE);
    uint32_t(*wcnt)[256] = reinterpret_cast<uint32_t(*)[256]>(svals + RS_TILE);
    uint32_t *tstart = &wcnt[RS_WARPS][0];   // 256
    uint32_t *gbase = tstart + 256;          // 256
    uint32_t *sh = gbase + 256;              // 33

    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    const uint32_t base = blockIdx.x * RS_TILE;
    const uint32_t tile_n = min((uint32_t)RS_TILE, n - base);
    for (int t = threadIdx.x; t < RS_WARPS * 256; t += RS_THREADS) (&wcnt[0][0])[t] = 0;
    __syncthreads();

    uint64_t key[RS_ITEMS];
    uint32_t val[RS_ITEMS], rank[RS_ITEMS];
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int it = 0; it < RS_ITEMS; ++it) {
        uint32_t k = base + warp * RS_WARP_SPAN + it * 32 + lane;
        bool valid = k < n;
        key[it] = valid ? kin[k] : 0ull;
        val[it] = valid ? vin[k] : 0u;
        uint32_t d = valid ? dg(key[it], val[it], shift) : 256u;
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t before = d < 256u ? wcnt[warp][d] : 0u;
        rank[it] = before + __popc(peers & lt);
        __syncwarp();
        if (d < 256u && lane == (unsigned)(__ffs(peers) - 1)) wcnt[warp][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive prefix over warps, tile-local digit start, and the
    // global base of this tile's run of the digit
    {
        const int d = threadIdx.x;
        uint32_t s = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) {
            uint32_t c = wcnt[w][d];
            wcnt[w][d] = s;
            s += c;
        }
        uint32_t dummy;
        uint32_t ts = block_excl_scan(s, sh, &dummy);
        uint32_t dp = block_excl_scan(tot[d], sh, &dummy);
        tstart[d] = ts;
        gbase[d] = dp + hist[(size_t)d * ntiles + blockIdx.x] - ts;
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < RS_ITEMS; ++it) {
        uint32_t k = base + warp * RS_WARP_SPAN + it * 32 + lane;
        if (k < n) {
            uint32_t d = dg(key[it], val[it], shift);
            uint32_t lp = tstart[d] + wcnt[warp][d] + rank[it];
            skeys[lp] = key[it];
            svals[lp] = val[it];
        }
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < tile_n; t += RS_THREADS) {
        uint64_t kk = skeys[t];
        uint32_t vv = svals[t];
        uint32_t d = dg(kk, vv, shift);
        uint32_t g = gbase[d] + t;
        kout[g] = kk;
        vout[g] = vv;
    }
}

static size_t rs_down_smem()
{
    return (size_t)RS_TILE * 8 + (size_t)RS_TILE * 4 + (size_t)RS_WARPS * 256 * 4 + 256 * 4 * 2 +
           33 * 4;
}

cudaError_t radix_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt,
                             uint32_t n, int bits, uint32_t *hist, cudaStream_t s)
{
    if (n <= 1) return cudaSuccess;
    cudaError_t e = set_max_dynamic_smem((const void *)k_rs_downsweep, rs_down_smem());
    if (e != cudaSuccess) return e;
    const uint32_t ntiles = rs_tiles(n);
    uint32_t *tot = hist + (size_t)256 * ntiles;
    uint64_t *ka = keys, *kb = keys_alt;
    uint32_t *va = vals, *vb = vals_alt;
    int passes = (bits + 7) / 8;
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        k_rs_upsweep<<<ntiles, RS_THREADS, 0, s>>>(ka, n, shift, hist, ntiles);
        k_rs_scan<<<256, 1024, 0, s>>>(hist, ntiles, tot);
        k_rs_downsweep<<<ntiles, RS_THREADS, rs_down_smem(), s>>>(ka, va, kb, vb, n, shift, hist,
                                                                 tot, ntiles, DigitSrc{nullptr, 0});
        uint64_t *tk = ka; ka = kb; kb = tk;
        uint32_t *tv = va; va = vb; vb = tv;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ka != keys) {
        // odd number of passes: copy back
        e = cudaMemcpyAsync(keys, ka, (size_t)n * 8, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(vals, va, (size_t)n * 4, cudaMemcpyDeviceToDevice, s);
    }
    return e;
}

cudaError_t radix_sort_by_system(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt,
                                 uint32_t *vals_alt, uint32_t n, const uint32_t *sys_off,
                                 uint32_t nsys, uint32_t *hist, cudaStream_t s)
{
    if (n <= 1 || nsys <= 1) return cudaSuccess;
    cudaError_t e = set_max_dynamic_smem((const void *)k_rs_downsweep, rs_down_smem());
    if (e != cudaSuccess) return e;
    const uint32_t ntiles = rs_tiles(n);
    uint32_t *tot = hist + (size_t)256 * ntiles;
    const DigitSrc dg{sys_off, nsys};
    const int passes = nsys <= 256 ? 1 : (nsys <= 65536 ? 2 : 3);
    uint64_t *ka = keys, *kb = keys_alt;
    uint32_t *va = vals, *vb = vals_alt;
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        k_rs_upsweep_sys<<<ntiles, RS_THREADS, 0, s>>>(va, n, shift, dg, hist, ntiles);
        k_rs_scan<<<256, 1024, 0, s>>>(hist, ntiles, tot);
        k_rs_downsweep<<<ntiles, RS_THREADS, rs_down_smem(), s>>>(ka, va, kb, vb, n, shift, hist,
                                                                 tot, ntiles, dg);
        uint64_t *tk = ka; ka = kb; kb = tk;
        uint32_t *tv = va; va = vb; vb = tv;
    }
    e = cudaGetLastError();
    if (e == cudaSuccess && ka != keys) {
        e = cudaMemcpyAsync(keys, ka, (size_t)n * 8, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(vals, va, (size_t)n * 4, cudaMemcpyDeviceToDevice, s);
    }
    return e;
}

}  // namespace nlg
