// SFC key generation with input validation, and a stable LSD radix sort of
// (key, index) pairs (Sec. II-A: particles in SFC order; stability makes
// equal keys keep their original order).
//
// Sort design (one read and one write of the pairs per 8-bit digit): one
// kernel counts every digit of every pass up front and a second scans the
// counts into digit starts; then one kernel per digit takes 5120-pair tiles
// in launch order, ranks each tile's pairs stably (warp ballots + per-warp
// counters), publishes its digit counts, finds the counts of all earlier
// tiles by a chained scan over their published words (decoupled look-back,
// a bounded wait), reorders the tile in shared memory and writes each
// digit's run contiguously.
#include <algorithm>

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

// ghist (optional): the digit counts of all eight 8-bit passes of the key
// sort that follows are added there (ghist[p * 256 + d]), so the sort does
// not read the keys once more to count them.  The grid then strides over
// the particles and each block adds its counts once.
template <int KIND, bool HIST>
__global__ void __launch_bounds__(256) k_keys_batch(int64_t n, const float *__restrict__ x,
                                                    const float *__restrict__ y,
                                                    const float *__restrict__ z,
                                                    const float *__restrict__ h, SysTables t,
                                                    float support, uint64_t *__restrict__ keys,
                                                    uint32_t *__restrict__ vals, Status *st,
                                                    uint32_t *__restrict__ ghist)
{
    __shared__ uint32_t hs[HIST ? 8 * 256 : 1];
    if constexpr (HIST) {
        for (int q = threadIdx.x; q < 8 * 256; q += blockDim.x) hs[q] = 0;
        __syncthreads();
    }
    unsigned bad = 0;
    const int64_t step = HIST ? (int64_t)gridDim.x * blockDim.x : n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += step) {
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
        const uint64_t key = KIND == NL_KEY_MORTON ? morton_key(qx, qy, qz) : hilbert_key(qx, qy, qz);
        keys[i] = key;
        vals[i] = (uint32_t)i;
        if constexpr (HIST) {
#pragma unroll
            for (int p = 0; p < 8; ++p) atomicAdd(&hs[p * 256 + ((unsigned)(key >> (8 * p)) & 0xffu)], 1u);
        }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    if (lane_id() == 0 && bad) atomicOr(&st->bad_input, bad);
    if constexpr (HIST) {
        __syncthreads();
        for (int q = threadIdx.x; q < 8 * 256; q += blockDim.x)
            if (hs[q]) atomicAdd(&ghist[q], hs[q]);
    }
}

cudaError_t launch_keys_batch(int64_t n, const float *x, const float *y, const float *z,
                              const float *h, const SysTables &t, float support, int kind,
                              uint64_t *keys, uint32_t *vals, Status *st, uint32_t *ghist,
                              cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (ghist) {
        const unsigned grid = std::min(blocks, 152u * 8u);
        if (kind == NL_KEY_MORTON)
            k_keys_batch<NL_KEY_MORTON, true><<<grid, 256, 0, s>>>(n, x, y, z, h, t, support, keys, vals, st, ghist);
        else
            k_keys_batch<NL_KEY_HILBERT, true><<<grid, 256, 0, s>>>(n, x, y, z, h, t, support, keys, vals, st, ghist);
    } else if (kind == NL_KEY_MORTON) {
        k_keys_batch<NL_KEY_MORTON, false><<<blocks, 256, 0, s>>>(n, x, y, z, h, t, support, keys, vals, st, nullptr);
    } else {
        k_keys_batch<NL_KEY_HILBERT, false><<<blocks, 256, 0, s>>>(n, x, y, z, h, t, support, keys, vals, st, nullptr);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Radix sort
// ---------------------------------------------------------------------------
constexpr int RS_THREADS = 512;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 10;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;  // 5120 pairs
constexpr int RS_WARP_SPAN = 32 * RS_ITEMS;     // 320 consecutive pairs per warp
constexpr int RS_R = 256;                       // 8-bit digits
constexpr int RS_MAXP = 8;                      // passes for 64 key bits
constexpr int RS_LOOK = 4;                      // earlier tiles read per look-back round trip
constexpr uint32_t RS_AGG = 1u << 30;           // status word: this tile's count is published
constexpr uint32_t RS_PRE = 2u << 30;           // ... the inclusive prefix is published
constexpr uint32_t RS_CNT = RS_AGG - 1u;
constexpr uint32_t RS_SPIN_LIMIT = 1u << 22;    // look-back polls before giving up

static uint32_t rs_tiles(uint32_t n) { return (n + RS_TILE - 1) / RS_TILE; }

// Scratch words: digit starts (RS_MAXP x 256), tile tickets (64), and one
// status word per (pass, tile, digit).
size_t radix_hist_words(uint32_t n)
{
    return (size_t)RS_MAXP * RS_R + 64 + (size_t)RS_MAXP * rs_tiles(n) * RS_R;
}

// Digit of an element: 8 key bits, or 8 bits of the system owning the value
// (a caller index) for the final by-system passes.
template <bool SYS>
struct DigitSrc {
    const uint32_t *sys_off;  // SYS: system offsets of the caller indices
    uint32_t nsys;
    __device__ __forceinline__ uint32_t operator()(uint64_t key, uint32_t val, int shift) const
    {
        if constexpr (!SYS) return (unsigned)(key >> shift) & 0xffu;
        return (sys_of(sys_off, nsys, val) >> shift) & 0xffu;
    }
};

__device__ __forceinline__ uint32_t ld_relaxed_gpu(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_gpu(uint32_t *p, uint32_t v)
{
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Counts of every digit of every pass: ghist[p * 256 + d] (eight pairs per
// thread and round, their loads issued together).
template <bool SYS>
__global__ void __launch_bounds__(256) k_rs_hist(const uint64_t *__restrict__ keys,
                                                 const uint32_t *__restrict__ vals, uint32_t n,
                                                 int passes, DigitSrc<SYS> dg, uint32_t *__restrict__ ghist)
{
    __shared__ uint32_t hs[RS_MAXP * RS_R];
    for (int t = threadIdx.x; t < passes * RS_R; t += blockDim.x) hs[t] = 0;
    __syncthreads();
    const uint32_t step = gridDim.x * blockDim.x * 8u;
    for (uint32_t b = blockIdx.x * blockDim.x * 8u + threadIdx.x; b < n; b += step) {
        uint64_t k[8];
        uint32_t v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const uint32_t i = b + u * blockDim.x;
            k[u] = (!SYS && i < n) ? keys[i] : 0ull;
            v[u] = (SYS && i < n) ? vals[i] : 0u;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (b + u * blockDim.x >= n) continue;
            for (int p = 0; p < passes; ++p) atomicAdd(&hs[p * RS_R + dg(k[u], v[u], 8 * p)], 1u);
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < passes * RS_R; t += blockDim.x)
        if (hs[t]) atomicAdd(&ghist[t], hs[t]);
}

// Digit starts: exclusive scan of each pass's 256 counts (one block per pass).
__global__ void __launch_bounds__(RS_R) k_rs_starts(uint32_t *ghist)
{
    __shared__ uint32_t sh[33];
    uint32_t *row = ghist + blockIdx.x * RS_R;
    uint32_t tot;
    const uint32_t e = block_excl_scan(row[threadIdx.x], sh, &tot);
    row[threadIdx.x] = e;
}

static size_t rs_pass_smem()
{
    return (size_t)RS_TILE * 12 + (size_t)RS_WARPS * RS_R * 4 + (size_t)RS_R * 8 + 64 * 4;
}

// One digit pass.  Tiles are numbered in the order their blocks start
// (ticket), so a tile waits only on tiles that are already running, and each
// of those publishes its counts before it waits on anything itself.
template <bool SYS>
__global__ void __launch_bounds__(RS_THREADS, 2) k_rs_pass(
    const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint64_t *__restrict__ kout,
    uint32_t *__restrict__ vout, uint32_t n, int shift, DigitSrc<SYS> dg,
    const uint32_t *__restrict__ gstart, uint32_t *status, uint32_t *ticket, unsigned int *stall)
{
    extern __shared__ __align__(16) unsigned char rs_smem[];
    uint64_t *skeys = reinterpret_cast<uint64_t *>(rs_smem);
    uint32_t *svals = reinterpret_cast<uint32_t *>(skeys + RS_TILE);
    uint32_t(*wc)[RS_R] = reinterpret_cast<uint32_t(*)[RS_R]>(svals + RS_TILE);
    uint32_t *dpre = &wc[RS_WARPS][0];  // tile-local start of each digit
    uint32_t *goff = dpre + RS_R;       // output index of tile slot 0 for each digit
    uint32_t *sh = goff + RS_R;         // scan words, tile number

    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) sh[40] = atomicAdd(ticket, 1u);
    for (int t = threadIdx.x; t < RS_WARPS * RS_R; t += RS_THREADS) (&wc[0][0])[t] = 0;
    __syncthreads();
    const uint32_t tile = sh[40];
    const uint32_t base = tile * RS_TILE;
    const uint32_t tile_n = min((uint32_t)RS_TILE, n - base);

    uint64_t key[RS_ITEMS];
    uint32_t val[RS_ITEMS], rank[RS_ITEMS];
#pragma unroll
    for (int it = 0; it < RS_ITEMS; ++it) {
        const uint32_t k = base + warp * RS_WARP_SPAN + it * 32 + lane;
        key[it] = k < n ? kin[k] : 0ull;
        val[it] = k < n ? vin[k] : 0u;
    }
    // stable rank within the warp: lanes holding the same digit found by one
    // ballot per digit bit; the leader of each group adds the group's size to
    // the warp's counter (a warp's atomics on one word apply in issue order)
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int it = 0; it < RS_ITEMS; ++it) {
        const uint32_t k = base + warp * RS_WARP_SPAN + it * 32 + lane;
        const bool valid = k < n;
        const uint32_t d = valid ? dg(key[it], val[it], shift) : 0u;
        const uint32_t vb = __ballot_sync(0xffffffffu, valid);
        uint32_t peers = valid ? vb : ~vb;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const bool bit = (d >> b) & 1u;
            const uint32_t bb = __ballot_sync(0xffffffffu, bit);
            peers &= bit ? bb : ~bb;
        }
        const int leader = __ffs(peers) - 1;
        uint32_t old = 0;
        if (valid && lane == (unsigned)leader) old = atomicAdd(&wc[warp][d], (uint32_t)__popc(peers));
        rank[it] = __shfl_sync(0xffffffffu, old, leader) + __popc(peers & lt);
    }
    __syncthreads();
    // per digit (threads 0..255): exclusive over warps, the tile's count,
    // published at once; then the tile-local digit starts
    uint32_t cnt = 0;
    const int d = threadIdx.x;
    if (d < RS_R) {
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) {
            const uint32_t c = wc[w][d];
            wc[w][d] = cnt;
            cnt += c;
        }
        st_relaxed_gpu(&status[(size_t)tile * RS_R + d], (tile == 0 ? RS_PRE : RS_AGG) | cnt);
    }
    uint32_t tot;
    const uint32_t ex = block_excl_scan(cnt, sh, &tot);
    if (d < RS_R) {
        // look-back: sum the counts of earlier tiles back to the nearest
        // published prefix, RS_LOOK words per round trip; a window with a
        // word still unpublished is read again (bounded)
        uint32_t sum = 0;
        if (tile > 0) {
            int32_t t = (int32_t)tile - 1;
            uint32_t spins = 0;
            for (;;) {
                uint32_t v[RS_LOOK];
#pragma unroll
                for (int q = 0; q < RS_LOOK; ++q)
                    v[q] = t - q >= 0 ? ld_relaxed_gpu(&status[(size_t)(t - q) * RS_R + d]) : RS_PRE;
                uint32_t part = 0;
                bool done = false, missing = false;
#pragma unroll
                for (int q = 0; q < RS_LOOK; ++q) {
                    if (done || missing) continue;
                    const uint32_t f = v[q] & ~RS_CNT;
                    if (f == 0u) {
                        missing = true;
                        continue;
                    }
                    part += v[q] & RS_CNT;
                    done = f == RS_PRE;
                }
                if (missing) {
                    if (++spins > RS_SPIN_LIMIT) {
                        atomicExch(stall, 1u);
                        break;
                    }
                    if (spins > 32u) __nanosleep(100);
                    continue;
                }
                sum += part;
                if (done) break;
                t -= RS_LOOK;
            }
            st_relaxed_gpu(&status[(size_t)tile * RS_R + d], RS_PRE | (sum + cnt));
        }
        dpre[d] = ex;
        goff[d] = gstart[d] + sum - ex;
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < RS_ITEMS; ++it) {
        const uint32_t k = base + warp * RS_WARP_SPAN + it * 32 + lane;
        if (k < n) {
            const uint32_t dd = dg(key[it], val[it], shift);
            const uint32_t lp = dpre[dd] + wc[warp][dd] + rank[it];
            skeys[lp] = key[it];
            svals[lp] = val[it];
        }
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < tile_n; t += RS_THREADS) {
        const uint64_t kk = skeys[t];
        const uint32_t vv = svals[t];
        const uint32_t g = goff[dg(kk, vv, shift)] + t;
        if (g < n) {  // always, unless a look-back gave up (reported in *stall)
            kout[g] = kk;
            vout[g] = vv;
        }
    }
}

// passes of 8 bits with digits from dg; keys/vals end in the input arrays
template <bool SYS>
static cudaError_t rs_run(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt,
                          uint32_t n, int passes, DigitSrc<SYS> dg, uint32_t *scratch,
                          unsigned int *stall, bool counted, cudaStream_t s)
{
    cudaError_t e = set_max_dynamic_smem((const void *)k_rs_pass<SYS>, rs_pass_smem());
    if (e != cudaSuccess) return e;
    const uint32_t ntiles = rs_tiles(n);
    uint32_t *ghist = scratch, *tickets = scratch + RS_MAXP * RS_R;
    uint32_t *status = tickets + 64;
    if (!counted) {
        e = radix_sort_clear(scratch, n, 8 * passes, s);
        if (e != cudaSuccess) return e;
        const uint32_t hgrid = min((n + 2047u) / 2048u, 152u * 8u);
        k_rs_hist<SYS><<<hgrid, 256, 0, s>>>(keys, vals, n, passes, dg, ghist);
    }
    k_rs_starts<<<passes, RS_R, 0, s>>>(ghist);
    uint64_t *ka = keys, *kb = keys_alt;
    uint32_t *va = vals, *vb = vals_alt;
    for (int p = 0; p < passes; ++p) {
        k_rs_pass<SYS><<<ntiles, RS_THREADS, rs_pass_smem(), s>>>(ka, va, kb, vb, n, 8 * p, dg,
                                                            ghist + p * RS_R,
                                                            status + (size_t)p * ntiles * RS_R,
                                                            tickets + p, stall);
        uint64_t *tk = ka; ka = kb; kb = tk;
        uint32_t *tv = va; va = vb; vb = tv;
    }
    e = cudaGetLastError();
    if (e == cudaSuccess && ka != keys) {
        // odd number of passes: copy back
        e = cudaMemcpyAsync(keys, ka, (size_t)n * 8, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(vals, va, (size_t)n * 4, cudaMemcpyDeviceToDevice, s);
    }
    return e;
}

cudaError_t radix_sort_clear(uint32_t *hist, uint32_t n, int bits, cudaStream_t s)
{
    const int passes = min((bits + 7) / 8, RS_MAXP);
    return cudaMemsetAsync(hist, 0, (RS_MAXP * RS_R + 64 + (size_t)passes * rs_tiles(n) * RS_R) * 4, s);
}

cudaError_t radix_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt,
                             uint32_t n, int bits, uint32_t *hist, unsigned int *stall, cudaStream_t s,
                             bool counted)
{
    if (n <= 1) return cudaSuccess;
    const int passes = min((bits + 7) / 8, RS_MAXP);
    return rs_run(keys, vals, keys_alt, vals_alt, n, passes, DigitSrc<false>{nullptr, 0}, hist, stall,
                  counted, s);
}

cudaError_t radix_sort_by_system(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt,
                                 uint32_t *vals_alt, uint32_t n, const uint32_t *sys_off,
                                 uint32_t nsys, uint32_t *hist, unsigned int *stall, cudaStream_t s)
{
    if (n <= 1 || nsys <= 1) return cudaSuccess;
    const int passes = nsys <= 256 ? 1 : (nsys <= 65536 ? 2 : 3);
    return rs_run(keys, vals, keys_alt, vals_alt, n, passes, DigitSrc<true>{sys_off, nsys}, hist, stall,
                  false, s);
}

}  // namespace nlg
