// Internal declarations of the sm_103a neighbor-list library (not installed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nl.h"

namespace nlg {

constexpr int kKeyBits = 21;         // bits per axis of the 63-bit SFC key
constexpr int kMaxLevel = 21;        // deepest octree level
constexpr int kSC = 8;               // clusters per super-cluster (8-bit masks, Sec. II-A)
constexpr uint32_t kBadRecord = 0xffffffffu;

// Box with the derived FP32 quantities every kernel uses.  len = hi - lo,
// half = 0.5f * len, qs = 2^21 / len, all rounded to nearest in FP32.
struct DevBox {
    float lo[3], hi[3], len[3], half[3], qs[3];
    int per[3];
};

// Tables of a batch of independent systems (a single system is a batch of
// one).  Caller arrays hold the systems back to back: system s owns caller
// (and, after the sort, sorted) indices [off[s], off[s+1]).  In SFC-sorted
// padded order every system starts on a super-cluster boundary: system s
// owns padded indices [pad_off[s], pad_off[s+1]), the tail filled with NaN
// dummies.  root[s] is the index of the system's octree root.
struct SysTables {
    const uint32_t *off;
    const uint32_t *pad_off;
    const DevBox *box;
    uint32_t *root;
    uint32_t nsys;
};

// system owning index k of an offset table t (t[0] = 0, t[nsys] = total)
__device__ __forceinline__ uint32_t sys_of(const uint32_t *t, uint32_t nsys, uint32_t k)
{
    uint32_t lo = 0, hi = nsys;  // invariant: t[lo] <= k < t[hi]
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (t[mid] <= k) lo = mid; else hi = mid;
    }
    return lo;
}

// Device status words written by the build kernels and read back once.
struct Status {
    // build words (keys, octree)
    unsigned int bad_input;   // bit0 non-finite coordinate, bit1 outside box, bit2 bad h,
                              // bit3 radius >= L/2 on a periodic axis
    unsigned int rmax_bits;   // max over particles of support*h (FP32 bits, >= 0)
    unsigned int n_leaves;
    unsigned int n_nodes;
    unsigned int node_overflow;  // nodes beyond the preallocated capacity (graph replays)
    unsigned int sort_stall;     // a radix-sort look-back gave up its bounded wait
    unsigned int pad0[2];
    // search words (reset before every search); ticket is the first of them
    unsigned int ticket;      // work counter of persistent kernels
    unsigned int stage_overflow;
    unsigned int max_count;   // longest super-cluster list seen when staging overflowed
    unsigned int list_overflow;
    unsigned long long list_used;  // bytes reserved in the list buffer
    unsigned long long n_entries;
    unsigned long long n_tiles;
    unsigned int pass_ticket;
    unsigned int pad;
    unsigned long long fail_off;   // lowest failed list reservation (host sets ~0 first)
    // search work counters
    unsigned long long node_visits;
    unsigned long long leaf_visits;
    unsigned long long j_examined;     // j-clusters box-tested against the 8 i-clusters
    unsigned long long tile_tests;     // (i-cluster, j-cluster) tiles decided by the exact predicate
    // half search (symmetric lists): reservations in the upper-entry and
    // transposed-tuple buffers (counted even when they do not fit)
    unsigned long long up_used;
    unsigned long long tu_used;
    unsigned int half_overflow;        // some reservation did not fit
    unsigned int asm_ticket;           // work counter of the record assembly
    unsigned int seg_total;            // total of the lower-entry scan
    unsigned int pad2;
    // periodic super-clusters whose neighbors cannot wrap (interior) and the rest
    unsigned int n_int, n_bnd;
    // half-list density: bits of the largest |m| (sets the fixed-point scale)
    unsigned int m_absmax, pad3;
};

// ---------------------------------------------------------------------------
// The canonical FP32 pair arithmetic (no FMA contraction anywhere).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float wrap_axis(float d, float len, float half, int per)
{
    if (per) {
        if (d > half)
            d = __fsub_rn(d, len);
        else if (d < -half)
            d = __fadd_rn(d, len);
    }
    return d;
}

template <bool PER>
__device__ __forceinline__ float pair_d2(const float4 &pi, const float4 &pj, const DevBox &b)
{
    float dx = __fsub_rn(pj.x, pi.x);
    float dy = __fsub_rn(pj.y, pi.y);
    float dz = __fsub_rn(pj.z, pi.z);
    if (PER) {
        dx = wrap_axis(dx, b.len[0], b.half[0], b.per[0]);
        dy = wrap_axis(dy, b.len[1], b.half[1], b.per[1]);
        dz = wrap_axis(dz, b.len[2], b.half[2], b.per[2]);
    }
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

template <bool PER>
__device__ __forceinline__ float3 pair_dx(const float4 &pi, const float4 &pj, const DevBox &b)
{
    float dx = __fsub_rn(pj.x, pi.x);
    float dy = __fsub_rn(pj.y, pi.y);
    float dz = __fsub_rn(pj.z, pi.z);
    if (PER) {
        dx = wrap_axis(dx, b.len[0], b.half[0], b.per[0]);
        dy = wrap_axis(dy, b.len[1], b.half[1], b.per[1]);
        dz = wrap_axis(dz, b.len[2], b.half[2], b.per[2]);
    }
    return make_float3(dx, dy, dz);
}

// Accurate pair vector for the sums.  The canonical wrap adds or subtracts
// L from the rounded difference, which loses up to ulp(L)/2 for pairs across
// a periodic face.  Here the coordinate near L is shifted first: when
// xj - xi > L/2 it is xj, when xj - xi < -L/2 it is xi, and in both cases
// the shift is exact (Sterbenz: the operand lies in [L/2, L]), so one
// rounding remains.  The decision to wrap is the canonical one, so the pair
// set is unchanged.
__device__ __forceinline__ float wrap_axis_acc(float xi, float xj, float len, float half, int per)
{
    float d = __fsub_rn(xj, xi);
    if (per) {
        if (d > half)
            d = __fsub_rn(__fsub_rn(xj, len), xi);
        else if (d < -half)
            d = __fsub_rn(xj, __fsub_rn(xi, len));
    }
    return d;
}

template <bool PER>
__device__ __forceinline__ float3 pair_dx_acc(const float4 &pi, const float4 &pj, const DevBox &b)
{
    if (!PER) return make_float3(__fsub_rn(pj.x, pi.x), __fsub_rn(pj.y, pi.y), __fsub_rn(pj.z, pi.z));
    return make_float3(wrap_axis_acc(pi.x, pj.x, b.len[0], b.half[0], b.per[0]),
                       wrap_axis_acc(pi.y, pj.y, b.len[1], b.half[1], b.per[1]),
                       wrap_axis_acc(pi.z, pj.z, b.len[2], b.half[2], b.per[2]));
}

__device__ __forceinline__ float d2_of(const float3 &d)
{
    return __fadd_rn(__fadd_rn(__fmul_rn(d.x, d.x), __fmul_rn(d.y, d.y)), __fmul_rn(d.z, d.z));
}

// Lower bound of |dx| after the wrap for any xi in [a0,a1], xj in [b0,b1].
// Every operation is round-to-nearest and monotone, so the bound never
// exceeds the canonical per-pair value (conservative box rounding).
__device__ __forceinline__ float axis_gap(float a0, float a1, float b0, float b1, float len,
                                          int per)
{
    float g = fmaxf(0.f, fmaxf(__fsub_rn(b0, a1), __fsub_rn(a0, b1)));
    if (per) {
        float down = __fsub_rn(len, __fsub_rn(b1, a0));  // j wrapped by -L
        float up = __fadd_rn(__fsub_rn(b0, a1), len);    // j wrapped by +L
        g = fminf(g, fmaxf(0.f, fminf(down, up)));
    }
    return g;
}

// Could some particle of box A be a symmetric neighbor of some particle of
// box B?  lo.w = largest radius of the box.  NaN/inf boxes (empty clusters)
// never pass.
template <bool PER>
__device__ __forceinline__ bool boxes_near(const float4 &alo, const float4 &ahi, const float4 &blo,
                                           const float4 &bhi, const DevBox &b)
{
    float gx = axis_gap(alo.x, ahi.x, blo.x, bhi.x, b.len[0], PER ? b.per[0] : 0);
    float gy = axis_gap(alo.y, ahi.y, blo.y, bhi.y, b.len[1], PER ? b.per[1] : 0);
    float gz = axis_gap(alo.z, ahi.z, blo.z, bhi.z, b.len[2], PER ? b.per[2] : 0);
    float d2 = __fadd_rn(__fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy)), __fmul_rn(gz, gz));
    float r = fmaxf(alo.w, blo.w);
    return d2 <= __fmul_rn(r, r);
}

// Could particle (x, radius r) be a symmetric neighbor of a particle inside
// box B (blo.w = largest radius in B)?  Same monotone rounding as above.
template <bool PER>
__device__ __forceinline__ bool point_near(const float4 &p, float r, const float4 &blo,
                                           const float4 &bhi, const DevBox &b)
{
    float gx = axis_gap(p.x, p.x, blo.x, bhi.x, b.len[0], PER ? b.per[0] : 0);
    float gy = axis_gap(p.y, p.y, blo.y, bhi.y, b.len[1], PER ? b.per[1] : 0);
    float gz = axis_gap(p.z, p.z, blo.z, bhi.z, b.len[2], PER ? b.per[2] : 0);
    float d2 = __fadd_rn(__fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy)), __fmul_rn(gz, gz));
    float rr = fmaxf(r, blo.w);
    return d2 <= __fmul_rn(rr, rr);
}

// ---------------------------------------------------------------------------
// The same arithmetic on a compact per-system form for the hot loops: the
// periodic lengths L (+inf on an open axis) in three registers.  L/2 is
// rounded as 0.5f * L exactly as in DevBox; with L = +inf an open axis never
// wraps and its periodic gap terms are +inf, so every value equals the one of
// the DevBox form without reading any flag.
// ---------------------------------------------------------------------------
struct PerLen {
    float x, y, z;
};

__device__ __forceinline__ PerLen per_len(const DevBox &b)
{
    return PerLen{b.per[0] ? b.len[0] : INFINITY, b.per[1] ? b.len[1] : INFINITY,
                  b.per[2] ? b.len[2] : INFINITY};
}

__device__ __forceinline__ float wrap_len(float d, float len)
{
    const float half = __fmul_rn(0.5f, len);
    if (d > half)
        d = __fsub_rn(d, len);
    else if (d < -half)
        d = __fadd_rn(d, len);
    return d;
}

// ---------------------------------------------------------------------------
// Two FP32 values in one 64-bit register for the packed arithmetic of sm_100
// and later.  One sub / mul .rn.f32x2 rounds each half to nearest exactly as
// the scalar __fsub_rn / __fmul_rn (checked bit for bit on 8.4M random
// operand pairs each).  A packed product whose only use is a packed sum is
// however contracted into a fused multiply-add by the code generator, .rn
// notwithstanding (22.6 % of random squared distances came out different,
// mostly equal to the fused value), so the sums of the canonical predicate
// are taken in scalar add.rn, which is never contracted (0 differences in
// 79.7M).  No packed add is used for it.
// ---------------------------------------------------------------------------
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pk2(float lo, float hi)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void unpk2(f32x2 v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

__device__ __forceinline__ f32x2 sub2_rn(f32x2 a, f32x2 b)
{
    f32x2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ f32x2 mul2_rn(f32x2 a, f32x2 b)
{
    f32x2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

template <bool PER>
__device__ __forceinline__ float pair_d2(const float4 &pi, const float4 &pj, const PerLen &L)
{
    float dx = __fsub_rn(pj.x, pi.x);
    float dy = __fsub_rn(pj.y, pi.y);
    float dz = __fsub_rn(pj.z, pi.z);
    if (PER) {
        dx = wrap_len(dx, L.x);
        dy = wrap_len(dy, L.y);
        dz = wrap_len(dz, L.z);
    }
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// (x^2 + y^2) + z^2 of both halves, the squares packed and the sums in
// scalar add.rn (see above: a packed sum of packed products is contracted)
__device__ __forceinline__ void sum_sq_x2(f32x2 x, f32x2 y, f32x2 z, float &da, float &db)
{
    float xa, xb, ya, yb, za, zb;
    unpk2(mul2_rn(x, x), xa, xb);
    unpk2(mul2_rn(y, y), ya, yb);
    unpk2(mul2_rn(z, z), za, zb);
    da = __fadd_rn(__fadd_rn(xa, ya), za);
    db = __fadd_rn(__fadd_rn(xb, yb), zb);
}

// Canonical d2 of two pairs at once: (xa, xb) - (xi, xi) etc. in packed
// registers; the periodic wrap of each half is the scalar one.  Bit for bit
// the scalar pair_d2 of each pair.
template <bool PER>
__device__ __forceinline__ void pair_d2_x2(f32x2 jx, f32x2 jy, f32x2 jz, f32x2 ix, f32x2 iy,
                                           f32x2 iz, const PerLen &L, float &d2a, float &d2b)
{
    f32x2 dx = sub2_rn(jx, ix), dy = sub2_rn(jy, iy), dz = sub2_rn(jz, iz);
    if (PER) {
        float a, b;
        unpk2(dx, a, b);
        dx = pk2(wrap_len(a, L.x), wrap_len(b, L.x));
        unpk2(dy, a, b);
        dy = pk2(wrap_len(a, L.y), wrap_len(b, L.y));
        unpk2(dz, a, b);
        dz = pk2(wrap_len(a, L.z), wrap_len(b, L.z));
    }
    sum_sq_x2(dx, dy, dz, d2a, d2b);
}

template <bool PER>
__device__ __forceinline__ float3 pair_dx_acc(const float4 &pi, const float4 &pj, const PerLen &L)
{
    if (!PER) return make_float3(__fsub_rn(pj.x, pi.x), __fsub_rn(pj.y, pi.y), __fsub_rn(pj.z, pi.z));
    return make_float3(wrap_axis_acc(pi.x, pj.x, L.x, __fmul_rn(0.5f, L.x), 1),
                       wrap_axis_acc(pi.y, pj.y, L.y, __fmul_rn(0.5f, L.y), 1),
                       wrap_axis_acc(pi.z, pj.z, L.z, __fmul_rn(0.5f, L.z), 1));
}

template <bool PER>
__device__ __forceinline__ float axis_gap_len(float a0, float a1, float b0, float b1, float len)
{
    float g = fmaxf(0.f, fmaxf(__fsub_rn(b0, a1), __fsub_rn(a0, b1)));
    if (PER) {
        float down = __fsub_rn(len, __fsub_rn(b1, a0));  // j wrapped by -L
        float up = __fadd_rn(__fsub_rn(b0, a1), len);    // j wrapped by +L
        g = fminf(g, fmaxf(0.f, fminf(down, up)));
    }
    return g;
}

template <bool PER>
__device__ __forceinline__ bool boxes_near(const float4 &alo, const float4 &ahi, const float4 &blo,
                                           const float4 &bhi, const PerLen &L)
{
    float gx = axis_gap_len<PER>(alo.x, ahi.x, blo.x, bhi.x, L.x);
    float gy = axis_gap_len<PER>(alo.y, ahi.y, blo.y, bhi.y, L.y);
    float gz = axis_gap_len<PER>(alo.z, ahi.z, blo.z, bhi.z, L.z);
    float d2 = __fadd_rn(__fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy)), __fmul_rn(gz, gz));
    float r = fmaxf(alo.w, blo.w);
    return d2 <= __fmul_rn(r, r);
}

// A real (finite) particle only: the periodic gap of a point at infinity
// is not meaningful.
template <bool PER>
__device__ __forceinline__ bool point_near(const float4 &p, float r, const float4 &blo,
                                           const float4 &bhi, const PerLen &L)
{
    float gx = axis_gap_len<PER>(p.x, p.x, blo.x, bhi.x, L.x);
    float gy = axis_gap_len<PER>(p.y, p.y, blo.y, bhi.y, L.y);
    float gz = axis_gap_len<PER>(p.z, p.z, blo.z, bhi.z, L.z);
    float d2 = __fadd_rn(__fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy)), __fmul_rn(gz, gz));
    float rr = fmaxf(r, blo.w);
    return d2 <= __fmul_rn(rr, rr);
}

// ---------------------------------------------------------------------------
// SFC keys
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t quantize21(float x, float lo, float qs)
{
    float t = __fmul_rn(__fsub_rn(x, lo), qs);
    if (!(t > 0.f)) return 0u;
    if (t >= 2097151.f) return 2097151u;
    return __float2uint_rz(t);
}

// Spread the low 21 bits of v so that bit b lands on bit 3b.
__device__ __forceinline__ uint64_t spread3(uint32_t v)
{
    uint64_t x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x001f00000000ffffull;
    x = (x | (x << 16)) & 0x001f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

__device__ __forceinline__ uint64_t morton_key(uint32_t qx, uint32_t qy, uint32_t qz)
{
    return (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
}

// Hilbert key: Skilling's axes-to-transpose transform (J. Skilling,
// "Programming the Hilbert curve", AIP Conf. Proc. 707, 2004) on 21-bit
// coordinates; the transposed words are then bit-interleaved, x first.
__device__ __forceinline__ uint64_t hilbert_key(uint32_t x0, uint32_t x1, uint32_t x2)
{
#pragma unroll
    for (int q = kKeyBits - 1; q >= 1; --q) {
        const uint32_t Q = 1u << q, P = Q - 1u;
        if (x0 & Q) x0 ^= P;
        if (x1 & Q) {
            x0 ^= P;
        } else {
            uint32_t t = (x0 ^ x1) & P;
            x0 ^= t;
            x1 ^= t;
        }
        if (x2 & Q) {
            x0 ^= P;
        } else {
            uint32_t t = (x0 ^ x2) & P;
            x0 ^= t;
            x2 ^= t;
        }
    }
    x1 ^= x0;
    x2 ^= x1;
    // t = xor of (Q-1) over the set bits Q >= 2 of x2: bit b of t is the
    // parity of the bits of x2 above b.
    uint32_t t = x2 >> 1;
    t ^= t >> 1;
    t ^= t >> 2;
    t ^= t >> 4;
    t ^= t >> 8;
    t ^= t >> 16;
    x0 ^= t;
    x1 ^= t;
    x2 ^= t;
    return (spread3(x0) << 2) | (spread3(x1) << 1) | spread3(x2);
}

// Octree level of the longest common key prefix (21 when the keys are equal).
__device__ __forceinline__ int lcp_level(uint64_t a, uint64_t b)
{
    uint64_t d = a ^ b;
    if (d == 0) return kMaxLevel;
    return (__clzll((long long)d) - 1) / 3;
}

// ---------------------------------------------------------------------------
// Warp helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if ((int)lane_id() >= o) v += t;
    }
    return v;
}

__device__ __forceinline__ uint32_t warp_sum(uint32_t v)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Exclusive scan of one value per thread across the block (blockDim.x a
// multiple of 32, <= 1024).  Returns the exclusive prefix; *total gets the
// block sum.  `sh` needs 33 words.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *sh, uint32_t *total)
{
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t inc = warp_incl_scan(v);
    if (lane == 31) sh[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < nw ? sh[lane] : 0u;
        uint32_t wi = warp_incl_scan(w);
        if (lane < nw) sh[lane] = wi - w;
        if (lane == 31) sh[32] = wi;
    }
    __syncthreads();
    uint32_t r = inc - v + sh[warp];
    *total = sh[32];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------
// Host-side launchers implemented in the .cu files
// ---------------------------------------------------------------------------
// Raise a kernel's dynamic shared-memory limit to `bytes` on the current
// device.  The attribute belongs to the device's context, so it is recorded
// per (kernel, device) under a lock: a second device, or several host threads
// on first use, each get it set before their launch.  Returns the error of
// cudaFuncSetAttribute (or of cudaGetDevice).
cudaError_t set_max_dynamic_smem(const void *func, size_t bytes);

cudaError_t launch_keys(int64_t n, const float *x, const float *y, const float *z, const float *h,
                        const DevBox &box, float support, int kind, uint64_t *keys, uint32_t *vals,
                        Status *st, cudaStream_t s);
// batch form: each particle uses its own system's box
// ghist (optional): add the counts of all eight 8-bit digits of the keys for
// a following radix_sort_pairs(..., counted = true) (ghist cleared first).
cudaError_t launch_keys_batch(int64_t n, const float *x, const float *y, const float *z,
                              const float *h, const SysTables &t, float support, int kind,
                              uint64_t *keys, uint32_t *vals, Status *st, uint32_t *ghist,
                              cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs on the low `bits` key bits.
// Scratch: keys_alt/vals_alt (n each), hist (radix_hist_words(n) words,
// cleared by the sort itself).  A look-back that gives up its bounded wait
// sets *stall to 1 (the order is then wrong; callers report NL_ERR_TIMEOUT).
// counted: hist was cleared by radix_sort_clear and the digit counts of all
// passes were added to it (launch_keys_batch with ghist = hist).
size_t radix_hist_words(uint32_t n);
cudaError_t radix_sort_clear(uint32_t *hist, uint32_t n, int bits, cudaStream_t s);
cudaError_t radix_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt,
                             uint32_t n, int bits, uint32_t *hist, unsigned int *stall,
                             cudaStream_t s, bool counted = false);
// Final stable passes by system (digit = system of the value, a caller index):
// sorts (system, key) when run after radix_sort_pairs.
cudaError_t radix_sort_by_system(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt,
                                 uint32_t *vals_alt, uint32_t n, const uint32_t *sys_off,
                                 uint32_t nsys, uint32_t *hist, unsigned int *stall,
                                 cudaStream_t s);

// Boxes of the aligned groups of M consecutive lanes (one particle per lane,
// M | 32, whole warps present): lo = (min xyz, max r), hi = (max xyz, min r),
// empty boxes for all-dummy groups (real == false everywhere).  With
// jlo != NULL the boxes of the aligned sub-groups of MJ < M lanes (the
// j-clusters) are written too.
template <int M>
__device__ __forceinline__ void cluster_box_reduce(uint32_t k, bool real, float4 p, float r,
                                                   int MJ, float4 *clo, float4 *chi,
                                                   float4 *jlo, float4 *jhi)
{
    float lx = real ? p.x : INFINITY, ly = real ? p.y : INFINITY, lz = real ? p.z : INFINITY;
    float hx = real ? p.x : -INFINITY, hy = real ? p.y : -INFINITY, hz = real ? p.z : -INFINITY;
    float rmin = real ? r : INFINITY;
    if (!real) r = 0.f;
#pragma unroll
    for (int o = 1; o < M; o <<= 1) {
        if (jlo && o == MJ && (k & (uint32_t)(MJ - 1)) == 0) {
            jlo[k / MJ] = make_float4(lx, ly, lz, r);
            jhi[k / MJ] = make_float4(hx, hy, hz, rmin);
        }
        rmin = fminf(rmin, __shfl_xor_sync(0xffffffffu, rmin, o));
        lx = fminf(lx, __shfl_xor_sync(0xffffffffu, lx, o));
        ly = fminf(ly, __shfl_xor_sync(0xffffffffu, ly, o));
        lz = fminf(lz, __shfl_xor_sync(0xffffffffu, lz, o));
        hx = fmaxf(hx, __shfl_xor_sync(0xffffffffu, hx, o));
        hy = fmaxf(hy, __shfl_xor_sync(0xffffffffu, hy, o));
        hz = fmaxf(hz, __shfl_xor_sync(0xffffffffu, hz, o));
        r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, o));
    }
    if ((k & (uint32_t)(M - 1)) == 0) {
        clo[k / M] = make_float4(lx, ly, lz, r);
        chi[k / M] = make_float4(hx, hy, hz, rmin);
    }
}

// Permute into padded SFC order as float4 (x, y, z, h) with NaN dummies,
// record the caller index of every padded slot (perm_pad, ~0 for dummies),
// and per-cluster boxes: clo = (lo, max r), chi = (hi, min r) per i-cluster
// of M particles, jlo / jhi the same per j-cluster of MJ < M particles
// (NULL when MJ == M: the i-cluster boxes serve both).
cudaError_t launch_permute(uint32_t npad, int M, int MJ, const SysTables &t, const uint32_t *perm,
                           const float *x, const float *y, const float *z, const float *h,
                           float support, float4 *pos, uint32_t *perm_pad, float4 *clo,
                           float4 *chi, float4 *jlo, float4 *jhi, cudaStream_t s);

// Octree, steps 1-2: leaf level per particle, leaf starts; n_leaves lands
// in st->n_leaves.  Scratch: lev (n bytes), bsum (scan_bsum_words(n)).
size_t scan_bsum_words(uint32_t n);
cudaError_t octree_leaves(const uint64_t *keys, uint32_t n, int bucket, const SysTables &t,
                          uint8_t *lcp, uint8_t *lev, uint32_t *leaf_first, uint8_t *leaf_lev,
                          uint32_t *bsum, Status *st, cudaStream_t s);
// step 3: node offsets per leaf; n_nodes lands in st->n_nodes.
// The leaf count is read on the device (st->n_leaves <= n).
cudaError_t octree_count_nodes(const uint64_t *keys, uint32_t n, const SysTables &t,
                               const uint32_t *leaf_first, const uint8_t *leaf_lev,
                               uint32_t *nodeoff, uint32_t *bsum, Status *st, cudaStream_t s);
// step 4: emit pre-order nodes and their boxes.
struct OctreeOut {
    float4 *nlo;      // (lo.xyz, max r)
    float4 *nhi;      // (hi.xyz, skip as int bits)
    int2 *nrng;       // (first, end) particle range in padded indices
    uint8_t *nlevel;
    int32_t *nparent;
    uint32_t *nchild;
    uint32_t *narrive;
};
// Leaf and node counts are read on the device; node_cap is the capacity of
// the node arrays (nodes beyond it are counted in st->node_overflow).
cudaError_t octree_emit(const uint64_t *keys, uint32_t n, uint32_t node_cap, const SysTables &t,
                        const uint32_t *leaf_first, const uint8_t *leaf_lev,
                        const uint32_t *nodeoff, const float4 *pos, float support,
                        const OctreeOut &o, Status *st, cudaStream_t s);

struct SearchArgs {
    const float4 *pos;
    const float4 *clo, *chi;   // i-cluster boxes (M particles)
    const float4 *jlo, *jhi;   // j-cluster boxes (MJ particles; == clo, chi when MJ == M)
    int mj;                    // j-cluster size MJ
    const float4 *nlo, *nhi;
    const int2 *nrng;
    uint32_t n, nsc, nnodes;
    SysTables sys;
    float support;
    uint32_t *stageJ;
    uint8_t *stageM;
    uint32_t stage_cap;
    uint32_t stage_slots;          // warp slots the staging arrays hold (stage_cap entries each)
    uint8_t *list;
    unsigned long long list_cap;
    uint32_t *rec_off;
    int compress;
    Status *st;
    // half search (MJ == M): super-cluster s searches only j-clusters J >= 8s,
    // keeps them as its upper entries and sends every tile (8s+k, J) with J
    // beyond its own clusters to super-cluster J/8 as a transposed tuple
    // (key = (J/8) * ncl + 8s+k, value = bit J%8 of the rows, merged per key)
    // half = 1; half = 2 stores the entries J >= 8s themselves as the record
    // (half list, every cluster pair once) and emits no tuples
    int half;
    uint32_t ncl;                  // clusters in total (padded)
    uint32_t *uJ;                  // upper entries (j-cluster, mask)
    uint8_t *uM;
    unsigned long long up_cap;
    uint32_t *up_off, *up_cnt;     // per super-cluster: first upper entry, count
    uint64_t *tkey;                // transposed tuples
    uint32_t *tval;
    unsigned long long tu_cap;
    uint32_t *lower_cnt;           // per super-cluster: tuples addressed to it
    const uint32_t *seg_off;       // exclusive scan of lower_cnt (record assembly)
};
cudaError_t launch_search_ctl(const SearchArgs &a, const uint32_t *work, uint32_t count,
                              uint32_t *redo, int M, int any_periodic, int grid_blocks,
                              int threads, cudaStream_t s, const uint32_t *count_dev = nullptr);
// Splits the super-clusters list[0..n) (NULL: 0..n-1) of periodic systems:
// interior ones (their box widened by the system's largest radius, plus a
// rounding margin, stays inside the box on every periodic axis, so no
// neighbor pair of theirs wraps and the open-axis arithmetic gives the same
// results) go to out_int, the others to out_bnd; counts in st->n_int, n_bnd.
cudaError_t launch_classify(const uint32_t *list, uint32_t n, int M, const SysTables &t,
                            const float4 *clo, const float4 *chi, const float4 *nlo,
                            uint32_t node_cap, uint32_t *out_int, uint32_t *out_bnd, Status *st,
                            cudaStream_t s);
// Record assembly of the half search: the record of super-cluster t is its
// sorted tuples (lower j-clusters) followed by its upper entries, encoded as
// by the search.  tkey/tval sorted by key; seg_off from seg_offsets().
cudaError_t launch_assemble(const SearchArgs &a, int grid_blocks, cudaStream_t s);
// keys[k] = fill for min(*used, cap) <= k < cap (unused tuple slots of a graph replay)
cudaError_t launch_fill_keys(uint64_t *keys, uint32_t cap, const unsigned long long *used,
                             uint64_t fill, cudaStream_t s);
// seg_off[k] = sum of cnt[0..k) over k < n; the total lands in *total.
cudaError_t exclusive_scan_u32(const uint32_t *cnt, uint32_t *seg_off, uint32_t n, uint32_t *bsum,
                               uint32_t *total, cudaStream_t s);

enum PassKind { PASS_DENSITY = 0, PASS_COUNT = 1, PASS_SPH = 2, PASS_LJ = 3, PASS_LJC = 4, PASS_MIN = 5 };
struct PassArgs {
    const float4 *pos;
    const uint8_t *list;
    const uint32_t *rec_off;
    const uint32_t *perm;  // caller index of every padded slot, ~0 for dummies
    const float2 *aux;     // per padded particle: density m; SPH (m, P/rho^2); LJ + Coulomb (q, 0)
    uint32_t n, nsc;
    SysTables sys;
    float support;
    int compress;
    int mj;                // j-cluster size MJ (units of the stored indices)
    float p0, p1;          // LJ: eps, sigma
    float p2, p3;          // LJ + Coulomb: rc^2 (interaction cutoff, +inf: the list radius), kc
    float *out0, *out1, *out2;
    uint32_t *outc;
    Status *st;
    const float *hq;         // optional query h per sorted particle (count pass)
    int sorted_out;          // write outputs at the sorted index instead of perm[i]
    const uint32_t *work;    // optional list of super-clusters to process
    uint32_t nwork;
    const uint32_t *nwork_dev;  // optional device count of work (at most nwork)
    // half list (every cluster pair once): both particles of a pair take
    // their share.  Density sums are added as 64-bit fixed point (integer
    // additions in any order give the same bits), counts as integers; a
    // finishing kernel turns them into the outputs.
    int half;
    unsigned long long *hsum;   // density: per sorted particle, sum m_j w in units of 2^-scale
    uint32_t *hcnt;             // counts (or nearest squared distance, float bits): per sorted particle
    double *hf;                 // forces: per sorted particle, 3 FP64 sums
};

// Fixed-point scale of the half-list density: 2^(40 - e) with |m| < 2^e for
// the largest mass, so one neighbor adds at most 2^40 units (w <= 1) and 2^23
// neighbors fit in 63 bits; clamped to the FP32 range.
__device__ __forceinline__ int half_scale_exp(unsigned int mbits)
{
    const int e = (int)((mbits >> 23) & 0xffu) - 126;
    return max(-126, min(127, 40 - e));
}
// threads 0 = 256; blocks_per_sm 0 = default
cudaError_t launch_pass(const PassArgs &a, int kind, int M, int any_periodic, int num_sms,
                        cudaStream_t s, int threads = 0, int blocks_per_sm = 0);
// aux[k] = (a[perm[k]], ...) for real padded slots, zero for dummies;
// amax (optional): atomic max of the bits of |aux.x| (zero it first).
cudaError_t launch_gather_aux(uint32_t npad, const uint32_t *perm_pad, const float *a,
                              const float *b, const float *c, int mode, float2 *aux,
                              cudaStream_t s, unsigned int *amax = nullptr);
// Outputs of a half-list pass from its sums (any pass kind).
cudaError_t launch_half_finish(const PassArgs &a, int kind, uint32_t npad, cudaStream_t s);

// pos[k].xyz = caller position perm_pad[k] (h kept); *max_disp (device, may be
// NULL) = largest |x_new - pos_ref| over real slots, minimum image per system.
cudaError_t launch_refresh(uint32_t npad, const uint32_t *perm_pad, const SysTables &t,
                           const float *x, const float *y, const float *z, float4 *pos,
                           const float4 *pos_ref, float *max_disp, cudaStream_t s);

// Octree node boxes only (topology unchanged), e.g. after new radii.
cudaError_t octree_boxes(uint32_t node_cap, const float4 *pos, float support, const OctreeOut &o,
                         const Status *st, cudaStream_t s);

// h iteration helpers (hiter.cu); all arrays in padded SFC order (npad).
cudaError_t launch_fill(float *a, uint32_t n, float v, cudaStream_t s);
cudaError_t launch_pos_h(uint32_t npad, const float *hs, float4 *pos, cudaStream_t s);
cudaError_t launch_pos_h_to(uint32_t npad, const float4 *pos, float *hq, cudaStream_t s);
cudaError_t launch_cluster_boxes(uint32_t npad, int M, int MJ, const float4 *pos, float support,
                                 float4 *clo, float4 *chi, float4 *jlo, float4 *jhi,
                                 cudaStream_t s);
cudaError_t launch_plain_h0(uint32_t nsc, int M, const uint32_t *perm_pad, const float4 *clo,
                            const float4 *chi, float n_target, float *hq, cudaStream_t s);
cudaError_t launch_hsearch(uint32_t npad, const float *hq, const float *hhi, const uint8_t *conv,
                           float margin, const float *hcap_sys, const SysTables &t, float *hs,
                           cudaStream_t s);
struct HIterState {
    float *hq, *hlo, *hhi, *hs;
    uint32_t *counts;
    uint8_t *conv;
    uint32_t *active_flag;   // per super-cluster
    uint32_t *active_list;
    unsigned int *words;     // [0] unconverged, [1] rebuild needed, [2] active count
    const uint32_t *perm_pad;
    const float *hcap_sys;   // per system: largest h keeping the search radius < L/2
};
cudaError_t launch_hupdate(uint32_t npad, int M, float n_target, float tol, const SysTables &t,
                           const HIterState &h, cudaStream_t s);
cudaError_t launch_active_list(uint32_t nsc, const HIterState &h, cudaStream_t s);
cudaError_t launch_scatter_h(uint32_t npad, const uint32_t *perm_pad, const float *hq,
                             const uint8_t *conv, float *h_out, uint8_t *conv_out, cudaStream_t s);

}  // namespace nlg
