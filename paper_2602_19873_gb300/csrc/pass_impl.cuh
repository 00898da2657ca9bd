// Neighborhood passes over the compressed list (Sec. II-A: loop in parallel
// over super-clusters, decode the list iteratively as needed, process each
// cluster-cluster interaction; Sec. II-D: pure pair function + a sum or a
// minimum).
//
// One warp per super-cluster (atomic work counter, persistent grid).  The
// warp decodes 32 differences at a time: the block mask is read at its
// nibble offset with a funnel shift, each lane finds its info nibble by
// popcount and its data nibbles by a warp scan of data lengths, and a warp
// scan of the differences rebuilds the j-cluster indices.  For every decoded
// (J, mask) entry the lanes hold one i particle of each of the 8 i-clusters
// (lane % M) and 1..8 of the MJ particles of j-cluster J, and accumulate per
// i-cluster in registers; masked-off i-clusters cost nothing (warp-uniform
// branches).  The j particles of 16 or 32 entries are staged in shared memory
// (16 where the super-cluster's own particles sit there too).  The self pair
// is excluded on the fly by index (Sec. II-A).
#pragma once
#include "nl_internal.cuh"

namespace nlg {

constexpr int PS_THREADS = 256;

__device__ __forceinline__ uint32_t get_nibble(const uint8_t *body, uint32_t p)
{
    uint32_t b = body[p >> 1];
    return (p & 1u) ? (b >> 4) : (b & 0xfu);
}

// sqrt.approx.f32: the hardware square root approximation (relative error
// about 2^-22); exact 0 for 0, so coincident particles need no guard
__device__ __forceinline__ float sqrt_approx(float x)
{
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// cubic spline shape on q < 2 (a gather pair of the density pass has
// q < 2 up to one rounding, where the outer branch is 0 to within 1e-20)
__device__ __forceinline__ float spline_w_inside(float q)
{
    const float a = 2.f - q;
    const float inner = fmaf(q * q, fmaf(0.75f, q, -1.5f), 1.f);
    const float outer = 0.25f * a * a * a;
    return q < 1.f ? inner : outer;
}

// 4 w(q) of two arguments q < 2 at once (packed products; inner part as
// 4 - 3 q^2 (2 - q), outer (2 - q)^3): four times the spline shape, exactly
// (scaling by 4 commutes with rounding), so sums of m 4w are exactly four
// times the sums of m w and the caller scales by 1/4 once at the end
__device__ __forceinline__ void spline_w4_inside_x2(f32x2 q, float &w0, float &w1)
{
    const f32x2 a = sub2_rn(pk2(2.f, 2.f), q);  // 2 - q
    const f32x2 t = mul2_rn(mul2_rn(q, q), a);
    const f32x2 a3 = mul2_rn(mul2_rn(a, a), a);
    float q0, q1, t0, t1, o0, o1;
    unpk2(q, q0, q1);
    unpk2(t, t0, t1);
    unpk2(a3, o0, o1);
    w0 = q0 < 1.f ? fmaf(-3.f, t0, 4.f) : o0;
    w1 = q1 < 1.f ? fmaf(-3.f, t1, 4.f) : o1;
}

// cubic spline shape w(q) (support q < 2) and its derivative
__device__ __forceinline__ float spline_w(float q)
{
    float a = 2.f - q;
    float outer = 0.25f * a * a * a;
    float inner = 1.f - 1.5f * q * q + 0.75f * q * q * q;
    return q < 1.f ? inner : (q < 2.f ? outer : 0.f);
}

__device__ __forceinline__ float spline_dw(float q)
{
    float a = 2.f - q;
    float outer = -0.75f * a * a;
    float inner = -3.f * q + 2.25f * q * q;
    return q < 1.f ? inner : (q < 2.f ? outer : 0.f);
}

// Decode the next 32 entries of a record (one per lane; Sec. II-B): the
// block mask is read at nibble offset pos with a funnel shift, each lane
// finds its info nibble by popcount and its data nibbles by a warp scan of
// data lengths, and a warp scan of the differences rebuilds the j-cluster
// indices from prevJ.  Advances pos and prevJ; uncompressed records hold
// the u32 indices (entry t of lane).
__device__ __forceinline__ uint32_t decode_block(const uint32_t *body, int compress, uint32_t t,
                                                 bool valid, uint32_t &pos, uint32_t &prevJ)
{
    const unsigned lane = lane_id();
    uint32_t J;
    if (compress) {
        const uint8_t *bodyb = reinterpret_cast<const uint8_t *>(body);
        const uint32_t w0 = body[pos >> 3];
        const uint32_t w1 = (pos & 7u) ? body[(pos >> 3) + 1] : 0u;
        const uint32_t bm = __funnelshift_r(w0, w1, (pos & 7u) * 4u);
        const bool bit = (bm >> lane) & 1u;
        const uint32_t nbits = __popc(bm);
        uint32_t info = bit ? get_nibble(bodyb, pos + 8 + __popc(bm & lanemask_lt())) : 0u;
        uint32_t ndat = (bit && info < 8u) ? info + 1u : 0u;
        uint32_t incl = warp_incl_scan(ndat);
        uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
        uint32_t pd = pos + 8 + nbits + incl - ndat;
        uint32_t v = 0;
        for (uint32_t q = 0; q < ndat; ++q) v = (v << 4) | get_nibble(bodyb, pd + q);
        uint32_t d = !bit ? 1u : (info >= 8u ? info - 6u : v);
        J = prevJ + warp_incl_scan(d);
        pos += 8 + nbits + tot;
    } else {
        J = valid ? body[t] : 0u;
    }
    prevJ = __shfl_sync(0xffffffffu, J, 31);
    return J;
}

// Accumulators per i-cluster.  Floating sums are two-level: terms of one
// block of 32 list entries go to a plain FP32 partial (b*), and each
// partial is added to the running sum with Kahan compensation (density)
// or plainly (forces), so the rounding error stays near that of ~32*NP
// terms however long the neighbor list is.  The density pass keeps its
// running sums and compensations (v, c) in shared memory instead (they are
// touched once per block), which frees their registers; v and c here serve
// only the final combination across lanes.
template <int KIND>
struct Acc;
template <>
struct Acc<PASS_DENSITY> { float v[kSC], c[kSC], b[kSC]; };
template <>
struct Acc<PASS_COUNT> { uint32_t v[kSC]; };
template <>
struct Acc<PASS_SPH> { float x[kSC], y[kSC], z[kSC], bx[kSC], by[kSC], bz[kSC]; };
template <>
struct Acc<PASS_LJ> { float x[kSC], y[kSC], z[kSC], bx[kSC], by[kSC], bz[kSC]; };
template <>
struct Acc<PASS_LJC> { float x[kSC], y[kSC], z[kSC], bx[kSC], by[kSC], bz[kSC]; };
template <>
struct Acc<PASS_MIN> { float v[kSC]; };  // smallest squared distance

template <int KIND>
__device__ __forceinline__ void acc_begin_block(Acc<KIND> &acc)
{
    if constexpr (KIND == PASS_DENSITY) {
#pragma unroll
        for (int k = 0; k < kSC; ++k) acc.b[k] = 0.f;
    } else if constexpr (KIND == PASS_SPH || KIND == PASS_LJ || KIND == PASS_LJC) {
#pragma unroll
        for (int k = 0; k < kSC; ++k) { acc.bx[k] = 0.f; acc.by[k] = 0.f; acc.bz[k] = 0.f; }
    }
}

template <int KIND>
__device__ __forceinline__ void acc_end_block(Acc<KIND> &acc)
{
    if constexpr (KIND == PASS_DENSITY) {
#pragma unroll
        for (int k = 0; k < kSC; ++k) {
            float y = __fsub_rn(acc.b[k], acc.c[k]);
            float t = __fadd_rn(acc.v[k], y);
            acc.c[k] = __fsub_rn(__fsub_rn(t, acc.v[k]), y);
            acc.v[k] = t;
        }
    } else if constexpr (KIND == PASS_SPH || KIND == PASS_LJ || KIND == PASS_LJC) {
#pragma unroll
        for (int k = 0; k < kSC; ++k) {
            acc.x[k] += acc.bx[k]; acc.y[k] += acc.by[k]; acc.z[k] += acc.bz[k];
        }
    }
}

// The passes keep the super-cluster's own particles in shared memory
// (position and r^2, 1/h and what the pass needs besides) instead of
// registers, read once per listed tile: 48 or more fewer registers per lane,
// so the scalar passes run 4 blocks per SM with few spills and the force
// passes 3; the j particles are staged 16 entries at a time to leave room
// for that.
template <int KIND, bool HL>
constexpr bool pass_i_in_smem() { return !(KIND == PASS_LJ && !HL); }  // full-list LJ: measured faster in registers

// bytes per own particle beside (x, y, z, r^2): (1/h, m) on a half-list
// density pass, (1/h, c_i, r_i, m_i) on the force passes, else 1/h
template <int KIND, bool HL>
constexpr size_t pass_own_extra_bytes()
{
    return (HL && KIND == PASS_DENSITY) ? 8
           : (KIND == PASS_SPH || KIND == PASS_LJ || KIND == PASS_LJC) ? 16 : 4;
}

// list entries whose j particles are staged together
template <int KIND, bool HL>
constexpr int pass_stage_entries() { return pass_i_in_smem<KIND, HL>() ? 16 : 32; }

// Shared memory per warp: the j particles (and pass inputs) of one stage of
// list entries, loaded in bulk before they are computed; on a half list also
// the masses of the super-cluster's own particles, and (half-list density)
// their positions, r^2 and 1/h.
template <int M, int MJ, int KIND, bool HL = false>
constexpr size_t pass_smem_per_warp()
{
    return (size_t)pass_stage_entries<KIND, HL>() * MJ *
               (sizeof(float4) + ((KIND == PASS_DENSITY || KIND == PASS_SPH || KIND == PASS_LJC) ? sizeof(float2) : 0)) +
           (HL ? (size_t)kSC * MJ * sizeof(float) : 0) +
           (pass_i_in_smem<KIND, HL>() ? (size_t)kSC * M * (sizeof(float4) + pass_own_extra_bytes<KIND, HL>()) : 0) +
           (KIND == PASS_DENSITY ? (size_t)2 * kSC * 32 * sizeof(float) : 0);
}

// Resident blocks per SM the register budget is cut for (measured at the
// benchmark sizes): the scalar passes run at 64 registers (4 blocks of 256;
// 5 blocks were slower); the force passes at 128 (2 blocks) on half lists
// and for LJ, at 85 (3 blocks) for SPH and LJ + Coulomb on full lists.
template <int KIND, bool HL>
constexpr int ps_min_blocks()
{
    return (KIND == PASS_DENSITY || KIND == PASS_COUNT || KIND == PASS_MIN) ? 4
           : (HL || KIND == PASS_LJ) ? 2 : 3;
}

// Nearest integer of x (ties away from zero) as a 64-bit two's complement
// word, with integer operations only; |x| < 2^62.  Subnormal x give 0.
__device__ __forceinline__ unsigned long long fixed_of(float x)
{
    const uint32_t b = __float_as_uint(x);
    const int e = (int)((b >> 23) & 0xffu) - 150;  // |x| = mant * 2^e
    const unsigned long long m = (unsigned long long)((b & 0x7fffffu) | 0x800000u);
    unsigned long long q;
    if (e >= 0)
        q = m << e;
    else if (e > -25)
        q = (m + (1ull << (-e - 1))) >> (-e);
    else
        q = 0ull;
    if (((b >> 23) & 0xffu) == 0u) q = 0ull;
    return (b >> 31) ? (0ull - q) : q;
}

// The same for 0 <= x < 2^63 in two 32-bit conversions: hi = floor(x / 2^32)
// (exact: x / 2^32 is a float), then the remainder x - hi 2^32, exact in
// FP32 (below 2^32 it is x itself; above, a multiple of ulp(x) >= 2^9 below
// 2^32), rounded to the nearest integer (ties to even; a remainder of x >=
// 2^32 is already an integer)
__device__ __forceinline__ unsigned long long fixed_of_nonneg(float x)
{
    const uint32_t hi = __float2uint_rz(__fmul_rn(x, 0x1p-32f));
    const uint32_t lo = __float2uint_rn(__fmaf_rn(-__uint2float_rn(hi), 0x1p32f, x));
    return ((unsigned long long)hi << 32) | lo;
}

// The FP64 value of x with integer operations only (exact for normal x;
// zero and subnormals, below 1.2e-38, give 0; inf and NaN stay so).
__device__ __forceinline__ double f64_of(float x)
{
    const uint32_t b = __float_as_uint(x);
    const uint32_t e = (b >> 23) & 0xffu;
    if (e == 0u) return 0.0;
    const unsigned long long d = ((unsigned long long)(b >> 31) << 63) |
                                 ((unsigned long long)(e == 255u ? 2047u : e + 896u) << 52) |
                                 ((unsigned long long)(b & 0x7fffffu) << 29);
    return __longlong_as_double((long long)d);
}

// HL: the list holds every cluster pair once (half list, MJ = M).  Entries
// of the super-cluster's own clusters are complete as they are (both orders
// of every pair are listed); an entry J beyond them is a pair of clusters
// listed only here, so its pairs also add to the j particles: d2 < rj^2 gives
// particle j the term with its own h (density, counts, LJ; SPH pairs share
// one symmetric predicate).  Those j shares are summed over the entry's i
// particles in a fixed shuffle order and added as integers (fixed point for
// density), so the result does not depend on the order of the adds; forces
// are added in FP64 and rounded once to FP32 by the finishing kernel.
template <int M, int MJ, bool PER, int KIND, bool HL>
__global__ void __launch_bounds__(PS_THREADS, (ps_min_blocks<KIND, HL>())) k_pass(PassArgs a)
{
    constexpr int NP = (M * MJ) / 32 > 0 ? (M * MJ) / 32 : 1;
    constexpr int JSTEP = 32 / M;
    constexpr bool AUX = (KIND == PASS_DENSITY || KIND == PASS_SPH || KIND == PASS_LJC);
    static_assert(!HL || M == MJ, "half lists have j-clusters of the i-cluster size");
    constexpr bool FORCE = (KIND == PASS_SPH || KIND == PASS_LJ || KIND == PASS_LJC);
    extern __shared__ __align__(16) unsigned char pass_smem[];
    constexpr bool ISM = pass_i_in_smem<KIND, HL>();
    constexpr uint32_t SE = pass_stage_entries<KIND, HL>();
    float4 *sp = reinterpret_cast<float4 *>(pass_smem + (threadIdx.x >> 5) * pass_smem_per_warp<M, MJ, KIND, HL>());
    float2 *sa = reinterpret_cast<float2 *>(sp + SE * MJ);
    float *smi = AUX ? reinterpret_cast<float *>(sa + SE * MJ) : reinterpret_cast<float *>(sp + SE * MJ);
    // ISM: own particle k*M + II at sip (x, y, z, r^2) and its 1/h in shm,
    // with its mass beside it on a half-list density pass (1/h, m)
    constexpr bool HM = HL && KIND == PASS_DENSITY;
    float4 *sip = reinterpret_cast<float4 *>(smi + (HL ? kSC * MJ : 0));
    float2 *shm = reinterpret_cast<float2 *>(sip + (ISM ? kSC * M : 0));
    float *shv = reinterpret_cast<float *>(shm);
    float4 *sxv = reinterpret_cast<float4 *>(shm);  // force passes: (1/h, c_i, r_i, m_i)
    // density: the running Kahan sums (v, c) of the 8 i-clusters, lane-minor,
    // updated once per block of 32 entries and kept out of the registers
    float *skv = reinterpret_cast<float *>(pass_smem + (threadIdx.x >> 5) * pass_smem_per_warp<M, MJ, KIND, HL>() +
                                           pass_smem_per_warp<M, MJ, KIND, HL>() -
                                           (KIND == PASS_DENSITY ? 2 * kSC * 32 * sizeof(float) : 0));
    // fixed-point scale of the half-list density (2^ex)
    // density sums taken in units of 4 w (the packed spline; WSC = 4) or w
    constexpr bool W4 = (HL && KIND == PASS_DENSITY) || (!HL && !PER && KIND == PASS_DENSITY && NP == 2);
    constexpr float WSC = W4 ? 4.f : 1.f;
    // fixed-point scale of the half-list density (2^ex), per unit of the sums
    const float hscale = (HL && KIND == PASS_DENSITY)
                             ? __int_as_float((half_scale_exp(a.st->m_absmax) + 127) << 23) / WSC
                             : 0.f;
    const unsigned lane = lane_id();
    const uint32_t II = lane % M;
    const uint32_t JJ0 = (lane / M) % MJ;
    auto own_hm = [&](int k) {
        return HM ? shm[k * M + II] : make_float2(shv[k * M + II], 0.f);
    };
    // lanes that hold a distinct (i, j) pair; for M x MJ = 4 x 4 lanes 16..31 repeat
    const bool owner = (M * MJ >= 32) || lane < (uint32_t)(M * MJ);

    const uint32_t nwork = a.work ? (a.nwork_dev ? min(a.nwork, *a.nwork_dev) : a.nwork) : a.nsc;
    for (;;) {
        uint32_t s = 0;
        if (lane == 0) s = atomicAdd(&a.st->pass_ticket, 1u);
        s = __shfl_sync(0xffffffffu, s, 0);
        if (s >= nwork) break;
        if (a.work) s = a.work[s];
        const PerLen box = per_len(a.sys.box[sys_of(a.sys.pad_off, a.sys.nsys, s * kSC * M)]);

        float4 pi[kSC];
        float ri2[kSC], hinv[kSC], ci[kSC], ri[kSC];
#pragma unroll
        for (int k = 0; k < kSC; ++k) {
            uint32_t i = (s * kSC + k) * M + II;
            pi[k] = a.pos[i];
            float r = __fmul_rn(a.support, (KIND == PASS_COUNT && a.hq) ? a.hq[i] : pi[k].w);
            ri[k] = r;
            ri2[k] = __fmul_rn(r, r);
            // LJ + Coulomb: pairs inside the list radius and the interaction cutoff
            if constexpr (KIND == PASS_LJC) ri2[k] = fminf(ri2[k], a.p2);
            hinv[k] = 1.f / pi[k].w;
            ci[k] = (KIND == PASS_SPH) ? a.aux[i].y : (KIND == PASS_LJC) ? a.p3 * a.aux[i].x : 0.f;
        }
        if constexpr (ISM) {
            // own particles for the tile terms (written once per super-cluster)
            __syncwarp();
            if (lane < (uint32_t)M) {
#pragma unroll
                for (int k = 0; k < kSC; ++k) {
                    const uint32_t i = (s * kSC + k) * M + II;
                    sip[k * M + II] = make_float4(pi[k].x, pi[k].y, pi[k].z, ri2[k]);
                    if constexpr (HM)
                        shm[k * M + II] = make_float2(hinv[k], a.aux[i].x);
                    else if constexpr (FORCE)
                        sxv[k * M + II] = make_float4(hinv[k], ci[k], ri[k], (HL && AUX) ? a.aux[i].x : 0.f);
                    else
                        shv[k * M + II] = hinv[k];
                }
            }
        }
        if constexpr (ISM) __syncwarp();
        Acc<KIND> acc;
        // density and counts take the self pair i = j inside the loop when the
        // j-cluster holding i is listed against its i-cluster (d2 = 0, w(0) = 1);
        // bit k: that entry was seen, so the explicit self term is not added
        constexpr bool SELF_IN_LOOP = (KIND == PASS_DENSITY || KIND == PASS_COUNT);
        constexpr uint32_t RJ = M / MJ;
        uint32_t selfseen = 0;
#pragma unroll
        for (int k = 0; k < kSC; ++k) {
            if constexpr (KIND == PASS_DENSITY) {
                skv[k * 32 + lane] = 0.f;
                skv[(kSC + k) * 32 + lane] = 0.f;
            } else if constexpr (KIND == PASS_COUNT) {
                acc.v[k] = 0;
            } else if constexpr (KIND == PASS_MIN) {
                acc.v[k] = INFINITY;
            } else {
                acc.x[k] = 0.f; acc.y[k] = 0.f; acc.z[k] = 0.f;
            }
        }

        // a super-cluster whose list was not stored (an overflow inside a graph
        // replay, reported by nl_graph_check) is read as an empty list
        const uint32_t roff = a.rec_off[s];
        const uint32_t *rec = reinterpret_cast<const uint32_t *>(a.list) + (roff == kBadRecord ? 0u : roff);
        const uint32_t cnt = roff == kBadRecord ? 0u : rec[0];
        const uint8_t *masks = reinterpret_cast<const uint8_t *>(rec + 1);
        const uint32_t *body = rec + 1 + ((cnt + 3u) >> 2);
        uint32_t pos = 0;
        uint32_t prevJ = 0xffffffffu;

        for (uint32_t b0 = 0; b0 < cnt; b0 += 32) {
            const uint32_t t = b0 + lane;
            const bool valid = t < cnt;
            const uint32_t J = decode_block(body, a.compress, t, valid, pos, prevJ);
            const uint32_t mk = valid ? masks[t] : 0u;
            const uint32_t nb = min(32u, cnt - b0);
            acc_begin_block<KIND>(acc);
            // stage the j clusters of entries c0 .. c0 + SE - 1 of the block:
            // entry c0 + e's particles at sp[e*MJ ..]
            auto stage = [&](uint32_t c0) {
            const uint32_t ns = min(SE, nb - c0);
            __syncwarp();
#pragma unroll 4
            for (uint32_t q0 = 0; q0 < ns * MJ; q0 += 32) {  // whole warp in every shuffle
                const uint32_t q = q0 + lane;
                const uint32_t e = min(c0 + q / MJ, 31u);
                const uint32_t src = __shfl_sync(0xffffffffu, J, e) * MJ + (q % MJ);
                if (q < ns * MJ) {
                    if constexpr (HL && (KIND == PASS_DENSITY || KIND == PASS_COUNT || KIND == PASS_MIN)) {
                        // half list: w holds rj^2, and the density input's
                        // second word 1/h_j (dummies: rj = 0, never a pair)
                        const float4 p = a.pos[src];
                        const float rj = __fmul_rn(a.support, p.w);
                        sp[q] = make_float4(p.x, p.y, p.z, __fmul_rn(rj, rj));
                        if constexpr (AUX) sa[q] = make_float2(a.aux[src].x, 1.f / p.w);
                    } else if constexpr (HL && (KIND == PASS_LJ || KIND == PASS_LJC)) {
                        // half list: w holds particle j's own squared cutoff
                        const float4 p = a.pos[src];
                        const float rj = __fmul_rn(a.support, p.w);
                        float rj2 = __fmul_rn(rj, rj);
                        if constexpr (KIND == PASS_LJC) rj2 = fminf(rj2, a.p2);
                        sp[q] = make_float4(p.x, p.y, p.z, rj2);
                        if constexpr (AUX) sa[q] = a.aux[src];
                    } else {
                        sp[q] = a.pos[src];
                        if constexpr (AUX) sa[q] = a.aux[src];
                    }
                }
            }
            __syncwarp();
            };
            // half list: the current entry feeds its j particles too (js), with
            // the shares of this lane's j particles in jsh (density), jcn
            // (counts) or jfx, jfy, jfz (forces)
            bool js = false;
            float jsh[NP] = {};
            uint32_t jcn[NP] = {};
            float jfx[NP] = {}, jfy[NP] = {}, jfz[NP] = {};
            float jmn[NP];
#pragma unroll
            for (int tt = 0; tt < NP; ++tt) jmn[tt] = INFINITY;
            // one (i-cluster k, j particle) term per lane
            // pik, hik, mik: i particle (x, y, z; w = r^2 when in shared memory),
            // its 1/h and (half-list density) its mass
            // ex: the force passes' (1/h, c_i, r_i, m_i)
            auto term = [&](int k, const float4 &pik, float hik, float mik, const float4 &ex,
                            const float4 &pj, const float2 &aj, uint32_t jj, int tt) {
                const uint32_t ii = (s * kSC + k) * M + II;
                // canonical distance decides the pair; the sums use the
                // accurate vector (identical unless wrapped)
                const float d2 = pair_d2<PER>(pik, pj, box);
                if constexpr (HL && KIND == PASS_DENSITY) {
                    static_assert(ISM, "the half-list density pass reads its i particles from shared memory");
                    const bool ini = d2 < pik.w;         // i = j included (see selfseen)
                    const bool inj = js && d2 < pj.w;    // the j share (entries beyond the own clusters)
                    if (owner && (ini || inj)) {
                        const float e2 = PER ? d2_of(pair_dx_acc<PER>(pik, pj, box)) : d2;
                        const float r = sqrt_approx(e2);
                        // both sides' kernel values in one packed evaluation
                        float wi, wj;
                        spline_w4_inside_x2(mul2_rn(pk2(r, r), pk2(hik, aj.y)), wi, wj);
                        if (ini) acc.b[k] += aj.x * wi;
                        if (inj) jsh[tt] += mik * wj;
                    }
                } else if constexpr (HL && KIND == PASS_COUNT) {
                    if (owner) {
                        if (d2 < pik.w) acc.v[k] += 1u;  // i = j included (see selfseen)
                        if (js && d2 < pj.w) jcn[tt] += 1u;
                    }
                } else if constexpr (KIND == PASS_DENSITY) {
                    if (owner && d2 < pik.w) {  // i = j included (see selfseen)
                        const float e2 = PER ? d2_of(pair_dx_acc<PER>(pik, pj, box)) : d2;
                        acc.b[k] += aj.x * spline_w_inside(sqrt_approx(e2) * hik);
                    }
                } else if constexpr (KIND == PASS_COUNT) {
                    if (owner && d2 < pik.w) acc.v[k] += 1u;  // i = j included (see selfseen)
                } else if constexpr (HL && KIND == PASS_MIN) {
                    const bool ini = d2 < pik.w;
                    const bool inj = js && d2 < pj.w;
                    if (owner && ii != jj && (ini || inj)) {
                        const float e2 = PER ? d2_of(pair_dx_acc<PER>(pik, pj, box)) : d2;
                        if (ini) acc.v[k] = fminf(acc.v[k], e2);
                        if (inj) jmn[tt] = fminf(jmn[tt], e2);
                    }
                } else if constexpr (KIND == PASS_MIN) {  // nearest gather neighbor
                    if (owner && ii != jj && d2 < pik.w) {
                        const float e2 = PER ? d2_of(pair_dx_acc<PER>(pik, pj, box)) : d2;
                        acc.v[k] = fminf(acc.v[k], e2);
                    }
                } else if constexpr (KIND == PASS_SPH) {
                    const float rj = __fmul_rn(a.support, pj.w);
                    const float rr = fmaxf(ex.z, rj);
                    if (owner && ii != jj && d2 < __fmul_rn(rr, rr)) {
                        // a_i -= m_j (c_i gW_i + c_j gW_j) (x_i - x_j) / r
                        const float3 dv = pair_dx_acc<PER>(pik, pj, box);
                        const float e2 = d2_of(dv);
                        const float ir = e2 > 0.f ? rsqrtf(e2) : 0.f;  // grad W(0) = 0
                        const float r = e2 * ir;
                        const float hji = 1.f / pj.w;
                        const float gi = spline_dw(r * ex.x) * ex.x * ex.x * ex.x * ex.x;
                        const float gj = spline_dw(r * hji) * hji * hji * hji * hji;
                        const float bsym = (ex.y * gi + aj.y * gj) * 0.318309886183790672f * ir;
                        const float sc = aj.x * bsym;
                        // x_i - x_j = -dv
                        acc.bx[k] += sc * dv.x;
                        acc.by[k] += sc * dv.y;
                        acc.bz[k] += sc * dv.z;
                        if constexpr (HL) {
                            if (js) {  // a_j -= m_i (same bracket) (x_j - x_i) / r
                                const float sj = ex.w * bsym;
                                jfx[tt] -= sj * dv.x;
                                jfy[tt] -= sj * dv.y;
                                jfz[tt] -= sj * dv.z;
                            }
                        }
                    }
                } else if constexpr (HL && KIND == PASS_LJ) {  // both particles, F_j = -F_ij
                    const bool ini = d2 < pik.w;
                    const bool inj = js && d2 < pj.w;
                    if (owner && ii != jj && (ini || inj)) {
                        const float3 dv = pair_dx_acc<PER>(pik, pj, box);
                        const float ir2 = 1.f / d2_of(dv);
                        const float s2 = a.p1 * a.p1 * ir2;
                        const float s6 = s2 * s2 * s2;
                        const float c = 24.f * a.p0 * ir2 * s6 * (2.f * s6 - 1.f);
                        if (ini) { acc.bx[k] -= c * dv.x; acc.by[k] -= c * dv.y; acc.bz[k] -= c * dv.z; }
                        if (inj) { jfx[tt] += c * dv.x; jfy[tt] += c * dv.y; jfz[tt] += c * dv.z; }
                    }
                } else if constexpr (HL && KIND == PASS_LJC) {  // both particles, F_j = -F_ij
                    const bool ini = d2 < pik.w;
                    const bool inj = js && d2 < pj.w;
                    if (owner && ii != jj && (ini || inj)) {
                        const float3 dv = pair_dx_acc<PER>(pik, pj, box);
                        const float ir = rsqrtf(d2_of(dv));
                        const float ir2 = ir * ir;
                        const float s2 = a.p1 * a.p1 * ir2;
                        const float s6 = s2 * s2 * s2;
                        const float c = ir2 * (24.f * a.p0 * s6 * (2.f * s6 - 1.f) + ex.y * aj.x * ir);
                        if (ini) { acc.bx[k] -= c * dv.x; acc.by[k] -= c * dv.y; acc.bz[k] -= c * dv.z; }
                        if (inj) { jfx[tt] += c * dv.x; jfy[tt] += c * dv.y; jfz[tt] += c * dv.z; }
                    }
                } else if constexpr (KIND == PASS_LJ) {  // F_i += 24 eps (2 s^12/r^14 - s^6/r^8)(x_i - x_j)
                    if (owner && ii != jj && d2 < pik.w) {
                        const float3 dv = pair_dx_acc<PER>(pik, pj, box);
                        const float ir2 = 1.f / d2_of(dv);
                        const float s2 = a.p1 * a.p1 * ir2;
                        const float s6 = s2 * s2 * s2;
                        const float c = 24.f * a.p0 * ir2 * s6 * (2.f * s6 - 1.f);
                        acc.bx[k] -= c * dv.x;
                        acc.by[k] -= c * dv.y;
                        acc.bz[k] -= c * dv.z;
                    }
                } else {  // LJ + Coulomb: the LJ term plus kc q_i q_j (x_i - x_j) / r^3
                    if (owner && ii != jj && d2 < pik.w) {
                        const float3 dv = pair_dx_acc<PER>(pik, pj, box);
                        const float ir = rsqrtf(d2_of(dv));
                        const float ir2 = ir * ir;
                        const float s2 = a.p1 * a.p1 * ir2;
                        const float s6 = s2 * s2 * s2;
                        const float c = ir2 * (24.f * a.p0 * s6 * (2.f * s6 - 1.f) + ex.y * aj.x * ir);
                        acc.bx[k] -= c * dv.x;
                        acc.by[k] -= c * dv.y;
                        acc.bz[k] -= c * dv.z;
                    }
                }
            };
            for (uint32_t e = 0; e < nb; ++e) {
                if (e % SE == 0) stage(e);
                const uint32_t el = e % SE;  // staged slot of the entry
                const uint32_t Je = __shfl_sync(0xffffffffu, J, e);
                const uint32_t me = __shfl_sync(0xffffffffu, mk, e);
                // half list: an entry beyond the own clusters also feeds its j particles
                js = HL && Je >= (s + 1) * kSC * RJ;
#pragma unroll
                for (int tt = 0; tt < NP; ++tt) {
                    jsh[tt] = 0.f; jcn[tt] = 0u;
                    jfx[tt] = 0.f; jfy[tt] = 0.f; jfz[tt] = 0.f;
                    jmn[tt] = INFINITY;
                }
                if constexpr (SELF_IN_LOOP) {
                    const uint32_t rel = Je - s * kSC * RJ;  // j-cluster within the own ones
                    if (rel < (uint32_t)(kSC * RJ)) {
                        const uint32_t kk = rel / RJ;
                        if (((me >> kk) & 1u) && (RJ == 1 || II / MJ == rel % RJ))
                            selfseen |= 1u << kk;
                    }
                }
                if constexpr (NP <= 2) {
                    // the entry's j particles in registers; the NP terms of one
                    // i-cluster are independent (instruction-level parallelism)
                    float4 pj[NP];
                    float2 aj[NP];
#pragma unroll
                    for (int tt = 0; tt < NP; ++tt) {
                        pj[tt] = sp[el * MJ + JJ0 + tt * JSTEP];
                        aj[tt] = AUX ? sa[el * MJ + JJ0 + tt * JSTEP] : make_float2(0.f, 0.f);
                    }
#pragma unroll
                    for (int k = 0; k < kSC; ++k) {
                        if (!((me >> k) & 1u)) continue;
                        const float4 pik = ISM ? sip[k * M + II] : make_float4(pi[k].x, pi[k].y, pi[k].z, ri2[k]);
                        const float4 ex = !FORCE ? make_float4(0.f, 0.f, 0.f, 0.f)
                                          : ISM ? sxv[k * M + II] : make_float4(hinv[k], ci[k], ri[k], 0.f);
                        const float2 hm = FORCE ? make_float2(ex.x, ex.w) : ISM ? own_hm(k) : make_float2(hinv[k], 0.f);
                        if constexpr (!HL && !PER && KIND == PASS_DENSITY && NP == 2) {
                            // full-list density on open systems: the lane's two
                            // pairs share one branch and one packed kernel evaluation
                            const float d2a = pair_d2<PER>(pik, pj[0], box), d2b = pair_d2<PER>(pik, pj[1], box);
                            const bool ina = owner && d2a < pik.w, inb = owner && d2b < pik.w;  // i = j included
                            if (ina || inb) {
                                float wa, wb;
                                spline_w4_inside_x2(mul2_rn(pk2(sqrt_approx(d2a), sqrt_approx(d2b)), pk2(hm.x, hm.x)),
                                                   wa, wb);
                                if (ina) acc.b[k] += aj[0].x * wa;
                                if (inb) acc.b[k] += aj[1].x * wb;
                            }
                        } else {
#pragma unroll
                            for (int tt = 0; tt < NP; ++tt)
                                term(k, pik, hm.x, hm.y, ex, pj[tt], aj[tt], Je * MJ + JJ0 + tt * JSTEP, tt);
                        }
                    }
                } else {
#pragma unroll
                    for (int tt = 0; tt < NP; ++tt) {
                        const float4 pj = sp[el * MJ + JJ0 + tt * JSTEP];
                        const float2 aj = AUX ? sa[el * MJ + JJ0 + tt * JSTEP] : make_float2(0.f, 0.f);
#pragma unroll
                        for (int k = 0; k < kSC; ++k)
                            if ((me >> k) & 1u) {
                                const float4 pik = ISM ? sip[k * M + II] : make_float4(pi[k].x, pi[k].y, pi[k].z, ri2[k]);
                                const float4 ex = !FORCE ? make_float4(0.f, 0.f, 0.f, 0.f)
                                                  : ISM ? sxv[k * M + II] : make_float4(hinv[k], ci[k], ri[k], 0.f);
                                const float2 hm = FORCE ? make_float2(ex.x, ex.w) : ISM ? own_hm(k) : make_float2(hinv[k], 0.f);
                                term(k, pik, hm.x, hm.y, ex, pj, aj, Je * MJ + JJ0 + tt * JSTEP, tt);
                            }
                    }
                }
                if constexpr (HL && NP == 2 && (KIND == PASS_DENSITY || KIND == PASS_COUNT)) {
                    if (js) {
                        // sum each j particle's share over the M lanes of its i
                        // particles in a fixed order: the first step trades the
                        // lane's two shares with lane II ^ 1 (even lanes keep the
                        // first j particle, odd lanes the second), two more steps
                        // finish; lanes II = 0 and 1 then add one integer each
                        const bool odd = II & 1u;
                        if constexpr (KIND == PASS_DENSITY) {
                            float v = (odd ? jsh[1] : jsh[0]) +
                                      __shfl_xor_sync(0xffffffffu, odd ? jsh[0] : jsh[1], 1);
#pragma unroll
                            for (int o = 2; o < M; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                            // a share is a sum of m 4w >= 0 (up to a rounding of
                            // the square root at the edge of the support, where
                            // w is below 1e-20: clamped to 0)
                            if (II < 2u && v > 0.f)
                                atomicAdd(&a.hsum[Je * MJ + JJ0 + II * JSTEP], fixed_of_nonneg(v * hscale));
                        } else {
                            uint32_t v = (odd ? jcn[1] : jcn[0]) +
                                         __shfl_xor_sync(0xffffffffu, odd ? jcn[0] : jcn[1], 1);
#pragma unroll
                            for (int o = 2; o < M; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                            if (II < 2u && v != 0u) atomicAdd(&a.hcnt[Je * MJ + JJ0 + II * JSTEP], v);
                        }
                    }
                } else if constexpr (HL) {
                    if (js) {
                        // sum each j particle's share over the M lanes of its i
                        // particles (fixed order), one integer add per j particle
#pragma unroll
                        for (int tt = 0; tt < NP; ++tt) {
                            const uint32_t jj = Je * MJ + JJ0 + tt * JSTEP;
                            if constexpr (KIND == PASS_DENSITY) {
                                float v = jsh[tt];
#pragma unroll
                                for (int o = 1; o < M; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                                if (owner && II == 0 && v != 0.f)
                                    atomicAdd(&a.hsum[jj], fixed_of(v * hscale));
                            } else if constexpr (FORCE) {
                                // FP64 adds: their order changes the sum by about
                                // 1e-16 of it, below the FP32 rounding of the output
                                float vx = jfx[tt], vy = jfy[tt], vz = jfz[tt];
#pragma unroll
                                for (int o = 1; o < M; o <<= 1) {
                                    vx += __shfl_xor_sync(0xffffffffu, vx, o);
                                    vy += __shfl_xor_sync(0xffffffffu, vy, o);
                                    vz += __shfl_xor_sync(0xffffffffu, vz, o);
                                }
                                if (owner && II == 0 && (vx != 0.f || vy != 0.f || vz != 0.f)) {
                                    atomicAdd(&a.hf[3 * (size_t)jj + 0], f64_of(vx));
                                    atomicAdd(&a.hf[3 * (size_t)jj + 1], f64_of(vy));
                                    atomicAdd(&a.hf[3 * (size_t)jj + 2], f64_of(vz));
                                }
                            } else if constexpr (KIND == PASS_MIN) {
                                // a minimum is the same in any order: integer
                                // minimum of the bits of non-negative floats
                                float v = jmn[tt];
#pragma unroll
                                for (int o = 1; o < M; o <<= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
                                if (owner && II == 0 && v < INFINITY) atomicMin(&a.hcnt[jj], __float_as_uint(v));
                            } else {
                                uint32_t v = jcn[tt];
#pragma unroll
                                for (int o = 1; o < M; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                                if (owner && II == 0 && v != 0u) atomicAdd(&a.hcnt[jj], v);
                            }
                        }
                    }
                }
            }
            if constexpr (KIND == PASS_DENSITY) {
                // the block partial into the running sum, Kahan-compensated
#pragma unroll
                for (int k = 0; k < kSC; ++k) {
                    const float v = skv[k * 32 + lane], c = skv[(kSC + k) * 32 + lane];
                    const float y = __fsub_rn(acc.b[k], c);
                    const float t = __fadd_rn(v, y);
                    skv[(kSC + k) * 32 + lane] = __fsub_rn(__fsub_rn(t, v), y);
                    skv[k * 32 + lane] = t;
                }
            } else {
                acc_end_block<KIND>(acc);
            }
        }
        if constexpr (KIND == PASS_DENSITY) {
#pragma unroll
            for (int k = 0; k < kSC; ++k) {
                acc.v[k] = skv[k * 32 + lane];
                acc.c[k] = skv[(kSC + k) * 32 + lane];
            }
        }

        // combine lanes holding the same i particle, write in caller order
#pragma unroll
        for (int k = 0; k < kSC; ++k) {
#pragma unroll
            for (int o = M; o < 32; o <<= 1) {
                if constexpr (KIND == PASS_DENSITY) {
                    if (o == M) acc.v[k] = __fsub_rn(acc.v[k], acc.c[k]);
                    acc.v[k] += __shfl_xor_sync(0xffffffffu, acc.v[k], o);
                } else if constexpr (KIND == PASS_COUNT) {
                    acc.v[k] += __shfl_xor_sync(0xffffffffu, acc.v[k], o);
                } else if constexpr (KIND == PASS_MIN) {
                    acc.v[k] = fminf(acc.v[k], __shfl_xor_sync(0xffffffffu, acc.v[k], o));
                } else {
                    acc.x[k] += __shfl_xor_sync(0xffffffffu, acc.x[k], o);
                    acc.y[k] += __shfl_xor_sync(0xffffffffu, acc.y[k], o);
                    acc.z[k] += __shfl_xor_sync(0xffffffffu, acc.z[k], o);
                }
            }
        }
        // lane (II, g) with g = lane / M writes the i-clusters k = g (mod 32/M)
        constexpr uint32_t G = 32 / M;
        const uint32_t g = lane / M;
#pragma unroll
        for (int k = 0; k < kSC; ++k) {
            if ((uint32_t)k % G != g) continue;
            const uint32_t i = (s * kSC + k) * M + II;
            const uint32_t pc = a.perm[i];
            if (pc == 0xffffffffu) continue;  // dummy slot
            const uint32_t o = a.sorted_out ? i : pc;
            // the loop took i = j iff its entry was listed and the radius is
            // nonzero (d2 = 0 < r^2)
            const bool took_self = ((selfseen >> k) & 1u) && (ISM ? sip[k * M + II].w : ri2[k]) > 0.f;
            if constexpr (HL && KIND == PASS_DENSITY) {
                const float self = took_self ? 0.f : WSC * a.aux[i].x;  // m_i w(0) = m_i
                atomicAdd(&a.hsum[i], fixed_of((acc.v[k] + self) * hscale));
            } else if constexpr (HL && KIND == PASS_COUNT) {
                atomicAdd(&a.hcnt[i], acc.v[k] - (took_self ? 1u : 0u));
            } else if constexpr (HL && FORCE) {
                atomicAdd(&a.hf[3 * (size_t)i + 0], f64_of(acc.x[k]));
                atomicAdd(&a.hf[3 * (size_t)i + 1], f64_of(acc.y[k]));
                atomicAdd(&a.hf[3 * (size_t)i + 2], f64_of(acc.z[k]));
            } else if constexpr (KIND == PASS_DENSITY) {
                const float self = took_self ? 0.f : WSC * a.aux[i].x;  // m_i w(0) = m_i
                const float hk = ISM ? own_hm(k).x : hinv[k];
                a.out0[o] = (acc.v[k] + self) * (1.f / WSC) * (0.318309886183790672f * hk * hk * hk);
            } else if constexpr (KIND == PASS_COUNT) {
                a.outc[o] = acc.v[k] - (took_self ? 1u : 0u);
            } else if constexpr (HL && KIND == PASS_MIN) {
                if (acc.v[k] < INFINITY) atomicMin(&a.hcnt[i], __float_as_uint(acc.v[k]));
            } else if constexpr (KIND == PASS_MIN) {
                a.out0[o] = sqrtf(acc.v[k]);  // +inf without a neighbor
            } else if constexpr (KIND == PASS_SPH) {
                a.out0[o] = acc.x[k];
                a.out1[o] = acc.y[k];
                a.out2[o] = acc.z[k];
            } else {  // LJ, LJ + Coulomb
                a.out0[o] = acc.x[k];
                a.out1[o] = acc.y[k];
                a.out2[o] = acc.z[k];
            }
        }
    }
}

template <int M, int MJ, int KIND, bool HL = false>
static cudaError_t launch_mk(const PassArgs &a, int per, int grid, int threads, cudaStream_t s)
{
    // the attribute is set for the largest block so that any shape fits
    const size_t smax = (size_t)(PS_THREADS / 32) * pass_smem_per_warp<M, MJ, KIND, HL>();
    const size_t smem = (size_t)(threads / 32) * pass_smem_per_warp<M, MJ, KIND, HL>();
    const void *fn = per ? (const void *)k_pass<M, MJ, true, KIND, HL>
                         : (const void *)k_pass<M, MJ, false, KIND, HL>;
    cudaError_t e = set_max_dynamic_smem(fn, smax);
    if (e != cudaSuccess) return e;
    if (per)
        k_pass<M, MJ, true, KIND, HL><<<grid, threads, smem, s>>>(a);
    else
        k_pass<M, MJ, false, KIND, HL><<<grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int KIND>
static cudaError_t launch_k(const PassArgs &a, int M, int per, int grid, int threads, cudaStream_t s)
{
    if (threads != 128 && threads != PS_THREADS) return cudaErrorInvalidValue;
    if (a.half) {
        switch (M * 100 + a.mj) {
        case 404: return launch_mk<4, 4, KIND, true>(a, per, grid, threads, s);
        case 808: return launch_mk<8, 8, KIND, true>(a, per, grid, threads, s);
        case 1616: return launch_mk<16, 16, KIND, true>(a, per, grid, threads, s);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (M * 100 + a.mj) {
    case 404: return launch_mk<4, 4, KIND>(a, per, grid, threads, s);
    case 808: return launch_mk<8, 8, KIND>(a, per, grid, threads, s);
    case 804: return launch_mk<8, 4, KIND>(a, per, grid, threads, s);
    case 1616: return launch_mk<16, 16, KIND>(a, per, grid, threads, s);
    case 1608: return launch_mk<16, 8, KIND>(a, per, grid, threads, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace nlg
