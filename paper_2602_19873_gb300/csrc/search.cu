// Cluster-pair search and list encoding (Sec. II-A, II-B, II-C).
//
// One warp per super-cluster (8 i-clusters of M particles), taken from an
// atomic work counter by a persistent grid.  The warp walks the pre-order
// octree without a stack (skip indices), reading nodes in coalesced chunks
// of 32 staged in shared memory.  Every particle of the super-cluster (1 to
// 4 per lane) is tested against the node box inflated by the larger of its
// radius and the node's maximum radius, with monotone round-to-nearest gaps
// so that no pair accepted by the FP32 predicate can be pruned.  Accepted leaves append
// their j-clusters (MJ particles each, MJ = M or M / 2: the M x MJ tiles of
// Sec. II-A / III-A) to a per-warp queue, drained 4 j-clusters at a time:
// their particles are staged in shared memory, 4 x 8 (i-cluster, j-cluster)
// box pairs are tested in one round (one lane each), and each candidate tile
// is decided by the exact FP32 predicate on its M x MJ pairs, stopping at the
// first pair found.  (Finer filters between the two, every i particle against
// the j-cluster box and a test for tiles whose pairs are all neighbors, cost
// more than the tile tests they saved.)  Depth-first order yields
// ascending j-clusters (Sec. II-A), so the (J, mask) list is produced
// sorted; it is staged per warp (L2 resident) and then encoded:
// u32 count | u8 masks | nibble blocks of 32 differences (Sec. II-B, the
// layout of Sec. II-C with w = 32), reserved with one atomicAdd in the list
// buffer.  Super-clusters whose list exceeds the staging capacity or the
// list buffer are queued in a redo list and re-run by the host after growth.
#include "nl_internal.cuh"

namespace nlg {

constexpr int SR_THREADS = 256;
constexpr int SR_WARPS = SR_THREADS / 32;
constexpr int WIN_WORDS = 64;
constexpr uint32_t SR_QCAP = 128;   // j-cluster queue entries per warp (multiple of 4)

struct SearchCtl {
    const uint32_t *work;   // NULL: super-clusters 0..count-1, else ids
    uint32_t count;
    uint32_t *redo;         // ids that could not be stored this time
    const uint32_t *count_dev;  // optional device count (at most count)
};

__device__ __forceinline__ uint32_t hex_digits(uint32_t v) { return (32u - __clz(v) + 3u) >> 2; }

__device__ __forceinline__ void win_put(uint32_t *win, uint32_t W0, uint32_t p, uint32_t v)
{
    uint32_t l = p - W0;
    atomicOr(&win[l >> 3], v << ((l & 7u) * 4u));
}

// Encode the list of one super-cluster: entry t is (getJ(t), getM(t)),
// ascending in J.  Returns false when the list buffer is full (nothing
// written for this super-cluster).
template <class GJ, class GM>
__device__ bool encode_record(uint32_t cnt, GJ getJ, GM getM, uint32_t *win, const SearchArgs &a,
                              uint32_t s)
{
    const unsigned lane = lane_id();
    const unsigned lt = lanemask_lt();
    uint32_t nib = 0;
    if (a.compress) {
        uint32_t carry = 0xffffffffu;  // J_{-1} = -1
        for (uint32_t b0 = 0; b0 < cnt; b0 += 32) {
            uint32_t t = b0 + lane;
            uint32_t J = t < cnt ? getJ(t) : 0u;
            uint32_t prev = __shfl_up_sync(0xffffffffu, J, 1);
            if (lane == 0) prev = carry;
            uint32_t d = t < cnt ? J - prev : 1u;
            uint32_t nb = d == 1u ? 0u : (d <= 9u ? 1u : 1u + hex_digits(d));
            nib += 8u + warp_sum(nb);
            carry = __shfl_sync(0xffffffffu, J, 31);
        }
    }
    const uint32_t mask_words = (cnt + 3u) >> 2;
    const uint32_t body_words = a.compress ? (nib + 7u) >> 3 : cnt;
    const uint32_t words = 1u + mask_words + body_words;
    unsigned long long off = 0;
    if (lane == 0) off = atomicAdd(&a.st->list_used, (unsigned long long)words * 4ull);
    off = __shfl_sync(0xffffffffu, off, 0);
    if (off + (unsigned long long)words * 4ull > a.list_cap) {
        // reservations only grow, so every record below the lowest failed
        // offset was stored; the host resumes allocation there
        if (lane == 0) atomicMin(&a.st->fail_off, off);
        return false;
    }
    uint32_t *rec = reinterpret_cast<uint32_t *>(a.list + off);
    if (lane == 0) {
        rec[0] = cnt;
        a.rec_off[s] = (uint32_t)(off >> 2);
    }
    for (uint32_t w = lane; w < mask_words; w += 32) {
        uint32_t v = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t t = 4 * w + q;
            if (t < cnt) v |= (getM(t) & 0xffu) << (8 * q);
        }
        rec[1 + w] = v;
    }
    uint32_t *body = rec + 1 + mask_words;
    if (!a.compress) {
        for (uint32_t t = lane; t < cnt; t += 32) body[t] = getJ(t);
        return true;
    }
    win[lane] = 0u;
    win[lane + 32] = 0u;
    __syncwarp();
    uint32_t W0 = 0, pos = 0, carry = 0xffffffffu;
    for (uint32_t b0 = 0; b0 < cnt; b0 += 32) {
        uint32_t t = b0 + lane;
        bool valid = t < cnt;
        uint32_t J = valid ? getJ(t) : 0u;
        uint32_t prev = __shfl_up_sync(0xffffffffu, J, 1);
        if (lane == 0) prev = carry;
        uint32_t d = valid ? J - prev : 1u;
        bool bit = d != 1u;
        uint32_t bm = __ballot_sync(0xffffffffu, bit);
        uint32_t ndat = (bit && d > 9u) ? hex_digits(d) : 0u;
        uint32_t info = !bit ? 0u : (d <= 9u ? d + 6u : ndat - 1u);
        uint32_t incl = warp_incl_scan(ndat);
        uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
        uint32_t nbits = __popc(bm);
        if (lane < 8) win_put(win, W0, pos + lane, (bm >> (4 * lane)) & 0xfu);
        if (bit) win_put(win, W0, pos + 8 + __popc(bm & lt), info);
        uint32_t pd = pos + 8 + nbits + (incl - ndat);
        for (uint32_t q = 0; q < ndat; ++q) win_put(win, W0, pd + q, (d >> (4 * (ndat - 1 - q))) & 0xfu);
        __syncwarp();
        uint32_t pend = pos + 8 + nbits + tot;
        uint32_t full = (pend - W0) >> 3;
        for (uint32_t w = lane; w < full; w += 32) body[(W0 >> 3) + w] = win[w];
        __syncwarp();
        uint32_t keep = win[full];
        __syncwarp();
        win[lane] = 0u;
        win[lane + 32] = 0u;
        __syncwarp();
        if (lane == 0) win[0] = keep;
        __syncwarp();
        W0 += full * 8u;
        pos = pend;
        carry = __shfl_sync(0xffffffffu, J, 31);
    }
    if (pos > W0 && lane == 0) body[W0 >> 3] = win[0];
    __syncwarp();
    return true;
}

// Half search output of super-cluster s (MJ == M): the staged upper entries
// (J >= 8s, ascending) go to the upper buffer, and every tile (8s+k, J) with
// J beyond the own clusters becomes part of a transposed tuple for
// super-cluster t = J/8: key t * ncl + (8s+k), value = the bits J%8 of all
// such J with the same t (entries of one t are consecutive, at most 8 of
// them, so a group spans at most two 32-entry chunks and is carried over).
// Returns false when a buffer was too small (the reservations still count,
// so the host learns the sizes it needs).
__device__ bool half_output(uint32_t cnt, const uint32_t *stJ, const uint8_t *stM,
                            const SearchArgs &a, uint32_t s)
{
    const unsigned lane = lane_id();
    constexpr uint32_t NONE = 0xffffffffu;
    unsigned long long off = 0;
    if (lane == 0) off = atomicAdd(&a.st->up_used, (unsigned long long)cnt);
    off = __shfl_sync(0xffffffffu, off, 0);
    if (off + cnt > a.up_cap) {
        if (lane == 0) atomicExch(&a.st->half_overflow, 1u);
        return false;
    }
    for (uint32_t t = lane; t < cnt; t += 32) {
        a.uJ[off + t] = stJ[t];
        a.uM[off + t] = stM[t];
    }
    if (lane == 0) {
        a.up_off[s] = (uint32_t)off;
        a.up_cnt[s] = cnt;
    }
    const uint32_t own_end = (s + 1) * kSC;  // first cluster after the own ones
    const uint32_t i0 = s * kSC;
    bool ok = true;
    uint32_t carry_t = NONE, carry[kSC];
#pragma unroll
    for (int k = 0; k < kSC; ++k) carry[k] = 0u;
    // reserve and write n tuples of group t from this lane
    auto emit = [&](bool on, uint32_t t, const uint32_t *rows) {
        uint32_t nrow = 0;
#pragma unroll
        for (int k = 0; k < kSC; ++k) nrow += (on && rows[k]) ? 1u : 0u;
        const uint32_t incl = warp_incl_scan(nrow);
        const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
        if (tot == 0) return;
        unsigned long long tb = 0;
        if (lane == 0) tb = atomicAdd(&a.st->tu_used, (unsigned long long)tot);
        tb = __shfl_sync(0xffffffffu, tb, 0);
        if (tb + tot > a.tu_cap) {
            ok = false;
            return;
        }
        if (nrow) {
            unsigned long long w = tb + incl - nrow;
#pragma unroll
            for (int k = 0; k < kSC; ++k)
                if (rows[k]) {
                    a.tkey[w] = (uint64_t)t * a.ncl + (i0 + k);
                    a.tval[w] = rows[k];
                    ++w;
                }
            atomicAdd(&a.lower_cnt[t], nrow);
        }
    };
    for (uint32_t b0 = 0; b0 < cnt; b0 += 32) {
        const uint32_t e = b0 + lane;
        const uint32_t J = e < cnt ? stJ[e] : 0u;
        const bool valid = e < cnt && J >= own_end;
        const uint32_t m = valid ? (uint32_t)stM[e] : 0u;
        const uint32_t t = valid ? J / kSC : NONE;
        // a carried group that does not continue here is complete
        if (carry_t != NONE && __shfl_sync(0xffffffffu, t, 0) != carry_t) {
            emit(lane == 0, carry_t, carry);
            carry_t = NONE;
        }
        const uint32_t gm = __match_any_sync(0xffffffffu, t);
        uint32_t rows[kSC];
#pragma unroll
        for (int k = 0; k < kSC; ++k) {
            rows[k] = __reduce_or_sync(gm, ((m >> k) & 1u) << (J & 7u));
            if (valid && t == carry_t) rows[k] |= carry[k];
        }
        // the group of the chunk's last entry may continue in the next chunk
        const uint32_t t31 = __shfl_sync(0xffffffffu, t, 31);
        const bool more = b0 + 32 < cnt;
        const bool hold = more && t31 != NONE && t == t31;
#pragma unroll
        for (int k = 0; k < kSC; ++k) carry[k] = __shfl_sync(0xffffffffu, rows[k], 31);
        carry_t = (more && t31 != NONE) ? t31 : NONE;
        emit(valid && lane == (uint32_t)(__ffs(gm) - 1) && !hold, t, rows);
    }
    if (carry_t != NONE) emit(lane == 0, carry_t, carry);
    if (!ok && lane == 0) atomicExch(&a.st->half_overflow, 1u);
    return ok;
}

// Shared memory of one warp: the super-cluster's particles, a chunk of 32
// consecutive octree nodes, the queue of candidate j-clusters, the particles
// and boxes of the 4 j-clusters being tested, and the encoder window.
// The tile operands are laid out for packed (two-pair) arithmetic: an i
// particle as (x, y, z, r^2), one 16-byte load per tile (the tile tests are
// bound by shared-memory bandwidth); the j particles of a lane's two pairs a
// and b as (xa, xb, ya, yb) and (za, zb, ra^2, rb^2), loaded once per
// j-cluster.  Squared radii suffice: fl(max(ri, rj)^2) = max(fl(ri^2),
// fl(rj^2)), squaring being monotone.
template <int M, int MJ>
struct SearchSmem {
    float4 ip[kSC * M];            // i particles
    float4 nlo[32], nhi[32];       // node chunk
    int2 nrg[32];
    uint32_t jq[SR_QCAP];          // candidate j-clusters, ascending
    float4 jpA[4 * MJ], jpB[4 * MJ];  // particles of the 4 j-clusters under test
    float4 ilo[kSC], ihi[kSC];     // boxes of the 8 i-clusters
    uint32_t win[WIN_WORDS];
};

// MODE 0: full list.  MODE 1: half search, upper entries and transposed
// tuples for the record assembly.  MODE 2: half list (each pair stored once,
// Sec. II-D): the half search's upper entries encoded as the record.
template <int M, int MJ, bool PER, int MODE>
__global__ void __launch_bounds__(SR_THREADS, 4) k_search(SearchArgs a, SearchCtl ctl)
{
    constexpr bool HALF = MODE != 0;  // only j-clusters from the own first one on
    constexpr int NP = (M * MJ) / 32 > 0 ? (M * MJ) / 32 : 1;  // pairs per lane per tile
    constexpr int JSTEP = 32 / M;
    constexpr uint32_t R = M / MJ;        // j-clusters per i-cluster
    constexpr int NPI = (kSC * M) / 32;   // i particles per lane for the pruning tests
    extern __shared__ __align__(16) unsigned char search_smem[];
    SearchSmem<M, MJ> &S = reinterpret_cast<SearchSmem<M, MJ> *>(search_smem)[threadIdx.x >> 5];
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    const uint32_t slot = blockIdx.x * (blockDim.x >> 5) + warp;
    // a warp without staging room stays idle; the work counter hands its
    // super-clusters to the others (warps never wait on each other here)
    if (slot >= a.stage_slots) return;
    uint32_t *stJ = a.stageJ + (size_t)slot * a.stage_cap;
    uint8_t *stM = a.stageM + (size_t)slot * a.stage_cap;
    const uint32_t II = lane % M;
    const uint32_t JJ0 = (lane / M) % MJ;
    const uint32_t grp = lane >> 3;       // j-cluster slot of this lane in the box round
    const uint32_t count = ctl.count_dev ? min(ctl.count, *ctl.count_dev) : ctl.count;

    for (;;) {
        uint32_t tk = 0;
        if (lane == 0) tk = atomicAdd(&a.st->ticket, 1u);
        tk = __shfl_sync(0xffffffffu, tk, 0);
        if (tk >= count) break;
        const uint32_t s = ctl.work ? ctl.work[tk] : tk;
        const uint32_t base = s * kSC * M;
        // the super-cluster's system: its box and its own octree subtree
        const uint32_t sy = sys_of(a.sys.pad_off, a.sys.nsys, base);
        const PerLen box = per_len(a.sys.box[sy]);
        // (clamped to the node arrays: after a node overflow in a graph replay
        // the tables may be stale, and the replay is reported as failed)
        const uint32_t vroot = min(a.sys.root[sy], a.nnodes - 1);
        const uint32_t vend = min((uint32_t)__float_as_int(a.nhi[vroot].w), a.nnodes);

        // i-cluster box of this lane's cluster (lane & 7)
        if (lane < kSC) {
            S.ilo[lane] = a.clo[s * kSC + lane];
            S.ihi[lane] = a.chi[s * kSC + lane];
        }
        // pruning particles base + lane + 32 t, staged as (x, y, z, r) for
        // the tile tests.  Dummies sit at infinity, which no open axis comes
        // near; on periodic systems they are flagged off as well (a point at
        // infinity has no meaningful periodic gap).  Per-particle tests, not boxes of several particles:
        // particles adjacent on the curve can lie far apart in sparse
        // regions, and a box around them would admit far too many nodes.
        float4 qp[NPI];
        float qr[NPI];
        uint32_t qok = 0;  // bit t: particle t of this lane is real
        __syncwarp();
#pragma unroll
        for (int t = 0; t < NPI; ++t) {
            const float4 p = a.pos[base + lane + 32 * t];
            const float r = __fmul_rn(a.support, p.w);
            const float rr = __fmul_rn(r, r);
            S.ip[lane + 32 * t] = make_float4(p.x, p.y, p.z, rr);
            const bool real = p.x == p.x;
            qp[t] = real ? p : make_float4(INFINITY, INFINITY, INFINITY, 0.f);
            qr[t] = real ? r : 0.f;
            qok |= real ? 1u << t : 0u;
        }

        // open systems, two pruning particles per lane: their coordinates as
        // packed pairs for the node tests
        f32x2 qx2 = 0, qy2 = 0, qz2 = 0;
        if constexpr (!PER && NPI == 2) {
            qx2 = pk2(qp[0].x, qp[1].x);
            qy2 = pk2(qp[0].y, qp[1].y);
            qz2 = pk2(qp[0].z, qp[1].z);
        }
        uint32_t cnt = 0, tiles = 0, nvis = 0, lvis = 0, jex = 0, ttests = 0, qn = 0;
        // the half search takes only j-clusters from its own first one on
        int lastJ = HALF ? (int)(base / MJ) - 1 : -1;

        // Test the queued j-clusters, 4 per round, and stage the hits.
        auto flush = [&]() {
            for (uint32_t b = 0; b < qn; b += 4) {
                const uint32_t nq = min(4u, qn - b);
                // stage the particles and boxes of up to 4 j-clusters
                __syncwarp();
                bool cand = false;
                if (grp < nq) {
                    const uint32_t Jl = S.jq[b + grp];
#pragma unroll
                    for (uint32_t jl = lane & 7; jl < (uint32_t)MJ; jl += 8) {
                        const float4 p = a.pos[Jl * MJ + jl];
                        const float r = __fmul_rn(a.support, p.w);
                        // slot of the lane's pair (a, b) holding jl, and its half
                        uint32_t slot = jl, half = 0;
                        if constexpr (NP >= 2) {
                            const uint32_t t = jl / JSTEP;
                            slot = (jl - t * JSTEP) + (t >> 1) * 2u * JSTEP;
                            half = t & 1u;
                        }
                        float *pa = reinterpret_cast<float *>(&S.jpA[grp * MJ + slot]);
                        float *pb = reinterpret_cast<float *>(&S.jpB[grp * MJ + slot]);
                        pa[half] = p.x;
                        pa[2 + half] = p.y;
                        pb[half] = p.z;
                        pb[2 + half] = __fmul_rn(r, r);
                    }
                    // 4 j-clusters x 8 i-cluster boxes, one per lane: may some
                    // pair be neighbors?
                    cand = boxes_near<PER>(S.ilo[lane & 7], S.ihi[lane & 7], a.jlo[Jl], a.jhi[Jl],
                                           box);
                }
                const uint32_t bal = __ballot_sync(0xffffffffu, cand);
                __syncwarp();
                for (uint32_t q = 0; q < nq; ++q) {
                    const uint32_t cm = (bal >> (8 * q)) & 0xffu;
                    if (!cm) continue;
                    const uint32_t J = S.jq[b + q];
                    // exact FP32 test of the candidate M x MJ tiles; the j
                    // operands of the first two pairs stay in registers
                    uint32_t mask = 0;
                    ttests += __popc(cm);
                    const float4 jA0 = S.jpA[q * MJ + JJ0], jB0 = S.jpB[q * MJ + JJ0];
                    for (uint32_t bits = cm; bits; bits &= bits - 1u) {
                        const int k = __ffs(bits) - 1;  // candidate tiles only, ascending
                        const float4 pi = S.ip[k * M + II];
                        // pair (i, j) is a self pair iff II - jl == delta
                        const int delta = (int)(J * MJ) - (int)(base + k * M);
                        bool hit = false;
                        if constexpr (NP >= 2) {
                            const f32x2 ix = pk2(pi.x, pi.x), iy = pk2(pi.y, pi.y);
                            const f32x2 iz = pk2(pi.z, pi.z);
#pragma unroll
                            for (int u = 0; u < NP / 2; ++u) {  // stops at the first hit
                                const uint32_t slot = JJ0 + 2u * u * JSTEP;
                                const float4 jA = u == 0 ? jA0 : S.jpA[q * MJ + slot];
                                const float4 jB = u == 0 ? jB0 : S.jpB[q * MJ + slot];
                                float d2a, d2b;
                                pair_d2_x2<PER>(pk2(jA.x, jA.y), pk2(jA.z, jA.w), pk2(jB.x, jB.y), ix, iy,
                                                iz, box, d2a, d2b);
                                const int ca = (int)II - (int)slot, cb = ca - JSTEP;
                                const bool h = (d2a < fmaxf(pi.w, jB.z) && ca != delta) ||
                                               (d2b < fmaxf(pi.w, jB.w) && cb != delta);
                                if (__any_sync(0xffffffffu, h)) {
                                    hit = true;
                                    break;
                                }
                            }
                        } else {
                            const float d2 = pair_d2<PER>(pi, make_float4(jA0.x, jA0.z, jB0.x, 0.f), box);
                            hit = __any_sync(0xffffffffu, d2 < fmaxf(pi.w, jB0.z) &&
                                                              (int)II - (int)JJ0 != delta);
                        }
                        if (hit) mask |= 1u << k;
                    }
                    if (mask) {
                        if (lane == 0 && cnt < a.stage_cap) {
                            stJ[cnt] = J;
                            stM[cnt] = (uint8_t)mask;
                        }
                        ++cnt;
                        tiles += __popc(mask);
                    }
                }
            }
            qn = 0;
        };

        // Stackless pre-order walk of the system's subtree; nodes are read in
        // coalesced chunks of 32 consecutive nodes staged in shared memory.
        uint32_t v = vroot, cb = 0;
        bool have = false, past = false;
        while (v < vend) {
            if (!have || v - cb >= 32u) {
                cb = v;
                have = true;
                __syncwarp();
                const uint32_t u = cb + lane;
                if (u < vend) {
                    S.nlo[lane] = a.nlo[u];
                    S.nhi[lane] = a.nhi[u];
                    S.nrg[lane] = a.nrng[u];
                }
                __syncwarp();
            }
            const float4 nlo = S.nlo[v - cb];
            const float4 nhi = S.nhi[v - cb];
            const uint32_t skip = (uint32_t)__float_as_int(nhi.w);
            // wholly before the own particles: only nodes ahead of the first
            // accepted leaf can be (that leaf holds particle base, and every
            // later node in pre-order holds later particles)
            if (HALF && !past && (uint32_t)S.nrg[v - cb].y <= base) {
                v = skip > v ? skip : v + 1;
                continue;
            }
            ++nvis;
            bool near = false;
            if constexpr (!PER && NPI == 2) {
                // the gap of each particle to the node box per axis, packed
                float g[3][2];
                const f32x2 lo2[3] = {pk2(nlo.x, nlo.x), pk2(nlo.y, nlo.y), pk2(nlo.z, nlo.z)};
                const f32x2 hi2[3] = {pk2(nhi.x, nhi.x), pk2(nhi.y, nhi.y), pk2(nhi.z, nhi.z)};
                const f32x2 q2[3] = {qx2, qy2, qz2};
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) {
                    float a0, a1, b0, b1;
                    unpk2(sub2_rn(lo2[ax], q2[ax]), a0, a1);
                    unpk2(sub2_rn(q2[ax], hi2[ax]), b0, b1);
                    g[ax][0] = fmaxf(0.f, fmaxf(a0, b0));
                    g[ax][1] = fmaxf(0.f, fmaxf(a1, b1));
                }
                const f32x2 gx = pk2(g[0][0], g[0][1]), gy = pk2(g[1][0], g[1][1]);
                const f32x2 gz = pk2(g[2][0], g[2][1]);
                float d2a, d2b, rra, rrb;
                sum_sq_x2(gx, gy, gz, d2a, d2b);
                const float ra = fmaxf(qr[0], nlo.w), rb = fmaxf(qr[1], nlo.w);
                unpk2(mul2_rn(pk2(ra, rb), pk2(ra, rb)), rra, rrb);
                near = d2a <= rra || d2b <= rrb;
            } else {
#pragma unroll
                for (int t = 0; t < NPI; ++t)
                    near |= (!PER || ((qok >> t) & 1u)) && point_near<PER>(qp[t], qr[t], nlo, nhi, box);
            }
            if (!__any_sync(0xffffffffu, near)) {
                v = skip > v ? skip : v + 1;  // always advances
                continue;
            }
            if (skip != v + 1) {  // internal node: descend to its first child
                ++v;
                continue;
            }
            // leaf: queue its j-clusters not queued yet (leaves can share one)
            const int2 rg = S.nrg[v - cb];
            past = true;
            int Jlo = max(rg.x / MJ, lastJ + 1);
            const int Jhi = (rg.y - 1) / MJ;
            ++lvis;
            if (Jhi >= Jlo) {
                jex += (uint32_t)(Jhi - Jlo + 1);
                lastJ = Jhi;
                while (Jlo <= Jhi) {
                    if (qn == SR_QCAP) flush();
                    const uint32_t c = min((uint32_t)(Jhi - Jlo + 1), SR_QCAP - qn);
                    __syncwarp();
                    for (uint32_t e = lane; e < c; e += 32) S.jq[qn + e] = (uint32_t)Jlo + e;
                    __syncwarp();
                    qn += c;
                    Jlo += (int)c;
                }
            }
            ++v;
        }
        flush();
        __syncwarp();
        const bool staged = cnt <= a.stage_cap;
        bool ok = staged;
        if (!staged) {
            if (lane == 0) atomicMax(&a.st->max_count, cnt);
        } else if constexpr (MODE == 1) {
            // a buffer overflow here makes the host re-run every super-cluster
            ok = half_output(cnt, stJ, stM, a, s);
        } else {
            ok = encode_record(
                cnt, [&](uint32_t t) { return stJ[t]; },
                [&](uint32_t t) { return (uint32_t)stM[t]; }, S.win, a, s);
            if (!ok && lane == 0) atomicExch(&a.st->list_overflow, 1u);
        }
        if (lane == 0) {
            if (!ok) {
                if (MODE != 1 || !staged) {
                    uint32_t r = atomicAdd(&a.st->stage_overflow, 1u);
                    ctl.redo[r] = s;
                }
                a.rec_off[s] = kBadRecord;
            } else if (MODE != 1) {
                atomicAdd(&a.st->n_entries, (unsigned long long)cnt);
                atomicAdd(&a.st->n_tiles, (unsigned long long)tiles);
            }
            atomicAdd(&a.st->node_visits, (unsigned long long)nvis);
            atomicAdd(&a.st->leaf_visits, (unsigned long long)lvis);
            atomicAdd(&a.st->j_examined, (unsigned long long)jex);
            atomicAdd(&a.st->tile_tests, (unsigned long long)ttests);
        }
    }
}

template <int M, int MJ, int MODE>
static cudaError_t launch_m(const SearchArgs &a, const SearchCtl &c, int per, int grid, int threads,
                            cudaStream_t s)
{
    const size_t smem = (size_t)(threads / 32) * sizeof(SearchSmem<M, MJ>);
    const size_t smax = (size_t)SR_WARPS * sizeof(SearchSmem<M, MJ>);
    const void *fn = per ? (const void *)k_search<M, MJ, true, MODE>
                         : (const void *)k_search<M, MJ, false, MODE>;
    cudaError_t e = set_max_dynamic_smem(fn, smax);
    if (e != cudaSuccess) return e;
    if (per)
        k_search<M, MJ, true, MODE><<<grid, threads, smem, s>>>(a, c);
    else
        k_search<M, MJ, false, MODE><<<grid, threads, smem, s>>>(a, c);
    return cudaGetLastError();
}

cudaError_t launch_search_ctl(const SearchArgs &a, const uint32_t *work, uint32_t count,
                              uint32_t *redo, int M, int any_periodic, int grid, int threads,
                              cudaStream_t s, const uint32_t *count_dev)
{
    SearchCtl c{work, count, redo, count_dev};
    if (threads != 128 && threads != SR_THREADS) return cudaErrorInvalidValue;
    if (a.half && a.mj != M) return cudaErrorInvalidValue;  // needs j-clusters = i-clusters
    if (a.half < 0 || a.half > 2) return cudaErrorInvalidValue;
    switch (M * 100 + a.mj) {
    case 404:
        if (a.half == 1) return launch_m<4, 4, 1>(a, c, any_periodic, grid, threads, s);
        if (a.half == 2) return launch_m<4, 4, 2>(a, c, any_periodic, grid, threads, s);
        return launch_m<4, 4, 0>(a, c, any_periodic, grid, threads, s);
    case 808:
        if (a.half == 1) return launch_m<8, 8, 1>(a, c, any_periodic, grid, threads, s);
        if (a.half == 2) return launch_m<8, 8, 2>(a, c, any_periodic, grid, threads, s);
        return launch_m<8, 8, 0>(a, c, any_periodic, grid, threads, s);
    case 804: return launch_m<8, 4, 0>(a, c, any_periodic, grid, threads, s);
    case 1616:
        if (a.half == 1) return launch_m<16, 16, 1>(a, c, any_periodic, grid, threads, s);
        if (a.half == 2) return launch_m<16, 16, 2>(a, c, any_periodic, grid, threads, s);
        return launch_m<16, 16, 0>(a, c, any_periodic, grid, threads, s);
    case 1608: return launch_m<16, 8, 0>(a, c, any_periodic, grid, threads, s);
    default: return cudaErrorInvalidValue;
    }
}

// Record assembly of the half search: one warp per super-cluster t.  Its
// record is the sorted tuples addressed to it (j-clusters below its own
// clusters; keys t * ncl + J, values the mask bits) followed by its upper
// entries, encoded exactly like a record of the full search.
__global__ void __launch_bounds__(SR_THREADS) k_assemble(SearchArgs a)
{
    __shared__ uint32_t wins[SR_WARPS][WIN_WORDS];
    const unsigned lane = lane_id();
    uint32_t *win = wins[threadIdx.x >> 5];
    for (;;) {
        uint32_t t = 0;
        if (lane == 0) t = atomicAdd(&a.st->asm_ticket, 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= a.nsc) break;
        if (a.st->half_overflow || a.st->stage_overflow) {
            // incomplete tuples or upper entries (a graph replay that outgrew
            // its buffers, reported by nl_graph_check): empty records
            if (lane == 0) a.rec_off[t] = kBadRecord;
            continue;
        }
        const uint32_t lc = a.lower_cnt[t], so = a.seg_off[t];
        const uint32_t uc = a.up_cnt[t], uo = a.up_off[t];
        const uint32_t cnt = lc + uc;
        const uint64_t kb = (uint64_t)t * a.ncl;
        auto getJ = [&](uint32_t i) -> uint32_t {
            return i < lc ? (uint32_t)(a.tkey[so + i] - kb) : a.uJ[uo + (i - lc)];
        };
        auto getM = [&](uint32_t i) -> uint32_t {
            return i < lc ? a.tval[so + i] : (uint32_t)a.uM[uo + (i - lc)];
        };
        const bool ok = encode_record(cnt, getJ, getM, win, a, t);
        uint32_t tiles = 0;
        for (uint32_t i = lane; i < cnt; i += 32) tiles += __popc(getM(i));
        tiles = warp_sum(tiles);
        if (lane == 0) {
            if (!ok) {
                atomicExch(&a.st->list_overflow, 1u);
                a.rec_off[t] = kBadRecord;
            } else {
                atomicAdd(&a.st->n_entries, (unsigned long long)cnt);
                atomicAdd(&a.st->n_tiles, (unsigned long long)tiles);
            }
        }
    }
}

__global__ void k_classify(const uint32_t *__restrict__ list, uint32_t n, int M, SysTables t,
                           const float4 *__restrict__ clo, const float4 *__restrict__ chi,
                           const float4 *__restrict__ nlo, uint32_t node_cap,
                           uint32_t *__restrict__ out_int, uint32_t *__restrict__ out_bnd,
                           Status *st)
{
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const uint32_t s = list ? list[k] : k;
    const uint32_t sy = sys_of(t.pad_off, t.nsys, s * kSC * M);
    const DevBox &b = t.box[sy];
    // largest radius of the system: its octree root (clamped as in the search)
    const float R = nlo[min(t.root[sy], node_cap - 1)].w;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int c = 0; c < kSC; ++c) {
        const float4 a = clo[s * kSC + c], z = chi[s * kSC + c];
        lo[0] = fminf(lo[0], a.x); lo[1] = fminf(lo[1], a.y); lo[2] = fminf(lo[2], a.z);
        hi[0] = fmaxf(hi[0], z.x); hi[1] = fmaxf(hi[1], z.y); hi[2] = fmaxf(hi[2], z.z);
    }
    bool interior = true;
    for (int a = 0; a < 3; ++a) {
        if (!b.per[a]) continue;
        // a wrapped pair needs a particle within R of a face; the margin covers
        // the roundings of the gaps here and of the wrapped differences
        const float m = R + R * 1e-5f + b.len[a] * 1e-6f;
        interior = interior && (lo[a] - b.lo[a] > m) && (b.hi[a] - hi[a] > m);
    }
    if (interior)
        out_int[atomicAdd(&st->n_int, 1u)] = s;
    else
        out_bnd[atomicAdd(&st->n_bnd, 1u)] = s;
}

cudaError_t launch_classify(const uint32_t *list, uint32_t n, int M, const SysTables &t,
                            const float4 *clo, const float4 *chi, const float4 *nlo,
                            uint32_t node_cap, uint32_t *out_int, uint32_t *out_bnd, Status *st,
                            cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_classify<<<(n + 255) / 256, 256, 0, s>>>(list, n, M, t, clo, chi, nlo, node_cap, out_int,
                                               out_bnd, st);
    return cudaGetLastError();
}

// keys[k] = fill for min(*used, cap) <= k < cap
__global__ void k_fill_keys(uint64_t *keys, uint32_t cap, const unsigned long long *used,
                            uint64_t fill)
{
    const unsigned long long u = *used;
    const uint32_t from = u < cap ? (uint32_t)u : cap;
    for (uint32_t k = from + blockIdx.x * blockDim.x + threadIdx.x; k < cap; k += gridDim.x * blockDim.x)
        keys[k] = fill;
}

cudaError_t launch_fill_keys(uint64_t *keys, uint32_t cap, const unsigned long long *used,
                             uint64_t fill, cudaStream_t s)
{
    k_fill_keys<<<1024, 256, 0, s>>>(keys, cap, used, fill);
    return cudaGetLastError();
}

cudaError_t launch_assemble(const SearchArgs &a, int grid, cudaStream_t s)
{
    k_assemble<<<grid, SR_THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace nlg
