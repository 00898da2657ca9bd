// SFC permutation with cluster boxes, and the octree built from the sorted
// keys (Sec. II-A: clusters are consecutive packs of M SFC particles; the
// octree is traversed from the root to collect neighbor clusters).
//
// Octree definition: leaves are the maximal key-prefix cells holding at most
// B particles (level-21 cells are leaves whatever their count); internal
// nodes are all non-empty cells above them; nodes are stored in pre-order
// with a skip index (first node after the subtree), so traversal needs no
// stack.  Construction is data-parallel:
//   1. the cell of particle k at level l holds more than B particles iff
//      some window of B+1 consecutive sorted keys containing k shares the
//      level-l prefix, so k's leaf level is 1 + max over those windows of
//      lcp_level(key[s], key[s+B]);
//   2. a particle starts a leaf where (level, prefix) changes; a scan numbers
//      the leaves;
//   3. leaf i opens the nodes at levels lcp(leaf i-1, leaf i)+1 .. level_i,
//      which is exactly the pre-order; a scan places them;
//   4. subtree ends come from binary searches of the key prefix; boxes are
//      reduced bottom-up by "last child to arrive" counters (no waiting).
#include "nl_internal.cuh"

namespace nlg {

// ---------------------------------------------------------------------------
// Permute + cluster boxes
// ---------------------------------------------------------------------------
template <int M>
__global__ void __launch_bounds__(256) k_permute(uint32_t npad, SysTables t,
                                                 const uint32_t *__restrict__ perm,
                                                 const float *__restrict__ x,
                                                 const float *__restrict__ y,
                                                 const float *__restrict__ z,
                                                 const float *__restrict__ h, float support,
                                                 float4 *__restrict__ pos,
                                                 uint32_t *__restrict__ perm_pad,
                                                 float4 *__restrict__ clo,
                                                 float4 *__restrict__ chi, int MJ,
                                                 float4 *__restrict__ jlo,
                                                 float4 *__restrict__ jhi)
{
    uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;  // npad is a multiple of 32
    if (k >= npad) return;
    const uint32_t sy = sys_of(t.pad_off, t.nsys, k);
    const uint32_t local = k - t.pad_off[sy];
    const bool real = local < t.off[sy + 1] - t.off[sy];
    float4 p;
    float r;
    const float nan = __int_as_float(0x7fc00000);
    if (real) {
        uint32_t o = perm[t.off[sy] + local];
        p = make_float4(x[o], y[o], z[o], h[o]);
        r = __fmul_rn(support, p.w);
        perm_pad[k] = o;
    } else {
        p = make_float4(nan, nan, nan, 0.f);
        r = 0.f;
        perm_pad[k] = 0xffffffffu;
    }
    pos[k] = p;
    cluster_box_reduce<M>(k, real, p, r, MJ, clo, chi, jlo, jhi);
}

cudaError_t launch_permute(uint32_t npad, int M, int MJ, const SysTables &t, const uint32_t *perm,
                           const float *x, const float *y, const float *z, const float *h,
                           float support, float4 *pos, uint32_t *perm_pad, float4 *clo,
                           float4 *chi, float4 *jlo, float4 *jhi, cudaStream_t s)
{
    unsigned grid = (npad + 255) / 256;
    if (MJ == M) jlo = jhi = nullptr;
    else if (!jlo || !jhi || MJ < 1 || M % MJ) return cudaErrorInvalidValue;
    switch (M) {
    case 4: k_permute<4><<<grid, 256, 0, s>>>(npad, t, perm, x, y, z, h, support, pos, perm_pad, clo, chi, MJ, jlo, jhi); break;
    case 8: k_permute<8><<<grid, 256, 0, s>>>(npad, t, perm, x, y, z, h, support, pos, perm_pad, clo, chi, MJ, jlo, jhi); break;
    case 16: k_permute<16><<<grid, 256, 0, s>>>(npad, t, perm, x, y, z, h, support, pos, perm_pad, clo, chi, MJ, jlo, jhi); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Device-wide exclusive scan over values produced by a functor.
// ---------------------------------------------------------------------------
constexpr int SC_THREADS = 256;
constexpr int SC_ITEMS = 8;
constexpr int SC_TILE = SC_THREADS * SC_ITEMS;

size_t scan_bsum_words(uint32_t n) { return (size_t)(n + SC_TILE - 1) / SC_TILE + 2; }

template <class F>
__global__ void __launch_bounds__(SC_THREADS) k_scan_reduce(F f, uint32_t n, const uint32_t *n_dev,
                                                           uint32_t *bsum)
{
    __shared__ uint32_t sh[33];
    if (n_dev) n = min(n, *n_dev);
    uint32_t base = blockIdx.x * SC_TILE, v = 0;
#pragma unroll
    for (int it = 0; it < SC_ITEMS; ++it) {
        uint32_t k = base + it * SC_THREADS + threadIdx.x;
        if (k < n) v += f(k);
    }
    uint32_t t;
    block_excl_scan(v, sh, &t);
    if (threadIdx.x == 0) bsum[blockIdx.x] = t;
}

__global__ void __launch_bounds__(1024) k_scan_bsums(uint32_t *bsum, uint32_t nb, uint32_t *total)
{
    __shared__ uint32_t sh[33];
    uint32_t carry = 0;
    for (uint32_t b = 0; b < nb; b += 1024) {
        uint32_t i = b + threadIdx.x;
        uint32_t v = i < nb ? bsum[i] : 0u;
        uint32_t t;
        uint32_t e = block_excl_scan(v, sh, &t);
        if (i < nb) bsum[i] = carry + e;
        carry += t;
    }
    if (threadIdx.x == 0) *total = carry;
}

// Every element k gets sink(k, exclusive prefix, value); elements are
// processed in blocked order (thread t owns SC_ITEMS consecutive elements).
template <class F, class S>
__global__ void __launch_bounds__(SC_THREADS) k_scan_apply(F f, S sink, uint32_t n,
                                                          const uint32_t *n_dev,
                                                          const uint32_t *bsum)
{
    __shared__ uint32_t sh[33];
    if (n_dev) n = min(n, *n_dev);
    uint32_t base = blockIdx.x * SC_TILE + threadIdx.x * SC_ITEMS;
    uint32_t v[SC_ITEMS], s = 0;
#pragma unroll
    for (int it = 0; it < SC_ITEMS; ++it) {
        uint32_t k = base + it;
        v[it] = k < n ? f(k) : 0u;
        s += v[it];
    }
    uint32_t t;
    uint32_t e = block_excl_scan(s, sh, &t) + bsum[blockIdx.x];
#pragma unroll
    for (int it = 0; it < SC_ITEMS; ++it) {
        uint32_t k = base + it;
        if (k < n) sink(k, e, v[it]);
        e += v[it];
    }
}

// n: element count, or an upper bound when n_dev points at the count on the
// device (launches cover the bound; elements past *n_dev contribute zero).
template <class F, class S>
static cudaError_t scan_exclusive(F f, S sink, uint32_t n, const uint32_t *n_dev, uint32_t *bsum,
                                  uint32_t *total, cudaStream_t s)
{
    uint32_t nb = (n + SC_TILE - 1) / SC_TILE;
    if (nb == 0) {
        return cudaMemsetAsync(total, 0, 4, s);
    }
    k_scan_reduce<<<nb, SC_THREADS, 0, s>>>(f, n, n_dev, bsum);
    k_scan_bsums<<<1, 1024, 0, s>>>(bsum, nb, total);
    k_scan_apply<<<nb, SC_THREADS, 0, s>>>(f, sink, n, n_dev, bsum);
    return cudaGetLastError();
}

struct ArrayVal {
    const uint32_t *a;
    __device__ uint32_t operator()(uint32_t k) const { return a[k]; }
};
struct ArraySink {
    uint32_t *o;
    __device__ void operator()(uint32_t k, uint32_t e, uint32_t) const { o[k] = e; }
};

cudaError_t exclusive_scan_u32(const uint32_t *cnt, uint32_t *seg_off, uint32_t n, uint32_t *bsum,
                               uint32_t *total, cudaStream_t s)
{
    return scan_exclusive(ArrayVal{cnt}, ArraySink{seg_off}, n, nullptr, bsum, total, s);
}

// ---------------------------------------------------------------------------
// Step 1: leaf level of every particle
// ---------------------------------------------------------------------------
// lcp level of the window [s, s+B], 0xff when it spans two systems
__global__ void k_lcp_window(const uint64_t *__restrict__ keys, uint32_t n, int B, SysTables t,
                             uint8_t *__restrict__ lcp)
{
    uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s + (uint32_t)B < n) {
        bool same = t.nsys == 1 || sys_of(t.off, t.nsys, s) == sys_of(t.off, t.nsys, s + B);
        lcp[s] = same ? (uint8_t)lcp_level(keys[s], keys[s + B]) : (uint8_t)0xffu;
    }
}

constexpr int LL_THREADS = 512;

// lev[k] = min(21, 1 + max_{s in [k-B, k], 0 <= s < n-B} lcp[s]); n <= B -> 0
__global__ void __launch_bounds__(LL_THREADS) k_leaf_level(const uint8_t *__restrict__ lcp,
                                                           uint32_t n, int B,
                                                           uint8_t *__restrict__ lev)
{
    // window values v = lcp + 1, 0 where no window (spans systems or out of
    // range), so lev = max v over the B+1 windows ending at k (0: no window,
    // the system root is a leaf).  The sliding maximum comes from a doubling
    // table: after the steps q = 1, 2, .., P/2 entry i holds max v[i, i+P),
    // P the largest power of two <= B+1, and two entries cover a window.
    extern __shared__ uint8_t win[];  // LL_THREADS + B entries
    constexpr int PER = 3;            // entries per thread (B <= 1024)
    const int L = LL_THREADS + B;
    const int64_t k0 = (int64_t)blockIdx.x * LL_THREADS;
    const int64_t nw = (int64_t)n - B;  // number of windows
    for (int t = threadIdx.x; t < L; t += LL_THREADS) {
        int64_t s = k0 - B + t;
        uint8_t v = (s >= 0 && s < nw) ? lcp[s] : 0xffu;
        win[t] = v == 0xffu ? (uint8_t)0 : (uint8_t)(v + 1);
    }
    __syncthreads();
    int P = 1;
    while (2 * P <= B + 1) P *= 2;
    for (int q = 1; q < P; q *= 2) {
        uint8_t r[PER];
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const int i = threadIdx.x + j * LL_THREADS;
            r[j] = 0;
            if (i < L) r[j] = (i + q < L) ? max(win[i], win[i + q]) : win[i];
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const int i = threadIdx.x + j * LL_THREADS;
            if (i < L) win[i] = r[j];
        }
        __syncthreads();
    }
    const int64_t k = k0 + threadIdx.x;
    if (k >= n) return;
    const int l = max(win[threadIdx.x], win[threadIdx.x + (B + 1) - P]);
    lev[k] = (uint8_t)(l > kMaxLevel ? kMaxLevel : l);
}

// ---------------------------------------------------------------------------
// Step 2: leaf starts
// ---------------------------------------------------------------------------
struct LeafFlag {
    const uint64_t *keys;
    const uint8_t *lev;
    SysTables t;
    __device__ uint32_t operator()(uint32_t k) const
    {
        if (k == 0) return 1u;
        if (t.nsys > 1 && sys_of(t.off, t.nsys, k) != sys_of(t.off, t.nsys, k - 1)) return 1u;
        int l = lev[k];
        if (l != lev[k - 1]) return 1u;
        if (l == 0) return 0u;
        int sh = 63 - 3 * l;
        return (keys[k] >> sh) != (keys[k - 1] >> sh) ? 1u : 0u;
    }
};

struct LeafSink {
    const uint8_t *lev;
    uint32_t n;
    uint32_t *leaf_first;
    uint8_t *leaf_lev;
    __device__ void operator()(uint32_t k, uint32_t excl, uint32_t v) const
    {
        if (v) {
            leaf_first[excl] = k;
            leaf_lev[excl] = lev[k];
        }
        if (k == n - 1) leaf_first[excl + v] = n;
    }
};

cudaError_t octree_leaves(const uint64_t *keys, uint32_t n, int bucket, const SysTables &t,
                          uint8_t *lcp, uint8_t *lev, uint32_t *leaf_first, uint8_t *leaf_lev,
                          uint32_t *bsum, Status *st, cudaStream_t s)
{
    if (n > (uint32_t)bucket)
        k_lcp_window<<<(n - bucket + 255) / 256, 256, 0, s>>>(keys, n, bucket, t, lcp);
    k_leaf_level<<<(n + LL_THREADS - 1) / LL_THREADS, LL_THREADS, LL_THREADS + bucket, s>>>(
        lcp, n, bucket, lev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return scan_exclusive(LeafFlag{keys, lev, t}, LeafSink{lev, n, leaf_first, leaf_lev}, n,
                          nullptr, bsum, &st->n_leaves, s);
}

// ---------------------------------------------------------------------------
// Step 3: nodes opened by each leaf
// ---------------------------------------------------------------------------
// lcp level of leaf i with the previous leaf; -1 for the first leaf of a
// system (it opens that system's root)
__device__ __forceinline__ int leaf_lcp(const uint64_t *keys, const uint32_t *leaf_first,
                                        const SysTables &t, uint32_t i)
{
    if (i == 0) return -1;
    const uint32_t a = leaf_first[i - 1], b = leaf_first[i];
    if (t.nsys > 1 && sys_of(t.off, t.nsys, a) != sys_of(t.off, t.nsys, b)) return -1;
    return lcp_level(keys[a], keys[b]);
}

struct NodeCount {
    const uint64_t *keys;
    const uint32_t *leaf_first;
    const uint8_t *leaf_lev;
    SysTables t;
    __device__ uint32_t operator()(uint32_t i) const
    {
        return (uint32_t)((int)leaf_lev[i] - leaf_lcp(keys, leaf_first, t, i));
    }
};

struct NodeSink {
    const uint32_t *nl;   // leaf count on the device
    uint32_t *nodeoff;
    __device__ void operator()(uint32_t i, uint32_t excl, uint32_t v) const
    {
        nodeoff[i] = excl;
        if (i == *nl - 1) nodeoff[i + 1] = excl + v;
    }
};

cudaError_t octree_count_nodes(const uint64_t *keys, uint32_t n, const SysTables &t,
                               const uint32_t *leaf_first, const uint8_t *leaf_lev,
                               uint32_t *nodeoff, uint32_t *bsum, Status *st, cudaStream_t s)
{
    return scan_exclusive(NodeCount{keys, leaf_first, leaf_lev, t},
                          NodeSink{&st->n_leaves, nodeoff}, n, &st->n_leaves, bsum, &st->n_nodes, s);
}

// ---------------------------------------------------------------------------
// Step 4: emit nodes, then boxes bottom-up
// ---------------------------------------------------------------------------
// first index in [lo, hi) with keys[idx] >= bound
__device__ __forceinline__ uint32_t lower_bound_u64(const uint64_t *keys, uint32_t lo, uint32_t hi,
                                                    uint64_t bound)
{
    while (lo < hi) {
        uint32_t mid = lo + ((hi - lo) >> 1);
        if (keys[mid] < bound) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// leaf index whose first particle is exactly p (p is a leaf start)
__device__ __forceinline__ uint32_t leaf_of(const uint32_t *leaf_first, uint32_t nl, uint32_t p)
{
    uint32_t lo = 0, hi = nl;
    while (lo < hi) {
        uint32_t mid = lo + ((hi - lo) >> 1);
        if (leaf_first[mid] < p) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void k_emit_nodes(const uint64_t *__restrict__ keys, uint32_t n, uint32_t node_cap,
                             SysTables t, const uint32_t *__restrict__ leaf_first,
                             const uint8_t *__restrict__ leaf_lev,
                             const uint32_t *__restrict__ nodeoff, OctreeOut o, Status *st)
{
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t nl = st->n_leaves, nn = st->n_nodes;
    if (i >= nl) return;
    if (nodeoff[i + 1] > node_cap) {  // no room: counted, nothing written
        atomicAdd(&st->node_overflow, nodeoff[i + 1] - max(nodeoff[i], node_cap));
        return;
    }
    const int c = leaf_lcp(keys, leaf_first, t, i);
    const uint32_t v0 = nodeoff[i], e = nodeoff[i + 1] - v0;
    const uint32_t first = leaf_first[i];
    const uint32_t sy = sys_of(t.off, t.nsys, first);
    const uint32_t sbeg = t.off[sy], send = t.off[sy + 1];
    const int shift_pad = (int)(t.pad_off[sy] - sbeg);  // sorted -> padded index
    const uint64_t kf = keys[first];
    for (uint32_t tt = 0; tt < e; ++tt) {
        const uint32_t v = v0 + tt;
        const int l = c + 1 + (int)tt;
        uint32_t end, skip;
        if (tt == e - 1) {
            end = leaf_first[i + 1];
            skip = v + 1;
        } else {
            if (l == 0) {
                end = send;
            } else {
                int sh = 63 - 3 * l;
                uint64_t bound = ((kf >> sh) + 1ull) << sh;
                end = lower_bound_u64(keys, first, send, bound);
            }
            skip = end >= n ? nn : nodeoff[leaf_of(leaf_first, nl, end)];
        }
        int32_t parent;
        if (tt > 0) {
            parent = (int32_t)(v - 1);
        } else if (c < 0) {
            parent = -1;  // the root of system sy
            t.root[sy] = v;
        } else {
            // ancestor of leaf i at level c, opened by the leaf holding its
            // first particle
            uint32_t pf;
            if (c == 0) {
                pf = sbeg;
            } else {
                int sh = 63 - 3 * c;
                pf = lower_bound_u64(keys, sbeg, first, (kf >> sh) << sh);
            }
            uint32_t j = leaf_of(leaf_first, nl, pf);
            int cj = leaf_lcp(keys, leaf_first, t, j);
            parent = (int32_t)(nodeoff[j] + (uint32_t)(c - cj - 1));
        }
        o.nrng[v] = make_int2((int)first + shift_pad, (int)end + shift_pad);
        o.nlevel[v] = (uint8_t)l;
        o.nparent[v] = parent;
        o.nhi[v] = make_float4(0.f, 0.f, 0.f, __int_as_float((int)skip));
        if (parent >= 0) atomicAdd(&o.nchild[parent], 1u);
    }
}

__global__ void k_node_boxes(uint32_t node_cap, const float4 *__restrict__ pos, float support,
                             OctreeOut o, const Status *st)
{
    uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= min(node_cap, st->n_nodes) || st->node_overflow) return;
    int skip = __float_as_int(o.nhi[v].w);
    if ((uint32_t)skip != v + 1) return;  // internal nodes are reduced by their last child
    int2 rg = o.nrng[v];
    float lx = INFINITY, ly = INFINITY, lz = INFINITY, r = 0.f;
    float hx = -INFINITY, hy = -INFINITY, hz = -INFINITY;
    for (int k = rg.x; k < rg.y; ++k) {
        float4 p = pos[k];
        lx = fminf(lx, p.x); ly = fminf(ly, p.y); lz = fminf(lz, p.z);
        hx = fmaxf(hx, p.x); hy = fmaxf(hy, p.y); hz = fmaxf(hz, p.z);
        r = fmaxf(r, __fmul_rn(support, p.w));
    }
    o.nlo[v] = make_float4(lx, ly, lz, r);
    o.nhi[v] = make_float4(hx, hy, hz, __int_as_float(skip));
    int32_t p = o.nparent[v];
    while (p >= 0) {
        __threadfence();
        uint32_t arrived = atomicAdd(&o.narrive[p], 1u);
        if (arrived + 1 != o.nchild[p]) return;
        __threadfence();
        float4 lo = make_float4(INFINITY, INFINITY, INFINITY, 0.f);
        float3 hi = make_float3(-INFINITY, -INFINITY, -INFINITY);
        const uint32_t pend = (uint32_t)__float_as_int(__ldcg(&o.nhi[p].w));
        uint32_t c = (uint32_t)p + 1;
        while (c < pend) {
            float4 cl = __ldcg(&o.nlo[c]);
            float4 ch = __ldcg(&o.nhi[c]);
            lo.x = fminf(lo.x, cl.x); lo.y = fminf(lo.y, cl.y); lo.z = fminf(lo.z, cl.z);
            lo.w = fmaxf(lo.w, cl.w);
            hi.x = fmaxf(hi.x, ch.x); hi.y = fmaxf(hi.y, ch.y); hi.z = fmaxf(hi.z, ch.z);
            const uint32_t nx = (uint32_t)__float_as_int(ch.w);
            c = nx > c ? nx : c + 1;  // always advances
        }
        o.nlo[p] = lo;
        o.nhi[p] = make_float4(hi.x, hi.y, hi.z, __int_as_float((int)pend));
        p = o.nparent[p];
    }
}

cudaError_t octree_emit(const uint64_t *keys, uint32_t n, uint32_t node_cap, const SysTables &t,
                        const uint32_t *leaf_first, const uint8_t *leaf_lev,
                        const uint32_t *nodeoff, const float4 *pos, float support,
                        const OctreeOut &o, Status *st, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(o.nchild, 0, (size_t)node_cap * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(o.narrive, 0, (size_t)node_cap * 4, s);
    if (e != cudaSuccess) return e;
    // one thread per leaf (n bounds the leaf count), one per node slot
    k_emit_nodes<<<(n + 127) / 128, 128, 0, s>>>(keys, n, node_cap, t, leaf_first, leaf_lev,
                                                 nodeoff, o, st);
    k_node_boxes<<<(node_cap + 127) / 128, 128, 0, s>>>(node_cap, pos, support, o, st);
    return cudaGetLastError();
}

cudaError_t octree_boxes(uint32_t node_cap, const float4 *pos, float support, const OctreeOut &o,
                         const Status *st, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(o.narrive, 0, (size_t)node_cap * 4, s);
    if (e != cudaSuccess) return e;
    k_node_boxes<<<(node_cap + 127) / 128, 128, 0, s>>>(node_cap, pos, support, o, st);
    return cudaGetLastError();
}

}  // namespace nlg
