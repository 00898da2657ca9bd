// C ABI of the neighbor-list library: argument checks, device workspace,
// the build pipeline on one stream, passes, inspection copies.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstddef>
#include <cstdlib>
#include <chrono>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <random>

#include "mlp.cuh"
#include "nl_internal.cuh"

using namespace nlg;

namespace {

thread_local std::string g_err = "no error";

nl_status fail(nl_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

nl_status cuda_fail(cudaError_t e, const char *what, int line)
{
    (void)cudaGetLastError();  // clear a non-sticky error
    nl_status st = e == cudaErrorMemoryAllocation ? NL_ERR_OOM : NL_ERR_CUDA;
    return fail(st, "CUDA error %d (%s) in %s (capi.cu:%d)", (int)e, cudaGetErrorString(e), what,
                line);
}

#define CK(x)                                                   \
    do {                                                        \
        cudaError_t e_ = (x);                                   \
        if (e_ != cudaSuccess) return cuda_fail(e_, #x, __LINE__); \
    } while (0)

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
    cudaError_t ensure(size_t bytes)
    {
        if (p && bytes <= cap) return cudaSuccess;
        release();
        size_t b = ((bytes ? bytes : 16) + 255) / 256 * 256;
        cudaError_t e = cudaMalloc(&p, b);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            p = nullptr;
            return e;
        }
        cap = b;
        return cudaSuccess;
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
    template <class T>
    T *as() const
    {
        return reinterpret_cast<T *>(p);
    }
};

constexpr uint32_t kStageCap0 = 4096;
constexpr int kSearchBlocksPerSM = 4;
constexpr int kMaxRedoRounds = 8;

}  // namespace

namespace nlg {
// Sets the thread-local message returned by nl_last_error (other entry files).
nl_status report_error(nl_status st, const char *msg)
{
    g_err = msg;
    return st;
}

cudaError_t set_max_dynamic_smem(const void *func, size_t bytes)
{
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, size_t> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    size_t &have = done[std::make_pair(func, dev)];
    if (have >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) have = bytes;
    return e;
}
}  // namespace nlg

struct nl_list {
    int dev = -1, num_sms = 0;
    int64_t n = 0;
    uint32_t npad = 0, ncl = 0, nsc = 0, n_leaves = 0, n_nodes = 0;
    nl_params p{};
    nl_box box{};
    DevBox dbox{};
    int any_per = 0;
    unsigned long long list_bytes = 0, n_entries = 0, n_tiles = 0;
    unsigned long long node_visits = 0, leaf_visits = 0, j_examined = 0, tile_tests = 0;
    std::vector<nl_hiter_step> hiter_trace;  // one entry per count pass of the last h iteration
    uint32_t stage_cap = kStageCap0;
    int stage_grown = 0;
    int64_t n_prepared = 0;
    DevBuf keys, keys_alt, vals, vals_alt, hist, pos, clo, chi, jlo, jhi, lcp, lev, leaf_first,
        leaf_lev, nodeoff, bsum;
    DevBuf nlo, nhi, nrng, nlevel, nparent, nchild, narrive;
    DevBuf stageJ, stageM, list, rec_off, redo, work, aux, status;
    // half search: upper entries, transposed tuples (+ sort buffers), per super-cluster tables
    DevBuf uJ, uM, up_off, up_cnt, lower_cnt, seg_off, tkey, tkey_alt, tval, tval_alt, thist;
    // batches mixing periodic and open systems: their super-clusters, so that
    // the open ones run the kernels without periodic arithmetic
    DevBuf sc_open, sc_per;
    uint32_t n_open = 0, n_per = 0;
    // periodic super-clusters split by the last search: interior / boundary
    DevBuf sc_int, sc_bnd;
    DevBuf perm_pad, sys_off, sys_pad, sys_box, sys_root, sys_hcap;
    int32_t nsys = 1;
    // positions replaced since the search (nl_refresh_positions); pos_ref
    // keeps the positions the list was built on
    int moved = 0;
    DevBuf pos_ref;
    // half-list passes: per sorted particle fixed-point density sums, counts,
    // FP64 force sums
    DevBuf hsum, hcnt, hf;
    uint32_t node_cap = 0;
    const struct nl_mlp *mlp = nullptr;
    DevBuf ml_X, ml_e64, ml_pred, ml_slo, ml_shi;
    int graph_mode = 0;   // build without host reads or allocations (stream capture)
    size_t graph_up_cap = 0, graph_tu_cap = 0;  // half search capacities of a capture
    Status *hst = nullptr;

    SysTables tables() const
    {
        return SysTables{sys_off.as<uint32_t>(), sys_pad.as<uint32_t>(), sys_box.as<DevBox>(),
                         sys_root.as<uint32_t>(), (uint32_t)nsys};
    }
    OctreeOut octree_out() const
    {
        return OctreeOut{nlo.as<float4>(), nhi.as<float4>(), nrng.as<int2>(), nlevel.as<uint8_t>(),
                         nparent.as<int32_t>(), nchild.as<uint32_t>(), narrive.as<uint32_t>()};
    }
    // stage timing (CUDA events on the launching stream)
    static constexpr int kStages = 8;
    int profiling = 0;
    cudaEvent_t ev[kStages + 1] = {};
    float stage_ms[kStages] = {};
    int pass_timed = 0;   // the pass events (5..7) have been recorded
    // device copies of host inputs for nl_density_from_host; the masses are
    // uploaded on a side stream while the list is built
    DevBuf hx, hy, hz, hh, hm, hrho;
    cudaStream_t side = nullptr, side2 = nullptr;
    cudaEvent_t ev_in = nullptr, ev_m = nullptr, ev_zh = nullptr;
    // h iteration state (sorted order)
    DevBuf it_hq, it_hlo, it_hhi, it_hs, it_counts, it_conv, it_aflag, it_alist, it_words, it_tmp;

    cudaError_t mark(int k, cudaStream_t s)
    {
        if (!profiling) return cudaSuccess;
        for (int i = 0; i <= kStages; ++i)
            if (!ev[i]) {
                cudaError_t e = cudaEventCreate(&ev[i]);
                if (e != cudaSuccess) return e;
            }
        if (k == kStages) pass_timed = 1;
        return cudaEventRecord(ev[k], s);
    }
    void collect(int from, int to)
    {
        if (!profiling) return;
        cudaEventSynchronize(ev[to]);
        for (int k = from; k < to; ++k) cudaEventElapsedTime(&stage_ms[k], ev[k], ev[k + 1]);
    }

    void release_all()
    {
        DevBuf *all[] = {&keys, &keys_alt, &vals, &vals_alt, &hist, &pos, &clo, &chi, &jlo, &jhi,
                         &lcp, &lev,
                         &leaf_first, &leaf_lev, &nodeoff, &bsum, &nlo, &nhi, &nrng, &nlevel,
                         &nparent, &nchild, &narrive, &stageJ, &stageM, &list, &rec_off, &redo,
                         &work, &aux, &status, &hx, &hy, &hz, &hh, &hm, &hrho, &perm_pad,
                         &sys_off, &sys_pad, &sys_box, &sys_root, &sys_hcap, &it_hq,
                         &it_hlo, &it_hhi, &it_hs, &it_counts, &it_conv, &it_aflag, &it_alist,
                         &it_words, &it_tmp, &ml_X, &ml_e64, &ml_pred, &ml_slo, &ml_shi,
                         &uJ, &uM, &up_off, &up_cnt, &lower_cnt, &seg_off, &tkey, &tkey_alt,
                         &tval, &tval_alt, &thist, &sc_open, &sc_per, &sc_int, &sc_bnd,
                         &pos_ref, &hsum, &hcnt, &hf};
        for (DevBuf *b : all) b->release();
        for (int i = 0; i <= kStages; ++i)
            if (ev[i]) cudaEventDestroy(ev[i]);
        if (ev_in) cudaEventDestroy(ev_in);
        if (ev_m) cudaEventDestroy(ev_m);
        if (ev_zh) cudaEventDestroy(ev_zh);
        if (side) cudaStreamDestroy(side);
        if (side2) cudaStreamDestroy(side2);
        ev_in = ev_m = ev_zh = nullptr;
        side = side2 = nullptr;
        if (hst) cudaFreeHost(hst);
        hst = nullptr;
    }
};

namespace {

// j-cluster size MJ (0 in the parameters means MJ = M)
inline int jcl(const nl_params *p) { return p->j_cluster ? p->j_cluster : p->cluster; }

nl_status check_params(const nl_params *p, const nl_box *box)
{
    if (!p || !box) return fail(NL_ERR_ARG, "params or box is NULL");
    if (p->key != NL_KEY_MORTON && p->key != NL_KEY_HILBERT)
        return fail(NL_ERR_ARG, "unknown key kind %d", p->key);
    if (p->cluster != 4 && p->cluster != 8 && p->cluster != 16)
        return fail(NL_ERR_ARG, "cluster size must be 4, 8 or 16 (got %d)", p->cluster);
    if (p->j_cluster != 0 && p->j_cluster != p->cluster &&
        !(p->cluster >= 8 && p->j_cluster * 2 == p->cluster))
        return fail(NL_ERR_ARG, "j_cluster must be 0, cluster or cluster / 2 >= 4 (got %d for cluster %d)",
                    p->j_cluster, p->cluster);
    if (p->half_list != 0 && p->half_list != 1) return fail(NL_ERR_ARG, "half_list must be 0 or 1");
    if (p->half_list && p->j_cluster != 0 && p->j_cluster != p->cluster)
        return fail(NL_ERR_ARG, "a half list needs j-clusters of the i-cluster size");
    if (!(p->support > 0.f) || !std::isfinite(p->support))
        return fail(NL_ERR_ARG, "support must be finite and > 0");
    if (p->compress != 0 && p->compress != 1) return fail(NL_ERR_ARG, "compress must be 0 or 1");
    if (p->leaf_bucket < 8 || p->leaf_bucket > 1024)
        return fail(NL_ERR_ARG, "leaf_bucket must be in [8, 1024] (got %d)", p->leaf_bucket);
    if (p->threads_per_block != 0 && p->threads_per_block != 128 && p->threads_per_block != 256)
        return fail(NL_ERR_ARG, "threads_per_block must be 0, 128 or 256");
    if (p->blocks_per_sm < 0 || p->blocks_per_sm > 8)
        return fail(NL_ERR_ARG, "blocks_per_sm must be in [0, 8]");
    for (int a = 0; a < 3; ++a) {
        if (!std::isfinite(box->lo[a]) || !std::isfinite(box->hi[a]) || !(box->lo[a] < box->hi[a]))
            return fail(NL_ERR_ARG, "box axis %d: need finite lo < hi", a);
        float len = box->hi[a] - box->lo[a];
        if (!(len > 0.f) || !std::isfinite(len)) return fail(NL_ERR_ARG, "box axis %d degenerate", a);
    }
    return NL_OK;
}

DevBox make_devbox(const nl_box &b)
{
    DevBox d{};
    for (int a = 0; a < 3; ++a) {
        volatile float lo = b.lo[a], hi = b.hi[a];
        float len = hi - lo;
        d.lo[a] = lo;
        d.hi[a] = hi;
        d.len[a] = len;
        d.half[a] = 0.5f * len;
        volatile float num = 2097152.0f;
        d.qs[a] = num / len;
        d.per[a] = b.periodic[a] ? 1 : 0;
    }
    return d;
}

nl_status read_status(nl_list *nl, cudaStream_t s)
{
    CK(cudaMemcpyAsync(nl->hst, nl->status.p, sizeof(Status), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (nl->hst->sort_stall)
        return fail(NL_ERR_TIMEOUT, "a radix-sort look-back gave up its bounded wait; rebuild");
    return NL_OK;
}

// Keys, stable sort (by system, then key), padded permutation with cluster
// boxes, octree.  Systems: nsys >= 1; offs[0..nsys] caller offsets (host),
// boxes[0..nsys-1] (host).
nl_status do_prep(nl_list *nl, const float *x, const float *y, const float *z, const float *h,
                  int64_t n, int32_t nsys, const int64_t *offs, const nl_box *boxes,
                  const nl_params *p, cudaStream_t s)
{
    if (!x || !y || !z || !h) return fail(NL_ERR_ARG, "NULL particle array");
    if (n < 1) return fail(NL_ERR_ARG, "n must be >= 1 (got %lld)", (long long)n);
    if (n > (int64_t)1 << 30) return fail(NL_ERR_ARG, "n must be <= 2^30");
    if (nsys < 1 || nsys > (1 << 20)) return fail(NL_ERR_ARG, "need 1 <= nsys <= 2^20");
    if (!offs || !boxes) return fail(NL_ERR_ARG, "NULL system table");
    if (offs[0] != 0 || offs[nsys] != n)
        return fail(NL_ERR_ARG, "system offsets must start at 0 and end at n");
    for (int32_t k = 0; k < nsys; ++k) {
        if (offs[k + 1] <= offs[k]) return fail(NL_ERR_ARG, "system %d is empty", k);
        nl_status st = check_params(p, &boxes[k]);
        if (st != NL_OK) return st;
    }

    int dev;
    CK(cudaGetDevice(&dev));
    if (dev != nl->dev) {
        CK(cudaDeviceGetAttribute(&nl->num_sms, cudaDevAttrMultiProcessorCount, dev));
        nl->dev = dev;
    }
    if (!nl->hst) CK(cudaMallocHost(&nl->hst, sizeof(Status)));

    const uint32_t N = (uint32_t)n;
    const int M = p->cluster;
    const uint32_t scp = (uint32_t)(kSC * M);
    // host tables: offsets, padded offsets, boxes, periodic h caps
    std::vector<uint32_t> off(nsys + 1), pad(nsys + 1);
    std::vector<DevBox> dbox(nsys);
    std::vector<float> hcap(nsys);
    nl->any_per = 0;
    pad[0] = 0;
    for (int32_t k = 0; k <= nsys; ++k) off[k] = (uint32_t)offs[k];
    for (int32_t k = 0; k < nsys; ++k) {
        uint64_t nk = off[k + 1] - off[k];
        uint64_t padded = (nk + scp - 1) / scp * scp;
        if ((uint64_t)pad[k] + padded > 0xffffffffull) return fail(NL_ERR_ARG, "batch too large");
        pad[k + 1] = pad[k] + (uint32_t)padded;
        dbox[k] = make_devbox(boxes[k]);
        float cap = 3.0e38f;
        for (int a = 0; a < 3; ++a) {
            if (boxes[k].periodic[a]) {
                nl->any_per = 1;
                cap = std::min(cap, dbox[k].half[a] / p->support * 0.999999f);
            }
        }
        hcap[k] = cap;
    }
    const int MJ = jcl(p);
    const uint32_t npad = pad[nsys], ncl = npad / M, nsc = npad / scp;
    nl->p = *p;
    nl->box = boxes[0];
    nl->dbox = dbox[0];
    nl->nsys = nsys;

    if (!nl->graph_mode) {
    CK(nl->keys.ensure((size_t)N * 8));
    CK(nl->keys_alt.ensure((size_t)N * 8));
    CK(nl->vals.ensure((size_t)N * 4));
    CK(nl->vals_alt.ensure((size_t)N * 4));
    CK(nl->hist.ensure(radix_hist_words(N) * 4));
    CK(nl->pos.ensure((size_t)npad * 16));
    CK(nl->perm_pad.ensure((size_t)npad * 4));
    CK(nl->clo.ensure((size_t)ncl * 16));
    CK(nl->chi.ensure((size_t)ncl * 16));
    if (MJ != M) {
        CK(nl->jlo.ensure((size_t)(npad / MJ) * 16));
        CK(nl->jhi.ensure((size_t)(npad / MJ) * 16));
    }
    CK(nl->lcp.ensure((size_t)N));
    CK(nl->lev.ensure((size_t)N));
    CK(nl->leaf_first.ensure((size_t)(N + 1) * 4));
    CK(nl->leaf_lev.ensure((size_t)N));
    CK(nl->nodeoff.ensure((size_t)(N + 1) * 4));
    CK(nl->bsum.ensure(scan_bsum_words(N) * 4));
    CK(nl->rec_off.ensure((size_t)nsc * 4));
    CK(nl->redo.ensure((size_t)nsc * 4));
    CK(nl->work.ensure((size_t)nsc * 4));
    CK(nl->status.ensure(sizeof(Status)));
    CK(nl->sys_off.ensure((size_t)(nsys + 1) * 4));
    CK(nl->sys_pad.ensure((size_t)(nsys + 1) * 4));
    CK(nl->sys_box.ensure((size_t)nsys * sizeof(DevBox)));
    CK(nl->sys_root.ensure((size_t)nsys * 4));
    CK(nl->sys_hcap.ensure((size_t)nsys * 4));
    CK(cudaMemcpyAsync(nl->sys_off.p, off.data(), (size_t)(nsys + 1) * 4, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(nl->sys_pad.p, pad.data(), (size_t)(nsys + 1) * 4, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(nl->sys_box.p, dbox.data(), (size_t)nsys * sizeof(DevBox),
                       cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(nl->sys_hcap.p, hcap.data(), (size_t)nsys * 4, cudaMemcpyHostToDevice, s));
    // super-clusters of open and of periodic systems, when a batch has both
    std::vector<uint32_t> lo_sc, pe_sc;
    bool has_open = false;
    for (int32_t k = 0; k < nsys; ++k)
        if (!(boxes[k].periodic[0] || boxes[k].periodic[1] || boxes[k].periodic[2])) has_open = true;
    if (nl->any_per && has_open) {
        for (int32_t k = 0; k < nsys; ++k) {
            const bool per = boxes[k].periodic[0] || boxes[k].periodic[1] || boxes[k].periodic[2];
            for (uint32_t c = pad[k] / scp; c < pad[k + 1] / scp; ++c) (per ? pe_sc : lo_sc).push_back(c);
        }
        CK(nl->sc_open.ensure(lo_sc.size() * 4));
        CK(nl->sc_per.ensure(pe_sc.size() * 4));
        CK(cudaMemcpyAsync(nl->sc_open.p, lo_sc.data(), lo_sc.size() * 4, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(nl->sc_per.p, pe_sc.data(), pe_sc.size() * 4, cudaMemcpyHostToDevice, s));
    }
    nl->n_open = (uint32_t)lo_sc.size();
    nl->n_per = (uint32_t)pe_sc.size();
    if (nl->any_per) {
        CK(nl->sc_int.ensure((size_t)(npad / scp) * 4));
        CK(nl->sc_bnd.ensure((size_t)(npad / scp) * 4));
    }
    }
    const SysTables T = nl->tables();
    Status *dst = nl->status.as<Status>();
    CK(cudaMemsetAsync(dst, 0, sizeof(Status), s));

    // 1. keys (+ validation), 2. stable sort, 3. permute + cluster boxes
    CK(nl->mark(0, s));
    // the key kernel also counts the sort's digits (scratch cleared first)
    CK(radix_sort_clear(nl->hist.as<uint32_t>(), N, 3 * kKeyBits, s));
    CK(launch_keys_batch(n, x, y, z, h, T, p->support, p->key, nl->keys.as<uint64_t>(),
                         nl->vals.as<uint32_t>(), dst, nl->hist.as<uint32_t>(), s));
    CK(nl->mark(1, s));
    CK(radix_sort_pairs(nl->keys.as<uint64_t>(), nl->vals.as<uint32_t>(),
                        nl->keys_alt.as<uint64_t>(), nl->vals_alt.as<uint32_t>(), N,
                        3 * kKeyBits, nl->hist.as<uint32_t>(), &dst->sort_stall, s, true));
    CK(radix_sort_by_system(nl->keys.as<uint64_t>(), nl->vals.as<uint32_t>(),
                            nl->keys_alt.as<uint64_t>(), nl->vals_alt.as<uint32_t>(), N,
                            nl->sys_off.as<uint32_t>(), (uint32_t)nsys, nl->hist.as<uint32_t>(),
                            &dst->sort_stall, s));
    // test knob NLGB_SORT_STALL=1: report a look-back wait of the key sort that
    // gave up, without one, so that the error path runs on the host
    if (const char *e = std::getenv("NLGB_SORT_STALL"))
        if (e[0] == '1') CK(cudaMemsetAsync(&dst->sort_stall, 1, 1, s));
    CK(nl->mark(2, s));
    CK(launch_permute(npad, M, MJ, T, nl->vals.as<uint32_t>(), x, y, z, h, p->support,
                      nl->pos.as<float4>(), nl->perm_pad.as<uint32_t>(), nl->clo.as<float4>(),
                      nl->chi.as<float4>(), nl->jlo.as<float4>(), nl->jhi.as<float4>(), s));
    // 4. octree
    CK(nl->mark(3, s));
    CK(octree_leaves(nl->keys.as<uint64_t>(), N, p->leaf_bucket, T, nl->lcp.as<uint8_t>(),
                     nl->lev.as<uint8_t>(), nl->leaf_first.as<uint32_t>(),
                     nl->leaf_lev.as<uint8_t>(), nl->bsum.as<uint32_t>(), dst, s));
    CK(octree_count_nodes(nl->keys.as<uint64_t>(), N, T, nl->leaf_first.as<uint32_t>(),
                          nl->leaf_lev.as<uint8_t>(), nl->nodeoff.as<uint32_t>(),
                          nl->bsum.as<uint32_t>(), dst, s));
    uint32_t nleaves = 0, nnodes = 0;
    if (!nl->graph_mode) {
        nl_status st = read_status(nl, s);  // validation and sizes, one read
        if (st != NL_OK) return st;
        if (nl->hst->bad_input & 7u) {
            unsigned b = nl->hst->bad_input;
            return fail(NL_ERR_ARG, "invalid particle input:%s%s%s",
                        (b & 1) ? " non-finite coordinate" : "",
                        (b & 2) ? " coordinate outside the box" : "",
                        (b & 4) ? " h <= 0 or non-finite" : "");
        }
        if (nl->hst->bad_input & 8u)
            return fail(NL_ERR_RADIUS, "support*h >= L/2 on a periodic axis for some particle");
        nleaves = nl->hst->n_leaves;
        nnodes = nl->hst->n_nodes;
        const size_t cap = (size_t)nnodes + nnodes / 8 + 64;  // slack for graph replays
        if (nl->node_cap < nnodes) {
            CK(nl->nlo.ensure(cap * 16));
            CK(nl->nhi.ensure(cap * 16));
            CK(nl->nrng.ensure(cap * 8));
            CK(nl->nlevel.ensure(cap));
            CK(nl->nparent.ensure(cap * 4));
            CK(nl->nchild.ensure(cap * 4));
            CK(nl->narrive.ensure(cap * 4));
            nl->node_cap = (uint32_t)cap;
        }
    }
    CK(octree_emit(nl->keys.as<uint64_t>(), N, nl->node_cap, T, nl->leaf_first.as<uint32_t>(),
                   nl->leaf_lev.as<uint8_t>(), nl->nodeoff.as<uint32_t>(), nl->pos.as<float4>(),
                   p->support, nl->octree_out(), dst, s));
    nl->npad = npad;
    nl->ncl = ncl;
    nl->nsc = nsc;
    nl->n_leaves = nleaves;
    nl->n_nodes = nnodes;
    nl->n_prepared = n;
    return NL_OK;
}

// Warp slots the staging arrays hold at the current per-slot capacity.
uint32_t stage_slots(const nl_list *nl)
{
    const size_t c = (size_t)nl->stage_cap;
    const size_t slots = std::min(nl->stageJ.cap / (4 * c), nl->stageM.cap / c);
    return (uint32_t)std::min<size_t>(slots, 0xffffffffu);
}

// First search round over all super-clusters.  Open systems run without
// periodic arithmetic; so do the interior super-clusters of periodic systems
// (classified here, on the device, from this build's boxes and radii); only
// the boundary ones run the periodic kernels.  The classification stays valid
// for the passes over this list.
cudaError_t search_all(nl_list *nl, const SearchArgs &sa, int M, int grid, int tpb, cudaStream_t s)
{
    uint32_t *redo = nl->redo.as<uint32_t>();
    if (!nl->any_per)
        return launch_search_ctl(sa, nullptr, nl->nsc, redo, M, 0, grid, tpb, s);
    const bool mixed = nl->n_open && nl->n_per;
    const uint32_t *plist = mixed ? nl->sc_per.as<uint32_t>() : nullptr;
    const uint32_t np = mixed ? nl->n_per : nl->nsc;
    cudaError_t e = launch_classify(plist, np, M, sa.sys, sa.clo, sa.chi, sa.nlo, sa.nnodes,
                                    nl->sc_int.as<uint32_t>(), nl->sc_bnd.as<uint32_t>(), sa.st, s);
    if (e != cudaSuccess) return e;
    if (mixed) {
        e = launch_search_ctl(sa, nl->sc_open.as<uint32_t>(), nl->n_open, redo, M, 0, grid, tpb, s);
        if (e != cudaSuccess) return e;
        e = cudaMemsetAsync(&sa.st->ticket, 0, sizeof(sa.st->ticket), s);
        if (e != cudaSuccess) return e;
    }
    e = launch_search_ctl(sa, nl->sc_int.as<uint32_t>(), np, redo, M, 0, grid, tpb, s, &sa.st->n_int);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(&sa.st->ticket, 0, sizeof(sa.st->ticket), s);
    if (e != cudaSuccess) return e;
    return launch_search_ctl(sa, nl->sc_bnd.as<uint32_t>(), np, redo, M, 1, grid, tpb, s, &sa.st->n_bnd);
}

// A pass over all super-clusters (a.work == NULL) or over a.work; split by
// system kind and interior / boundary as the last search was.
cudaError_t run_pass(const nl_list *nl, const PassArgs &a, int kind, cudaStream_t s)
{
    const int M = nl->p.cluster;
    const int tpb = nl->p.threads_per_block, bps = nl->p.blocks_per_sm;
    if (a.work || !nl->any_per)
        return launch_pass(a, kind, M, nl->any_per, nl->num_sms, s, tpb, bps);
    const bool mixed = nl->n_open && nl->n_per;
    const uint32_t np = mixed ? nl->n_per : nl->nsc;
    cudaError_t e;
    if (mixed) {
        PassArgs o = a;
        o.work = nl->sc_open.as<uint32_t>();
        o.nwork = nl->n_open;
        e = launch_pass(o, kind, M, 0, nl->num_sms, s, tpb, bps);
        if (e != cudaSuccess) return e;
    }
    PassArgs q = a;
    q.work = nl->sc_int.as<uint32_t>();
    q.nwork = np;
    q.nwork_dev = &a.st->n_int;
    e = launch_pass(q, kind, M, 0, nl->num_sms, s, tpb, bps);
    if (e != cudaSuccess) return e;
    q.work = nl->sc_bnd.as<uint32_t>();
    q.nwork_dev = &a.st->n_bnd;
    return launch_pass(q, kind, M, 1, nl->num_sms, s, tpb, bps);
}

// Half search (j-clusters = i-clusters): every super-cluster searches only
// the j-clusters from its own first one on and sends the transposed tiles to
// the later super-clusters; the tuples are sorted by (target, j-cluster) and
// each record is assembled from its tuples and its own upper entries.  The
// records equal those of the full search byte for byte.  Buffer overflows of
// the upper entries or tuples re-run every super-cluster with buffers of the
// size the failed run asked for; staging overflows re-run only the
// super-clusters concerned, as in the full search.
nl_status do_search_half(nl_list *nl, cudaStream_t s)
{
    nl_status st;
    const nl_params *p = &nl->p;
    const uint32_t N = (uint32_t)nl->n_prepared, nsc = nl->nsc, ncl = nl->ncl;
    const int M = p->cluster;
    Status *dst = nl->status.as<Status>();
    const size_t search_words = sizeof(Status) - offsetof(Status, ticket);
    CK(cudaMemsetAsync(&dst->ticket, 0, search_words, s));
    size_t upc = 0, tuc = 0;
    const int tpb = p->threads_per_block ? p->threads_per_block : 256;
    const int wpb = tpb / 32;
    const int grid0 = nl->num_sms * (p->blocks_per_sm ? p->blocks_per_sm : kSearchBlocksPerSM);
    int grid = grid0;
    size_t slots = (size_t)grid * wpb;
    if (!nl->graph_mode) {
        CK(nl->up_off.ensure((size_t)nsc * 4));
        CK(nl->up_cnt.ensure((size_t)nsc * 4));
        CK(nl->lower_cnt.ensure((size_t)nsc * 4));
        CK(nl->seg_off.ensure((size_t)nsc * 4));
        upc = std::max(nl->uM.cap, (size_t)N * 2 + 4096);
        tuc = std::max(nl->tval.cap / 4, (size_t)N * 2 + 4096);
        if (const char *e = std::getenv("NLGB_HALF_CAP0")) upc = tuc = std::strtoull(e, nullptr, 10) + 1;
        CK(nl->uJ.ensure(upc * 4));
        CK(nl->uM.ensure(upc));
        CK(nl->tkey.ensure(tuc * 8));
        CK(nl->tval.ensure(tuc * 4));
        if (const char *e = std::getenv("NLGB_STAGE_CAP0"))
            if (!nl->stage_grown) nl->stage_cap = (uint32_t)std::strtoul(e, nullptr, 10);
        CK(nl->stageJ.ensure(slots * nl->stage_cap * 4));
        CK(nl->stageM.ensure(slots * nl->stage_cap));
    }
    CK(cudaMemsetAsync(nl->lower_cnt.p, 0, (size_t)nsc * 4, s));
    CK(nl->mark(4, s));

    SearchArgs sa{};
    sa.pos = nl->pos.as<float4>();
    sa.clo = nl->clo.as<float4>();
    sa.chi = nl->chi.as<float4>();
    sa.mj = M;
    sa.jlo = sa.clo;
    sa.jhi = sa.chi;
    sa.nlo = nl->nlo.as<float4>();
    sa.nhi = nl->nhi.as<float4>();
    sa.nrng = nl->nrng.as<int2>();
    sa.n = N;
    sa.nsc = nsc;
    sa.nnodes = nl->node_cap;
    sa.sys = nl->tables();
    sa.support = p->support;
    sa.compress = p->compress;
    sa.st = dst;
    sa.rec_off = nl->rec_off.as<uint32_t>();
    sa.half = 1;
    sa.ncl = ncl;
    sa.up_off = nl->up_off.as<uint32_t>();
    sa.up_cnt = nl->up_cnt.as<uint32_t>();
    sa.lower_cnt = nl->lower_cnt.as<uint32_t>();
    sa.seg_off = nl->seg_off.as<uint32_t>();

    int bits = 1;
    while (bits < 64 && ((unsigned long long)nsc * ncl >> bits) != 0) ++bits;
    if (nl->graph_mode) {
        // one pass with the capacities reserved before the capture; the sort
        // covers the whole tuple capacity (unused slots hold the largest key)
        // and overflows are reported by nl_graph_check
        const size_t gcap = nl->graph_tu_cap;
        sa.stageJ = nl->stageJ.as<uint32_t>();
        sa.stageM = nl->stageM.as<uint8_t>();
        sa.stage_cap = nl->stage_cap;
        sa.stage_slots = stage_slots(nl);
        sa.uJ = nl->uJ.as<uint32_t>();
        sa.uM = nl->uM.as<uint8_t>();
        sa.up_cap = nl->graph_up_cap;
        sa.tkey = nl->tkey.as<uint64_t>();
        sa.tval = nl->tval.as<uint32_t>();
        sa.tu_cap = gcap;
        sa.list = nl->list.as<uint8_t>();
        sa.list_cap = nl->list.cap - 8;
        CK(search_all(nl, sa, M, grid0, tpb, s));
        CK(launch_fill_keys(nl->tkey.as<uint64_t>(), (uint32_t)gcap, &dst->tu_used,
                            bits >= 64 ? ~0ull : (1ull << bits) - 1ull, s));
        CK(radix_sort_pairs(nl->tkey.as<uint64_t>(), nl->tval.as<uint32_t>(),
                            nl->tkey_alt.as<uint64_t>(), nl->tval_alt.as<uint32_t>(),
                            (uint32_t)gcap, bits, nl->thist.as<uint32_t>(), &dst->sort_stall, s));
        CK(exclusive_scan_u32(nl->lower_cnt.as<uint32_t>(), nl->seg_off.as<uint32_t>(), nsc,
                              nl->bsum.as<uint32_t>(), &dst->seg_total, s));
        CK(launch_assemble(sa, grid0, s));
        return NL_OK;
    }

    unsigned long long nv = 0, lv = 0, jx = 0, tt = 0;
    const uint32_t *work = nullptr;
    uint32_t count = nsc;
    for (int round = 0;; ++round) {
        if (round >= kMaxRedoRounds)
            return fail(NL_ERR_CAPACITY, "half search still overflowing after %d rounds", round);
        sa.stageJ = nl->stageJ.as<uint32_t>();
        sa.stageM = nl->stageM.as<uint8_t>();
        sa.stage_cap = nl->stage_cap;
        sa.stage_slots = stage_slots(nl);
        sa.uJ = nl->uJ.as<uint32_t>();
        sa.uM = nl->uM.as<uint8_t>();
        sa.up_cap = upc;
        sa.tkey = nl->tkey.as<uint64_t>();
        sa.tval = nl->tval.as<uint32_t>();
        sa.tu_cap = tuc;
        if (work)
            CK(launch_search_ctl(sa, work, count, nl->redo.as<uint32_t>(), M, nl->any_per, grid, tpb, s));
        else
            CK(search_all(nl, sa, M, grid, tpb, s));
        st = read_status(nl, s);
        if (st != NL_OK) return st;
        nv += nl->hst->node_visits;
        lv += nl->hst->leaf_visits;
        jx += nl->hst->j_examined;
        tt += nl->hst->tile_tests;
        if (nl->hst->max_count > nl->stage_cap) {
            nl->stage_cap = nl->hst->max_count + nl->hst->max_count / 4 + 64;
            nl->stage_grown = 1;
        }
        if (nl->hst->half_overflow) {
            // start over with the sizes the failed run asked for
            upc = std::max(upc, (size_t)(nl->hst->up_used + nl->hst->up_used / 4 + 4096));
            tuc = std::max(tuc, (size_t)(nl->hst->tu_used + nl->hst->tu_used / 4 + 4096));
            CK(nl->uJ.ensure(upc * 4));
            CK(nl->uM.ensure(upc));
            CK(nl->tkey.ensure(tuc * 8));
            CK(nl->tval.ensure(tuc * 4));
            grid = grid0;
            slots = (size_t)grid * wpb;
            CK(nl->stageJ.ensure(slots * nl->stage_cap * 4));
            CK(nl->stageM.ensure(slots * nl->stage_cap));
            CK(cudaMemsetAsync(&dst->ticket, 0, search_words, s));
            CK(cudaMemsetAsync(nl->lower_cnt.p, 0, (size_t)nsc * 4, s));
            work = nullptr;
            count = nsc;
            nv = lv = jx = tt = 0;
            continue;
        }
        const uint32_t nredo = nl->hst->stage_overflow;
        if (nredo == 0) break;
        // staging overflow only: re-run the listed super-clusters after growth
        CK(cudaMemcpyAsync(nl->work.p, nl->redo.p, (size_t)nredo * 4, cudaMemcpyDeviceToDevice, s));
        work = nl->work.as<uint32_t>();
        count = nredo;
        grid = (int)std::min<uint32_t>((uint32_t)grid, (nredo + wpb - 1) / wpb);
        slots = (size_t)grid * wpb;
        CK(nl->stageJ.ensure(slots * nl->stage_cap * 4));
        CK(nl->stageM.ensure(slots * nl->stage_cap));
        const unsigned long long keep_up = nl->hst->up_used, keep_tu = nl->hst->tu_used;
        const unsigned int keep_int = nl->hst->n_int, keep_bnd = nl->hst->n_bnd;
        std::memset(&nl->hst->ticket, 0, search_words);
        nl->hst->up_used = keep_up;
        nl->hst->tu_used = keep_tu;
        nl->hst->n_int = keep_int;  // the passes use the first round's split
        nl->hst->n_bnd = keep_bnd;
        CK(cudaMemcpyAsync(&dst->ticket, &nl->hst->ticket, search_words, cudaMemcpyHostToDevice, s));
    }
    const uint32_t ntu = (uint32_t)nl->hst->tu_used;
    CK(nl->mark(5, s));
    // sort the tuples by (target super-cluster, j-cluster)
    if (ntu > 1) {
        CK(nl->tkey_alt.ensure((size_t)ntu * 8));
        CK(nl->tval_alt.ensure((size_t)ntu * 4));
        CK(nl->thist.ensure(radix_hist_words(ntu) * 4));
        CK(radix_sort_pairs(nl->tkey.as<uint64_t>(), nl->tval.as<uint32_t>(),
                            nl->tkey_alt.as<uint64_t>(), nl->tval_alt.as<uint32_t>(), ntu, bits,
                            nl->thist.as<uint32_t>(), &dst->sort_stall, s));
    }
    CK(nl->bsum.ensure(scan_bsum_words(nsc) * 4));
    CK(exclusive_scan_u32(nl->lower_cnt.as<uint32_t>(), nl->seg_off.as<uint32_t>(), nsc,
                          nl->bsum.as<uint32_t>(), &dst->seg_total, s));
    // assemble and encode the records
    size_t est = (size_t)N * (p->compress ? 12 : 48) + 65536;
    if (const char *e = std::getenv("NLGB_LIST_CAP0")) est = std::strtoull(e, nullptr, 10) + 8;
    if (nl->list.cap < est) CK(nl->list.ensure(est));
    for (int round = 0;; ++round) {
        if (round >= kMaxRedoRounds)
            return fail(NL_ERR_CAPACITY, "list still overflowing after %d rounds", round);
        CK(cudaMemsetAsync(&dst->list_used, 0, sizeof(dst->list_used), s));
        CK(cudaMemsetAsync(&dst->n_entries, 0, sizeof(dst->n_entries), s));
        CK(cudaMemsetAsync(&dst->n_tiles, 0, sizeof(dst->n_tiles), s));
        CK(cudaMemsetAsync(&dst->list_overflow, 0, sizeof(dst->list_overflow), s));
        CK(cudaMemsetAsync(&dst->asm_ticket, 0, sizeof(dst->asm_ticket), s));
        sa.list = nl->list.as<uint8_t>();
        sa.list_cap = nl->list.cap - 8;  // 8 bytes of slack behind the last record
        CK(launch_assemble(sa, grid0, s));
        st = read_status(nl, s);
        if (st != NL_OK) return st;
        if (!nl->hst->list_overflow) break;
        const size_t need = (size_t)nl->hst->list_used + nl->hst->list_used / 8 + 65536;
        nl->list.release();
        CK(nl->list.ensure(need));
    }
    CK(nl->mark(6, s));
    nl->collect(0, 6);
    nl->n = nl->n_prepared;
    nl->list_bytes = nl->hst->list_used;
    nl->n_entries = nl->hst->n_entries;
    nl->n_tiles = nl->hst->n_tiles;
    nl->node_visits = nv;
    nl->leaf_visits = lv;
    nl->j_examined = jx;
    nl->tile_tests = tt;
    return NL_OK;
}

// Cluster-pair search + encoding over the prepared structures, with redo
// rounds for overflows.  Sets nl->n on success.
nl_status do_search(nl_list *nl, cudaStream_t s)
{
    nl->moved = 0;  // the list is built on the positions it holds
    {
        // the half search needs j-clusters = i-clusters; NLGB_SEARCH=full
        // forces the full search (tests run both)
        const char *e = std::getenv("NLGB_SEARCH");
        const bool full = e && std::strcmp(e, "full") == 0;
        if (!nl->p.half_list && !full && jcl(&nl->p) == nl->p.cluster) return do_search_half(nl, s);
    }
    nl_status st;
    const nl_params *p = &nl->p;
    const uint32_t N = (uint32_t)nl->n_prepared, nsc = nl->nsc;
    const int M = p->cluster;
    Status *dst = nl->status.as<Status>();
    const size_t search_words = sizeof(Status) - offsetof(Status, ticket);
    CK(cudaMemsetAsync(&dst->ticket, 0, search_words, s));
    size_t est = (size_t)N * (p->compress ? 12 : 48) + 65536;
    // test knobs: start from tiny buffers to exercise the overflow rounds
    if (const char *e = std::getenv("NLGB_LIST_CAP0")) est = std::strtoull(e, nullptr, 10) + 8;
    if (const char *e = std::getenv("NLGB_STAGE_CAP0"))
        if (!nl->stage_grown) nl->stage_cap = (uint32_t)std::strtoul(e, nullptr, 10);
    const int tpb = p->threads_per_block ? p->threads_per_block : 256;
    const int wpb = tpb / 32;
    int grid = nl->num_sms * (p->blocks_per_sm ? p->blocks_per_sm : kSearchBlocksPerSM);
    size_t slots = (size_t)grid * wpb;
    if (!nl->graph_mode) {
        if (nl->list.cap < est) CK(nl->list.ensure(est));
        CK(nl->stageJ.ensure(slots * nl->stage_cap * 4));
        CK(nl->stageM.ensure(slots * nl->stage_cap));
    }
    CK(cudaMemsetAsync(&dst->fail_off, 0xff, sizeof(dst->fail_off), s));
    CK(nl->mark(4, s));

    SearchArgs sa{};
    sa.pos = nl->pos.as<float4>();
    sa.clo = nl->clo.as<float4>();
    sa.chi = nl->chi.as<float4>();
    sa.mj = jcl(p);
    sa.jlo = sa.mj == M ? sa.clo : nl->jlo.as<float4>();
    sa.jhi = sa.mj == M ? sa.chi : nl->jhi.as<float4>();
    sa.nlo = nl->nlo.as<float4>();
    sa.nhi = nl->nhi.as<float4>();
    sa.nrng = nl->nrng.as<int2>();
    sa.n = N;
    sa.nsc = nsc;
    sa.nnodes = nl->node_cap;  // node array capacity (bounds every node index)
    sa.sys = nl->tables();
    sa.support = p->support;
    sa.compress = p->compress;
    sa.st = dst;
    sa.rec_off = nl->rec_off.as<uint32_t>();
    sa.half = p->half_list ? 2 : 0;  // the half list: the half search's own entries as records

    unsigned long long entries = 0, tiles = 0, used = 0, nv = 0, lv = 0, jx = 0, tt = 0;
    const uint32_t *work = nullptr;
    uint32_t count = nsc;
    for (int round = 0;; ++round) {
        sa.stageJ = nl->stageJ.as<uint32_t>();
        sa.stageM = nl->stageM.as<uint8_t>();
        sa.stage_cap = nl->stage_cap;
        sa.stage_slots = stage_slots(nl);
        sa.list = nl->list.as<uint8_t>();
        sa.list_cap = nl->list.cap - 8;  // 8 bytes of slack behind the last record
        if (work)
            CK(launch_search_ctl(sa, work, count, nl->redo.as<uint32_t>(), M, nl->any_per, grid, tpb, s));
        else
            CK(search_all(nl, sa, M, grid, tpb, s));
        if (nl->graph_mode) return NL_OK;  // overflow is reported by nl_graph_check
        st = read_status(nl, s);
        if (st != NL_OK) return st;
        entries += nl->hst->n_entries;
        tiles += nl->hst->n_tiles;
        nv += nl->hst->node_visits;
        lv += nl->hst->leaf_visits;
        jx += nl->hst->j_examined;
        tt += nl->hst->tile_tests;
        used = nl->hst->list_used;
        const uint32_t nredo = nl->hst->stage_overflow;
        if (nredo == 0) break;
        if (round + 1 >= kMaxRedoRounds)
            return fail(NL_ERR_CAPACITY, "list still overflowing after %d rounds", round + 1);
        // grow what overflowed, then re-run only the listed super-clusters
        CK(cudaMemcpyAsync(nl->work.p, nl->redo.p, (size_t)nredo * 4, cudaMemcpyDeviceToDevice, s));
        work = nl->work.as<uint32_t>();
        count = nredo;
        grid = (int)std::min<uint32_t>((uint32_t)grid, (nredo + wpb - 1) / wpb);
        slots = (size_t)grid * wpb;
        if (nl->hst->max_count > nl->stage_cap) {
            nl->stage_cap = nl->hst->max_count + nl->hst->max_count / 4 + 64;
            nl->stage_grown = 1;
        }
        CK(nl->stageJ.ensure(slots * nl->stage_cap * 4));
        CK(nl->stageM.ensure(slots * nl->stage_cap));
        unsigned long long keep = used;
        if (nl->hst->list_overflow) {
            keep = nl->hst->fail_off;
            size_t ncap = std::max((size_t)nl->list.cap * 2, (size_t)(used + used / 2 + 4096));
            DevBuf bigger;
            CK(bigger.ensure(ncap));
            CK(cudaMemcpyAsync(bigger.p, nl->list.p, keep, cudaMemcpyDeviceToDevice, s));
            CK(cudaStreamSynchronize(s));
            nl->list.release();
            nl->list = bigger;
            bigger.p = nullptr;
        }
        const unsigned int keep_int = nl->hst->n_int, keep_bnd = nl->hst->n_bnd;
        std::memset(&nl->hst->ticket, 0, search_words);
        nl->hst->list_used = keep;
        nl->hst->fail_off = ~0ull;
        nl->hst->n_int = keep_int;  // the passes use the first round's split
        nl->hst->n_bnd = keep_bnd;
        CK(cudaMemcpyAsync(&dst->ticket, &nl->hst->ticket, search_words, cudaMemcpyHostToDevice, s));
    }
    CK(nl->mark(5, s));
    CK(nl->mark(6, s));  // the full search has no assembly stage
    nl->collect(0, 6);
    nl->n = nl->n_prepared;
    nl->list_bytes = used;
    nl->n_entries = entries;
    nl->n_tiles = tiles;
    nl->node_visits = nv;
    nl->leaf_visits = lv;
    nl->j_examined = jx;
    nl->tile_tests = tt;
    return NL_OK;
}

nl_status do_build(nl_list *nl, const float *x, const float *y, const float *z, const float *h,
                   int64_t n, int32_t nsys, const int64_t *offs, const nl_box *boxes,
                   const nl_params *p, cudaStream_t s)
{
    nl_status st = do_prep(nl, x, y, z, h, n, nsys, offs, boxes, p, s);
    if (st != NL_OK) return st;
    return do_search(nl, s);
}

nl_status check_list(const nl_list *nl)
{
    if (!nl) return fail(NL_ERR_ARG, "list is NULL");
    if (nl->n <= 0) return fail(NL_ERR_ARG, "list is empty (not built or last build failed)");
    return NL_OK;
}

PassArgs pass_args(const nl_list *nl)
{
    PassArgs a{};
    a.pos = nl->pos.as<float4>();
    a.list = nl->list.as<uint8_t>();
    a.rec_off = nl->rec_off.as<uint32_t>();
    a.perm = nl->perm_pad.as<uint32_t>();
    a.aux = nl->aux.as<float2>();
    a.n = (uint32_t)nl->n;
    a.nsc = nl->nsc;
    a.sys = nl->tables();
    a.support = nl->p.support;
    a.compress = nl->p.compress;
    a.mj = jcl(&nl->p);
    a.st = nl->status.as<Status>();
    a.half = nl->p.half_list;
    a.hsum = nl->hsum.as<unsigned long long>();
    a.hcnt = nl->hcnt.as<uint32_t>();
    a.hf = nl->hf.as<double>();
    return a;
}

}  // namespace

extern "C" {

void nl_default_params(nl_params *p)
{
    if (!p) return;
    p->key = NL_KEY_HILBERT;
    p->cluster = 8;
    p->support = 2.0f;
    p->compress = 1;
    p->leaf_bucket = 256;
    p->threads_per_block = 0;
    p->blocks_per_sm = 0;
    p->j_cluster = 0;
    p->half_list = 0;
}

const char *nl_last_error(void) { return g_err.c_str(); }

nl_status nl_rebuild(nl_list *nl, const float *x, const float *y, const float *z, const float *h,
                     int64_t n, const nl_box *box, const nl_params *p, void *stream)
{
    if (!nl) return fail(NL_ERR_ARG, "list is NULL");
    if (!box) return fail(NL_ERR_ARG, "box is NULL");
    nl->n = 0;
    const int64_t offs[2] = {0, n};
    nl_status st = do_build(nl, x, y, z, h, n, 1, offs, box, p, (cudaStream_t)stream);
    if (st != NL_OK) nl->n = 0;
    return st;
}

nl_status nl_rebuild_batch(nl_list *nl, const float *x, const float *y, const float *z,
                           const float *h, int32_t nsys, const int64_t *offsets,
                           const nl_box *boxes, const nl_params *p, void *stream)
{
    if (!nl) return fail(NL_ERR_ARG, "list is NULL");
    if (!offsets || nsys < 1) return fail(NL_ERR_ARG, "need nsys >= 1 and offsets");
    nl->n = 0;
    nl_status st = do_build(nl, x, y, z, h, offsets[nsys], nsys, offsets, boxes, p,
                            (cudaStream_t)stream);
    if (st != NL_OK) nl->n = 0;
    return st;
}

nl_status nl_build_batch(const float *x, const float *y, const float *z, const float *h,
                         int32_t nsys, const int64_t *offsets, const nl_box *boxes,
                         const nl_params *p, void *stream, nl_list **out)
{
    if (!out) return fail(NL_ERR_ARG, "out is NULL");
    *out = nullptr;
    nl_list *nl = new (std::nothrow) nl_list();
    if (!nl) return fail(NL_ERR_OOM, "host allocation failed");
    nl_status st = nl_rebuild_batch(nl, x, y, z, h, nsys, offsets, boxes, p, stream);
    if (st != NL_OK) {
        nl->release_all();
        delete nl;
        return st;
    }
    *out = nl;
    return NL_OK;
}

nl_status nl_build(const float *x, const float *y, const float *z, const float *h, int64_t n,
                   const nl_box *box, const nl_params *p, void *stream, nl_list **out)
{
    if (!out) return fail(NL_ERR_ARG, "out is NULL");
    *out = nullptr;
    nl_list *nl = new (std::nothrow) nl_list();
    if (!nl) return fail(NL_ERR_OOM, "host allocation failed");
    nl_status st = nl_rebuild(nl, x, y, z, h, n, box, p, stream);
    if (st != NL_OK) {
        nl->release_all();
        delete nl;
        return st;
    }
    *out = nl;
    return NL_OK;
}

nl_status nl_create(nl_list **out)
{
    if (!out) return fail(NL_ERR_ARG, "out is NULL");
    *out = new (std::nothrow) nl_list();
    if (!*out) return fail(NL_ERR_OOM, "host allocation failed");
    return NL_OK;
}

nl_status nl_set_profiling(nl_list *nl, int32_t on)
{
    if (!nl) return fail(NL_ERR_ARG, "list is NULL");
    nl->profiling = on ? 1 : 0;
    return NL_OK;
}

nl_status nl_get_stage_times(const nl_list *cnl, float *ms, int32_t cap, int32_t *count)
{
    if (!cnl) return fail(NL_ERR_ARG, "list is NULL");
    nl_list *nl = const_cast<nl_list *>(cnl);
    if (nl->profiling && nl->pass_timed) {
        CK(cudaEventSynchronize(nl->ev[nl_list::kStages]));
        CK(cudaEventElapsedTime(&nl->stage_ms[6], nl->ev[6], nl->ev[7]));
        CK(cudaEventElapsedTime(&nl->stage_ms[7], nl->ev[7], nl->ev[8]));
    }
    for (int k = 0; k < nl_list::kStages && k < cap; ++k) ms[k] = nl->stage_ms[k];
    if (count) *count = nl_list::kStages;
    return NL_OK;
}

nl_status nl_density_from_host(nl_list *nl, const float *x, const float *y, const float *z,
                               const float *h, const float *m, int64_t n, const nl_box *box,
                               const nl_params *p, float *rho, void *stream)
{
    if (!nl) return fail(NL_ERR_ARG, "list is NULL");
    if (!x || !y || !z || !h || !m || !rho) return fail(NL_ERR_ARG, "NULL host array");
    if (n < 1 || n > (int64_t)1 << 30) return fail(NL_ERR_ARG, "bad n %lld", (long long)n);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t b = (size_t)n * 4;
    DevBuf *bufs[] = {&nl->hx, &nl->hy, &nl->hz, &nl->hh, &nl->hm, &nl->hrho};
    for (DevBuf *d : bufs) CK(d->ensure(b));
    if (!nl->side) {
        CK(cudaStreamCreateWithFlags(&nl->side, cudaStreamNonBlocking));
        CK(cudaStreamCreateWithFlags(&nl->side2, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&nl->ev_in, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&nl->ev_m, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&nl->ev_zh, cudaEventDisableTiming));
    }
    // the side streams start after earlier work on `stream` (which may still
    // read the previous inputs): one uploads m while the list is built, the
    // other z and h beside x and y on `stream`, so that the copies overlap
    CK(cudaEventRecord(nl->ev_in, s));
    CK(cudaStreamWaitEvent(nl->side, nl->ev_in, 0));
    CK(cudaStreamWaitEvent(nl->side2, nl->ev_in, 0));
    CK(cudaMemcpyAsync(nl->hz.p, z, b, cudaMemcpyHostToDevice, nl->side2));
    CK(cudaMemcpyAsync(nl->hh.p, h, b, cudaMemcpyHostToDevice, nl->side2));
    CK(cudaEventRecord(nl->ev_zh, nl->side2));
    CK(cudaMemcpyAsync(nl->hm.p, m, b, cudaMemcpyHostToDevice, nl->side));
    CK(cudaEventRecord(nl->ev_m, nl->side));
    CK(cudaMemcpyAsync(nl->hx.p, x, b, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(nl->hy.p, y, b, cudaMemcpyHostToDevice, s));
    CK(cudaStreamWaitEvent(s, nl->ev_zh, 0));
    nl_status st = nl_rebuild(nl, nl->hx.as<float>(), nl->hy.as<float>(), nl->hz.as<float>(),
                              nl->hh.as<float>(), n, box, p, stream);
    CK(cudaStreamWaitEvent(s, nl->ev_m, 0));  // also on failure: m stays owned by us
    if (st != NL_OK) return st;
    st = nl_density_pass(nl, nl->hm.as<float>(), nl->hrho.as<float>(), stream);
    if (st != NL_OK) return st;
    CK(cudaMemcpyAsync(rho, nl->hrho.p, b, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return NL_OK;
}

}  // extern "C"

struct nl_mlp {
    DevBuf P, m, v, grad, partial, loss, idx;
    int64_t step = 0;
    int slots = 0;
};

namespace {
nl_status mlp_slots(nl_mlp *mlp, int slots)
{
    if (mlp->slots >= slots) return NL_OK;
    CK(mlp->partial.ensure((size_t)slots * kMlpParams * 4));
    CK(mlp->loss.ensure((size_t)slots * 4));
    mlp->slots = slots;
    return NL_OK;
}

nl_status features_of(const nl_list *cnl, cudaStream_t s)
{
    nl_list *nl = const_cast<nl_list *>(cnl);
    CK(nl->ml_X.ensure((size_t)nl->ncl * kMlpF * 4));
    CK(nl->ml_e64.ensure((size_t)nl->nsc * 4));
    CK(nl->ml_slo.ensure((size_t)nl->nsc * 16));
    CK(nl->ml_shi.ensure((size_t)nl->nsc * 16));
    CK(mlp_features(nl->nsc, nl->p.cluster, nl->tables(), nl->clo.as<float4>(), nl->chi.as<float4>(),
                    nl->perm_pad.as<uint32_t>(), nl->ml_slo.as<float4>(), nl->ml_shi.as<float4>(),
                    nl->ml_X.as<float>(), nl->ml_e64.as<float>(), s));
    return NL_OK;
}

nl_status learned_start(nl_list *nl, float *hq, cudaStream_t s)
{
    nl_status st = features_of(nl, s);
    if (st != NL_OK) return st;
    CK(nl->ml_pred.ensure((size_t)nl->ncl * 4));
    CK(mlp_predict(nl->ncl, nl->ml_X.as<float>(), nl->mlp->P.as<float>(), nl->ml_pred.as<float>(),
                   nl->num_sms, s));
    CK(mlp_apply_h0(nl->npad, nl->p.cluster, nl->perm_pad.as<uint32_t>(), nl->ml_pred.as<float>(),
                    nl->ml_e64.as<float>(), hq, s));
    return NL_OK;
}
}  // namespace

extern "C" {

int64_t nl_mlp_nparams(void) { return kMlpParams; }

nl_status nl_mlp_create(uint64_t seed, nl_mlp **out)
{
    if (!out) return fail(NL_ERR_ARG, "out is NULL");
    *out = nullptr;
    nl_mlp *mlp = new (std::nothrow) nl_mlp();
    if (!mlp) return fail(NL_ERR_OOM, "host allocation failed");
    std::vector<float> P(kMlpParams, 0.f);
    std::mt19937_64 rng(seed);
    std::normal_distribution<float> nd(0.f, 1.f);
    size_t o = 0;
    const int fan[4] = {kMlpF, kMlpH, kMlpH, kMlpH}, outs[4] = {kMlpH, kMlpH, kMlpH, 1};
    for (int l = 0; l < 4; ++l) {
        const float sd = 1.f / std::sqrt((float)fan[l]);
        for (int k = 0; k < outs[l] * fan[l]; ++k) P[o++] = sd * nd(rng);
        o += outs[l];  // biases stay zero
    }
    cudaError_t e = mlp->P.ensure(kMlpParams * 4);
    if (e == cudaSuccess) e = mlp->m.ensure(kMlpParams * 4);
    if (e == cudaSuccess) e = mlp->v.ensure(kMlpParams * 4);
    if (e == cudaSuccess) e = mlp->grad.ensure(kMlpParams * 4);
    if (e == cudaSuccess) e = cudaMemcpy(mlp->P.p, P.data(), kMlpParams * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(mlp->m.p, 0, kMlpParams * 4);
    if (e == cudaSuccess) e = cudaMemset(mlp->v.p, 0, kMlpParams * 4);
    if (e != cudaSuccess) {
        delete mlp;
        return cuda_fail(e, "nl_mlp_create", __LINE__);
    }
    *out = mlp;
    return NL_OK;
}

nl_status nl_mlp_free(nl_mlp *mlp)
{
    if (!mlp) return NL_OK;
    cudaDeviceSynchronize();
    DevBuf *all[] = {&mlp->P, &mlp->m, &mlp->v, &mlp->grad, &mlp->partial, &mlp->loss, &mlp->idx};
    for (DevBuf *b : all) b->release();
    delete mlp;
    return NL_OK;
}

nl_status nl_mlp_get_params(const nl_mlp *mlp, float *params)
{
    if (!mlp || !params) return fail(NL_ERR_ARG, "NULL argument");
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(params, mlp->P.p, kMlpParams * 4, cudaMemcpyDeviceToHost));
    return NL_OK;
}

nl_status nl_mlp_set_params(nl_mlp *mlp, const float *params)
{
    if (!mlp || !params) return fail(NL_ERR_ARG, "NULL argument");
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(mlp->P.p, params, kMlpParams * 4, cudaMemcpyHostToDevice));
    CK(cudaMemset(mlp->m.p, 0, kMlpParams * 4));
    CK(cudaMemset(mlp->v.p, 0, kMlpParams * 4));
    mlp->step = 0;
    return NL_OK;
}

nl_status nl_mlp_features(const nl_list *nl, float *X, float *e64, void *stream)
{
    nl_status st = check_list(nl);
    if (st != NL_OK) return st;
    if (!X || !e64) return fail(NL_ERR_ARG, "NULL output");
    cudaStream_t s = (cudaStream_t)stream;
    st = features_of(nl, s);
    if (st != NL_OK) return st;
    CK(cudaMemcpyAsync(X, nl->ml_X.p, (size_t)nl->ncl * kMlpF * 4, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(e64, nl->ml_e64.p, (size_t)nl->nsc * 4, cudaMemcpyDeviceToDevice, s));
    return NL_OK;
}

nl_status nl_mlp_targets(const nl_list *nl, const float *h, const float *e64, float *y, float *w,
                         void *stream)
{
    nl_status st = check_list(nl);
    if (st != NL_OK) return st;
    if (!h || !e64 || !y || !w) return fail(NL_ERR_ARG, "NULL argument");
    CK(mlp_targets(nl->ncl, nl->p.cluster, nl->perm_pad.as<uint32_t>(), h, e64, y, w,
                   (cudaStream_t)stream));
    return NL_OK;
}

static nl_status mlp_run(nl_mlp *mlp, const float *X, const float *y, const float *w, int64_t n,
                         const int64_t *idx_dev, int64_t nb, float *grad, int adam, float lr,
                         float inv_n, float *loss_host, cudaStream_t s)
{
    const int slots = (int)std::min<int64_t>((nb + 63) / 64, 4096);
    nl_status st = mlp_slots(mlp, slots);
    if (st != NL_OK) return st;
    if (adam) ++mlp->step;
    CK(mlp_train_step(nb, idx_dev, X, y, w, mlp->P.as<float>(), mlp->m.as<float>(),
                      mlp->v.as<float>(), mlp->partial.as<float>(), slots, grad,
                      mlp->loss.as<float>(), adam, lr, (int)std::max<int64_t>(mlp->step, 1), inv_n, s));
    if (loss_host) {
        std::vector<float> l(slots);
        CK(cudaMemcpyAsync(l.data(), mlp->loss.p, (size_t)slots * 4, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        double t = 0.0;
        for (float v : l) t += v;
        *loss_host = (float)(t * inv_n);
    }
    (void)n;
    return NL_OK;
}

nl_status nl_mlp_grad(nl_mlp *mlp, const float *X, const float *y, const float *w, int64_t n,
                      float *grad, float *loss, void *stream)
{
    if (!mlp || !X || !y || !w || !grad || n < 1) return fail(NL_ERR_ARG, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int64_t> idx(n);
    for (int64_t k = 0; k < n; ++k) idx[k] = k;
    CK(mlp->idx.ensure((size_t)n * 8));
    CK(cudaMemcpyAsync(mlp->idx.p, idx.data(), (size_t)n * 8, cudaMemcpyHostToDevice, s));
    nl_status st = mlp_run(mlp, X, y, w, n, mlp->idx.as<int64_t>(), n, grad, 0, 0.f,
                           1.f / (float)n, loss, s);
    if (st != NL_OK) return st;
    CK(cudaStreamSynchronize(s));
    return NL_OK;
}

nl_status nl_mlp_train(nl_mlp *mlp, const float *X, const float *y, const float *w, int64_t n,
                       int32_t epochs, int32_t batch, float lr, uint64_t seed, float *loss,
                       void *stream)
{
    if (!mlp || !X || !y || !w || n < 1 || epochs < 1 || batch < 64 || !(lr > 0.f))
        return fail(NL_ERR_ARG, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int64_t> idx(n);
    for (int64_t k = 0; k < n; ++k) idx[k] = k;
    std::mt19937_64 rng(seed);
    CK(mlp->idx.ensure((size_t)n * 8));
    float last = 0.f;
    for (int ep = 0; ep < epochs; ++ep) {
        std::shuffle(idx.begin(), idx.end(), rng);
        CK(cudaMemcpyAsync(mlp->idx.p, idx.data(), (size_t)n * 8, cudaMemcpyHostToDevice, s));
        double tot = 0.0;
        for (int64_t b0 = 0; b0 < n; b0 += batch) {
            const int64_t nb = std::min<int64_t>(batch, n - b0);
            float lb = 0.f;
            const bool want = (ep == epochs - 1);
            nl_status st = mlp_run(mlp, X, y, w, n, mlp->idx.as<int64_t>() + b0, nb, nullptr, 1, lr,
                                   1.f / (float)nb, want ? &lb : nullptr, s);
            if (st != NL_OK) return st;
            tot += (double)lb * nb;
        }
        if (ep == epochs - 1) last = (float)(tot / (double)n);
        CK(cudaStreamSynchronize(s));  // idx is rewritten by the next epoch
    }
    if (loss) *loss = last;
    return NL_OK;
}

nl_status nl_mlp_predict(const nl_mlp *mlp, const float *X, int64_t n, float *pred, void *stream)
{
    if (!mlp || !X || !pred || n < 1) return fail(NL_ERR_ARG, "bad argument");
    int dev, sms;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CK(mlp_predict(n, X, mlp->P.as<float>(), pred, sms, (cudaStream_t)stream));
    return NL_OK;
}

nl_status nl_set_mlp(nl_list *nl, const nl_mlp *mlp)
{
    if (!nl) return fail(NL_ERR_ARG, "list is NULL");
    nl->mlp = mlp;
    return NL_OK;
}

static nl_status do_iterate_h(nl_list *nl, const float *x, const float *y, const float *z,
                              float *h, int64_t n, int32_t nsys, const int64_t *offs,
                              const nl_box *boxes, const nl_params *p, float n_target, float tol,
                              int32_t max_iter, float margin, int32_t start, uint8_t *converged,
                              nl_hiter_info *info, cudaStream_t s)
{
    if (!nl) return fail(NL_ERR_ARG, "list is NULL");
    if (!h) return fail(NL_ERR_ARG, "h is NULL");
    if (!(n_target >= 1.f) || !(tol >= 0.f) || max_iter < 1 || !(margin >= 0.f) || !(margin < 4.f))
        return fail(NL_ERR_ARG, "need n_target >= 1, tol >= 0, max_iter >= 1, 0 <= margin < 4");
    if (start != NL_HSTART_GIVEN && start != NL_HSTART_PLAIN && start != NL_HSTART_LEARNED)
        return fail(NL_ERR_ARG, "unknown start %d", start);
    if (start == NL_HSTART_LEARNED && !nl->mlp) return fail(NL_ERR_ARG, "no model attached");
    if (n < 1 || n > (int64_t)1 << 30) return fail(NL_ERR_ARG, "bad n %lld", (long long)n);
    nl->n = 0;
    const uint32_t N = (uint32_t)n;
    const float *hin = h;
    if (start != NL_HSTART_GIVEN) {
        CK(nl->it_tmp.ensure((size_t)N * 4));
        CK(launch_fill(nl->it_tmp.as<float>(), N, 1e-30f, s));
        hin = nl->it_tmp.as<float>();
    }
    // the iteration re-runs single super-clusters on full lists
    nl_params pf = p ? *p : nl_params{};
    pf.half_list = 0;
    nl_status st = do_prep(nl, x, y, z, hin, n, nsys, offs, boxes, p ? &pf : nullptr, s);
    if (st != NL_OK) return st;
    const int M = p->cluster;
    const uint32_t nsc = nl->nsc, npad = nl->npad;
    CK(nl->it_hq.ensure((size_t)npad * 4));
    CK(nl->it_hlo.ensure((size_t)npad * 4));
    CK(nl->it_hhi.ensure((size_t)npad * 4));
    CK(nl->it_hs.ensure((size_t)npad * 4));
    CK(nl->it_counts.ensure((size_t)npad * 4));
    CK(nl->it_conv.ensure((size_t)npad));
    CK(nl->it_aflag.ensure((size_t)nsc * 4));
    CK(nl->it_alist.ensure((size_t)nsc * 4));
    CK(nl->it_words.ensure(16));
    const SysTables T = nl->tables();
    HIterState hs{nl->it_hq.as<float>(), nl->it_hlo.as<float>(), nl->it_hhi.as<float>(),
                  nl->it_hs.as<float>(), nl->it_counts.as<uint32_t>(), nl->it_conv.as<uint8_t>(),
                  nl->it_aflag.as<uint32_t>(), nl->it_alist.as<uint32_t>(),
                  nl->it_words.as<unsigned int>(), nl->perm_pad.as<uint32_t>(),
                  nl->sys_hcap.as<float>()};
    if (start == NL_HSTART_GIVEN) {
        CK(launch_pos_h_to(npad, nl->pos.as<float4>(), hs.hq, s));
    } else if (start == NL_HSTART_PLAIN) {
        CK(launch_plain_h0(nsc, M, hs.perm_pad, nl->clo.as<float4>(), nl->chi.as<float4>(),
                           n_target, hs.hq, s));
    } else {
        st = learned_start(nl, hs.hq, s);
        if (st != NL_OK) return st;
    }
    CK(cudaMemsetAsync(hs.hlo, 0, (size_t)npad * 4, s));
    CK(launch_fill(hs.hhi, npad, INFINITY, s));
    CK(cudaMemsetAsync(hs.conv, 0, (size_t)npad, s));
    CK(cudaMemsetAsync(hs.active_flag, 0, (size_t)nsc * 4, s));
    const OctreeOut oo = nl->octree_out();
    bool rebuild = true, first = true;
    int iters = 0, rebuilds = 0;
    unsigned int words[4] = {0, 0, 0, 0};
    nl->hiter_trace.clear();
    for (; iters < max_iter;) {
        const auto t_iter = std::chrono::steady_clock::now();
        nl_hiter_step step{};
        step.rebuilt = rebuild ? 1 : 0;
        step.active = first ? (int64_t)nsc : (int64_t)words[2];
        if (rebuild) {
            CK(launch_hsearch(npad, hs.hq, hs.hhi, hs.conv, margin, hs.hcap_sys, T, hs.hs, s));
            CK(launch_pos_h(npad, hs.hs, nl->pos.as<float4>(), s));
            CK(launch_cluster_boxes(npad, M, jcl(p), nl->pos.as<float4>(), p->support,
                                    nl->clo.as<float4>(), nl->chi.as<float4>(),
                                    nl->jlo.as<float4>(), nl->jhi.as<float4>(), s));
            CK(octree_boxes(nl->node_cap, nl->pos.as<float4>(), p->support, oo,
                            nl->status.as<Status>(), s));
            st = do_search(nl, s);
            if (st != NL_OK) return st;
            ++rebuilds;
        }
        PassArgs a = pass_args(nl);
        a.outc = hs.counts;
        a.hq = hs.hq;
        a.sorted_out = 1;
        if (!first) {
            a.work = hs.active_list;
            a.nwork = words[2];
        }
        CK(run_pass(nl, a, PASS_COUNT, s));
        ++iters;
        first = false;
        CK(cudaMemsetAsync(hs.words, 0, 16, s));
        CK(launch_hupdate(npad, M, n_target, tol, T, hs, s));
        CK(launch_active_list(nsc, hs, s));
        CK(cudaMemcpyAsync(words, hs.words, 16, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        step.unconverged = words[0];
        step.entries = (int64_t)nl->n_entries;
        step.tiles = (int64_t)nl->n_tiles;
        step.ms = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t_iter).count();
        nl->hiter_trace.push_back(step);
        if (words[0] == 0) break;
        rebuild = words[1] != 0;
    }
    CK(launch_scatter_h(npad, hs.perm_pad, hs.hq, hs.conv, h, converged, s));
    CK(cudaStreamSynchronize(s));
    if (info) {
        info->iterations = iters;
        info->rebuilds = rebuilds;
        info->unconverged = words[0];
    }
    if (words[0] != 0)
        return fail(NL_ERR_NOT_CONVERGED, "%u particles outside the neighbor window after %d passes",
                    words[0], iters);
    return NL_OK;
}

nl_status nl_iterate_h(nl_list *nl, const float *x, const float *y, const float *z, float *h,
                       int64_t n, const nl_box *box, const nl_params *p, float n_target, float tol,
                       int32_t max_iter, float margin, int32_t start, uint8_t *converged,
                       nl_hiter_info *info, void *stream)
{
    if (!box) return fail(NL_ERR_ARG, "box is NULL");
    const int64_t offs[2] = {0, n};
    return do_iterate_h(nl, x, y, z, h, n, 1, offs, box, p, n_target, tol, max_iter, margin, start,
                        converged, info, (cudaStream_t)stream);
}

nl_status nl_iterate_h_batch(nl_list *nl, const float *x, const float *y, const float *z, float *h,
                             int32_t nsys, const int64_t *offsets, const nl_box *boxes,
                             const nl_params *p, float n_target, float tol, int32_t max_iter,
                             float margin, int32_t start, uint8_t *converged, nl_hiter_info *info,
                             void *stream)
{
    if (!offsets || nsys < 1) return fail(NL_ERR_ARG, "need nsys >= 1 and offsets");
    return do_iterate_h(nl, x, y, z, h, offsets[nsys], nsys, offsets, boxes, p, n_target, tol,
                        max_iter, margin, start, converged, info, (cudaStream_t)stream);
}

}  // extern "C"

struct nl_graph {
    nl_list *nl = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" {

nl_status nl_graph_create(nl_list *nl, const float *x, const float *y, const float *z,
                          const float *h, const float *m, float *rho, int32_t nsys,
                          const int64_t *offsets, const nl_box *boxes, const nl_params *p,
                          void *stream, nl_graph **out)
{
    if (!out) return fail(NL_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!nl || !m || !rho) return fail(NL_ERR_ARG, "NULL list, m or rho");
    cudaStream_t s = (cudaStream_t)stream;
    if (!s) return fail(NL_ERR_ARG, "graph capture needs a non-default stream");
    // 1. a normal build and pass size every buffer and validate the inputs
    nl_status st = nl_rebuild_batch(nl, x, y, z, h, nsys, offsets, boxes, p, stream);
    if (st != NL_OK) return st;
    st = nl_density_pass(nl, m, rho, stream);
    if (st != NL_OK) return st;
    // slack for the replays: list bytes; the node arrays already carry 1/8
    const size_t want = (size_t)nl->list_bytes + nl->list_bytes / 4 + 65536;
    if (nl->list.cap < want) {
        DevBuf bigger;
        CK(bigger.ensure(want));
        nl->list.release();
        nl->list = bigger;
    }
    {
        // staging for the full persistent grid (the redo rounds of the build
        // above may have grown the per-slot capacity on a smaller grid)
        const int tpb = p->threads_per_block ? p->threads_per_block : 256;
        const size_t slots = (size_t)nl->num_sms *
                             (p->blocks_per_sm ? p->blocks_per_sm : kSearchBlocksPerSM) * (tpb / 32);
        CK(nl->stageJ.ensure(slots * nl->stage_cap * 4));
        CK(nl->stageM.ensure(slots * nl->stage_cap));
    }
    {
        // half search buffers: slack over the sizes of this build, and sort
        // buffers for the whole tuple capacity (a replay sorts all of it)
        const Status &hs = *nl->hst;
        const size_t up = (size_t)hs.up_used + hs.up_used / 4 + 4096;
        const size_t tu = (size_t)hs.tu_used + hs.tu_used / 4 + 4096;
        CK(nl->uJ.ensure(up * 4));
        CK(nl->uM.ensure(up));
        CK(nl->tkey.ensure(tu * 8));
        CK(nl->tval.ensure(tu * 4));
        CK(nl->tkey_alt.ensure(tu * 8));
        CK(nl->tval_alt.ensure(tu * 4));
        CK(nl->thist.ensure(radix_hist_words((uint32_t)tu) * 4));
        nl->graph_up_cap = up;
        nl->graph_tu_cap = tu;
    }
    CK(cudaStreamSynchronize(s));
    const int64_t n = offsets[nsys];
    const int prof = nl->profiling;
    nl->profiling = 0;
    // 2. capture the sync-free step
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    nl->graph_mode = 1;
    st = do_prep(nl, x, y, z, h, n, nsys, offsets, boxes, p, s);
    if (st == NL_OK) st = do_search(nl, s);
    if (st == NL_OK) st = nl_density_pass(nl, m, rho, stream);
    nl->graph_mode = 0;
    nl->profiling = prof;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &g);
    if (st != NL_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture", __LINE__);
    cudaGraphExec_t ge = nullptr;
    e = cudaGraphInstantiate(&ge, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(e, "cudaGraphInstantiate", __LINE__);
    }
    nl_graph *G = new (std::nothrow) nl_graph();
    if (!G) {
        cudaGraphExecDestroy(ge);
        cudaGraphDestroy(g);
        return fail(NL_ERR_OOM, "host allocation failed");
    }
    G->nl = nl;
    G->graph = g;
    G->exec = ge;
    *out = G;
    return NL_OK;
}

nl_status nl_graph_launch(nl_graph *g, void *stream)
{
    if (!g) return fail(NL_ERR_ARG, "graph is NULL");
    CK(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
    return NL_OK;
}

nl_status nl_graph_check(nl_graph *g, void *stream)
{
    if (!g) return fail(NL_ERR_ARG, "graph is NULL");
    nl_list *nl = g->nl;
    nl_status st = read_status(nl, (cudaStream_t)stream);
    if (st != NL_OK) return st;
    const Status &h = *nl->hst;
    if (h.bad_input & 7u) return fail(NL_ERR_ARG, "invalid particle input in the last replay");
    if (h.bad_input & 8u) return fail(NL_ERR_RADIUS, "support*h >= L/2 on a periodic axis");
    if (h.node_overflow)
        return fail(NL_ERR_CAPACITY, "octree needs %u more nodes than the graph reserved",
                    h.node_overflow);
    if (h.stage_overflow)
        return fail(NL_ERR_CAPACITY, "%u super-cluster lists did not fit the graph's buffers",
                    h.stage_overflow);
    if (h.half_overflow || h.list_overflow)
        return fail(NL_ERR_CAPACITY, "the lists outgrew the buffers the graph reserved");
    nl->n_leaves = h.n_leaves;
    nl->n_nodes = h.n_nodes;
    nl->list_bytes = h.list_used;
    nl->n_entries = h.n_entries;
    nl->n_tiles = h.n_tiles;
    nl->node_visits = h.node_visits;
    nl->leaf_visits = h.leaf_visits;
    nl->j_examined = h.j_examined;
    nl->tile_tests = h.tile_tests;
    return NL_OK;
}

nl_status nl_graph_free(nl_graph *g)
{
    if (!g) return NL_OK;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return NL_OK;
}

nl_status nl_autotune_batch(const float *x, const float *y, const float *z, const float *h,
                            const float *m, int32_t nsys, const int64_t *offsets,
                            const nl_box *boxes, const nl_params *base, int32_t reps,
                            nl_params *best, float *best_ms, void *stream)
{
    if (!base || !best || !m || !offsets || nsys < 1) return fail(NL_ERR_ARG, "NULL argument");
    if (reps < 1) return fail(NL_ERR_ARG, "reps must be >= 1");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = offsets[nsys];
    DevBuf rho;
    CK(rho.ensure((size_t)n * 4));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    nl_list *nl = new (std::nothrow) nl_list();
    if (!nl) return fail(NL_ERR_OOM, "host allocation failed");
    // tile shapes M x MJ
    const int Ms[5] = {4, 8, 8, 16, 16}, MJs[5] = {4, 8, 4, 16, 8};
    const int T[2] = {128, 256}, B[3] = {2, 3, 4};
    float bms = INFINITY;
    nl_params bp = *base;
    nl_status st = NL_OK;
    for (int mi = 0; mi < 5 && st == NL_OK; ++mi)
        for (int ti = 0; ti < 2 && st == NL_OK; ++ti)
            for (int bi = 0; bi < 3 && st == NL_OK; ++bi) {
                if (base->half_list && MJs[mi] != Ms[mi]) continue;  // half lists need MJ = M
                nl_params c = *base;
                c.cluster = Ms[mi];
                c.j_cluster = MJs[mi];
                c.threads_per_block = T[ti];
                c.blocks_per_sm = B[bi];
                float tot = 0.f;
                for (int r = 0; r <= reps && st == NL_OK; ++r) {
                    cudaEventRecord(e0, s);
                    st = nl_rebuild_batch(nl, x, y, z, h, nsys, offsets, boxes, &c, stream);
                    if (st == NL_OK) st = nl_density_pass(nl, m, rho.as<float>(), stream);
                    cudaEventRecord(e1, s);
                    cudaEventSynchronize(e1);
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (r > 0) tot += ms;  // r = 0 warms up
                }
                if (st == NL_OK && tot / reps < bms) {
                    bms = tot / reps;
                    bp = c;
                }
            }
    nl->release_all();
    delete nl;
    rho.release();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != NL_OK) return st;
    *best = bp;
    if (best_ms) *best_ms = bms;
    return NL_OK;
}

nl_status nl_free(nl_list *nl)
{
    if (!nl) return NL_OK;
    cudaDeviceSynchronize();
    nl->release_all();
    delete nl;
    return NL_OK;
}

nl_status nl_density_pass(const nl_list *cnl, const float *m, float *rho, void *stream)
{
    nl_status st = check_list(cnl);
    if (st != NL_OK) return st;
    if (!m || !rho) return fail(NL_ERR_ARG, "NULL m or rho");
    nl_list *nl = const_cast<nl_list *>(cnl);
    cudaStream_t s = (cudaStream_t)stream;
    const bool half = nl->p.half_list != 0;
    CK(nl->aux.ensure((size_t)nl->npad * 8));
    if (half) CK(nl->hsum.ensure((size_t)nl->npad * 8));
    Status *dst = nl->status.as<Status>();
    CK(nl->mark(6, s));
    if (half) CK(cudaMemsetAsync(&dst->m_absmax, 0, sizeof(unsigned int), s));
    CK(launch_gather_aux(nl->npad, nl->perm_pad.as<uint32_t>(), m, nullptr, nullptr, 0,
                         nl->aux.as<float2>(), s, half ? &dst->m_absmax : nullptr));
    if (half) CK(cudaMemsetAsync(nl->hsum.p, 0, (size_t)nl->npad * 8, s));
    CK(nl->mark(7, s));
    PassArgs a = pass_args(nl);
    a.out0 = rho;
    CK(run_pass(nl, a, PASS_DENSITY, s));
    if (half) CK(launch_half_finish(a, PASS_DENSITY, nl->npad, s));
    CK(nl->mark(8, s));
    return NL_OK;
}

nl_status nl_force_pass(const nl_list *cnl, int32_t kind, const float *params, const float *m,
                        const float *rho, const float *pres, float *ax, float *ay, float *az,
                        void *stream)
{
    nl_status st = check_list(cnl);
    if (st != NL_OK) return st;
    if (!ax || !ay || !az) return fail(NL_ERR_ARG, "NULL force output");
    nl_list *nl = const_cast<nl_list *>(cnl);
    cudaStream_t s = (cudaStream_t)stream;
    const bool half = nl->p.half_list != 0;
    if (half) CK(nl->hf.ensure((size_t)nl->npad * 24));
    if (kind == NL_FORCE_SPH_PRESSURE) {
        if (!m || !rho || !pres) return fail(NL_ERR_ARG, "SPH force needs m, rho and pres");
        CK(nl->aux.ensure((size_t)nl->npad * 8));
    }
    PassArgs a = pass_args(nl);  // after every buffer it points to exists
    a.out0 = ax;
    a.out1 = ay;
    a.out2 = az;
    if (kind == NL_FORCE_SPH_PRESSURE) {
        CK(nl->mark(6, s));
        CK(launch_gather_aux(nl->npad, nl->perm_pad.as<uint32_t>(), m, pres, rho, 1,
                             nl->aux.as<float2>(), s));
        CK(nl->mark(7, s));
        if (half) CK(cudaMemsetAsync(nl->hf.p, 0, (size_t)nl->npad * 24, s));
        CK(run_pass(nl, a, PASS_SPH, s));
        if (half) CK(launch_half_finish(a, PASS_SPH, nl->npad, s));
        CK(nl->mark(8, s));
    } else if (kind == NL_FORCE_LJ) {
        if (!params) return fail(NL_ERR_ARG, "LJ force needs params {eps, sigma}");
        if (!std::isfinite(params[0]) || !(params[1] > 0.f))
            return fail(NL_ERR_ARG, "LJ needs finite eps and sigma > 0");
        a.p0 = params[0];
        a.p1 = params[1];
        CK(nl->mark(6, s));
        CK(nl->mark(7, s));
        if (half) CK(cudaMemsetAsync(nl->hf.p, 0, (size_t)nl->npad * 24, s));
        CK(run_pass(nl, a, PASS_LJ, s));
        if (half) CK(launch_half_finish(a, PASS_LJ, nl->npad, s));
        CK(nl->mark(8, s));
    } else if (kind == NL_FORCE_LJ_COULOMB) {
        if (!params) return fail(NL_ERR_ARG, "LJ + Coulomb needs params {eps, sigma, rc, kc}");
        if (!std::isfinite(params[0]) || !(params[1] > 0.f) || !(params[2] >= 0.f) ||
            !std::isfinite(params[2]) || !std::isfinite(params[3]))
            return fail(NL_ERR_ARG, "LJ + Coulomb needs finite eps, kc, sigma > 0 and rc >= 0");
        CK(nl->aux.ensure((size_t)nl->npad * 8));
        a = pass_args(nl);
        a.out0 = ax;
        a.out1 = ay;
        a.out2 = az;
        a.p0 = params[0];
        a.p1 = params[1];
        a.p2 = params[2] > 0.f ? params[2] * params[2] : INFINITY;  // rounded once, as the predicate's r^2
        a.p3 = params[3];
        CK(nl->mark(6, s));
        if (m)
            CK(launch_gather_aux(nl->npad, nl->perm_pad.as<uint32_t>(), m, nullptr, nullptr, 0,
                                 nl->aux.as<float2>(), s));
        else
            CK(cudaMemsetAsync(nl->aux.p, 0, (size_t)nl->npad * 8, s));
        CK(nl->mark(7, s));
        if (half) CK(cudaMemsetAsync(nl->hf.p, 0, (size_t)nl->npad * 24, s));
        CK(run_pass(nl, a, PASS_LJC, s));
        if (half) CK(launch_half_finish(a, PASS_LJC, nl->npad, s));
        CK(nl->mark(8, s));
    } else {
        return fail(NL_ERR_ARG, "unknown force kind %d", kind);
    }
    return NL_OK;
}

nl_status nl_refresh_positions(nl_list *nl, const float *x, const float *y, const float *z,
                               float *max_disp, void *stream)
{
    nl_status st = check_list(nl);
    if (st != NL_OK) return st;
    if (!x || !y || !z) return fail(NL_ERR_ARG, "NULL position array");
    cudaStream_t s = (cudaStream_t)stream;
    if (!nl->moved) {
        CK(nl->pos_ref.ensure((size_t)nl->npad * sizeof(float4)));
        CK(cudaMemcpyAsync(nl->pos_ref.p, nl->pos.p, (size_t)nl->npad * sizeof(float4),
                           cudaMemcpyDeviceToDevice, s));
    }
    CK(launch_refresh(nl->npad, nl->perm_pad.as<uint32_t>(), nl->tables(), x, y, z,
                      nl->pos.as<float4>(), nl->pos_ref.as<float4>(), max_disp, s));
    nl->moved = 1;
    if (nl->any_per) {
        // the passes split periodic super-clusters into interior ones (no
        // wrapped pair within the largest radius R of the system: the box of
        // their particles stays more than R from every periodic face) and
        // boundary ones; the split is redone for the new positions, from the
        // cluster boxes of those positions
        const int M = nl->p.cluster;
        CK(launch_cluster_boxes(nl->npad, M, jcl(&nl->p), nl->pos.as<float4>(), nl->p.support,
                                nl->clo.as<float4>(), nl->chi.as<float4>(),
                                nl->jlo.as<float4>(), nl->jhi.as<float4>(), s));
        Status *dst = nl->status.as<Status>();
        CK(cudaMemsetAsync(&dst->n_int, 0, 2 * sizeof(unsigned int), s));
        const bool mixed = nl->n_open && nl->n_per;
        CK(launch_classify(mixed ? nl->sc_per.as<uint32_t>() : nullptr, mixed ? nl->n_per : nl->nsc,
                           M, nl->tables(), nl->clo.as<float4>(), nl->chi.as<float4>(),
                           nl->nlo.as<float4>(), nl->node_cap, nl->sc_int.as<uint32_t>(),
                           nl->sc_bnd.as<uint32_t>(), dst, s));
    }
    return NL_OK;
}

nl_status nl_neighbor_counts(const nl_list *cnl, uint32_t *counts, void *stream)
{
    nl_status st = check_list(cnl);
    if (st != NL_OK) return st;
    if (!counts) return fail(NL_ERR_ARG, "NULL counts");
    nl_list *nl = const_cast<nl_list *>(cnl);
    cudaStream_t s = (cudaStream_t)stream;
    const bool half = nl->p.half_list != 0;
    if (half) {
        CK(nl->hcnt.ensure((size_t)nl->npad * 4));
        CK(cudaMemsetAsync(nl->hcnt.p, 0, (size_t)nl->npad * 4, s));
    }
    PassArgs a = pass_args(nl);
    a.outc = counts;
    CK(run_pass(nl, a, PASS_COUNT, s));
    if (half) CK(launch_half_finish(a, PASS_COUNT, nl->npad, s));
    return NL_OK;
}

nl_status nl_nearest_distance(const nl_list *cnl, float *dist, void *stream)
{
    nl_status st = check_list(cnl);
    if (st != NL_OK) return st;
    if (!dist) return fail(NL_ERR_ARG, "NULL dist");
    nl_list *nl = const_cast<nl_list *>(cnl);
    cudaStream_t s = (cudaStream_t)stream;
    const bool half = nl->p.half_list != 0;
    if (half) {
        CK(nl->hcnt.ensure((size_t)nl->npad * 4));
        CK(launch_fill(nl->hcnt.as<float>(), nl->npad, INFINITY, s));
    }
    PassArgs a = pass_args(nl);
    a.out0 = dist;
    CK(run_pass(nl, a, PASS_MIN, s));
    if (half) CK(launch_half_finish(a, PASS_MIN, nl->npad, s));
    return NL_OK;
}

nl_status nl_get_hiter_trace(const nl_list *nl, nl_hiter_step *steps, int32_t cap, int32_t *count)
{
    if (!nl || !count || cap < 0 || (cap > 0 && !steps))
        return fail(NL_ERR_ARG, "nl_get_hiter_trace: bad argument");
    const int32_t k = (int32_t)nl->hiter_trace.size();
    for (int32_t i = 0; i < k && i < cap; ++i) steps[i] = nl->hiter_trace[(size_t)i];
    *count = k;
    return NL_OK;
}

nl_status nl_get_sizes(const nl_list *nl, nl_sizes *out)
{
    nl_status st = check_list(nl);
    if (st != NL_OK) return st;
    if (!out) return fail(NL_ERR_ARG, "NULL out");
    out->n = nl->n;
    out->n_clusters = nl->ncl;
    out->n_superclusters = nl->nsc;
    out->n_leaves = nl->n_leaves;
    out->n_nodes = nl->n_nodes;
    out->n_entries = (int64_t)nl->n_entries;
    out->n_tiles = (int64_t)nl->n_tiles;
    out->list_bytes = (int64_t)nl->list_bytes;
    out->cluster = nl->p.cluster;
    out->compress = nl->p.compress;
    out->j_cluster = jcl(&nl->p);
    out->node_visits = (int64_t)nl->node_visits;
    out->leaf_visits = (int64_t)nl->leaf_visits;
    out->j_examined = (int64_t)nl->j_examined;
    out->tile_tests = (int64_t)nl->tile_tests;
    return NL_OK;
}

nl_status nl_copy_sorted(const nl_list *nl, uint64_t *keys, int32_t *perm)
{
    nl_status st = check_list(nl);
    if (st != NL_OK) return st;
    CK(cudaDeviceSynchronize());
    if (keys) CK(cudaMemcpy(keys, nl->keys.p, (size_t)nl->n * 8, cudaMemcpyDeviceToHost));
    if (perm) CK(cudaMemcpy(perm, nl->vals.p, (size_t)nl->n * 4, cudaMemcpyDeviceToHost));
    return NL_OK;
}

nl_status nl_copy_octree(const nl_list *nl, int32_t *level, int32_t *first, int32_t *end,
                         int32_t *leaf, int32_t *skip)
{
    nl_status st = check_list(nl);
    if (st != NL_OK) return st;
    CK(cudaDeviceSynchronize());
    const size_t nn = nl->n_nodes;
    std::vector<uint8_t> lv(nn);
    std::vector<int2> rg(nn);
    std::vector<float4> hi(nn);
    CK(cudaMemcpy(lv.data(), nl->nlevel.p, nn, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(rg.data(), nl->nrng.p, nn * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(hi.data(), nl->nhi.p, nn * 16, cudaMemcpyDeviceToHost));
    for (size_t v = 0; v < nn; ++v) {
        int sk = __builtin_bit_cast(int, hi[v].w);
        if (level) level[v] = lv[v];
        if (first) first[v] = rg[v].x;
        if (end) end[v] = rg[v].y;
        if (leaf) leaf[v] = (size_t)sk == v + 1;
        if (skip) skip[v] = sk;
    }
    return NL_OK;
}

nl_status nl_copy_records(const nl_list *nl, uint64_t *rec_off, uint8_t *bytes)
{
    nl_status st = check_list(nl);
    if (st != NL_OK) return st;
    CK(cudaDeviceSynchronize());
    if (rec_off) {
        std::vector<uint32_t> w(nl->nsc);
        CK(cudaMemcpy(w.data(), nl->rec_off.p, (size_t)nl->nsc * 4, cudaMemcpyDeviceToHost));
        for (uint32_t s = 0; s < nl->nsc; ++s) rec_off[s] = (uint64_t)w[s] * 4u;
    }
    if (bytes) CK(cudaMemcpy(bytes, nl->list.p, nl->list_bytes, cudaMemcpyDeviceToHost));
    return NL_OK;
}

}  // extern "C"
