// SFC ordering without device allocation: Hilbert/Morton keys and the stable
// radix-sort permutation for at most NL_NOALLOC_MAX_N particles, with every
// scratch buffer (ping-pong keys and indices, per-tile digit counts, status
// words) taken from one file-scope device array instead of cudaMalloc.
//
// Why: some callers cannot allocate device memory at the point where they
// need an SFC order -- latency-critical simulation loops where cudaMalloc's
// implicit device synchronisation is not acceptable, and host frameworks that
// own all device memory through their own pool and forbid driver allocations
// by the libraries they call.  They pass their own output arrays and get the
// same keys and permutation as nl_build computes.
//
// The array is part of this library's device image, so every GPU that loads
// the library holds it (about 14.7 MB) until the process exits.  Its device
// address is looked up once per device with cudaGetSymbolAddress, on the
// first call made with that device current; that first call belongs before
// any stream capture begins.  All calls share the one array:
// the status words are cleared at the start of each call, and calls that
// overlap on the GPU (different streams, or several host threads) race on it.
#include <mutex>

#include "nl_internal.cuh"

namespace nlg {
nl_status report_error(nl_status st, const char *msg);
}

using namespace nlg;

namespace {

constexpr uint32_t kMaxN = NL_NOALLOC_MAX_N;
constexpr size_t kStatusBytes = 256;
constexpr size_t kKeysBytes = (size_t)kMaxN * 8;
constexpr size_t kValsBytes = (size_t)kMaxN * 4;
constexpr size_t kHistWords = 8 * 256 + 64 + (size_t)8 * 256 * ((kMaxN + 4095) / 4096);
constexpr size_t kScratchBytes = kStatusBytes + kKeysBytes + kValsBytes + kHistWords * 4;
static_assert(sizeof(Status) <= kStatusBytes, "status words must fit their slot");

std::mutex g_mu;
constexpr int kMaxDevices = 256;
unsigned char *g_dev_ptr[kMaxDevices] = {};

}  // namespace

// The scratch itself.  In host code this name is only a stand-in for the
// symbol; kernels are given the address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_sfc_scratch[kScratchBytes];

namespace {

nl_status scratch_of_current_device(unsigned char **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        (void)cudaGetLastError();
        return report_error(NL_ERR_CUDA, "nl_sfc_order_noalloc: no current CUDA device");
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_dev_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_sfc_scratch);
        if (e != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return report_error(NL_ERR_CUDA,
                                "nl_sfc_order_noalloc: cudaGetSymbolAddress of the scratch failed");
        }
        g_dev_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_dev_ptr[dev];
    return NL_OK;
}

}  // namespace

extern "C" nl_status nl_sfc_order_noalloc(const float *x, const float *y, const float *z,
                                          const float *h, int64_t n, const nl_box *box,
                                          int32_t key, float support, uint64_t *keys,
                                          uint32_t *perm, void *stream)
{
    if (!x || !y || !z || !h || !keys || !perm || !box)
        return report_error(NL_ERR_ARG, "nl_sfc_order_noalloc: NULL argument");
    if (n < 1) return report_error(NL_ERR_ARG, "nl_sfc_order_noalloc: n must be >= 1");
    if (n > (int64_t)kMaxN)
        return report_error(NL_ERR_ARG,
                            "nl_sfc_order_noalloc: n exceeds NL_NOALLOC_MAX_N (1048576); "
                            "use nl_build for larger systems");
    if (key != NL_KEY_MORTON && key != NL_KEY_HILBERT)
        return report_error(NL_ERR_ARG, "nl_sfc_order_noalloc: unknown key kind");
    if (!(support > 0.f) || !(support < 3.0e38f))
        return report_error(NL_ERR_ARG, "nl_sfc_order_noalloc: support must be finite and > 0");
    DevBox b{};
    for (int a = 0; a < 3; ++a) {
        volatile float lo = box->lo[a], hi = box->hi[a];
        if (!(lo < hi) || !(hi - lo < 3.0e38f) || !(lo > -3.0e38f))
            return report_error(NL_ERR_ARG, "nl_sfc_order_noalloc: need finite box lo < hi");
        float len = hi - lo;
        volatile float num = 2097152.0f;
        b.lo[a] = lo;
        b.hi[a] = hi;
        b.len[a] = len;
        b.half[a] = 0.5f * len;
        b.qs[a] = num / len;
        b.per[a] = box->periodic[a] ? 1 : 0;
    }
    unsigned char *base = nullptr;
    nl_status st = scratch_of_current_device(&base);
    if (st != NL_OK) return st;
    Status *dst = reinterpret_cast<Status *>(base);
    uint64_t *keys_alt = reinterpret_cast<uint64_t *>(base + kStatusBytes);
    uint32_t *vals_alt = reinterpret_cast<uint32_t *>(base + kStatusBytes + kKeysBytes);
    uint32_t *hist = reinterpret_cast<uint32_t *>(base + kStatusBytes + kKeysBytes + kValsBytes);
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t N = (uint32_t)n;

    cudaError_t e = cudaMemsetAsync(dst, 0, sizeof(Status), s);
    if (e == cudaSuccess) e = launch_keys(n, x, y, z, h, b, support, key, keys, perm, dst, s);
    if (e == cudaSuccess) e = radix_sort_pairs(keys, perm, keys_alt, vals_alt, N, 3 * kKeyBits, hist,
                                                      &dst->sort_stall, s);
    Status hs{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, dst, sizeof(Status), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return report_error(NL_ERR_CUDA, cudaGetErrorString(e));
    }
    if (hs.sort_stall)
        return report_error(NL_ERR_TIMEOUT, "nl_sfc_order_noalloc: a radix-sort look-back gave up "
                                            "its bounded wait");
    if (hs.bad_input)
        return report_error(NL_ERR_ARG, "nl_sfc_order_noalloc: invalid particle input "
                                        "(non-finite or out-of-box coordinate, or h <= 0)");
    float rmax = __builtin_bit_cast(float, hs.rmax_bits);
    for (int a = 0; a < 3; ++a)
        if (b.per[a] && !(rmax < b.half[a]))
            return report_error(NL_ERR_RADIUS,
                                "nl_sfc_order_noalloc: support*max(h) >= L/2 on a periodic axis");
    return NL_OK;
}
