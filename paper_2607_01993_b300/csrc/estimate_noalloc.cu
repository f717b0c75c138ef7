// silh_estimate_noalloc: Phase 2 with its column scratch in a fixed,
// file-scope device array instead of stream-ordered allocations.
//
// Who needs it: callers that must not allocate device memory while they run --
// code that executes under a memory budget owned entirely by another allocator
// (a framework that has already reserved the device's memory), latency-bound
// loops that cannot absorb an allocation or its possible failure in the middle
// of a stream, and callers inside allocator or driver callbacks where calling
// back into the allocator is not allowed.  This entry point makes no cudaMalloc,
// cudaMallocAsync, cudaFree or other allocating call; the caller still passes
// every input and output buffer.
//
// The scratch array lives in this library's device image: every GPU that loads
// the library holds it until the process exits.  Every call shares it.  The
// gather kernel rewrites every element a call reads (all m x D entries of the
// column operand, including padding, and all m weights), so nothing needs to be
// cleared between calls; two calls whose work overlaps on the GPU (different
// streams, no ordering between them) race on the array and must be serialised
// by the caller.
#include <mutex>

#include "kernels.cuh"

namespace silh {
namespace {

constexpr int64_t kNoAllocMaxColumns = SILH_NOALLOC_MAX_COLUMNS;  // include/silh.h
constexpr int64_t kNoAllocMaxFloats = SILH_NOALLOC_MAX_FLOATS;

// Column operand Y (m x D), then wY (m) and zY (m).
static __device__ __align__(256) float g_noalloc_scratch[kNoAllocMaxFloats + 2 * kNoAllocMaxColumns];

std::mutex g_noalloc_mu;
float *g_noalloc_ptr[64] = {nullptr};

// Device address of the scratch array for the current device.  The array's
// name is only a host-side stand-in in host code; the address must come from
// cudaGetSymbolAddress with the device current.  Done once per device.
silh_status noalloc_scratch(int dev, float **out) {
    if (dev < 0 || dev >= 64) return fail(SILH_EINVAL, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (g_noalloc_ptr[dev] == nullptr) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return fail(SILH_ECUDA, "cudaGetSymbolAddress(no-alloc scratch) failed: %s",
                        cudaGetErrorString(e));
        g_noalloc_ptr[dev] = static_cast<float *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return SILH_OK;
}

}  // namespace
}  // namespace silh

using namespace silh;

extern "C" silh_status silh_estimate_noalloc(const void *X, silh_dtype dtype, int64_t n, int32_t d,
                                             int64_t ld, const int32_t *labels, int32_t k,
                                             silh_metric metric, silh_prec prec,
                                             const silh_sample *S, const int64_t *rows,
                                             int64_t nrows, float *s_hat, float *a_hat,
                                             float *b_hat, void *stream_) {
    cudaStream_t stream = (cudaStream_t)stream_;
    silh_status st = SILH_OK;
    int dev = 0;
    int D = 0;
    int64_t m = 0;
    float *base = nullptr, *Y = nullptr, *wY = nullptr, *zY = nullptr;

    SILH_REQ(X && labels, "null pointer argument");
    SILH_REQ(n >= 2 && n < (int64_t(1) << 31), "n must be in [2, 2^31)");
    SILH_REQ(d >= 1 && d <= 128 && ld >= d, "need 1 <= d <= 128 and ld >= d");
    SILH_REQ(k >= 2 && k <= SILH_MAX_K, "k must be in [2, %d]", SILH_MAX_K);
    SILH_REQ(metric >= SILH_EUCLIDEAN && metric <= SILH_CANBERRA, "unknown metric");
    SILH_REQ(dtype == SILH_F32 || dtype == SILH_BF16, "unknown dtype");
    SILH_REQ(prec >= SILH_PREC_FP32 && prec <= SILH_PREC_BF16X3, "unknown precision");
    SILH_REQ(S && S->k == k && S->sizes && S->offsets, "sample missing or k mismatch");
    m = S->size;
    SILH_REQ(m >= 0 && m <= S->cap && (m == 0 || (S->idx && S->p)), "bad sample size");
    SILH_REQ(s_hat, "s_hat is null");
    SILH_DEVPTR(X, "X");
    SILH_DEVPTR(labels, "labels");
    SILH_REQ(sample_accessible(S), "sample arrays are not device-accessible memory");
    SILH_DEVPTR(s_hat, "s_hat");
    SILH_DEVPTR_OPT(a_hat, "a_hat");
    SILH_DEVPTR_OPT(b_hat, "b_hat");
    SILH_DEVPTR_OPT(rows, "rows");
    D = padded_dim(d);
    if (m > kNoAllocMaxColumns || m * D > kNoAllocMaxFloats) {
        st = fail(SILH_ECAPACITY,
                  "sample of %lld columns x %d padded coordinates exceeds the no-alloc scratch "
                  "(at most %lld columns and %lld floats)",
                  (long long)m, D, (long long)kNoAllocMaxColumns, (long long)kNoAllocMaxFloats);
        goto done;
    }
    if (rows == nullptr) nrows = n;
    SILH_REQ(nrows >= 0, "nrows < 0");
    SILH_CK(cudaGetDevice(&dev));
    st = noalloc_scratch(dev, &base);
    if (st != SILH_OK) goto done;
    Y = base;
    wY = base + kNoAllocMaxFloats;
    zY = wY + kNoAllocMaxColumns;
    st = gather_columns(X, dtype, d, ld, S->idx, S->p, m, D, metric, Y, wY, zY, stream);
    if (st != SILH_OK) goto done;
    st = phase2_sweep(X, dtype, n, d, ld, labels, k, metric, prec, S->sizes, S->offsets, Y, wY, zY,
                      m, D, rows, nrows, s_hat, a_hat, b_hat, stream);
done:
    return st;
}
