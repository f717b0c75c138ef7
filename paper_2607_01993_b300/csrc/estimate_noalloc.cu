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
// column operand, including padding, and all m weights), and a Canberra call
// resets the two words of its data range before it reduces into them, so nothing
// carries over between calls; two calls whose work overlaps on the GPU (different
// streams, no ordering between them) race on the array and must be serialised
// by the caller.
//
// Precision: the column scratch holds the FP32 operand of the CUDA-core sweep,
// so every call evaluates distances in FP32 on the CUDA cores, whatever prec
// asks for.  The results equal silh_estimate with SILH_PREC_FP32 bit for bit;
// for a tensor-core precision they are the more accurate FP32 values, not that
// mode's.
#include "kernels.cuh"

namespace silh {
namespace {

constexpr int64_t kNoAllocMaxColumns = SILH_NOALLOC_MAX_COLUMNS;  // include/silh.h
constexpr int64_t kNoAllocMaxFloats = SILH_NOALLOC_MAX_FLOATS;

// Column operand Y (m x D), then wY (m), zY (m) and one 256-byte slot whose
// first two words hold the Canberra sweep's data range (largest and smallest
// nonzero magnitude).
static __device__ __align__(256) float
    g_noalloc_scratch[kNoAllocMaxFloats + 2 * kNoAllocMaxColumns + 64];

// Device address of the scratch array for the current device.  The array's
// name is only a host-side stand-in in host code; the address must come from
// cudaGetSymbolAddress with the device current.  It is looked up on every call
// (no allocation, a table lookup once the module is loaded), so a cached address
// can never outlive a device reset or a re-created context.
silh_status noalloc_scratch(float **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SILH_ECUDA,
                    "cudaGetSymbolAddress(no-alloc scratch) failed: %s (the first call on a "
                    "device loads the library's device code and maps the %.1f MiB scratch; "
                    "make it before reserving the device's memory)",
                    cudaGetErrorString(e), sizeof(g_noalloc_scratch) / 1048576.0);
    }
    *out = static_cast<float *>(p);
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
                                             float *b_hat, int32_t *nb, void *stream_) {
    cudaStream_t stream = (cudaStream_t)stream_;
    silh_status st = SILH_OK;
    int D = 0;
    int64_t m = 0;
    float *base = nullptr, *Y = nullptr, *wY = nullptr, *zY = nullptr;
    unsigned *crange = nullptr;

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
    SILH_DEVPTR_OPT(nb, "neighbour");
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
    st = noalloc_scratch(&base);
    if (st != SILH_OK) goto done;
    Y = base;
    wY = base + kNoAllocMaxFloats;
    zY = wY + kNoAllocMaxColumns;
    if (metric == SILH_CANBERRA) {
        crange = reinterpret_cast<unsigned *>(zY + kNoAllocMaxColumns);
        st = canberra_range(X, dtype, n, d, ld, crange, stream);
        if (st != SILH_OK) goto done;
    }
    st = gather_columns(X, dtype, d, ld, S->idx, S->p, m, D, metric, crange, Y, wY, zY, stream);
    if (st != SILH_OK) goto done;
    st = phase2_sweep(X, dtype, n, d, ld, labels, k, metric, SILH_PREC_FP32, S->sizes, S->offsets,
                      Y, wY, zY, crange, m, D, rows, nrows, s_hat, a_hat, b_hat, nb, stream);
done:
    return st;
}
