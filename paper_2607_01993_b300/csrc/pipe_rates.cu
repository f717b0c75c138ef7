// Throughput of the arithmetic pipes the sweeps are bound by, measured on the
// device itself: FP32 FMA (scalar and packed two-lane), the MUFU reciprocal and
// square root, FP32 min/max and FP64 FMA.  These rates turn the per-pair instruction
// counts of the CUDA-core and tensor-core epilogues into bounds.
//
// Each kernel runs as many 256-thread blocks per SM as fit at once (up to
// eight), every thread carrying eight independent dependency chains, so the
// pipe rather than the latency limits the rate.  The rate is the launch's
// total lane-operations over its CUDA-event duration (a few ms, so launch
// overhead is negligible); per-clock figures are formed by the caller from a
// sampled SM clock.
#include <algorithm>

#include "common.cuh"

namespace silh {
namespace {

constexpr int kRateThreads = 256;
constexpr int kRateBlocksPerSm = 8;
constexpr int kRateIters = 16384;
constexpr int kChains = 8;

enum { kFfma = 0, kFfma2 = 1, kRcp = 2, kSqrt = 3, kFmnmx = 4, kDfma = 5, kNumRates = 6 };

__device__ __forceinline__ float rcp_apx(float x) {
    float r;
    asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float sqrt_apx(float x) {
    float r;
    asm volatile("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Lane-operations of the chosen kind per thread: kRateIters * kChains (the
// packed form counts two lanes per instruction); sink keeps the results live.
template <int KIND>
__global__ void __launch_bounds__(kRateThreads)
k_rate(float seed, float *__restrict__ sink) {
    float v[kChains];
    float2 w[kChains];
    double u[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        v[c] = seed + 0.001f * (float)(threadIdx.x + c);
        w[c] = make_float2(v[c], v[c] + 0.5f);
        u[c] = (double)v[c];
    }
    const int iters = (KIND == kDfma) ? kRateIters / 16 : kRateIters;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            if (KIND == kFfma) v[c] = fmaf(v[c], 0.999f, 0.0001f);
            if (KIND == kFfma2) w[c] = __ffma2_rn(w[c], make_float2(0.999f, 0.999f),
                                                  make_float2(0.0001f, 0.0001f));
            if (KIND == kRcp) v[c] = rcp_apx(v[c] + 1.0f);
            if (KIND == kSqrt) v[c] = sqrt_apx(v[c] + 1.0f);
            if (KIND == kFmnmx) v[c] = fminf(fmaxf(v[c], -1.0f), 2.0f);
            if (KIND == kDfma) u[c] = fma(u[c], 0.999, 0.0001);
        }
    }
    float acc = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc += v[c] + w[c].x + w[c].y + (float)u[c];
    if (acc == 12345.678f) sink[blockIdx.x * kRateThreads + threadIdx.x] = acc;
}

}  // namespace
}  // namespace silh

using namespace silh;

// Measured lane-operations per second per SM: out[0] FP32 FMA, out[1] packed
// two-lane FP32 FMA (lanes), out[2] MUFU reciprocal, out[3] MUFU square root,
// out[4] FP32 min/max pairs counted as two operations, out[5] FP64 FMA.  Host
// array of 6 doubles.  Synchronous.  Diagnostic only (no counterpart in the paper).
extern "C" silh_status silh_pipe_rates(double *out, void *stream_) {
    cudaStream_t stream = (cudaStream_t)stream_;
    silh_status st = SILH_OK;
    int dev = 0, nsm = 0;
    float *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    Scratch sc(stream);
    SILH_REQ(out != nullptr, "out is null");
    SILH_CK(cudaGetDevice(&dev));
    SILH_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    SILH_CK(cudaEventCreate(&e0));
    SILH_CK(cudaEventCreate(&e1));
    {
        SILH_CK(sc.alloc(&sink, (size_t)nsm * kRateBlocksPerSm * kRateThreads));
        void (*kern[kNumRates])(float, float *) = {k_rate<kFfma>, k_rate<kFfma2>, k_rate<kRcp>,
                                                   k_rate<kSqrt>, k_rate<kFmnmx>, k_rate<kDfma>};
        for (int kind = 0; kind < kNumRates; ++kind) {
            // as many blocks as fit on every SM at once, so all run concurrently
            int per_sm = 0;
            SILH_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern[kind],
                                                                  kRateThreads, 0));
            per_sm = std::max(1, std::min(per_sm, kRateBlocksPerSm));
            const int blocks = nsm * per_sm;
            kern[kind]<<<blocks, kRateThreads, 0, stream>>>(1.0f, sink);   // warm-up
            SILH_CK(cudaEventRecord(e0, stream));
            kern[kind]<<<blocks, kRateThreads, 0, stream>>>(1.0f, sink);
            SILH_CK(cudaEventRecord(e1, stream));
            count_launches(2);
            SILH_CK(cudaGetLastError());
            SILH_CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            SILH_CK(cudaEventElapsedTime(&ms, e0, e1));
            const double lanes_per_thread = (double)(kind == kDfma ? kRateIters / 16 : kRateIters) *
                                            kChains * (kind == kFfma2 ? 2 : 1) *
                                            (kind == kFmnmx ? 2 : 1);
            out[kind] = lanes_per_thread * kRateThreads * blocks / ((double)ms * 1e-3) / nsm;
        }
    }
done:
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return st;
}
