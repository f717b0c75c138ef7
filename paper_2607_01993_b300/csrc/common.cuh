// Internal helpers of libsilh: status reporting, stream-ordered scratch,
// the counter-based generator, element loads.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <vector>

#include "../../include/silh.h"

namespace silh {

// ---------------------------------------------------------------- errors

void set_error(const char *fmt, ...);
silh_status fail(silh_status st, const char *fmt, ...);

// A failed CUDA call: SILH_ENOMEM when the device is out of memory (the error
// is cleared, the context stays usable), SILH_ECUDA otherwise.
#define SILH_CK(call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            if (e_ == cudaErrorMemoryAllocation) cudaGetLastError();                       \
            st = ::silh::fail(e_ == cudaErrorMemoryAllocation ? SILH_ENOMEM : SILH_ECUDA,   \
                              "%s:%d %s: %s", __FILE__, __LINE__, #call,                   \
                              cudaGetErrorString(e_));                                     \
            goto done;                                                                     \
        }                                                                                  \
    } while (0)

#define SILH_REQ(cond, ...)                                   \
    do {                                                      \
        if (!(cond)) {                                        \
            st = ::silh::fail(SILH_EINVAL, __VA_ARGS__);      \
            goto done;                                        \
        }                                                     \
    } while (0)

// --------------------------------------------------------------- scratch

// Stream-ordered scratch.  Every block is released with cudaFreeAsync on the
// same stream when the Scratch object goes out of scope, so the memory returns
// to the pool only after the kernels that use it have run.
struct Scratch {
    cudaStream_t stream;
    std::vector<void *> blocks;
    explicit Scratch(cudaStream_t s) : stream(s) {}
    ~Scratch() {
        for (void *p : blocks) cudaFreeAsync(p, stream);
    }
    template <class T>
    cudaError_t alloc(T **out, size_t count) {
        void *p = nullptr;
        size_t bytes = count * sizeof(T);
        if (bytes == 0) bytes = 16;
        bytes = (bytes + 255) & ~size_t(255);
        cudaError_t e = cudaMallocAsync(&p, bytes, stream);
        if (e != cudaSuccess) return e;
        blocks.push_back(p);
        *out = static_cast<T *>(p);
        return cudaSuccess;
    }
};

// True when p is memory a kernel may read or write: device, managed, or
// page-locked host memory (mapped into the unified address space).  Plain
// pageable host memory and null are not.
bool device_accessible(const void *p);

// The arrays of a sample set (sizes, offsets, and idx / p when non-empty).
bool sample_accessible(const silh_sample *S);

// A caller pointer that must be kernel-accessible (SILH_EINVAL otherwise);
// nullable ones are checked only when non-null.
#define SILH_DEVPTR(ptr, name) \
    SILH_REQ(::silh::device_accessible(ptr), "%s is not device-accessible memory", name)
#define SILH_DEVPTR_OPT(ptr, name) \
    SILH_REQ((ptr) == nullptr || ::silh::device_accessible(ptr), \
             "%s is not device-accessible memory", name)

// Keep freed scratch cached in the device's default pool between calls.
void ensure_pool_retains(int device);

// ------------------------------------------------- b_hat without division

// Running minimum over clusters of acc_j / |C_j| (b_hat, Eq. 8) with no
// division per cluster: a candidate (acc, size) replaces the best (bacc, bsz)
// when acc * bsz < bacc * size (sizes are positive; each product is rounded
// once), and the minimum itself is formed once, bacc / bsz.  Ties keep the
// lower cluster index (clusters are offered in increasing order), which is
// kept as the neighbouring cluster.  FP64 division is many times the cost of
// a multiply.
struct RatioMin {
    double acc, size;
    int arg;
    __device__ __forceinline__ RatioMin() : acc(INFINITY), size(1.0), arg(-1) {}
    __device__ __forceinline__ void add(double a, double sz, int j) {
        if (a * size < acc * sz) {
            acc = a;
            size = sz;
            arg = j;
        }
    }
    __device__ __forceinline__ double value() const { return acc / size; }
};

// ----------------------------------------------- warp column reduction

// Sums over the 32 lanes of CB per-lane values at once: halving exchanges
// (lanes below / above the offset keep the lower / upper half of the values)
// leave each lane one partial sum of column `col`, which plain butterfly steps
// then complete; lanes whose low log2(32 / CB) bits are zero hold the totals.
template <int CB>
__device__ __forceinline__ float transpose_reduce(float (&cs)[CB], int lane, int &col) {
    int base = 0, o = 16;
#pragma unroll
    for (int w = CB; w > 1; w >>= 1, o >>= 1) {
        const bool up = lane & o;
#pragma unroll
        for (int h = 0; h < w / 2; ++h) {
            const float send = up ? cs[h] : cs[h + w / 2];
            cs[h] = (up ? cs[h + w / 2] : cs[h]) + __shfl_xor_sync(0xffffffffu, send, o);
        }
        if (up) base += w / 2;
    }
#pragma unroll
    for (; o > 0; o >>= 1) cs[0] += __shfl_xor_sync(0xffffffffu, cs[0], o);
    col = base;
    return cs[0];
}

// ----------------------------------------------------------- Philox4x64-10

// Salmon et al., "Parallel random numbers: as easy as 1, 2, 3" (SC'11):
// 4x64 variant, 10 rounds.  Round: products of words 0 and 2 with the two
// multipliers; new words = (hi(w2*M1) ^ w1 ^ k0, lo(w2*M1), hi(w0*M0) ^ w3 ^ k1,
// lo(w0*M0)); the key advances by two Weyl increments between rounds.
__device__ __forceinline__ uint64_t philox_word0(uint64_t c0, uint64_t c1, uint64_t c2,
                                                 uint64_t c3, uint64_t k0, uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint64_t lo0 = M0 * c0, hi0 = __umul64hi(M0, c0);
        uint64_t lo1 = M1 * c2, hi1 = __umul64hi(M1, c2);
        uint64_t n0 = hi1 ^ c1 ^ k0;
        uint64_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += W0; k1 += W1;
    }
    return c0;
}

// U(seed, stream, cid, e) in [0, 1): key (seed, 0), counter (e, stream, cid, 0),
// top 53 bits of the first output word.
__device__ __forceinline__ double uniform01(uint64_t seed, uint64_t stream, uint64_t cid,
                                            uint64_t e) {
    uint64_t w = philox_word0(e, stream, cid, 0, seed, 0);
    return (double)(w >> 11) * 0x1.0p-53;
}

// ----------------------------------------------------------------- loads

template <class T>
__device__ __forceinline__ float to_f32(T v);
template <>
__device__ __forceinline__ float to_f32<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 v) {
    return __bfloat162float(v);
}

inline int ceil_div_i(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Number of kernels this library has launched in the process (all threads).
void count_launches(int nlaunch);

}  // namespace silh
