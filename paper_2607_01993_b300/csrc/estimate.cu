// Phase 2 of Algorithm 1 (W_hat, a_hat, b_hat, s_hat), the exact silhouette
// (Eq. 1-2, the same sweep with F_Cj = Cj and p = 1) and the FP64 global mean
// (Eq. 3 / Eq. 6).
//
// Column operand: the sampled rows gathered into a dense cluster-major matrix
// Y (m x D floats, D = d rounded up, zero padded) with per-column weights
// wY = 1/p.  A CTA owns a tile of rows and streams the columns of one cluster
// after another through shared memory, so the per-row state is constant:
// the running FP32 sum of the current column chunk, the FP64 sum of the
// current cluster, the own-cluster weight and the running minimum for b_hat.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>

#include "kernels.cuh"

namespace silh {

int padded_dim(int d) {
    if (d <= 8) return 8;
    if (d <= 16) return 16;
    if (d <= 32) return 32;
    if (d <= 64) return 64;
    return 128;
}

namespace {

// ------------------------------------------------ Canberra at any scale
// A Canberra term |x_c - y_c| / (|x_c| + |y_c|) (Sec. 5.1.1) does not change
// when both coordinates are multiplied by the same factor.  The sweeps multiply
// every coordinate by one power of two, 2^-E with 2^E above the data's largest
// magnitude (exact, except below FP32's normal range), so every scaled
// magnitude is below 1 (at most 4 for data above 2^125) and the pair fraction
// (n1 d2 + n2 d1) / (d1 d2) cannot overflow, whatever the data's scale.  Each
// staged |y| carries +2^-63, which makes a 0/0 term 0 and keeps d1 d2 >= 2^-126,
// a normal FP32 number; the guard is below 2^-24 of every denominator whose
// coordinates are zero or at least 2^-39 in scaled magnitude.  A point with a
// nonzero coordinate below that ("tiny") has its pairs evaluated term by term
// from the unscaled values instead (canb_direct).
constexpr float kCanbGuard = 0x1p-63f;
constexpr float kCanbTiny = 0x1p-39f;

// 2^-E for the largest magnitude, range[0] (bits of a non-negative float;
// non-negative floats order like their bit patterns): range[0] 2^-E lands in
// [1/2, 1).
__host__ __device__ __forceinline__ float canb_scale_of(unsigned b) {
    if (b == 0u) return 1.0f;
    const int e = (int)(b >> 23);
    const int field = 253 - e < 1 ? 1 : (253 - e > 253 ? 253 : 253 - e);
    const unsigned bits = (unsigned)field << 23;
    float f;
    memcpy(&f, &bits, sizeof f);
    return f;
}

__device__ __forceinline__ float canb_scale(const unsigned *__restrict__ range) {
    return canb_scale_of(range ? range[0] : 0u);
}

// Whether any nonzero coordinate of the data is tiny at that scale: the
// smallest nonzero magnitude, range[1], times the scale is below 2^-39 (when
// the data have no nonzero value range[1] holds a sentinel near FLT_MAX).
__host__ __device__ __forceinline__ bool canb_tiny_of(unsigned min_bits, float scale) {
    float mn;
    memcpy(&mn, &min_bits, sizeof mn);
    return mn * scale < kCanbTiny;
}

__device__ __forceinline__ bool canb_tiny_data(const unsigned *__restrict__ range, float scale) {
    return range != nullptr && canb_tiny_of(range[1], scale);
}

__device__ __forceinline__ bool canb_is_tiny(float v, float scale) {
    return v != 0.f && fabsf(v * scale) < kCanbTiny;
}

// Canberra distance of one pair term by term from the unscaled coordinates
// (the path for points with tiny coordinates): each term's two coordinates are
// multiplied by a power of two that brings the larger magnitude into
// [2^-49, 2^64] (exact for the larger; the smaller only loses bits that are
// below FP32 resolution of the term), then |x - y| / (|x| + |y|) by the
// approximate reciprocal and one Newton step; a 0/0 term is 0.
__device__ __forceinline__ float rcp_nr(float den) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(den));
    return r;
}

template <class T>
__device__ __forceinline__ float canb_direct(const T *__restrict__ x, const float *__restrict__ y,
                                             int d) {
    float acc = 0.f;
    for (int c = 0; c < d; ++c) {
        const float xv = to_f32<T>(x[c]), yv = y[c];
        const float m = fmaxf(fabsf(xv), fabsf(yv));
        const float sc = m > 0x1p64f ? 0x1p-64f
                         : (m < 0x1p-100f ? 0x1p100f : (m < 0x1p-64f ? 0x1p64f : 1.0f));
        const float xs = xv * sc, ys = yv * sc;
        const float num = fabsf(xs - ys), den = fabsf(xs) + fabsf(ys);
        if (den > 0.f) {
            const float r = rcp_nr(den);
            float q = num * r;
            q = fmaf(r, fmaf(-q, den, num), q);
            acc += q;
        }
    }
    return acc;
}

// Largest and smallest nonzero |x| over the n x d data, as the bits of
// non-negative floats: range[0] (atomicMax, starts at 0) and range[1]
// (atomicMin, starts at a sentinel near FLT_MAX).  NaN is skipped.
template <class T>
__global__ void k_range(const T *__restrict__ X, int64_t n, int d, int64_t ld,
                        unsigned *__restrict__ range) {
    float mx = 0.f, mn = FLT_MAX;
    const int64_t total = n * (int64_t)d;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / d;
        const int c = (int)(i - r * d);
        const float a = fabsf(to_f32<T>(X[r * ld + c]));
        mx = fmaxf(mx, a);
        if (a > 0.f) mn = fminf(mn, a);
    }
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (mx > 0.f) atomicMax(&range[0], __float_as_uint(mx));
        if (mn < FLT_MAX) atomicMin(&range[1], __float_as_uint(mn));
    }
}

// ------------------------------------------------------------- gather

// zY: cosine, 0.5 wY for a zero column (below); Canberra, 1 for a column with a
// tiny coordinate at the data's scale (*crange), else 0.
template <class T>
__global__ void k_gather(const T *__restrict__ X, int d, int64_t ld, const int32_t *__restrict__ idx,
                         const double *__restrict__ p, int64_t m, int D, int metric,
                         const unsigned *__restrict__ crange, float *__restrict__ Y,
                         float *__restrict__ wY, float *__restrict__ zY,
                         const int64_t *__restrict__ d_m) {
    int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    int lane = threadIdx.x & 31;
    if (i >= m || (d_m != nullptr && i >= *d_m)) return;
    int64_t e = idx ? idx[i] : i;
    const T *x = X + e * ld;
    float scale = 1.0f;
    if (metric == SILH_COSINE) {
        float s = 0.f;
        for (int c = lane; c < d; c += 32) {
            const float v = to_f32<T>(x[c]);
            s = fmaf(v, v, s);
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        scale = s > 0.f ? rsqrtf(s) : 0.0f;
    }
    const float cs = (metric == SILH_CANBERRA) ? canb_scale(crange) : 1.0f;
    bool tiny = false;
    for (int c = lane; c < D; c += 32) {
        const float v = (c < d) ? to_f32<T>(x[c]) : 0.0f;
        if (metric == SILH_CANBERRA) tiny = tiny || canb_is_tiny(v, cs);
        Y[i * D + c] = v * scale;
    }
    tiny = __any_sync(0xffffffffu, tiny);
    if (lane == 0) {
        float w = p ? (float)(1.0 / p[i]) : 1.0f;
        wY[i] = w;
        // cosine: a zero column is at distance 1 from everything; the unit-vector
        // form 0.5 |x - y|^2 gives 0.5 for it, so it carries +0.5 w here.
        zY[i] = (metric == SILH_COSINE && scale == 0.0f) ? 0.5f * w : (tiny ? 1.0f : 0.0f);
    }
}

// ------------------------------------------------------- pair kernels

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Register / shared-memory slot layout of the coordinates.  Canberra stores
// each group of four coordinates as (c0, c2, c1, c3), so that the two-lane
// registers hold (c0, c2) and (c1, c3): the terms of the pairs (c0, c1) and
// (c2, c3), which share one reciprocal each, then sit in the same lane of two
// registers, and the pair fractions of both pairs are single packed
// instructions.  Other metrics keep the natural order.  The map is its own
// inverse: slot s holds coordinate canb_slot<METRIC>(s).
template <int METRIC>
__device__ __forceinline__ int canb_slot(int s) {
    return METRIC == SILH_CANBERRA ? (s & ~3) | ((s & 1) << 1) | ((s >> 1) & 1) : s;
}

// Distance of one row (registers, coordinate pairs) to one column (shared
// memory, float4 of NEGATED coordinates, so x - y is one packed add).
// Euclidean: sqrt(sum (x - y)^2).  Manhattan: sum |x - y|.  Cosine: rows and
// columns are unit-normalised and 1 - <x,y> is evaluated as 0.5 |x - y|^2
// (equal for unit vectors, and free of the cancellation of 1 - <x,y> for
// nearly parallel pairs).  Canberra: terms |x - y| / (|x| + |y|) taken two at a
// time as (n1 d2 + n2 d1)/(d1 d2) so that one reciprocal serves two
// coordinates, on coordinates scaled by the data's power-of-two scale; each
// denominator carries +2^-63 (added to |y| when the column is staged) so that
// an all-zero coordinate pair (including padding) contributes 0 and d1 d2
// stays a normal float (see "Canberra at any scale").  ax holds |x| when the caller
// keeps it in registers (NA = D / 2), else NA = 1 and |x| is formed here.
// Everything but the reciprocals is packed two-lane FP32 (one instruction for
// two coordinates, or for two Canberra pairs in the (c0, c2, c1, c3) slot
// order): the sweep is issue-bound, and packing halves the issue slots.
template <int METRIC, int D, int NA>
__device__ __forceinline__ float pair_dist(const float2 (&x)[D / 2], const float2 (&ax)[NA],
                                           const float4 *__restrict__ ny4,
                                           const float4 *__restrict__ ya4) {
    float2 sq0 = make_float2(0.f, 0.f), sq1 = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < D / 4; ++q) {
        const float4 y = ny4[q];
        const float2 t0 = __fadd2_rn(x[2 * q], make_float2(y.x, y.y));
        const float2 t1 = __fadd2_rn(x[2 * q + 1], make_float2(y.z, y.w));
        if (METRIC == SILH_EUCLIDEAN || METRIC == SILH_COSINE) {
            sq0 = __ffma2_rn(t0, t0, sq0);
            sq1 = __ffma2_rn(t1, t1, sq1);
        } else if (METRIC == SILH_MANHATTAN) {
            sq0 = __fadd2_rn(sq0, make_float2(fabsf(t0.x), fabsf(t0.y)));
            sq1 = __fadd2_rn(sq1, make_float2(fabsf(t1.x), fabsf(t1.y)));
        } else {
            const float4 ya = ya4[q];
            float2 a0, a1;
            if (NA == D / 2) {
                a0 = ax[(2 * q) % NA];
                a1 = ax[(2 * q + 1) % NA];
            } else {
                a0 = make_float2(fabsf(x[2 * q].x), fabsf(x[2 * q].y));
                a1 = make_float2(fabsf(x[2 * q + 1].x), fabsf(x[2 * q + 1].y));
            }
            // slots (c0, c2) and (c1, c3): t0 = (n0, n2), t1 = (n1, n3) are the
            // numerators |x - y|, d0 = (d0, d2), d1 = (d1, d3) the denominators
            const float2 d0 = __fadd2_rn(a0, make_float2(ya.x, ya.y));   // |x| + (|y| + 2^-63)
            const float2 d1 = __fadd2_rn(a1, make_float2(ya.z, ya.w));
            const float2 n0 = make_float2(fabsf(t0.x), fabsf(t0.y));
            const float2 n1 = make_float2(fabsf(t1.x), fabsf(t1.y));
            // pairs (c0, c1) and (c2, c3): (n0 d1 + n1 d0) / (d0 d1) in each lane
            const float2 num = __ffma2_rn(n0, d1, __fmul2_rn(n1, d0));
            const float2 den = __fmul2_rn(d0, d1);
            const float2 r = make_float2(rcp_approx(den.x), rcp_approx(den.y));
            if (q & 1) sq1 = __ffma2_rn(num, r, sq1);
            else sq0 = __ffma2_rn(num, r, sq0);
        }
    }
    if (METRIC == SILH_EUCLIDEAN) return sqrt_approx((sq0.x + sq0.y) + (sq1.x + sq1.y));
    if (METRIC == SILH_COSINE) return 0.5f * ((sq0.x + sq0.y) + (sq1.x + sq1.y));
    return (sq0.x + sq0.y) + (sq1.x + sq1.y);     // Manhattan, Canberra
}

// Whether a row tile keeps |x| in registers for Canberra (register budget).
template <int METRIC, int D, int RPT>
struct RowAbs {
    static constexpr int NA = (METRIC == SILH_CANBERRA && D * RPT <= 32) ? D / 2 : 1;
};

// Stage nq float4 of column coordinates as their negation (and, for Canberra,
// scaled by cscale, with |y| + 2^-63 beside them), in the slot order of
// canb_slot.
template <int METRIC>
__device__ __forceinline__ void stage_columns(const float4 *__restrict__ src, int nq,
                                              float *__restrict__ sh_ny, float *__restrict__ sh_ya,
                                              int tid, int nthreads, float cscale) {
    for (int q = tid; q < nq; q += nthreads) {
        float4 v = src[q];
        if (METRIC == SILH_CANBERRA)                                          // slot order
            v = make_float4(v.x * cscale, v.z * cscale, v.y * cscale, v.w * cscale);
        reinterpret_cast<float4 *>(sh_ny)[q] = make_float4(-v.x, -v.y, -v.z, -v.w);
        if (METRIC == SILH_CANBERRA)
            reinterpret_cast<float4 *>(sh_ya)[q] =
                make_float4(fabsf(v.x) + kCanbGuard, fabsf(v.y) + kCanbGuard,
                            fabsf(v.z) + kCanbGuard, fabsf(v.w) + kCanbGuard);
    }
}

constexpr int kThreads = 128;

// One CTA's tile of BM = 128 RPT rows [r0, r0 + BM) against the whole
// cluster-major column operand (Y, wY, zY, offsets): W_hat_j for every cluster
// and the silhouette of Eq. 8.  Shared by the single and the batched sweeps.
template <class T, int METRIC, int D, int RPT, int BN, bool CHECK_TINY = true>
__device__ __forceinline__ void sweep_rows(
        int64_t r0, const T *__restrict__ X, int d, int64_t ld, int64_t n,
        const int32_t *__restrict__ labels, int k, const int64_t *__restrict__ sizes,
        const int64_t *__restrict__ offsets, const float *__restrict__ Y,
        const float *__restrict__ wY, const float *__restrict__ zY,
        const unsigned *__restrict__ crange, const int64_t *__restrict__ rows, int64_t nrows,
        float *__restrict__ s_out,
        float *__restrict__ a_out, float *__restrict__ b_out, int32_t *__restrict__ nb_out,
        double *__restrict__ wown_out = nullptr, double *__restrict__ wsep_out = nullptr) {
    __shared__ __align__(16) float sh_y[BN * D];
    __shared__ __align__(16) float sh_ya[METRIC == SILH_CANBERRA ? BN * D : 4];
    __shared__ float sh_w[BN];
    __shared__ float sh_z[BN];
    constexpr int NA = RowAbs<METRIC, D, RPT>::NA;
    float2 x[RPT][D / 2];
    float2 ax[RPT][NA];
    float zx[RPT];   // cosine: 0.5 for a zero row (distance 1 to everything)
    int own[RPT];
    double wown[RPT];
    RatioMin bmin[RPT];
    double wsep[RPT];   // sum of W_hat_j over clusters j > own (separation numerator)
    bool rslow[RPT];    // Canberra: the row has a tiny coordinate
    const float cscale = (METRIC == SILH_CANBERRA) ? canb_scale(crange) : 1.0f;
    // Canberra: some coordinate of the data is tiny at that scale (uniform); only
    // then are rows and columns checked and flagged pairs evaluated directly
    // (CHECK_TINY = false: the caller has established that no coordinate is)
    const bool tiny_data =
        METRIC == SILH_CANBERRA && CHECK_TINY && canb_tiny_data(crange, cscale);
    int any_slow = 0;
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        int64_t rr = r0 + threadIdx.x + r * kThreads;
        int64_t e = (rr < nrows) ? (rows ? rows[rr] : rr) : -1;
        rslow[r] = false;
        own[r] = -1;
        if (e >= 0 && e < n) {
            int l = labels[e];
            own[r] = (l >= 0 && l < k) ? l : -2;
        }
        float sc = 0.f;
#pragma unroll
        for (int c = 0; c < D; c += 2) {
            const bool ok = e >= 0 && e < n;
            const int c0 = canb_slot<METRIC>(c), c1 = canb_slot<METRIC>(c + 1);
            x[r][c / 2].x = (ok && c0 < d) ? to_f32<T>(X[e * ld + c0]) : 0.f;
            x[r][c / 2].y = (ok && c1 < d) ? to_f32<T>(X[e * ld + c1]) : 0.f;
            if (METRIC == SILH_CANBERRA) {
                if (tiny_data)
                    rslow[r] = rslow[r] || canb_is_tiny(x[r][c / 2].x, cscale) ||
                               canb_is_tiny(x[r][c / 2].y, cscale);
                x[r][c / 2].x *= cscale;
                x[r][c / 2].y *= cscale;
            }
            sc = fmaf(x[r][c / 2].x, x[r][c / 2].x, sc);
            sc = fmaf(x[r][c / 2].y, x[r][c / 2].y, sc);
        }
        zx[r] = 0.f;
        if (METRIC == SILH_COSINE) {
            float inv = sc > 0.f ? rsqrtf(sc) : 0.f;
            zx[r] = sc > 0.f ? 0.f : 0.5f;
#pragma unroll
            for (int c = 0; c < D / 2; ++c) {
                x[r][c].x *= inv;
                x[r][c].y *= inv;
            }
        }
#pragma unroll
        for (int c = 0; c < NA; ++c)
            ax[r][c] = make_float2(fabsf(x[r][c].x), fabsf(x[r][c].y));
        wown[r] = 0.0;
        bmin[r] = RatioMin();
        wsep[r] = 0.0;
        any_slow |= rslow[r] ? 1 : 0;
    }
    // Canberra: whether any row of the CTA has a tiny coordinate (uniform)
    if (tiny_data) any_slow = __syncthreads_or(any_slow);
    for (int j = 0; j < k; ++j) {
        int64_t cs = offsets[j], ce = offsets[j + 1];
        double accd[RPT];
#pragma unroll
        for (int r = 0; r < RPT; ++r) accd[r] = 0.0;
        for (int64_t cb = cs; cb < ce; cb += BN) {
            int nb = (int)min((int64_t)BN, ce - cb);
            __syncthreads();
            stage_columns<METRIC>(reinterpret_cast<const float4 *>(Y + cb * D), nb * (D / 4), sh_y,
                                  sh_ya, threadIdx.x, kThreads, cscale);
            int chunk_slow = 0;
            for (int q = threadIdx.x; q < BN; q += kThreads) {
                sh_w[q] = (q < nb) ? wY[cb + q] : 0.f;
                // cosine: the zero-column term; Canberra: the tiny-column flag
                if (METRIC == SILH_COSINE) sh_z[q] = (q < nb) ? zY[cb + q] : 0.f;
                if (tiny_data && q < nb && zY[cb + q] != 0.f) chunk_slow = 1;
            }
            if (tiny_data) chunk_slow = __syncthreads_or(chunk_slow | any_slow);
            else __syncthreads();
            float accf[RPT];
            float accz = 0.f, accw = 0.f;
#pragma unroll
            for (int r = 0; r < RPT; ++r) accf[r] = 0.f;
            if (METRIC == SILH_CANBERRA && chunk_slow) {
                // a tiny row or column in the CTA's rows or this chunk: every
                // pair of the chunk term by term from the unscaled coordinates
                for (int col = 0; col < nb; ++col) {
                    const float w = sh_w[col];
#pragma unroll
                    for (int r = 0; r < RPT; ++r) {
                        const int64_t rr = r0 + threadIdx.x + r * kThreads;
                        const int64_t e = (rr < nrows) ? (rows ? rows[rr] : rr) : -1;
                        const float dd = (e >= 0 && e < n)
                                             ? canb_direct<T>(X + e * ld, Y + (cb + col) * D, d)
                                             : 0.f;
                        accf[r] = fmaf(w, dd, accf[r]);
                    }
                }
            } else {
                for (int col = 0; col < nb; ++col) {
                    const float4 *y4 = reinterpret_cast<const float4 *>(sh_y + col * D);
                    const float4 *ya4 = reinterpret_cast<const float4 *>(sh_ya + col * D);
                    float w = sh_w[col];
                    if (METRIC == SILH_COSINE) {
                        accz += sh_z[col];
                        accw += w;
                    }
#pragma unroll
                    for (int r = 0; r < RPT; ++r)
                        accf[r] = fmaf(w, pair_dist<METRIC, D, NA>(x[r], ax[r], y4, ya4), accf[r]);
                }
            }
#pragma unroll
            for (int r = 0; r < RPT; ++r) {
                if (METRIC == SILH_COSINE) accf[r] += accz + zx[r] * accw;
                accd[r] += (double)accf[r];
            }
        }
        double csz = (double)sizes[j];
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            if (j == own[r]) wown[r] = accd[r];
            else bmin[r].add(accd[r], csz, j);
            if (j > own[r]) wsep[r] += accd[r];
        }
    }
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        int64_t rr = r0 + threadIdx.x + r * kThreads;
        if (rr >= nrows) continue;
        float sv, av, bv;
        if (own[r] < 0) {
            sv = av = bv = NAN;
        } else {
            int64_t nc = sizes[own[r]];
            double a = (nc > 1) ? wown[r] / (double)(nc - 1) : 0.0;
            double b = bmin[r].value();
            double mx = fmax(a, b);
            double s = (nc > 1 && mx > 0.0) ? (b - a) / mx : 0.0;
            sv = (float)s; av = (float)a; bv = (float)b;
        }
        if (s_out) s_out[rr] = sv;
        if (a_out) a_out[rr] = av;
        if (b_out) b_out[rr] = bv;
        if (nb_out) nb_out[rr] = (own[r] < 0) ? -1 : bmin[r].arg;
        if (wown_out) wown_out[rr] = (own[r] >= 0) ? wown[r] : 0.0;
        if (wsep_out) wsep_out[rr] = (own[r] >= 0) ? wsep[r] : 0.0;
    }
}

// Per-row own-cluster and separation sums for Coh/Sep (all rows, in order).
template <class T, int METRIC, int D, int RPT, int BN>
__global__ void __launch_bounds__(kThreads)
k_sweep_cohsep(const T *__restrict__ X, int d, int64_t ld, int64_t n,
               const int32_t *__restrict__ labels, int k, const int64_t *__restrict__ sizes,
               const int64_t *__restrict__ offsets, const float *__restrict__ Y,
               const float *__restrict__ wY, const float *__restrict__ zY,
               const unsigned *__restrict__ crange, double *__restrict__ wown,
               double *__restrict__ wsep) {
    sweep_rows<T, METRIC, D, RPT, BN>((int64_t)blockIdx.x * kThreads * RPT, X, d, ld, n, labels, k,
                                      sizes, offsets, Y, wY, zY, crange, nullptr, n, nullptr,
                                      nullptr, nullptr, nullptr, wown, wsep);
}

// Coh = (1/2) sum wown / sum_j C(|Cj|,2), Sep = sum wsep / sum_{j1<j2} |Cj1||Cj2|
// (single block, fixed reduction order).
__global__ void k_cohsep_final(const double *__restrict__ wown, const double *__restrict__ wsep,
                               int64_t n, const int64_t *__restrict__ sizes, int k,
                               double *__restrict__ out) {
    __shared__ double sh[3][256];
    double a = 0.0, b = 0.0, c = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += 256) {
        a += wown[i];
        b += wsep[i];
    }
    for (int j = threadIdx.x; j < k; j += 256) c += (double)sizes[j];
    sh[0][threadIdx.x] = a;
    sh[1][threadIdx.x] = b;
    sh[2][threadIdx.x] = c;
    __syncthreads();
    for (int off = 128; off > 0; off >>= 1) {
        if (threadIdx.x < off)
            for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double pairs_in = 0.0, sq = 0.0;
        for (int j = 0; j < k; ++j) {
            const double s = (double)sizes[j];
            pairs_in += 0.5 * s * (s - 1.0);
            sq += s * s;
        }
        const double tot = sh[2][0];
        const double pairs_out = 0.5 * (tot * tot - sq);          // sum_{j1<j2} |Cj1||Cj2|
        out[0] = pairs_in > 0.0 ? 0.5 * sh[0][0] / pairs_in : 0.0;
        out[1] = pairs_out > 0.0 ? sh[1][0] / pairs_out : 0.0;
    }
}

// TINY selects the instantiation for Canberra data with (true) or without
// (false) tiny coordinates; both are launched, and the one that does not match
// the data (read from crange) returns at once, so the common case runs a
// kernel without the direct-evaluation path.  Other metrics: TINY = false.
template <class T, int METRIC, int D, int RPT, int BN, bool TINY>
__global__ void __launch_bounds__(kThreads)
k_sweep(const T *__restrict__ X, int d, int64_t ld, int64_t n, const int32_t *__restrict__ labels,
        int k, const int64_t *__restrict__ sizes, const int64_t *__restrict__ offsets,
        const float *__restrict__ Y, const float *__restrict__ wY, const float *__restrict__ zY,
        const unsigned *__restrict__ crange, const int64_t *__restrict__ rows, int64_t nrows,
        float *__restrict__ s_out, float *__restrict__ a_out, float *__restrict__ b_out,
        int32_t *__restrict__ nb_out) {
    if (METRIC == SILH_CANBERRA && canb_tiny_data(crange, canb_scale(crange)) != TINY) return;
    sweep_rows<T, METRIC, D, RPT, BN, TINY>((int64_t)blockIdx.x * kThreads * RPT, X, d, ld, n, labels, k,
                                      sizes, offsets, Y, wY, zY, crange, rows, nrows, s_out, a_out,
                                      b_out, nb_out);
}

template <class T, int METRIC>
void launch_cohsep_d(int D, cudaStream_t stream, const T *X, int d, int64_t ld, int64_t n,
                     const int32_t *labels, int k, const int64_t *sizes, const int64_t *offsets,
                     const float *Y, const float *wY, const float *zY, const unsigned *crange,
                     double *wown, double *wsep) {
    const int grid1 = (int)((n + kThreads - 1) / kThreads), grid2 = (int)((n + 2 * kThreads - 1) / (2 * kThreads));
    switch (D) {
        case 8: k_sweep_cohsep<T, METRIC, 8, 2, 64><<<grid2, kThreads, 0, stream>>>(X, d, ld, n, labels, k, sizes, offsets, Y, wY, zY, crange, wown, wsep); break;
        case 16: k_sweep_cohsep<T, METRIC, 16, 2, 64><<<grid2, kThreads, 0, stream>>>(X, d, ld, n, labels, k, sizes, offsets, Y, wY, zY, crange, wown, wsep); break;
        case 32: k_sweep_cohsep<T, METRIC, 32, 2, 64><<<grid2, kThreads, 0, stream>>>(X, d, ld, n, labels, k, sizes, offsets, Y, wY, zY, crange, wown, wsep); break;
        case 64: k_sweep_cohsep<T, METRIC, 64, 1, 32><<<grid1, kThreads, 0, stream>>>(X, d, ld, n, labels, k, sizes, offsets, Y, wY, zY, crange, wown, wsep); break;
        default: k_sweep_cohsep<T, METRIC, 128, 1, 32><<<grid1, kThreads, 0, stream>>>(X, d, ld, n, labels, k, sizes, offsets, Y, wY, zY, crange, wown, wsep); break;
    }
    count_launches(1);
}

// ------------------------------------------------------------ batched

// Many clusterings of one dataset in one persistent launch: item c has its own
// labels, cluster sizes, sample offsets (relative to its block of the
// concatenated column operand, starting at col_base) and output.  Work item w
// is (item, row tile); CTAs claim work items from a global counter, items in
// decreasing order of their column count (longest tiles first).
struct BatchItem {
    const int32_t *labels;
    const int64_t *sizes;
    const int64_t *offsets;
    const int32_t *idx;
    const double *p;
    float *s_out;
    int64_t col_base;
    int64_t m;
    int64_t tile_base;
    int32_t k;
    int32_t pad_;
};

constexpr int kMaxBatch = 256;

struct BatchParams {
    int32_t nitems;
    int64_t total_tiles;
    int64_t total_cols;
    BatchItem items[kMaxBatch];
};

template <class T, int METRIC, int D, int RPT, int BN>
__global__ void __launch_bounds__(kThreads)
k_sweep_batched(const __grid_constant__ BatchParams bp, const T *__restrict__ X, int d, int64_t ld,
                int64_t n, const float *__restrict__ Y, const float *__restrict__ wY,
                const float *__restrict__ zY, const unsigned *__restrict__ crange,
                unsigned long long *__restrict__ next_work) {
    __shared__ int64_t sh_work;
    for (;;) {
        // dynamic schedule: claim the next work item (items are ordered by cost, largest first)
        __syncthreads();
        if (threadIdx.x == 0) sh_work = (int64_t)atomicAdd(next_work, 1ull);
        __syncthreads();
        const int64_t w = sh_work;
        if (w >= bp.total_tiles) break;
        int lo = 0, hi = bp.nitems - 1;          // last item with tile_base <= w
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (bp.items[mid].tile_base <= w) lo = mid; else hi = mid - 1;
        }
        const BatchItem &it = bp.items[lo];
        const int64_t rt = w - it.tile_base;
        sweep_rows<T, METRIC, D, RPT, BN>(rt * kThreads * RPT, X, d, ld, n, it.labels, it.k,
                                          it.sizes, it.offsets, Y + it.col_base * D,
                                          wY + it.col_base, zY + it.col_base, crange, nullptr, n,
                                          it.s_out, nullptr, nullptr, nullptr);
    }
}

// Concatenated column operand of all items (one warp per column).
template <class T>
__global__ void k_gather_batched(const __grid_constant__ BatchParams bp, const T *__restrict__ X,
                                 int d, int64_t ld, int D, int metric,
                                 const unsigned *__restrict__ crange, float *__restrict__ Y,
                                 float *__restrict__ wY, float *__restrict__ zY) {
    const int64_t g = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (g >= bp.total_cols) return;
    int lo = 0, hi = bp.nitems - 1;              // last item with col_base <= g
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (bp.items[mid].col_base <= g) lo = mid; else hi = mid - 1;
    }
    const BatchItem &it = bp.items[lo];
    const int64_t i = g - it.col_base;
    const T *x = X + (int64_t)it.idx[i] * ld;
    float scale = 1.0f;
    if (metric == SILH_COSINE) {
        float sq = 0.f;
        for (int c = lane; c < d; c += 32) {
            const float v = to_f32<T>(x[c]);
            sq = fmaf(v, v, sq);
        }
        for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
        scale = sq > 0.f ? rsqrtf(sq) : 0.0f;
    }
    const float cs = (metric == SILH_CANBERRA) ? canb_scale(crange) : 1.0f;
    bool tiny = false;
    for (int c = lane; c < D; c += 32) {
        const float v = (c < d) ? to_f32<T>(x[c]) : 0.0f;
        if (metric == SILH_CANBERRA) tiny = tiny || canb_is_tiny(v, cs);
        Y[g * D + c] = v * scale;
    }
    tiny = __any_sync(0xffffffffu, tiny);
    if (lane == 0) {
        const float w = (float)(1.0 / it.p[i]);
        wY[g] = w;
        zY[g] = (metric == SILH_COSINE && scale == 0.0f) ? 0.5f * w : (tiny ? 1.0f : 0.0f);
    }
}

template <class T, int METRIC, int D, int RPT, int BN>
cudaError_t launch_batched_v(const BatchParams &bp, cudaStream_t stream, const T *X, int d,
                             int64_t ld, int64_t n, const float *Y, const float *wY,
                             const float *zY, const unsigned *crange,
                             unsigned long long *next_work) {
    auto kern = k_sweep_batched<T, METRIC, D, RPT, BN>;
    int dev = 0, nsm = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, 0);
    if (e != cudaSuccess) return e;
    const int64_t grid = std::min<int64_t>(bp.total_tiles, (int64_t)nsm * std::max(per_sm, 1));
    e = cudaMemsetAsync(next_work, 0, sizeof(unsigned long long), stream);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)std::max<int64_t>(grid, 1), kThreads, 0, stream>>>(bp, X, d, ld, n, Y, wY, zY,
                                                                       crange, next_work);
    count_launches(1);
    return cudaGetLastError();
}

// Tile-shape variants the autotuner chooses from: (rows per thread, columns per stage).
constexpr int kBatchVariants = 4;

template <class T, int METRIC, int D>
cudaError_t launch_batched(int variant, const BatchParams &bp, cudaStream_t stream, const T *X,
                           int d, int64_t ld, int64_t n, const float *Y, const float *wY,
                           const float *zY, const unsigned *crange, unsigned long long *nw) {
    // default: as the single sweep, (2, 128) for rows of up to 32 elements, else
    // (1, 64), or (1, 32) for Canberra rows of 128
    if (variant < 0) variant = (D <= 32) ? 3 : (D == 64 || METRIC != SILH_CANBERRA) ? 1 : 0;
    switch (variant) {
        case 0: return launch_batched_v<T, METRIC, D, 1, 32>(bp, stream, X, d, ld, n, Y, wY, zY, crange, nw);
        case 1:   // Canberra rows of 128 keep 32 columns (two staged copies in 48 KB)
            return launch_batched_v<T, METRIC, D, 1, (D >= 128 && METRIC == SILH_CANBERRA) ? 32 : 64>(
                bp, stream, X, d, ld, n, Y, wY, zY, crange, nw);
        case 2: return launch_batched_v<T, METRIC, D, 2, 32>(bp, stream, X, d, ld, n, Y, wY, zY, crange, nw);
        default: return launch_batched_v<T, METRIC, D, 2, (D <= 32 ? 128 : D >= 128 ? 32 : 64)>(
            bp, stream, X, d, ld, n, Y, wY, zY, crange, nw);
    }
}

template <class T, int METRIC>
cudaError_t launch_batched_d(int D, int variant, const BatchParams &bp, cudaStream_t stream,
                             const T *X, int d, int64_t ld, int64_t n, const float *Y,
                             const float *wY, const float *zY, const unsigned *crange, unsigned long long *nw) {
    switch (D) {
        case 8: return launch_batched<T, METRIC, 8>(variant, bp, stream, X, d, ld, n, Y, wY, zY, crange, nw);
        case 16: return launch_batched<T, METRIC, 16>(variant, bp, stream, X, d, ld, n, Y, wY, zY, crange, nw);
        case 32: return launch_batched<T, METRIC, 32>(variant, bp, stream, X, d, ld, n, Y, wY, zY, crange, nw);
        case 64: return launch_batched<T, METRIC, 64>(variant, bp, stream, X, d, ld, n, Y, wY, zY, crange, nw);
        default: return launch_batched<T, METRIC, 128>(variant, bp, stream, X, d, ld, n, Y, wY, zY, crange, nw);
    }
}

template <class T>
cudaError_t launch_batched_m(int metric, int D, int variant, const BatchParams &bp,
                             cudaStream_t stream, const T *X, int d, int64_t ld, int64_t n,
                             const float *Y, const float *wY, const float *zY,
                             const unsigned *crange, unsigned long long *nw) {
    switch (metric) {
        case SILH_EUCLIDEAN:
            return launch_batched_d<T, SILH_EUCLIDEAN>(D, variant, bp, stream, X, d, ld, n, Y, wY, zY, crange, nw);
        case SILH_COSINE:
            return launch_batched_d<T, SILH_COSINE>(D, variant, bp, stream, X, d, ld, n, Y, wY, zY, crange, nw);
        case SILH_MANHATTAN:
            return launch_batched_d<T, SILH_MANHATTAN>(D, variant, bp, stream, X, d, ld, n, Y, wY, zY, crange, nw);
        default:
            return launch_batched_d<T, SILH_CANBERRA>(D, variant, bp, stream, X, d, ld, n, Y, wY, zY, crange, nw);
    }
}

template <class T, int METRIC, int D>
void launch_sweep(cudaStream_t stream, const T *X, int d, int64_t ld, int64_t n,
                  const int32_t *labels, int k, const int64_t *sizes, const int64_t *offsets,
                  const float *Y, const float *wY, const float *zY, const unsigned *crange,
                  const int64_t *rows, int64_t nrows, float *s, float *a, float *b,
                  int32_t *nb) {
    constexpr int RPT = (D <= 32) ? 2 : 1;
    constexpr int BN = (D <= 32) ? 128 : (D == 64 || METRIC != SILH_CANBERRA) ? 64 : 32;
    int grid = (int)((nrows + kThreads * RPT - 1) / (kThreads * RPT));
    k_sweep<T, METRIC, D, RPT, BN, false><<<grid, kThreads, 0, stream>>>(
        X, d, ld, n, labels, k, sizes, offsets, Y, wY, zY, crange, rows, nrows, s, a, b, nb);
    count_launches(1);
    if (METRIC == SILH_CANBERRA) {
        k_sweep<T, METRIC, D, RPT, BN, METRIC == SILH_CANBERRA><<<grid, kThreads, 0, stream>>>(
            X, d, ld, n, labels, k, sizes, offsets, Y, wY, zY, crange, rows, nrows, s, a, b, nb);
        count_launches(1);
    }
}

template <class T, int METRIC>
void launch_sweep_d(int D, cudaStream_t stream, const T *X, int d, int64_t ld, int64_t n,
                    const int32_t *labels, int k, const int64_t *sizes, const int64_t *offsets,
                    const float *Y, const float *wY, const float *zY, const unsigned *crange,
                    const int64_t *rows, int64_t nrows, float *s, float *a, float *b,
                    int32_t *nb) {
#define SILH_SWEEP_D(DD)                                                                      \
    case DD:                                                                                  \
        launch_sweep<T, METRIC, DD>(stream, X, d, ld, n, labels, k, sizes, offsets, Y, wY, zY, \
                                    crange, rows, nrows, s, a, b, nb);                      \
        break;
    switch (D) {
        SILH_SWEEP_D(8)
        SILH_SWEEP_D(16)
        SILH_SWEEP_D(32)
        SILH_SWEEP_D(64)
        SILH_SWEEP_D(128)
        default: break;
    }
#undef SILH_SWEEP_D
}

template <class T>
void launch_sweep_m(int metric, int D, cudaStream_t stream, const T *X, int d, int64_t ld,
                    int64_t n, const int32_t *labels, int k, const int64_t *sizes,
                    const int64_t *offsets, const float *Y, const float *wY, const float *zY,
                    const unsigned *crange, const int64_t *rows, int64_t nrows, float *s, float *a,
                    float *b, int32_t *nb) {
    switch (metric) {
        case SILH_EUCLIDEAN:
            launch_sweep_d<T, SILH_EUCLIDEAN>(D, stream, X, d, ld, n, labels, k, sizes, offsets,
                                              Y, wY, zY, crange, rows, nrows, s, a, b, nb);
            break;
        case SILH_COSINE:
            launch_sweep_d<T, SILH_COSINE>(D, stream, X, d, ld, n, labels, k, sizes, offsets, Y,
                                           wY, zY, crange, rows, nrows, s, a, b, nb);
            break;
        case SILH_MANHATTAN:
            launch_sweep_d<T, SILH_MANHATTAN>(D, stream, X, d, ld, n, labels, k, sizes, offsets,
                                              Y, wY, zY, crange, rows, nrows, s, a, b, nb);
            break;
        default:
            launch_sweep_d<T, SILH_CANBERRA>(D, stream, X, d, ld, n, labels, k, sizes, offsets,
                                             Y, wY, zY, crange, rows, nrows, s, a, b, nb);
            break;
    }
}


// ----------------------------------------------------- exact, symmetric

// Column tiles one block of the symmetric exact sweep takes in a row (the row
// tile's registers and running sums carry over from one to the next).
constexpr int64_t kSymSeg = 4;

// Whether the symmetric exact sweep takes a straight-line form for blocks of
// columns that continue the running cluster (32-element Manhattan and
// Canberra rows), and the CTAs per SM such an instance is held to (0: no
// bound, the compiler's own register choice).
template <int METRIC, int D>
constexpr bool kSymFast = D == 32 && (METRIC == SILH_MANHATTAN || METRIC == SILH_CANBERRA);
template <int METRIC, int D>
constexpr int kSymMinBlocks = !kSymFast<METRIC, D> ? 0 : (METRIC == SILH_CANBERRA ? 3 : 4);

// Exact silhouette over all n rows: d(x, y) = d(y, x), so each pair of
// cluster-sorted position tiles (I <= J) is evaluated once.  A CTA owns the
// T = 128 RPT positions of tile I as rows and streams a segment of up to
// kSymSeg tiles J >= I as columns: every distance is added to its row's sum
// for the column's cluster (registers, flushed at cluster changes) and, for
// I < J, to its column's sum for the row's cluster (reduced over the CTA's rows
// with warp shuffles and shared memory).  Both land in the n x k FP64 weight
// matrix W with atomic adds (so results are reproducible to rounding order,
// not bitwise).

template <int METRIC, int D, int RPT, bool TINY>
__global__ void __launch_bounds__(kThreads, kSymMinBlocks<METRIC, D>)
k_exact_sym(const float *__restrict__ Y, const float *__restrict__ zY,
            const int32_t *__restrict__ lab_s, int64_t n, int k, int64_t ntiles,
            const unsigned *__restrict__ crange, double *__restrict__ W) {
    constexpr int T = kThreads * RPT;
    // columns per stage (static shared memory under 48 KB; Canberra measured
    // faster with 64 at D = 32, the others with 128)
    constexpr int BN = (D <= 32 && METRIC != SILH_CANBERRA) ? 128 : (D >= 128) ? 32 : 64;
    constexpr int NW = kThreads / 32;
    __shared__ __align__(16) float sh_y[BN * D];
    __shared__ __align__(16) float sh_ya[METRIC == SILH_CANBERRA ? BN * D : 4];
    __shared__ float sh_z[BN];
    __shared__ int sh_lab[BN];
    __shared__ float sh_col[NW][BN];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // Row tile I and a segment of up to kSymSeg of its column tiles J >= I from
    // the linear block index: row tile i has ceil((ntiles - i) / kSymSeg)
    // segments, so the blocks before row tile I number F(ntiles) - F(ntiles - I)
    // with F(x) = sum_{m <= x} ceil(m / kSymSeg).
    const int64_t b = blockIdx.x;
    auto segs_upto = [](int64_t x) -> int64_t {
        const int64_t q = x / kSymSeg, r = x % kSymSeg;
        return kSymSeg * q * (q + 1) / 2 + r * (q + 1);
    };
    const int64_t ftot = segs_upto(ntiles);
    int64_t lo = 0, hi = ntiles - 1;   // largest I with F(ntiles) - F(ntiles - I) <= b
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (ftot - segs_upto(ntiles - mid) <= b) lo = mid; else hi = mid - 1;
    }
    const int64_t I = lo;
    const int64_t J_begin = I + (b - (ftot - segs_upto(ntiles - I))) * kSymSeg;
    const int64_t J_end = min(J_begin + kSymSeg, ntiles);
    constexpr int NA = RowAbs<METRIC, D, RPT>::NA;
    float2 x[RPT][D / 2];
    float2 ax[RPT][NA];
    int lp[RPT];
    float zx[RPT];
    int64_t prow[RPT];
    float rv[RPT];                     // 1 for a row of the input, 0 past n
    const float cscale = (METRIC == SILH_CANBERRA) ? canb_scale(crange) : 1.0f;
    // Canberra with some coordinate of the data tiny at that scale (the host
    // picks this instantiation from crange): rows and columns are checked and
    // flagged chunks evaluated directly
    constexpr bool tiny_data = METRIC == SILH_CANBERRA && TINY;
    int any_slow = 0;
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int64_t p = I * T + threadIdx.x + r * kThreads;
        prow[r] = p;
        rv[r] = p < n ? 1.f : 0.f;
        const bool v = p < n;
        lp[r] = v ? lab_s[p] : -1;
        zx[r] = (METRIC == SILH_COSINE && v) ? zY[p] : 0.f;
        if (tiny_data && v && zY[p] != 0.f) any_slow = 1;    // a tiny row
        // float4 loads of the padded row; Canberra's slot order (c0, c2, c1, c3)
        // pairs the loaded lanes (x, z) and (y, w)
#pragma unroll
        for (int q = 0; q < D / 4; ++q) {
            const float4 u = v ? reinterpret_cast<const float4 *>(Y + p * D)[q]
                               : make_float4(0.f, 0.f, 0.f, 0.f);
            if (METRIC == SILH_CANBERRA) {
                x[r][2 * q] = make_float2(u.x * cscale, u.z * cscale);
                x[r][2 * q + 1] = make_float2(u.y * cscale, u.w * cscale);
            } else {
                x[r][2 * q] = make_float2(u.x, u.y);
                x[r][2 * q + 1] = make_float2(u.z, u.w);
            }
        }
#pragma unroll
        for (int c = 0; c < NA; ++c) ax[r][c] = make_float2(fabsf(x[r][c].x), fabsf(x[r][c].y));
    }
    if (tiny_data) any_slow = __syncthreads_or(any_slow);
    const int64_t rlast = min(I * T + T, n) - 1;
    const int cI0 = lab_s[I * T], cI1 = lab_s[rlast];
    int cur = -1;                      // column cluster of the running row sums
    float accr[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) accr[r] = 0.f;
    for (int64_t J = J_begin; J < J_end; ++J) {
    const bool diag = (I == J);
    const int64_t c_begin = J * T, c_end = min(J * T + T, n);
    for (int64_t cb = c_begin; cb < c_end; cb += BN) {
        const int nb = (int)min((int64_t)BN, c_end - cb);
        __syncthreads();
        stage_columns<METRIC>(reinterpret_cast<const float4 *>(Y + cb * D), nb * (D / 4), sh_y,
                              sh_ya, threadIdx.x, kThreads, cscale);
        int chunk_slow = 0;
        for (int q = threadIdx.x; q < BN; q += kThreads) {
            sh_lab[q] = (q < nb) ? lab_s[cb + q] : -1;
            sh_z[q] = (METRIC == SILH_COSINE && q < nb) ? zY[cb + q] : 0.f;
            // Canberra: a column with a tiny coordinate
            if (tiny_data && q < nb && zY[cb + q] != 0.f) chunk_slow = 1;
        }
        if (tiny_data) chunk_slow = __syncthreads_or(chunk_slow | any_slow);
        else __syncthreads();
        // Canberra with a tiny row in the CTA or a tiny column in this chunk
        // takes the per-column branch, every pair term by term (canb_direct).
        const bool direct = METRIC == SILH_CANBERRA && chunk_slow;
        if (!diag && cI0 == cI1 && !direct) {
            // One row cluster: the column sums are reduced across the warp CB
            // columns at a time (transpose-reduce: 16 shuffles for 16 columns,
            // 9 for 8; Canberra's larger body takes 8 to stay in the
            // instruction cache -- measured: 16 is 22 % slower, 4 2 % slower).
            constexpr int CB = (METRIC == SILH_CANBERRA) ? 8 : 16;
            // A block of CB columns that all continue the running cluster
            // (columns are cluster-sorted: its first and last do) takes the
            // straight-line form, without the per-column cluster checks.
            for (int col0 = 0; col0 < nb; col0 += CB) {
                float cs[CB];
                const bool fast = kSymFast<METRIC, D> && col0 + CB <= nb && sh_lab[col0] == cur &&
                                  sh_lab[col0 + CB - 1] == cur;
                if (fast) {
#pragma unroll
                    for (int c = 0; c < CB; ++c) {
                        const float4 *y4 = reinterpret_cast<const float4 *>(sh_y + (col0 + c) * D);
                        const float4 *ya4 = reinterpret_cast<const float4 *>(sh_ya + (col0 + c) * D);
                        cs[c] = 0.f;
#pragma unroll
                        for (int r = 0; r < RPT; ++r) {
                            float dd = pair_dist<METRIC, D, NA>(x[r], ax[r], y4, ya4);
                            if (METRIC == SILH_COSINE) dd += zx[r] + sh_z[col0 + c];
                            accr[r] += dd;
                            cs[c] = fmaf(rv[r], dd, cs[c]);
                        }
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < CB; ++c) {
                        const int col = col0 + c;
                        cs[c] = 0.f;
                        if (col < nb) {
                            const int lq = sh_lab[col];
                            if (lq != cur) {
                                if (cur >= 0) {
#pragma unroll
                                    for (int r = 0; r < RPT; ++r)
                                        if (prow[r] < n)
                                            atomicAdd(&W[prow[r] * k + cur], (double)accr[r]);
                                }
#pragma unroll
                                for (int r = 0; r < RPT; ++r) accr[r] = 0.f;
                                cur = lq;
                            }
                            const float4 *y4 = reinterpret_cast<const float4 *>(sh_y + col * D);
                            const float4 *ya4 = reinterpret_cast<const float4 *>(sh_ya + col * D);
#pragma unroll
                            for (int r = 0; r < RPT; ++r) {
                                float dd = pair_dist<METRIC, D, NA>(x[r], ax[r], y4, ya4);
                                if (METRIC == SILH_COSINE) dd += zx[r] + sh_z[col];
                                accr[r] += dd;                  // flushed only for rows < n
                                cs[c] = fmaf(rv[r], dd, cs[c]); // rows past n add nothing
                            }
                        }
                    }
                }
                int mine = 0;
                const float tot = transpose_reduce<CB>(cs, lane, mine);
                if ((lane & (32 / CB - 1)) == 0 && col0 + mine < nb) sh_col[warp][col0 + mine] = tot;
            }
        } else {
            // Diagonal tile (row sums only), or rows of several clusters (a tile
            // at a cluster boundary): one column sum per row cluster.
            for (int col = 0; col < nb; ++col) {
                const int lq = sh_lab[col];
                if (lq != cur) {           // uniform: columns are cluster-sorted
                    if (cur >= 0) {
#pragma unroll
                        for (int r = 0; r < RPT; ++r)
                            if (prow[r] < n) atomicAdd(&W[prow[r] * k + cur], (double)accr[r]);
                    }
#pragma unroll
                    for (int r = 0; r < RPT; ++r) accr[r] = 0.f;
                    cur = lq;
                }
                const float4 *y4 = reinterpret_cast<const float4 *>(sh_y + col * D);
                const float4 *ya4 = reinterpret_cast<const float4 *>(sh_ya + col * D);
                float dr[RPT];
#pragma unroll
                for (int r = 0; r < RPT; ++r) {
                    float dd;
                    if (METRIC == SILH_CANBERRA && direct)
                        dd = prow[r] < n ? canb_direct<float>(Y + prow[r] * D, Y + (cb + col) * D, D)
                                         : 0.f;
                    else
                        dd = pair_dist<METRIC, D, NA>(x[r], ax[r], y4, ya4);
                    if (METRIC == SILH_COSINE) dd += zx[r] + sh_z[col];
                    dr[r] = (prow[r] < n) ? dd : 0.f;
                    accr[r] += dr[r];
                }
                if (!diag) {
                    for (int c = cI0; c <= cI1; ++c) {
                        float v = 0.f;
#pragma unroll
                        for (int r = 0; r < RPT; ++r) v += (lp[r] == c) ? dr[r] : 0.f;
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                        if (lane == 0 && v != 0.f) atomicAdd(&W[(cb + col) * k + c], (double)v);
                    }
                }
            }
        }
        if (!diag && cI0 == cI1 && !direct) {
            __syncthreads();
            for (int q = threadIdx.x; q < nb; q += kThreads) {
                float v = 0.f;
#pragma unroll
                for (int w = 0; w < NW; ++w) v += sh_col[w][q];
                atomicAdd(&W[(cb + q) * k + cI0], (double)v);
            }
        }
    }
    }
    if (cur >= 0) {
#pragma unroll
        for (int r = 0; r < RPT; ++r)
            if (prow[r] < n) atomicAdd(&W[prow[r] * k + cur], (double)accr[r]);
    }
}

// s, a, b of every sorted position from its row of W; written at the element's
// original index order[pos].
__global__ void k_exact_finalize(const double *__restrict__ W, const int32_t *__restrict__ lab_s,
                                 const int32_t *__restrict__ order, const int64_t *__restrict__ sizes,
                                 int64_t n, int k, float *__restrict__ s_out,
                                 float *__restrict__ a_out, float *__restrict__ b_out,
                                 int32_t *__restrict__ nb_out) {
    const int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= n) return;
    const int own = lab_s[pos];
    const double *w = W + pos * k;
    RatioMin bm;
    for (int j = 0; j < k; ++j)
        if (j != own) bm.add(w[j], (double)sizes[j], j);
    const double bmin = bm.value();
    const int64_t nc = sizes[own];
    const double a = (nc > 1) ? w[own] / (double)(nc - 1) : 0.0;
    const double mx = fmax(a, bmin);
    const int64_t o = order[pos];
    s_out[o] = (float)((nc > 1 && mx > 0.0) ? (bmin - a) / mx : 0.0);
    if (a_out) a_out[o] = (float)a;
    if (b_out) b_out[o] = (float)bmin;
    if (nb_out) nb_out[o] = bm.arg;
}

__global__ void k_sorted_labels(const int32_t *__restrict__ labels, const int32_t *__restrict__ order,
                                int64_t n, int32_t *__restrict__ lab_s) {
    const int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pos < n) lab_s[pos] = labels[order[pos]];
}

template <int METRIC, int D>
void launch_exact_sym(cudaStream_t stream, const float *Y, const float *zY, const int32_t *lab_s,
                      int64_t n, int k, const unsigned *crange, bool tiny, double *W) {
    constexpr int RPT = (D <= 32) ? 2 : 1;
    constexpr int T = kThreads * RPT;
    const int64_t nt = (n + T - 1) / T;
    const int64_t q = nt / kSymSeg, r = nt % kSymSeg;
    const int64_t nblk = kSymSeg * q * (q + 1) / 2 + r * (q + 1);   // row-tile segments
    if (METRIC == SILH_CANBERRA && tiny)
        k_exact_sym<METRIC, D, RPT, METRIC == SILH_CANBERRA><<<(unsigned)nblk, kThreads, 0, stream>>>(
            Y, zY, lab_s, n, k, nt, crange, W);
    else
        k_exact_sym<METRIC, D, RPT, false><<<(unsigned)nblk, kThreads, 0, stream>>>(
            Y, zY, lab_s, n, k, nt, crange, W);
    count_launches(1);
}

template <int METRIC>
void launch_exact_sym_d(int D, cudaStream_t stream, const float *Y, const float *zY,
                        const int32_t *lab_s, int64_t n, int k, const unsigned *crange, bool tiny,
                        double *W) {
    switch (D) {
        case 8: launch_exact_sym<METRIC, 8>(stream, Y, zY, lab_s, n, k, crange, tiny, W); break;
        case 16: launch_exact_sym<METRIC, 16>(stream, Y, zY, lab_s, n, k, crange, tiny, W); break;
        case 32: launch_exact_sym<METRIC, 32>(stream, Y, zY, lab_s, n, k, crange, tiny, W); break;
        case 64: launch_exact_sym<METRIC, 64>(stream, Y, zY, lab_s, n, k, crange, tiny, W); break;
        default: launch_exact_sym<METRIC, 128>(stream, Y, zY, lab_s, n, k, crange, tiny, W); break;
    }
}

// ------------------------------------------------------------- global

constexpr int kSumThreads = 256;

__global__ void k_sum_partial(const float *__restrict__ s, int64_t n, double *__restrict__ part) {
    __shared__ double sh[kSumThreads];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kSumThreads + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kSumThreads)
        acc += (double)s[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int off = kSumThreads / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_sum_final(const double *__restrict__ part, int np, int64_t n,
                            double *__restrict__ out) {
    __shared__ double sh[kSumThreads];
    double acc = 0.0;
    for (int i = threadIdx.x; i < np; i += kSumThreads) acc += part[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int off = kSumThreads / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0] / (double)n;
}

}  // namespace

silh_status canberra_range(const void *X, silh_dtype dtype, int64_t n, int32_t d, int64_t ld,
                           unsigned *range, cudaStream_t stream) {
    silh_status st = SILH_OK;
    int grid = ceil_div_i(std::max<int64_t>(n * (int64_t)d, 1), 256 * 8);
    grid = std::min(grid, 148 * 8);
    SILH_CK(cudaMemsetAsync(range, 0, sizeof(unsigned), stream));
    SILH_CK(cudaMemsetAsync(range + 1, 0x7F, sizeof(unsigned), stream));   // 0x7F7F7F7F
    if (dtype == SILH_F32)
        k_range<float><<<grid, 256, 0, stream>>>((const float *)X, n, d, ld, range);
    else
        k_range<__nv_bfloat16><<<grid, 256, 0, stream>>>((const __nv_bfloat16 *)X, n, d, ld, range);
    count_launches(1);
    SILH_CK(cudaGetLastError());
done:
    return st;
}

silh_status gather_columns(const void *X, silh_dtype dtype, int32_t d, int64_t ld,
                           const int32_t *idx, const double *p, int64_t m, int D, int metric,
                           const unsigned *crange, float *Y, float *wY, float *zY,
                           cudaStream_t stream, const int64_t *d_m) {
    silh_status st = SILH_OK;
    if (m > 0) {
        int grid = ceil_div_i(m, 8);
        if (dtype == SILH_F32)
            k_gather<float><<<grid, 256, 0, stream>>>((const float *)X, d, ld, idx, p, m, D,
                                                      metric, crange, Y, wY, zY, d_m);
        else
            k_gather<__nv_bfloat16><<<grid, 256, 0, stream>>>((const __nv_bfloat16 *)X, d, ld,
                                                              idx, p, m, D, metric, crange, Y, wY,
                                                              zY, d_m);
        count_launches(1);
    }
    SILH_CK(cudaGetLastError());
done:
    return st;
}

silh_status phase2_sweep(const void *X, silh_dtype dtype, int64_t n, int32_t d, int64_t ld,
                         const int32_t *labels, int32_t k, int metric, int prec,
                         const int64_t *sizes, const int64_t *offsets, const float *Y,
                         const float *wY, const float *zY, const unsigned *crange, int64_t m, int D,
                         const int64_t *rows, int64_t nrows, float *s, float *a, float *b,
                         int32_t *nb, cudaStream_t stream) {
    silh_status st = SILH_OK;
    (void)prec;
    (void)m;
    if (nrows > 0) {
        if (dtype == SILH_F32)
            launch_sweep_m<float>(metric, D, stream, (const float *)X, d, ld, n, labels, k, sizes,
                                  offsets, Y, wY, zY, crange, rows, nrows, s, a, b, nb);
        else
            launch_sweep_m<__nv_bfloat16>(metric, D, stream, (const __nv_bfloat16 *)X, d, ld, n,
                                          labels, k, sizes, offsets, Y, wY, zY, crange, rows, nrows,
                                          s, a, b, nb);
    }
    SILH_CK(cudaGetLastError());
done:
    return st;
}

}  // namespace silh

using namespace silh;

static silh_status check_data_args(const void *X, silh_dtype dtype, int64_t n, int32_t d,
                                   int64_t ld, const int32_t *labels, int32_t k,
                                   silh_metric metric, silh_prec prec) {
    if (!X || !labels) return fail(SILH_EINVAL, "null pointer argument");
    if (!device_accessible(X)) return fail(SILH_EINVAL, "X is not device-accessible memory");
    if (!device_accessible(labels)) return fail(SILH_EINVAL, "labels is not device-accessible memory");
    if (n < 2 || n >= (int64_t(1) << 31)) return fail(SILH_EINVAL, "n must be in [2, 2^31)");
    if (d < 1 || d > 128 || ld < d) return fail(SILH_EINVAL, "need 1 <= d <= 128 and ld >= d");
    if (k < 2 || k > SILH_MAX_K) return fail(SILH_EINVAL, "k must be in [2, %d]", SILH_MAX_K);
    if (metric < SILH_EUCLIDEAN || metric > SILH_CANBERRA) return fail(SILH_EINVAL, "unknown metric");
    if (dtype != SILH_F32 && dtype != SILH_BF16) return fail(SILH_EINVAL, "unknown dtype");
    if (prec < SILH_PREC_FP32 || prec > SILH_PREC_BF16X3) return fail(SILH_EINVAL, "unknown precision");
    return SILH_OK;
}

// Phase 2 for a sample of m columns (S->size), or, when d_m is given, of *d_m
// columns with m = S->cap bounding it (scratch sized for m; the kernels read
// the actual size from the device).
static silh_status estimate_impl(const void *X, silh_dtype dtype, int64_t n, int32_t d, int64_t ld,
                                 const int32_t *labels, int32_t k, silh_metric metric,
                                 silh_prec prec, const silh_sample *S, const int64_t *d_m,
                                 const int64_t *rows, int64_t nrows, float *s_hat, float *a_hat,
                                 float *b_hat, int32_t *nb, cudaStream_t stream) {
    silh_status st = check_data_args(X, dtype, n, d, ld, labels, k, metric, prec);
    if (st != SILH_OK) return st;
    int dev = 0;
    int D = padded_dim(d);
    Scratch sc(stream);
    float *Y = nullptr, *wY = nullptr, *zY = nullptr;
    unsigned *crange = nullptr;
    int64_t m = 0;
    SILH_REQ(S && S->k == k && S->sizes && S->offsets, "sample missing or k mismatch");
    m = d_m ? S->cap : S->size;
    SILH_REQ(m >= 0 && m <= S->cap && (m == 0 || (S->idx && S->p)), "bad sample size");
    SILH_REQ(s_hat, "s_hat is null");
    SILH_REQ(sample_accessible(S), "sample arrays are not device-accessible memory");
    SILH_DEVPTR(s_hat, "s_hat");
    SILH_DEVPTR_OPT(a_hat, "a_hat");
    SILH_DEVPTR_OPT(b_hat, "b_hat");
    SILH_DEVPTR_OPT(nb, "neighbour");
    SILH_DEVPTR_OPT(rows, "rows");
    SILH_DEVPTR_OPT(d_m, "d_size");
    if (rows == nullptr) nrows = n;
    SILH_REQ(nrows >= 0, "nrows < 0");
    SILH_CK(cudaGetDevice(&dev));
    ensure_pool_retains(dev);
    if (m > 0 && nrows > 0 && tc_eligible(metric, prec, d)) {
        // a cluster holds at most all m sampled columns
        st = tc_sweep(X, dtype, n, d, ld, labels, k, metric, prec, S->sizes, S->offsets, S->idx,
                      S->p, m, m, rows, nrows, s_hat, a_hat, b_hat, nb, sc, stream, d_m);
        goto done;
    }
    SILH_CK(sc.alloc(&Y, (size_t)m * D));
    SILH_CK(sc.alloc(&wY, (size_t)m));
    SILH_CK(sc.alloc(&zY, (size_t)m));
    if (metric == SILH_CANBERRA) {
        SILH_CK(sc.alloc(&crange, 2));
        st = canberra_range(X, dtype, n, d, ld, crange, stream);
        if (st != SILH_OK) goto done;
    }
    st = gather_columns(X, dtype, d, ld, S->idx, S->p, m, D, metric, crange, Y, wY, zY, stream,
                        d_m);
    if (st != SILH_OK) goto done;
    st = phase2_sweep(X, dtype, n, d, ld, labels, k, metric, prec, S->sizes, S->offsets, Y, wY, zY,
                      crange, m, D, rows, nrows, s_hat, a_hat, b_hat, nb, stream);
done:
    return st;
}

extern "C" silh_status silh_estimate(const void *X, silh_dtype dtype, int64_t n, int32_t d,
                                     int64_t ld, const int32_t *labels, int32_t k,
                                     silh_metric metric, silh_prec prec, const silh_sample *S,
                                     const int64_t *rows, int64_t nrows, float *s_hat,
                                     float *a_hat, float *b_hat, int32_t *nb, void *stream_) {
    return estimate_impl(X, dtype, n, d, ld, labels, k, metric, prec, S, nullptr, rows, nrows,
                         s_hat, a_hat, b_hat, nb, (cudaStream_t)stream_);
}

extern "C" silh_status silh_estimate_async(const void *X, silh_dtype dtype, int64_t n, int32_t d,
                                           int64_t ld, const int32_t *labels, int32_t k,
                                           silh_metric metric, silh_prec prec,
                                           const silh_sample *S, const int64_t *d_size,
                                           const int64_t *rows, int64_t nrows, float *s_hat,
                                           float *a_hat, float *b_hat, int32_t *nb,
                                           void *stream_) {
    if (d_size == nullptr) return fail(SILH_EINVAL, "d_size is null");
    return estimate_impl(X, dtype, n, d, ld, labels, k, metric, prec, S, d_size, rows, nrows,
                         s_hat, a_hat, b_hat, nb, (cudaStream_t)stream_);
}

extern "C" silh_status silh_exact(const void *X, silh_dtype dtype, int64_t n, int32_t d,
                                  int64_t ld, const int32_t *labels, int32_t k, silh_metric metric,
                                  silh_prec prec, const int64_t *rows, int64_t nrows, float *s,
                                  float *a, float *b, int32_t *nb, void *stream_) {
    cudaStream_t stream = (cudaStream_t)stream_;
    silh_status st = check_data_args(X, dtype, n, d, ld, labels, k, metric, prec);
    if (st != SILH_OK) return st;
    int dev = 0;
    int D = padded_dim(d);
    Scratch sc(stream);
    std::vector<int64_t> h_sizes, h_coff;
    int64_t *sizes = nullptr, *coff = nullptr;
    int32_t *order = nullptr, *lab_s = nullptr;
    double *W = nullptr;
    unsigned *crange = nullptr;
    unsigned h_range[2] = {0u, 0u};
    bool tiny = false;
    float *Y = nullptr, *wY = nullptr, *zY = nullptr;
    SILH_REQ(s, "s is null");
    SILH_DEVPTR(s, "s");
    SILH_DEVPTR_OPT(a, "a");
    SILH_DEVPTR_OPT(b, "b");
    SILH_DEVPTR_OPT(nb, "neighbour");
    SILH_DEVPTR_OPT(rows, "rows");
    if (rows == nullptr) nrows = n;
    SILH_REQ(nrows >= 0, "nrows < 0");
    SILH_CK(cudaGetDevice(&dev));
    ensure_pool_retains(dev);
    SILH_CK(sc.alloc(&sizes, (size_t)k));
    if (metric == SILH_CANBERRA) {
        // the data range, read back under cluster_sort's synchronisation
        SILH_CK(sc.alloc(&crange, 2));
        st = canberra_range(X, dtype, n, d, ld, crange, stream);
        if (st != SILH_OK) goto done;
        SILH_CK(cudaMemcpyAsync(h_range, crange, sizeof(h_range), cudaMemcpyDeviceToHost, stream));
    }
    st = cluster_sort(labels, n, k, sc, stream, sizes, &coff, &order, h_sizes, h_coff);
    if (st != SILH_OK) goto done;
    tiny = metric == SILH_CANBERRA && canb_tiny_of(h_range[1], canb_scale_of(h_range[0]));
    if (nrows > 0 && tc_eligible(metric, prec, d)) {
        const int64_t maxc = *std::max_element(h_sizes.begin(), h_sizes.end());
        if (rows == nullptr &&
            (double)(n + 31.0 * k) * (double)k * 8.0 <= 4294967296.0) {
            // all points: each pair once, row and column sums into an FP64 matrix
            st = tc_exact_sym(X, dtype, n, d, ld, k, metric, prec, sizes, coff, order, h_sizes, s,
                              a, b, nb, sc, stream);
        } else {
            st = tc_sweep(X, dtype, n, d, ld, labels, k, metric, prec, sizes, coff, order, nullptr,
                          n, maxc, rows, nrows, s, a, b, nb, sc, stream);
        }
        goto done;
    }
    SILH_CK(sc.alloc(&Y, (size_t)n * D));
    SILH_CK(sc.alloc(&wY, (size_t)n));
    SILH_CK(sc.alloc(&zY, (size_t)n));
    st = gather_columns(X, dtype, d, ld, order, nullptr, n, D, metric, crange, Y, wY, zY, stream);
    if (st != SILH_OK) goto done;
    if (rows == nullptr && (double)n * (double)k * 8.0 <= 2147483648.0) {
        // all rows: the symmetric sweep evaluates each pair once
        SILH_CK(sc.alloc(&lab_s, (size_t)n));
        SILH_CK(sc.alloc(&W, (size_t)n * k));
        SILH_CK(cudaMemsetAsync(W, 0, sizeof(double) * (size_t)n * k, stream));
        k_sorted_labels<<<ceil_div_i(n, 256), 256, 0, stream>>>(labels, order, n, lab_s);
        count_launches(1);
        switch (metric) {
            case SILH_EUCLIDEAN: launch_exact_sym_d<SILH_EUCLIDEAN>(D, stream, Y, zY, lab_s, n, k, crange, tiny, W); break;
            case SILH_COSINE: launch_exact_sym_d<SILH_COSINE>(D, stream, Y, zY, lab_s, n, k, crange, tiny, W); break;
            case SILH_MANHATTAN: launch_exact_sym_d<SILH_MANHATTAN>(D, stream, Y, zY, lab_s, n, k, crange, tiny, W); break;
            default: launch_exact_sym_d<SILH_CANBERRA>(D, stream, Y, zY, lab_s, n, k, crange, tiny, W); break;
        }
        k_exact_finalize<<<ceil_div_i(n, 256), 256, 0, stream>>>(W, lab_s, order, sizes, n, k, s, a,
                                                                 b, nb);
        count_launches(1);
        SILH_CK(cudaGetLastError());
        goto done;
    }
    st = phase2_sweep(X, dtype, n, d, ld, labels, k, metric, prec, sizes, coff, Y, wY, zY, crange, n,
                      D, rows, nrows, s, a, b, nb, stream);
done:
    return st;
}

extern "C" silh_status silh_estimate_batched(const void *X, silh_dtype dtype, int64_t n,
                                             int32_t d, int64_t ld, silh_metric metric,
                                             silh_prec prec, int32_t nitems,
                                             const silh_batch_item *items, int32_t variant,
                                             void *stream_) {
    cudaStream_t stream = (cudaStream_t)stream_;
    silh_status st = SILH_OK;
    const int D = padded_dim(d);
    Scratch sc(stream);
    float *Y = nullptr, *wY = nullptr, *zY = nullptr;
    unsigned long long *next_work = nullptr;
    unsigned *crange = nullptr;
    std::vector<BatchParams> parts;
    std::vector<int32_t> order;
    SILH_REQ(X && items, "null pointer argument");
    SILH_DEVPTR(X, "X");
    SILH_REQ(n >= 2 && n < (int64_t(1) << 31), "n must be in [2, 2^31)");
    SILH_REQ(d >= 1 && d <= 128 && ld >= d, "need 1 <= d <= 128 and ld >= d");
    SILH_REQ(metric >= SILH_EUCLIDEAN && metric <= SILH_CANBERRA, "unknown metric");
    SILH_REQ(dtype == SILH_F32 || dtype == SILH_BF16, "unknown dtype");
    SILH_REQ(prec >= SILH_PREC_FP32 && prec <= SILH_PREC_BF16X3, "unknown precision");
    SILH_REQ(nitems >= 1, "need at least one item");
    SILH_REQ(variant >= -1 && variant < kBatchVariants, "variant must be -1 .. %d",
             kBatchVariants - 1);
    // largest items first (longest row tiles), then kMaxBatch per launch as launch parameters
    for (int32_t i = 0; i < nitems; ++i) {
        SILH_REQ(items[i].sample, "item %d: null sample", i);
        order.push_back(i);
    }
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        return items[a].sample->size > items[b].sample->size;
    });
    for (int32_t c0 = 0; c0 < nitems; c0 += kMaxBatch) {
        parts.emplace_back();
        BatchParams &b = parts.back();
        std::memset(&b, 0, sizeof(b));
        b.nitems = std::min<int32_t>(kMaxBatch, nitems - c0);
        int64_t tiles = 0, cols = 0;
        const int64_t bm = kThreads * ((variant < 0 ? (D <= 32 ? 3 : 0) : variant) >= 2 ? 2 : 1);
        for (int i = 0; i < b.nitems; ++i) {
            const silh_batch_item &src = items[order[c0 + i]];
            SILH_REQ(src.labels && src.s_hat && src.sample, "item %d: null pointer", c0 + i);
            const silh_sample *S = src.sample;
            SILH_REQ(S->k >= 2 && S->k <= SILH_MAX_K && S->sizes && S->offsets,
                     "item %d: bad sample", c0 + i);
            SILH_REQ(S->size >= 1 && S->size <= S->cap && S->idx && S->p, "item %d: empty sample",
                     c0 + i);
            SILH_REQ(device_accessible(src.labels) && device_accessible(src.s_hat) &&
                         sample_accessible(S),
                     "item %d: buffers are not device-accessible memory", c0 + i);
            BatchItem &it = b.items[i];
            it.labels = src.labels;
            it.sizes = S->sizes;
            it.offsets = S->offsets;
            it.idx = S->idx;
            it.p = S->p;
            it.s_out = src.s_hat;
            it.k = S->k;
            it.col_base = cols;
            it.m = S->size;
            it.tile_base = tiles;
            cols += S->size;
            tiles += (n + bm - 1) / bm;
        }
        b.total_tiles = tiles;
        b.total_cols = cols;
    }
    if (tc_eligible(metric, prec, d)) {
        st = tc_sweep_batched(X, dtype, n, d, ld, metric, prec, items, order, variant, stream);
        goto done;
    }
    SILH_CK(sc.alloc(&next_work, 1));
    if (metric == SILH_CANBERRA) {
        SILH_CK(sc.alloc(&crange, 2));
        st = canberra_range(X, dtype, n, d, ld, crange, stream);
        if (st != SILH_OK) goto done;
    }
    for (BatchParams &b : parts) {
        SILH_CK(sc.alloc(&Y, (size_t)b.total_cols * D));
        SILH_CK(sc.alloc(&wY, (size_t)b.total_cols));
        SILH_CK(sc.alloc(&zY, (size_t)b.total_cols));
        if (dtype == SILH_F32) {
            k_gather_batched<float><<<ceil_div_i(b.total_cols, 8), 256, 0, stream>>>(
                b, (const float *)X, d, ld, D, metric, crange, Y, wY, zY);
            count_launches(1);
            SILH_CK(launch_batched_m<float>(metric, D, variant, b, stream, (const float *)X, d, ld,
                                            n, Y, wY, zY, crange, next_work));
        } else {
            k_gather_batched<__nv_bfloat16><<<ceil_div_i(b.total_cols, 8), 256, 0, stream>>>(
                b, (const __nv_bfloat16 *)X, d, ld, D, metric, crange, Y, wY, zY);
            count_launches(1);
            SILH_CK(launch_batched_m<__nv_bfloat16>(metric, D, variant, b, stream,
                                                    (const __nv_bfloat16 *)X, d, ld, n, Y, wY,
                                                    zY, crange, next_work));
        }
    }
done:
    return st;
}

extern "C" silh_status silh_cohsep(const void *X, silh_dtype dtype, int64_t n, int32_t d,
                                   int64_t ld, const int32_t *labels, int32_t k, silh_metric metric,
                                   const silh_sample *S, double *out, void *stream_) {
    cudaStream_t stream = (cudaStream_t)stream_;
    silh_status st = check_data_args(X, dtype, n, d, ld, labels, k, metric, SILH_PREC_FP32);
    if (st != SILH_OK) return st;
    const int D = padded_dim(d);
    Scratch sc(stream);
    float *Y = nullptr, *wY = nullptr, *zY = nullptr;
    double *wown = nullptr, *wsep = nullptr;
    unsigned *crange = nullptr;
    int64_t m = 0;
    SILH_REQ(S && S->k == k && S->sizes && S->offsets && out, "sample or output missing");
    m = S->size;
    SILH_REQ(m >= 0 && m <= S->cap && (m == 0 || (S->idx && S->p)), "bad sample size");
    SILH_REQ(sample_accessible(S), "sample arrays are not device-accessible memory");
    SILH_DEVPTR(out, "out");
    SILH_CK(sc.alloc(&Y, (size_t)m * D));
    SILH_CK(sc.alloc(&wY, (size_t)m));
    SILH_CK(sc.alloc(&zY, (size_t)m));
    SILH_CK(sc.alloc(&wown, (size_t)n));
    SILH_CK(sc.alloc(&wsep, (size_t)n));
    if (metric == SILH_CANBERRA) {
        SILH_CK(sc.alloc(&crange, 2));
        st = canberra_range(X, dtype, n, d, ld, crange, stream);
        if (st != SILH_OK) goto done;
    }
    st = gather_columns(X, dtype, d, ld, S->idx, S->p, m, D, metric, crange, Y, wY, zY, stream);
    if (st != SILH_OK) goto done;
    if (dtype == SILH_F32) {
        switch (metric) {
            case SILH_EUCLIDEAN: launch_cohsep_d<float, SILH_EUCLIDEAN>(D, stream, (const float *)X, d, ld, n, labels, k, S->sizes, S->offsets, Y, wY, zY, crange, wown, wsep); break;
            case SILH_COSINE: launch_cohsep_d<float, SILH_COSINE>(D, stream, (const float *)X, d, ld, n, labels, k, S->sizes, S->offsets, Y, wY, zY, crange, wown, wsep); break;
            case SILH_MANHATTAN: launch_cohsep_d<float, SILH_MANHATTAN>(D, stream, (const float *)X, d, ld, n, labels, k, S->sizes, S->offsets, Y, wY, zY, crange, wown, wsep); break;
            default: launch_cohsep_d<float, SILH_CANBERRA>(D, stream, (const float *)X, d, ld, n, labels, k, S->sizes, S->offsets, Y, wY, zY, crange, wown, wsep); break;
        }
    } else {
        const __nv_bfloat16 *Xb = (const __nv_bfloat16 *)X;
        switch (metric) {
            case SILH_EUCLIDEAN: launch_cohsep_d<__nv_bfloat16, SILH_EUCLIDEAN>(D, stream, Xb, d, ld, n, labels, k, S->sizes, S->offsets, Y, wY, zY, crange, wown, wsep); break;
            case SILH_COSINE: launch_cohsep_d<__nv_bfloat16, SILH_COSINE>(D, stream, Xb, d, ld, n, labels, k, S->sizes, S->offsets, Y, wY, zY, crange, wown, wsep); break;
            case SILH_MANHATTAN: launch_cohsep_d<__nv_bfloat16, SILH_MANHATTAN>(D, stream, Xb, d, ld, n, labels, k, S->sizes, S->offsets, Y, wY, zY, crange, wown, wsep); break;
            default: launch_cohsep_d<__nv_bfloat16, SILH_CANBERRA>(D, stream, Xb, d, ld, n, labels, k, S->sizes, S->offsets, Y, wY, zY, crange, wown, wsep); break;
        }
    }
    k_cohsep_final<<<1, 256, 0, stream>>>(wown, wsep, n, S->sizes, k, out);
    count_launches(1);
    SILH_CK(cudaGetLastError());
done:
    return st;
}

extern "C" silh_status silh_stream_status(void *stream_) {
    silh_status st = SILH_OK;
    int e = 0;
    SILH_CK(cudaStreamSynchronize((cudaStream_t)stream_));
    e = tc_take_error();
    if (e < 0) st = fail(SILH_ECUDA, "reading the device error word failed");
    else if (e > 0) st = fail(SILH_ETIMEOUT, "a bounded device wait gave up");
done:
    return st;
}

extern "C" silh_status silh_wait_selftest(int32_t arrive, uint64_t timeout_ns, void *stream_) {
    silh_status st = SILH_OK;
    SILH_REQ(timeout_ns >= 1000 && timeout_ns <= 1000000000ull,
             "timeout_ns must be in [1 us, 1 s]");
    st = tc_wait_selftest(arrive != 0, timeout_ns, (cudaStream_t)stream_);
done:
    return st;
}

extern "C" silh_status silh_global(const float *s, int64_t n, double *out, void *stream_) {
    cudaStream_t stream = (cudaStream_t)stream_;
    silh_status st = SILH_OK;
    Scratch sc(stream);
    double *part = nullptr;
    int np = 0;
    SILH_REQ(s && out, "null pointer argument");
    SILH_REQ(n >= 1, "n must be >= 1");
    SILH_DEVPTR(s, "s");
    SILH_DEVPTR(out, "out");
    np = (int)std::min<int64_t>(1024, (n + kSumThreads - 1) / kSumThreads);
    SILH_CK(sc.alloc(&part, np));
    k_sum_partial<<<np, kSumThreads, 0, stream>>>(s, n, part); count_launches(1);
    k_sum_final<<<1, kSumThreads, 0, stream>>>(part, np, n, out); count_launches(1);
    SILH_CK(cudaGetLastError());
done:
    return st;
}
