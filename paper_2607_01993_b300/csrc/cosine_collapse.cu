// Phase 2 of Algorithm 1 for the cosine distance in O(n k d) instead of
// O(n |S| d).
//
// With unit vectors, d_cos(x, y) = 1 - <x^, y^> = 0.5 |x^ - y^|^2, so the
// estimated weight of a cluster is a weighted sum of squared Euclidean
// distances to the cluster's sampled unit vectors.  The parallel-axis
// identity splits it exactly (in real arithmetic) into a per-row part and a
// per-cluster constant:
//   sum_{y in F_j} w_y |x^ - y^|^2 = S_j |x^ - mu_j|^2 + R_j,
//   S_j = sum w_y,  mu_j = sum w_y y^ / S_j,  R_j = sum w_y |y^ - mu_j|^2
// (sums over the non-zero sampled vectors; a zero vector is at distance 1 from
// everything and contributes its weight Z_j directly).  Unlike the expanded
// form S_j - <x^, sum w y^>, both terms are non-negative, so nothing cancels:
// the per-row arithmetic can stay FP32.  The result equals Eq. 8's per-pair
// estimate up to rounding; the per-pair sweep remains the primary path.
#include <cmath>

#include "kernels.cuh"

namespace silh {
namespace {

constexpr int kClThreads = 256;   // per-cluster reduction block
constexpr int kRowThreads = 128;

// Partial sums over one slice of a cluster's sample: grid (k, kSlices); the
// block (j, g) takes members b + g*NW + warp, stepping kSlices*NW, and writes
// (sum w y^ [D], S, Z) in FP64 to part[(j * kSlices + g) * (D + 2)].  Fixed
// order throughout (lanes over coordinates, warps combined in index order).
constexpr int kSlices = 16;

template <class T>
__global__ void __launch_bounds__(kClThreads)
k_collapse_partial(const T *__restrict__ X, int d, int64_t ld, const int64_t *__restrict__ offsets,
                   const int32_t *__restrict__ idx, const double *__restrict__ p, int D,
                   double *__restrict__ part) {
    constexpr int NW = kClThreads / 32;
    __shared__ double sh_v[NW][128];
    __shared__ double sh_s[NW], sh_z[NW];
    const int j = blockIdx.x, g = blockIdx.y, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t b = offsets[j], e = offsets[j + 1];
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    double s = 0.0, z = 0.0;
    for (int64_t i = b + g * NW + warp; i < e; i += kSlices * NW) {
        const T *x = X + (int64_t)idx[i] * ld;
        double xv[4], nrm = 0.0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int c = lane + 32 * q;
            xv[q] = (c < d) ? (double)to_f32<T>(x[c]) : 0.0;
            nrm += xv[q] * xv[q];
        }
        for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
        const double w = 1.0 / p[i];
        if (nrm > 0.0) {
            const double inv = 1.0 / sqrt(nrm);
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] += w * (xv[q] * inv);
            s += w;
        } else {
            z += w;
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) sh_v[warp][lane + 32 * q] = v[q];
    if (lane == 0) {
        sh_s[warp] = s;
        sh_z[warp] = z;
    }
    __syncthreads();
    double *out = part + ((int64_t)j * kSlices + g) * (D + 2);
    if ((int)threadIdx.x < D) {
        double V = 0.0;
        for (int w = 0; w < NW; ++w) V += sh_v[w][threadIdx.x];
        out[threadIdx.x] = V;
    } else if ((int)threadIdx.x == D) {
        double S = 0.0, Z = 0.0;
        for (int w = 0; w < NW; ++w) {
            S += sh_s[w];
            Z += sh_z[w];
        }
        out[D] = S;
        out[D + 1] = Z;
    }
}

// One block (128 threads) per cluster: combine the slices in index order;
// mu_j = V / S_j goes to the row kernel negated and split into two FP32 words
// (hi + lo carries it to ~2^-48), zero padded to D.  Since every sampled
// non-zero y^ is a unit vector, R_j = sum w |y^ - mu_j|^2 = S_j (1 - |mu_j|^2);
// in FP64 its rounding error stays ~1e-16 S_j even for a tight cluster.
__global__ void k_collapse_final(const double *__restrict__ part, int d, int D,
                                 float *__restrict__ nmu_hi, float *__restrict__ nmu_lo,
                                 double *__restrict__ Sw, double *__restrict__ Zw,
                                 double *__restrict__ Rw) {
    __shared__ double sh_sq[128];
    const int j = blockIdx.x, c = threadIdx.x;
    const double *pj = part + (int64_t)j * kSlices * (D + 2);
    double S = 0.0, Z = 0.0, V = 0.0;
    for (int g = 0; g < kSlices; ++g) {
        S += pj[g * (D + 2) + D];
        Z += pj[g * (D + 2) + D + 1];
        if (c < D) V += pj[g * (D + 2) + c];
    }
    const double m = (S > 0.0 && c < d) ? V / S : 0.0;
    if (c < D) {
        const float hi = (float)m;
        nmu_hi[(int64_t)j * D + c] = -hi;
        nmu_lo[(int64_t)j * D + c] = -(float)(m - (double)hi);
    }
    sh_sq[c] = m * m;
    __syncthreads();
    if (c == 0) {
        double q = 0.0;
        for (int i = 0; i < 128; ++i) q += sh_sq[i];
        Sw[j] = S;
        Zw[j] = Z;
        Rw[j] = S > 0.0 ? S * fmax(0.0, 1.0 - q) : 0.0;
    }
}

// One row per thread: W_hat_j = Z_j + 0.5 (S_j |x^ - mu_j|^2 + R_j) for every
// cluster (a zero row is at distance 1 from everything: S_j + Z_j), then
// a_hat, b_hat, s_hat of Eq. 8.  The cluster constants are staged through
// shared memory CH clusters at a time.
template <class T, int D>
__global__ void __launch_bounds__(kRowThreads)
k_collapse_rows(const T *__restrict__ X, int d, int64_t ld, int64_t n,
                const int32_t *__restrict__ labels, int k, const int64_t *__restrict__ sizes,
                const float *__restrict__ nmu_hi, const float *__restrict__ nmu_lo,
                const double *__restrict__ Sw,
                const double *__restrict__ Zw, const double *__restrict__ Rw,
                const int64_t *__restrict__ rows, int64_t nrows, float *__restrict__ s_out,
                float *__restrict__ a_out, float *__restrict__ b_out,
                int32_t *__restrict__ nb_out) {
    constexpr int CH = (D <= 32) ? 64 : 16;
    __shared__ __align__(16) float sh_hi[CH * D];
    __shared__ __align__(16) float sh_lo[CH * D];
    __shared__ float sh_s[CH], sh_c[CH];    // 0.5 S_j and Z_j + 0.5 R_j (FP32)
    __shared__ float sh_all[CH];            // S_j + Z_j
    __shared__ float sh_inv[CH];            // 1 / |C_j|
    const int64_t rr = (int64_t)blockIdx.x * kRowThreads + threadIdx.x;
    const int64_t e = (rr < nrows) ? (rows ? rows[rr] : rr) : -1;
    int own = -1;
    if (e >= 0 && e < n) {
        const int l = labels[e];
        own = (l >= 0 && l < k) ? l : -2;
    }
    float2 x[D / 2];
    float2 sq = make_float2(0.f, 0.f);
#pragma unroll
    for (int c = 0; c < D; c += 2) {
        const bool ok = own >= 0;
        const float a = (ok && c < d) ? to_f32<T>(X[e * ld + c]) : 0.f;
        const float b = (ok && c + 1 < d) ? to_f32<T>(X[e * ld + c + 1]) : 0.f;
        x[c / 2] = make_float2(a, b);
        sq = __ffma2_rn(x[c / 2], x[c / 2], sq);
    }
    // unit row in FP32: rsqrt refined by one Newton step (inv (1.5 - 0.5 n inv^2))
    const float nrm = sq.x + sq.y;
    const bool zero = !(nrm > 0.f);
    float inv = zero ? 0.f : rsqrtf(nrm);
    inv = zero ? 0.f : inv * fmaf(-0.5f * nrm * inv, inv, 1.5f);
#pragma unroll
    for (int c = 0; c < D / 2; ++c) x[c] = __fmul2_rn(x[c], make_float2(inv, inv));
    // every term below is non-negative and carries a few FP32 roundings, so
    // W_hat_j and its ratio to |C_j| stay FP32; a_hat, b_hat, s_hat are FP64
    float wown = 0.f, bmin = INFINITY;
    int barg = -1;                          // neighbouring cluster (lowest j on ties)
    for (int j0 = 0; j0 < k; j0 += CH) {
        const int nb = min(CH, k - j0);
        __syncthreads();
        for (int q = threadIdx.x; q < nb * D / 4; q += kRowThreads) {
            reinterpret_cast<float4 *>(sh_hi)[q] =
                reinterpret_cast<const float4 *>(nmu_hi + (int64_t)j0 * D)[q];
            reinterpret_cast<float4 *>(sh_lo)[q] =
                reinterpret_cast<const float4 *>(nmu_lo + (int64_t)j0 * D)[q];
        }
        for (int q = threadIdx.x; q < nb; q += kRowThreads) {
            const int j = j0 + q;
            sh_s[q] = (float)(0.5 * Sw[j]);
            sh_c[q] = (float)(Zw[j] + 0.5 * Rw[j]);
            sh_all[q] = (float)(Sw[j] + Zw[j]);
            sh_inv[q] = (float)(1.0 / (double)sizes[j]);
        }
        __syncthreads();
        if (own < 0) continue;
        for (int q = 0; q < nb; ++q) {
            const float2 *h2 = reinterpret_cast<const float2 *>(sh_hi + q * D);
            const float2 *l2 = reinterpret_cast<const float2 *>(sh_lo + q * D);
            float2 acc0 = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
#pragma unroll
            for (int c = 0; c < D / 2; c += 2) {
                // (x - mu_hi) is exact where x is close to mu_hi; then - mu_lo
                const float2 t0 = __fadd2_rn(__fadd2_rn(x[c], h2[c]), l2[c]);
                const float2 t1 = __fadd2_rn(__fadd2_rn(x[c + 1], h2[c + 1]), l2[c + 1]);
                acc0 = __ffma2_rn(t0, t0, acc0);
                acc1 = __ffma2_rn(t1, t1, acc1);
            }
            const float dist = (acc0.x + acc0.y) + (acc1.x + acc1.y);
            const float w = zero ? sh_all[q] : fmaf(sh_s[q], dist, sh_c[q]);
            if (j0 + q == own) wown = w;
            else if (w * sh_inv[q] < bmin) {
                bmin = w * sh_inv[q];
                barg = j0 + q;
            }
        }
    }
    if (rr >= nrows) return;
    float sv, av, bv;
    if (own < 0) {
        sv = av = bv = NAN;
    } else {
        const int64_t nc = sizes[own];
        const double a = (nc > 1) ? (double)wown / (double)(nc - 1) : 0.0;
        const double bd = (double)bmin;
        const double mx = fmax(a, bd);
        sv = (float)((nc > 1 && mx > 0.0) ? (bd - a) / mx : 0.0);
        av = (float)a;
        bv = bmin;
    }
    s_out[rr] = sv;
    if (a_out) a_out[rr] = av;
    if (b_out) b_out[rr] = bv;
    if (nb_out) nb_out[rr] = (own < 0) ? -1 : barg;
}

template <class T>
void launch_rows(int D, cudaStream_t stream, const T *X, int d, int64_t ld, int64_t n,
                 const int32_t *labels, int k, const int64_t *sizes, const float *nmu_hi,
                 const float *nmu_lo, const double *Sw, const double *Zw, const double *Rw, const int64_t *rows,
                 int64_t nrows, float *s, float *a, float *b, int32_t *nb) {
    const int grid = (int)((nrows + kRowThreads - 1) / kRowThreads);
    switch (D) {
        case 8: k_collapse_rows<T, 8><<<grid, kRowThreads, 0, stream>>>(X, d, ld, n, labels, k, sizes, nmu_hi, nmu_lo, Sw, Zw, Rw, rows, nrows, s, a, b, nb); break;
        case 16: k_collapse_rows<T, 16><<<grid, kRowThreads, 0, stream>>>(X, d, ld, n, labels, k, sizes, nmu_hi, nmu_lo, Sw, Zw, Rw, rows, nrows, s, a, b, nb); break;
        case 32: k_collapse_rows<T, 32><<<grid, kRowThreads, 0, stream>>>(X, d, ld, n, labels, k, sizes, nmu_hi, nmu_lo, Sw, Zw, Rw, rows, nrows, s, a, b, nb); break;
        case 64: k_collapse_rows<T, 64><<<grid, kRowThreads, 0, stream>>>(X, d, ld, n, labels, k, sizes, nmu_hi, nmu_lo, Sw, Zw, Rw, rows, nrows, s, a, b, nb); break;
        default: k_collapse_rows<T, 128><<<grid, kRowThreads, 0, stream>>>(X, d, ld, n, labels, k, sizes, nmu_hi, nmu_lo, Sw, Zw, Rw, rows, nrows, s, a, b, nb); break;
    }
    count_launches(1);
}

}  // namespace
}  // namespace silh

using namespace silh;

extern "C" silh_status silh_estimate_cosine_collapsed(
        const void *X, silh_dtype dtype, int64_t n, int32_t d, int64_t ld, const int32_t *labels,
        int32_t k, const silh_sample *S, const int64_t *rows, int64_t nrows, float *s_hat,
        float *a_hat, float *b_hat, int32_t *nb, void *stream_) {
    cudaStream_t stream = (cudaStream_t)stream_;
    silh_status st = SILH_OK;
    Scratch sc(stream);
    float *nmu_hi = nullptr, *nmu_lo = nullptr;
    double *Sw = nullptr, *Zw = nullptr, *Rw = nullptr, *part = nullptr;
    int D = 0, dev = 0;
    SILH_REQ(X && labels, "null pointer argument");
    SILH_REQ(n >= 2 && n < (int64_t(1) << 31), "n must be in [2, 2^31)");
    SILH_REQ(d >= 1 && d <= 128 && ld >= d, "need 1 <= d <= 128 and ld >= d");
    SILH_REQ(k >= 2 && k <= SILH_MAX_K, "k must be in [2, %d]", SILH_MAX_K);
    SILH_REQ(dtype == SILH_F32 || dtype == SILH_BF16, "unknown dtype");
    SILH_REQ(S && S->k == k && S->sizes && S->offsets, "sample missing or k mismatch");
    SILH_REQ(S->size >= 0 && S->size <= S->cap && (S->size == 0 || (S->idx && S->p)),
             "bad sample size");
    SILH_REQ(s_hat, "s_hat is null");
    SILH_DEVPTR(X, "X");
    SILH_DEVPTR(labels, "labels");
    SILH_REQ(sample_accessible(S), "sample arrays are not device-accessible memory");
    SILH_DEVPTR(s_hat, "s_hat");
    SILH_DEVPTR_OPT(a_hat, "a_hat");
    SILH_DEVPTR_OPT(b_hat, "b_hat");
    SILH_DEVPTR_OPT(nb, "neighbour");
    SILH_DEVPTR_OPT(rows, "rows");
    if (rows == nullptr) nrows = n;
    SILH_REQ(nrows >= 0, "nrows < 0");
    SILH_CK(cudaGetDevice(&dev));
    ensure_pool_retains(dev);
    D = padded_dim(d);
    SILH_CK(sc.alloc(&nmu_hi, (size_t)k * D));
    SILH_CK(sc.alloc(&nmu_lo, (size_t)k * D));
    SILH_CK(sc.alloc(&Sw, (size_t)k));
    SILH_CK(sc.alloc(&Zw, (size_t)k));
    SILH_CK(sc.alloc(&Rw, (size_t)k));
    SILH_CK(sc.alloc(&part, (size_t)k * kSlices * (D + 2)));
    if (dtype == SILH_F32)
        k_collapse_partial<float><<<dim3(k, kSlices), kClThreads, 0, stream>>>(
            (const float *)X, d, ld, S->offsets, S->idx, S->p, D, part);
    else
        k_collapse_partial<__nv_bfloat16><<<dim3(k, kSlices), kClThreads, 0, stream>>>(
            (const __nv_bfloat16 *)X, d, ld, S->offsets, S->idx, S->p, D, part);
    k_collapse_final<<<k, 128, 0, stream>>>(part, d, D, nmu_hi, nmu_lo, Sw, Zw, Rw);
    count_launches(2);
    SILH_CK(cudaGetLastError());
    if (nrows > 0) {
        if (dtype == SILH_F32)
            launch_rows<float>(D, stream, (const float *)X, d, ld, n, labels, k, S->sizes, nmu_hi, nmu_lo,
                               Sw, Zw, Rw, rows, nrows, s_hat, a_hat, b_hat, nb);
        else
            launch_rows<__nv_bfloat16>(D, stream, (const __nv_bfloat16 *)X, d, ld, n, labels, k,
                                       S->sizes, nmu_hi, nmu_lo, Sw, Zw, Rw, rows, nrows, s_hat,
                                       a_hat, b_hat, nb);
        SILH_CK(cudaGetLastError());
    }
done:
    return st;
}
