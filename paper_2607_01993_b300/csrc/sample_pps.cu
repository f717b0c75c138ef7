// Phase 1 of Algorithm 1 (PPS sampling) and the cluster bookkeeping it needs.
//
// Layout: every per-element array of Phase 1 is indexed by the element's
// position in cluster-major order ("pos"): order[pos] is the element id,
// coff[j] .. coff[j+1]-1 are the positions of cluster j, ascending element id
// inside a cluster.  Distances from cluster members to the initial sample F0_j
// are kept in an FP64 matrix D_j of |F0_j| x |Cj| (F0-major, so that the W sums
// and the gamma sweep both read it coalesced).
//
// Precision: Phase 1 decides which elements are sampled (u < p_e), so it runs
// at FP64-class accuracy.  Pair distances use double-float arithmetic (an FP32
// pair hi + lo carried with error-free transformations: Knuth's two-sum, the
// FMA two-product), about 2^-44 relative (cosine: its inner product and norms,
// then 1 - <x,y>/(|x||y|) in FP64), which B300 evaluates an order of magnitude
// faster than native FP64.  W sums, gamma and p are FP64.
#include <algorithm>
#include <cmath>

#include "kernels.cuh"

namespace silh {

namespace {

constexpr int kHistWarps = 1;

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Per-tile histograms: counts[j * ntiles + tile] (cluster-major).
__global__ void k_tile_hist(const int32_t *__restrict__ labels, int64_t n, int k, int tile,
                            int ntiles, int32_t *__restrict__ counts, int32_t *__restrict__ bad) {
    extern __shared__ int32_t sh_cnt[];
    for (int j = threadIdx.x; j < k; j += blockDim.x) sh_cnt[j] = 0;
    __syncwarp();
    int64_t base = (int64_t)blockIdx.x * tile;
    int64_t end = min(base + (int64_t)tile, n);
    for (int64_t i = base + threadIdx.x; i < end; i += blockDim.x) {
        int32_t l = labels[i];
        if (l < 0 || l >= k) {
            atomicOr(bad, 1);
            continue;
        }
        atomicAdd(&sh_cnt[l], 1);
    }
    __syncwarp();
    for (int j = threadIdx.x; j < k; j += blockDim.x)
        counts[(int64_t)j * ntiles + blockIdx.x] = sh_cnt[j];
}

// Block j: exclusive scan over tiles of cluster j's tile counts; sizes[j] = total.
__global__ void k_cluster_scan(const int32_t *__restrict__ counts, int ntiles,
                               int64_t *__restrict__ tile_base, int64_t *__restrict__ sizes) {
    __shared__ int64_t sh[1024];
    int j = blockIdx.x;
    const int32_t *c = counts + (int64_t)j * ntiles;
    int64_t *o = tile_base + (int64_t)j * ntiles;
    int per = (ntiles + blockDim.x - 1) / blockDim.x;
    int lo = threadIdx.x * per, hi = min(lo + per, ntiles);
    int64_t s = 0;
    for (int i = lo; i < hi; ++i) s += c[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    // Hillis-Steele inclusive scan of the per-thread sums.
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        int64_t v = (threadIdx.x >= (unsigned)off) ? sh[threadIdx.x - off] : 0;
        __syncthreads();
        sh[threadIdx.x] += v;
        __syncthreads();
    }
    int64_t run = sh[threadIdx.x] - s;
    for (int i = lo; i < hi; ++i) {
        o[i] = run;
        run += c[i];
    }
    if (threadIdx.x == blockDim.x - 1) sizes[j] = sh[threadIdx.x];
}

// Stable scatter: one warp walks its tile in element order; lanes with the same
// label are ranked by lane id.
__global__ void k_scatter(const int32_t *__restrict__ labels, int64_t n, int k, int tile,
                          int ntiles, const int64_t *__restrict__ tile_base,
                          const int64_t *__restrict__ coff, int32_t *__restrict__ order) {
    extern __shared__ int32_t sh_cnt[];
    for (int j = threadIdx.x; j < k; j += 32) sh_cnt[j] = 0;
    __syncwarp();
    int64_t base = (int64_t)blockIdx.x * tile;
    int64_t end = min(base + (int64_t)tile, n);
    unsigned lt = lanemask_lt();
    for (int64_t i0 = base; i0 < end; i0 += 32) {
        int64_t i = i0 + threadIdx.x;
        int32_t l = (i < end) ? labels[i] : -1;
        bool ok = (l >= 0 && l < k);
        int key = ok ? l : -1;
        unsigned peers = __match_any_sync(0xffffffffu, key);
        int rank = __popc(peers & lt);
        int cnt = ok ? sh_cnt[l] : 0;
        __syncwarp();
        if (ok) {
            int64_t pos = coff[l] + tile_base[(int64_t)l * ntiles + blockIdx.x] + cnt + rank;
            order[pos] = (int32_t)i;
            if (rank == 0) sh_cnt[l] = cnt + __popc(peers);
        }
        __syncwarp();
    }
}

// ----------------------------------------------- asynchronous Phase 1
// The asynchronous entry point sizes everything on the device: a status word
// (SILH_OK or an error) gates every later kernel, which returns at once when it
// is set, so an invalid clustering or an exhausted capacity never leads to an
// out-of-range access; the sample is then written as an empty one.

__device__ __forceinline__ bool gated(const int32_t *status) {
    return status != nullptr && *status != SILH_OK;
}

// coff[j] = exclusive prefix of the sizes (one block); an invalid label seen by
// the histogram (*bad) or an empty cluster sets *status = SILH_EINVAL.
__global__ void k_coff_async(const int64_t *__restrict__ sizes, int k,
                             const int32_t *__restrict__ bad, int64_t *__restrict__ coff,
                             int32_t *__restrict__ status) {
    __shared__ int64_t sh[1024];
    __shared__ int empty;
    if (threadIdx.x == 0) empty = 0;
    __syncthreads();
    const int per = (k + 1023) / 1024;
    const int lo = threadIdx.x * per, hi = min(lo + per, k);
    int64_t s = 0;
    for (int j = lo; j < hi; ++j) {
        s += sizes[j];
        if (sizes[j] == 0) empty = 1;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int64_t v = (threadIdx.x >= (unsigned)off) ? sh[threadIdx.x - off] : 0;
        __syncthreads();
        sh[threadIdx.x] += v;
        __syncthreads();
    }
    int64_t run = sh[threadIdx.x] - s;
    for (int j = lo; j < hi; ++j) {
        coff[j] = run;
        run += sizes[j];
    }
    if (threadIdx.x == 1023) coff[k] = sh[1023];
    if (threadIdx.x == 0 && (*bad != 0 || empty)) *status = SILH_EINVAL;
}

// Plan of the member x F0 distance matrices on the device (one block): doff[j] =
// exclusive prefix of |Cj| |F0_j| and item_base[j] = exclusive prefix of the
// 128-member chunks of the clusters with a non-empty F0; a total beyond the
// matrix capacity sets *status = SILH_ECAPACITY.
__global__ void k_plan_f0(const int64_t *__restrict__ coff, const int64_t *__restrict__ f0off,
                          int k, int64_t dcap, int64_t *__restrict__ doff,
                          int64_t *__restrict__ item_base, int32_t *__restrict__ status) {
    __shared__ int64_t shd[1024], shi[1024];
    if (gated(status)) return;
    const int per = (k + 1023) / 1024;
    const int lo = threadIdx.x * per, hi = min(lo + per, k);
    int64_t sd = 0, si = 0;
    for (int j = lo; j < hi; ++j) {
        const int64_t nc = coff[j + 1] - coff[j], nf = f0off[j + 1] - f0off[j];
        sd += nc * nf;
        si += nf > 0 ? (nc + 127) / 128 : 0;
    }
    shd[threadIdx.x] = sd;
    shi[threadIdx.x] = si;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int64_t vd = (threadIdx.x >= (unsigned)off) ? shd[threadIdx.x - off] : 0;
        const int64_t vi = (threadIdx.x >= (unsigned)off) ? shi[threadIdx.x - off] : 0;
        __syncthreads();
        shd[threadIdx.x] += vd;
        shi[threadIdx.x] += vi;
        __syncthreads();
    }
    int64_t rd = shd[threadIdx.x] - sd, ri = shi[threadIdx.x] - si;
    for (int j = lo; j < hi; ++j) {
        const int64_t nc = coff[j + 1] - coff[j], nf = f0off[j + 1] - f0off[j];
        doff[j] = rd;
        item_base[j] = ri;
        rd += nc * nf;
        ri += nf > 0 ? (nc + 127) / 128 : 0;
    }
    if (threadIdx.x == 1023) {
        doff[k] = shd[1023];
        item_base[k] = shi[1023];
        if (shd[1023] > dcap) *status = SILH_ECAPACITY;
    }
}

// |S| to *d_size, or SILH_ECAPACITY when it exceeds the caller's capacity.
__global__ void k_finish_size(const int64_t *__restrict__ total, int64_t cap,
                              int64_t *__restrict__ d_size, int32_t *__restrict__ status) {
    if (*status == SILH_OK && *total > cap) *status = SILH_ECAPACITY;
    *d_size = (*status == SILH_OK) ? *total : 0;
}

// ------------------------------------------------------------------- scan

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ int64_t block_excl_scan(int64_t v, int64_t *sh, int64_t *total) {
    int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int off = 1; off < kScanThreads; off <<= 1) {
        int64_t u = (t >= off) ? sh[t - off] : 0;
        __syncthreads();
        sh[t] += u;
        __syncthreads();
    }
    int64_t incl = sh[t];
    if (total) *total = sh[kScanThreads - 1];
    __syncthreads();
    return incl - v;
}

__global__ void k_scan_reduce(const int32_t *__restrict__ f, int64_t n, int64_t *__restrict__ bsum) {
    __shared__ int64_t sh[kScanThreads];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t s = 0;
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) s += f[base + i];
    int64_t tot;
    block_excl_scan(s, sh, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_scan_top(int64_t *__restrict__ bsum, int nb, int64_t *__restrict__ total) {
    __shared__ int64_t sh[kScanThreads];
    int per = (nb + kScanThreads - 1) / kScanThreads;
    int lo = threadIdx.x * per, hi = min(lo + per, nb);
    int64_t s = 0;
    for (int i = lo; i < hi; ++i) s += bsum[i];
    int64_t tot;
    int64_t run = block_excl_scan(s, sh, &tot);
    for (int i = lo; i < hi; ++i) {
        int64_t v = bsum[i];
        bsum[i] = run;
        run += v;
    }
    if (threadIdx.x == 0) *total = tot;
}

__global__ void k_scan_down(const int32_t *__restrict__ f, int64_t n,
                            const int64_t *__restrict__ bsum, int64_t *__restrict__ out) {
    __shared__ int64_t sh[kScanThreads];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int32_t v[kScanItems];
    int64_t s = 0;
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < n) ? f[base + i] : 0;
        s += v[i];
    }
    int64_t run = block_excl_scan(s, sh, nullptr) + bsum[blockIdx.x];
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
}

// ---------------------------------------------------------------- Phase 1

// Initial Poisson sample F0 (stream 0) for clusters with |Cj| > t.
__global__ void k_draw_f0(const int32_t *__restrict__ order, const int32_t *__restrict__ labels,
                          const int64_t *__restrict__ sizes, int64_t n, double t, double m0,
                          uint64_t seed, uint64_t cid, int32_t *__restrict__ flag0,
                          const int32_t *__restrict__ status = nullptr) {
    int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= n || gated(status)) return;
    int32_t e = order[pos];
    int64_t nc = sizes[labels[e]];
    int32_t f = 0;
    if ((double)nc > t) {
        double q = __ddiv_rn(m0, (double)nc);
        if (q > 1.0) q = 1.0;
        f = uniform01(seed, 0, cid, (uint64_t)e) < q ? 1 : 0;
    }
    flag0[pos] = f;
}

__global__ void k_compact(const int32_t *__restrict__ flag, const int64_t *__restrict__ pos_of,
                          const int32_t *__restrict__ order, int64_t n, int32_t *__restrict__ ids,
                          const double *__restrict__ pv, double *__restrict__ pout,
                          const int32_t *__restrict__ status = nullptr) {
    int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= n || gated(status) || !flag[pos]) return;
    int64_t o = pos_of[pos];
    ids[o] = order[pos];
    if (pout) pout[o] = pv[pos];
}

// off[j] = pos_of[coff[j]] (j < k), off[k] = total; all zero (an empty sample)
// when the status word is set.
__global__ void k_seg_offsets(const int64_t *__restrict__ pos_of, const int64_t *__restrict__ coff,
                              int k, int64_t n, const int64_t *__restrict__ total,
                              int64_t *__restrict__ off,
                              const int32_t *__restrict__ status = nullptr) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j > k) return;
    if (gated(status)) {
        off[j] = 0;
        return;
    }
    off[j] = (j == k || coff[j] >= n) ? *total : pos_of[coff[j]];
}

constexpr int kF0Group = 8;     // F0 rows staged in shared memory at a time
constexpr int kDistThreads = 128;

// ------------------------------------------------ double-float arithmetic
// A value is carried as hi + lo (two FP32 numbers).  two_sum (Knuth) and
// two_prod (one FMA) return the exact rounding error of an add / a multiply;
// df_acc adds a nonnegative FP32 term to a nonnegative accumulator and
// renormalises.  All operations are explicitly rounded (no contraction).

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {  // |a| >= |b|
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

__device__ __forceinline__ void df_acc(float &hi, float &lo, float b) {
    float s, e;
    two_sum(hi, b, s, e);
    e = __fadd_rn(e, lo);
    fast_two_sum(s, e, hi, lo);
}

// The same operations on two independent values at once (packed two-lane
// FP32, each lane's operation rounded to nearest like the scalar one).  The
// adds, subtracts and multiplies carry an explicit rounding mode in PTX,
// which keeps the compiler from fusing a multiply into a later add.
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

__device__ __forceinline__ float2 add2_rn(float2 a, float2 b) {
    unsigned long long r;
    const unsigned long long x = *reinterpret_cast<const unsigned long long *>(&a);
    const unsigned long long y = *reinterpret_cast<const unsigned long long *>(&b);
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(x), "l"(y));
    return *reinterpret_cast<const float2 *>(&r);
}

__device__ __forceinline__ float2 sub2_rn(float2 a, float2 b) {
    unsigned long long r;
    const unsigned long long x = *reinterpret_cast<const unsigned long long *>(&a);
    const unsigned long long y = *reinterpret_cast<const unsigned long long *>(&b);
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(x), "l"(y));
    return *reinterpret_cast<const float2 *>(&r);
}

__device__ __forceinline__ float2 mul2_rn(float2 a, float2 b) {
    unsigned long long r;
    const unsigned long long x = *reinterpret_cast<const unsigned long long *>(&a);
    const unsigned long long y = *reinterpret_cast<const unsigned long long *>(&b);
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(x), "l"(y));
    return *reinterpret_cast<const float2 *>(&r);
}

__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2 &s, float2 &e) {
    s = add2_rn(a, b);
    const float2 bb = sub2_rn(s, a);
    e = add2_rn(sub2_rn(a, sub2_rn(s, bb)), sub2_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum2(float2 a, float2 b, float2 &s, float2 &e) {
    s = add2_rn(a, b);
    e = sub2_rn(b, sub2_rn(s, a));
}

__device__ __forceinline__ void two_prod2(float2 a, float2 b, float2 &p, float2 &e) {
    p = mul2_rn(a, b);
    e = __ffma2_rn(a, b, neg2(p));
}

__device__ __forceinline__ void df_acc2(float2 &hi, float2 &lo, float2 b) {
    float2 s, e;
    two_sum2(hi, b, s, e);
    e = add2_rn(e, lo);
    fast_two_sum2(s, e, hi, lo);
}

__device__ __forceinline__ float rcp_apx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float sqrt_apx(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// One Canberra term |x - y| / (|x| + |y|) added to the double-float sum
// (hi, lo), given x - y = s + t (s >= 0) and |x| + |y| = ds + de: in FP32 with
// one residual step when ds is in [2^-100, 2^100], else (or for a zero pair,
// which adds nothing) in FP64 from the coordinates.
__device__ __forceinline__ void canb_df_lane(float xv, float yv, float s, float t, float ds,
                                             float de, bool in_range, float &hi, float &lo) {
    if (!in_range) {
        if (ds != 0.f) {
            const double xd = xv, yd = yv;
            const double q = fabs(xd - yd) / (fabs(xd) + fabs(yd));
            const float qh = (float)q;
            df_acc(hi, lo, qh);
            lo = __fadd_rn(lo, (float)(q - (double)qh));
        }
    } else {
        const float rc = rcp_apx(ds);
        const float q0 = __fmul_rn(s, rc);
        float rr = __fmaf_rn(-q0, ds, s);     // residual of s / ds
        rr = __fadd_rn(rr, t);
        rr = __fmaf_rn(-q0, de, rr);
        const float q1 = __fmul_rn(rr, rc);
        df_acc(hi, lo, q0);
        lo = __fadd_rn(lo, q1);
    }
}

// Phase-1 pair distances for Euclidean, Manhattan and Canberra in double-float
// arithmetic.  D_j[f, i] = d(member i, F0_j[f]), one thread per member, F0
// rows staged in shared memory kF0Group at a time; work item w covers members
// [chunk*128, chunk*128+128) of cluster item_cluster[w].  The staged rows
// are interleaved in pairs (element c of rows 2h and 2h + 1 side by side) and
// each thread carries the two rows of a pair in the two lanes of packed FP32
// registers, every lane with the scalar sequence of operations (measured on
// the large workload: the samples of Euclidean, cosine and Manhattan are
// bit-identical to the one-row-at-a-time form, Canberra's inclusion
// probabilities agree to 2e-14 relative, the accuracy of the double-float
// sums, and its sample sets are identical).
// Work items from item_cluster / item_chunk (planned on the host), or, when
// item_cluster is null, from item_base[k + 1] (planned on the device: block b is
// chunk b - item_base[j] of the last cluster j with item_base[j] <= b; blocks
// past item_base[k] have none).
template <class T, int METRIC>
__global__ void k_dist_f0_df(const T *__restrict__ X, int d, int64_t ld,
                             const int32_t *__restrict__ order, const int64_t *__restrict__ coff,
                             const int32_t *__restrict__ f0_elem, const int64_t *__restrict__ f0off,
                             const int64_t *__restrict__ doff, const int32_t *__restrict__ item_cluster,
                             const int32_t *__restrict__ item_chunk, double *__restrict__ D,
                             const int64_t *__restrict__ item_base = nullptr, int k = 0,
                             const int32_t *__restrict__ status = nullptr) {
    extern __shared__ float sh_yf[];            // kF0Group x d, rows interleaved in pairs,
                                                // negated (x + (-y)) but for cosine
    static_assert(kF0Group % 2 == 0, "rows are paired");
    constexpr int NP = kF0Group / 2;
    __shared__ double sh_inv[kF0Group];         // cosine: 1/|y| of the staged rows (0: zero row)
    int j;
    int64_t chunk;
    if (item_cluster != nullptr) {
        j = item_cluster[blockIdx.x];
        chunk = item_chunk[blockIdx.x];
    } else {
        const int64_t b = blockIdx.x;
        if (gated(status) || b >= item_base[k]) return;
        int lo = 0, hi = k - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (item_base[mid] <= b) lo = mid;
            else hi = mid - 1;
        }
        j = lo;
        chunk = b - item_base[lo];
    }
    const int64_t c0 = coff[j], nc = coff[j + 1] - c0;
    const int64_t i = chunk * kDistThreads + threadIdx.x;
    const bool live = i < nc;
    const int64_t e = live ? order[c0 + i] : 0;
    const int64_t g0 = f0off[j], nf = f0off[j + 1] - g0;
    double *Dj = D + doff[j];
    double inv_x = 0.0;                         // cosine: 1/|x| of this member (0: zero row)
    if (METRIC == SILH_COSINE && live) {
        float nh = 0.f, nl = 0.f;
        for (int c = 0; c < d; ++c) {
            const float xv = to_f32<T>(X[e * ld + c]);
            float p, pe;
            two_prod(xv, xv, p, pe);
            df_acc(nh, nl, p);
            nl = __fadd_rn(nl, pe);
        }
        const double n2 = (double)nh + (double)nl;
        inv_x = n2 > 0.0 ? __ddiv_rn(1.0, __dsqrt_rn(n2)) : 0.0;
    }
    for (int64_t gb = 0; gb < nf; gb += kF0Group) {
        const int gc = (int)min((int64_t)kF0Group, nf - gb);
        __syncthreads();
        for (int q = threadIdx.x; q < kF0Group * d; q += blockDim.x) {
            const int g = q / d, c = q % d;
            const float yv = (g < gc) ? to_f32<T>(X[(int64_t)f0_elem[g0 + gb + g] * ld + c]) : 0.f;
            sh_yf[((g >> 1) * d + c) * 2 + (g & 1)] = (METRIC == SILH_COSINE) ? yv : -yv;
        }
        __syncthreads();
        if (METRIC == SILH_COSINE && threadIdx.x < kF0Group) {
            float nh = 0.f, nl = 0.f;
            for (int c = 0; c < d; ++c) {
                const float yv = sh_yf[((threadIdx.x >> 1) * d + c) * 2 + (threadIdx.x & 1)];
                float p, pe;
                two_prod(yv, yv, p, pe);
                df_acc(nh, nl, p);
                nl = __fadd_rn(nl, pe);
            }
            const double n2 = (double)nh + (double)nl;
            sh_inv[threadIdx.x] = n2 > 0.0 ? __ddiv_rn(1.0, __dsqrt_rn(n2)) : 0.0;
        }
        __syncthreads();
        if (!live) continue;
        float2 hi2[NP], lo2[NP];
#pragma unroll
        for (int h = 0; h < NP; ++h) hi2[h] = lo2[h] = make_float2(0.f, 0.f);
        const T *xr = X + e * ld;
        const float2 *sy2 = reinterpret_cast<const float2 *>(sh_yf);
        for (int c = 0; c < d; ++c) {
            const float xv = to_f32<T>(xr[c]);
            const float2 xv2 = make_float2(xv, xv);
#pragma unroll
            for (int h = 0; h < NP; ++h) {
                const float2 yv = sy2[h * d + c];       // rows 2h, 2h + 1 (negated but for cosine)
                if (METRIC == SILH_COSINE) {            // signed double-float dot product
                    float2 p, pe, s2, e2;
                    two_prod2(xv2, yv, p, pe);
                    two_sum2(hi2[h], p, s2, e2);
                    e2 = add2_rn(add2_rn(e2, pe), lo2[h]);
                    two_sum2(s2, e2, hi2[h], lo2[h]);
                    continue;
                }
                float2 s, t;
                two_sum2(xv2, yv, s, t);                // x - y = s + t exactly
                if (METRIC == SILH_EUCLIDEAN) {
                    float2 p, pe;
                    two_prod2(s, s, p, pe);             // s^2 = p + pe exactly
                    // (s + t)^2 = p + pe + 2 s t + t^2; t^2 < 2^-46 p is dropped
                    const float2 small = __ffma2_rn(mul2_rn(make_float2(2.f, 2.f), s), t, pe);
                    df_acc2(hi2[h], lo2[h], p);
                    lo2[h] = add2_rn(lo2[h], small);
                } else {
                    if (s.x < 0.f) {                    // |x - y| = |s + t|
                        s.x = -s.x;
                        t.x = -t.x;
                    }
                    if (s.y < 0.f) {
                        s.y = -s.y;
                        t.y = -t.y;
                    }
                    if (METRIC == SILH_MANHATTAN) {
                        df_acc2(hi2[h], lo2[h], s);
                        lo2[h] = add2_rn(lo2[h], t);
                    } else {                            // Canberra
                        float2 ds, de;                  // |x| + |y| exactly
                        two_sum2(make_float2(fabsf(xv), fabsf(xv)),
                                 make_float2(fabsf(yv.x), fabsf(yv.y)), ds, de);
                        const bool in0 = ds.x >= 0x1p-100f && ds.x <= 0x1p+100f;
                        const bool in1 = ds.y >= 0x1p-100f && ds.y <= 0x1p+100f;
                        if (in0 && in1) {
                            const float2 rc = make_float2(rcp_apx(ds.x), rcp_apx(ds.y));
                            const float2 q0 = mul2_rn(s, rc);
                            float2 rr = __ffma2_rn(neg2(q0), ds, s);   // residual of s / ds
                            rr = add2_rn(rr, t);
                            rr = __ffma2_rn(neg2(q0), de, rr);
                            const float2 q1 = mul2_rn(rr, rc);
                            df_acc2(hi2[h], lo2[h], q0);
                            lo2[h] = add2_rn(lo2[h], q1);
                        } else {
                            // a lane with magnitudes outside the range the FP32
                            // reciprocal and residual steps keep exact (or a zero
                            // pair): that lane's term in FP64 from the coordinates
                            canb_df_lane(xv, -yv.x, s.x, t.x, ds.x, de.x, in0, hi2[h].x, lo2[h].x);
                            canb_df_lane(xv, -yv.y, s.y, t.y, ds.y, de.y, in1, hi2[h].y, lo2[h].y);
                        }
                    }
                }
            }
        }
        float hi[kF0Group], lo[kF0Group];
#pragma unroll
        for (int h = 0; h < NP; ++h) {
            hi[2 * h] = hi2[h].x;
            hi[2 * h + 1] = hi2[h].y;
            lo[2 * h] = lo2[h].x;
            lo[2 * h + 1] = lo2[h].y;
        }
#pragma unroll
        for (int g = 0; g < kF0Group; ++g) {
            if (g >= gc) break;
            double v;
            if (METRIC == SILH_EUCLIDEAN) {
                // sqrt(hi + lo): FP32 estimate y0, one Newton step on the double-float value
                const float h = hi[g];
                if (h > 0.f) {
                    const float y0 = sqrt_apx(h);
                    float p, pe;
                    two_prod(y0, y0, p, pe);
                    const float r = __fadd_rn(__fsub_rn(__fsub_rn(h, p), pe), lo[g]);
                    const float corr = __fmul_rn(r, __fmul_rn(0.5f, rcp_apx(y0)));
                    v = (double)y0 + (double)corr;
                } else {
                    v = 0.0;
                }
            } else if (METRIC == SILH_COSINE) {
                const double iy = sh_inv[g];
                if (inv_x == 0.0 || iy == 0.0) {
                    v = 1.0;                             // a zero-norm operand
                } else {
                    const double dot = (double)hi[g] + (double)lo[g];
                    v = __dsub_rn(1.0, __dmul_rn(__dmul_rn(dot, inv_x), iy));
                    v = v < 0.0 ? 0.0 : (v > 2.0 ? 2.0 : v);
                }
            } else {
                v = (double)hi[g] + (double)lo[g];
            }
            Dj[(gb + g) * nc + i] = v;
        }
    }
}

// W(e0) = sum over the members of column e0 of D_j, fixed reduction tree.
// Initial-sample points g = blockIdx.x, blockIdx.x + gridDim.x, ... below nf0
// (*d_nf0 when given, else gridDim.x: one block per point).
__global__ void k_w0(const int32_t *__restrict__ f0_elem, const int32_t *__restrict__ labels,
                     const int64_t *__restrict__ coff, const int64_t *__restrict__ f0off,
                     const int64_t *__restrict__ doff, const double *__restrict__ D,
                     double *__restrict__ W0, double *__restrict__ invW0,
                     const int64_t *__restrict__ d_nf0 = nullptr,
                     const int32_t *__restrict__ status = nullptr) {
    __shared__ double sh[256];
    if (gated(status)) return;
    const int64_t nf0 = d_nf0 ? *d_nf0 : (int64_t)gridDim.x;
    for (int64_t g = blockIdx.x; g < nf0; g += gridDim.x) {
        int j = labels[f0_elem[g]];
        int64_t nc = coff[j + 1] - coff[j];
        int64_t f = g - f0off[j];
        const double *col = D + doff[j] + f * nc;
        double s = 0.0;
        for (int64_t i = threadIdx.x; i < nc; i += 256) s += col[i];
        __syncthreads();
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int off = 128; off > 0; off >>= 1) {
            if (threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            W0[g] = sh[0];
            invW0[g] = sh[0] > 0.0 ? __ddiv_rn(1.0, sh[0]) : 0.0;   // W = 0: the term d/W is 0
        }
    }
}

// gamma_e, p_e and the final Poisson draw (stream 1), one thread per position.
__global__ void k_gamma_draw(const int32_t *__restrict__ order, const int32_t *__restrict__ labels,
                             const int64_t *__restrict__ coff, const int64_t *__restrict__ sizes,
                             const int64_t *__restrict__ f0off, const int64_t *__restrict__ doff,
                             const double *__restrict__ D, const double *__restrict__ invW0, int64_t n,
                             double t, int uniform, uint64_t seed, uint64_t cid,
                             double *__restrict__ pS, int32_t *__restrict__ flag1,
                             const int32_t *__restrict__ status = nullptr) {
    int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= n || gated(status)) return;
    int32_t e = order[pos];
    int j = labels[e];
    int64_t nc = sizes[j];
    double p;
    if ((double)nc <= t) {
        p = 1.0;
    } else if (uniform) {
        p = __ddiv_rn(t, (double)nc);
        if (p > 1.0) p = 1.0;
    } else {
        int64_t i = pos - coff[j];
        int64_t g0 = f0off[j], nf = f0off[j + 1] - g0;
        const double *Dj = D + doff[j];
        double g2 = 0.0;
        for (int64_t f = 0; f < nf; ++f) {
            const double r = __dmul_rn(Dj[f * nc + i], invW0[g0 + f]);   // d(e, e0) / W(e0)
            if (r > g2) g2 = r;
        }
        double g1 = __ddiv_rn(1.0, (double)nc);
        double g = g1 > g2 ? g1 : g2;
        p = __dmul_rn(t, g);
        if (!(p < 1.0)) p = 1.0;
    }
    pS[pos] = p;
    flag1[pos] = (p >= 1.0 || uniform01(seed, 1, cid, (uint64_t)e) < p) ? 1 : 0;
}

template <class T>
void launch_dist_f0(int metric, int nitems, size_t smem, cudaStream_t stream, const T *X, int d,
                    int64_t ld, const int32_t *order, const int64_t *coff, const int32_t *f0_elem,
                    const int64_t *f0off, const int64_t *doff, const int32_t *ic,
                    const int32_t *ik, double *D, const int64_t *item_base = nullptr, int k = 0,
                    const int32_t *status = nullptr) {
    const size_t smem_f = smem / 2;       // FP32 staging for the double-float kernels
    switch (metric) {
        case SILH_EUCLIDEAN:
            k_dist_f0_df<T, SILH_EUCLIDEAN><<<nitems, kDistThreads, smem_f, stream>>>(
                X, d, ld, order, coff, f0_elem, f0off, doff, ic, ik, D, item_base, k, status);
            break;
        case SILH_COSINE:
            k_dist_f0_df<T, SILH_COSINE><<<nitems, kDistThreads, smem_f, stream>>>(
                X, d, ld, order, coff, f0_elem, f0off, doff, ic, ik, D, item_base, k, status);
            break;
        case SILH_MANHATTAN:
            k_dist_f0_df<T, SILH_MANHATTAN><<<nitems, kDistThreads, smem_f, stream>>>(
                X, d, ld, order, coff, f0_elem, f0off, doff, ic, ik, D, item_base, k, status);
            break;
        default:
            k_dist_f0_df<T, SILH_CANBERRA><<<nitems, kDistThreads, smem_f, stream>>>(
                X, d, ld, order, coff, f0_elem, f0off, doff, ic, ik, D, item_base, k, status);
            break;
    }
    count_launches(1);
}

// Shared-memory opt-in of the Phase-1 distance kernels for wide rows.
template <class T>
cudaError_t dist_f0_smem_optin(size_t smem_f) {
    if (smem_f <= 48 * 1024) return cudaSuccess;
    for (auto f : {k_dist_f0_df<T, 0>, k_dist_f0_df<T, 1>, k_dist_f0_df<T, 2>, k_dist_f0_df<T, 3>}) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem_f);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

// ------------------------------------------------------------ host helpers

cudaError_t scan_flags(const int32_t *flags, int64_t n, int64_t *out, int64_t *d_total,
                       Scratch &sc, cudaStream_t stream) {
    int nb = (int)std::max<int64_t>(1, (n + kScanTile - 1) / kScanTile);
    int64_t *bsum = nullptr;
    cudaError_t e = sc.alloc(&bsum, nb);
    if (e != cudaSuccess) return e;
    k_scan_reduce<<<nb, kScanThreads, 0, stream>>>(flags, n, bsum); count_launches(1);
    k_scan_top<<<1, kScanThreads, 0, stream>>>(bsum, nb, d_total); count_launches(1);
    k_scan_down<<<nb, kScanThreads, 0, stream>>>(flags, n, bsum, out); count_launches(1);
    return cudaGetLastError();
}

silh_status cluster_sort(const int32_t *labels, int64_t n, int k, Scratch &sc,
                         cudaStream_t stream, int64_t *d_sizes, int64_t **d_coff,
                         int32_t **d_order, std::vector<int64_t> &h_sizes,
                         std::vector<int64_t> &h_coff) {
    silh_status st = SILH_OK;
    int tile = (k <= 512) ? 1024 : 8192;
    int ntiles = (int)((n + tile - 1) / tile);
    int32_t *counts = nullptr, *bad = nullptr;
    int64_t *tile_base = nullptr;
    int32_t h_bad = 0;
    size_t smem = sizeof(int32_t) * (size_t)k;
    SILH_CK(sc.alloc(&counts, (size_t)k * ntiles));
    SILH_CK(sc.alloc(&tile_base, (size_t)k * ntiles));
    SILH_CK(sc.alloc(&bad, 1));
    SILH_CK(sc.alloc(d_coff, (size_t)k + 1));
    SILH_CK(sc.alloc(d_order, (size_t)n));
    SILH_CK(cudaMemsetAsync(bad, 0, sizeof(int32_t), stream));
    if (smem > 48 * 1024) {
        SILH_CK(cudaFuncSetAttribute(k_tile_hist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
        SILH_CK(cudaFuncSetAttribute(k_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    }
    k_tile_hist<<<ntiles, 32 * kHistWarps, smem, stream>>>(labels, n, k, tile, ntiles, counts, bad); count_launches(1);
    k_cluster_scan<<<k, 256, 0, stream>>>(counts, ntiles, tile_base, d_sizes); count_launches(1);
    SILH_CK(cudaGetLastError());
    h_sizes.assign(k, 0);
    SILH_CK(cudaMemcpyAsync(h_sizes.data(), d_sizes, sizeof(int64_t) * k, cudaMemcpyDeviceToHost,
                            stream));
    SILH_CK(cudaMemcpyAsync(&h_bad, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
    SILH_CK(cudaStreamSynchronize(stream));
    SILH_REQ(h_bad == 0, "a label is outside [0, k)");
    for (int j = 0; j < k; ++j) SILH_REQ(h_sizes[j] > 0, "cluster %d is empty", j);
    h_coff.assign(k + 1, 0);
    for (int j = 0; j < k; ++j) h_coff[j + 1] = h_coff[j] + h_sizes[j];
    SILH_CK(cudaMemcpyAsync(*d_coff, h_coff.data(), sizeof(int64_t) * (k + 1),
                            cudaMemcpyHostToDevice, stream));
    k_scatter<<<ntiles, 32, smem, stream>>>(labels, n, k, tile, ntiles, tile_base, *d_coff,
                                            *d_order); count_launches(1);
    SILH_CK(cudaGetLastError());
done:
    return st;
}

}  // namespace silh

using namespace silh;

extern "C" silh_status silh_sample_pps(const void *X, silh_dtype dtype, int64_t n, int32_t d,
                                       int64_t ld, const int32_t *labels, int32_t k,
                                       silh_metric metric, double t, double m0, double delta,
                                       uint64_t seed, uint32_t clustering_id, int32_t uniform,
                                       silh_sample *out, void *stream_) {
    cudaStream_t stream = (cudaStream_t)stream_;
    silh_status st = SILH_OK;
    int dev = 0;
    Scratch sc(stream);
    std::vector<int64_t> h_sizes, h_coff, h_f0off, h_doff, h_off;
    std::vector<int32_t> h_ic, h_ik;
    int64_t *coff = nullptr, *pos0 = nullptr, *pos1 = nullptr, *tot = nullptr, *f0off = nullptr;
    int64_t *doff = nullptr;
    int32_t *order = nullptr, *flag0 = nullptr, *flag1 = nullptr, *f0_elem = nullptr;
    int32_t *ic = nullptr, *ik = nullptr;
    double *D = nullptr, *W0 = nullptr, *invW0 = nullptr, *pS = nullptr;
    int64_t nf0 = 0, dtot = 0, size = 0;
    int nblk = 0;

    SILH_REQ(X && labels && out, "null pointer argument");
    SILH_REQ(n >= 2 && n < (int64_t(1) << 31), "n must be in [2, 2^31)");
    SILH_REQ(d >= 1 && ld >= d, "need d >= 1 and ld >= d");
    SILH_REQ(k >= 2 && k <= SILH_MAX_K, "k must be in [2, %d]", SILH_MAX_K);
    SILH_REQ(out->k == k && out->sizes && out->offsets && out->idx && out->p,
             "silh_sample buffers missing or k mismatch");
    SILH_REQ(t > 0.0 && std::isfinite(t), "t must be positive");
    SILH_REQ(metric >= SILH_EUCLIDEAN && metric <= SILH_CANBERRA, "unknown metric");
    SILH_REQ(dtype == SILH_F32 || dtype == SILH_BF16, "unknown dtype");
    SILH_DEVPTR(X, "X");
    SILH_DEVPTR(labels, "labels");
    SILH_DEVPTR(out->sizes, "sample sizes");
    SILH_DEVPTR(out->offsets, "sample offsets");
    SILH_DEVPTR(out->idx, "sample idx");
    SILH_DEVPTR(out->p, "sample p");
    if (!(m0 > 0.0)) {
        SILH_REQ(delta > 0.0 && delta < 1.0, "delta must be in (0, 1)");
        m0 = 2.0 * std::log(5.0 * (double)k / delta);
    }
    SILH_CK(cudaGetDevice(&dev));
    ensure_pool_retains(dev);

    st = cluster_sort(labels, n, k, sc, stream, out->sizes, &coff, &order, h_sizes, h_coff);
    if (st != SILH_OK) goto done;
    nblk = ceil_div_i(n, 256);
    SILH_CK(sc.alloc(&flag0, n));
    SILH_CK(sc.alloc(&flag1, n));
    SILH_CK(sc.alloc(&pos0, n));
    SILH_CK(sc.alloc(&pos1, n));
    SILH_CK(sc.alloc(&tot, 2));
    SILH_CK(sc.alloc(&f0off, (size_t)k + 1));
    SILH_CK(sc.alloc(&pS, n));

    h_f0off.assign(k + 1, 0);
    if (!uniform) {
        k_draw_f0<<<nblk, 256, 0, stream>>>(order, labels, out->sizes, n, t, m0, seed,
                                            clustering_id, flag0); count_launches(1);
        SILH_CK(scan_flags(flag0, n, pos0, tot, sc, stream));
        k_seg_offsets<<<ceil_div_i(k + 1, 256), 256, 0, stream>>>(pos0, coff, k, n, tot, f0off); count_launches(1);
        SILH_CK(cudaGetLastError());
        SILH_CK(cudaMemcpyAsync(h_f0off.data(), f0off, sizeof(int64_t) * (k + 1),
                                cudaMemcpyDeviceToHost, stream));
        SILH_CK(cudaStreamSynchronize(stream));
        nf0 = h_f0off[k];
    } else {
        SILH_CK(cudaMemsetAsync(f0off, 0, sizeof(int64_t) * (k + 1), stream));
    }
    // Plan the member x F0 distance matrices and the work items.
    h_doff.assign(k + 1, 0);
    for (int j = 0; j < k; ++j) {
        int64_t nc = h_sizes[j], nf = h_f0off[j + 1] - h_f0off[j];
        h_doff[j + 1] = h_doff[j] + nc * nf;
        if (nf > 0)
            for (int64_t c = 0; c * kDistThreads < nc; ++c) {
                h_ic.push_back(j);
                h_ik.push_back((int32_t)c);
            }
    }
    dtot = h_doff[k];
    SILH_CK(sc.alloc(&doff, (size_t)k + 1));
    SILH_CK(cudaMemcpyAsync(doff, h_doff.data(), sizeof(int64_t) * (k + 1),
                            cudaMemcpyHostToDevice, stream));
    SILH_CK(sc.alloc(&D, (size_t)std::max<int64_t>(dtot, 1)));
    SILH_CK(sc.alloc(&W0, (size_t)std::max<int64_t>(nf0, 1)));
    SILH_CK(sc.alloc(&invW0, (size_t)std::max<int64_t>(nf0, 1)));
    SILH_CK(sc.alloc(&f0_elem, (size_t)std::max<int64_t>(nf0, 1)));
    if (nf0 > 0) {
        k_compact<<<nblk, 256, 0, stream>>>(flag0, pos0, order, n, f0_elem, nullptr, nullptr); count_launches(1);
        int nitems = (int)h_ic.size();
        SILH_CK(sc.alloc(&ic, nitems));
        SILH_CK(sc.alloc(&ik, nitems));
        SILH_CK(cudaMemcpyAsync(ic, h_ic.data(), sizeof(int32_t) * nitems, cudaMemcpyHostToDevice,
                                stream));
        SILH_CK(cudaMemcpyAsync(ik, h_ik.data(), sizeof(int32_t) * nitems, cudaMemcpyHostToDevice,
                                stream));
        size_t smem = sizeof(double) * kF0Group * (size_t)d;
        SILH_REQ(smem <= 200 * 1024, "d too large for Phase 1 (d <= 3200)");
        if (dtype == SILH_F32) {
            SILH_CK(dist_f0_smem_optin<float>(smem / 2));
            launch_dist_f0<float>(metric, nitems, smem, stream, (const float *)X, d, ld, order,
                                  coff, f0_elem, f0off, doff, ic, ik, D);
        } else {
            SILH_CK(dist_f0_smem_optin<__nv_bfloat16>(smem / 2));
            launch_dist_f0<__nv_bfloat16>(metric, nitems, smem, stream,
                                          (const __nv_bfloat16 *)X, d, ld, order, coff, f0_elem,
                                          f0off, doff, ic, ik, D);
        }
        SILH_CK(cudaGetLastError());
        k_w0<<<(int)nf0, 256, 0, stream>>>(f0_elem, labels, coff, f0off, doff, D, W0, invW0); count_launches(1);
        SILH_CK(cudaGetLastError());
    }
    k_gamma_draw<<<nblk, 256, 0, stream>>>(order, labels, coff, out->sizes, f0off, doff, D, invW0, n,
                                           t, uniform ? 1 : 0, seed, clustering_id, pS, flag1); count_launches(1);
    SILH_CK(scan_flags(flag1, n, pos1, tot + 1, sc, stream));
    SILH_CK(cudaMemcpyAsync(&size, tot + 1, sizeof(int64_t), cudaMemcpyDeviceToHost, stream));
    SILH_CK(cudaStreamSynchronize(stream));
    out->size = size;
    if (size > out->cap) {
        st = fail(SILH_ECAPACITY, "sample has %lld elements, capacity %lld", (long long)size,
                  (long long)out->cap);
        goto done;
    }
    k_compact<<<nblk, 256, 0, stream>>>(flag1, pos1, order, n, out->idx, pS, out->p); count_launches(1);
    k_seg_offsets<<<ceil_div_i(k + 1, 256), 256, 0, stream>>>(pos1, coff, k, n, tot + 1,
                                                              out->offsets); count_launches(1);
    SILH_CK(cudaGetLastError());
    SILH_CK(cudaStreamSynchronize(stream));
done:
    return st;
}

// Phase 1 with every size kept on the device: the same kernels and arithmetic as
// silh_sample_pps (so the same sample), planned by device kernels instead of the
// host, with scratch sized from n, k and m0.  The member x F0 distance matrices
// get n (m0 + 8 sqrt(m0) + 16) entries: |F0_j| exceeds m0 + 8 sqrt(m0) + 16 with
// probability below 1e-15 (Poisson tail), and a larger total only sets
// SILH_ECAPACITY in *d_status.
extern "C" silh_status silh_sample_pps_async(const void *X, silh_dtype dtype, int64_t n,
                                             int32_t d, int64_t ld, const int32_t *labels,
                                             int32_t k, silh_metric metric, double t, double m0,
                                             double delta, uint64_t seed, uint32_t clustering_id,
                                             int32_t uniform, silh_sample *out, int64_t *d_size,
                                             int32_t *d_status, void *stream_) {
    cudaStream_t stream = (cudaStream_t)stream_;
    silh_status st = SILH_OK;
    int dev = 0;
    Scratch sc(stream);
    int64_t *coff = nullptr, *pos0 = nullptr, *pos1 = nullptr, *tot = nullptr, *f0off = nullptr;
    int64_t *doff = nullptr, *item_base = nullptr, *tile_base = nullptr;
    int32_t *order = nullptr, *flag0 = nullptr, *flag1 = nullptr, *f0_elem = nullptr;
    int32_t *counts = nullptr, *bad = nullptr;
    double *D = nullptr, *W0 = nullptr, *invW0 = nullptr, *pS = nullptr;
    int64_t dcap = 0;
    int nblk = 0, tile = 0, ntiles = 0;
    size_t hsmem = 0;

    SILH_REQ(X && labels && out && d_size && d_status, "null pointer argument");
    SILH_REQ(n >= 2 && n < (int64_t(1) << 31), "n must be in [2, 2^31)");
    SILH_REQ(d >= 1 && ld >= d, "need d >= 1 and ld >= d");
    SILH_REQ(k >= 2 && k <= SILH_MAX_K, "k must be in [2, %d]", SILH_MAX_K);
    SILH_REQ(out->k == k && out->sizes && out->offsets && out->idx && out->p && out->cap >= 1,
             "silh_sample buffers missing, k mismatch or no capacity");
    SILH_REQ(t > 0.0 && std::isfinite(t), "t must be positive");
    SILH_REQ(metric >= SILH_EUCLIDEAN && metric <= SILH_CANBERRA, "unknown metric");
    SILH_REQ(dtype == SILH_F32 || dtype == SILH_BF16, "unknown dtype");
    SILH_DEVPTR(X, "X");
    SILH_DEVPTR(labels, "labels");
    SILH_DEVPTR(out->sizes, "sample sizes");
    SILH_DEVPTR(out->offsets, "sample offsets");
    SILH_DEVPTR(out->idx, "sample idx");
    SILH_DEVPTR(out->p, "sample p");
    SILH_DEVPTR(d_size, "d_size");
    SILH_DEVPTR(d_status, "d_status");
    if (!(m0 > 0.0)) {
        SILH_REQ(delta > 0.0 && delta < 1.0, "delta must be in (0, 1)");
        m0 = 2.0 * std::log(5.0 * (double)k / delta);
    }
    SILH_REQ((size_t)sizeof(double) * kF0Group * (size_t)d <= 200 * 1024,
             "d too large for Phase 1 (d <= 3200)");
    SILH_CK(cudaGetDevice(&dev));
    ensure_pool_retains(dev);
    dcap = uniform ? 1 : (int64_t)std::ceil((double)n * (m0 + 8.0 * std::sqrt(m0) + 16.0));
    tile = (k <= 512) ? 1024 : 8192;
    ntiles = (int)((n + tile - 1) / tile);
    hsmem = sizeof(int32_t) * (size_t)k;
    nblk = ceil_div_i(n, 256);
    SILH_CK(sc.alloc(&counts, (size_t)k * ntiles));
    SILH_CK(sc.alloc(&tile_base, (size_t)k * ntiles));
    SILH_CK(sc.alloc(&bad, 1));
    SILH_CK(sc.alloc(&coff, (size_t)k + 1));
    SILH_CK(sc.alloc(&order, (size_t)n));
    SILH_CK(sc.alloc(&flag0, n));
    SILH_CK(sc.alloc(&flag1, n));
    SILH_CK(sc.alloc(&pos0, n));
    SILH_CK(sc.alloc(&pos1, n));
    SILH_CK(sc.alloc(&tot, 2));
    SILH_CK(sc.alloc(&f0off, (size_t)k + 1));
    SILH_CK(sc.alloc(&doff, (size_t)k + 1));
    SILH_CK(sc.alloc(&item_base, (size_t)k + 1));
    SILH_CK(sc.alloc(&pS, n));
    SILH_CK(sc.alloc(&D, (size_t)dcap));
    SILH_CK(sc.alloc(&W0, n));
    SILH_CK(sc.alloc(&invW0, n));
    SILH_CK(sc.alloc(&f0_elem, n));
    SILH_CK(cudaMemsetAsync(bad, 0, sizeof(int32_t), stream));
    SILH_CK(cudaMemsetAsync(d_status, 0, sizeof(int32_t), stream));
    if (hsmem > 48 * 1024) {
        SILH_CK(cudaFuncSetAttribute(k_tile_hist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)hsmem));
        SILH_CK(cudaFuncSetAttribute(k_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)hsmem));
    }
    // cluster bookkeeping: sizes, offsets (validated on the device), stable order
    k_tile_hist<<<ntiles, 32 * kHistWarps, hsmem, stream>>>(labels, n, k, tile, ntiles, counts, bad);
    k_cluster_scan<<<k, 256, 0, stream>>>(counts, ntiles, tile_base, out->sizes);
    k_coff_async<<<1, 1024, 0, stream>>>(out->sizes, k, bad, coff, d_status);
    k_scatter<<<ntiles, 32, hsmem, stream>>>(labels, n, k, tile, ntiles, tile_base, coff, order);
    count_launches(4);
    SILH_CK(cudaGetLastError());
    if (!uniform) {
        // initial sample, its offsets, the device plan of the distance matrices
        k_draw_f0<<<nblk, 256, 0, stream>>>(order, labels, out->sizes, n, t, m0, seed,
                                            clustering_id, flag0, d_status);
        count_launches(1);
        SILH_CK(scan_flags(flag0, n, pos0, tot, sc, stream));
        k_seg_offsets<<<ceil_div_i(k + 1, 256), 256, 0, stream>>>(pos0, coff, k, n, tot, f0off,
                                                                  d_status);
        k_plan_f0<<<1, 1024, 0, stream>>>(coff, f0off, k, dcap, doff, item_base, d_status);
        k_compact<<<nblk, 256, 0, stream>>>(flag0, pos0, order, n, f0_elem, nullptr, nullptr,
                                            d_status);
        count_launches(3);
        const size_t smem = sizeof(double) * kF0Group * (size_t)d;
        const int items_cap = ceil_div_i(n, kDistThreads) + k;
        if (dtype == SILH_F32) {
            SILH_CK(dist_f0_smem_optin<float>(smem / 2));
            launch_dist_f0<float>(metric, items_cap, smem, stream, (const float *)X, d, ld, order,
                                  coff, f0_elem, f0off, doff, nullptr, nullptr, D, item_base, k,
                                  d_status);
        } else {
            SILH_CK(dist_f0_smem_optin<__nv_bfloat16>(smem / 2));
            launch_dist_f0<__nv_bfloat16>(metric, items_cap, smem, stream,
                                          (const __nv_bfloat16 *)X, d, ld, order, coff, f0_elem,
                                          f0off, doff, nullptr, nullptr, D, item_base, k,
                                          d_status);
        }
        k_w0<<<(int)std::min<int64_t>(n, 148 * 16), 256, 0, stream>>>(
            f0_elem, labels, coff, f0off, doff, D, W0, invW0, tot, d_status);
        count_launches(1);
        SILH_CK(cudaGetLastError());
    } else {
        SILH_CK(cudaMemsetAsync(f0off, 0, sizeof(int64_t) * (k + 1), stream));
    }
    k_gamma_draw<<<nblk, 256, 0, stream>>>(order, labels, coff, out->sizes, f0off, doff, D, invW0,
                                           n, t, uniform ? 1 : 0, seed, clustering_id, pS, flag1,
                                           d_status);
    count_launches(1);
    SILH_CK(scan_flags(flag1, n, pos1, tot + 1, sc, stream));
    k_finish_size<<<1, 1, 0, stream>>>(tot + 1, out->cap, d_size, d_status);
    k_compact<<<nblk, 256, 0, stream>>>(flag1, pos1, order, n, out->idx, pS, out->p, d_status);
    k_seg_offsets<<<ceil_div_i(k + 1, 256), 256, 0, stream>>>(pos1, coff, k, n, tot + 1,
                                                              out->offsets, d_status);
    count_launches(3);
    SILH_CK(cudaGetLastError());
done:
    return st;
}
