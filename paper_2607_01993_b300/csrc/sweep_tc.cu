// Tensor-core Phase-2 / exact sweep for the Euclidean and cosine distances.
//
// The inner products x.y of a 128-row tile against a 64-column tile of the
// cluster-major sample are one tcgen05 MMA chain (FP32 accumulate in tensor
// memory).  SILH_PREC_3XTF32 splits every operand into a TF32 head and an
// FP32 tail (x = hi + lo, kind::tf32) and accumulates hi.hi + hi.lo + lo.hi,
// which leaves an inner-product error of a few 2^-22 |x||y|; SILH_PREC_TF32
// uses the heads only.  SILH_PREC_BF16X3 / SILH_PREC_BF16 do the same with
// BF16 heads and BF16 tails (kind::f16; x = hi + lo to ~2^-17, so an
// inner-product error of ~2^-17 |x||y|), or BF16 heads only (2^-8).  Both
// operand kinds fill 128-byte shared-memory rows (32 TF32 or 64 BF16
// elements), so the layouts, TMA boxes and descriptors are shared; each MMA
// consumes 32 bytes of K (8 TF32 or 16 BF16 elements).  The epilogue turns each inner product into a distance
//   Euclidean: d = sqrt(|x|^2 + |y|^2 - 2 x.y)   cosine: d = 1 - x^.y^
// multiplies by the inclusion weight 1/p and adds it to the running sum of the
// current cluster (Algorithm 1, Phase 2); W_hat never leaves the SM.  Pairs
// whose distance is small against the magnitudes that cancel in it
// (Euclidean: d^2 < tau (|x|^2 + |y|^2); cosine: d < tau) are recomputed
// directly in FP32 from the coordinates, so close pairs (mostly a row's own
// cluster) keep FP32 relative accuracy.
//
// Roles (one persistent CTA per SM, 6 warps): warp 0 issues TMA loads of the
// row tile and of the column tiles into a ring of shared-memory stages, warp 1
// issues the MMAs into two TMEM accumulators (so the MMA of tile t+1 overlaps
// the epilogue of tile t), warps 2-5 (128 threads, one per row / TMEM lane) run
// the epilogue.  Every wait is bounded; on a timeout the CTA records an error
// and stops.
//
// Rows are processed in cluster-sorted order so that a warp's rows share their
// own cluster and the recompute branch rarely diverges.
//
// Many clusterings of one dataset run as one persistent launch (BATCH): each
// gets its own sorted rows and padded columns in shared buffers, and the
// kernel's work items become (clustering, row group) pairs.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>

#include "kernels.cuh"
#include "tc_util.cuh"

namespace silh {

namespace {

using namespace tc;

constexpr int kTileM = 128;       // rows per tile = TMEM lanes
constexpr int kTileN = 64;        // columns per tile
constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s per wait

__device__ int g_tc_error = 0;    // set when a bounded wait gives up

#define SMEM_CHECK(bytes) ((bytes) + 1024 <= 200 * 1024)

// KD: padded FP32 row length (32 or 64); BF: BF16 operands (one 128-byte K
// block of 64 elements) instead of TF32 (KD / 32 blocks of 32 elements).
// WIDE: 128-column tiles (one MMA covers N = 128, so each read of the 128-row
// A tile from shared memory serves twice the columns) with one accumulator
// per slot where two would not fit in tensor memory; otherwise 64-column
// tiles, two accumulators per slot.
// Row tiles a CTA sweeps at once (each with its own epilogue warpgroup and
// accumulators): four where a row is one 128-byte K block (BF16 operands, or
// TF32 rows of 32 elements), two for two-block TF32 rows.  (Two slots for
// one-block rows, with deeper B staging and two accumulators per slot, were
// slower: fewer epilogue warps per column tile.)
__host__ __device__ constexpr int tc_slots(int KD, bool BF) { return (BF || KD == 32) ? 4 : 2; }

// Close-pair recompute form: rows of 32 elements evaluate a flagged chunk's
// 32 x 32 pairs with one column per lane, from lane-interleaved FP32 copies of
// rows and columns; 64-element rows recompute only the flagged pairs, each lane
// its own row from the row-major operands (there, typically one lane of a chunk
// is flagged, and a whole row-major row is two cache lines where its
// interleaved form is sixteen).
__host__ __device__ constexpr bool tc_col_redo(int KD) { return KD == 32; }
// 64-element rows: a chunk whose close pairs average more than this many per
// marked column is recomputed lane by lane (each lane its row, the marked
// columns one after another), else pair by pair with the whole warp.  For
// TF32 operands (a row is hi + lo, two loads per coordinate) the pair-by-pair
// form measured faster at every density, so the threshold is never reached.
__host__ __device__ constexpr uint32_t coop_pairs_per_column(bool bf) { return bf ? 12u : 33u; }

template <int KD, bool SPLIT, bool BF = false, bool WIDE = false>
struct TcCfg {
    static constexpr int KB = BF ? 1 : KD / 32;                 // 128-byte K blocks
    static constexpr int KSTEPS = BF ? KD / 16 : 4;             // 32-byte MMA K steps per block
    static constexpr int KELEM = BF ? 64 : 32;                  // elements per 128-byte row
    static constexpr int PARTS = SPLIT ? 2 : 1;                 // hi (+ lo)
    static constexpr int SLOTS = tc_slots(KD, BF);              // row tiles per CTA pass
    static constexpr int TN = WIDE ? 128 : kTileN;              // columns per tile
    static constexpr int NACC = (SLOTS * 2 * TN <= 512) ? 2 : 1;  // accumulators per slot
    static constexpr int A_SLOT = PARTS * KB * kTileM * 128;
    static constexpr int A_BYTES = SLOTS * A_SLOT;
    static constexpr int B_BYTES = PARTS * KB * TN * 128;       // one stage
    static constexpr int STAGES_FIT = (199 * 1024 - A_BYTES) / B_BYTES;
    static constexpr int STAGES = WIDE ? (STAGES_FIT < 8 ? STAGES_FIT : 8)
                                       : ((KB == 1) ? (SPLIT ? 4 : 8) : (SPLIT ? 2 : 4));
    static_assert(STAGES >= 2, "fewer than two B stages fit");
    static_assert(SMEM_CHECK(A_BYTES + STAGES * B_BYTES), "dynamic shared memory over budget");
    static constexpr int SMEM = 1024 + A_BYTES + STAGES * B_BYTES;
    static constexpr int THREADS = 64 + 128 * SLOTS;            // TMA, MMA, epilogue groups
    static constexpr uint32_t TMEM_COLS = SLOTS * NACC * TN;
};

__device__ __forceinline__ float sqrt_apx(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Distance of a row (row-major; TF32 operands: x = hi + lo exactly, BF16
// operands and the symmetric layout: xh is the FP32 row and xl is unused) to a
// column (y, global), directly from the coordinates in FP32.
template <int METRIC, int KD, bool FULL>
__device__ __noinline__ float direct_dist_rows(const float *__restrict__ xh,
                                               const float *__restrict__ xl,
                                               const float *__restrict__ y) {
    const float4 *y4 = reinterpret_cast<const float4 *>(y);
    const float4 *h4 = reinterpret_cast<const float4 *>(xh);
    const float4 *l4 = reinterpret_cast<const float4 *>(xl);
    float a0 = 0.f, a1 = 0.f;
#pragma unroll 4
    for (int q = 0; q < KD / 4; ++q) {
        const float4 v = __ldg(y4 + q), h = __ldg(h4 + q);
        const float4 l = FULL ? make_float4(0.f, 0.f, 0.f, 0.f) : __ldg(l4 + q);
        const float t0 = (h.x + l.x) - v.x, t1 = (h.y + l.y) - v.y;
        const float t2 = (h.z + l.z) - v.z, t3 = (h.w + l.w) - v.w;
        a0 = fmaf(t0, t0, a0); a1 = fmaf(t1, t1, a1);
        a0 = fmaf(t2, t2, a0); a1 = fmaf(t3, t3, a1);
    }
    const float s = a0 + a1;
    return METRIC == SILH_EUCLIDEAN ? sqrtf(s) : 0.5f * s;
}

// Lane-interleaved FP32 copy of a row or column operand (the dense close-pair
// recompute of 32-element rows reads it): rows in blocks of 32 (one epilogue
// warp), element c of row r at
//   il[(r / 32) * 32 KD + (c / 4) * 128 + (r % 32) * 4 + c % 4],
// so a warp reading four elements of one row (every lane the same row) or of
// its 32 rows (every lane its own) touches consecutive bytes.  For TF32
// operands the values are hi + lo.  il_index gives that position.
__device__ __forceinline__ int64_t il_index(int64_t r, int c, int KD) {
    return (r >> 5) * (int64_t)(KD * 32) + (c >> 2) * 128 + (r & 31) * 4 + (c & 3);
}

// Fast-path epilogue of 16 accumulator columns (inner products r) of one row,
// two columns per packed two-lane FP32 instruction: part += sum w d, and the
// sign bit of flag is set when a pair needs the direct recompute (Euclidean:
// d^2 - tau (|x|^2 + |y|^2) < 0, OR-ed over the raw bits of that difference;
// cosine: d - tau < 0).  wn4 holds (w_2i, w_2i+1, |y_2i|^2, |y_2i+1|^2).
template <int METRIC>
__device__ __forceinline__ void half_chunk(const uint32_t (&r)[16], const float4 *wn4, float xn,
                                           float tau, float &part, uint32_t &flag) {
    float2 acc0 = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
    float dmin = INFINITY;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float4 wn = wn4[i];
        const float2 v = make_float2(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]));
        float2 d;
        if (METRIC == SILH_EUCLIDEAN) {
            const float2 s = __fadd2_rn(make_float2(xn, xn), make_float2(wn.z, wn.w));
            const float2 q = __ffma2_rn(make_float2(-2.f, -2.f), v, s);
            const float2 f = __ffma2_rn(make_float2(-tau, -tau), s, q);
            flag |= __float_as_uint(f.x) | __float_as_uint(f.y);
            d = make_float2(sqrt_apx(q.x), sqrt_apx(q.y));
        } else {
            d = __ffma2_rn(v, make_float2(-1.f, -1.f), make_float2(1.f, 1.f));   // 1 - x^.y^
            dmin = fminf(dmin, fminf(d.x, d.y));
        }
        if (i & 1) acc1 = __ffma2_rn(make_float2(wn.x, wn.y), d, acc1);
        else acc0 = __ffma2_rn(make_float2(wn.x, wn.y), d, acc0);
    }
    if (METRIC == SILH_COSINE) flag |= __float_as_uint(dmin - tau);
    part += (acc0.x + acc0.y) + (acc1.x + acc1.y);
}

// half_chunk for the symmetric exact sweep: also returns, for the column
// `col` this lane ends up holding, the sum over the warp's 32 rows of d times
// the row weight rw (1 for a point, 0 for padding) -- the column side of the
// pairs; lanes with an odd index hold a duplicate.
template <int METRIC>
__device__ __forceinline__ float half_chunk_sym(const uint32_t (&r)[16], const float4 *wn4,
                                                float xn, float tau, float rw, int lane,
                                                float &part, uint32_t &flag, int &col) {
    float2 acc0 = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
    float cs[16];
    float dmin = INFINITY;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float4 wn = wn4[i];
        const float2 v = make_float2(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]));
        float2 d;
        if (METRIC == SILH_EUCLIDEAN) {
            const float2 s = __fadd2_rn(make_float2(xn, xn), make_float2(wn.z, wn.w));
            const float2 q = __ffma2_rn(make_float2(-2.f, -2.f), v, s);
            const float2 f = __ffma2_rn(make_float2(-tau, -tau), s, q);
            flag |= __float_as_uint(f.x) | __float_as_uint(f.y);
            d = make_float2(sqrt_apx(q.x), sqrt_apx(q.y));
        } else {
            d = __ffma2_rn(v, make_float2(-1.f, -1.f), make_float2(1.f, 1.f));   // 1 - x^.y^
            dmin = fminf(dmin, fminf(d.x, d.y));
        }
        if (i & 1) acc1 = __ffma2_rn(make_float2(wn.x, wn.y), d, acc1);
        else acc0 = __ffma2_rn(make_float2(wn.x, wn.y), d, acc0);
        cs[2 * i] = d.x * rw;
        cs[2 * i + 1] = d.y * rw;
    }
    if (METRIC == SILH_COSINE) flag |= __float_as_uint(dmin - tau);
    part += (acc0.x + acc0.y) + (acc1.x + acc1.y);
    return transpose_reduce<16>(cs, lane, col);
}

// Column layout: cluster j occupies padded columns [poff[j], poff[j+1]), its
// |F_j| sampled columns first, then zero columns of weight 0 up to a multiple
// of 32, so every 32-column chunk belongs to exactly one cluster.
//
// SYM (the exact silhouette over all points, rows = columns in the padded
// layout): each unordered pair is evaluated once.  A row group streams only
// the column tiles from its own first row on, split into work items of about
// equal length (sym_work: row group, first tile, end tile); a warp's 32-row
// block takes a 32-column chunk only when the chunk lies entirely after the
// block (blocks are 32-aligned and never straddle clusters, so the diagonal
// blocks are own cluster pairs, which the direct pass covers).  Row sums per
// cluster and the column sums (per column, over the warp's rows, which share
// one cluster) are added to W (FP64, position x cluster); a separate pass forms
// s, a, b.
//
// BATCH (many clusterings of one dataset in one launch): clustering b has its
// own cluster-sorted row operand, rows [arow, arow + nrows) of the shared row
// buffers (zero padded to whole row groups), its own padded column range from
// column ccol (a multiple of the tile width, zero padded to whole tiles), its
// padded cluster offsets at poff + pbase, its cluster sizes and its output.
// Work items are (clustering, row group), numbered clustering by clustering
// from work_base; each is swept exactly as the single-clustering kernel sweeps
// that row group, so a batched result equals the single call's bit for bit.
struct TcItem {
    int64_t work_base;
    int64_t arow;
    int64_t ccol;
    int64_t nrows;
    int64_t pbase;
    const int64_t *sizes;
    float *s_out;
    int32_t k;
    int32_t pad_;
};
// Close pairs of 64-element rows, deferred from the sweep's epilogue: a lane
// whose chunk holds close pairs records them (the row, the chunk's first
// operand column, the mask of close columns) instead of evaluating them, and
// the cluster they belong to is "dirty" for that row: at its end the partial
// W_hat_j (without those pairs) is recorded too (mask 0), in a slot reserved
// with the cluster's first record.  Each row's records are chained (prev), in
// the order the sweep met them.  A row with any dirty cluster leaves its
// running minimum over the clean clusters in a row record instead of its
// outputs.  k_defer_fix then evaluates every recorded chunk's close pairs
// directly in FP32, and k_defer_final walks each dirty row's chain in a fixed
// order, completes its dirty clusters, merges them into the minimum and writes
// the outputs -- so results are deterministic and a batched item equals its
// single call.  Lanes beyond the record capacity evaluate their pairs in the
// epilogue as before.
struct TcDeferEntry {
    int32_t row;       // operand row
    int32_t col;       // first operand column of the chunk
    uint32_t mask;     // close columns of the chunk; 0: the end of a dirty cluster
    int32_t prev;      // the row's previous record, -1 for its first
    int32_t j;         // the cluster
    int32_t pad_;
    double val;        // chunk: sum of w d over its close pairs; end: partial W_hat_j
};
struct TcDeferRow {
    double bacc, bsize;    // minimum over the clean clusters of W_hat_j / |Cj| (as RatioMin)
    int32_t barg, head;    // its cluster; the row's last record
    int32_t row, item;     // operand row; clustering (batched) or 0
    int64_t out;           // output index
};
struct TcDefer {
    TcDeferEntry *ent;          // nullptr: no deferral (the epilogue evaluates close pairs)
    TcDeferRow *rec;
    unsigned long long *ctr;    // [0] records reserved, [1] dirty rows
    int64_t ent_cap, rec_cap;
    int64_t nrows_ops, ncols_ops;   // rows and columns of the operands (bounds of the records)
};

constexpr int kMaxTcBatch = 256;
// Column tiles of (w, |y|^2) the producer may stage ahead of the epilogue.
constexpr int kWnRing = 8;
// Device memory of one batched launch's operands; a batch that needs more is
// split into several launches (a single clustering always fits one).
constexpr size_t kTcBatchBytes = size_t(16) << 30;
template <bool BATCH>
struct TcBatchArg {            // one clustering: everything is in the kernel arguments
    int32_t unused;
};
template <>
struct TcBatchArg<true> {
    int32_t nitems;
    int64_t total_work;
    TcItem items[kMaxTcBatch];
};

__device__ __forceinline__ int64_t bt_total_work(const TcBatchArg<false> &) { return 0; }
__device__ __forceinline__ int64_t bt_total_work(const TcBatchArg<true> &b) { return b.total_work; }

// NB: the instantiation that also writes the neighbouring cluster (its
// running argmin is a register the others do without).
template <int METRIC, int KD, bool SPLIT, bool BF, bool SYM = false, bool WIDE = false,
          bool BATCH = false, bool NB = false>
__global__ void __launch_bounds__(TcCfg<KD, SPLIT, BF, WIDE>::THREADS, 1)
k_sweep_tc(const __grid_constant__ CUtensorMap m_ahi, const __grid_constant__ CUtensorMap m_alo,
           const __grid_constant__ CUtensorMap m_bhi, const __grid_constant__ CUtensorMap m_blo,
           const float *__restrict__ a_hi, const float *__restrict__ a_lo,
           const float *__restrict__ a_il,
           const float *__restrict__ a_norm, const int32_t *__restrict__ a_lab,
           const int64_t *__restrict__ a_out, int64_t nrows, const float *__restrict__ y_full,
           const float *__restrict__ y_il,
           const float2 *__restrict__ y_wn, const float4 *__restrict__ y_wn4,
           const int64_t *__restrict__ poff,
           const int64_t *__restrict__ sizes, int k, float tau, int dq,
           const double *__restrict__ w_own, float *__restrict__ s_out,
           float *__restrict__ a_out_v, float *__restrict__ b_out_v,
           int32_t *__restrict__ nb_out_v, double *__restrict__ W,
           const int4 *__restrict__ sym_work, int64_t n_sym_work, const TcDefer df,
           const __grid_constant__ TcBatchArg<BATCH> bt) {
    static_assert(!(BATCH && SYM), "the symmetric exact sweep is not batched");
    using C = TcCfg<KD, SPLIT, BF, WIDE>;
    constexpr int TN = C::TN;
    constexpr bool kColRedo = tc_col_redo(KD);
    constexpr bool kDefer = !SYM && !kColRedo;    // 64-element rows may defer close pairs
    // 32-element rows: the accumulator is released after the tile's last
    // tensor-memory load, before that chunk's arithmetic (64-element rows
    // re-read a flagged chunk from tensor memory; keeping the last chunk's
    // products in registers for that instead measured slower)
    constexpr bool kEarlyRelease = kColRedo;
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t bar_full[C::STAGES], bar_empty[C::STAGES];
    __shared__ uint64_t bar_afull, bar_aempty, bar_accf[C::SLOTS][C::NACC], bar_acce[C::SLOTS][C::NACC];
    __shared__ uint64_t bar_drain;      // the MMA issuer's last commit, after an abort
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;
    // (w, |y|^2) of the column tiles in flight: a ring of kWnRing tiles that the
    // producer fills by bulk copies from y_wn4, two columns per float4 as
    // (w_2i, w_2i+1, n_2i, n_2i+1) so that the epilogue reads lane pairs; a
    // slot is refilled once every epilogue warp has released it
    __shared__ __align__(16) float4 sh_wn[kWnRing][TN / 2];
    __shared__ uint64_t bar_wnf[kWnRing], bar_wne[kWnRing];

    const uint32_t raw = smem_u32(smem_raw);
    uint8_t *sm = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    uint8_t *sA = sm;                   // [slot][part][kb][128 rows][128 B]
    uint8_t *sB = sm + C::A_BYTES;      // [stage][part][kb][128 cols][128 B]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ngroups = BATCH ? bt_total_work(bt)
                          : SYM   ? n_sym_work
                                  : ((nrows + kTileM - 1) / kTileM + C::SLOTS - 1) / C::SLOTS;
    // Work item w as (clustering, row group): its row group rg, the first row
    // (arow) and column (ccol) of its clustering in the operands, the row
    // count, padded cluster offsets, sizes, cluster count, output, the padded
    // column count mp with its column-tile count nct, and the column tiles
    // [ct_b, ct_e) the item sweeps: all of them, or for SYM one segment of the
    // row group's triangle (sym_work[w] = (row group, first tile, end tile)).
    struct View {
        int64_t rg, arow, ccol, nrows, mp, nct, ct_b, ct_e;
        const int64_t *poff, *sizes;
        float *s_out;
        int k, item;
    };
    auto view_of = [&](int64_t w) -> View {
        View v;
        if constexpr (BATCH) {
            int lo = 0, hi = bt.nitems - 1;           // last clustering with work_base <= w
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (bt.items[mid].work_base <= w) lo = mid;
                else hi = mid - 1;
            }
            const TcItem &it = bt.items[lo];
            v.rg = w - it.work_base;
            v.arow = it.arow;
            v.ccol = it.ccol;
            v.nrows = it.nrows;
            v.poff = poff + it.pbase;
            v.sizes = it.sizes;
            v.s_out = it.s_out;
            v.k = it.k;
            v.item = lo;
        } else {
            v.rg = w;
            v.arow = 0;
            v.ccol = 0;
            v.nrows = nrows;
            v.poff = poff;
            v.sizes = sizes;
            v.s_out = s_out;
            v.k = k;
            v.item = 0;
        }
        v.mp = v.poff[v.k];
        v.nct = (v.mp + TN - 1) / TN;
        v.ct_b = 0;
        v.ct_e = v.nct;
        if constexpr (SYM) {
            const int4 e = sym_work[w];
            v.rg = e.x;
            v.ct_b = e.y;
            v.ct_e = e.z;
        }
        return v;
    };
    // Work item of this CTA's it-th round: blockIdx.x + it * gridDim.x; -1
    // when the round has none for it, -2 past the last round.
    auto group_of = [&](int64_t it) -> int64_t {
        const int64_t base = it * gridDim.x;
        if (base >= ngroups) return -2;
        const int64_t w = base + blockIdx.x;
        return w < ngroups ? w : -1;
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; ++s) {
            mbar_init(&bar_full[s], 1);
            mbar_init(&bar_empty[s], 1);
        }
        mbar_init(&bar_afull, 1);
        mbar_init(&bar_aempty, 1);
        mbar_init(&bar_drain, 1);
        for (int g = 0; g < C::SLOTS; ++g)
            for (int a = 0; a < C::NACC; ++a) {
                mbar_init(&bar_accf[g][a], 1);
                mbar_init(&bar_acce[g][a], 4);
            }
        for (int r = 0; r < kWnRing; ++r) {
            mbar_init(&bar_wnf[r], 1);
            mbar_init(&bar_wne[r], 4 * C::SLOTS);
        }
        abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) tmem_alloc(&tmem_base, C::TMEM_COLS);
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = tmem_base;
    // TMA loads the producer thread has issued: per B stage whether one was and
    // the phase parity it completes, and the same for the A tile (drained on abort)
    uint32_t ld_issued = 0, ld_parity = 0;
    bool a_issued = false;
    uint32_t a_parity = 0;
    uint32_t wn_issued = 0, wn_parity = 0;    // the same for the (w, |y|^2) ring
    static_assert(C::STAGES <= 32 && kWnRing <= 32, "stage masks are 32-bit");

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            tma_prefetch_desc(&m_ahi);
            tma_prefetch_desc(&m_bhi);
            if (SPLIT) {
                tma_prefetch_desc(&m_alo);
                tma_prefetch_desc(&m_blo);
            }
            int stage = 0;
            uint32_t phase = 0;
            int64_t idx = 0;
            uint64_t wt = 0;                      // column tiles staged into the ring so far
            for (int64_t it = 0; !abort_flag; ++it) {
                const int64_t w = group_of(it);
                if (w == -2) break;
                if (w < 0) continue;
                const View v = view_of(w);
                const int64_t rg = v.rg;
                if (idx > 0 && !mbar_wait(&bar_aempty, (uint32_t)((idx - 1) & 1), kWaitNs)) {
                    abort_flag = 1;
                    break;
                }
                mbar_expect_tx(&bar_afull, C::A_BYTES);
                a_issued = true;
                a_parity = (uint32_t)(idx & 1);
                for (int g = 0; g < C::SLOTS; ++g) {
                    const int y = (int)(v.arow + (rg * C::SLOTS + g) * kTileM);
                    uint8_t *a = sA + g * C::A_SLOT;
                    for (int kb = 0; kb < C::KB; ++kb) {
                        tma_load_2d(&m_ahi, &bar_afull, a + kb * kTileM * 128, kb * C::KELEM, y);
                        if (SPLIT)
                            tma_load_2d(&m_alo, &bar_afull, a + (C::KB + kb) * kTileM * 128,
                                        kb * C::KELEM, y);
                    }
                }
                for (int64_t ct = v.ct_b; ct < v.ct_e; ++ct) {
                    if (!mbar_wait(&bar_empty[stage], phase ^ 1u, kWaitNs)) {
                        abort_flag = 1;
                        break;
                    }
                    uint8_t *dst = sB + stage * C::B_BYTES;
                    mbar_expect_tx(&bar_full[stage], C::B_BYTES);
                    ld_issued |= 1u << stage;
                    ld_parity = (ld_parity & ~(1u << stage)) | (phase << stage);
                    for (int kb = 0; kb < C::KB; ++kb) {
                        tma_load_2d(&m_bhi, &bar_full[stage], dst + kb * TN * 128,
                                    kb * C::KELEM, (int)(v.ccol + ct * TN));
                        if (SPLIT)
                            tma_load_2d(&m_blo, &bar_full[stage],
                                        dst + (C::KB + kb) * TN * 128, kb * C::KELEM,
                                        (int)(v.ccol + ct * TN));
                    }
                    if (++stage == C::STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                    // this tile's (w, |y|^2) into ring slot ws, once every
                    // epilogue warp has released the tile kWnRing earlier
                    const int ws = (int)(wt % kWnRing);
                    const uint32_t wpar = (uint32_t)((wt / kWnRing) & 1);
                    if (wt >= (uint64_t)kWnRing && !mbar_wait(&bar_wne[ws], wpar ^ 1u, kWaitNs)) {
                        abort_flag = 1;
                        break;
                    }
                    mbar_expect_tx(&bar_wnf[ws], TN * 8);
                    wn_issued |= 1u << ws;
                    wn_parity = (wn_parity & ~(1u << ws)) | (wpar << ws);
                    bulk_load(&sh_wn[ws][0], y_wn4 + (v.ccol + ct * TN) / 2, TN * 8, &bar_wnf[ws]);
                    ++wt;
                }
                ++idx;
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = BF ? idesc_bf16(kTileM, TN) : idesc_tf32(kTileM, TN);
            const uint64_t adesc0 = sw128_kmajor_desc(smem_u32(sA));
            const uint64_t bdesc0 = sw128_kmajor_desc(smem_u32(sB));
            int stage = 0;
            uint32_t phase = 0, acc = 0, acc_phase = 0;
            int64_t idx = 0;
            for (int64_t it = 0; !abort_flag; ++it) {
                const int64_t w = group_of(it);
                if (w == -2) break;
                if (w < 0) continue;
                const View v = view_of(w);
                if (!mbar_wait(&bar_afull, (uint32_t)(idx & 1), kWaitNs)) {
                    abort_flag = 1;
                    break;
                }
                for (int64_t ct = v.ct_b; ct < v.ct_e; ++ct) {
                    if (!mbar_wait(&bar_full[stage], phase, kWaitNs)) {
                        abort_flag = 1;
                        break;
                    }
                    // descriptors differ from the stage / slot bases only in the
                    // start-address field (bits 0-13, address >> 4), so each one
                    // is a base plus a compile-time offset
                    const uint64_t bd = bdesc0 + (uint64_t)((stage * C::B_BYTES) >> 4);
                    bool ok = true;
#pragma unroll
                    for (int g = 0; g < C::SLOTS; ++g) {
                        if (!mbar_wait(&bar_acce[g][acc], acc_phase ^ 1u, kWaitNs)) {
                            ok = false;
                            break;
                        }
                        fence_after_sync();
                        const uint32_t d_tmem = tmem + (uint32_t)(g * C::NACC + acc) * TN;
                        const uint64_t ad = adesc0 + (uint64_t)((g * C::A_SLOT) >> 4);
#pragma unroll
                        for (int kb = 0; kb < C::KB; ++kb) {
#pragma unroll
                            for (int ks = 0; ks < C::KSTEPS; ++ks) {
                                const uint32_t first = (kb == 0 && ks == 0) ? 0u : 1u;
                                const uint64_t ahi = ad + (uint64_t)((kb * kTileM * 128 + ks * 32) >> 4);
                                const uint64_t bhi = bd + (uint64_t)((kb * TN * 128 + ks * 32) >> 4);
                                if (SPLIT) {
                                    const uint64_t alo =
                                        ad + (uint64_t)(((C::KB + kb) * kTileM * 128 + ks * 32) >> 4);
                                    const uint64_t blo =
                                        bd + (uint64_t)(((C::KB + kb) * TN * 128 + ks * 32) >> 4);
                                    if (BF) {
                                        mma_bf16(d_tmem, alo, bhi, idesc, first);
                                        mma_bf16(d_tmem, ahi, blo, idesc, 1);
                                        mma_bf16(d_tmem, ahi, bhi, idesc, 1);
                                    } else {
                                        mma_tf32(d_tmem, alo, bhi, idesc, first);
                                        mma_tf32(d_tmem, ahi, blo, idesc, 1);
                                        mma_tf32(d_tmem, ahi, bhi, idesc, 1);
                                    }
                                } else {
                                    if (BF) mma_bf16(d_tmem, ahi, bhi, idesc, first);
                                    else mma_tf32(d_tmem, ahi, bhi, idesc, first);
                                }
                            }
                        }
                        mma_commit(&bar_accf[g][acc]);
                    }
                    if (!ok) {
                        abort_flag = 1;
                        break;
                    }
                    mma_commit(&bar_empty[stage]);
                    if (++stage == C::STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                    acc = (acc + 1 == (uint32_t)C::NACC) ? 0u : acc + 1;
                    if (acc == 0) acc_phase ^= 1u;
                }
                mma_commit(&bar_aempty);
                ++idx;
                if (abort_flag) break;
            }
            // The last A-release arrival must land before the CTA exits.
            if (!abort_flag && idx > 0 &&
                !mbar_wait(&bar_aempty, (uint32_t)((idx - 1) & 1), kWaitNs))
                abort_flag = 1;
        }
    } else {
        // ------------------------------------------------ epilogue groups
        const int g = (warp - 2) >> 2;          // row-tile slot of this group
        const int q = warp & 3;                 // TMEM lane quarter of this warp
        const int r_local = 32 * q + lane;
        const uint32_t tlane = (uint32_t)(32 * q) << 16;
        uint32_t acc = 0, acc_phase = 0;
        uint64_t wt = 0;                         // column tiles consumed from the ring so far
        for (int64_t it = 0;; ++it) {
            const int64_t w = group_of(it);
            if (w == -2) break;
            if (w < 0) continue;
            const View v = view_of(w);
            const int64_t rg = v.rg;
            const int64_t ct_end = v.ct_e;
            const int64_t *vpoff = v.poff;
            const int vk = v.k;
            const int64_t pos = (rg * C::SLOTS + g) * kTileM + r_local;   // within the clustering
            const bool valid = pos < v.nrows;
            const int64_t apos = v.arow + pos;                            // row of the operands
            const int own = valid ? a_lab[apos] : -1;
            const float xn = valid ? a_norm[apos] : 0.f;
            if (!kColRedo && valid) {
                // the row-form recompute reads this row's FP32 coordinates (hi and,
                // for TF32 operands, lo): bring them into L2 now, so that a close
                // pair later in the sweep does not wait on DRAM for them
                const float *xr = a_hi + apos * KD;
                asm volatile("prefetch.global.L2 [%0];" ::"l"(xr));
                asm volatile("prefetch.global.L2 [%0];" ::"l"(xr + 32));
                if (!(BF || SYM)) {
                    const float *lr = a_lo + apos * KD;
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(lr));
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(lr + 32));
                }
            }
            // the warp's block of 32 rows in the lane-interleaved FP32 copy (for
            // the direct recompute; a warp past the last row never recomputes)
            const int64_t blk0 = pos - lane;
            const float *xblk =
                kColRedo ? a_il + il_index(v.arow + (blk0 < v.nrows ? blk0 : 0), 0, KD) : nullptr;
            // SYM: this warp's 32-row block starts at wblk; rows are the padded
            // columns, so a row's weight (1 point / 0 padding) is its column weight
            const int64_t wblk = (rg * C::SLOTS + g) * kTileM + 32 * q;
            const float rw = (SYM && valid) ? y_wn[pos].x : 0.f;
            const int64_t ct0 = v.ct_b;
            int j = 0;
            if (SYM) {                                // first cluster ending after column ct0 TN
                int lo = 0, hi = vk;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (vpoff[mid + 1] <= ct0 * TN) lo = mid + 1;
                    else hi = mid;
                }
                j = lo;
            }
            int64_t pbnd = (j < vk) ? vpoff[j + 1] : LLONG_MAX;
            double accd = 0.0;
            RatioMin bmin;
            int32_t dlast = -1, dmark = -1;           // deferral: last record; dirty cluster's end slot
            bool ddirty = false;                      // the row has a dirty cluster
            float accf = 0.f;                         // current cluster, this tile
            bool dead = false;
            for (int64_t ct = ct0; ct < ct_end; ++ct) {
                // the tile's accumulator and its (w, |y|^2) in ring slot ws
                const int ws = (int)(wt % kWnRing);
                const bool ok = !abort_flag && mbar_wait(&bar_accf[g][acc], acc_phase, kWaitNs) &&
                                mbar_wait(&bar_wnf[ws], (uint32_t)((wt / kWnRing) & 1), kWaitNs);
                if (!__all_sync(0xffffffffu, ok)) {     // the warp stops as one
                    abort_flag = 1;
                    dead = true;
                    break;
                }
                fence_after_sync();
                const uint32_t tcol = tmem + tlane + (uint32_t)(g * C::NACC + acc) * TN;
                // The tile's 64 accumulator columns are read in four 16-column
                // halves; each half's load is issued before the previous half's
                // arithmetic, so the TMEM latency overlaps it.
                uint32_t ra[16], rb[16];
                __syncwarp();
                tmem_ld16_issue(tcol, ra);
#pragma unroll
                for (int ch = 0; ch < TN / 32; ++ch) {
                    const int64_t c0 = ct * TN + ch * 32;
                    // clusters that end here (empty ones included) are complete;
                    // the own cluster's sum comes from the direct pass (w_own)
                    while (j < vk && c0 == pbnd) {
                        accd += (double)accf;
                        accf = 0.f;
                        if (SYM) {
                            if (accd != 0.0 && rw != 0.f) atomicAdd(&W[pos * k + j], accd);
                        } else if (j != own) {
                            if (kDefer && dmark >= 0) {   // a dirty cluster ends: its partial sum
                                df.ent[dmark] = TcDeferEntry{(int32_t)apos, 0, 0u, dlast, j, 0, accd};
                                dlast = dmark;
                                dmark = -1;
                            } else {
                                bmin.add(accd, (double)v.sizes[j], j);
                            }
                        }
                        accd = 0.0;
                        ++j;
                        pbnd = (j < vk) ? vpoff[j + 1] : LLONG_MAX;
                    }
                    const bool live = j < vk;             // else padding beyond the last cluster
                    const bool mine = live && (j == own); // own-cluster pairs: skipped here
                    // SYM: own is uniform over the warp (one cluster per 32-row block)
                    const bool skip = SYM ? (!live || mine || c0 <= wblk)
                                          : (!live || __all_sync(0xffffffffu, mine));
                    const float4 *wn4 = &sh_wn[ws][ch * 16];
                    float part = 0.f;
                    uint32_t flag = 0;
                    float cs0 = 0.f, cs1 = 0.f;           // SYM: column sums of the two halves
                    int col0 = 0, col1 = 0;
                    tmem_wait_16(ra);                     // first half of this chunk
                    __syncwarp();
                    tmem_ld16_issue(tcol + ch * 32 + 16, rb);
                    if (!skip) {
                        if (SYM) cs0 = half_chunk_sym<METRIC>(ra, wn4, xn, tau, rw, lane, part, flag, col0);
                        else half_chunk<METRIC>(ra, wn4, xn, tau, part, flag);
                    }
                    tmem_wait_16(rb);                     // second half
                    if (ch + 1 < TN / 32) {
                        __syncwarp();
                        tmem_ld16_issue(tcol + (ch + 1) * 32, ra);
                    } else if (kEarlyRelease) {
                        // the tile's last read of tensor memory (the close-pair
                        // recompute of 32-element rows reads coordinates only): the
                        // accumulator goes back to the MMA issuer now, so the next
                        // tile's MMAs overlap this chunk's arithmetic
                        fence_before_sync();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&bar_acce[g][acc]);
                    }
                    if (!skip) {
                        if (SYM) cs1 = half_chunk_sym<METRIC>(rb, wn4 + 8, xn, tau, rw, lane, part, flag, col1);
                        else half_chunk<METRIC>(rb, wn4 + 8, xn, tau, part, flag);
                    }
                    const bool redo = !skip && __any_sync(0xffffffffu, !mine && (flag >> 31) != 0u);
                    if (SYM && !skip && !redo && (lane & 1) == 0) {
                        atomicAdd(&W[(c0 + col0) * k + own], (double)cs0);
                        atomicAdd(&W[(c0 + 16 + col1) * k + own], (double)cs1);
                    }
                    if (redo && kColRedo) {
                        // A lane has a close pair in this chunk: the warp evaluates the
                        // chunk's 32 x 32 pairs directly from the coordinates in FP32.
                        // Lane c takes column c and the 32 rows pass by: each step loads
                        // one row's four coordinates as a broadcast and the 32 columns'
                        // four as one coalesced run (both copies lane-interleaved and
                        // L1-resident), so every pair is an independent FMA chain over
                        // the d real coordinates; a butterfly gives each row's sum of
                        // w d to its own lane.
                        const float *ycl = y_il + il_index(v.ccol + c0, 0, KD) + 4 * lane;
                        const float *fw = reinterpret_cast<const float *>(
                            &sh_wn[ws][ch * 16 + (lane >> 1)]);
                        const float wc = fw[lane & 1], nyc = fw[2 + (lane & 1)];
                        float colsum = 0.f;
                        part = 0.f;
#pragma unroll 2
                        for (int r = 0; r < 32; ++r) {
                            const float *xr = xblk + 4 * r;
                            float a0 = 0.f, a1 = 0.f;
#pragma unroll
                            for (int q = 0; q < KD / 4; ++q) {
                                if (q < dq) {
                                    const float4 h = __ldg(reinterpret_cast<const float4 *>(xr + 128 * q));
                                    const float4 y = __ldg(reinterpret_cast<const float4 *>(ycl + 128 * q));
                                    const float t0 = h.x - y.x, t1 = h.y - y.y;
                                    const float t2 = h.z - y.z, t3 = h.w - y.w;
                                    a0 = fmaf(t0, t0, a0); a1 = fmaf(t1, t1, a1);
                                    a0 = fmaf(t2, t2, a0); a1 = fmaf(t3, t3, a1);
                                }
                            }
                            float dist;
                            if (METRIC == SILH_EUCLIDEAN) {
                                dist = sqrt_apx(a0 + a1);
                            } else {     // a zero vector is at distance 1 from everything
                                const float nxr = __shfl_sync(0xffffffffu, xn, r);
                                dist = (nxr == 0.f || nyc == 0.f) ? 1.f : 0.5f * (a0 + a1);
                            }
                            if (SYM) colsum = fmaf(__shfl_sync(0xffffffffu, rw, r), dist, colsum);
                            float rs = wc * dist;
#pragma unroll
                            for (int o = 16; o > 0; o >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, o);
                            if (lane == r) part = rs;
                        }
                        if (SYM) atomicAdd(&W[(c0 + lane) * k + own], (double)colsum);
                    } else if (redo && !SYM) {
                        // 64-element rows, close pairs in a few lanes and columns: each
                        // lane first takes its 32 pairs from the inner products (four
                        // columns per TMEM load) and only marks the close ones; then
                        // the warp evaluates the marked pairs together, one pair at a
                        // time with two coordinates per lane -- the row's and the
                        // column's loads are coalesced and issued at once, and a
                        // shuffle sum gives the distance.
                        uint32_t fm = 0u;
                        part = 0.f;
                        uint32_t rr0[16], rr1[16];
                        __syncwarp();
                        tmem_ld16_issue(tcol + ch * 32, rr0);
                        tmem_ld16_issue(tcol + ch * 32 + 16, rr1);
                        tmem_wait_16(rr0);
                        tmem_wait_16(rr1);
#pragma unroll
                        for (int hh = 0; hh < 8; ++hh) {
#pragma unroll
                            for (int ii = 0; ii < 4; ++ii) {
                                const int i = 4 * hh + ii;
                                const float dot = __uint_as_float(i < 16 ? rr0[i] : rr1[i - 16]);
                                const float *f = reinterpret_cast<const float *>(
                                    &sh_wn[ws][ch * 16 + (i >> 1)]);
                                const float2 wn = make_float2(f[i & 1], f[2 + (i & 1)]);
                                bool close;
                                float dist;
                                if (METRIC == SILH_EUCLIDEAN) {
                                    const float s2 = xn + wn.y;
                                    const float d2 = fmaf(-2.f, dot, s2);
                                    close = d2 < tau * s2;
                                    dist = sqrt_apx(d2);
                                } else {
                                    dist = 1.f - dot;
                                    close = dist < tau;
                                }
                                if (close) fm |= 1u << i;
                                else part = fmaf(wn.x, dist, part);
                            }
                        }
                        if (mine || !valid) fm = 0u;     // own-cluster sums come from w_own
                        if (kDefer && df.ent != nullptr) {
                            // record the close pairs instead (a cluster's first record also
                            // reserves its end slot); slots are taken for the warp at once
                            const uint32_t need = (fm != 0u) ? (dmark >= 0 ? 1u : 2u) : 0u;
                            uint32_t incl = need;
#pragma unroll
                            for (int o = 1; o < 32; o <<= 1) {
                                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                                if (lane >= o) incl += t;
                            }
                            const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
                            if (tot != 0u) {
                                unsigned long long b0 = 0ull;
                                if (lane == 0) b0 = atomicAdd(&df.ctr[0], (unsigned long long)tot);
                                b0 = __shfl_sync(0xffffffffu, b0, 0);
                                const unsigned long long my = b0 + incl - need;
                                const unsigned long long cap = (unsigned long long)df.ent_cap;
                                if (need != 0u && my + need <= cap) {
                                    df.ent[my] = TcDeferEntry{(int32_t)apos, (int32_t)(v.ccol + c0), fm,
                                                              dlast, j, 0, 0.0};
                                    dlast = (int32_t)my;
                                    if (dmark < 0) {
                                        dmark = (int32_t)(my + 1);
                                        ddirty = true;
                                    }
                                    fm = 0u;                // done here; k_defer_fix evaluates them
                                } else {
                                    // past the capacity: this lane evaluates its pairs below;
                                    // slots of its reservation that lie inside are left empty
                                    for (unsigned long long q = my; q < my + need && q < cap; ++q)
                                        df.ent[q].mask = 0u, df.ent[q].row = -1;
                                }
                            }
                        }
                        constexpr bool kFullRows = BF;
                        // Dense chunks (many close pairs per marked column): each lane
                        // evaluates its own marked pairs column by column, the lanes in
                        // parallel (one direct distance per marked column and lane).
                        const uint32_t npairs = __reduce_add_sync(0xffffffffu, (uint32_t)__popc(fm));
                        const uint32_t colmask = __reduce_or_sync(0xffffffffu, fm);
                        if (npairs > coop_pairs_per_column(BF) * (uint32_t)__popc(colmask)) {
                            const float *xh = a_hi + apos * KD;
                            const float *xl = kFullRows ? xh : a_lo + apos * KD;
                            uint32_t cm = colmask;
                            while (cm != 0u) {
                                const int i = __ffs(cm) - 1;
                                cm &= cm - 1u;
                                if ((fm >> i) & 1u) {
                                    const float *yc = y_full + (v.ccol + c0 + i) * KD;
                                    const float dist = direct_dist_rows<METRIC, KD, kFullRows>(xh, xl, yc);
                                    const float wc = reinterpret_cast<const float *>(
                                        &sh_wn[ws][ch * 16 + (i >> 1)])[i & 1];
                                    part = fmaf(wc, dist, part);
                                }
                            }
                            fm = 0u;
                        }
                        // the marked (row, column) pairs in lane order, four per round:
                        // every round issues the rows' and columns' loads of its four
                        // pairs before any arithmetic
                        uint32_t todo = __ballot_sync(0xffffffffu, fm != 0u);
                        uint32_t m = 0u;
                        int rl = -1;
                        while (todo != 0u || m != 0u) {
                            int pr[4], pc[4];
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                if (m == 0u && todo != 0u) {
                                    rl = __ffs(todo) - 1;
                                    todo &= todo - 1u;
                                    m = __shfl_sync(0xffffffffu, fm, rl);
                                }
                                pr[u] = (m != 0u) ? rl : -1;
                                pc[u] = (m != 0u) ? __ffs(m) - 1 : 0;
                                if (m != 0u) m &= m - 1u;
                            }
                            float x0[4], x1[4], y0[4], y1[4];
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                const int64_t rp = __shfl_sync(0xffffffffu, apos, pr[u] < 0 ? 0 : pr[u]);
                                const float *xr = a_hi + rp * KD;
                                const float *yc = y_full + (v.ccol + c0 + pc[u]) * KD;
                                x0[u] = xr[lane];
                                x1[u] = (KD > 32) ? xr[lane + 32] : 0.f;
                                if (!kFullRows) {          // TF32 operands: x = hi + lo exactly
                                    const float *xq = a_lo + rp * KD;
                                    x0[u] += xq[lane];
                                    if (KD > 32) x1[u] += xq[lane + 32];
                                }
                                y0[u] = yc[lane];
                                y1[u] = (KD > 32) ? yc[lane + 32] : 0.f;
                            }
                            float ss[4];
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                const float t0 = x0[u] - y0[u], t1 = x1[u] - y1[u];
                                ss[u] = fmaf(t0, t0, t1 * t1);
                            }
#pragma unroll
                            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                                for (int u = 0; u < 4; ++u)
                                    ss[u] += __shfl_xor_sync(0xffffffffu, ss[u], o);
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                if (lane != pr[u]) continue;
                                const float dist = (METRIC == SILH_EUCLIDEAN) ? sqrtf(ss[u]) : 0.5f * ss[u];
                                const float wc = reinterpret_cast<const float *>(
                                    &sh_wn[ws][ch * 16 + (pc[u] >> 1)])[pc[u] & 1];
                                part = fmaf(wc, dist, part);
                            }
                        }
                    } else if (redo) {
                        // the same chunk column by column, each lane its own row; the
                        // flagged pairs directly from the coordinates
                        const float *xh = a_hi + (valid ? apos : 0) * KD;
                        constexpr bool kFull = BF || SYM;
                        const float *xl = kFull ? xh : a_lo + (valid ? apos : 0) * KD;
                        part = 0.f;
#pragma unroll 1
                        for (int i = 0; i < 32; ++i) {
                            __syncwarp();
                            const float dot = tmem_ld_32x1(tcol + ch * 32 + i);
                            const float *f = reinterpret_cast<const float *>(
                                &sh_wn[ws][ch * 16 + (i >> 1)]);
                            const float2 wn = make_float2(f[i & 1], f[2 + (i & 1)]);
                            const float *yc = y_full + (v.ccol + c0 + i) * KD;
                            float dist;
                            if (METRIC == SILH_EUCLIDEAN) {
                                const float s2 = xn + wn.y;
                                const float d2 = fmaf(-2.f, dot, s2);
                                dist = (d2 < tau * s2) ? direct_dist_rows<METRIC, KD, kFull>(xh, xl, yc)
                                                       : sqrt_apx(d2);
                            } else {
                                dist = 1.f - dot;
                                if (dist < tau) dist = direct_dist_rows<METRIC, KD, kFull>(xh, xl, yc);
                            }
                            part = fmaf(wn.x, dist, part);
                            if (SYM) {                // column side of this pair
                                float cv = dist * rw;
#pragma unroll
                                for (int o = 16; o > 0; o >>= 1) cv += __shfl_xor_sync(0xffffffffu, cv, o);
                                if (lane == 0) atomicAdd(&W[(c0 + i) * k + own], (double)cv);
                            }
                        }
                    }
                    if (live && !mine) accf += part;
                }
                fence_before_sync();
                __syncwarp();
                if (lane == 0) {
                    if (!kEarlyRelease) mbar_arrive(&bar_acce[g][acc]);
                    mbar_arrive(&bar_wne[ws]);
                }
                acc = (acc + 1 == (uint32_t)C::NACC) ? 0u : acc + 1;
                if (acc == 0) acc_phase ^= 1u;
                ++wt;
                accd += (double)accf;                    // FP64 fold once per tile
                accf = 0.f;
            }
            if (dead) break;
            if (SYM) {                                // row side of the last cluster reached
                accd += (double)accf;
                if (j < k && accd != 0.0 && rw != 0.f) atomicAdd(&W[pos * k + j], accd);
            } else {
                // clusters after the last processed chunk (the current one and empty ones)
                while (j < vk) {
                    accd += (double)accf;
                    accf = 0.f;
                    if (j != own) {
                        if (kDefer && dmark >= 0) {
                            df.ent[dmark] = TcDeferEntry{(int32_t)apos, 0, 0u, dlast, j, 0, accd};
                            dlast = dmark;
                            dmark = -1;
                        } else {
                            bmin.add(accd, (double)v.sizes[j], j);
                        }
                    }
                    accd = 0.0;
                    ++j;
                }
                const double wown = (valid && own >= 0) ? w_own[apos] : 0.0;
                if (kDefer && valid && ddirty) {
                    // outputs come from k_defer_final, which completes the dirty clusters
                    const unsigned long long ri = atomicAdd(&df.ctr[1], 1ull);
                    if (ri < (unsigned long long)df.rec_cap)
                        df.rec[ri] = TcDeferRow{bmin.acc, bmin.size, bmin.arg, dlast, (int32_t)apos,
                                                v.item, a_out[apos]};
                } else if (valid) {
                    const int64_t o = a_out[apos];
                    float sv, av, bv;
                    if (own < 0 || own >= vk) {
                        sv = av = bv = NAN;
                    } else {
                        const int64_t nc = v.sizes[own];
                        const double a = (nc > 1) ? wown / (double)(nc - 1) : 0.0;
                        const double b = bmin.value();
                        const double mx = fmax(a, b);
                        sv = (float)((nc > 1 && mx > 0.0) ? (b - a) / mx : 0.0);
                        av = (float)a;
                        bv = (float)b;
                    }
                    v.s_out[o] = sv;
                    if (a_out_v) a_out_v[o] = av;
                    if (b_out_v) b_out_v[o] = bv;
                    if (NB) nb_out_v[o] = (own < 0 || own >= vk) ? -1 : bmin.arg;
                }
            }
        }
    }
    if (threadIdx.x == 0 && abort_flag) atomicExch(&g_tc_error, 1);
    fence_before_sync();
    __syncthreads();
    if (abort_flag) {
        // A wait gave up: before shared and tensor memory are released, wait
        // (bounded) for every TMA load the producer issued and for the MMAs the
        // issuer issued (one more commit tracks all of them).
        if (warp == 0 && lane == 0) {
            for (int st = 0; st < C::STAGES; ++st)
                if ((ld_issued >> st) & 1u)
                    mbar_wait(&bar_full[st], (ld_parity >> st) & 1u, kWaitNs);
            for (int r = 0; r < kWnRing; ++r)
                if ((wn_issued >> r) & 1u) mbar_wait(&bar_wnf[r], (wn_parity >> r) & 1u, kWaitNs);
            if (a_issued) mbar_wait(&bar_afull, a_parity, kWaitNs);
        } else if (warp == 1 && lane == 0) {
            mma_commit(&bar_drain);
            mbar_wait(&bar_drain, 0u, kWaitNs);
        }
        fence_before_sync();
        __syncthreads();
    }
    if (warp == 1) {
        __syncwarp();
        tmem_dealloc(tmem, C::TMEM_COLS);
    }
}

// Deferred close pairs, step 1: every recorded chunk's close pairs evaluated
// directly in FP32 from the coordinates, a warp per record and two pairs at a
// time (each half-warp one pair, four coordinates per lane, a four-step
// shuffle sum), the terms added in column order; the sum of w d goes to the
// record.  Rows: a_hi (+ a_lo for TF32 operands: x = hi + lo exactly);
// columns: y_full, weights from y_wn.  Records outside the operands (left
// empty by a reservation past the capacity) are skipped.
template <int METRIC, int KD, bool BF>
__global__ void __launch_bounds__(256)
k_defer_fix(const TcDefer df, const float *__restrict__ a_hi, const float *__restrict__ a_lo,
            int64_t nrows_ops, const float *__restrict__ y_full,
            const float2 *__restrict__ y_wn, int64_t ncols_ops) {
    static_assert(KD == 64, "deferral is for 64-element rows (16 lanes x 4 coordinates)");
    const int lane = threadIdx.x & 31, h = lane & 15;
    const bool upper = lane >= 16;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t count = min((int64_t)df.ctr[0], df.ent_cap);
    for (int64_t e = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); e < count;
         e += nw) {
        const uint32_t mask = df.ent[e].mask;
        const int64_t row = df.ent[e].row, col = df.ent[e].col;
        if (mask == 0u || row < 0 || row >= nrows_ops || col < 0 || col + 32 > ncols_ops) continue;
        float4 x = reinterpret_cast<const float4 *>(a_hi + row * KD)[h];
        if (!BF) {
            const float4 l = reinterpret_cast<const float4 *>(a_lo + row * KD)[h];
            x = make_float4(x.x + l.x, x.y + l.y, x.z + l.z, x.w + l.w);
        }
        float acc = 0.f;
        uint32_t m = mask;
        while (m != 0u) {
            const int ia = __ffs(m) - 1;          // this round's pairs: the next two columns
            m &= m - 1u;
            const int ib = (m != 0u) ? __ffs(m) - 1 : -1;
            if (m != 0u) m &= m - 1u;
            const int i = upper ? (ib < 0 ? ia : ib) : ia;
            const float4 y = reinterpret_cast<const float4 *>(y_full + (col + i) * KD)[h];
            const float t0 = x.x - y.x, t1 = x.y - y.y, t2 = x.z - y.z, t3 = x.w - y.w;
            float ss = fmaf(t0, t0, t1 * t1) + fmaf(t2, t2, t3 * t3);
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
            const float dist = (METRIC == SILH_EUCLIDEAN) ? sqrtf(ss) : 0.5f * ss;
            const float term = y_wn[col + i].x * dist;
            const float tb = __shfl_sync(0xffffffffu, term, 16);   // the upper half's pair
            acc += term;                                            // column order: a, then b
            if (ib >= 0) acc += tb;
        }
        if (lane == 0) df.ent[e].val = (double)acc;
    }
}

// Deferred close pairs, step 2: per dirty row, its records walked from the
// last one back (a fixed order): each dirty cluster's partial W_hat_j plus its
// chunks' sums, merged into the row's minimum over the clean clusters (lower
// cluster index on equal ratios), then s_hat, a_hat, b_hat and the neighbour
// as the sweep writes them.
template <bool BATCH>
__global__ void __launch_bounds__(256)
k_defer_final(const TcDefer df, const int32_t *__restrict__ a_lab, const double *__restrict__ w_own,
              const int64_t *__restrict__ sizes, int k, float *__restrict__ s_out,
              float *__restrict__ a_out_v, float *__restrict__ b_out_v, int32_t *__restrict__ nb_out_v,
              const __grid_constant__ TcBatchArg<BATCH> bt) {
    const int64_t count = min((int64_t)df.ctr[1], df.rec_cap);
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < count;
         r += (int64_t)gridDim.x * blockDim.x) {
        const TcDeferRow R = df.rec[r];
        const int64_t *sz = sizes;
        float *so = s_out;
        int kk = k;
        if constexpr (BATCH) {
            sz = bt.items[R.item].sizes;
            so = bt.items[R.item].s_out;
            kk = bt.items[R.item].k;
        }
        double acc = R.bacc, bsz = R.bsize;
        int arg = R.barg;
        auto merge = [&](int j, double w) {
            const double sj = (double)sz[j];
            const double lhs = w * bsz, rhs = acc * sj;
            if (lhs < rhs || (lhs == rhs && j < arg)) {
                acc = w;
                bsz = sj;
                arg = j;
            }
        };
        int cj = -1;
        double csum = 0.0;
        for (int32_t e = R.head; e >= 0; e = df.ent[e].prev) {
            if (df.ent[e].mask == 0u) {           // the end of a dirty cluster
                if (cj >= 0) merge(cj, csum);
                cj = df.ent[e].j;
                csum = df.ent[e].val;
            } else {
                csum += df.ent[e].val;
            }
        }
        if (cj >= 0) merge(cj, csum);
        const int own = a_lab[R.row];
        float sv, av, bv;
        if (own < 0 || own >= kk) {
            sv = av = bv = NAN;
        } else {
            const int64_t nc = sz[own];
            const double a = (nc > 1) ? w_own[R.row] / (double)(nc - 1) : 0.0;
            const double b = acc / bsz;
            const double mx = fmax(a, b);
            sv = (float)((nc > 1 && mx > 0.0) ? (b - a) / mx : 0.0);
            av = (float)a;
            bv = (float)b;
        }
        so[R.out] = sv;
        if (a_out_v) a_out_v[R.out] = av;
        if (b_out_v) b_out_v[R.out] = bv;
        if (nb_out_v) nb_out_v[R.out] = (own < 0 || own >= kk) ? -1 : arg;
    }
}

// Own-cluster pass: W_own[pos] = sum over the row's own cluster's sampled
// columns of w d(x, y), evaluated directly in FP32 from the coordinates (these
// are the close pairs where |x|^2 + |y|^2 - 2 x.y cancels).  Two rows per
// thread in sorted order; a CTA streams one chunk (blockIdx.y) of the column
// blocks of the clusters its rows belong to (contiguous, as rows are sorted by
// cluster) and adds its partial sums to W_own (zeroed beforehand).
template <int METRIC, int KD, bool BF>
__global__ void __launch_bounds__(128)
k_own_direct(const float *__restrict__ a_hi, const float *__restrict__ a_lo,
             const float *__restrict__ a_norm, const int32_t *__restrict__ a_lab, int64_t nrows,
             const float *__restrict__ y_full, const float2 *__restrict__ y_wn,
             const int64_t *__restrict__ poff, int k, int64_t chunk_cols,
             double *__restrict__ w_own) {
    constexpr int BN = 64;
    constexpr int RPT = 2;                       // rows per thread: two 128-row halves
    __shared__ __align__(16) float sh_y[BN * KD];
    __shared__ float2 sh_w[BN];
    const int64_t base = (int64_t)blockIdx.x * 128 * RPT;
    // cluster range of this CTA's rows (labels are sorted; invalid rows last)
    const int64_t last = min(base + 128 * RPT - 1, nrows - 1);
    const int j0 = a_lab[base];
    int j1 = a_lab[last];
    for (int64_t p = last; p >= base && j1 < 0; --p) j1 = a_lab[p];
    if (j0 < 0) return;
    {   // nothing to do when this column chunk is empty for every cluster of the rows
        bool work = false;
        for (int j = j0; j <= j1 && !work; ++j)
            work = poff[j] + (int64_t)blockIdx.y * chunk_cols < poff[j + 1];
        if (!work) return;
    }
    float2 x[RPT][KD / 2];     // coordinate pairs (packed two-lane FP32 arithmetic)
    int own[RPT];
    float zx[RPT];
    int64_t pos[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        pos[r] = base + threadIdx.x + r * 128;
        const bool valid = pos[r] < nrows;
        own[r] = valid ? a_lab[pos[r]] : -1;
        // the row as float4 loads (hi + lo for TF32 operands)
#pragma unroll
        for (int q = 0; q < KD / 4; ++q) {
            float4 h = make_float4(0.f, 0.f, 0.f, 0.f);
            if (valid) {
                h = reinterpret_cast<const float4 *>(a_hi + pos[r] * KD)[q];
                if (!BF) {
                    const float4 l = reinterpret_cast<const float4 *>(a_lo + pos[r] * KD)[q];
                    h = make_float4(h.x + l.x, h.y + l.y, h.z + l.z, h.w + l.w);
                }
            }
            x[r][2 * q] = make_float2(h.x, h.y);
            x[r][2 * q + 1] = make_float2(h.z, h.w);
        }
        zx[r] = (METRIC == SILH_COSINE && valid && a_norm[pos[r]] == 0.f) ? 0.5f : 0.f;
    }
    double acc[RPT] = {};
    if (j0 >= 0) {
        for (int j = j0; j <= j1; ++j) {
            // this block's chunk of cluster j's columns (blockIdx.y-th of chunk_cols)
            const int64_t cs = poff[j] + (int64_t)blockIdx.y * chunk_cols;
            const int64_t ce = min(cs + chunk_cols, poff[j + 1]);
            if (cs >= ce) continue;
            bool any = false;
#pragma unroll
            for (int r = 0; r < RPT; ++r) any |= (own[r] == j);
            for (int64_t cb = cs; cb < ce; cb += BN) {
                const int nb = (int)min((int64_t)BN, ce - cb);
                __syncthreads();
                const float4 *src = reinterpret_cast<const float4 *>(y_full + cb * KD);
                float4 *dst = reinterpret_cast<float4 *>(sh_y);
                for (int q = threadIdx.x; q < nb * (KD / 4); q += 128) {
                    const float4 v = src[q];                 // staged negated: x + (-y)
                    dst[q] = make_float4(-v.x, -v.y, -v.z, -v.w);
                }
                for (int q = threadIdx.x; q < BN; q += 128)
                    sh_w[q] = (q < nb) ? y_wn[cb + q] : make_float2(0.f, 0.f);
                __syncthreads();
                if (!any) continue;
                float part[RPT] = {};
                for (int col = 0; col < nb; ++col) {
                    const float4 *y4 = reinterpret_cast<const float4 *>(sh_y + col * KD);
                    float2 b0[RPT], b1[RPT];
#pragma unroll
                    for (int r = 0; r < RPT; ++r) b0[r] = b1[r] = make_float2(0.f, 0.f);
#pragma unroll
                    for (int q = 0; q < KD / 4; ++q) {
                        const float4 y = y4[q];
#pragma unroll
                        for (int r = 0; r < RPT; ++r) {
                            const float2 t0 = __fadd2_rn(x[r][2 * q], make_float2(y.x, y.y));
                            const float2 t1 = __fadd2_rn(x[r][2 * q + 1], make_float2(y.z, y.w));
                            b0[r] = __ffma2_rn(t0, t0, b0[r]);
                            b1[r] = __ffma2_rn(t1, t1, b1[r]);
                        }
                    }
                    const float2 wn = sh_w[col];
                    const float zy = (METRIC == SILH_COSINE && wn.y == 0.f) ? 0.5f : 0.f;
#pragma unroll
                    for (int r = 0; r < RPT; ++r) {
                        // zero vectors sit at cosine distance 1 from everything
                        const float q2 = (b0[r].x + b0[r].y) + (b1[r].x + b1[r].y);
                        const float dist = (METRIC == SILH_EUCLIDEAN) ? sqrt_apx(q2)
                                                                      : 0.5f * q2 + zx[r] + zy;
                        part[r] = fmaf(wn.x, dist, part[r]);
                    }
                }
#pragma unroll
                for (int r = 0; r < RPT; ++r)
                    if (own[r] == j) acc[r] += (double)part[r];
            }
        }
    }
#pragma unroll
    for (int r = 0; r < RPT; ++r)
        if (pos[r] < nrows && acc[r] != 0.0) atomicAdd(&w_own[pos[r]], acc[r]);
}

// Own-cluster pairs of the symmetric exact, each unordered pair once.  Work
// item (j, I, J), I <= J: the rows of tile I and the columns of tile J of
// cluster j's padded range [poff[j], poff[j+1]) (tiles of 128 * RPT points).
// Row sums of d go to W[row * k + j]; off the diagonal the column sums (over
// the tile's rows, weighted by the row weight, 0 for padding) go to
// W[col * k + j] through a warp transpose-reduce.  Distances directly in FP32
// from the FP32 layout yf, as the row-streaming own pass does.
struct OwnItem {
    int32_t j, I, J, pad_;
};

template <int METRIC, int KD>
__global__ void __launch_bounds__(128)
k_own_sym(const float *__restrict__ yf, const float2 *__restrict__ ywn,
          const int64_t *__restrict__ poff, const OwnItem *__restrict__ items, int k,
          double *__restrict__ W) {
    constexpr int RPT = (KD == 32) ? 2 : 1;
    constexpr int T = 128 * RPT, BN = 64, CB = 8, NW = 4;
    __shared__ __align__(16) float sh_y[BN * KD];      // negated columns
    __shared__ float2 sh_w[BN];                        // (weight, squared norm)
    __shared__ float sh_col[NW][BN];
    const OwnItem it = items[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = poff[it.j], end = poff[it.j + 1];
    const bool diag = it.I == it.J;
    float2 x[RPT][KD / 2];
    float rw[RPT], zx[RPT], accr[RPT];
    int64_t pos[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        pos[r] = base + (int64_t)it.I * T + threadIdx.x + r * 128;
        const bool valid = pos[r] < end;
        const float2 wn = valid ? ywn[pos[r]] : make_float2(0.f, 0.f);
        rw[r] = wn.x;
        zx[r] = (METRIC == SILH_COSINE && valid && wn.y == 0.f) ? 0.5f : 0.f;
        accr[r] = 0.f;
#pragma unroll
        for (int q = 0; q < KD / 4; ++q) {
            const float4 h = valid ? reinterpret_cast<const float4 *>(yf + pos[r] * KD)[q]
                                   : make_float4(0.f, 0.f, 0.f, 0.f);
            x[r][2 * q] = make_float2(h.x, h.y);
            x[r][2 * q + 1] = make_float2(h.z, h.w);
        }
    }
    const int64_t cs_ = base + (int64_t)it.J * T, ce = min(cs_ + T, end);
    for (int64_t cb = cs_; cb < ce; cb += BN) {
        const int nb = (int)min((int64_t)BN, ce - cb);
        __syncthreads();
        for (int q = threadIdx.x; q < nb * (KD / 4); q += 128) {
            const float4 v = reinterpret_cast<const float4 *>(yf + cb * KD)[q];
            reinterpret_cast<float4 *>(sh_y)[q] = make_float4(-v.x, -v.y, -v.z, -v.w);
        }
        for (int q = threadIdx.x; q < BN; q += 128)
            sh_w[q] = (q < nb) ? ywn[cb + q] : make_float2(0.f, 0.f);
        __syncthreads();
        for (int col0 = 0; col0 < nb; col0 += CB) {
            float cs[CB];
#pragma unroll
            for (int c = 0; c < CB; ++c) {
                const int col = col0 + c;
                cs[c] = 0.f;
                if (col < nb) {
                    const float4 *y4 = reinterpret_cast<const float4 *>(sh_y + col * KD);
                    const float2 wn = sh_w[col];
                    const float zy = (METRIC == SILH_COSINE && wn.y == 0.f) ? 0.5f : 0.f;
#pragma unroll
                    for (int r = 0; r < RPT; ++r) {
                        float2 b0 = make_float2(0.f, 0.f), b1 = make_float2(0.f, 0.f);
#pragma unroll
                        for (int q = 0; q < KD / 4; ++q) {
                            const float4 y = y4[q];
                            const float2 t0 = __fadd2_rn(x[r][2 * q], make_float2(y.x, y.y));
                            const float2 t1 = __fadd2_rn(x[r][2 * q + 1], make_float2(y.z, y.w));
                            b0 = __ffma2_rn(t0, t0, b0);
                            b1 = __ffma2_rn(t1, t1, b1);
                        }
                        const float q2 = (b0.x + b0.y) + (b1.x + b1.y);
                        const float dist = (METRIC == SILH_EUCLIDEAN) ? sqrt_apx(q2)
                                                                      : 0.5f * q2 + zx[r] + zy;
                        accr[r] = fmaf(wn.x, dist, accr[r]);
                        cs[c] = fmaf(rw[r], dist, cs[c]);
                    }
                }
            }
            if (!diag) {
                int mine = 0;
                const float tot = transpose_reduce<CB>(cs, lane, mine);
                if ((lane & (32 / CB - 1)) == 0 && col0 + mine < nb) sh_col[warp][col0 + mine] = tot;
            }
        }
        if (!diag) {
            __syncthreads();
            for (int q = threadIdx.x; q < nb; q += 128) {
                float v = 0.f;
#pragma unroll
                for (int w = 0; w < NW; ++w) v += sh_col[w][q];
                if (v != 0.f) atomicAdd(&W[(cb + q) * k + it.j], (double)v);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < RPT; ++r)
        if (pos[r] < end && accr[r] != 0.f) atomicAdd(&W[pos[r] * k + it.j], (double)accr[r]);
}

// Mean of the m sampled columns (Euclidean centring): per-block partial sums
// over a fixed slice of columns, then one block adds them in order.
// (m, per_block) come from the host, or, when d_m is given, m = *d_m and
// per_block = ceil(m / gridDim.x), the host's formula.
template <class T>
__global__ void k_col_mean_partial(const T *__restrict__ X, int d, int64_t ld,
                                   const int32_t *__restrict__ idx, int64_t m, int per_block,
                                   double *__restrict__ part, const int64_t *__restrict__ d_m) {
    const int c = threadIdx.x;                  // coordinate
    if (c >= d) return;
    if (d_m != nullptr) {
        m = *d_m;
        per_block = (int)((m + gridDim.x - 1) / gridDim.x);
    }
    const int64_t lo = (int64_t)blockIdx.x * per_block, hi = min(lo + per_block, m);
    double s = 0.0;
    for (int64_t i = lo; i < hi; ++i) {
        const int64_t e = idx ? idx[i] : i;
        s += (double)to_f32<T>(X[e * ld + c]);
    }
    part[(int64_t)blockIdx.x * d + c] = s;
}

__global__ void k_col_mean_final(const double *__restrict__ part, int nb, int d, int64_t m,
                                 float *__restrict__ mu, const int64_t *__restrict__ d_m) {
    const int c = threadIdx.x;
    if (c >= d) return;
    if (d_m != nullptr) m = *d_m;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[(int64_t)b * d + c];
    mu[c] = m > 0 ? (float)(s / (double)m) : 0.f;     // an empty sample centres nothing
}

// --------------------------------------------------------- row ordering

// Row r of the listed rows (rows == nullptr: row r) gets key = its label, or k
// when the label is outside [0, k); rows are ordered by key, stably.
__global__ void k_key_hist(const int32_t *__restrict__ labels, const int64_t *__restrict__ rows,
                           int64_t nrows, int64_t n, int k, int tile, int ntiles,
                           int32_t *__restrict__ counts) {
    extern __shared__ int32_t sh_cnt[];
    for (int j = threadIdx.x; j <= k; j += 32) sh_cnt[j] = 0;
    __syncwarp();
    const int64_t base = (int64_t)blockIdx.x * tile, end = min(base + (int64_t)tile, nrows);
    for (int64_t r = base + threadIdx.x; r < end; r += 32) {
        const int64_t e = rows ? rows[r] : r;
        const int32_t l = (e >= 0 && e < n) ? labels[e] : -1;
        atomicAdd(&sh_cnt[(l >= 0 && l < k) ? l : k], 1);
    }
    __syncwarp();
    for (int j = threadIdx.x; j <= k; j += 32) counts[(int64_t)j * ntiles + blockIdx.x] = sh_cnt[j];
}

__global__ void k_key_scan(const int32_t *__restrict__ counts, int ntiles,
                           int64_t *__restrict__ tile_base, int64_t *__restrict__ totals) {
    __shared__ int64_t sh[256];
    const int j = blockIdx.x;
    const int32_t *c = counts + (int64_t)j * ntiles;
    int64_t *o = tile_base + (int64_t)j * ntiles;
    const int per = (ntiles + 255) / 256;
    const int lo = threadIdx.x * per, hi = min(lo + per, ntiles);
    int64_t s = 0;
    for (int i = lo; i < hi; ++i) s += c[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 256; off <<= 1) {
        const int64_t v = (threadIdx.x >= (unsigned)off) ? sh[threadIdx.x - off] : 0;
        __syncthreads();
        sh[threadIdx.x] += v;
        __syncthreads();
    }
    int64_t run = sh[threadIdx.x] - s;
    for (int i = lo; i < hi; ++i) {
        o[i] = run;
        run += c[i];
    }
    if (threadIdx.x == 255) totals[j] = sh[255];
}

// boff[j] = sum of totals[0..j), j = 0..nb (single block).
__global__ void k_key_offsets(const int64_t *__restrict__ totals, int nb, int64_t *__restrict__ boff) {
    __shared__ int64_t sh[1024];
    const int per = (nb + 1023) / 1024;
    const int lo = threadIdx.x * per, hi = min(lo + per, nb);
    int64_t s = 0;
    for (int i = lo; i < hi; ++i) s += totals[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int64_t v = (threadIdx.x >= (unsigned)off) ? sh[threadIdx.x - off] : 0;
        __syncthreads();
        sh[threadIdx.x] += v;
        __syncthreads();
    }
    int64_t run = sh[threadIdx.x] - s;
    for (int i = lo; i < hi; ++i) {
        boff[i] = run;
        run += totals[i];
    }
    if (threadIdx.x == 1023) boff[nb] = sh[1023];
}

__global__ void k_key_scatter(const int32_t *__restrict__ labels, const int64_t *__restrict__ rows,
                              int64_t nrows, int64_t n, int k, int tile, int ntiles,
                              const int64_t *__restrict__ tile_base, const int64_t *__restrict__ boff,
                              int64_t *__restrict__ perm) {
    extern __shared__ int32_t sh_cnt[];
    for (int j = threadIdx.x; j <= k; j += 32) sh_cnt[j] = 0;
    __syncwarp();
    unsigned lt;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
    const int64_t base = (int64_t)blockIdx.x * tile, end = min(base + (int64_t)tile, nrows);
    for (int64_t r0 = base; r0 < end; r0 += 32) {
        const int64_t r = r0 + threadIdx.x;
        int key = -1;
        if (r < end) {
            const int64_t e = rows ? rows[r] : r;
            const int32_t l = (e >= 0 && e < n) ? labels[e] : -1;
            key = (l >= 0 && l < k) ? l : k;
        }
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        const int rank = __popc(peers & lt);
        const int cnt = (key >= 0) ? sh_cnt[key] : 0;
        __syncwarp();
        if (key >= 0) {
            perm[boff[key] + tile_base[(int64_t)key * ntiles + blockIdx.x] + cnt + rank] = r;
            if (rank == 0) sh_cnt[key] = cnt + __popc(peers);
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------- gathers

__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Operand split of one (scaled, centred) coordinate v at element c of a row:
// TF32 head + FP32 tail into float rows of KD elements, or BF16 head + BF16
// tail into 64-element BF16 rows (128 bytes).
template <bool BF>
__device__ __forceinline__ void store_split(float v, int64_t row, int c, int KD, void *hi, void *lo) {
    if (BF) {
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
        reinterpret_cast<__nv_bfloat16 *>(hi)[row * 64 + c] = h;
        reinterpret_cast<__nv_bfloat16 *>(lo)[row * 64 + c] = l;
    } else {
        const float h = to_tf32(v);
        reinterpret_cast<float *>(hi)[row * KD + c] = h;
        reinterpret_cast<float *>(lo)[row * KD + c] = v - h;
    }
}

// Row operand in sorted order: hi/lo split (zero padded), the FP32 row when
// the operands are BF16 (full, KD columns; the own-cluster pass reads it),
// the lane-interleaved FP32 copy (il, when given; the direct recompute of
// 32-element rows reads it), squared norm (Euclidean) or unit scaling
// (cosine), label, output index.
// Positions nrows .. nrows_pad - 1 get zero hi/lo rows (the tail of a row
// group that the tile loads read).  A warp per position, grid-stride with two
// positions in flight per warp (each position's loads -- its permutation
// entry, then its row and label -- depend on one another, so the second
// position's chain overlaps the first's); lane c holds elements c, c + 32, ...
template <class T, bool BF>
__global__ void __launch_bounds__(256)
k_gather_rows_tc(const T *__restrict__ X, int d, int64_t ld, int64_t n,
                 const int32_t *__restrict__ labels, const int64_t *__restrict__ rows,
                 const int64_t *__restrict__ perm, int64_t nrows, int64_t nrows_pad,
                 int KD, int k, int metric, const float *__restrict__ mu,
                 void *__restrict__ hi, void *__restrict__ lo,
                 float *__restrict__ full, float *__restrict__ il,
                 float *__restrict__ nrm, int32_t *__restrict__ lab,
                 int64_t *__restrict__ outi) {
    constexpr int U = 2;                      // positions in flight per warp
    constexpr int NE = 4;                     // elements per lane (rows of up to 128)
    const int lane = threadIdx.x & 31;
    const int KE = BF ? 64 : KD;              // elements stored per row
    const int64_t wstride = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t p0 = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; p0 < nrows_pad;
         p0 += U * wstride) {
        int64_t r[U], e[U];
        bool ok[U];
        float v[U][NE];
        int32_t l[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t p = p0 + u * wstride;
            r[u] = (p < nrows) ? perm[p] : -1;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            e[u] = (r[u] >= 0) ? (rows ? rows[r[u]] : r[u]) : -1;
            ok[u] = e[u] >= 0 && e[u] < n;
            const T *x = X + (ok[u] ? e[u] : 0) * ld;
#pragma unroll
            for (int i = 0; i < NE; ++i) {
                const int c = lane + 32 * i;
                v[u][i] = (ok[u] && c < d) ? to_f32<T>(x[c]) : 0.f;
            }
            l[u] = ok[u] ? labels[e[u]] : -1;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t p = p0 + u * wstride;
            if (p >= nrows_pad) continue;         // uniform over the warp
            if (p >= nrows) {
                for (int c = lane; c < (BF ? 64 : KD); c += 32) {
                    store_split<BF>(0.f, p, c, KD, hi, lo);
                    if (il != nullptr && c < KD) il[il_index(p, c, KD)] = 0.f;
                }
                continue;
            }
            // norms in FP32 (pairwise over the lanes): they enter the epilogue in FP32
            float s = 0.f;
            if (metric == SILH_COSINE) {
#pragma unroll
                for (int i = 0; i < NE; ++i)
                    if (lane + 32 * i < d) s = fmaf(v[u][i], v[u][i], s);
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            }
            const float scale = (metric == SILH_COSINE) ? (s > 0.f ? rsqrtf(s) : 0.f) : 1.f;
            float ss = 0.f;
#pragma unroll
            for (int i = 0; i < NE; ++i) {
                const int c = lane + 32 * i;
                if (c < KE) {
                    float w = (c < d) ? v[u][i] * scale : 0.f;
                    if (mu != nullptr && c < d) w = w - mu[c];
                    store_split<BF>(w, p, c, KD, hi, lo);
                    if (BF && c < KD) full[p * KD + c] = w;
                    if (il != nullptr && c < KD) il[il_index(p, c, KD)] = w;
                    ss = fmaf(w, w, ss);
                }
            }
            for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
            if (lane == 0) {
                // Euclidean: squared norm of the (centred) row; cosine: 1, or 0 for a zero row
                nrm[p] = (metric == SILH_COSINE) ? (s > 0.f ? 1.f : 0.f) : ss;
                lab[p] = (l[u] >= 0 && l[u] < k) ? l[u] : -1;
                outi[p] = r[u];
            }
        }
    }
}

// Padded per-cluster column offsets: poff[j+1] = poff[j] + roundup(|F_j|, 32)
// (single block).
__global__ void k_col_poff(const int64_t *__restrict__ offsets, int k, int64_t *__restrict__ poff) {
    __shared__ int64_t sh[1024];
    const int per = (k + 1023) / 1024;
    const int lo = threadIdx.x * per, hi = min(lo + per, k);
    int64_t s = 0;
    for (int j = lo; j < hi; ++j) s += (offsets[j + 1] - offsets[j] + 31) & ~int64_t(31);
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
        poff[j] = run;
        run += (offsets[j + 1] - offsets[j] + 31) & ~int64_t(31);
    }
    if (threadIdx.x == 1023) poff[k] = sh[1023];
}

// Column operand in the padded layout (one warp per padded column): full FP32
// copy, hi/lo split, (weight, squared norm), and when il is given the
// lane-interleaved FP32 copy (the symmetric exact, whose rows are these
// columns).  Padding columns are zero with weight 0.  Source column of sampled
// position t is idx[t] (idx == nullptr: t).
template <class T, bool BF>
__global__ void k_gather_cols_tc(const T *__restrict__ X, int d, int64_t ld,
                                 const int32_t *__restrict__ idx, const double *__restrict__ p,
                                 const int64_t *__restrict__ offsets,
                                 const int64_t *__restrict__ poff, int k, int64_t mp_max, int KD,
                                 int metric, const float *__restrict__ mu, float *__restrict__ full,
                                 void *__restrict__ hi, void *__restrict__ lo,
                                 float2 *__restrict__ wn, float *__restrict__ wn4,
                                 float *__restrict__ il) {
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (i >= mp_max) return;
    int64_t t = -1;
    if (i < poff[k]) {
        int lo_j = 0, hi_j = k - 1;            // last j with poff[j] <= i
        while (lo_j < hi_j) {
            const int mid = (lo_j + hi_j + 1) >> 1;
            if (poff[mid] <= i) lo_j = mid;
            else hi_j = mid - 1;
        }
        const int64_t local = i - poff[lo_j];
        if (local < offsets[lo_j + 1] - offsets[lo_j]) t = offsets[lo_j] + local;
    }
    const int KE = BF ? 64 : KD;
    if (t < 0) {
        for (int c = lane; c < KE; c += 32) {
            if (c < KD) full[i * KD + c] = 0.f;
            if (il != nullptr && c < KD) il[il_index(i, c, KD)] = 0.f;
            store_split<BF>(0.f, i, c, KD, hi, lo);
        }
        if (lane == 0) {
            wn[i] = make_float2(0.f, 0.f);
            if (wn4 != nullptr) wn4[(i >> 1) * 4 + (i & 1)] = wn4[(i >> 1) * 4 + 2 + (i & 1)] = 0.f;
        }
        return;
    }
    const int64_t e = idx ? idx[t] : t;
    const T *x = X + e * ld;
    float s = 0.f;
    if (metric == SILH_COSINE) {
        for (int c = lane; c < d; c += 32) {
            const float v = to_f32<T>(x[c]);
            s = fmaf(v, v, s);
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    const float scale = (metric == SILH_COSINE) ? (s > 0.f ? rsqrtf(s) : 0.f) : 1.f;
    float ss = 0.f;
    for (int c = lane; c < KE; c += 32) {
        float v = (c < d) ? to_f32<T>(x[c]) * scale : 0.f;
        if (mu != nullptr && c < d) v = v - mu[c];
        if (c < KD) full[i * KD + c] = v;
        if (il != nullptr && c < KD) il[il_index(i, c, KD)] = v;
        store_split<BF>(v, i, c, KD, hi, lo);
        ss = fmaf(v, v, ss);
    }
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if (lane == 0) {
        const float w = p ? (float)(1.0 / p[t]) : 1.0f;
        // Euclidean: squared norm of the (centred) column; cosine: 1, or 0 for a zero column
        wn[i] = make_float2(w, (metric == SILH_COSINE) ? (s > 0.f ? 1.f : 0.f) : ss);
        if (wn4 != nullptr) {                    // (w_2i, w_2i+1, n_2i, n_2i+1) per column pair
            wn4[(i >> 1) * 4 + (i & 1)] = wn[i].x;
            wn4[(i >> 1) * 4 + 2 + (i & 1)] = wn[i].y;
        }
    }
}

// Symmetric exact: per padded position i, the cluster of its 32-aligned block
// (padding included, so a warp's rows share it; -1 past the last cluster), the
// original element index (-1 for padding) and the squared norm (from wn).
__global__ void k_padded_meta(const int64_t *__restrict__ offsets, const int64_t *__restrict__ poff,
                              const int32_t *__restrict__ order, int k, int64_t mp_max,
                              const float2 *__restrict__ wn, int32_t *__restrict__ plab,
                              int64_t *__restrict__ outi, float *__restrict__ nrm) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= mp_max) return;
    int32_t lab = -1;
    int64_t o = -1;
    if (i < poff[k]) {
        int lo = 0, hi = k - 1;                // last j with poff[j] <= i
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (poff[mid] <= i) lo = mid;
            else hi = mid - 1;
        }
        lab = lo;
        const int64_t local = i - poff[lo];
        if (local < offsets[lo + 1] - offsets[lo]) o = order[offsets[lo] + local];
    }
    plab[i] = lab;
    outi[i] = o;
    nrm[i] = wn[i].y;
}

// s, a, b of every point from its row of W (the cross-cluster sums, and at
// its own cluster the own-cluster sum), written at the point's original index.
__global__ void k_tc_sym_finalize(const double *__restrict__ W,
                                  const int32_t *__restrict__ plab, const int64_t *__restrict__ outi,
                                  const int64_t *__restrict__ sizes, int64_t mp_max, int k,
                                  float *__restrict__ s_out, float *__restrict__ a_out,
                                  float *__restrict__ b_out, int32_t *__restrict__ nb_out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= mp_max) return;
    const int64_t o = outi[i];
    if (o < 0) return;
    const int own = plab[i];
    const double *w = W + i * k;
    RatioMin bm;
    for (int j = 0; j < k; ++j)
        if (j != own) bm.add(w[j], (double)sizes[j], j);
    const double bmin = bm.value();
    const int64_t nc = sizes[own];
    const double a = (nc > 1) ? w[own] / (double)(nc - 1) : 0.0;    // own-cluster sum
    const double mx = fmax(a, bmin);
    s_out[o] = (float)((nc > 1 && mx > 0.0) ? (bmin - a) / mx : 0.0);
    if (a_out) a_out[o] = (float)a;
    if (b_out) b_out[o] = (float)bmin;
    if (nb_out) nb_out[o] = bm.arg;
}

// ------------------------------------------------------------- host side

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

// 2-D map over a row-major operand with 128-byte boxes along K: FP32 rows of
// KD elements (box 32 x box_rows), or BF16 rows of 64 elements (box 64 x
// box_rows); 128-byte swizzle, matching sw128_kmajor_desc.
bool make_map(CUtensorMap *map, const void *ptr, int KD, int64_t rows, int box_rows, bool bf) {
    auto enc = encode_fn();
    if (!enc) return false;
    const int ke = bf ? 64 : KD, es_bytes = bf ? 2 : 4;
    cuuint64_t gdim[2] = {(cuuint64_t)ke, (cuuint64_t)rows};
    cuuint64_t gstr[1] = {(cuuint64_t)ke * es_bytes};
    cuuint32_t box[2] = {(cuuint32_t)(128 / es_bytes), (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return enc(map, bf ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
               (void *)ptr, gdim, gstr, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 128-column tiles wherever the A operand is one 128-byte K block (split TF32
// at d <= 32 and every BF16 mode); 64-column tiles for two-block TF32 rows.
constexpr bool kWideTiles = true;
constexpr bool wide_tiles(int KD, bool BF) { return kWideTiles && (BF || KD == 32); }

// Own-cluster pass of the row-streaming sweep: W_own of every sorted row is
// zeroed, then set to the direct FP32 sums over its own cluster's columns.
template <int METRIC, int KD, bool BF>
cudaError_t launch_own(cudaStream_t stream, const float *a_hi, const float *a_lo,
                       const float *a_norm, const int32_t *a_lab, int64_t nrows,
                       const float *y_full, const float2 *y_wn, const int64_t *poff, int k,
                       int64_t max_cluster_cols, double *w_own) {
    constexpr int64_t kChunk = 2048;
    const int64_t nchunk = std::max<int64_t>(1, (max_cluster_cols + 31 + kChunk - 1) / kChunk);
    cudaError_t e = cudaMemsetAsync(w_own, 0, sizeof(double) * (size_t)nrows, stream);
    if (e != cudaSuccess) return e;
    // the own-cluster pass reads FP32 rows: hi + lo (TF32 operands) or the
    // FP32 copy (BF16 operands)
    k_own_direct<METRIC, KD, BF><<<dim3((unsigned)((nrows + 255) / 256), (unsigned)nchunk), 128, 0, stream>>>(
        a_hi, a_lo, a_norm, a_lab, nrows, y_full, y_wn, poff, k, kChunk, w_own);
    count_launches(1);
    return cudaGetLastError();
}

template <int METRIC, int KD, bool SPLIT, bool BF, bool SYM = false>
cudaError_t launch_tc(int nsm, cudaStream_t stream, const CUtensorMap &ahi, const CUtensorMap &alo,
                      const CUtensorMap &bhi, const CUtensorMap &blo, const float *a_hi,
                      const float *a_lo, const float *a_il, const float *a_norm,
                      const int32_t *a_lab, const int64_t *a_out, int64_t nrows,
                      const float *y_full, const float *y_il, const float2 *y_wn,
                      const float *y_wn4,
                      const int64_t *poff, const int64_t *sizes, int k, float tau, int dq,
                      int64_t max_cluster_cols, double *w_own, float *s, float *a, float *b,
                      int32_t *nb, double *W = nullptr, const OwnItem *own_items = nullptr,
                      int64_t n_own_items = 0, const int4 *sym_work = nullptr,
                      int64_t n_sym_work = 0, const TcDefer df = TcDefer{}) {
    constexpr bool WIDE = wide_tiles(KD, BF);
    using C = TcCfg<KD, SPLIT, BF, WIDE>;
    if (SYM) {
        // own-cluster pairs once each, into W at the own cluster
        if (n_own_items > 0) {
            k_own_sym<METRIC, KD><<<(unsigned)n_own_items, 128, 0, stream>>>(y_full, y_wn, poff,
                                                                             own_items, k, W);
            count_launches(1);
        }
    } else {
        cudaError_t e0 = launch_own<METRIC, KD, BF>(stream, a_hi, a_lo, a_norm, a_lab, nrows, y_full,
                                                    y_wn, poff, k, max_cluster_cols, w_own);
        if (e0 != cudaSuccess) return e0;
    }
    auto kern = (!SYM && nb != nullptr) ? k_sweep_tc<METRIC, KD, SPLIT, BF, SYM, WIDE, false, true>
                                        : k_sweep_tc<METRIC, KD, SPLIT, BF, SYM, WIDE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    const int64_t groups = SYM ? n_sym_work
                               : ((nrows + kTileM - 1) / kTileM + C::SLOTS - 1) / C::SLOTS;
    if (groups == 0) return cudaSuccess;
    const int grid = (int)std::min<int64_t>(groups, nsm);
    kern<<<grid, C::THREADS, C::SMEM, stream>>>(ahi, alo, bhi, blo, a_hi, a_lo, a_il, a_norm,
                                                a_lab, a_out, nrows, y_full, y_il, y_wn,
                                                reinterpret_cast<const float4 *>(y_wn4), poff,
                                                sizes, k, tau, dq, w_own, s, a, b, nb, W, sym_work,
                                                n_sym_work, df, TcBatchArg<false>{});
    count_launches(1);
    if constexpr (KD == 64 && !SYM) {
        if (df.ent != nullptr) {      // the close pairs the sweep recorded, then the dirty rows
            k_defer_fix<METRIC, KD, BF><<<nsm * 8, 256, 0, stream>>>(df, a_hi, a_lo, df.nrows_ops,
                                                                      y_full, y_wn, df.ncols_ops);
            k_defer_final<false><<<nsm * 4, 256, 0, stream>>>(df, a_lab, w_own, sizes, k, s, a, b,
                                                              nb, TcBatchArg<false>{});
            count_launches(2);
        }
    }
    return cudaGetLastError();
}

// One persistent sweep over the (clustering, row group) work items of a batch;
// the row and column operands, weights, offsets and W_own of all its
// clusterings live in shared buffers (bases in bt).
template <int METRIC, int KD, bool SPLIT, bool BF, bool WIDE>
cudaError_t launch_tc_batched(int nsm, cudaStream_t stream, const CUtensorMap &ahi,
                              const CUtensorMap &alo, const CUtensorMap &bhi,
                              const CUtensorMap &blo, const float *a_hi, const float *a_lo,
                              const float *a_il, const float *a_norm, const int32_t *a_lab,
                              const int64_t *a_out,
                              const float *y_full, const float *y_il, const float2 *y_wn,
                              const float *y_wn4, const int64_t *poff,
                              float tau, int dq, const double *w_own,
                              const TcBatchArg<true> &bt, const TcDefer df) {
    using C = TcCfg<KD, SPLIT, BF, WIDE>;
    auto kern = k_sweep_tc<METRIC, KD, SPLIT, BF, false, WIDE, true>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::min<int64_t>(bt.total_work, nsm);
    kern<<<grid, C::THREADS, C::SMEM, stream>>>(ahi, alo, bhi, blo, a_hi, a_lo, a_il, a_norm,
                                                a_lab, a_out, 0, y_full, y_il, y_wn,
                                                reinterpret_cast<const float4 *>(y_wn4), poff, nullptr,
                                                0, tau, dq, w_own, nullptr, nullptr, nullptr,
                                                nullptr, nullptr, nullptr, 0, df, bt);
    count_launches(1);
    if constexpr (KD == 64) {
        if (df.ent != nullptr) {
            k_defer_fix<METRIC, KD, BF><<<nsm * 8, 256, 0, stream>>>(df, a_hi, a_lo, df.nrows_ops,
                                                                      y_full, y_wn, df.ncols_ops);
            k_defer_final<true><<<nsm * 4, 256, 0, stream>>>(df, a_lab, w_own, nullptr, 0, nullptr,
                                                             nullptr, nullptr, nullptr, bt);
            count_launches(2);
        }
    }
    return cudaGetLastError();
}

// Operands of one clustering in the tensor-core layouts, written into
// caller-provided device buffers: the listed rows sorted by cluster (hi/lo
// split, the FP32 copy for BF16 operands, the lane-interleaved FP32 copy (whole
// blocks of 32 rows), norms, labels, output indices;
// nrows_pad rows, the tail zero) and the cluster-major sample columns padded
// per cluster to multiples of 32 (FP32 copy, lane-interleaved FP32 copy,
// hi/lo split, weight and norm, padded offsets; mp_pad columns, the tail zero
// with weight 0).
struct TcOps {
    uint8_t *rhi, *rlo;
    float *rfull, *ril, *rn;
    int32_t *lab;
    int64_t *outi;
    float *yf, *yil;
    uint8_t *yhi, *ylo;
    float2 *ywn;
    float *ywn4;       // (w, |y|^2) in column pairs, whole 128-column tiles
    int64_t *poff;
};

silh_status tc_prepare(const void *X, silh_dtype dtype, int64_t n, int32_t d, int64_t ld,
                       const int32_t *labels, int32_t k, int metric, int KD, bool bf,
                       const int64_t *offsets, const int32_t *col_idx, const double *col_p,
                       int64_t m, const int64_t *rows, int64_t nrows, int64_t nrows_pad,
                       int64_t mp_pad, const TcOps &o, cudaStream_t stream,
                       const int64_t *d_m = nullptr) {
    silh_status st = SILH_OK;
    Scratch sc(stream);                          // temporaries, released on return
    int gdev = 0, gsm = 0, gather_blocks = 1;
    const int tile = (k <= 512) ? 1024 : 8192;
    const int ntiles = (int)std::max<int64_t>(1, (nrows + tile - 1) / tile);
    const size_t hsmem = sizeof(int32_t) * (size_t)(k + 1);
    const int mean_blocks = 128;
    int32_t *counts = nullptr;
    int64_t *tbase = nullptr, *tot = nullptr, *boff = nullptr, *perm = nullptr;
    double *mpart = nullptr;
    float *mu = nullptr;
    SILH_CK(sc.alloc(&counts, (size_t)(k + 1) * ntiles));
    SILH_CK(sc.alloc(&tbase, (size_t)(k + 1) * ntiles));
    SILH_CK(sc.alloc(&tot, (size_t)k + 1));
    SILH_CK(sc.alloc(&boff, (size_t)k + 2));
    SILH_CK(sc.alloc(&perm, (size_t)nrows));
    SILH_CK(sc.alloc(&mpart, (size_t)mean_blocks * d));
    SILH_CK(sc.alloc(&mu, (size_t)d));
    if (hsmem > 48 * 1024) {
        SILH_CK(cudaFuncSetAttribute(k_key_hist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)hsmem));
        SILH_CK(cudaFuncSetAttribute(k_key_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)hsmem));
    }
    k_key_hist<<<ntiles, 32, hsmem, stream>>>(labels, rows, nrows, n, k, tile, ntiles, counts);
    k_key_scan<<<k + 1, 256, 0, stream>>>(counts, ntiles, tbase, tot);
    k_key_offsets<<<1, 1024, 0, stream>>>(tot, k + 1, boff);
    k_key_scatter<<<ntiles, 32, hsmem, stream>>>(labels, rows, nrows, n, k, tile, ntiles, tbase,
                                                  boff, perm);
    k_col_poff<<<1, 1024, 0, stream>>>(offsets, k, o.poff);
    count_launches(5);
    if (metric == SILH_EUCLIDEAN) {
        // distances are shift invariant: centre rows and columns on the sample mean
        const int per = (int)((m + mean_blocks - 1) / mean_blocks);
        if (dtype == SILH_F32)
            k_col_mean_partial<float><<<mean_blocks, 128, 0, stream>>>((const float *)X, d, ld,
                                                                       col_idx, m, per, mpart, d_m);
        else
            k_col_mean_partial<__nv_bfloat16><<<mean_blocks, 128, 0, stream>>>(
                (const __nv_bfloat16 *)X, d, ld, col_idx, m, per, mpart, d_m);
        k_col_mean_final<<<1, 128, 0, stream>>>(mpart, mean_blocks, d, m, mu, d_m);
        count_launches(2);
    } else {
        mu = nullptr;
    }
    if (o.ril != nullptr && nrows_pad % 32 != 0)   // rows of the last block past nrows_pad
        SILH_CK(cudaMemsetAsync(o.ril + (nrows_pad / 32) * 32 * KD, 0,   // are read, as zeros
                                sizeof(float) * 32 * KD, stream));
    if (o.yil != nullptr && mp_pad % 32 != 0)      // and so are columns past mp_pad
        SILH_CK(cudaMemsetAsync(o.yil + (mp_pad / 32) * 32 * KD, 0, sizeof(float) * 32 * KD,
                                stream));
    // row gather: grid-stride, eight CTAs of eight warps per SM at most
    SILH_CK(cudaGetDevice(&gdev));
    SILH_CK(cudaDeviceGetAttribute(&gsm, cudaDevAttrMultiProcessorCount, gdev));
    gather_blocks = (int)std::max<int64_t>(1, std::min<int64_t>((nrows_pad + 15) / 16,
                                                                (int64_t)gsm * 8));
#define SILH_TC_GATHER(T, BFV)                                                                  \
    k_gather_rows_tc<T, BFV><<<gather_blocks, 256, 0, stream>>>(                               \
        (const T *)X, d, ld, n, labels, rows, perm, nrows, nrows_pad, KD, k, metric, mu, o.rhi, \
        o.rlo, o.rfull, o.ril, o.rn, o.lab, o.outi);                                            \
    k_gather_cols_tc<T, BFV><<<ceil_div_i(mp_pad, 8), 256, 0, stream>>>(                       \
        (const T *)X, d, ld, col_idx, col_p, offsets, o.poff, k, mp_pad, KD, metric, mu, o.yf,  \
        o.yhi, o.ylo, o.ywn, o.ywn4, o.yil);
    if (dtype == SILH_F32) {
        if (bf) { SILH_TC_GATHER(float, true) } else { SILH_TC_GATHER(float, false) }
    } else {
        if (bf) { SILH_TC_GATHER(__nv_bfloat16, true) } else { SILH_TC_GATHER(__nv_bfloat16, false) }
    }
#undef SILH_TC_GATHER
    count_launches(2);
    SILH_CK(cudaGetLastError());
done:
    return st;
}

}  // namespace

bool tc_eligible(int metric, int prec, int d) {
    return (metric == SILH_EUCLIDEAN || metric == SILH_COSINE) &&
           (prec == SILH_PREC_TF32 || prec == SILH_PREC_3XTF32 || prec == SILH_PREC_BF16 ||
            prec == SILH_PREC_BF16X3) &&
           d <= 64 && encode_fn() != nullptr;
}

silh_status tc_sweep(const void *X, silh_dtype dtype, int64_t n, int32_t d, int64_t ld,
                     const int32_t *labels, int32_t k, int metric, int prec, const int64_t *sizes,
                     const int64_t *offsets, const int32_t *col_idx, const double *col_p, int64_t m,
                     int64_t max_cluster_cols, const int64_t *rows, int64_t nrows, float *s,
                     float *a, float *b, int32_t *nb, Scratch &sc, cudaStream_t stream,
                     const int64_t *d_m) {
    silh_status st = SILH_OK;
    const int KD = d <= 32 ? 32 : 64;
    const bool split = prec == SILH_PREC_3XTF32 || prec == SILH_PREC_BF16X3;
    const bool bf = prec == SILH_PREC_BF16 || prec == SILH_PREC_BF16X3;
    const int KE = bf ? 64 : KD;                  // operand row length (128 B per K block)
    const size_t ebytes = bf ? 2 : 4;
    const int64_t mp_max = m + 31 * (int64_t)k;   // padded columns, upper bound
    const int64_t wn_cols = (mp_max + 127) / 128 * 128;
    int dev = 0, nsm = 0;
    double *w_own = nullptr;
    TcOps o = {};
    TcDefer df = {};
    CUtensorMap m_ahi, m_alo, m_bhi, m_blo;
    const float tau = 0.25f;

    SILH_CK(sc.alloc(&o.outi, (size_t)nrows));
    SILH_CK(sc.alloc(&o.lab, (size_t)nrows));
    SILH_CK(sc.alloc(&o.rhi, (size_t)nrows * KE * ebytes));
    SILH_CK(sc.alloc(&o.rlo, (size_t)nrows * KE * ebytes));
    if (bf) SILH_CK(sc.alloc(&o.rfull, (size_t)nrows * KD));
    if (tc_col_redo(KD)) SILH_CK(sc.alloc(&o.ril, (size_t)((nrows + 31) & ~int64_t(31)) * KD));
    SILH_CK(sc.alloc(&o.rn, (size_t)nrows));
    SILH_CK(sc.alloc(&o.poff, (size_t)k + 1));
    SILH_CK(sc.alloc(&w_own, (size_t)nrows));
    SILH_CK(sc.alloc(&o.yf, (size_t)mp_max * KD));
    if (tc_col_redo(KD)) SILH_CK(sc.alloc(&o.yil, (size_t)((mp_max + 31) & ~int64_t(31)) * KD));
    SILH_CK(sc.alloc(&o.yhi, (size_t)mp_max * KE * ebytes));
    SILH_CK(sc.alloc(&o.ylo, (size_t)mp_max * KE * ebytes));
    SILH_CK(sc.alloc(&o.ywn, (size_t)mp_max));
    // the sweep stages whole 128-column tiles of (w, |y|^2): zeros past mp_max
    SILH_CK(sc.alloc(&o.ywn4, (size_t)2 * wn_cols));
    SILH_CK(cudaMemsetAsync(o.ywn4, 0, sizeof(float) * 2 * (size_t)wn_cols, stream));
    if (KD == 64) {        // records of deferred close pairs (a few per row covers the typical case)
        df.ent_cap = std::min<int64_t>(4 * nrows + (int64_t(1) << 20), int64_t(1) << 27);
        df.rec_cap = nrows;
        df.nrows_ops = nrows;
        df.ncols_ops = mp_max;
        SILH_CK(sc.alloc(&df.ent, (size_t)df.ent_cap));
        SILH_CK(sc.alloc(&df.rec, (size_t)nrows));
        SILH_CK(sc.alloc(&df.ctr, 2));
        SILH_CK(cudaMemsetAsync(df.ctr, 0, 2 * sizeof(unsigned long long), stream));
    }
    st = tc_prepare(X, dtype, n, d, ld, labels, k, metric, KD, bf, offsets, col_idx, col_p, m,
                    rows, nrows, nrows, mp_max, o, stream, d_m);
    if (st != SILH_OK) goto done;
    SILH_REQ(make_map(&m_ahi, o.rhi, KD, nrows, kTileM, bf) &&
                 make_map(&m_alo, o.rlo, KD, nrows, kTileM, bf) &&
                 make_map(&m_bhi, o.yhi, KD, mp_max, wide_tiles(KD, bf) ? 128 : kTileN, bf) &&
                 make_map(&m_blo, o.ylo, KD, mp_max, wide_tiles(KD, bf) ? 128 : kTileN, bf),
             "tensor map encoding failed");
    SILH_CK(cudaGetDevice(&dev));
    SILH_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    // the direct recompute and the own-cluster pass read FP32 rows: hi + lo for
    // TF32 operands (exact), the separate FP32 copy for BF16 operands
#define SILH_TC_CASE(MET, KDV, SP, BFV)                                                        \
    if (metric == MET && KD == KDV && split == SP && bf == BFV) {                              \
        SILH_CK((launch_tc<MET, KDV, SP, BFV>(                                                  \
            nsm, stream, m_ahi, m_alo, m_bhi, m_blo, BFV ? o.rfull : (const float *)o.rhi,     \
            BFV ? nullptr : (const float *)o.rlo, o.ril, o.rn, o.lab, o.outi, nrows, o.yf,      \
            o.yil, o.ywn, o.ywn4, o.poff, sizes, k, tau, (d + 3) / 4, max_cluster_cols, w_own, s, a, b, nb, \
            nullptr, nullptr, 0, nullptr, 0, df)));                                             \
    }
#define SILH_TC_CASES(MET, KDV)             \
    SILH_TC_CASE(MET, KDV, true, false)     \
    SILH_TC_CASE(MET, KDV, false, false)    \
    SILH_TC_CASE(MET, KDV, true, true)      \
    SILH_TC_CASE(MET, KDV, false, true)
    SILH_TC_CASES(SILH_EUCLIDEAN, 32)
    SILH_TC_CASES(SILH_EUCLIDEAN, 64)
    SILH_TC_CASES(SILH_COSINE, 32)
    SILH_TC_CASES(SILH_COSINE, 64)
#undef SILH_TC_CASES
#undef SILH_TC_CASE
done:
    return st;
}

silh_status tc_sweep_batched(const void *X, silh_dtype dtype, int64_t n, int32_t d, int64_t ld,
                             int metric, int prec, const silh_batch_item *items,
                             const std::vector<int32_t> &order, int variant,
                             cudaStream_t stream) {
    silh_status st = SILH_OK;
    const int KD = d <= 32 ? 32 : 64;
    const bool split = prec == SILH_PREC_3XTF32 || prec == SILH_PREC_BF16X3;
    const bool bf = prec == SILH_PREC_BF16 || prec == SILH_PREC_BF16X3;
    // tile shape: 128-column tiles, one accumulator per slot (variant 0), or,
    // for TF32 operands of 32-element rows, 64-column tiles with two (variant 1)
    const bool wide = wide_tiles(KD, bf) && !(variant == 1 && !bf && KD == 32);
    const int KE = bf ? 64 : KD;
    const size_t ebytes = bf ? 2 : 4;
    const int slots = tc_slots(KD, bf);           // row tiles per row group (TcCfg::SLOTS)
    const int64_t group_rows = (int64_t)slots * kTileM;
    const int64_t rows_pad = (n + 4 * kTileM - 1) / (4 * kTileM) * (4 * kTileM);
    const int64_t work_per_item = (n + group_rows - 1) / group_rows;
    const size_t il_bytes = tc_col_redo(KD) ? KD * 4 : 0;    // interleaved copies
    const size_t row_bytes = 2 * KE * ebytes + (bf ? KD * 4 : 0) + il_bytes + 4 + 4 + 8 + 8;
    const size_t col_bytes = KD * 4 + il_bytes + 2 * KE * ebytes + 8;
    const float tau = 0.25f;
    int dev = 0, nsm = 0;
    auto cols_of = [&](int32_t i) -> int64_t {     // padded column count, whole 128-column tiles
        const silh_sample *S = items[i].sample;
        return (S->size + 31 * (int64_t)S->k + 127) / 128 * 128;
    };
    // per row also the records of deferred close pairs (64-element rows)
    const size_t defer_row_bytes = (KD == 64) ? 4 * sizeof(TcDeferEntry) + sizeof(TcDeferRow) : 0;
    auto bytes_of = [&](int32_t i) -> size_t {
        return (size_t)rows_pad * (row_bytes + defer_row_bytes) + (size_t)cols_of(i) * col_bytes +
               8 * (size_t)(items[i].sample->k + 1);
    };
    SILH_CK(cudaGetDevice(&dev));
    SILH_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    for (size_t i0 = 0; i0 < order.size();) {
        // as many clusterings as fit the group budget (at least one)
        size_t i1 = i0, bytes = 0;
        while (i1 < order.size() && i1 - i0 < (size_t)kMaxTcBatch) {
            const size_t b = bytes_of(order[i1]);
            if (i1 > i0 && bytes + b > kTcBatchBytes) break;
            bytes += b;
            ++i1;
        }
        const int nb = (int)(i1 - i0);
        int64_t cols_total = 0, poff_total = 0;
        for (size_t i = i0; i < i1; ++i) {
            cols_total += cols_of(order[i]);
            poff_total += items[order[i]].sample->k + 1;
        }
        const int64_t rows_total = rows_pad * nb;
        Scratch gs(stream);                       // this group's operands
        TcOps g = {};
        TcDefer df = {};
        double *w_own = nullptr;
        CUtensorMap m_ahi, m_alo, m_bhi, m_blo;
        TcBatchArg<true> bt;
        std::memset(&bt, 0, sizeof(bt));
        bt.nitems = nb;
        bt.total_work = work_per_item * nb;
        SILH_CK(gs.alloc(&g.outi, (size_t)rows_total));
        SILH_CK(gs.alloc(&g.lab, (size_t)rows_total));
        SILH_CK(gs.alloc(&g.rhi, (size_t)rows_total * KE * ebytes));
        SILH_CK(gs.alloc(&g.rlo, (size_t)rows_total * KE * ebytes));
        if (bf) SILH_CK(gs.alloc(&g.rfull, (size_t)rows_total * KD));
        if (tc_col_redo(KD)) SILH_CK(gs.alloc(&g.ril, (size_t)rows_total * KD));
        SILH_CK(gs.alloc(&g.rn, (size_t)rows_total));
        SILH_CK(gs.alloc(&w_own, (size_t)rows_total));
        SILH_CK(gs.alloc(&g.poff, (size_t)poff_total));
        SILH_CK(gs.alloc(&g.yf, (size_t)cols_total * KD));
        if (tc_col_redo(KD)) SILH_CK(gs.alloc(&g.yil, (size_t)cols_total * KD));
        SILH_CK(gs.alloc(&g.yhi, (size_t)cols_total * KE * ebytes));
        SILH_CK(gs.alloc(&g.ylo, (size_t)cols_total * KE * ebytes));
        SILH_CK(gs.alloc(&g.ywn, (size_t)cols_total));
        SILH_CK(gs.alloc(&g.ywn4, (size_t)2 * cols_total));   // whole tiles, all written
        if (KD == 64) {    // deferred close pairs of every clustering of the group
            df.ent_cap = std::min<int64_t>(4 * rows_total + (int64_t(1) << 20), int64_t(1) << 27);
            df.rec_cap = rows_total;
            df.nrows_ops = rows_total;
            df.ncols_ops = cols_total;
            SILH_CK(gs.alloc(&df.ent, (size_t)df.ent_cap));
            SILH_CK(gs.alloc(&df.rec, (size_t)rows_total));
            SILH_CK(gs.alloc(&df.ctr, 2));
            SILH_CK(cudaMemsetAsync(df.ctr, 0, 2 * sizeof(unsigned long long), stream));
        }
        {
            int64_t ccol = 0, pbase = 0;
            for (int c = 0; c < nb; ++c) {
                const silh_batch_item &src = items[order[i0 + c]];
                const silh_sample *S = src.sample;
                const int64_t arow = rows_pad * c, mp_pad = cols_of(order[i0 + c]);
                TcOps o = g;
                o.rhi = g.rhi + arow * KE * ebytes;
                o.rlo = g.rlo + arow * KE * ebytes;
                o.rfull = bf ? g.rfull + arow * KD : nullptr;
                o.ril = g.ril ? g.ril + arow * KD : nullptr;
                o.rn = g.rn + arow;
                o.lab = g.lab + arow;
                o.outi = g.outi + arow;
                o.yf = g.yf + ccol * KD;
                o.yil = g.yil ? g.yil + ccol * KD : nullptr;
                o.yhi = g.yhi + ccol * KE * ebytes;
                o.ylo = g.ylo + ccol * KE * ebytes;
                o.ywn = g.ywn + ccol;
                o.ywn4 = g.ywn4 + 2 * ccol;
                o.poff = g.poff + pbase;
                st = tc_prepare(X, dtype, n, d, ld, src.labels, S->k, metric, KD, bf, S->offsets,
                                S->idx, S->p, S->size, nullptr, n, rows_pad, mp_pad, o, stream);
                if (st != SILH_OK) goto done;
                const float *rows32 = bf ? o.rfull : (const float *)o.rhi;
                const float *lo32 = bf ? nullptr : (const float *)o.rlo;
#define SILH_TC_OWN(MET, KDV, BFV)                                                              \
                if (metric == MET && KD == KDV && bf == BFV)                                    \
                    SILH_CK((launch_own<MET, KDV, BFV>(stream, rows32, lo32, o.rn, o.lab, n, o.yf, \
                                                       o.ywn, o.poff, S->k, S->size,            \
                                                       w_own + arow)));
                SILH_TC_OWN(SILH_EUCLIDEAN, 32, false)
                SILH_TC_OWN(SILH_EUCLIDEAN, 32, true)
                SILH_TC_OWN(SILH_EUCLIDEAN, 64, false)
                SILH_TC_OWN(SILH_EUCLIDEAN, 64, true)
                SILH_TC_OWN(SILH_COSINE, 32, false)
                SILH_TC_OWN(SILH_COSINE, 32, true)
                SILH_TC_OWN(SILH_COSINE, 64, false)
                SILH_TC_OWN(SILH_COSINE, 64, true)
#undef SILH_TC_OWN
                TcItem &it = bt.items[c];
                it.work_base = work_per_item * c;
                it.arow = arow;
                it.ccol = ccol;
                it.nrows = n;
                it.pbase = pbase;
                it.sizes = S->sizes;
                it.s_out = src.s_hat;
                it.k = S->k;
                ccol += mp_pad;
                pbase += S->k + 1;
            }
        }
        SILH_REQ(make_map(&m_ahi, g.rhi, KD, rows_total, kTileM, bf) &&
                     make_map(&m_alo, g.rlo, KD, rows_total, kTileM, bf) &&
                     make_map(&m_bhi, g.yhi, KD, cols_total, wide ? 128 : kTileN, bf) &&
                     make_map(&m_blo, g.ylo, KD, cols_total, wide ? 128 : kTileN, bf),
                 "tensor map encoding failed");
#define SILH_TC_BCASE_W(MET, KDV, SP, BFV, WV)                                                 \
        if (metric == MET && KD == KDV && split == SP && bf == BFV && wide == WV) {            \
            SILH_CK((launch_tc_batched<MET, KDV, SP, BFV, WV>(                                  \
                nsm, stream, m_ahi, m_alo, m_bhi, m_blo,                                        \
                BFV ? g.rfull : (const float *)g.rhi, BFV ? nullptr : (const float *)g.rlo,     \
                g.ril, g.rn, g.lab, g.outi, g.yf, g.yil, g.ywn, g.ywn4, g.poff, tau, (d + 3) / 4, w_own, \
                bt, df)));                                                                      \
        }
#define SILH_TC_BCASE(MET, KDV, SP, BFV) SILH_TC_BCASE_W(MET, KDV, SP, BFV, wide_tiles(KDV, BFV))
#define SILH_TC_BCASES(MET, KDV)             \
        SILH_TC_BCASE(MET, KDV, true, false)     \
        SILH_TC_BCASE(MET, KDV, false, false)    \
        SILH_TC_BCASE(MET, KDV, true, true)      \
        SILH_TC_BCASE(MET, KDV, false, true)
        SILH_TC_BCASES(SILH_EUCLIDEAN, 32)
        SILH_TC_BCASES(SILH_EUCLIDEAN, 64)
        SILH_TC_BCASES(SILH_COSINE, 32)
        SILH_TC_BCASES(SILH_COSINE, 64)
        // 64-column tiles for TF32 operands of 32-element rows (variant 1)
        SILH_TC_BCASE_W(SILH_EUCLIDEAN, 32, true, false, false)
        SILH_TC_BCASE_W(SILH_EUCLIDEAN, 32, false, false, false)
        SILH_TC_BCASE_W(SILH_COSINE, 32, true, false, false)
        SILH_TC_BCASE_W(SILH_COSINE, 32, false, false, false)
#undef SILH_TC_BCASES
#undef SILH_TC_BCASE
#undef SILH_TC_BCASE_W
        i0 = i1;
    }
done:
    return st;
}

// Exact silhouette of all n points on the tensor cores, each unordered pair
// once (the SYM sweep).  Points are laid out cluster-major and padded per
// cluster to multiples of 32 (the column layout of tc_sweep, weights 1), and
// that one layout is both the row and the column operand.  coff / order: the
// cluster offsets and the cluster-sorted element ids; h_sizes: the cluster
// sizes on the host.  Needs (n + 31 k) * k doubles of scratch for the sums.
silh_status tc_exact_sym(const void *X, silh_dtype dtype, int64_t n, int32_t d, int64_t ld,
                         int32_t k, int metric, int prec, const int64_t *sizes,
                         const int64_t *coff, const int32_t *order,
                         const std::vector<int64_t> &h_sizes, float *s, float *a, float *b,
                         int32_t *nb, Scratch &sc, cudaStream_t stream) {
    silh_status st = SILH_OK;
    const int KD = d <= 32 ? 32 : 64;
    const bool split = prec == SILH_PREC_3XTF32 || prec == SILH_PREC_BF16X3;
    const bool bf = prec == SILH_PREC_BF16 || prec == SILH_PREC_BF16X3;
    const int KE = bf ? 64 : KD;
    const size_t ebytes = bf ? 2 : 4;
    const int64_t mp_max = n + 31 * (int64_t)k;
    const int mean_blocks = 128;
    int dev = 0, nsm = 0;
    int64_t *poff = nullptr, *outi = nullptr;
    int32_t *plab = nullptr;
    double *W = nullptr, *mpart = nullptr;
    float *mu = nullptr, *yf = nullptr, *yil = nullptr, *rn = nullptr;
    OwnItem *own_items = nullptr;
    std::vector<OwnItem> h_items;
    int4 *sym_work = nullptr;
    std::vector<int4> h_work;
    uint8_t *yhi = nullptr, *ylo = nullptr;
    float2 *ywn = nullptr;
    float *ywn4 = nullptr;
    const int64_t wn_cols = (mp_max + 127) / 128 * 128;
    CUtensorMap m_ahi, m_alo, m_bhi, m_blo;
    const float tau = 0.25f;

    SILH_CK(sc.alloc(&poff, (size_t)k + 1));
    SILH_CK(sc.alloc(&outi, (size_t)mp_max));
    SILH_CK(sc.alloc(&plab, (size_t)mp_max));
    SILH_CK(sc.alloc(&rn, (size_t)mp_max));
    SILH_CK(sc.alloc(&W, (size_t)mp_max * k));
    SILH_CK(sc.alloc(&mpart, (size_t)mean_blocks * d));
    SILH_CK(sc.alloc(&mu, (size_t)d));
    SILH_CK(sc.alloc(&yf, (size_t)mp_max * KD));
    if (tc_col_redo(KD)) SILH_CK(sc.alloc(&yil, (size_t)((mp_max + 31) & ~int64_t(31)) * KD));
    SILH_CK(sc.alloc(&yhi, (size_t)mp_max * KE * ebytes));
    SILH_CK(sc.alloc(&ylo, (size_t)mp_max * KE * ebytes));
    SILH_CK(sc.alloc(&ywn, (size_t)mp_max));
    SILH_CK(sc.alloc(&ywn4, (size_t)2 * wn_cols));     // whole tiles: zeros past mp_max
    SILH_CK(cudaMemsetAsync(ywn4, 0, sizeof(float) * 2 * (size_t)wn_cols, stream));
    SILH_CK(cudaMemsetAsync(W, 0, sizeof(double) * (size_t)mp_max * k, stream));
    {   // own-cluster tile pairs (I <= J) over each cluster's padded range
        const int64_t T = (KD == 32) ? 256 : 128;
        for (int32_t j = 0; j < k; ++j) {
            const int64_t len = (h_sizes[j] + 31) & ~int64_t(31);
            const int64_t nt = (len + T - 1) / T;
            for (int64_t I = 0; I < nt; ++I)
                for (int64_t J = I; J < nt; ++J) h_items.push_back({j, (int32_t)I, (int32_t)J, 0});
        }
        if (!h_items.empty()) {
            SILH_CK(sc.alloc(&own_items, h_items.size()));
            SILH_CK(cudaMemcpyAsync(own_items, h_items.data(), sizeof(OwnItem) * h_items.size(),
                                    cudaMemcpyHostToDevice, stream));
        }
    }
    k_col_poff<<<1, 1024, 0, stream>>>(coff, k, poff);
    count_launches(1);
    if (metric == SILH_EUCLIDEAN) {
        // distances are shift invariant: centre on the mean of all points
        const int per = (int)((n + mean_blocks - 1) / mean_blocks);
        if (dtype == SILH_F32)
            k_col_mean_partial<float><<<mean_blocks, 128, 0, stream>>>((const float *)X, d, ld,
                                                                       order, n, per, mpart, nullptr);
        else
            k_col_mean_partial<__nv_bfloat16><<<mean_blocks, 128, 0, stream>>>(
                (const __nv_bfloat16 *)X, d, ld, order, n, per, mpart, nullptr);
        k_col_mean_final<<<1, 128, 0, stream>>>(mpart, mean_blocks, d, n, mu, nullptr);
        count_launches(2);
    } else {
        mu = nullptr;
    }
    if (yil != nullptr && mp_max % 32 != 0)   // positions of the last block past mp_max are
        SILH_CK(cudaMemsetAsync(yil + (mp_max / 32) * 32 * KD, 0,   // read, as zeros
                                sizeof(float) * 32 * KD, stream));
#define SILH_TC_GATHER_SYM(T, BFV)                                                              \
    k_gather_cols_tc<T, BFV><<<ceil_div_i(mp_max, 8), 256, 0, stream>>>(                       \
        (const T *)X, d, ld, order, nullptr, coff, poff, k, mp_max, KD, metric, mu, yf, yhi,    \
        ylo, ywn, ywn4, yil);
    if (dtype == SILH_F32) {
        if (bf) { SILH_TC_GATHER_SYM(float, true) } else { SILH_TC_GATHER_SYM(float, false) }
    } else {
        if (bf) { SILH_TC_GATHER_SYM(__nv_bfloat16, true) } else { SILH_TC_GATHER_SYM(__nv_bfloat16, false) }
    }
#undef SILH_TC_GATHER_SYM
    k_padded_meta<<<ceil_div_i(mp_max, 256), 256, 0, stream>>>(coff, poff, order, k, mp_max, ywn,
                                                               plab, outi, rn);
    count_launches(2);
    SILH_CK(cudaGetLastError());
    SILH_REQ(make_map(&m_ahi, yhi, KD, mp_max, kTileM, bf) &&
                 make_map(&m_alo, ylo, KD, mp_max, kTileM, bf) &&
                 make_map(&m_bhi, yhi, KD, mp_max, wide_tiles(KD, bf) ? 128 : kTileN, bf) &&
                 make_map(&m_blo, ylo, KD, mp_max, wide_tiles(KD, bf) ? 128 : kTileN, bf),
             "tensor map encoding failed");
    SILH_CK(cudaGetDevice(&dev));
    SILH_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    {   // The symmetric sweep's work: each row group takes the column tiles from
        // its own first row on (a triangle), cut into segments of about equal
        // length, so that the CTAs' totals even out; segments of one row group
        // add their row sums to W like the column sums.
        const int64_t TN = wide_tiles(KD, bf) ? 128 : kTileN;
        const int64_t slots = tc_slots(KD, bf);
        const int64_t step = slots * kTileM / TN;   // column tiles per row group on the diagonal
        int64_t mp = 0;
        for (int32_t j = 0; j < k; ++j) mp += (h_sizes[j] + 31) & ~int64_t(31);
        const int64_t nct = (mp + TN - 1) / TN;
        const int64_t ngroups = ((mp_max + kTileM - 1) / kTileM + slots - 1) / slots;
        int64_t total = 0;
        for (int64_t rg = 0; rg < ngroups && rg * step < nct; ++rg) total += nct - rg * step;
        const int64_t seg = std::max<int64_t>(8, (total + 8 * (int64_t)nsm - 1) / (8 * (int64_t)nsm));
        for (int64_t rg = 0; rg < ngroups; ++rg)
            for (int64_t c = rg * step; c < nct; c += seg)
                h_work.push_back(make_int4((int)rg, (int)c, (int)std::min(c + seg, nct), 0));
        if (!h_work.empty()) {
            SILH_CK(sc.alloc(&sym_work, h_work.size()));
            SILH_CK(cudaMemcpyAsync(sym_work, h_work.data(), sizeof(int4) * h_work.size(),
                                    cudaMemcpyHostToDevice, stream));
        }
    }
#define SILH_TC_SYM_CASE(MET, KDV, SP, BFV)                                                    \
    if (metric == MET && KD == KDV && split == SP && bf == BFV) {                              \
        SILH_CK((launch_tc<MET, KDV, SP, BFV, true>(                                            \
            nsm, stream, m_ahi, m_alo, m_bhi, m_blo, yf, nullptr, yil, rn, plab, outi, mp_max, yf, \
            yil, ywn, ywn4, poff, sizes, k, tau, (d + 3) / 4, 0, nullptr, nullptr, nullptr, nullptr, nullptr, W, \
            own_items, (int64_t)h_items.size(), sym_work, (int64_t)h_work.size())));            \
    }
#define SILH_TC_SYM_CASES(MET, KDV)             \
    SILH_TC_SYM_CASE(MET, KDV, true, false)     \
    SILH_TC_SYM_CASE(MET, KDV, false, false)    \
    SILH_TC_SYM_CASE(MET, KDV, true, true)      \
    SILH_TC_SYM_CASE(MET, KDV, false, true)
    SILH_TC_SYM_CASES(SILH_EUCLIDEAN, 32)
    SILH_TC_SYM_CASES(SILH_EUCLIDEAN, 64)
    SILH_TC_SYM_CASES(SILH_COSINE, 32)
    SILH_TC_SYM_CASES(SILH_COSINE, 64)
#undef SILH_TC_SYM_CASES
#undef SILH_TC_SYM_CASE
    k_tc_sym_finalize<<<ceil_div_i(mp_max, 256), 256, 0, stream>>>(W, plab, outi, sizes,
                                                                   mp_max, k, s, a, b, nb);
    count_launches(1);
    SILH_CK(cudaGetLastError());
done:
    return st;
}

namespace {

// Self-test of the bounded-wait error path (one thread, one mbarrier, no TMA and
// no tensor memory): waits for phase 0 of a barrier with one expected arrival,
// after arriving on it first when arrive != 0 (the wait then succeeds at once),
// else with nothing that ever arrives (the wait runs out after timeout_ns).  A
// wait that gives up is recorded exactly as the sweep records it.
__global__ void k_wait_selftest(int arrive, uint64_t timeout_ns) {
    __shared__ uint64_t bar;
    mbar_init(&bar, 1);
    fence_mbar_init();
    if (arrive) mbar_arrive(&bar);
    if (!mbar_wait(&bar, 0u, timeout_ns)) atomicExch(&g_tc_error, 1);
}

}  // namespace

silh_status tc_wait_selftest(int arrive, uint64_t timeout_ns, cudaStream_t stream) {
    silh_status st = SILH_OK;
    k_wait_selftest<<<1, 1, 0, stream>>>(arrive, timeout_ns);
    count_launches(1);
    SILH_CK(cudaGetLastError());
done:
    return st;
}

int tc_take_error() {
    int h = 0;
    if (cudaMemcpyFromSymbol(&h, g_tc_error, sizeof(int)) != cudaSuccess) return -1;
    if (h) {
        int z = 0;
        cudaMemcpyToSymbol(g_tc_error, &z, sizeof(int));
    }
    return h;
}

}  // namespace silh
