/*
 * silh.h -- C ABI of the B300 PPS silhouette library (libsilh.so).
 *
 * Implements the silh-pps-all estimator of Altieri, Pietracaprina, Pucci and
 * Vandin, "Scalable and Distributed Silhouette Approximation":
 *   Problem 1 (Sec. 4.1):  estimate s(e) for every element e of V;
 *   Problem 2 (Sec. 4.2):  estimate the silhouette s(C) of the clustering;
 *   Algorithm 1:           Phase 1 = PPS sampling, Phase 2 = estimation;
 *   Eq. 1-3:               exact silhouette of an element / of a clustering.
 *
 * Conventions shared by every entry point
 *   - Data X: n rows of d coordinates, row-major with a leading dimension of
 *     ld elements (ld >= d), in device memory, FP32 or BF16 (silh_dtype).
 *     Rows and the base pointer must be 16-byte aligned (ld * element size a
 *     multiple of 16 bytes).
 *   - labels: int32 device array of n cluster ids in [0, k).  A clustering is a
 *     partition of V into k >= 2 non-empty clusters (Sec. 2).
 *   - Every pointer argument is device memory owned by the caller, unless the
 *     comment says host.  The library allocates only temporary scratch
 *     (stream-ordered, released before the call's work completes on stream) and
 *     never frees caller memory.
 *   - stream: a cudaStream_t passed as void*; NULL is the legacy default stream.
 *     Work is enqueued on it; calls documented as synchronising wait for it.
 *   - Errors come back as a silh_status; silh_last_error() describes the last
 *     failure of the calling thread.  No entry point aborts or traps.
 *   - n < 2^31 and k <= SILH_MAX_K.
 */
#ifndef SILH_H
#define SILH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SILH_MAX_K 8192

/* Distances of Sec. 5.1.1.  d_cos is read as 1 - <x,y>/(|x||y|) (the printed
 * numerator is garbled); a zero-norm operand gives 1.  Canberra terms with
 * |x_i| + |y_i| = 0 contribute 0. */
typedef enum {
    SILH_EUCLIDEAN = 0,
    SILH_COSINE = 1,
    SILH_MANHATTAN = 2,
    SILH_CANBERRA = 3
} silh_metric;

/* Storage type of X. */
typedef enum { SILH_F32 = 0, SILH_BF16 = 1 } silh_dtype;

/* Arithmetic of the Phase-2 / exact distance evaluation.
 *   SILH_PREC_FP32    FP32 on CUDA cores (reference precision, |ds| <= 1e-5);
 *   SILH_PREC_TF32    Euclidean/cosine inner products on tensor cores (TF32);
 *   SILH_PREC_3XTF32  split-TF32 (hi*hi + hi*lo + lo*hi) on tensor cores;
 *   SILH_PREC_BF16    inner products of BF16-rounded operands on tensor cores;
 *   SILH_PREC_BF16X3  split-BF16 (BF16 head and tail, three products).
 * All tensor-core modes accumulate in FP32, keep the per-cluster sums in FP64
 * and recompute in FP32, from the coordinates, the pairs whose distance is
 * small against the magnitudes that cancel in it.  The tensor-core modes
 * apply to Euclidean and cosine with d <= 64; Manhattan, Canberra and d > 64
 * run on CUDA cores in FP32 whatever the mode. */
typedef enum {
    SILH_PREC_FP32 = 0,
    SILH_PREC_TF32 = 1,
    SILH_PREC_3XTF32 = 2,
    SILH_PREC_BF16 = 3,
    SILH_PREC_BF16X3 = 4
} silh_prec;

typedef enum {
    SILH_OK = 0,
    SILH_EINVAL = -1,    /* bad argument or clustering */
    SILH_ENOMEM = -2,    /* scratch allocation failed */
    SILH_ECUDA = -3,     /* CUDA runtime error (see silh_last_error) */
    SILH_ECAPACITY = -4, /* caller's sample buffers too small; size holds need */
    SILH_ETIMEOUT = -5   /* a bounded device wait gave up */
} silh_status;

/* The sample set S = union of F_Cj (Algorithm 1, Phase 1), as per-cluster
 * lists.  All arrays are device memory owned by the caller:
 *   sizes[k]        |Cj| (written by silh_sample_pps)
 *   offsets[k+1]    F_Cj occupies positions offsets[j] .. offsets[j+1]-1
 *   idx[cap]        element ids (rows of X), ascending within each cluster
 *   p[cap]          inclusion probability p_e of each sampled element (FP64)
 * size is the number of sampled elements |S| (host field).  cap = n is always
 * enough. */
typedef struct silh_sample {
    int32_t k;
    int64_t *sizes;
    int64_t *offsets;
    int32_t *idx;
    double *p;
    int64_t cap;
    int64_t size;
} silh_sample;

/* Phase 1 of Algorithm 1 (PPS sampling), for every cluster Cj:
 *   if |Cj| <= t: F_Cj = Cj with p = 1;
 *   else F0 = Poisson sample of Cj with probability min(1, m0/|Cj|);
 *        W(e0) = sum_{e' in Cj} d(e0, e') for e0 in F0;
 *        gamma_e = max(1/|Cj|, max_{e0 in F0} d(e, e0)/W(e0));
 *        p_e = min(1, t gamma_e); F_Cj = Poisson sample with probabilities p_e.
 * m0 <= 0 selects m0 = 2 ln(5k/delta) (Algorithm 1).  The uniforms are
 * Philox4x64-10 with key (seed, 0) and counter (e, stream, clustering_id, 0),
 * u = (word0 >> 11) 2^-53; stream 0 draws F0, stream 1 draws F.  Distances,
 * W, gamma and p are evaluated in FP64.
 * uniform != 0 runs the uniform-sampling variant of Sec. 4.1.3 instead:
 * p_e = min(1, t/|Cj|) for clusters with |Cj| > t, no initial sample.
 * Synchronising: returns after the sample is complete (reads |S| to out->size).
 * Errors: SILH_EINVAL (k < 2, n < 2, d < 1, t <= 0, a label outside [0, k),
 * an empty cluster, null pointers); SILH_ECAPACITY if out->cap < |S| (out->size
 * then holds |S|; sizes are written, the lists are not). */
silh_status silh_sample_pps(const void *X, silh_dtype dtype, int64_t n, int32_t d, int64_t ld,
                            const int32_t *labels, int32_t k, silh_metric metric, double t,
                            double m0, double delta, uint64_t seed, uint32_t clustering_id,
                            int32_t uniform, silh_sample *out, void *stream);

/* Phase 2 of Algorithm 1 for the listed rows (rows == NULL: all n rows, in
 * order; else nrows int64 device row ids):
 *   W_hat_j(e) = sum_{e' in F_Cj} d(e, e') / p_e';
 *   a_hat = W_hat_C(e)/(|C|-1), b_hat = min_{j != C} W_hat_j(e)/|Cj|,
 *   s_hat = (b_hat - a_hat)/max(a_hat, b_hat)   (Eq. 8); singleton -> 0.
 * Outputs are FP32 arrays of nrows entries; a_hat and b_hat may be NULL.
 * nb (may be NULL): int32 array of nrows entries, the neighbouring cluster --
 * the j != C that attains b_hat (the cluster Example 1 names as giving b(e)),
 * the lowest such j among equal ratios; -1 for a row whose label is invalid.
 * Where two clusters' ratios differ by less than the arithmetic's error the
 * choice between them follows the evaluated ratios.
 * Per-cluster sums are carried in FP64 across column tiles.
 * S must describe a sample of this clustering (sizes, offsets, idx, p).
 * Asynchronous.  Errors: SILH_EINVAL for bad sizes/pointers.  A label outside
 * [0, k) in a listed row yields NaN for that row. */
silh_status silh_estimate(const void *X, silh_dtype dtype, int64_t n, int32_t d, int64_t ld,
                          const int32_t *labels, int32_t k, silh_metric metric, silh_prec prec,
                          const silh_sample *S, const int64_t *rows, int64_t nrows,
                          float *s_hat, float *a_hat, float *b_hat, int32_t *nb, void *stream);

/* Phase 1 of Algorithm 1, as silh_sample_pps, with no host synchronisation: the
 * whole phase is enqueued on stream and the call returns at once, so a request
 * (this call, silh_estimate_async, silh_global) is one asynchronous chain and
 * several can run at once on different streams.  Same arguments, arithmetic
 * and sample as silh_sample_pps; in addition
 *   d_size    device int64: receives |S| (0 after any error);
 *   d_status  device int32: receives SILH_OK, SILH_EINVAL (a label outside
 *             [0, k) or an empty cluster), or SILH_ECAPACITY (|S| > out->cap,
 *             or initial samples beyond the planned capacity, below 1e-15 in
 *             probability); after an error the sample is written as an empty
 *             one (offsets all 0), so a following silh_estimate_async stays in
 *             bounds, and the caller may redo the request with
 *             silh_sample_pps.
 * out->cap bounds |S| (cap = n is always enough); out->size is not written.
 * Sizes, offsets and the plan of the initial-sample distance matrices are
 * computed on the device; their scratch is sized from n, k and m0 (n (m0 +
 * 8 sqrt(m0) + 16) FP64 entries for the matrices) and released in stream
 * order.  Errors returned by the call itself: invalid arguments (SILH_EINVAL)
 * and scratch allocation (SILH_ENOMEM), before anything is enqueued. */
silh_status silh_sample_pps_async(const void *X, silh_dtype dtype, int64_t n, int32_t d,
                                  int64_t ld, const int32_t *labels, int32_t k, silh_metric metric,
                                  double t, double m0, double delta, uint64_t seed,
                                  uint32_t clustering_id, int32_t uniform, silh_sample *out,
                                  int64_t *d_size, int32_t *d_status, void *stream);

/* silh_estimate for a sample whose size |S| is known only on the device
 * (*d_size, device int64, from silh_sample_pps_async); S->cap bounds it and sizes
 * the scratch, S->size is ignored.  Results equal silh_estimate's on the same
 * sample bit for bit.  Asynchronous, nothing waits for the device.  Errors: as
 * silh_estimate, and SILH_EINVAL for a null d_size. */
silh_status silh_estimate_async(const void *X, silh_dtype dtype, int64_t n, int32_t d, int64_t ld,
                                const int32_t *labels, int32_t k, silh_metric metric,
                                silh_prec prec, const silh_sample *S, const int64_t *d_size,
                                const int64_t *rows, int64_t nrows, float *s_hat, float *a_hat,
                                float *b_hat, int32_t *nb, void *stream);

/* Phase 2 of Algorithm 1 (Eq. 8) for the cosine distance in O(n k d): with unit
 * vectors d_cos = 1 - <x^, y^> = 0.5 |x^ - y^|^2 (the cosine distance of
 * Sec. 5.1.1, read as in the exact definition), and the weighted sum over a
 * cluster's sample collapses by the parallel-axis identity to
 *   W_hat_j(e) = Z_j + 0.5 (S_j |x^ - mu_j|^2 + R_j),
 * S_j = sum of 1/p over the non-zero sampled vectors, mu_j their weighted mean
 * direction, R_j = sum (1/p) |y^ - mu_j|^2, Z_j = sum of 1/p over zero sampled
 * vectors (distance 1 to everything; a zero row has W_hat_j = S_j + Z_j).
 * Per-cluster constants in FP64, per-row distances in FP32 with mu_j carried
 * as two FP32 words; no cancellation, since both terms are non-negative.  The
 * same real-arithmetic result as silh_estimate(metric = SILH_COSINE), which
 * stays the reference path; this one costs n k d instead of n |S| d.
 * Arguments, layouts and errors as silh_estimate (no metric or precision). */
silh_status silh_estimate_cosine_collapsed(const void *X, silh_dtype dtype, int64_t n, int32_t d,
                                           int64_t ld, const int32_t *labels, int32_t k,
                                           const silh_sample *S, const int64_t *rows,
                                           int64_t nrows, float *s_hat, float *a_hat,
                                           float *b_hat, int32_t *nb, void *stream);

/* Limits of silh_estimate_noalloc's fixed scratch (8.5 MiB per device). */
#define SILH_NOALLOC_MAX_COLUMNS 65536
#define SILH_NOALLOC_MAX_FLOATS 2097152

/* silh_estimate without any device allocation.  The paper has no counterpart:
 * this is a deployment variant of silh_estimate for callers that cannot
 * allocate device memory while they run -- a host framework that has already
 * reserved all of the device's memory for its own allocator, a latency-bound
 * loop that cannot take an allocation (or its failure) in the middle of a
 * stream, or code running inside an allocator or driver callback.  Arguments
 * and errors are those of silh_estimate; the caller still provides every input
 * and output buffer.
 * Precision: distances are always evaluated in FP32 on the CUDA cores, whatever
 * prec says (any valid mode is accepted).  The results equal silh_estimate
 * with SILH_PREC_FP32 bit for bit; where silh_estimate would run a tensor-core
 * mode (Euclidean or cosine, d <= 64) they are the more accurate FP32 values,
 * within that mode's tolerance of its results, not equal to them.
 * Scratch: a fixed array in the library's device image (every GPU that loads
 * libsilh holds it until the process exits) sized for |S| <=
 * SILH_NOALLOC_MAX_COLUMNS sampled columns and |S| x D <= SILH_NOALLOC_MAX_FLOATS
 * (D = d rounded up to 8, 16, 32, 64 or 128); larger samples are rejected with
 * SILH_ECAPACITY before any work is enqueued.  With lazy module loading (the
 * CUDA default) the first call on a device loads this part of the library's
 * device code and maps the 8.5 MiB array; that first call can fail with
 * SILH_ECUDA if the device has no memory left, so make it during
 * initialisation, before reserving the device's memory and before any stream
 * capture.  Every call looks the array's address up again (no allocation).
 * All calls share the array and it keeps the last call's contents; each call
 * rewrites everything it reads (and resets the two words it reduces into),
 * so nothing needs clearing by the caller, but calls whose work overlaps on
 * the GPU race on it and must be ordered by the caller.
 * Asynchronous. */
silh_status silh_estimate_noalloc(const void *X, silh_dtype dtype, int64_t n, int32_t d,
                                  int64_t ld, const int32_t *labels, int32_t k,
                                  silh_metric metric, silh_prec prec, const silh_sample *S,
                                  const int64_t *rows, int64_t nrows, float *s_hat, float *a_hat,
                                  float *b_hat, int32_t *nb, void *stream);

/* One clustering of the dataset in a batched call: its labels, its sample set
 * (from silh_sample_pps on these labels) and its FP32 output of n s_hat values. */
typedef struct silh_batch_item {
    const int32_t *labels;
    const silh_sample *sample;
    float *s_hat;
} silh_batch_item;

/* Phase 2 of Algorithm 1 for many clusterings of the same data X in one
 * persistent launch (the work items are (clustering, row tile) pairs, taken
 * round-robin by CTAs sized to fill the GPU), all rows of every item.
 * prec SILH_PREC_FP32 (or a tensor-core mode the metric or d rules out): CUDA
 * cores, the arithmetic of silh_estimate with SILH_PREC_FP32 on each item;
 * variant selects the tile shape (rows per thread x columns per stage: 0 =
 * 1x32, 1 = 1x64, 2 = 2x32, 3 = 2x128 (2x64 for d > 32, 2x32 for d > 64);
 * -1 = default, the single sweep's shape, whose results equal silh_estimate's
 * bit for bit; the other shapes group each cluster's FP32 partial sums
 * differently, so their last bits can differ) -- the choice an autotuner
 * makes by timing.  prec TF32 / 3XTF32 / BF16 / BF16X3 with the
 * Euclidean or cosine distance and d <= 64: tensor cores; each item first gets
 * the operands of the single-clustering tensor-core sweep (rows sorted by its
 * clusters, its padded sample columns, its own-cluster sums), then one
 * persistent sweep covers every (clustering, row group), and each result
 * equals silh_estimate with that prec bit for bit; variant 1 selects 64-column
 * tiles with two accumulators per row tile for TF32 operands of rows of up to
 * 32 elements (d <= 32), any other value the default 128-column tiles with one
 * (the choice an autotuner makes by timing; the results do not depend on it).
 * Operands above 16 GiB per launch are split over several launches.
 * Asynchronous and free of host synchronisation, so the call can be captured
 * in a CUDA graph; items are passed to the kernels as launch parameters, 256
 * per launch.  Errors: SILH_EINVAL for bad arguments, SILH_ENOMEM when the
 * scratch cannot be allocated. */
silh_status silh_estimate_batched(const void *X, silh_dtype dtype, int64_t n, int32_t d,
                                  int64_t ld, silh_metric metric, silh_prec prec, int32_t nitems,
                                  const silh_batch_item *items, int32_t variant, void *stream);

/* Exact silhouette (Eq. 1-2) of the listed rows against all n elements:
 * Phase 2 with F_Cj = Cj and p = 1; nb (may be NULL) as for silh_estimate.
 * Synchronising (validates labels).  Errors: as silh_sample_pps. */
silh_status silh_exact(const void *X, silh_dtype dtype, int64_t n, int32_t d, int64_t ld,
                       const int32_t *labels, int32_t k, silh_metric metric, silh_prec prec,
                       const int64_t *rows, int64_t nrows, float *s, float *a, float *b,
                       int32_t *nb, void *stream);

/* Cohesion and separation of the clustering estimated from the Phase-2 weights
 * (the paper's section on other clustering validation measures):
 *   Coh = (1/2) sum_j sum_{e in Cj} W_hat_Cj(e) / sum_j C(|Cj|, 2)
 *   Sep = sum_{j1<j2} sum_{e in Cj1} W_hat_Cj2(e) / sum_{j1<j2} |Cj1||Cj2|
 * (the printed |C_{j-1}| in Sep's denominator is read as |C_{j1}|).  With
 * every p = 1 (t >= max |Cj|) these are the exact values.  out: two doubles in
 * device memory, (Coh, Sep).  FP32 CUDA-core distances, FP64 sums.
 * Asynchronous.  Errors: as silh_estimate. */
silh_status silh_cohsep(const void *X, silh_dtype dtype, int64_t n, int32_t d, int64_t ld,
                        const int32_t *labels, int32_t k, silh_metric metric, const silh_sample *S,
                        double *out, void *stream);

/* Mean of n FP32 values in FP64 with a fixed reduction tree (Eq. 3 for exact
 * s, Eq. 6 for s_hat, Eq. 7 for a row subset).  out: one double, device memory.
 * Asynchronous.  Errors: SILH_EINVAL if n < 1 or a pointer is NULL. */
silh_status silh_global(const float *s, int64_t n, double *out, void *stream);

/* Waits for all work on stream, then reports whether any bounded device wait
 * of the library gave up since the previous call (SILH_ETIMEOUT; the results
 * of the affected call are then incomplete) and clears that record.  Kernels
 * never trap or spin without limit; this is how a stalled pipeline surfaces.
 * The record is one per device and process: with calls in flight on several
 * streams, a timeout is reported to whichever caller checks first, so a
 * multi-stream caller treats SILH_ETIMEOUT as "some call since the last check".
 * Synchronising. */
silh_status silh_stream_status(void *stream);

/* Self-test of the bounded-wait error path; no counterpart in the paper.  One
 * kernel of one thread initialises an mbarrier expecting one arrival and waits
 * for it with the limit timeout_ns (1 us .. 1 s): with arrive != 0 the thread
 * arrives first and the wait succeeds; with arrive == 0 nothing ever arrives,
 * the wait gives up after the limit and records the failure in the word that
 * silh_stream_status reads, exactly as the tensor-core sweep's waits do.  No
 * TMA copy, MMA or tensor memory is involved, so nothing is left in flight and
 * the context stays usable.  Asynchronous.  Errors: SILH_EINVAL for a limit
 * outside the range. */
silh_status silh_wait_selftest(int32_t arrive, uint64_t timeout_ns, void *stream);

/* Lemma 1: t = ceil((3c/eps^2) ln(5 n k / delta)) with c = 18.  Host-only. */
double silh_t_from_eps(double eps, double delta, int64_t n, int32_t k);

/* Description of the calling thread's last failure ("" if none). */
const char *silh_last_error(void);

/* Library version string. */
const char *silh_version(void);

/* Measured arithmetic rates of the current device, in lane-operations per
 * second per SM (device wall-clock time): out[0] FP32 FMA, out[1] packed
 * two-lane FP32 FMA (lanes), out[2] MUFU reciprocal (rcp.approx), out[3] MUFU
 * square root (sqrt.approx), out[4] FP32 min/max, out[5] FP64 FMA.  Divide by
 * the SM clock for per-clock figures.  out: host array of 6 doubles.
 * Synchronous.  Diagnostic with no counterpart in the paper: the bounds of the
 * Phase-2 kernels are stated in these units. */
silh_status silh_pipe_rates(double *out, void *stream);

/* Number of CUDA kernels this library has launched in the calling process
 * (all threads, all devices) -- for launch accounting in benchmarks. */
uint64_t silh_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* SILH_H */
