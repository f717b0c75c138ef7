// Host-side helpers shared by the entry points of libsilh.
#pragma once

#include <vector>

#include "common.cuh"

namespace silh {

// Stable counting sort of the labels.  On success:
//   d_sizes[k]   |Cj| (device, caller memory)
//   *d_coff      exclusive prefix of the sizes, k+1 entries (scratch)
//   *d_order     element ids grouped by cluster, ascending inside a cluster (scratch)
//   h_sizes/h_coff  host copies.
// Synchronises the stream once (validation of the clustering).
silh_status cluster_sort(const int32_t *labels, int64_t n, int k, Scratch &sc,
                         cudaStream_t stream, int64_t *d_sizes, int64_t **d_coff,
                         int32_t **d_order, std::vector<int64_t> &h_sizes,
                         std::vector<int64_t> &h_coff);

// Exclusive prefix sum of n int32 flags (0/1) into out[n] (int64); the total is
// written to *d_total (device).
cudaError_t scan_flags(const int32_t *flags, int64_t n, int64_t *out, int64_t *d_total,
                       Scratch &sc, cudaStream_t stream);

// Largest and smallest nonzero |x| over the n x d data, for the Canberra
// sweeps' power-of-two scale and their test for tiny coordinates:
// crange[0..1] (device, two words) receive the bits of those non-negative floats.
silh_status canberra_range(const void *X, silh_dtype dtype, int64_t n, int32_t d, int64_t ld,
                           unsigned *crange, cudaStream_t stream);

// Rows of the Phase-2 column operand: Y[i, :] = X[idx[i], :] for i < m (or
// i < *d_m <= m when the sample size is given on the device), padded
// with zeros to D columns; cosine rows are scaled to unit norm.  wY[i] = 1/p[i]
// (or 1 when p == nullptr); zY[i] = 0.5 wY[i] for a zero cosine column, 1 for a
// Canberra column with a coordinate that is tiny at the scale of crange (from
// canberra_range; read only for Canberra), else 0.
silh_status gather_columns(const void *X, silh_dtype dtype, int32_t d, int64_t ld,
                           const int32_t *idx, const double *p, int64_t m, int D, int metric,
                           const unsigned *crange, float *Y, float *wY, float *zY,
                           cudaStream_t stream, const int64_t *d_m = nullptr);

// Phase-2 sweep: for every listed row, W_hat_j over the cluster-major column
// operand (Y, wY, offsets) and the silhouette of Eq. 8 (crange as for
// gather_columns).
silh_status phase2_sweep(const void *X, silh_dtype dtype, int64_t n, int32_t d, int64_t ld,
                         const int32_t *labels, int32_t k, int metric, int prec,
                         const int64_t *sizes, const int64_t *offsets, const float *Y,
                         const float *wY, const float *zY, const unsigned *crange, int64_t m, int D,
                         const int64_t *rows, int64_t nrows, float *s, float *a, float *b,
                         int32_t *nb, cudaStream_t stream);

// Padded row width of the column operand for a given d.
int padded_dim(int d);

// Tensor-core sweep (Euclidean / cosine, TF32 or split TF32, d <= 64).
bool tc_eligible(int metric, int prec, int d);
silh_status tc_sweep(const void *X, silh_dtype dtype, int64_t n, int32_t d, int64_t ld,
                     const int32_t *labels, int32_t k, int metric, int prec, const int64_t *sizes,
                     const int64_t *offsets, const int32_t *col_idx, const double *col_p, int64_t m,
                     int64_t max_cluster_cols, const int64_t *rows, int64_t nrows, float *s,
                     float *a, float *b, int32_t *nb, Scratch &sc, cudaStream_t stream,
                     const int64_t *d_m = nullptr);
// Phase 2 of many clusterings of X (all rows each) on the tensor cores: per
// clustering the operands of tc_sweep, then one persistent sweep over every
// (clustering, row group); the results equal tc_sweep's bit for bit.  order:
// the items in launch order (largest first).  Batches beyond the operand
// budget are split into several launches.
// variant 1 selects 64-column tiles for TF32 operands of 32-element rows;
// any other variant the default 128-column tiles.
silh_status tc_sweep_batched(const void *X, silh_dtype dtype, int64_t n, int32_t d, int64_t ld,
                             int metric, int prec, const silh_batch_item *items,
                             const std::vector<int32_t> &order, int variant,
                             cudaStream_t stream);
// Exact silhouette of all n points on the tensor cores with each unordered
// pair evaluated once (Euclidean / cosine, the tc_sweep precisions, d <= 64).
// coff / order / h_sizes from cluster_sort.
silh_status tc_exact_sym(const void *X, silh_dtype dtype, int64_t n, int32_t d, int64_t ld,
                         int32_t k, int metric, int prec, const int64_t *sizes,
                         const int64_t *coff, const int32_t *order,
                         const std::vector<int64_t> &h_sizes, float *s, float *a, float *b,
                         int32_t *nb, Scratch &sc, cudaStream_t stream);
// 1 if a bounded wait in the tensor-core sweep gave up since the last call
// (and clears it), 0 if not, -1 on a CUDA error.  Synchronous.
int tc_take_error();
// One-thread kernel that waits (bounded) on an mbarrier that is either
// satisfied first (arrive != 0) or never (arrive == 0), and records a wait that
// gives up in the same error word as the tensor-core sweep.
silh_status tc_wait_selftest(int arrive, uint64_t timeout_ns, cudaStream_t stream);

}  // namespace silh
