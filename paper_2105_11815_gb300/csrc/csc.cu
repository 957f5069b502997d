// CSR -> CSC copy of a sparse A (Ski-LLS-sparse, Section 6: LSQR with sparse
// products), so that A^T t is a gather per column with a fixed summation
// order (row indices ascending) instead of scattered atomics.
#include "common.cuh"
#include "lsqr_impl.cuh"

__global__ void k_scan_counts(const int32_t* __restrict__ counts, int64_t m, int64_t* __restrict__ offsets);

namespace {

__global__ void k_col_count(int64_t nnz, const int32_t* __restrict__ colidx, int32_t* __restrict__ counts) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p < nnz) atomicAdd(&counts[colidx[p]], 1);
}

__global__ void k_col_fill(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                           const double* __restrict__ val, const int64_t* __restrict__ colptr,
                           int32_t* __restrict__ cursor, int32_t* __restrict__ trow, double* __restrict__ tval) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n) return;
  for (int64_t p = rowptr[j]; p < rowptr[j + 1]; ++p) {
    int32_t c = colidx[p];
    int64_t pos = colptr[c] + atomicAdd(&cursor[c], 1);
    trow[pos] = (int32_t)j;
    tval[pos] = val[p];
  }
}

// Rank sort of each column segment by row index (entries are distinct).
__global__ void __launch_bounds__(256) k_col_sort(int64_t d, const int64_t* __restrict__ colptr,
                                                  const int32_t* __restrict__ trow, const double* __restrict__ tval,
                                                  int32_t* __restrict__ rowidx, double* __restrict__ cval) {
  __shared__ int32_t keys[4096];
  const int64_t c = blockIdx.x;
  const int64_t lo = colptr[c], K = colptr[c + 1] - lo;
  const bool in_smem = K <= 4096;
  if (in_smem)
    for (int64_t a = threadIdx.x; a < K; a += blockDim.x) keys[a] = trow[lo + a];
  __syncthreads();
  for (int64_t a = threadIdx.x; a < K; a += blockDim.x) {
    const int32_t v = trow[lo + a];
    int64_t rank = 0;
    if (in_smem)
      for (int64_t b = 0; b < K; ++b) rank += keys[b] < v;
    else
      for (int64_t b = 0; b < K; ++b) rank += trow[lo + b] < v;
    rowidx[lo + rank] = v;
    cval[lo + rank] = tval[lo + a];
  }
}

}  // namespace

size_t ski_csc_ws_bytes(int64_t n, int64_t d, int64_t nnz) {
  (void)n;
  SkiArena ar{nullptr, 0, 0, true};
  ar.take<int32_t>(d);
  ar.take<int32_t>(d);
  ar.take<int32_t>(nnz);
  ar.take<double>(nnz);
  return ar.off;
}

ski_status ski_csc_build(const ski_matrix* A, int64_t* colptr, int32_t* rowidx, double* cval, SkiArena& ar,
                         cudaStream_t st) {
  const int64_t d = A->d, nnz = A->nnz, n = A->n;
  int32_t* counts = ar.take<int32_t>(d);
  int32_t* cursor = ar.take<int32_t>(d);
  int32_t* trow = ar.take<int32_t>(nnz);
  double* tval = ar.take<double>(nnz);
  if (!ar.ok() || !tval) return SKI_ENOMEM;
  SKI_CUDA_TRY(cudaMemsetAsync(counts, 0, d * sizeof(int32_t), st));
  SKI_CUDA_TRY(cudaMemsetAsync(cursor, 0, d * sizeof(int32_t), st));
  if (nnz > 0) {
    k_col_count<<<(unsigned)ski_cdiv(nnz, 256), 256, 0, st>>>(nnz, A->colidx, counts);
    SKI_LAUNCH_CHECK();
  }
  k_scan_counts<<<1, 1024, 0, st>>>(counts, d, colptr);
  SKI_LAUNCH_CHECK();
  if (nnz > 0) {
    k_col_fill<<<(unsigned)ski_cdiv(n, 256), 256, 0, st>>>(n, A->rowptr, A->colidx, A->val, colptr, cursor, trow,
                                                          tval);
    SKI_LAUNCH_CHECK();
    k_col_sort<<<(unsigned)d, 256, 0, st>>>(d, colptr, trow, tval, rowidx, cval);
    SKI_LAUNCH_CHECK();
  }
  return SKI_OK;
}
