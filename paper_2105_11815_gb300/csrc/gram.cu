// Step 2 of Ski-LLS-sparse from a sparse sketch (Section 6): SA kept sparse
// (CSR, duplicates merged), its Gram matrix G = SA^T SA formed from the
// sparse rows, and R the Cholesky factor of G (R^T R = G, upper, positive
// diagonal), which in exact arithmetic is the R of a QR factorization of SA
// -- the factor the paper takes from SPQR on the sparse SA.  Q^T Sb is then
// R^{-T} SA^T Sb.  Used for CSR A with ski_opts.factorization = 2.
//
//  1. Bucket lists of the s-hashing draw (as the dense sketch).
//  2. Row i of SA: the columns of the A rows hashed to bucket i, each entry
//     signed and scaled by 1/sqrt(s), sorted by column in shared memory
//     (bitonic, keyed by (column, load position) so that the summation order
//     of equal columns is fixed) and merged.  Rows longer than kRowCap
//     entries before merging make the path report failure.
//  3. Compact CSR, then its CSC (csc.cu: row indices ascending per column).
//  4. G, upper triangle: CTA per row i of G (a column chunk at a time) with a
//     shared-memory accumulator: for each nonzero SA[r, i] (r ascending), the
//     entries SA[r, c], c >= i, of row r are added times SA[r, i]; a barrier
//     between rows keeps every accumulator update in a fixed order.  Work is
//     sum_r nnz(row r)^2 / 2 (G of a dense SA would cost m d^2 / 2).
//  5. Blocked right-looking Cholesky in place (blocks of 64 columns): the
//     diagonal block in one CTA, R12 = R11^{-T} G12 by forward substitution
//     down each column of the panel (one thread per column), and
//     G22 -= R12^T R12 on the SIMT GEMM restricted to tiles that meet the
//     upper triangle.  A pivot that is not positive reports failure.
//  6. c = SA^T Sb by columns of SA, then Q^T Sb = R^{-T} c by blocked forward
//     substitution (the diagonal block in one CTA, the rest as GEMV updates).
// On failure the caller factors the dense sketch by Householder QR instead.
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "hash.cuh"
#include "lsqr_impl.cuh"
#include "sketch_impl.cuh"

__global__ void k_scan_counts(const int32_t* __restrict__ counts, int64_t m, int64_t* __restrict__ offsets);

namespace {

constexpr int kRowCap = 8192;  // entries of one SA row before merging (shared-memory sort)
constexpr int CB = 64;         // Cholesky block
constexpr int kGramChunk = 24576;  // columns of G per accumulator pass (192 KB of FP64)

// ---- 2. sparse sketch rows
__global__ void k_sa_row_bound(int64_t m, const int64_t* __restrict__ off, const uint32_t* __restrict__ list,
                               const int64_t* __restrict__ rowptr, int32_t* __restrict__ ub, int* __restrict__ fail) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  int64_t t = 0;
  for (int64_t e = off[i]; e < off[i + 1]; ++e) {
    const int64_t j = list[e] >> 1;
    t += rowptr[j + 1] - rowptr[j];
  }
  if (t > kRowCap) {
    atomicExch(fail, 1);
    t = 0;  // the path is abandoned; keep the layout small
  }
  ub[i] = (int32_t)t;
}

// CTA per SA row: gather, sort by (column, load position), merge.
__global__ void __launch_bounds__(256) k_sa_row_fill(int64_t m, const int64_t* __restrict__ off,
                                                     const uint32_t* __restrict__ list,
                                                     const int64_t* __restrict__ rowptr,
                                                     const int32_t* __restrict__ colidx,
                                                     const double* __restrict__ val, double scale,
                                                     const int64_t* __restrict__ ubptr, int32_t* __restrict__ rowlen,
                                                     int32_t* __restrict__ ocol, double* __restrict__ oval) {
  extern __shared__ __align__(16) unsigned char raw[];
  unsigned long long* key = reinterpret_cast<unsigned long long*>(raw);  // [kRowCap]
  double* v = reinterpret_cast<double*>(key + kRowCap);                 // [kRowCap], by load position
  __shared__ int64_t seg[257];
  __shared__ int s_heads[8];
  const int64_t i = blockIdx.x;
  const int64_t e0 = off[i], ne = off[i + 1] - e0;
  const int64_t K = ubptr[i + 1] - ubptr[i];
  if (K == 0) {
    if (threadIdx.x == 0) rowlen[i] = 0;
    return;
  }
  // load: bucket entries in chunks of 256, each thread one A row of the chunk
  int64_t pos0 = 0;
  for (int64_t c0 = 0; c0 < ne; c0 += 256) {
    const int64_t e = c0 + threadIdx.x;
    int64_t len = 0, j = 0;
    bool neg = false;
    if (e < ne) {
      const uint32_t en = list[e0 + e];
      j = en >> 1;
      neg = en & 1u;
      len = rowptr[j + 1] - rowptr[j];
    }
    // exclusive scan of the chunk's row lengths
    if (threadIdx.x == 0) seg[0] = 0;
    __syncthreads();
    seg[threadIdx.x + 1] = len;
    __syncthreads();
    if (threadIdx.x == 0)
      for (int t = 1; t <= 256; ++t) seg[t] += seg[t - 1];
    __syncthreads();
    if (e < ne) {
      const int64_t p0 = rowptr[j], base = pos0 + seg[threadIdx.x];
      for (int64_t p = 0; p < len; ++p) {
        const int64_t q = base + p;
        key[q] = ((unsigned long long)(uint32_t)colidx[p0 + p] << 32) | (unsigned long long)q;
        const double a = val[p0 + p] * scale;
        v[q] = neg ? -a : a;
      }
    }
    pos0 += seg[256];
    __syncthreads();
  }
  // bitonic sort of key[0 .. Kp) (padding keys sort last)
  int Kp = 1;
  while (Kp < K) Kp <<= 1;
  for (int64_t q = K + threadIdx.x; q < Kp; q += blockDim.x) key[q] = ~0ull;
  __syncthreads();
  for (int size = 2; size <= Kp; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = threadIdx.x; t < Kp / 2; t += blockDim.x) {
        const int lo = 2 * t - (t & (stride - 1));
        const int hi = lo + stride;
        const bool up = (lo & size) == 0;
        const unsigned long long a = key[lo], b = key[hi];
        if ((a > b) == up) {
          key[lo] = b;
          key[hi] = a;
        }
      }
      __syncthreads();
    }
  }
  // merge runs of equal columns: each run head sums its run in sorted order
  // and takes its rank among the heads as its output position; thread t
  // scans the contiguous range [t qc, (t + 1) qc) so that ranks follow q
  const int64_t qc = (K + blockDim.x - 1) / blockDim.x;
  const int64_t qa = threadIdx.x * qc, qb = std::min<int64_t>(K, qa + qc);
  int mycount = 0;
  for (int64_t q = qa; q < qb; ++q) mycount += (q == 0 || (key[q] >> 32) != (key[q - 1] >> 32)) ? 1 : 0;
  // block scan of the per-thread head counts (256 threads: 8 warps)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = mycount;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_heads[wid] = x;
  __syncthreads();
  int before = x - mycount;
  for (int w = 0; w < wid; ++w) before += s_heads[w];
  int total = 0;
  for (int w = 0; w < 8; ++w) total += s_heads[w];
  const int64_t ob = ubptr[i];
  int rank = before;
  for (int64_t q = qa; q < qb; ++q) {
    const uint32_t col = (uint32_t)(key[q] >> 32);
    if (q == 0 || (key[q - 1] >> 32) != col) {
      double s = 0.0;
      for (int64_t r = q; r < K && (uint32_t)(key[r] >> 32) == col; ++r) s += v[key[r] & 0xFFFFFFFFull];
      ocol[ob + rank] = (int32_t)col;
      oval[ob + rank] = s;
      ++rank;
    }
  }
  if (threadIdx.x == 0) rowlen[i] = total;
}

// ---- 3. compact CSR
__global__ void k_sa_compact(int64_t m, const int64_t* __restrict__ ubptr, const int64_t* __restrict__ rowptr,
                             const int32_t* __restrict__ icol, const double* __restrict__ ival,
                             int32_t* __restrict__ ocol, double* __restrict__ oval) {
  const int64_t i = blockIdx.x;
  const int64_t src = ubptr[i], dst = rowptr[i], len = rowptr[i + 1] - dst;
  for (int64_t p = threadIdx.x; p < len; p += blockDim.x) {
    ocol[dst + p] = icol[src + p];
    oval[dst + p] = ival[src + p];
  }
}

// ---- 4. G = SA^T SA, upper triangle, columns [c0, c0 + cw) of row i
__global__ void __launch_bounds__(256) k_gram_rows(int64_t d, const int64_t* __restrict__ colptr,
                                                   const int32_t* __restrict__ rowidx, const double* __restrict__ cval,
                                                   const int64_t* __restrict__ rowptr,
                                                   const int32_t* __restrict__ colidx, const double* __restrict__ val,
                                                   double* __restrict__ G, int64_t ldg, int64_t c0, int64_t cw) {
  extern __shared__ __align__(16) double acc[];
  const int64_t i = blockIdx.x;
  const int64_t lo = std::max<int64_t>(i, c0), hi = std::min<int64_t>(d, c0 + cw);
  if (lo >= hi) return;
  for (int64_t c = lo + threadIdx.x; c < hi; c += blockDim.x) acc[c - c0] = 0.0;
  __syncthreads();
  for (int64_t e = colptr[i]; e < colptr[i + 1]; ++e) {
    const int64_t r = rowidx[e];
    const double a = cval[e];
    // first entry of row r with column >= lo (columns ascending)
    int64_t p = rowptr[r], q = rowptr[r + 1];
    while (p < q) {
      const int64_t mid = (p + q) >> 1;
      if (colidx[mid] < lo) p = mid + 1;
      else q = mid;
    }
    for (int64_t t = p + threadIdx.x; t < rowptr[r + 1]; t += blockDim.x) {
      const int64_t c = colidx[t];
      if (c >= hi) break;
      acc[c - c0] = fma(a, val[t], acc[c - c0]);
    }
    __syncthreads();
  }
  for (int64_t c = lo + threadIdx.x; c < hi; c += blockDim.x) G[i * ldg + c] = acc[c - c0];
}

// ---- 5. Cholesky: diagonal block (nb <= CB) in place, one CTA
__global__ void __launch_bounds__(256) k_chol_diag(double* __restrict__ G, int64_t ldg, int nb,
                                                   int* __restrict__ fail) {
  __shared__ double a[CB][CB + 1];
  __shared__ double s_inv;
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int r = e / nb, c = e % nb;
    a[r][c] = c >= r ? G[r * ldg + c] : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (threadIdx.x == 0) {
      double piv = a[j][j];
      if (!(piv > 0.0)) {
        atomicExch(fail, 1);
        piv = 1.0;
      }
      const double r = sqrt(piv);
      a[j][j] = r;
      s_inv = 1.0 / r;
    }
    __syncthreads();
    for (int c = j + 1 + threadIdx.x; c < nb; c += blockDim.x) a[j][c] *= s_inv;
    __syncthreads();
    const int w = nb - j - 1;  // trailing upper triangle (i, c), j < i <= c
    for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
      const int i = j + 1 + e / w, c = j + 1 + e % w;
      if (c >= i) a[i][c] = fma(-a[j][i], a[j][c], a[i][c]);
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int r = e / nb, c = e % nb;
    if (c >= r) G[r * ldg + c] = a[r][c];
  }
}

// R12 = R11^{-T} G12 in place: thread per column of the panel (rows k0..k0+nb)
__global__ void __launch_bounds__(128) k_chol_panel(double* __restrict__ G, int64_t ldg, int nb, int64_t ncol) {
  __shared__ double r11[CB][CB + 1];
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int r = e / nb, c = e % nb;
    r11[r][c] = c >= r ? G[r * ldg + c] : 0.0;
  }
  __syncthreads();
  const int64_t c = nb + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;  // column of the block row
  if (c >= nb + ncol) return;
  double y[CB];
#pragma unroll
  for (int i = 0; i < CB; ++i) {
    if (i < nb) {
      double t = G[i * ldg + c];
#pragma unroll
      for (int k = 0; k < CB; ++k)
        if (k < i) t = fma(-r11[k][i], y[k], t);
      y[i] = t / r11[i][i];
    }
  }
#pragma unroll
  for (int i = 0; i < CB; ++i)
    if (i < nb) G[i * ldg + c] = y[i];
}

__global__ void k_zero_lower(int64_t d, double* __restrict__ R, int64_t ldr) {
  const int64_t r = blockIdx.y * (int64_t)blockDim.y + threadIdx.y;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < d && c < r;
       c += (int64_t)gridDim.x * blockDim.x)
    R[r * ldr + c] = 0.0;
}

// ---- 6. c = SA^T Sb (warp per column, rows ascending)
__global__ void k_sat_sb(int64_t d, const int64_t* __restrict__ colptr, const int32_t* __restrict__ rowidx,
                         const double* __restrict__ cval, const double* __restrict__ Sb, int64_t ldsb,
                         double* __restrict__ c) {
  const int64_t col = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (col >= d) return;
  double s = 0.0;
  for (int64_t e = colptr[col] + lane; e < colptr[col + 1]; e += 32) s = fma(cval[e], Sb[rowidx[e] * ldsb], s);
  s = ski_warp_sum(s);
  if (lane == 0) c[col] = s;
}

// forward substitution R11^T y = c for one diagonal block (in place in c)
__global__ void __launch_bounds__(256) k_trsv_t_diag(const double* __restrict__ R, int64_t ldr, int nb,
                                                     double* __restrict__ c) {
  __shared__ double y[256];
  __shared__ double part[8][33];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = 0; i < nb; ++i) {
    // y_i = (c_i - sum_{k<i} R[k][i] y_k) / R[i][i]
    double t = 0.0;
    for (int k = threadIdx.x; k < i; k += blockDim.x) t = fma(R[k * ldr + i], y[k], t);
    t = ski_warp_sum(t);
    if (lane == 0) part[wid][0] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < 8; ++w) s += part[w][0];
      y[i] = (c[i] - s) / R[i * ldr + i];
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < nb; i += blockDim.x) c[i] = y[i];
}

}  // namespace

size_t ski_gram_ws_bytes(int64_t n, int64_t d, int64_t nnz, int32_t s, int64_t m) {
  SkiArena ar{nullptr, 0, 0, true};
  const int64_t cap = (int64_t)s * nnz;
  ar.take<char>(ski_bucket_ws_bytes(n, s, m));
  ar.take<int32_t>(m);          // ub
  ar.take<int64_t>(m + 1);      // ubptr
  ar.take<int32_t>(m);          // rowlen
  ar.take<int32_t>(cap);        // ub-layout columns
  ar.take<double>(cap);         // ub-layout values
  ar.take<int64_t>(m + 1);      // compact rowptr
  ar.take<int32_t>(cap);        // compact columns
  ar.take<double>(cap);         // compact values
  ar.take<int64_t>(d + 1);      // CSC colptr
  ar.take<int32_t>(cap);        // CSC rows
  ar.take<double>(cap);         // CSC values
  ar.take<char>(ski_csc_ws_bytes(m, d, cap));
  ar.take<double>(d);           // SA^T Sb
  ar.take<int>(1);              // failure flag
  return ar.off;
}

ski_status ski_gram_chol_run(const ski_matrix* A, uint64_t seed, int32_t s, int32_t replace, int64_t m,
                             const double* Sb, int64_t ldsb, double* R, int64_t ldr, double* qtsb, bool* ok,
                             SkiArena& ar, cudaStream_t st) {
  *ok = false;
  const int64_t n = A->n, d = A->d, nnz = A->nnz, cap = (int64_t)s * nnz;
  if (A->kind != SKI_CSR || d < 1 || m < 1 || cap >= (1ll << 31)) return SKI_EINVAL;
  const size_t bkb = ski_bucket_ws_bytes(n, s, m);
  char* bkws = ar.take<char>(bkb);
  int32_t* ub = ar.take<int32_t>(m);
  int64_t* ubptr = ar.take<int64_t>(m + 1);
  int32_t* rowlen = ar.take<int32_t>(m);
  int32_t* ucol = ar.take<int32_t>(cap);
  double* uval = ar.take<double>(cap);
  int64_t* rowptr = ar.take<int64_t>(m + 1);
  int32_t* ccol = ar.take<int32_t>(cap);
  double* cvalr = ar.take<double>(cap);
  int64_t* colptr = ar.take<int64_t>(d + 1);
  int32_t* crow = ar.take<int32_t>(cap);
  double* cval = ar.take<double>(cap);
  const size_t cscb = ski_csc_ws_bytes(m, d, cap);
  char* cscws = ar.take<char>(cscb);
  double* cvec = ar.take<double>(d);
  int* fail = ar.take<int>(1);
  if (!ar.ok() || !fail) return SKI_ENOMEM;
  SKI_CUDA_TRY(cudaMemsetAsync(fail, 0, sizeof(int), st));
  // 1. bucket lists
  SkiArena bar{bkws, bkb, 0, false};
  SkiBuckets bk;
  SKI_TRY(ski_build_buckets(seed, s, replace, m, n, bar, st, &bk, 0));
  // 2. rows of SA
  k_sa_row_bound<<<(unsigned)ski_cdiv(m, 256), 256, 0, st>>>(m, bk.offsets, bk.list, A->rowptr, ub, fail);
  SKI_LAUNCH_CHECK();
  k_scan_counts<<<1, 1024, 0, st>>>(ub, m, ubptr);
  SKI_LAUNCH_CHECK();
  const size_t fsm = (size_t)kRowCap * (sizeof(unsigned long long) + sizeof(double));
  SKI_CUDA_TRY(cudaFuncSetAttribute(k_sa_row_fill, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm));
  k_sa_row_fill<<<(unsigned)m, 256, fsm, st>>>(m, bk.offsets, bk.list, A->rowptr, A->colidx, A->val,
                                              1.0 / sqrt((double)s), ubptr, rowlen, ucol, uval);
  SKI_LAUNCH_CHECK();
  // 3. compact CSR and its CSC
  k_scan_counts<<<1, 1024, 0, st>>>(rowlen, m, rowptr);
  SKI_LAUNCH_CHECK();
  k_sa_compact<<<(unsigned)m, 128, 0, st>>>(m, ubptr, rowptr, ucol, uval, ccol, cvalr);
  SKI_LAUNCH_CHECK();
  int64_t nnz_sa = 0;
  SKI_CUDA_TRY(cudaMemcpyAsync(&nnz_sa, rowptr + m, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  int hfail = 0;
  SKI_CUDA_TRY(cudaMemcpyAsync(&hfail, fail, sizeof(int), cudaMemcpyDeviceToHost, st));
  SKI_CUDA_TRY(cudaStreamSynchronize(st));
  if (hfail) return SKI_OK;  // a row too long for the shared-memory merge: *ok stays false
  ski_matrix sa{};
  sa.kind = SKI_CSR;
  sa.n = m;
  sa.d = d;
  sa.val = cvalr;
  sa.rowptr = rowptr;
  sa.colidx = ccol;
  sa.nnz = nnz_sa;
  SkiArena car{cscws, cscb, 0, false};
  SKI_TRY(ski_csc_build(&sa, colptr, crow, cval, car, st));
  // 4. G (upper) into R
  const int64_t chunk = std::min<int64_t>(d, kGramChunk);
  SKI_CUDA_TRY(cudaFuncSetAttribute(k_gram_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(chunk * sizeof(double))));
  for (int64_t c0 = 0; c0 < d; c0 += chunk) {
    k_gram_rows<<<(unsigned)std::min<int64_t>(d, c0 + chunk), 256, chunk * sizeof(double), st>>>(
        d, colptr, crow, cval, rowptr, ccol, cvalr, R, ldr, c0, chunk);
    SKI_LAUNCH_CHECK();
  }
  // 5. Cholesky in place
  for (int64_t k0 = 0; k0 < d; k0 += CB) {
    const int nb = (int)std::min<int64_t>(CB, d - k0);
    double* Gk = R + k0 * ldr + k0;
    k_chol_diag<<<1, 256, 0, st>>>(Gk, ldr, nb, fail);
    SKI_LAUNCH_CHECK();
    const int64_t rest = d - k0 - nb;
    if (rest > 0) {
      k_chol_panel<<<(unsigned)ski_cdiv(rest, 128), 128, 0, st>>>(Gk, ldr, nb, rest);
      SKI_LAUNCH_CHECK();
      // G22 -= R12^T R12 (tiles meeting the upper triangle only)
      const double* R12 = Gk + nb;
      SKI_TRY(ski_gemm_ex<double>(rest, rest, nb, -1.0, R12, 1, ldr, R12, ldr, 1, 1.0, Gk + nb * ldr + nb, ldr, 1,
                                  0, st, 4));
    }
  }
  {
    dim3 blk(32, 8), grid((unsigned)std::min<int64_t>(64, ski_cdiv(d, 32)), (unsigned)ski_cdiv(d, 8));
    k_zero_lower<<<grid, blk, 0, st>>>(d, R, ldr);
    SKI_LAUNCH_CHECK();
  }
  // 6. Q^T Sb = R^{-T} SA^T Sb
  if (qtsb) {
    k_sat_sb<<<(unsigned)ski_cdiv(d * 32, 256), 256, 0, st>>>(d, colptr, crow, cval, Sb, ldsb, cvec);
    SKI_LAUNCH_CHECK();
    constexpr int TB = 256;
    for (int64_t k0 = 0; k0 < d; k0 += TB) {
      const int nb = (int)std::min<int64_t>(TB, d - k0);
      k_trsv_t_diag<<<1, 256, 0, st>>>(R + k0 * ldr + k0, ldr, nb, cvec + k0);
      SKI_LAUNCH_CHECK();
      const int64_t rest = d - k0 - nb;
      if (rest > 0)  // c[k0+nb:] -= R[k0:k0+nb, k0+nb:]^T y
        SKI_TRY(ski_gemm<double>(rest, 1, nb, -1.0, R + k0 * ldr + k0 + nb, 1, ldr, cvec + k0, 1, 1, 1.0,
                                 cvec + k0 + nb, 1, st));
    }
    SKI_CUDA_TRY(cudaMemcpyAsync(qtsb, cvec, d * sizeof(double), cudaMemcpyDeviceToDevice, st));
  }
  SKI_CUDA_TRY(cudaMemcpyAsync(&hfail, fail, sizeof(int), cudaMemcpyDeviceToHost, st));
  SKI_CUDA_TRY(cudaStreamSynchronize(st));
  *ok = hfail == 0;
  return SKI_OK;
}
