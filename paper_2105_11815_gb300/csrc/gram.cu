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
//     down each column of the panel (four lanes per column in FP64), and
//     G22 -= R12^T R12 on the SIMT GEMM restricted to tiles that meet the
//     upper triangle.  For d > 1024 the FP64 factorisation runs in panels of
//     512 columns, the update across panels from exact FP16 slice products
//     on the tensor cores.  A pivot that is not positive reports failure.
//  6. c = SA^T Sb by columns of SA, then Q^T Sb = R^{-T} c by blocked forward
//     substitution (the diagonal block in one CTA, the rest as GEMV updates).
// On failure the caller factors the dense sketch by Householder QR instead.
// The same Cholesky serves a dense sketch (ski_gram_dense_run), whose Gram
// matrix is a product on the tensor cores: 3xTF32 for FP32, exact FP16 slice
// products summed in FP64 for FP64.
#include <cuda_fp16.h>
#include <math.h>

#include <algorithm>
#include <type_traits>

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

// ---- 5. Cholesky: diagonal block (nb <= CB) in place, 256 threads, in
// bands of RB rows.  Per band: warp 0 factors the RB rows over the block's
// columns with the band in registers (lane l: columns l and l + 32; pivot
// r_jj = sqrt(g_jj) and its reciprocal, row j scaled, the band's later rows
// updated, row entries broadcast by shuffles); then every
// thread applies the band's rank-RB update to its column of the trailing
// upper triangle, g_ic -= sum_q r_qi r_qc (threads over columns, rows strided
// by 4).  The reciprocals 1 / r_jj go to dinv for the block-row solve.
// *fail is set on a pivot that is not positive (1 is used for it).
template <class T>
__global__ void __launch_bounds__(256) k_chol_diag(T* __restrict__ G, int64_t ldg, int nb, T* __restrict__ dinv,
                                                   int* __restrict__ fail) {
  constexpr int RB = 8, RS = 256 / CB;  // band rows; row stride of the trailing update
  __shared__ T a[CB][CB + 1];
  const int tid = threadIdx.x, tx = tid & (CB - 1), ty = tid / CB;
  {
    constexpr int RPT = CB / RS;  // rows per thread
    T v[RPT];
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int r = ty + q * RS;
      v[q] = (r < nb && tx < nb && tx >= r) ? G[r * ldg + tx] : T(0);
    }
#pragma unroll
    for (int q = 0; q < RPT; ++q) a[ty + q * RS][tx] = v[q];
  }
  __syncthreads();
  for (int j0 = 0; j0 < nb; j0 += RB) {
    const int je = min(nb, j0 + RB);
    if (tid < 32) {
      // the band in registers: rows j0 + q, columns tid and tid + 32
      T v0[RB], v1[RB];
#pragma unroll
      for (int q = 0; q < RB; ++q) {
        v0[q] = a[j0 + q][tid];
        v1[q] = a[j0 + q][tid + 32];
      }
#pragma unroll
      for (int q = 0; q < RB; ++q) {
        const int j = j0 + q;
        if (j < je) {
          T piv = __shfl_sync(0xffffffffu, j < 32 ? v0[q] : v1[q], j & 31);
          const bool bad = !(piv > T(0));
          if (bad) piv = T(1);
          // one reciprocal square root and a product (within an ulp or two of
          // sqrt and its reciprocal): the shortest chain on the pivot's path
          const T ir = rsqrt(piv), r = piv * ir;
          if (tid == 0) {
            if (bad) atomicExch(fail, 1);
            dinv[j] = ir;
          }
          v0[q] = tid == j ? r : (tid > j ? v0[q] * ir : v0[q]);
          v1[q] = tid + 32 == j ? r : (tid + 32 > j ? v1[q] * ir : v1[q]);
#pragma unroll
          for (int p = q + 1; p < RB; ++p) {
            const int i = j0 + p;
            const T rji = __shfl_sync(0xffffffffu, i < 32 ? v0[q] : v1[q], i & 31);
            if (tid >= i) v0[p] = fma(-rji, v0[q], v0[p]);
            if (tid + 32 >= i) v1[p] = fma(-rji, v1[q], v1[p]);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < RB; ++q) {
        a[j0 + q][tid] = v0[q];
        a[j0 + q][tid + 32] = v1[q];
      }
    }
    __syncthreads();
    if (tx >= je && tx < nb) {
      T rc[RB];
#pragma unroll
      for (int q = 0; q < RB; ++q) rc[q] = j0 + q < je ? a[j0 + q][tx] : T(0);
      for (int i = je + ty; i <= tx; i += RS) {
        T s = a[i][tx];
#pragma unroll
        for (int q = 0; q < RB; ++q) s = fma(-(j0 + q < je ? a[j0 + q][i] : T(0)), rc[q], s);
        a[i][tx] = s;
      }
    }
    __syncthreads();
  }
  for (int r = ty; r < nb; r += RS)
    if (tx >= r && tx < nb) G[r * ldg + tx] = a[r][tx];
}

// block row R12 = R11^{-T} G12 in place, one thread per column of G12 (the
// column in registers, R11 broadcast from shared memory): forward
// substitution y_i = (g_i - sum_{k<i} r_ki y_k) / r_ii with the reciprocals
// from the diagonal kernel.  For the tensor-core update the column also goes
// to row c of Pt (rest x CB, zeros past nb).
template <class T>
__global__ void __launch_bounds__(32) k_trsm_row(T* __restrict__ Gk, int64_t ldg, int nb, int64_t rest,
                                                 const T* __restrict__ dinv, T* __restrict__ Pt) {
  __shared__ T r[CB][CB];
  __shared__ T di[CB];
  const int tid = threadIdx.x;
#pragma unroll 1
  for (int i0 = 0; i0 < CB; i0 += 16) {
    T v[16][2];
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = i0 + u, k = tid + 32 * h;
        v[u][h] = (i < nb && k > i && k < nb) ? Gk[i * ldg + k] : T(0);
      }
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int h = 0; h < 2; ++h) r[i0 + u][tid + 32 * h] = v[u][h];
  }
  for (int i = tid; i < CB; i += 32) di[i] = i < nb ? dinv[i] : T(0);
  __syncthreads();
  const int64_t c = blockIdx.x * 32ll + tid;
  if (c >= rest) return;
  T g[CB];
#pragma unroll
  for (int i = 0; i < CB; ++i) g[i] = i < nb ? Gk[i * ldg + nb + c] : T(0);
#pragma unroll
  for (int i = 0; i < CB; ++i) {
    const T y = g[i] * di[i];
    g[i] = y;
#pragma unroll
    for (int k = i + 1; k < CB; ++k) g[k] = fma(-r[i][k], y, g[k]);
  }
#pragma unroll
  for (int i = 0; i < CB; ++i)
    if (i < nb) Gk[i * ldg + nb + c] = g[i];
  if (Pt) {
#pragma unroll
    for (int i = 0; i < CB; ++i) Pt[c * CB + i] = g[i];
  }
}

// The same block-row solve with four lanes per column (FP64, where the
// FP64 pipe sets the pace): lane t of a column's group holds rows t + 4q; at
// step i the owner of row i forms y_i and a shuffle gives it to the group,
// which updates its later rows.  A warp takes 8 columns, so the columns
// spread over several CTAs per SM and nothing spills.
__global__ void __launch_bounds__(32) k_trsm_row4(double* __restrict__ Gk, int64_t ldg, int nb, int64_t rest,
                                                  const double* __restrict__ dinv) {
  __shared__ double r[CB][CB];
  __shared__ double di[CB];
  const int lane = threadIdx.x, t = lane & 3;
#pragma unroll 1
  for (int i0 = 0; i0 < CB; i0 += 16) {
    double v[16][2];
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = i0 + u, k = lane + 32 * h;
        v[u][h] = (i < nb && k > i && k < nb) ? Gk[i * ldg + k] : 0.0;
      }
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int h = 0; h < 2; ++h) r[i0 + u][lane + 32 * h] = v[u][h];
  }
  for (int i = lane; i < CB; i += 32) di[i] = i < nb ? dinv[i] : 0.0;
  __syncthreads();
  const int64_t c = blockIdx.x * 8ll + (lane >> 2);
  const bool on = c < rest;
  double g[CB / 4];
#pragma unroll
  for (int q = 0; q < CB / 4; ++q) {
    const int k = t + 4 * q;
    g[q] = (on && k < nb) ? Gk[k * ldg + nb + c] : 0.0;
  }
#pragma unroll
  for (int i = 0; i < CB; ++i) {
    const int qi = i >> 2, ti = i & 3;
    if (t == ti) g[qi] *= di[i];
    const double y = __shfl_sync(0xffffffffu, g[qi], (lane & ~3) | ti);
#pragma unroll
    for (int q = (i >> 2); q < CB / 4; ++q)
      if (t + 4 * q > i) g[q] = fma(-r[i][t + 4 * q], y, g[q]);
  }
  if (!on) return;
#pragma unroll
  for (int q = 0; q < CB / 4; ++q) {
    const int k = t + 4 * q;
    if (k < nb) Gk[k * ldg + nb + c] = g[q];
  }
}

__global__ void k_zero_lower(int64_t d, double* __restrict__ R, int64_t ldr) {
  const int64_t r = blockIdx.y * (int64_t)blockDim.y + threadIdx.y;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < d && c < r;
       c += (int64_t)gridDim.x * blockDim.x)
    R[r * ldr + c] = 0.0;
}

// R (FP64, upper, zeros below) from the upper triangle of an FP32 factor
__global__ void k_upper_to_f64(int64_t d, const float* __restrict__ G, int64_t ldg, double* __restrict__ R,
                               int64_t ldr) {
  const int64_t r = blockIdx.y * (int64_t)blockDim.y + threadIdx.y;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < d && c < d;
       c += (int64_t)gridDim.x * blockDim.x)
    R[r * ldr + c] = c >= r ? (double)G[r * ldg + c] : 0.0;
}

// SA^T Sb of a dense sketch [SA | Sb] (m x (d + 1), row stride lda), in
// FP64 accumulation: part[z][i] sums rows [z rows_per, (z + 1) rows_per) of
// SA[r][i] Sb[r] (threads over columns, rows in flight eight at a time), and
// k_sum_parts adds the chunks in order
template <class T>
__global__ void __launch_bounds__(128) k_sat_sb_part(int64_t m, int64_t d, const T* __restrict__ A, int64_t lda,
                                                     int64_t rows_per, double* __restrict__ part) {
  const int64_t i = blockIdx.x * 128ll + threadIdx.x;
  const int64_t r0 = blockIdx.y * rows_per, r1 = std::min<int64_t>(m, r0 + rows_per);
  if (i >= d) return;
  double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int64_t r = r0; r < r1; r += 8) {
    double a[8], b[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const bool in = r + u < r1;
      a[u] = in ? (double)A[(r + u) * lda + i] : 0.0;
      b[u] = in ? (double)A[(r + u) * lda + d] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] = fma(a[u], b[u], acc[u]);
  }
  part[blockIdx.y * d + i] = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
}

__global__ void k_sum_parts(int64_t d, int nz, const double* __restrict__ part, double* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= d) return;
  double s = 0.0;
  for (int z = 0; z < nz; ++z) s += part[z * d + i];
  out[i] = s;
}

constexpr int64_t kSatRows = 256;  // rows of the sketch per partial sum

// ---- FP64 Gram matrix from exact slice products on the tensor cores.
// Column j of SA is scaled by 2^-e_j (every |a_rj| < 2^e_j) and cut into
// integer slices of beta bits: x = a 2^-e_j = sum_k 2^(-beta k) S_k + rho,
// the S_k the balanced base-2^beta digits of round(2^(beta s) x), so
// |S_1| <= 2^beta, |S_k| <= 2^(beta-1) after it and |rho| <= 2^(-beta s - 1).  A product of
// slices summed over m rows stays below m 2^(2 beta) < 2^24, so the tensor
// cores' FP32 accumulation of FP16 slice products is exact; G = 2^(e_i + e_j)
// sum over k + l <= s + 1 of 2^(-beta (k + l)) S_k^T S_l, added in FP64 in
// decreasing order of magnitude.  Pairs of one weight k + l share an FP32
// accumulator while the bound on its sum stays below 2^24.  The dropped
// pairs are below 2^(-beta s) per row of the normalised columns.
int oz_beta(int64_t m) {
  int lg = 0;
  while ((1ll << lg) <= m) ++lg;  // m < 2^lg
  return (24 - lg) / 2;
}
int oz_slices(int beta) { return (54 + beta - 1) / beta; }
constexpr int kOzMinBeta = 4;  // below it (m >= 2^16) the FP64 SIMT GEMM forms G

// e_j: an exponent with every |a_rj| (r < m) below 2^e_j; the caller fills e
// with a very negative value first (a zero column keeps exponent 0).  A NaN
// or infinite entry sets *fail (the Gram factor is then not used).
__global__ void __launch_bounds__(128) k_col_exp(int64_t m, int64_t d, const double* __restrict__ A, int64_t lda,
                                                 int64_t rows_per, int* __restrict__ e, int* __restrict__ fail) {
  const int64_t j = blockIdx.x * 128ll + threadIdx.x;
  const int64_t r0 = blockIdx.y * rows_per, r1 = std::min<int64_t>(m, r0 + rows_per);
  if (j >= d) return;
  double mx = 0.0;
  bool bad = false;
  for (int64_t r = r0; r < r1; ++r) {
    const double a = fabs(A[r * lda + j]);
    bad |= !(a <= 1.7976931348623157e308);
    mx = fmax(mx, a);
  }
  if (bad) {
    atomicExch(fail, 1);
    return;
  }
  int ex = 0;
  frexp(mx, &ex);
  atomicMax(&e[j], ex);
}

// v = round(a 2^(bits - e)) as an integer, for |a| < 2^e (so |v| <= 2^bits),
// from a's bit pattern: a = +-M 2^(E - 1075) with the 53-bit M.  Integer
// operations only (the FP64 pipe is slow here).
__device__ __forceinline__ long long oz_fixed(double a, int e, int bits) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(a);
  const int E = (int)((u >> 52) & 0x7FF);
  unsigned long long M = u & 0xFFFFFFFFFFFFFull;
  if ((E == 0 && M == 0) || E == 0x7FF) return 0;  // zero; NaN / Inf are flagged by k_col_exp
  int ex = E;
  if (E != 0) M |= 1ull << 52;
  else ex = 1;  // subnormal
  const int sh = ex - 1075 - e + bits;
  unsigned long long v;
  if (sh >= 0) v = M << sh;  // |a| < 2^e keeps v below 2^bits
  else if (sh > -64) v = (M + (1ull << (-sh - 1))) >> -sh;
  else v = 0;
  return (u >> 63) ? -(long long)v : (long long)v;
}

// slices of a 64-row x 32-column tile of SA, transposed: Sl[k][j][r] (FP16,
// row stride lds, slice stride sstride).  Thread (tx, ty) takes column
// j0 + tx, rows r0 + ty + 8 q: v = round(x 2^(beta ns)) in int64, cut into
// balanced base-2^beta digits from the low end (each in [-2^(beta-1),
// 2^(beta-1)), the leading one what remains, |S_1| <= 2^beta); the tile is
// transposed through shared memory so that each slice row is written as
// 128-byte segments.
__global__ void __launch_bounds__(256) k_oz_slice(int64_t m, int64_t d, const double* __restrict__ A, int64_t lda,
                                                  const int* __restrict__ e, int beta, int ns,
                                                  __half* __restrict__ Sl, int64_t lds, int64_t sstride) {
  extern __shared__ __align__(16) unsigned char oz_raw[];
  __half* t = reinterpret_cast<__half*>(oz_raw);  // [ns][32][66]
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t j0 = (int64_t)blockIdx.y * 32, r0 = (int64_t)blockIdx.x * 64, j = j0 + tx;
  const int ej = j < d ? e[j] : 0;
  const long long mask = (1ll << beta) - 1, half_ = 1ll << (beta - 1);
  double av[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int64_t r = r0 + ty + 8 * q;
    av[q] = (r < m && j < d) ? A[r * lda + j] : 0.0;
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int rl = ty + 8 * q;
    long long v = oz_fixed(av[q], ej, beta * ns);
    for (int k = ns - 1; k >= 1; --k) {
      long long dg = v & mask;
      if (dg >= half_) dg -= (1ll << beta);
      v = (v - dg) >> beta;  // exact: v - dg is a multiple of 2^beta
      t[(k * 32 + tx) * 66 + rl] = __int2half_rn((int)dg);
    }
    t[tx * 66 + rl] = __int2half_rn((int)v);  // |v| <= 2^beta: exact
  }
  __syncthreads();
  // slice k, column jl: 64 halves = 32 words, one per lane
  for (int w = ty; w < ns * 32; w += 8) {
    const int k = w >> 5, jl = w & 31;
    const int64_t jj = j0 + jl, r = r0 + 2 * tx;
    if (jj >= d || r >= m) continue;
    const __half* src = t + (k * 32 + jl) * 66 + 2 * tx;
    __half* dst = Sl + k * sstride + jj * lds + r;
    if (r + 1 < m) {
      *reinterpret_cast<__half2*>(dst) = __halves2half2(src[0], src[1]);
    } else {
      dst[0] = src[0];
    }
  }
}

// G[i][j] *= 2^(e_i + e_j) on the upper triangle
__global__ void k_oz_scale(int64_t d, double* __restrict__ G, int64_t ldg, const int* __restrict__ e) {
  const int64_t i = blockIdx.y * (int64_t)blockDim.y + threadIdx.y;
  if (i >= d) return;
  const int ei = e[i];
  for (int64_t j = i + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d; j += (int64_t)gridDim.x * blockDim.x)
    G[i * ldg + j] = ldexp(G[i * ldg + j], ei + e[j]);
}

int64_t oz_lds(int64_t m) { return ski_round_up(m, 8); }

// Optional CUDA-event timing of the Gram matrix product (one span on the
// launching stream); ms() after the stream has been synchronised
struct SpanTimer {
  cudaEvent_t e[2] = {nullptr, nullptr};
  bool on;
  explicit SpanTimer(bool enable) : on(enable) {
    if (on && (cudaEventCreate(&e[0]) != cudaSuccess || cudaEventCreate(&e[1]) != cudaSuccess)) on = false;
  }
  ~SpanTimer() {
    for (auto x : e)
      if (x) cudaEventDestroy(x);
  }
  void mark(int i, cudaStream_t st) {
    if (on) cudaEventRecord(e[i], st);
  }
  double ms() {
    float t = 0.f;
    return on && cudaEventElapsedTime(&t, e[0], e[1]) == cudaSuccess ? t : 0.0;
  }
};

// P (upper triangle, d x d, row stride ldg) = the slice sum of A^T A for the
// FP64 A (m x d, row stride lda) without the column scales: P[i][j] 2^(e_i +
// e_j) = (A^T A)[i][j].  e: d ints, Sl: ns d lds halves of scratch.
ski_status oz_products(const double* A, int64_t lda, int64_t m, int64_t d, double* G, int64_t ldg, int* e,
                       __half* Sl, int* fail, SpanTimer& tm, cudaStream_t st) {
  const int beta = oz_beta(m), ns = oz_slices(beta);
  const int64_t lds = oz_lds(m), sstride = d * lds;
  SKI_CUDA_TRY(cudaMemsetAsync(e, 0x80, d * sizeof(int), st));
  const int64_t nz = ski_cdiv(m, kSatRows);
  k_col_exp<<<dim3((unsigned)ski_cdiv(d, 128), (unsigned)nz), 128, 0, st>>>(m, d, A, lda, kSatRows, e, fail);
  SKI_LAUNCH_CHECK();
  // the attribute is set once, for the most slices (the fewest bits) taken
  const size_t smem = (size_t)ns * 32 * 66 * sizeof(__half);
  SKI_CUDA_TRY(ski_attr_once((const void*)k_oz_slice, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              [] { return (int)((size_t)oz_slices(kOzMinBeta) * 32 * 66 * sizeof(__half)); }));
  k_oz_slice<<<dim3((unsigned)ski_cdiv(m, 64), (unsigned)ski_cdiv(d, 32)), 256, smem, st>>>(m, d, A, lda, e, beta, ns,
                                                                                           Sl, lds, sstride);
  SKI_LAUNCH_CHECK();
  SKI_CUDA_TRY(cudaMemset2DAsync(G, ldg * sizeof(double), 0, d * sizeof(double), d, st));
  tm.mark(0, st);
  // the pairs of one weight t = k + l share an accumulator while the bound
  // on its sum, m |S_k|max |S_l|max summed over them, stays below 2^24
  // (|S_1| <= 2^beta, |S_k| <= 2^(beta-1) after it)
  auto smax = [&](int k) { return k == 1 ? (double)(1 << beta) : (double)(1 << (beta - 1)); };
  for (int tt = 2; tt <= ns + 1; ++tt) {
    TcPairs pr{};
    double bound = 0.0;
    auto flush = [&]() -> ski_status {
      if (pr.n == 0) return SKI_OK;
      SKI_TRY(ski_gemm_f16_pairs_f64acc(Sl, lds, sstride, ns, d, m, pr, G, ldg, ldexp(1.0, -beta * tt), true, fail,
                                        st));
      pr.n = 0;
      bound = 0.0;
      return SKI_OK;
    };
    for (int k = std::max(1, tt - ns); k <= std::min(ns, tt - 1); ++k) {
      const double b = (double)m * smax(k) * smax(tt - k);
      if (pr.n == kTcMaxPairs || (pr.n > 0 && bound + b >= 16777216.0)) SKI_TRY(flush());
      pr.a[pr.n] = (int8_t)(k - 1);
      pr.b[pr.n] = (int8_t)(tt - k - 1);
      ++pr.n;
      bound += b;
    }
    SKI_TRY(flush());
  }
  tm.mark(1, st);
  return SKI_OK;
}

// G (upper triangle, d x d, row stride ldg) = SA^T SA for the FP64 SA (m x d,
// row stride lda), from exact slice products
ski_status oz_gram(const double* A, int64_t lda, int64_t m, int64_t d, double* G, int64_t ldg, int* e, __half* Sl,
                   int* fail, SpanTimer& tm, cudaStream_t st) {
  SKI_TRY(oz_products(A, lda, m, d, G, ldg, e, Sl, fail, tm, st));
  dim3 blk(32, 8), grid((unsigned)std::min<int64_t>(64, ski_cdiv(d, 32)), (unsigned)ski_cdiv(d, 8));
  k_oz_scale<<<grid, blk, 0, st>>>(d, G, ldg, e);
  SKI_LAUNCH_CHECK();
  return SKI_OK;
}

// C[i][j] -= P[i][j] 2^(e_i + e_j) on the upper triangle (n x n)
__global__ void k_oz_sub(int64_t n, double* __restrict__ C, int64_t ldc, const double* __restrict__ P, int64_t ldp,
                         const int* __restrict__ e) {
  const int64_t i = blockIdx.y * (int64_t)blockDim.y + threadIdx.y;
  if (i >= n) return;
  const int ei = e[i];
  for (int64_t j = i + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    C[i * ldc + j] -= ldexp(P[i * ldp + j], ei + e[j]);
}

template <class T>
ski_status sat_sb_dense(const T* A, int64_t lda, int64_t m, int64_t d, double* part, double* out, cudaStream_t st) {
  const int64_t nz = ski_cdiv(m, kSatRows);
  k_sat_sb_part<T><<<dim3((unsigned)ski_cdiv(d, 128), (unsigned)nz), 128, 0, st>>>(m, d, A, lda, kSatRows, part);
  SKI_LAUNCH_CHECK();
  k_sum_parts<<<(unsigned)ski_cdiv(d, 256), 256, 0, st>>>(d, (int)nz, part, out);
  SKI_LAUNCH_CHECK();
  return SKI_OK;
}

// rows [0, ncols) of X^T: X m x ncols (row-major, ldx) -> Xt ncols x ldt
__global__ void k_transpose_f32(int64_t m, int64_t ncols, const float* __restrict__ X, int64_t ldx,
                                float* __restrict__ Xt, int64_t ldt) {
  __shared__ float tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32, c0 = (int64_t)blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t r = r0 + k, c = c0 + threadIdx.x;
    tile[k][threadIdx.x] = (r < m && c < ncols) ? X[r * ldx + c] : 0.f;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t c = c0 + k, r = r0 + threadIdx.x;
    if (c < ncols && r < m) Xt[c * ldt + r] = tile[threadIdx.x][k];
  }
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

// gdiag[j] = G[j][j] (the Gram matrix's diagonal, before the factorisation)
template <class T>
__global__ void k_save_diag(int64_t d, const T* __restrict__ G, int64_t ld, double* __restrict__ gdiag) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j < d) gdiag[j] = (double)G[j * ld + j];
}

// *eq = max_j sqrt(g_jj) / r_jj: r_jj / |a_j| is the distance of column j of
// SA from the span of the columns before it, relative to its length, so eq is
// a lower bound on the condition number of SA with its columns scaled to unit
// length (infinite for a pivot that is not positive or not finite).  One CTA.
template <class T>
__global__ void __launch_bounds__(256) k_eq_ratio(int64_t d, const T* __restrict__ R, int64_t ld,
                                                  const double* __restrict__ gdiag, double* __restrict__ eq) {
  __shared__ double red[256];
  double mx = 0.0;
  for (int64_t j = threadIdx.x; j < d; j += 256) {
    const double r = (double)R[j * ld + j], g = gdiag[j];
    const double q = (r > 0.0 && isfinite(r) && isfinite(g)) ? sqrt(fmax(g, 0.0)) / r : INFINITY;
    mx = fmax(mx, q);
  }
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *eq = red[0];
}

// G (upper triangle, ld) := its Cholesky factor R (R^T R = G) in place:
// blocked right-looking, blocks of CB.  Per block: the diagonal factor (one
// CTA), the block row R12 = R11^{-T} G12 (one thread per column), and the
// trailing G22 -= R12^T R12 -- in FP32 on the tensor cores (three TF32
// passes) from the transposed block row Pt, in FP64 on the SIMT GEMM over the
// tiles that meet the upper triangle.  Scratch: dinv (CB), gdiag (d), and
// for FP32 Pt (d x CB).  *fail is set on a pivot that is not positive or a
// tensor-core wait that gave up; *eq receives the column-scaled diagonal
// ratio of k_eq_ratio.
template <class T>
ski_status chol_upper(T* G, int64_t ld, int64_t d, T* dinv, T* Pt, double* gdiag, double* eq, int* fail,
                      cudaStream_t st) {
  k_save_diag<T><<<(unsigned)ski_cdiv(d, 256), 256, 0, st>>>(d, G, ld, gdiag);
  SKI_LAUNCH_CHECK();
  for (int64_t k0 = 0; k0 < d; k0 += CB) {
    const int nb = (int)std::min<int64_t>(CB, d - k0);
    T* Gk = G + k0 * ld + k0;
    k_chol_diag<T><<<1, 256, 0, st>>>(Gk, ld, nb, dinv, fail);
    SKI_LAUNCH_CHECK();
    const int64_t rest = d - k0 - nb;
    if (rest <= 0) continue;
    if constexpr (std::is_same<T, float>::value) {
      k_trsm_row<T><<<(unsigned)ski_cdiv(rest, 32), 32, 0, st>>>(Gk, ld, nb, rest, dinv, Pt);
    } else {
      k_trsm_row4<<<(unsigned)ski_cdiv(rest, 8), 32, 0, st>>>(Gk, ld, nb, rest, dinv);
    }
    SKI_LAUNCH_CHECK();
    T* G22 = Gk + nb * ld + nb;
    if constexpr (std::is_same<T, float>::value) {
      SKI_TRY(ski_gemm_tf32(Pt, CB, Pt, CB, rest, rest, CB, G22, ld, 1 | 4, 1, 0, fail, st, true));
    } else {
      const T* R12 = Gk + nb;
      SKI_TRY(ski_gemm_ex<T>(rest, rest, nb, T(-1), R12, 1, ld, R12, ld, 1, T(1), G22, ld, 1, 0, st, 4));
    }
  }
  k_eq_ratio<T><<<1, 256, 0, st>>>(d, G, ld, gdiag, eq);
  SKI_LAUNCH_CHECK();
  return SKI_OK;
}

// FP64 Cholesky in two levels: panels of kOzPanel columns; inside a panel the
// blocks of CB as above, with the rank-CB update applied only to the panel's
// later rows (over every column to their right); across panels one update
// G22 -= R12^T R12 with K = the panel's rows, from exact FP16 slice products
// of R12 on the tensor cores (P = the unscaled product, then G22 -= P scaled
// by the column exponents).  Scratch (chol2_bytes): e (d ints), the slices
// of one panel's R12, P (d x d).
constexpr int64_t kOzPanel = 512;
size_t chol2_bytes(int64_t d) {
  SkiArena ar{nullptr, 0, 0, true};
  ar.take<int>(d);
  ar.take<__half>((int64_t)oz_slices(oz_beta(kOzPanel)) * d * oz_lds(kOzPanel));
  ar.take<double>(d * d);
  return ar.off;
}
bool chol2_applies(int64_t d) { return d > 2 * kOzPanel; }

ski_status chol_upper2(double* G, int64_t ld, int64_t d, double* dinv, double* gdiag, double* eq, int* fail,
                       SkiArena& ar, cudaStream_t st) {
  int* e = ar.take<int>(d);
  __half* Sl = ar.take<__half>((int64_t)oz_slices(oz_beta(kOzPanel)) * d * oz_lds(kOzPanel));
  double* P = ar.take<double>(d * d);
  if (!ar.ok() || !P) return SKI_ENOMEM;
  SpanTimer none(false);
  k_save_diag<double><<<(unsigned)ski_cdiv(d, 256), 256, 0, st>>>(d, G, ld, gdiag);
  SKI_LAUNCH_CHECK();
  for (int64_t K0 = 0; K0 < d; K0 += kOzPanel) {
    const int64_t Ke = std::min(d, K0 + kOzPanel);
    for (int64_t k0 = K0; k0 < Ke; k0 += CB) {
      const int nb = (int)std::min<int64_t>(CB, Ke - k0);
      double* Gk = G + k0 * ld + k0;
      k_chol_diag<double><<<1, 256, 0, st>>>(Gk, ld, nb, dinv, fail);
      SKI_LAUNCH_CHECK();
      const int64_t rest = d - k0 - nb;
      if (rest <= 0) continue;
      k_trsm_row4<<<(unsigned)ski_cdiv(rest, 8), 32, 0, st>>>(Gk, ld, nb, rest, dinv);
      SKI_LAUNCH_CHECK();
      const int64_t rows = Ke - k0 - nb;  // the panel's later rows
      if (rows > 0) {
        const double* R12 = Gk + nb;
        SKI_TRY(ski_gemm_ex<double>(rows, rest, nb, -1.0, R12, 1, ld, R12, ld, 1, 1.0, Gk + nb * ld + nb, ld, 1, 0,
                                    st, 4));
      }
    }
    const int64_t rest = d - Ke;
    if (rest <= 0) continue;
    // G22 -= R12^T R12: R12 = rows [K0, Ke), columns [Ke, d)
    SKI_TRY(oz_products(G + K0 * ld + Ke, ld, Ke - K0, rest, P, rest, e, Sl, fail, none, st));
    dim3 blk(32, 8), grid((unsigned)std::min<int64_t>(64, ski_cdiv(rest, 32)), (unsigned)ski_cdiv(rest, 8));
    k_oz_sub<<<grid, blk, 0, st>>>(rest, G + Ke * ld + Ke, ld, P, rest, e);
    SKI_LAUNCH_CHECK();
  }
  k_eq_ratio<double><<<1, 256, 0, st>>>(d, G, ld, gdiag, eq);
  SKI_LAUNCH_CHECK();
  return SKI_OK;
}

// forward substitution R11^T y = c for one diagonal block of nb <= 64 rows,
// in place in c: the block is staged in shared memory by 256 threads (all
// loads in flight at once), then one warp solves: the reciprocals of the
// diagonal are taken up front (two per lane); lane l holds c_l and c_{l+32}.
// Step i: the owner of c_i forms y_i = c_i / r_ii, a shuffle broadcasts it,
// and each lane subtracts r_ij y_i from its later c_j.
__global__ void __launch_bounds__(256) k_trsv_t_diag(const double* __restrict__ R, int64_t ldr, int nb,
                                                     double* __restrict__ c) {
  __shared__ double r[64][65];
  {
    const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
    double v[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int i = ty + 4 * q;
      v[q] = (i < nb && tx < nb) ? R[(int64_t)i * ldr + tx] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) r[ty + 4 * q][tx] = v[q];
  }
  __syncthreads();
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  const double inv0 = lane < nb ? 1.0 / r[lane][lane] : 0.0;
  const double inv1 = lane + 32 < nb ? 1.0 / r[lane + 32][lane + 32] : 0.0;
  double c0 = lane < nb ? c[lane] : 0.0, c1 = lane + 32 < nb ? c[lane + 32] : 0.0;
  for (int i = 0; i < nb; ++i) {
    const bool lo = i < 32;
    if (lane == (i & 31)) {
      if (lo) c0 *= inv0;
      else c1 *= inv1;
    }
    const double y = __shfl_sync(0xffffffffu, lo ? c0 : c1, i & 31);
    if (lane > i && lane < nb) c0 = fma(-r[i][lane], y, c0);
    if (lane + 32 > i && lane + 32 < nb) c1 = fma(-r[i][lane + 32], y, c1);
  }
  if (lane < nb) c[lane] = c0;
  if (lane + 32 < nb) c[lane + 32] = c1;
}

// c_j -= sum_{i < nb} r_ij y_i for the rest columns j: a CTA takes 32
// columns, its 8 warps 8 rows each (one load round trip), and the 8 partial
// sums of a column are added in shared memory in a fixed order
__global__ void __launch_bounds__(256) k_gemv_t_sub(const double* __restrict__ R, int64_t ldr, int nb, int64_t rest,
                                                    const double* __restrict__ y, double* __restrict__ c) {
  __shared__ double part[8][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t j = blockIdx.x * 32ll + lane;
  double v[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int i = w * 8 + u;
    v[u] = (i < nb && j < rest) ? R[(int64_t)i * ldr + j] * y[i] : 0.0;
  }
  part[w][lane] = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
  __syncthreads();
  if (w == 0 && j < rest) {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) s += part[q][lane];
    c[j] -= s;
  }
}

// R^T y = c in place (R upper, FP64): the diagonal blocks by one warp, the
// rest as GEMV updates
ski_status trsv_upper_t(const double* R, int64_t ldr, int64_t d, double* c, cudaStream_t st) {
  constexpr int TB = 64;
  for (int64_t k0 = 0; k0 < d; k0 += TB) {
    const int nb = (int)std::min<int64_t>(TB, d - k0);
    k_trsv_t_diag<<<1, 256, 0, st>>>(R + k0 * ldr + k0, ldr, nb, c + k0);
    SKI_LAUNCH_CHECK();
    const int64_t rest = d - k0 - nb;
    if (rest > 0) {  // c[k0+nb:] -= R[k0:k0+nb, k0+nb:]^T y
      k_gemv_t_sub<<<(unsigned)ski_cdiv(rest, 32), 256, 0, st>>>(R + k0 * ldr + k0 + nb, ldr, nb, rest, c + k0,
                                                                 c + k0 + nb);
      SKI_LAUNCH_CHECK();
    }
  }
  return SKI_OK;
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
  ar.take<double>(CB);          // Cholesky: 1 / r_jj of a block
  ar.take<double>(d + 1);       // Cholesky: diagonal of G, ratio
  if (chol2_applies(d)) ar.take<char>(chol2_bytes(d));
  return ar.off;
}

ski_status ski_gram_chol_run(const ski_matrix* A, uint64_t seed, int32_t s, int32_t replace, int64_t m,
                             const double* Sb, int64_t ldsb, double* R, int64_t ldr, double* qtsb, bool* ok,
                             double* eq_ratio, SkiArena& ar, cudaStream_t st) {
  *ok = false;
  *eq_ratio = INFINITY;
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
  double* dinv = ar.take<double>(CB);
  double* gdiag = ar.take<double>(d + 1);
  if (!ar.ok() || !gdiag) return SKI_ENOMEM;
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
  if (chol2_applies(d)) {
    const size_t cb = chol2_bytes(d);
    SkiArena car2{ar.take<char>(cb), cb, 0, false};
    if (!ar.ok()) return SKI_ENOMEM;
    SKI_TRY(chol_upper2(R, ldr, d, dinv, gdiag, gdiag + d, fail, car2, st));
  } else {
    SKI_TRY(chol_upper<double>(R, ldr, d, dinv, nullptr, gdiag, gdiag + d, fail, st));
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
    SKI_TRY(trsv_upper_t(R, ldr, d, cvec, st));
    SKI_CUDA_TRY(cudaMemcpyAsync(qtsb, cvec, d * sizeof(double), cudaMemcpyDeviceToDevice, st));
  }
  SKI_CUDA_TRY(cudaMemcpyAsync(&hfail, fail, sizeof(int), cudaMemcpyDeviceToHost, st));
  SKI_CUDA_TRY(cudaMemcpyAsync(eq_ratio, gdiag + d, sizeof(double), cudaMemcpyDeviceToHost, st));
  SKI_CUDA_TRY(cudaStreamSynchronize(st));
  *ok = hfail == 0;
  return SKI_OK;
}

// ---- dense sketch: R from the Cholesky factor of SA^T SA
// FP64: G = SA^T SA from exact FP16 slice products on the tensor cores
// (m < 2^16; above, on the FP64 SIMT GEMM), the tiles that meet the upper
// triangle, then the FP64 blocked Cholesky.  FP32 / TF32: SA^T (the
// GEMM's K-major operand) by a tile transpose, G on the tensor cores (three
// TF32 passes for FP32, one for TF32), the Cholesky in FP32, R cast to FP64.
// Work: m d^2 + d^3 / 3 multiply-adds against 2 m d^2 - 2 d^3 / 3 for the
// Householder QR.  Q^T Sb = R^{-T} SA^T Sb in FP64 (SA^T Sb accumulated in
// FP64 from the sketch's values).
size_t ski_gram_dense_ws_bytes(int64_t m, int64_t d, int32_t prec) {
  SkiArena ar{nullptr, 0, 0, true};
  ar.take<double>(d);                        // SA^T Sb
  ar.take<int>(1);                           // failure flag
  ar.take<double>(ski_cdiv(m, kSatRows) * d);  // SA^T Sb partial sums
  ar.take<double>(d + 1);                    // Cholesky: diagonal of G, ratio
  if (prec != SKI_F64) {
    const int64_t ldt = ski_round_up(m, 32), ldg = ski_round_up(d, 4);
    ar.take<float>(d * ldt);        // SA^T
    ar.take<float>(d * ldg);        // G, then R
    ar.take<float>(CB);             // Cholesky: 1 / r_jj of a block
    ar.take<float>(ldg * CB);       // Cholesky: block row transposed
  } else {
    ar.take<double>(CB);
    if (chol2_applies(d)) ar.take<char>(chol2_bytes(d));
    if (oz_beta(m) >= kOzMinBeta) {
      ar.take<int>(d);                                                    // column exponents
      ar.take<__half>((int64_t)oz_slices(oz_beta(m)) * d * oz_lds(m));  // slices
    }
  }
  return ar.off;
}

ski_status ski_gram_dense_run(const void* SA, int64_t ld_sa, int64_t m, int64_t d, int32_t prec, double* R,
                              int64_t ldr, double* qtsb, bool* ok, double* eq_ratio, SkiArena& ar, cudaStream_t st,
                              double* gemm_ms) {
  *ok = false;
  *eq_ratio = INFINITY;
  SpanTimer tm(gemm_ms != nullptr);
  if (d < 1 || m < d) return SKI_EINVAL;
  double* cvec = ar.take<double>(d);
  int* fail = ar.take<int>(1);
  double* part = ar.take<double>(ski_cdiv(m, kSatRows) * d);
  double* gdiag = ar.take<double>(d + 1);
  if (!ar.ok() || !gdiag) return SKI_ENOMEM;
  SKI_CUDA_TRY(cudaMemsetAsync(fail, 0, sizeof(int), st));
  if (prec == SKI_F64) {
    const double* A = (const double*)SA;
    // G = SA^T SA (upper tiles) into R, in place to its factor
    double* dinv = ar.take<double>(CB);
    const size_t c2b = chol2_applies(d) ? chol2_bytes(d) : 0;
    char* c2 = c2b ? ar.take<char>(c2b) : nullptr;
    if (!ar.ok() || !dinv) return SKI_ENOMEM;
    if (oz_beta(m) >= kOzMinBeta) {
      // G from exact FP16 slice products on the tensor cores
      int* e = ar.take<int>(d);
      __half* Sl = ar.take<__half>((int64_t)oz_slices(oz_beta(m)) * d * oz_lds(m));
      if (!ar.ok() || !Sl) return SKI_ENOMEM;
      SKI_TRY(oz_gram(A, ld_sa, m, d, R, ldr, e, Sl, fail, tm, st));
    } else {
      tm.mark(0, st);
      SKI_TRY(ski_gemm_ex<double>(d, d, m, 1.0, A, 1, ld_sa, A, ld_sa, 1, 0.0, R, ldr, 1, 0, st, 4));
      tm.mark(1, st);
    }
    if (chol2_applies(d)) {
      SkiArena car2{c2, c2b, 0, false};
      SKI_TRY(chol_upper2(R, ldr, d, dinv, gdiag, gdiag + d, fail, car2, st));
    } else {
      SKI_TRY(chol_upper<double>(R, ldr, d, dinv, nullptr, gdiag, gdiag + d, fail, st));
    }
    dim3 blk(32, 8), grid((unsigned)std::min<int64_t>(64, ski_cdiv(d, 32)), (unsigned)ski_cdiv(d, 8));
    k_zero_lower<<<grid, blk, 0, st>>>(d, R, ldr);
    SKI_LAUNCH_CHECK();
    // SA^T Sb (Sb = column d of the sketch)
    SKI_TRY(sat_sb_dense<double>(A, ld_sa, m, d, part, cvec, st));
  } else if (prec == SKI_F32 || prec == SKI_TF32) {
    const float* A = (const float*)SA;
    const int64_t ldt = ski_round_up(m, 32), ldg = ski_round_up(d, 4);
    float* At = ar.take<float>(d * ldt);
    float* G = ar.take<float>(d * ldg);
    float* dinv = ar.take<float>(CB);
    float* Pts = ar.take<float>(ldg * CB);
    if (!ar.ok() || !Pts) return SKI_ENOMEM;
    {
      dim3 grid((unsigned)ski_cdiv(m, 32), (unsigned)ski_cdiv(d, 32));
      k_transpose_f32<<<grid, dim3(32, 8), 0, st>>>(m, d, A, ld_sa, At, ldt);
      SKI_LAUNCH_CHECK();
    }
    // G = SA^T SA on the tensor cores (D = At At^T, stored; upper tiles only)
    tm.mark(0, st);
    SKI_TRY(ski_gemm_tf32(At, ldt, At, ldt, d, d, m, G, ldg, 0 | 4, 1, 0, fail, st, prec == SKI_F32));
    tm.mark(1, st);
    SKI_TRY(chol_upper<float>(G, ldg, d, dinv, Pts, gdiag, gdiag + d, fail, st));
    dim3 blk(32, 8), grid((unsigned)std::min<int64_t>(64, ski_cdiv(d, 32)), (unsigned)ski_cdiv(d, 8));
    k_upper_to_f64<<<grid, blk, 0, st>>>(d, G, ldg, R, ldr);
    SKI_LAUNCH_CHECK();
    SKI_TRY(sat_sb_dense<float>(A, ld_sa, m, d, part, cvec, st));
  } else {
    return SKI_EINVAL;
  }
  if (qtsb) {
    SKI_TRY(trsv_upper_t(R, ldr, d, cvec, st));
    SKI_CUDA_TRY(cudaMemcpyAsync(qtsb, cvec, d * sizeof(double), cudaMemcpyDeviceToDevice, st));
  }
  int hfail = 0;
  SKI_CUDA_TRY(cudaMemcpyAsync(&hfail, fail, sizeof(int), cudaMemcpyDeviceToHost, st));
  SKI_CUDA_TRY(cudaMemcpyAsync(eq_ratio, gdiag + d, sizeof(double), cudaMemcpyDeviceToHost, st));
  SKI_CUDA_TRY(cudaStreamSynchronize(st));
  if (gemm_ms) *gemm_ms = tm.ms();
  *ok = hfail == 0;
  return SKI_OK;
}
