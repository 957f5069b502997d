// SIMT GEMM used by the blocked Householder QR (trailing update, Algorithm 1
// Step 2) and by the triangular inverse: C = beta C + alpha op(A) op(B) with
// arbitrary element strides, so that transposed operands need no copy.
//
// FP64: GB300 issues 2 DFMA per clock per SM, so the kernel is bound by the
// FP64 pipe whatever the tiling; a 64x64 (or 32x64) tile with a 4x4 (2x4)
// register micro-tile keeps shared-memory traffic far below that bound.
// FP32: the same tiling; the TF32/BF16 tensor-core path lives in gemm_tc.cu.
#include "common.cuh"
#include "sketch_impl.cuh"

namespace {

template <class T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN)) k_gemm(
    int64_t M, int64_t N, int64_t K, int64_t kchunk, T alpha, const T* __restrict__ A, int64_t sa_m,
    int64_t sa_k, const T* __restrict__ B, int64_t sb_k, int64_t sb_n, T beta, T* __restrict__ C, int64_t ldc,
    int64_t c_zstride, int tri, int64_t a_zstride, int64_t b_zstride) {
  constexpr int NT = (BM / TM) * (BN / TN);
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % (BN / TN), ty = tid / (BN / TN);
  const int64_t m0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;
  // z: a K split (a_zstride = b_zstride = 0) or a batch of independent
  // products whose operands sit a_zstride / b_zstride elements apart
  const bool batch = a_zstride != 0 || b_zstride != 0;
  int64_t kbeg = batch ? 0 : (int64_t)blockIdx.z * kchunk;
  int64_t kend = batch ? K : min(K, kbeg + kchunk);
  A += (int64_t)blockIdx.z * a_zstride;
  B += (int64_t)blockIdx.z * b_zstride;
  // tri bit 0: A upper triangular (A[i,k] = 0 for k < i); bit 1: B upper
  // triangular (B[k,j] = 0 for k > j).  Skip the k-range that is all zero.
  if (tri & 1) kbeg = max(kbeg, m0 - (m0 % BK));
  if (tri & 2) kend = min(kend, n0 + BN);
  // tri bit 2: only C's upper triangle is wanted -- a tile wholly below the
  // diagonal (every row index above every column index) is skipped
  if ((tri & 4) && m0 >= n0 + BN) return;
  C += (int64_t)blockIdx.z * c_zstride;
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
  const bool a_m_fast = (sa_m == 1);
  const bool b_n_fast = (sb_n == 1);
  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
    // A tile BM x BK
    for (int e = tid; e < BM * BK; e += NT) {
      int mm, kk;
      if (a_m_fast) { mm = e % BM; kk = e / BM; } else { kk = e % BK; mm = e / BK; }
      int64_t gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < M && gk < kend) ? A[gm * sa_m + gk * sa_k] : T(0);
    }
    for (int e = tid; e < BN * BK; e += NT) {
      int nn, kk;
      if (b_n_fast) { nn = e % BN; kk = e / BN; } else { kk = e % BK; nn = e / BK; }
      int64_t gn = n0 + nn, gk = k0 + kk;
      Bs[kk][nn] = (gn < N && gk < kend) ? B[gk * sb_k + gn * sb_n] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + i * (BM / TM)];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + j * (BN / TN)];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    int64_t gm = m0 + ty + i * (BM / TM);
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int64_t gn = n0 + tx + j * (BN / TN);
      if (gn >= N) continue;
      T* cp = &C[gm * ldc + gn];
      *cp = (beta == T(0)) ? alpha * acc[i][j] : fma(alpha, acc[i][j], beta * *cp);
    }
  }
}

}  // namespace

// Plain GEMM (no split) or split-K into `splits` partial outputs at
// C + z * c_zstride (beta applies to each partial; callers pass beta = 0).
template <class T>
ski_status ski_gemm_ex(int64_t M, int64_t N, int64_t K, T alpha, const T* A, int64_t sa_m, int64_t sa_k,
                       const T* B, int64_t sb_k, int64_t sb_n, T beta, T* C, int64_t ldc, int splits,
                       int64_t c_zstride, cudaStream_t st, int tri) {
  if (M <= 0 || N <= 0) return SKI_OK;
  constexpr int BK = sizeof(T) == 8 ? 16 : 16;
  int64_t kchunk = ski_round_up(ski_cdiv(K > 0 ? K : 1, splits), BK);
  if (M <= 32) {
    dim3 grid((unsigned)ski_cdiv(N, 64), (unsigned)ski_cdiv(M, 32), (unsigned)splits);
    k_gemm<T, 32, 64, BK, 2, 4><<<grid, 256, 0, st>>>(M, N, K, kchunk, alpha, A, sa_m, sa_k, B, sb_k, sb_n, beta,
                                                      C, ldc, c_zstride, tri, 0, 0);
  } else {
    dim3 grid((unsigned)ski_cdiv(N, 64), (unsigned)ski_cdiv(M, 64), (unsigned)splits);
    k_gemm<T, 64, 64, BK, 4, 4><<<grid, 256, 0, st>>>(M, N, K, kchunk, alpha, A, sa_m, sa_k, B, sb_k, sb_n, beta,
                                                      C, ldc, c_zstride, tri, 0, 0);
  }
  SKI_LAUNCH_CHECK();
  return SKI_OK;
}

// `batch` independent products C_z = beta C_z + alpha op(A_z) op(B_z) with the
// operands of product z at A + z a_zs, B + z b_zs, C + z c_zs (one launch).
template <class T>
ski_status ski_gemm_batched(int64_t M, int64_t N, int64_t K, T alpha, const T* A, int64_t sa_m, int64_t sa_k,
                            int64_t a_zs, const T* B, int64_t sb_k, int64_t sb_n, int64_t b_zs, T beta, T* C,
                            int64_t ldc, int64_t c_zs, int64_t batch, int tri, cudaStream_t st) {
  if (M <= 0 || N <= 0 || batch <= 0) return SKI_OK;
  if (batch > 65535 || (a_zs == 0 && b_zs == 0 && batch > 1)) return SKI_EINVAL;
  constexpr int BK = 16;
  const int64_t kchunk = ski_round_up(K > 0 ? K : 1, BK);
  if (M <= 32) {
    dim3 grid((unsigned)ski_cdiv(N, 64), (unsigned)ski_cdiv(M, 32), (unsigned)batch);
    k_gemm<T, 32, 64, BK, 2, 4><<<grid, 256, 0, st>>>(M, N, K, kchunk, alpha, A, sa_m, sa_k, B, sb_k, sb_n, beta,
                                                      C, ldc, c_zs, tri, a_zs, b_zs);
  } else {
    dim3 grid((unsigned)ski_cdiv(N, 64), (unsigned)ski_cdiv(M, 64), (unsigned)batch);
    k_gemm<T, 64, 64, BK, 4, 4><<<grid, 256, 0, st>>>(M, N, K, kchunk, alpha, A, sa_m, sa_k, B, sb_k, sb_n, beta,
                                                      C, ldc, c_zs, tri, a_zs, b_zs);
  }
  SKI_LAUNCH_CHECK();
  return SKI_OK;
}
template ski_status ski_gemm_batched<double>(int64_t, int64_t, int64_t, double, const double*, int64_t, int64_t,
                                             int64_t, const double*, int64_t, int64_t, int64_t, double, double*,
                                             int64_t, int64_t, int64_t, int, cudaStream_t);
template ski_status ski_gemm_batched<float>(int64_t, int64_t, int64_t, float, const float*, int64_t, int64_t, int64_t,
                                            const float*, int64_t, int64_t, int64_t, float, float*, int64_t, int64_t,
                                            int64_t, int, cudaStream_t);

template <class T>
ski_status ski_gemm(int64_t M, int64_t N, int64_t K, T alpha, const T* A, int64_t sa_m, int64_t sa_k,
                    const T* B, int64_t sb_k, int64_t sb_n, T beta, T* C, int64_t ldc, cudaStream_t st) {
  return ski_gemm_ex<T>(M, N, K, alpha, A, sa_m, sa_k, B, sb_k, sb_n, beta, C, ldc, 1, 0, st, 0);
}

template <class T>
ski_status ski_gemm_tri(int64_t M, int64_t N, int64_t K, T alpha, const T* A, int64_t sa_m, int64_t sa_k,
                        const T* B, int64_t sb_k, int64_t sb_n, T beta, T* C, int64_t ldc, int tri, cudaStream_t st) {
  return ski_gemm_ex<T>(M, N, K, alpha, A, sa_m, sa_k, B, sb_k, sb_n, beta, C, ldc, 1, 0, st, tri);
}

template ski_status ski_gemm<double>(int64_t, int64_t, int64_t, double, const double*, int64_t, int64_t,
                                     const double*, int64_t, int64_t, double, double*, int64_t, cudaStream_t);
template ski_status ski_gemm<float>(int64_t, int64_t, int64_t, float, const float*, int64_t, int64_t,
                                    const float*, int64_t, int64_t, float, float*, int64_t, cudaStream_t);
template ski_status ski_gemm_ex<double>(int64_t, int64_t, int64_t, double, const double*, int64_t, int64_t,
                                        const double*, int64_t, int64_t, double, double*, int64_t, int, int64_t,
                                        cudaStream_t, int);
template ski_status ski_gemm_ex<float>(int64_t, int64_t, int64_t, float, const float*, int64_t, int64_t,
                                       const float*, int64_t, int64_t, float, float*, int64_t, int, int64_t,
                                       cudaStream_t, int);
template ski_status ski_gemm_tri<double>(int64_t, int64_t, int64_t, double, const double*, int64_t, int64_t,
                                         const double*, int64_t, int64_t, double, double*, int64_t, int, cudaStream_t);
template ski_status ski_gemm_tri<float>(int64_t, int64_t, int64_t, float, const float*, int64_t, int64_t,
                                        const float*, int64_t, int64_t, float, float*, int64_t, int, cudaStream_t);
