// Internal interfaces between the sketch, premix, QR, LSQR translation units
// and the C-ABI layer.
#pragma once
#include <cuda.h>

#include "common.cuh"

struct SkiBuckets {
  const int64_t* offsets;  // [m+1]
  const uint32_t* list;    // entries (j << 1) | neg, ascending inside a bucket
  int64_t m;
};

// scale * (S * 2^(E - 1075 - FX_LIFT)) with scale = c * 2^(-62 - e), c in [2^61, 2^62).
__device__ __forceinline__ double fx_scaled(const FxAcc& a, long long c, int e) {
  if (a.bad) return __longlong_as_double(0x7FF8000000000000ll);
  long long Sp = (long long)(((__int128)a.S * (__int128)c) >> 62);
  return fx_to_double(Sp, a.E, e);
}

// ---- sketch.cu
size_t ski_bucket_ws_bytes(int64_t nrows, int32_t s, int64_t m);
// row0: the global index of the first of the nrows rows (a row block of a
// larger A draws its rows' columns of S)
ski_status ski_build_buckets(uint64_t seed, int32_t s, int32_t replace, int64_t m, int64_t nrows, SkiArena& ar,
                             cudaStream_t st, SkiBuckets* out, int64_t row0 = 0);
ski_status ski_gather_dense(const double* A, int64_t lda, int64_t nrows, int64_t d, const double* b,
                            const SkiBuckets& bk, double scale, int32_t out_dtype, void* SA, int64_t ld_sa,
                            cudaStream_t st);
ski_status ski_gather_dense_f32in(const float* Y, int64_t ldy, int64_t ncols, const SkiBuckets& bk,
                                  double scale, int32_t out_dtype, void* SA, int64_t ld_sa, cudaStream_t st);
// Gather of a column slab (ncols <= 128) of the premix output Y (FP64 or
// FP32 per y_dtype) into the same columns of SA: one warp per bucket.
ski_status ski_gather_slab(const void* Y, int32_t y_dtype, int64_t ldy, int64_t ncols, const SkiBuckets& bk,
                           double scale, int32_t out_dtype, void* SA, int64_t ld_sa, cudaStream_t st);
ski_status ski_gather_csr(const ski_matrix* A, const double* b, const SkiBuckets& bk, double scale,
                          int32_t out_dtype, void* SA, int64_t ld_sa, cudaStream_t st);

// ---- wht.cu
// Y = 2^(-floor(L/2)) * Hu D [A b; 0] with Hu the unnormalised Walsh-Hadamard
// matrix of order n_pad = 2^L; the remaining factor (1 or 2^-1/2) is
// returned in *residual_scale for the caller to fold into the sketch scale.
size_t ski_premix_ws_bytes(int64_t n, int64_t ncols, int64_t n_pad, int32_t dtype);
// Buffers and pass plan of a premix over at most ncols_max columns at a time
// (D drawn once); ski_premix_cols then transforms any column range of A (A and
// Y offset by the caller), so a wide A can be premixed slab by slab through
// the same L2-sized buffers.
struct SkiPremixPlan {
  int64_t n, n_pad, ldq;
  int32_t dtype;
  int L, P, yshift;
  int nbs[8];
  double residual_scale;
  int8_t* D;
  int* nonfinite;  // [ldq + 1]: per column, set when the column holds a NaN or Inf; then any column
  int* err;  // set when a bounded wait of the TMA-fed pass gave up
  void *Qa, *Qb;
  int16_t *Xa, *Xb;
  int* ecol;
};
// err_flag: a device int the caller zeroes and reads (nullptr: one in the
// plan's scratch).
ski_status ski_premix_plan(int64_t n, int64_t ncols_max, int64_t n_pad, int32_t dtype, uint64_t seed, SkiArena& ar,
                           cudaStream_t st, SkiPremixPlan* plan, int* err_flag = nullptr);
ski_status ski_premix_cols(const SkiPremixPlan& plan, const double* A, int64_t lda, int64_t d, const double* b,
                           void* Y, int64_t ldy, cudaStream_t st);
// The FP64 premix output left in block-fixed-point form (one pass): row j,
// column c is Q[j * ldq + c] * 2^(X[tile(j) * ldx + c] - yshift), with tile(j)
// the tile of row j in the last pass (row bits [lo, lo + nb)).  Saves the
// last pass its FP64 conversion and the hash gather its FP64 decode.
// With two or more passes the last one aligns each column to a common
// exponent instead (X == nullptr): row j, column c is Q[j * ldq + c] *
// 2^(ecol[c] + headroom - yshift).
struct SkiPremixQ {
  const long long* Q;
  const int* nonfinite;  // per column: the column's sketch is NaN
  const int* err;        // set: a bounded wait of the premix gave up, the whole sketch is NaN
  const int16_t* X;
  const int* ecol;
  int headroom;
  int64_t ldq, ldx;
  int lo, nb, yshift;
};
ski_status ski_premix_cols_q(const SkiPremixPlan& plan, const double* A, int64_t lda, int64_t d, const double* b,
                             SkiPremixQ* out, cudaStream_t st);
ski_status ski_gather_q(const SkiPremixQ& y, int64_t ncols, const SkiBuckets& bk, double scale, double* SA,
                        int64_t ld_sa, cudaStream_t st);
ski_status ski_premix_run(const double* A, int64_t lda, int64_t n, int64_t d, const double* b, uint64_t seed,
                          int64_t n_pad, int32_t dtype, void* Y, int64_t ldy, SkiArena& ar, cudaStream_t st,
                          double* residual_scale);

// ---- qr.cu
size_t ski_qr_ws_bytes(int64_t m, int64_t ncols, int32_t dtype);
ski_status ski_qr_run(int64_t m, int64_t d, int32_t with_rhs, void* SA, int64_t ld_sa, int32_t dtype,
                      double* R, int64_t ldr, double* qtsb, SkiArena& ar, cudaStream_t st,
                      double* gemm_ms = nullptr);

ski_status ski_barrier_selftest(long long spin_limit, void* ws, cudaStream_t st);

// ---- gemm_tc.cu: D = A B^T on the TF32 tensor cores (see there for modes)
bool ski_tmap_f64_2d(CUtensorMap* map, const double* base, int64_t rows, int64_t cols, int64_t ld, int box_rows,
                     int box_cols);
ski_status ski_gemm_tf32(const float* A, int64_t lda, const float* B, int64_t ldb, int64_t M, int64_t N, int64_t K,
                         float* C, int64_t ldc, int mode, int splits, int64_t c_zstride, int* err, cudaStream_t st,
                         bool split3);

// C64 += scale * sum over pairs of S[a] S[b]^T on the tensor cores from a
// stack S of FP16 matrices (gemm_tc.cu): one FP32 accumulator for the pairs,
// exact for integer operands with partial sums below 2^24
constexpr int kTcMaxPairs = 16;
struct TcPairs {
  int n;
  int8_t a[kTcMaxPairs], b[kTcMaxPairs];
};
ski_status ski_gemm_f16_pairs_f64acc(const void* S, int64_t lds, int64_t sstride, int ns, int64_t rows, int64_t K,
                                     const TcPairs& pr, double* C64, int64_t ldc, double scale, bool upper, int* err,
                                     cudaStream_t st);

// ---- trinv.cu
size_t ski_trinv_ws_bytes(int64_t d, int32_t dtype);
ski_status ski_trinv_run(int64_t d, const double* R, int64_t ldr, double* M, double* Mt, int64_t ldm,
                         int32_t dtype, double perturb, SkiArena& ar, cudaStream_t st);

// ---- gemm.cu : C = beta*C + alpha * op(A) op(B), row-major element strides.
template <class T>
ski_status ski_gemm(int64_t M, int64_t N, int64_t K, T alpha, const T* A, int64_t sa_m, int64_t sa_k,
                    const T* B, int64_t sb_k, int64_t sb_n, T beta, T* C, int64_t ldc, cudaStream_t st);
template <class T>
ski_status ski_gemm_ex(int64_t M, int64_t N, int64_t K, T alpha, const T* A, int64_t sa_m, int64_t sa_k,
                       const T* B, int64_t sb_k, int64_t sb_n, T beta, T* C, int64_t ldc, int splits,
                       int64_t c_zstride, cudaStream_t st, int tri = 0);
template <class T>
ski_status ski_gemm_batched(int64_t M, int64_t N, int64_t K, T alpha, const T* A, int64_t sa_m, int64_t sa_k,
                            int64_t a_zs, const T* B, int64_t sb_k, int64_t sb_n, int64_t b_zs, T beta, T* C,
                            int64_t ldc, int64_t c_zs, int64_t batch, int tri, cudaStream_t st);
template <class T>
ski_status ski_gemm_tri(int64_t M, int64_t N, int64_t K, T alpha, const T* A, int64_t sa_m, int64_t sa_k,
                        const T* B, int64_t sb_k, int64_t sb_n, T beta, T* C, int64_t ldc, int tri, cudaStream_t st);

// Column-pivoted QR of [R | c] (cpqr.cu): R11 (p x p, row-major, ld11), c1
// (the first p entries of the reflected c), piv (the column of R at each
// pivoted position) and p under the rank rule; synchronises the stream.
size_t ski_cpqr_ws_bytes(int64_t d);
ski_status ski_cpqr_run(int64_t d, const double* R, int64_t ldr, const double* c, double rcond, double* R11,
                        int64_t ld11, double* c1, int32_t* piv, int32_t* p_out, SkiArena& ar, cudaStream_t st);
// dst[k] = src[idx[k]] for k < p
ski_status ski_gather_launch(int64_t p, const int32_t* idx, const double* src, double* dst, cudaStream_t st);
// dst = 0 (length d), then dst[idx[k]] = src[k] for k < p
ski_status ski_scatter_launch(int64_t d, int64_t p, const int32_t* idx, const double* src, double* dst,
                              cudaStream_t st);

// dht.cu: the DHT premix F D of Eq. HR-DHT (length N, prime factors <= 13)
// into Y (N x ldY, FP64 or FP32), and the sampling sketch S_s of Eq. SR-DHT
bool ski_dht_length_ok(int64_t N);
int64_t ski_dht_length(int64_t n);
size_t ski_dht_ws_bytes(int64_t n, int64_t ncols, int64_t N, int32_t dtype);
ski_status ski_dht_premix(const double* A, int64_t lda, int64_t n, int64_t d, const double* b, uint64_t seed,
                          int64_t N, int32_t dtype, void* Y, int64_t ldY, SkiArena& ar, cudaStream_t st);
// SA[i, :] = X[c_i, :] (and b[c_i] in column dx when b is given), i < m
ski_status ski_sample_rows(uint64_t seed, int64_t m, int64_t nrows, const void* X, int32_t x_dtype, int64_t ldx,
                           int64_t dx, const double* b, int32_t out_dtype, void* SA, int64_t ld_sa, cudaStream_t st);

// gram.cu: Step 2 of Ski-LLS-sparse from a sparse sketch -- SA in CSR, its Gram
// matrix SA^T SA, R = its Cholesky factor (d x d, upper, ldr; lower triangle
// zeroed) and qtsb = R^{-T} SA^T Sb (Sb: column of the dense sketch, stride
// ldsb).  *ok = false (R and qtsb unusable) when a sketch row is too long for
// the shared-memory merge or a Cholesky pivot is not positive; *eq_ratio =
// max_j sqrt(g_jj) / r_jj (infinite when not computed); synchronises st.
size_t ski_gram_ws_bytes(int64_t n, int64_t d, int64_t nnz, int32_t s, int64_t m);
ski_status ski_gram_chol_run(const ski_matrix* A, uint64_t seed, int32_t s, int32_t replace, int64_t m,
                             const double* Sb, int64_t ldsb, double* R, int64_t ldr, double* qtsb, bool* ok,
                             double* eq_ratio, SkiArena& ar, cudaStream_t st);
// R from the Cholesky factor of SA^T SA of a dense sketch (SA: m x (d + 1)
// row-major, FP64 for prec SKI_F64, else FP32; column d holds Sb); *ok as above
size_t ski_gram_dense_ws_bytes(int64_t m, int64_t d, int32_t prec);
// gemm_ms (optional): CUDA-event time of the Gram matrix product
ski_status ski_gram_dense_run(const void* SA, int64_t ld_sa, int64_t m, int64_t d, int32_t prec, double* R,
                              int64_t ldr, double* qtsb, bool* ok, double* eq_ratio, SkiArena& ar, cudaStream_t st,
                              double* gemm_ms = nullptr);
