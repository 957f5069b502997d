// R^{-1} for the upper-triangular factor of Step 2, formed once so that the
// two preconditioner applications per LSQR iteration (R^{-1} v, R^{-T} u) are
// bandwidth-bound triangular matrix-vector products instead of
// latency-bound back-substitutions.  2x2 blocking,
//   [R11 R12; 0 R22]^{-1} = [X11, -X11 R12 X22; 0, X22],  X11 = R11^{-1}, X22 = R22^{-1},
// with all 32 x 32 diagonal blocks inverted by back-substitution in one launch
// and the off-diagonal blocks formed level by level by batched GEMMs (gemm.cu).  With perturb > 0
// each diagonal entry r_ii is replaced by r_ii + perturb (the perturbed
// back-solve of Ski-LLS-sparse).  The FP32 inverse works on R * 2^-e, with
// 2^e the power of two of max |r_ij| (exact scaling), so that any FP64 R is in
// FP32 range; M = (R 2^-e)^{-1} 2^-e.
#include "common.cuh"
#include "sketch_impl.cuh"

namespace {

constexpr int LB = 32;

// Invert the LB x LB diagonal blocks of R (in X, same layout): one warp per
// block, lane = column of the inverse.
template <class T>
__global__ void k_diag_inv(int64_t d, const T* __restrict__ R, int64_t ldr, T* __restrict__ X, int64_t ldx,
                           double perturb) {
  const int64_t blk = blockIdx.x;
  const int lane = threadIdx.x;
  const int64_t o = blk * LB;
  const int nbk = (int)std::min<int64_t>(LB, d - o);
  __shared__ T Rs[LB][LB + 1];
  for (int i = 0; i < nbk; ++i) Rs[i][lane] = lane < nbk ? R[(o + i) * ldr + o + lane] : T(0);
  __syncwarp();
  // column `lane` of the inverse: solve R x = e_lane by back-substitution
  T x[LB];
#pragma unroll
  for (int i = 0; i < LB; ++i) x[i] = T(0);
  if (lane < nbk) {
#pragma unroll
    for (int i = LB - 1; i >= 0; --i) {
      if (i >= nbk || i > lane) continue;
      T acc = (i == lane) ? T(1) : T(0);
#pragma unroll
      for (int k = i + 1; k < LB; ++k)
        if (k <= lane && k < nbk) acc -= Rs[i][k] * x[k];
      x[i] = acc / (Rs[i][i] + (T)perturb);
    }
  }
  for (int i = 0; i < nbk; ++i)
    if (lane < nbk) X[(o + i) * ldx + o + lane] = x[i];
}

// Largest biased exponent field over the upper triangle of R (atomicMax into
// *emax, which starts at 0).
__global__ void k_upper_max_exp(int64_t d, const double* __restrict__ R, int64_t ldr, int* __restrict__ emax) {
  int e = 0;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < d * d;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / d, c = idx % d;
    if (c >= i) e = max(e, (int)((__double_as_longlong(R[i * ldr + c]) >> 52) & 0x7FF));
  }
  e = __reduce_max_sync(0xffffffffu, e);
  if ((threadIdx.x & 31) == 0 && e > 0) atomicMax(emax, e);
}
// Scale shift of R for the FP32 inverse: max |r_ij| * 2^-sh lies in [1, 2).
// No shift when R is all zero or holds a NaN / Inf (then the inverse is
// non-finite in either precision).
__device__ __forceinline__ int trinv_shift(const int* emax) {
  if (!emax) return 0;
  const int e = *emax;
  return (e == 0 || e == 0x7FF) ? 0 : e - 1023;
}
template <class T>
__global__ void k_cast_upper(int64_t d, const double* __restrict__ R, int64_t ldr, T* __restrict__ Rt, int64_t ldt,
                             const int* __restrict__ emax) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= d * d) return;
  int64_t i = idx / d, c = idx % d;
  const int sh = trinv_shift(emax);
  Rt[i * ldt + c] = c >= i ? (T)ldexp(R[i * ldr + c], -sh) : T(0);
}

template <class T>
__global__ void k_emit(int64_t d, const T* __restrict__ X, int64_t ldx, double* __restrict__ M,
                       double* __restrict__ Mt, int64_t ldm, const int* __restrict__ emax) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= d * d) return;
  int64_t i = idx / d, c = idx % d;
  const int sh = trinv_shift(emax);
  double v = c >= i ? ldexp((double)X[i * ldx + c], -sh) : 0.0;
  M[i * ldm + c] = v;
  if (Mt) Mt[c * ldm + i] = v;
}

// Off-diagonal blocks, bottom-up by doubling: after the level of block size
// b every aligned block [k 2b, (k+1) 2b) (and the tail) holds its inverse,
// formed from its two halves as X12 = -X11 (R12 X22).  All full-size nodes of
// a level are independent and go to one batched GEMM pair; a ragged tail node
// (right half shorter than b) takes one more pair.  Eight launches per
// doubling instead of two per node of a recursion tree.
template <class T>
ski_status levels(int64_t d, const T* R, int64_t ldr, T* X, int64_t ldx, T* tmp, cudaStream_t st) {
  for (int64_t b = LB; b < d; b *= 2) {
    const int64_t nfull = d / (2 * b);
    if (nfull > 0) {
      // node i: left block at o = 2 b i, right block at o + b, both of size b
      const int64_t zr = 2 * b * (ldr + 1), zx = 2 * b * (ldx + 1);
      SKI_TRY(ski_gemm_batched<T>(b, b, b, T(1), R + b, ldr, 1, zr, X + b * ldx + b, ldx, 1, zx, T(0), tmp, b, b * b,
                                  nfull, 2, st));
      SKI_TRY(ski_gemm_batched<T>(b, b, b, T(-1), X, ldx, 1, zx, tmp, b, 1, b * b, T(0), X + b, ldx, zx, nfull, 1,
                                  st));
    }
    const int64_t o = 2 * b * nfull;
    const int64_t n2 = d - o - b;
    if (n2 > 0) {
      const T* R12 = R + o * ldr + o + b;
      const T* X22 = X + (o + b) * ldx + o + b;
      const T* X11 = X + o * ldx + o;
      T* X12 = X + o * ldx + o + b;
      SKI_TRY(ski_gemm_tri<T>(b, n2, n2, T(1), R12, ldr, 1, X22, ldx, 1, T(0), tmp, n2, 2, st));
      SKI_TRY(ski_gemm_tri<T>(b, n2, b, T(-1), X11, ldx, 1, tmp, n2, 1, T(0), X12, ldx, 1, st));
    }
  }
  return SKI_OK;
}

template <class T>
ski_status trinv_impl(int64_t d, const double* R, int64_t ldr, double* M, double* Mt, int64_t ldm, double perturb,
                      SkiArena& ar, cudaStream_t st) {
  T* Rt = ar.take<T>(d * d);
  T* X = ar.take<T>(d * d);
  T* tmp = ar.take<T>(ski_cdiv(d, 2) * d + LB * d);
  int* emax = ar.take<int>(1);
  if (!ar.ok() || !emax) return SKI_ENOMEM;
  if (sizeof(T) == 8) emax = nullptr;  // the FP64 inverse needs no scaling
  SKI_CUDA_TRY(cudaMemsetAsync(X, 0, d * d * sizeof(T), st));
  if (emax) {
    SKI_CUDA_TRY(cudaMemsetAsync(emax, 0, sizeof(int), st));
    k_upper_max_exp<<<(unsigned)std::min<int64_t>(4 * 152, ski_cdiv(d * d, 256)), 256, 0, st>>>(d, R, ldr, emax);
    SKI_LAUNCH_CHECK();
  }
  k_cast_upper<T><<<ski_cdiv(d * d, 256), 256, 0, st>>>(d, R, ldr, Rt, d, emax);
  SKI_LAUNCH_CHECK();
  k_diag_inv<T><<<ski_cdiv(d, LB), 32, 0, st>>>(d, Rt, d, X, d, perturb);
  SKI_LAUNCH_CHECK();
  SKI_TRY(levels<T>(d, Rt, d, X, d, tmp, st));
  k_emit<T><<<ski_cdiv(d * d, 256), 256, 0, st>>>(d, X, d, M, Mt, ldm, emax);
  SKI_LAUNCH_CHECK();
  return SKI_OK;
}

}  // namespace

size_t ski_trinv_ws_bytes(int64_t d, int32_t dtype) {
  size_t es = dtype == SKI_F64 ? 8 : 4;
  SkiArena ar{nullptr, 0, 0, true};
  ar.take<char>(es * d * d);
  ar.take<char>(es * d * d);
  ar.take<char>(es * (ski_cdiv(d, 2) * d + LB * d));
  ar.take<int>(1);
  return ar.off;
}

ski_status ski_trinv_run(int64_t d, const double* R, int64_t ldr, double* M, double* Mt, int64_t ldm, int32_t dtype,
                         double perturb, SkiArena& ar, cudaStream_t st) {
  if (dtype == SKI_F64) return trinv_impl<double>(d, R, ldr, M, Mt, ldm, perturb, ar, st);
  if (dtype == SKI_F32) return trinv_impl<float>(d, R, ldr, M, Mt, ldm, perturb, ar, st);
  return SKI_EINVAL;
}
