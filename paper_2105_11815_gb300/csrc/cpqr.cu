// Step 2 of Algorithm 1 with a rank-revealing factorization: the column-
// pivoted Householder QR (Businger & Golub) named by Remark (i), for a sketch
// whose plain QR fails the rank rule.
//
// SA = Q R has already been factored without pivoting.  Pivoting R itself,
// R P = Q' R', gives SA P = (Q Q') R': the pivots and the leading rows of R'
// are those of the column-pivoted QR of SA, because the orthonormal Q keeps
// every partial column norm.  So only the d x d triangle is pivoted, not the
// m x d sketch.  The reflectors are applied to Q^T Sb as well, so that the
// first p entries of the result are Q1^T Sb for Step 3.
//
// Step j takes the column of largest Euclidean norm over rows j.. among those
// not yet pivoted (the smallest column index on ties), reflects it onto
// beta e_j with beta = -sign(x_0) ||x||, and applies the reflector to every
// other column.  The norms are recomputed from the updated columns at every
// step, not downdated.  The factorization stops at the first step whose
// |beta| is below rcond |beta_0|: since |beta| does not increase along the
// pivoted diagonal, p = that step is the numerical rank under the rank rule
// |r_qq| >= rcond |r_11|.
//
// One cooperative launch, one CTA per SM, one grid barrier per step.  Column
// c belongs to CTA c mod nCTA, which alone writes it; every CTA reads the
// pivot column through L2 and forms the same reflector redundantly (same
// data, same reduction order), so all CTAs agree on every pivot and on the
// stopping step.  Each barrier wait is bounded: after the spin limit the
// error flag is set and the kernel returns (SKI_ETIMEOUT on the host).
#include "common.cuh"
#include "lsqr_impl.cuh"
#include "sketch_impl.cuh"

namespace {

constexpr int CP_THREADS = 256;
constexpr int CP_WARPS = CP_THREADS / 32;

struct CpqrArgs {
  int64_t d, ldb;
  double* B;        // column-major [R | c]: column c at B + c * ldb, rows 0..d-1
  double* beta;     // [d] diagonal of the pivoted factor
  int32_t* piv;     // [d] column of R at pivoted position j
  int8_t* done;     // [d] column already pivoted (read and written by its owner only)
  double* slot_v;   // [2 nCTA] each CTA's largest squared norm, by step parity
  int32_t* slot_i;  // [2 nCTA] its column
  int32_t* steps;   // out: p
  double rcond;
  GridBar* gb;
  long long spin_limit;
};

// (v, i) <- the larger norm, the smaller column on ties; i < 0 is empty
__device__ __forceinline__ void cp_better(double& v, int& i, double v2, int i2) {
  if (i2 < 0) return;
  if (i < 0 || v2 > v || (v2 == v && i2 < i)) {
    v = v2;
    i = i2;
  }
}

// Block-wide arg-max; every thread returns the same pair.
__device__ __forceinline__ void cp_block_argmax(double& v, int& i, double* sv, int* si) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
    const int i2 = __shfl_xor_sync(0xffffffffu, i, o);
    cp_better(v, i, v2, i2);
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    sv[threadIdx.x >> 5] = v;
    si[threadIdx.x >> 5] = i;
  }
  __syncthreads();
  v = sv[0];
  i = si[0];
  for (int w = 1; w < CP_WARPS; ++w) cp_better(v, i, sv[w], si[w]);
}

// Block-wide sum in a fixed order; every thread returns the same value.
__device__ __forceinline__ double cp_block_sum(double x, double* sbuf) {
  x = ski_warp_sum(x);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sbuf[threadIdx.x >> 5] = x;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < CP_WARPS; ++w) s += sbuf[w];
  return s;
}

__global__ void __launch_bounds__(CP_THREADS) k_cpqr(CpqrArgs a) {
  extern __shared__ __align__(16) double s_v[];  // the reflector, rows j..d-1
  __shared__ double s_red[CP_WARPS];
  __shared__ double s_av[CP_WARPS];
  __shared__ int s_ai[CP_WARPS];
  const int nb = gridDim.x, bid = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t d = a.d, ldb = a.ldb;
  unsigned my_gen = 0;
  // squared norms of this CTA's columns, whole height
  double bv = -1.0;
  int bi = -1;
  for (int64_t c = bid + (int64_t)warp * nb; c < d; c += (int64_t)CP_WARPS * nb) {
    const double* col = a.B + c * ldb;
    double s = 0.0;
    for (int64_t i = lane; i < d; i += 32) {
      const double x = col[i];
      s += x * x;
    }
    s = ski_warp_sum(s);
    if (lane == 0) a.done[c] = 0;
    cp_better(bv, bi, s, (int)c);
  }
  cp_block_argmax(bv, bi, s_av, s_ai);
  if (threadIdx.x == 0) {
    a.slot_v[bid] = bv;
    a.slot_i[bid] = bi;
  }
  if (!grid_sync(a.gb, nb, my_gen, a.spin_limit)) return;
  double r11 = 0.0;
  int64_t j = 0;
  for (; j < d; ++j) {
    const int par = (int)(j & 1);
    double pv = -1.0;
    int pk = -1;
    for (int t = threadIdx.x; t < nb; t += CP_THREADS)
      cp_better(pv, pk, __ldcg(a.slot_v + par * nb + t), __ldcg(a.slot_i + par * nb + t));
    cp_block_argmax(pv, pk, s_av, s_ai);
    if (pk < 0 || !(pv > 0.0)) break;  // every remaining column is zero
    const double* colk = a.B + (int64_t)pk * ldb + j;
    const int64_t len = d - j;
    double ss = 0.0;
    for (int64_t i = threadIdx.x; i < len; i += CP_THREADS) {
      const double x = __ldcg(colk + i);
      s_v[i] = x;
      ss += x * x;
    }
    const double normx = sqrt(cp_block_sum(ss, s_red));
    const double x0 = s_v[0];
    const double beta = x0 >= 0.0 ? -normx : normx;
    if (j == 0) r11 = fabs(beta);
    if (normx == 0.0 || !(fabs(beta) >= a.rcond * r11)) break;  // rank rule: p = j
    __syncthreads();
    if (threadIdx.x == 0) s_v[0] = x0 - beta;
    __syncthreads();
    double vv = 0.0;
    for (int64_t i = threadIdx.x; i < len; i += CP_THREADS) vv += s_v[i] * s_v[i];
    const double tau = 2.0 / cp_block_sum(vv, s_red);
    if (threadIdx.x == 0) {
      if (bid == 0) {
        a.piv[j] = pk;
        a.beta[j] = beta;
      }
      if (pk % nb == bid) a.done[pk] = 1;
    }
    __syncthreads();
    // reflect this CTA's unpivoted columns and the right-hand side (column d);
    // the new squared norms over rows j+1.. choose the next pivot
    bv = -1.0;
    bi = -1;
    for (int64_t c = bid + (int64_t)warp * nb; c <= d; c += (int64_t)CP_WARPS * nb) {
      if (c < d && a.done[c]) continue;
      double* col = a.B + c * ldb + j;
      double w = 0.0;
      for (int64_t i = lane; i < len; i += 32) w += s_v[i] * col[i];
      w = ski_warp_sum(w) * tau;
      double s = 0.0;
      for (int64_t i = lane; i < len; i += 32) {
        const double x = col[i] - w * s_v[i];
        col[i] = x;
        if (i > 0) s += x * x;
      }
      if (c < d) {
        s = ski_warp_sum(s);
        cp_better(bv, bi, s, (int)c);
      }
    }
    cp_block_argmax(bv, bi, s_av, s_ai);
    if (threadIdx.x == 0) {
      a.slot_v[(1 - par) * nb + bid] = bv;
      a.slot_i[(1 - par) * nb + bid] = bi;
    }
    if (!grid_sync(a.gb, nb, my_gen, a.spin_limit)) return;
  }
  if (bid == 0 && threadIdx.x == 0) *a.steps = (int32_t)j;
}

// B (column-major, ldb) <- [R | c] from R row-major (upper triangle) and c.
__global__ void k_cpqr_load(int64_t d, const double* __restrict__ R, int64_t ldr, const double* __restrict__ c,
                            double* __restrict__ B, int64_t ldb) {
  __shared__ double tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int k = ty; k < 32; k += 8) {
    const int64_t i = r0 + k, col = c0 + tx;
    double v = 0.0;
    if (i < d && col <= d) v = col < d ? (i <= col ? R[i * ldr + col] : 0.0) : c[i];
    tile[k][tx] = v;
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const int64_t col = c0 + k, i = r0 + tx;
    if (i < d && col <= d) B[col * ldb + i] = tile[tx][k];
  }
}

// R11 (p x p, row-major, ld11) and c1 = the first p entries of the reflected c.
__global__ void k_cpqr_extract(int64_t d, const double* __restrict__ B, int64_t ldb, const double* __restrict__ beta,
                               const int32_t* __restrict__ piv, const int32_t* __restrict__ steps,
                               double* __restrict__ R11, int64_t ld11, double* __restrict__ c1) {
  const int64_t p = *steps;
  const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t i = blockIdx.y;
  if (i >= p || l >= p) return;
  R11[i * ld11 + l] = i < l ? B[(int64_t)piv[l] * ldb + i] : (i == l ? beta[l] : 0.0);
  if (l == 0) c1[i] = B[d * ldb + i];
}

}  // namespace

size_t ski_cpqr_ws_bytes(int64_t d) {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaGetLastError();
  SkiArena ar{nullptr, 0, 0, true};
  ar.take<double>((d + 1) * d);
  ar.take<double>(d);
  ar.take<int8_t>(d);
  ar.take<double>(2 * (size_t)std::max(sms, 152));
  ar.take<int32_t>(2 * (size_t)std::max(sms, 152));
  ar.take<int32_t>(1);
  ar.take<GridBar>(1);
  return ar.off;
}

ski_status ski_cpqr_run(int64_t d, const double* R, int64_t ldr, const double* c, double rcond, double* R11,
                        int64_t ld11, double* c1, int32_t* piv, int32_t* p_out, SkiArena& ar, cudaStream_t st) {
  if (d < 1 || d > SKI_DENSE_DMAX || ldr < d || ld11 < 1) return SKI_EINVAL;
  int dev = 0, sms = 0, per_sm = 0;
  SKI_CUDA_TRY(cudaGetDevice(&dev));
  SKI_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const size_t smem = (size_t)d * sizeof(double);
  SKI_CUDA_TRY(cudaFuncSetAttribute((const void*)k_cpqr, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(SKI_DENSE_DMAX * sizeof(double))));
  SKI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k_cpqr, CP_THREADS, smem));
  if (per_sm < 1) return SKI_EINVAL;
  const int ncta = std::min(sms, 152 * 4);
  const int64_t ldb = d;
  CpqrArgs a{};
  a.d = d;
  a.ldb = ldb;
  a.B = ar.take<double>((d + 1) * ldb);
  a.beta = ar.take<double>(d);
  a.done = ar.take<int8_t>(d);
  a.slot_v = ar.take<double>(2 * (size_t)std::max(sms, 152));
  a.slot_i = ar.take<int32_t>(2 * (size_t)std::max(sms, 152));
  a.steps = ar.take<int32_t>(1);
  a.gb = ar.take<GridBar>(1);
  if (!ar.ok() || !a.B || !a.gb) return SKI_ENOMEM;
  a.piv = piv;
  a.rcond = rcond;
  a.spin_limit = 1ll << 24;
  SKI_CUDA_TRY(cudaMemsetAsync(a.gb, 0, sizeof(GridBar), st));
  SKI_CUDA_TRY(cudaMemsetAsync(a.steps, 0, sizeof(int32_t), st));
  {
    dim3 grid((unsigned)ski_cdiv(d + 1, 32), (unsigned)ski_cdiv(d, 32));
    k_cpqr_load<<<grid, dim3(32, 8), 0, st>>>(d, R, ldr, c, a.B, ldb);
    SKI_LAUNCH_CHECK();
  }
  void* args[] = {&a};
  SKI_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_cpqr, dim3(ncta), dim3(CP_THREADS), args, smem, st));
  ski_count_launch();
  {
    dim3 grid((unsigned)ski_cdiv(d, 256), (unsigned)d);
    k_cpqr_extract<<<grid, 256, 0, st>>>(d, a.B, ldb, a.beta, piv, a.steps, R11, ld11, c1);
    SKI_LAUNCH_CHECK();
  }
  GridBar h;
  int32_t p = 0;
  SKI_CUDA_TRY(cudaMemcpyAsync(&h, a.gb, sizeof(h), cudaMemcpyDeviceToHost, st));
  SKI_CUDA_TRY(cudaMemcpyAsync(&p, a.steps, sizeof(p), cudaMemcpyDeviceToHost, st));
  SKI_CUDA_TRY(cudaStreamSynchronize(st));
  if (h.err) return SKI_ETIMEOUT;
  *p_out = p;
  return SKI_OK;
}

namespace {
__global__ void k_gather(int64_t p, const int32_t* __restrict__ idx, const double* __restrict__ src,
                         double* __restrict__ dst) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k < p) dst[k] = src[idx[k]];
}
__global__ void k_scatter(int64_t p, const int32_t* __restrict__ idx, const double* __restrict__ src,
                          double* __restrict__ dst) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k < p) dst[idx[k]] = src[k];
}
}  // namespace

ski_status ski_gather_launch(int64_t p, const int32_t* idx, const double* src, double* dst, cudaStream_t st) {
  if (p < 1) return SKI_OK;
  k_gather<<<(unsigned)ski_cdiv(p, 256), 256, 0, st>>>(p, idx, src, dst);
  SKI_LAUNCH_CHECK();
  return SKI_OK;
}

ski_status ski_scatter_launch(int64_t d, int64_t p, const int32_t* idx, const double* src, double* dst,
                              cudaStream_t st) {
  SKI_CUDA_TRY(cudaMemsetAsync(dst, 0, d * sizeof(double), st));
  if (p < 1) return SKI_OK;
  k_scatter<<<(unsigned)ski_cdiv(p, 256), 256, 0, st>>>(p, idx, src, dst);
  SKI_LAUNCH_CHECK();
  return SKI_OK;
}
