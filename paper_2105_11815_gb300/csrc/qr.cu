// Step 2 of Algorithm 1: Householder QR of the sketch SA (m x d, m >= d),
// blocked in panels of NB = 32 columns (compact WY form, Schreiber & Van Loan).
//
// The factorisation works on the transpose Ct = [SA | Sb]^T (column j of SA
// contiguous), so that both trailing-update GEMMs read K-major operands:
//   W^T = C^T V   (K = rows of the panel)   and   C^T -= B'^T V^T (K = 32),
// which is the layout the TF32 tensor-core GEMM (gemm_tc.cu) consumes.  Each
// panel is copied to a row-major scratch, factored there, and copied back.
//
// Panel: column j of the panel is reduced by one launch that (a) finalises
// the reflector of column j-1 from the previous launch's partial sums --
// beta = -sign(x0) ||x||, tau = (beta - x0) / beta, v = [1; x_rest / (x0 - beta)]
// -- and applies it to the remaining panel columns, then (b) accumulates the
// partial dot products of column j with the panel for the next launch.  Each
// CTA owns a slab of rows; one warp handles one row, one lane one panel
// column, so every access is a coalesced 256 B row segment and the only
// cross-CTA exchange is the partials buffer between launches (no inter-CTA
// waits).  Partial sums are combined in a fixed order (deterministic).
//
// Trailing update: C <- (I - V T V^T)^T C = C - V (T^T (V^T C)), with V the
// explicit unit-lower-trapezoidal reflector block and T upper triangular
// (forward accumulation: T_ii = tau_i, T[0:i, i] = -tau_i T[0:i,0:i] V[:,0:i]^T v_i).
// V^T C is a split-K GEMM, C -= V (T^T W) a plain GEMM (gemm.cu).
// Applying the reflectors to column d of [SA | Sb] yields Q^T Sb for Step 3.
#include <cooperative_groups.h>

#include <type_traits>
#include <vector>

#include "common.cuh"
#include "sketch_impl.cuh"

namespace {

constexpr int NB = 32;
constexpr int PW = 2 * NB;  // partial slot: g[32] then the diagonal row[32]
constexpr int64_t kClusterRowsF64 = 16384;  // FP64 panels up to this height may take the cluster kernel
constexpr int WARPS = 8;
constexpr long long kSpinLimit = 1ll << 24;  // ~1 s of polling at ~64 ns per poll

template <class T>
struct PanelArgs {
  T* P;           // &B[k0, k0]
  int64_t ld;
  int64_t mr;     // rows of the panel (m - k0)
  int w;          // panel width <= NB
  int64_t rows_per;
  int ncta;
  const T* part_prev;
  T* part_cur;
  T* tau;
  T* V;           // explicit reflectors, mr x NB (row-major), written by the last step
  T* Vt;          // the same, transposed: NB x ldvt
  int64_t ldvt;
  T* Ct;          // &Ct[k0][k0]: panel column c, row r at Ct[c * ldt + r]
  int64_t ldt;
};

template <class T>
__device__ __forceinline__ T sgn_nrm(T x0, T nrm) { return x0 >= T(0) ? -nrm : nrm; }

// One column step s of the panel (see the file comment): finalise column
// s-1 from the partials of step s-1 and accumulate those of column s.
// Partials are read with L1-bypassing loads: in the persistent kernel they
// were written by other SMs during this launch.
// Where a step reads the previous step's per-CTA partials and writes its own:
// global memory (launch-per-step and grid-barrier kernels) or distributed
// shared memory (cluster kernel).
template <class T>
struct GlobalParts {
  const T* prev;
  T* cur;
  __device__ __forceinline__ int rank() const { return blockIdx.x; }
  __device__ __forceinline__ T get(int b, int idx) const { return __ldcg(&prev[(int64_t)b * PW + idx]); }
  __device__ __forceinline__ void put(int idx, T v) const { cur[(int64_t)blockIdx.x * PW + idx] = v; }
};

template <class T, int NW = WARPS, class Parts = GlobalParts<T>>
__device__ __forceinline__ void panel_step_body(PanelArgs<T> a, int s, const Parts& parts) {
  constexpr int WARPS = NW;
  __shared__ T red[NW][NB];
  __shared__ T s_par[4];  // tau, beta, scl
  __shared__ T s_wc[NB];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rank = parts.rank();
  const int j = s - 1;
  T tau = T(0), beta = T(0), scl = T(0), wc = T(0);
  if (s > 0) {
    // partial sums of the previous launch, split over the warps (fixed order)
    T g = T(0);
#pragma unroll 8
    for (int b = warp; b < a.ncta; b += WARPS) g += parts.get(b, lane);
    red[warp][lane] = g;
    __syncthreads();
    if (warp == 0) {
      g = T(0);
#pragma unroll
      for (int q = 0; q < WARPS; ++q) g += red[q][lane];
      const int owner = (int)(j / a.rows_per);
      const T dr = parts.get(owner, NB + lane);
      const T x0 = __shfl_sync(0xffffffffu, dr, j);
      const T gj = __shfl_sync(0xffffffffu, g, j);
      T tau_, beta_, scl_;
      if (gj == T(0)) {
        tau_ = T(0);
        beta_ = x0;
        scl_ = T(0);
      } else {
        const T nrm = sqrt(x0 * x0 + gj);
        beta_ = sgn_nrm(x0, nrm);
        tau_ = (beta_ - x0) / beta_;
        scl_ = T(1) / (x0 - beta_);
      }
      s_wc[lane] = dr + scl_ * g;  // v^T p_c for lanes c > j
      if (lane == 0) {
        s_par[0] = tau_;
        s_par[1] = beta_;
        s_par[2] = scl_;
        if (rank == 0) a.tau[j] = tau_;
      }
    }
    __syncthreads();
    tau = s_par[0];
    beta = s_par[1];
    scl = s_par[2];
    wc = s_wc[lane];
  }
  const int64_t r0 = (int64_t)rank * a.rows_per;
  const int64_t r1 = min(a.mr, r0 + a.rows_per);
  T acc = T(0);
  // independent rows: unrolled so the shuffles and shared-memory round trips
  // of several rows overlap (each step's latency is on the QR's critical path)
#pragma unroll 4
  for (int64_t r = r0 + warp; r < r1; r += WARPS) {
    T val = lane < a.w ? a.P[r * a.ld + lane] : T(0);
    if (s > 0 && r >= j) {
      T nv;
      if (r == j) {
        nv = lane == j ? beta : (lane > j ? val - tau * wc : val);
      } else {
        const T vr = scl * __shfl_sync(0xffffffffu, val, j);
        nv = lane == j ? vr : (lane > j ? val - (tau * wc) * vr : val);
      }
      if (lane < a.w && lane >= j) a.P[r * a.ld + lane] = nv;
      val = nv;
    }
    if (s < a.w) {
      const T ps = __shfl_sync(0xffffffffu, val, s);
      if (r == s) {
        parts.put(NB + lane, val);
      } else if (r > s) {
        acc = fma(ps, val, acc);
      }
    } else {
      // last step: explicit reflector block
      T v = (lane >= a.w || r < lane) ? T(0) : (r == lane ? T(1) : val);
      a.V[r * NB + lane] = v;
      a.Vt[(int64_t)lane * a.ldvt + r] = v;
    }
  }
  if (s < a.w) {
    __syncthreads();  // red[] may still be read by warp 0 of the finalisation above
    red[warp][lane] = acc;
    __syncthreads();
    if (warp == 0) {
      T t = T(0);
#pragma unroll
      for (int q = 0; q < WARPS; ++q) t += red[q][lane];
      parts.put(lane, t);
    }
  }
}

// Rows [r0, r1) of the panel between the column-major Ct and the row-major
// scratch P (ld = NB); columns >= w of P are zero.  Moved in 32 x 32 tiles
// through shared memory so that both sides are accessed in 128-byte rows.
template <class T>
__device__ __forceinline__ void panel_copy(const PanelArgs<T>& a, bool in) {
  __shared__ T tile[NB][NB + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t r0 = (int64_t)blockIdx.x * a.rows_per;
  const int64_t r1 = min(a.mr, r0 + a.rows_per);
  for (int64_t rb = r0; rb < r1; rb += NB) {
    if (in) {
      for (int c = warp; c < NB; c += WARPS) {
        const int64_t r = rb + lane;
        tile[c][lane] = (c < a.w && r < r1) ? a.Ct[(int64_t)c * a.ldt + r] : T(0);
      }
      __syncthreads();
      for (int i = warp; i < NB; i += WARPS)
        if (rb + i < r1) a.P[(rb + i) * NB + lane] = tile[lane][i];
    } else {
      for (int i = warp; i < NB; i += WARPS)
        if (rb + i < r1) tile[lane][i] = a.P[(rb + i) * NB + lane];
      __syncthreads();
      for (int c = warp; c < a.w; c += WARPS) {
        const int64_t r = rb + lane;
        if (r < r1) a.Ct[(int64_t)c * a.ldt + r] = tile[c][lane];
      }
    }
    __syncthreads();
  }
}

template <class T>
__global__ void __launch_bounds__(32 * WARPS) k_panel_copy(PanelArgs<T> a, int in) {
  panel_copy(a, in != 0);
}

template <class T>
__global__ void __launch_bounds__(32 * WARPS) k_panel_step(PanelArgs<T> a, int s) {
  panel_step_body<T>(a, s, GlobalParts<T>{a.part_prev, a.part_cur});
}

// The whole panel in one cooperative launch: the w + 1 column steps are
// separated by grid barriers instead of kernel boundaries, and each CTA keeps
// its slab of panel rows in shared memory for all of them (row stride
// NB + 1 against bank conflicts), so a step's row sweep never leaves the SM.
template <class T>
__global__ void __launch_bounds__(32 * WARPS) k_panel_coop(PanelArgs<T> a, T* partA, T* partB, GridBar* gb,
                                                          long long spin_limit) {
  extern __shared__ __align__(16) unsigned char slab_raw[];
  T* slab = reinterpret_cast<T*>(slab_raw);
  unsigned my_gen = 0;
  const int64_t r0 = (int64_t)blockIdx.x * a.rows_per;
  const int64_t r1 = min(a.mr, r0 + a.rows_per);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // copy-in: column c of the panel (contiguous in Ct) -> slab row-major
  for (int c = warp; c < NB; c += WARPS)
    for (int64_t r = r0 + lane; r < r1; r += 32)
      slab[(r - r0) * (NB + 1) + c] = c < a.w ? a.Ct[(int64_t)c * a.ldt + r] : T(0);
  __syncthreads();
  PanelArgs<T> b = a;
  b.P = slab - r0 * (NB + 1);  // indexed with global panel rows r in [r0, r1)
  b.ld = NB + 1;
  for (int s = 0; s <= a.w; ++s) {
    b.part_prev = (s & 1) ? partA : partB;
    b.part_cur = (s & 1) ? partB : partA;
    panel_step_body<T>(b, s, GlobalParts<T>{b.part_prev, b.part_cur});
    if (s < a.w && !grid_sync(gb, gridDim.x, my_gen, spin_limit)) return;
  }
  __syncthreads();
  for (int c = warp; c < a.w; c += WARPS)
    for (int64_t r = r0 + lane; r < r1; r += 32) a.Ct[(int64_t)c * a.ldt + r] = slab[(r - r0) * (NB + 1) + c];
}

// Distributed-shared-memory partials of the cluster kernel: step s writes
// slot s & 1 of its own CTA, step s + 1 reads slot s & 1 of every CTA.
template <class T>
struct ClusterParts {
  T* mine_prev;
  T* mine_cur;
  __device__ __forceinline__ int rank() const { return (int)cooperative_groups::this_cluster().block_rank(); }
  __device__ __forceinline__ T get(int b, int idx) const {
    return *cooperative_groups::this_cluster().map_shared_rank(mine_prev + idx, (unsigned)b);
  }
  __device__ __forceinline__ void put(int idx, T v) const { mine_cur[idx] = v; }
};

// The whole panel in one thread-block cluster (one cluster, up to 16 CTAs):
// slabs in shared memory, partials exchanged through distributed shared
// memory, one hardware cluster barrier per column step.
template <class T, int NW>
__global__ void __launch_bounds__(32 * NW) k_panel_cluster(PanelArgs<T> a) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char cl_raw[];
  T* slots = reinterpret_cast<T*>(cl_raw);  // [2][PW]
  T* slab = slots + 2 * PW;
  const int rank = (int)cl.block_rank();
  const int64_t r0 = (int64_t)rank * a.rows_per;
  const int64_t r1 = min(a.mr, r0 + a.rows_per);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = warp; c < NB; c += NW)
    for (int64_t r = r0 + lane; r < r1; r += 32)
      slab[(r - r0) * (NB + 1) + c] = c < a.w ? a.Ct[(int64_t)c * a.ldt + r] : T(0);
  __syncthreads();
  PanelArgs<T> b = a;
  b.P = slab - r0 * (NB + 1);
  b.ld = NB + 1;
  for (int s = 0; s <= a.w; ++s) {
    ClusterParts<T> parts{slots + ((s + 1) & 1) * PW, slots + (s & 1) * PW};
    panel_step_body<T, NW>(b, s, parts);
    // also after the last step, which still reads the other CTAs' partials:
    // no CTA may leave (and release its shared memory) while a peer reads it
    cl.sync();
  }
  __syncthreads();
  for (int c = warp; c < a.w; c += NW)
    for (int64_t r = r0 + lane; r < r1; r += 32) a.Ct[(int64_t)c * a.ldt + r] = slab[(r - r0) * (NB + 1) + c];
}

// ---- FP32 panel by Cholesky QR twice and Householder reconstruction
//
// The column-by-column panel meets a cluster barrier per column (4.5 us each
// at 8000 rows, the QR's critical path).  For FP32 the panel is instead
// factored with two cluster-wide reductions:
//   (1) CholeskyQR2 (Yamamoto, Nakatsukasa, Yanagisawa & Fukaya 2015):
//       G = P^T P, R1 = chol(G) (columns equilibrated by diag(G)^{-1/2}),
//       Q1 = P R1^{-1}, then the same on Q1: Q = Q1 R2^{-1}, R = R2 R1;
//   (2) Householder reconstruction (Ballard, Demmel, Grigori, Jacquelin,
//       Knight & Nguyen, "Reconstructing Householder vectors from tall-skinny
//       QR", 2015): LU without pivoting of Q - [S; 0], S = diag(s_i) with s_i =
//       -sign of the i-th pivot, gives Q - [S; 0] = Y U with Y unit lower
//       trapezoidal; then I - Y T Y^T with T = -U S Y1^{-T} is orthogonal, maps
//       [S; 0] to Q, and H^T P = [S R; 0].
// Y is the panel's reflector block V, T its compact-WY factor and S R its R
// (the signs of R's rows are arbitrary in any Householder QR).  The 32 x 32
// factorisations are done redundantly by every CTA of the cluster from the
// same reduced Gram matrices (fixed reduction order), so all CTAs agree.
// If an equilibrated Cholesky pivot falls below 2^-24 (panel condition above
// about 4e3, where CholeskyQR2 in FP32 loses orthogonality) the kernel
// restores the panel and takes the column-by-column steps instead, then
// forms T from V^T V and the reflector scalars; either way it writes V, V^T,
// T and the panel's R.
constexpr int HM = NB + 1;  // row stride of the 32 x 32 work matrices

// G (all CTAs) = sum over the cluster of the w x w Gram of this CTA's rows,
// with element (r, c) of a row given by val(r, c).  1024 threads: (i, j).
// Warps 0..7 each take every 8th row: lane j holds the row's entry j and
// accumulates column j of the Gram from the other entries by shuffles (no
// shared-memory traffic in the row loop); the 8 warp partials are then summed
// in a fixed order.  Wg: [8][NB][HM] scratch.
constexpr int GRAM_WARPS = 8;
template <class F>
__device__ __forceinline__ void cl_gram(int nrows, F val, float* Wg, float* Gp, float* G,
                                        const cooperative_groups::cluster_group& cl) {
  const int i = threadIdx.x >> 5, j = threadIdx.x & 31;
  if (i < GRAM_WARPS) {
    float acc[NB];
#pragma unroll
    for (int k = 0; k < NB; ++k) acc[k] = 0.f;
    for (int r = i; r < nrows; r += GRAM_WARPS) {
      const float pj = val(r, j);
#pragma unroll
      for (int k = 0; k < NB; ++k) acc[k] = fmaf(__shfl_sync(0xffffffffu, pj, k), pj, acc[k]);
    }
    float* wp = Wg + i * NB * HM;
#pragma unroll
    for (int k = 0; k < NB; ++k) wp[k * HM + j] = acc[k];
  }
  __syncthreads();
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < GRAM_WARPS; ++q) s += Wg[q * NB * HM + i * HM + j];
  Gp[i * HM + j] = s;
  cl.sync();
  float g = 0.f;
  for (unsigned b = 0; b < cl.num_blocks(); ++b) g += *cl.map_shared_rank(Gp + i * HM + j, b);
  G[i * HM + j] = g;
  cl.sync();  // every CTA has read every partial: Gp is free again
}

// The 32 x 32 factorisations below use the whole CTA (1024 threads; thread
// (i, j) = (threadIdx.x / 32, threadIdx.x % 32)) with two barriers per
// elimination step, or one warp per column for the triangular inverses:
// they are on the panel's critical path.

// R (upper, w x w) = chol(D A D) D^{-1}, D = diag(A)^{-1/2}; A is destroyed.
// False (the same in every thread) when a scaled pivot is below 2^-24 or not
// finite.  Dv: [NB] scratch.
__device__ __forceinline__ bool cta_chol(float* A, float* R, float* Dv, int w) {
  const int i = threadIdx.x >> 5, j = threadIdx.x & 31;
  if (i == 0) {
    const float a = j < w ? A[j * HM + j] : 1.f;
    Dv[j] = (a > 0.f && isfinite(a)) ? rsqrtf(a) : 0.f;
  }
  __syncthreads();
  for (int k = 0; k < w; ++k)
    if (!(Dv[k] > 0.f)) return false;  // uniform: every thread reads the same Dv
  if (i < w && j < w) A[i * HM + j] *= Dv[i] * Dv[j];
  R[i * HM + j] = 0.f;
  __syncthreads();
  for (int k = 0; k < w; ++k) {
    const float piv = A[k * HM + k];
    if (!(piv > 0x1p-24f) || !isfinite(piv)) return false;  // uniform
    const float rkk = sqrtf(piv);
    if (i == k && j >= k && j < w) R[k * HM + j] = j == k ? rkk : A[k * HM + j] / rkk;
    __syncthreads();
    if (i > k && i < w && j >= i && j < w) A[i * HM + j] -= R[k * HM + i] * R[k * HM + j];
    __syncthreads();
  }
  if (i < w && j < w && i <= j) R[i * HM + j] /= Dv[j];
  __syncthreads();
  return true;
}

// X = U^{-1} for upper triangular U (w x w): warp c forms column c by back
// substitution, the inner sums as warp reductions.
__device__ __forceinline__ void cta_upper_inv(const float* U, float* X, int w) {
  const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (c < NB) {
    float x = 0.f;  // lane l holds X[l][c]
    if (c < w)
      for (int k = c; k >= 0; --k) {
        const float s = ski_warp_sumf(lane > k && lane <= c ? U[k * HM + lane] * x : 0.f);
        if (lane == k) x = ((k == c ? 1.f : 0.f) - s) / U[k * HM + k];
      }
    X[lane * HM + c] = x;
  }
  __syncthreads();
}

// X = L^{-1} for unit lower triangular L (w x w), warp c forming column c.
__device__ __forceinline__ void cta_unit_lower_inv(const float* L, float* X, int w) {
  const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (c < NB) {
    float x = lane == c ? 1.f : 0.f;  // lane l holds X[l][c]
    if (c < w)
      for (int k = c + 1; k < w; ++k) {
        const float s = ski_warp_sumf(lane >= c && lane < k ? L[k * HM + lane] * x : 0.f);
        if (lane == k) x = -s;
      }
    X[lane * HM + c] = x;
  }
  __syncthreads();
}

// LU without pivoting of Q - S (Q: the top w x w block, destroyed), s_k = -sign
// of the k-th pivot, so |pivot| >= 1: L1 unit lower, U upper, S the signs.
__device__ __forceinline__ void cta_mod_lu(float* Q, float* L1, float* U, float* S, int w) {
  const int i = threadIdx.x >> 5, j = threadIdx.x & 31;
  L1[i * HM + j] = i == j ? 1.f : 0.f;
  U[i * HM + j] = 0.f;
  __syncthreads();
  for (int k = 0; k < w; ++k) {
    const float akk = Q[k * HM + k];
    const float sk = akk >= 0.f ? -1.f : 1.f;
    const float piv = akk - sk;
    if (i == k && j >= k && j < w) U[k * HM + j] = j == k ? piv : Q[k * HM + j];
    if (j == k && i > k && i < w) L1[i * HM + k] = Q[i * HM + k] / piv;
    if (i == k && j == k) S[k] = sk;
    __syncthreads();
    if (i > k && i < w && j > k && j < w) Q[i * HM + j] -= L1[i * HM + k] * U[k * HM + j];
    __syncthreads();
  }
}

// Rows [0, nrows) of the slab times an upper triangular X from the right;
// lane j keeps column j of X in registers, so the row loop is shuffles and
// FMAs only.
template <int NW>
__device__ __forceinline__ void rows_times_upper(float* slab, int nrows, const float* X, int w) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float xc[NB];
#pragma unroll
  for (int i = 0; i < NB; ++i) xc[i] = (i <= lane && lane < w && i < w) ? X[i * HM + lane] : 0.f;
  for (int r = warp; r < nrows; r += NW) {
    const float p = lane < w ? slab[r * HM + lane] : 0.f;
    float q = 0.f;
#pragma unroll
    for (int i = 0; i < NB; ++i) q = fmaf(__shfl_sync(0xffffffffu, p, i), xc[i], q);
    if (lane < w) slab[r * HM + lane] = q;
  }
}

template <int NW>
__global__ void __launch_bounds__(32 * NW) k_panel_chol(PanelArgs<float> a, float* Tm) {
  static_assert(NW == 32, "the Gram kernels map one thread to each of the 32 x 32 entries");
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char ch_raw[];
  float* slots = reinterpret_cast<float*>(ch_raw);  // [2][PW] for the column-by-column fallback
  float* Gp = slots + 2 * PW;                        // this CTA's Gram partial
  float* G = Gp + NB * HM;
  float* R1 = G + NB * HM;
  float* X = R1 + NB * HM;                           // inverses
  float* R2 = X + NB * HM;
  float* Qt = R2 + NB * HM;                          // top w rows of Q, then the LU work
  float* L1 = Qt + NB * HM;
  float* U = L1 + NB * HM;
  float* L1i = U + NB * HM;
  float* Ts = L1i + NB * HM;
  float* S = Ts + NB * HM;                           // [NB] signs
  float* Wg = S + NB;                                // [GRAM_WARPS][NB][HM] Gram partials
  float* slab = Wg + GRAM_WARPS * NB * HM;
  const int rank = (int)cl.block_rank();
  const int64_t r0 = (int64_t)rank * a.rows_per;
  const int64_t r1 = min(a.mr, r0 + a.rows_per);
  const int nrows = (int)max((int64_t)0, r1 - r0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int w = a.w;
  const int i2 = threadIdx.x >> 5, j2 = threadIdx.x & 31;  // (row, column) of the 32 x 32 products
  for (int c = warp; c < NB; c += NW)
    for (int64_t r = r0 + lane; r < r1; r += 32)
      slab[(r - r0) * HM + c] = c < w ? a.Ct[(int64_t)c * a.ldt + r] : 0.f;
  __syncthreads();
  auto plain = [&](int r, int c) { return slab[r * HM + c]; };
  // (1) CholeskyQR2
  cl_gram(nrows, plain, Wg, Gp, G, cl);
  bool ok = cta_chol(G, R1, S, w);
  if (ok) {
    cta_upper_inv(R1, X, w);
    rows_times_upper<NW>(slab, nrows, X, w);  // Q1 = P R1^{-1}
    __syncthreads();
    cl_gram(nrows, plain, Wg, Gp, G, cl);
    ok = cta_chol(G, R2, S, w);
    if (ok) cta_upper_inv(R2, X, w);
    if (!ok) {
      rows_times_upper<NW>(slab, nrows, R1, w);  // restore P = Q1 R1 for the fallback
      __syncthreads();
    }
  }
  if (ok) {
    rows_times_upper<NW>(slab, nrows, X, w);  // Q = Q1 R2^{-1}
    // R = R2 R1 into R2's place after the product (thread (i, j), k in [i, j])
    float rij = 0.f;
    if (i2 < w && j2 < w && i2 <= j2)
      for (int k = i2; k <= j2; ++k) rij = fmaf(R2[i2 * HM + k], R1[k * HM + j2], rij);
    __syncthreads();
    if (i2 < NB && j2 < NB) R2[i2 * HM + j2] = (i2 < w && j2 < w && i2 <= j2) ? rij : 0.f;
    // (2) Householder reconstruction: the top w rows of Q from their CTAs
    cl.sync();
    if (i2 < w && j2 < NB) {
      const int64_t owner = i2 / a.rows_per;
      const float* src = cl.map_shared_rank(slab + (i2 - owner * a.rows_per) * HM + j2, (unsigned)owner);
      Qt[i2 * HM + j2] = j2 < w ? *src : 0.f;
    }
    cl.sync();  // all have read the top rows: the slabs may change
    cta_mod_lu(Qt, L1, U, S, w);
    cta_upper_inv(U, X, w);       // X = U^{-1}
    cta_unit_lower_inv(L1, L1i, w);
    // T = -U S L1^{-T}: T[i][j] = -sum_{k=i..j} U[i][k] s_k L1i[j][k]
    {
      float t = 0.f;
      if (i2 < w && j2 < w && i2 <= j2)
        for (int k = i2; k <= j2; ++k) t = fmaf(U[i2 * HM + k] * S[k], L1i[j2 * HM + k], t);
      Ts[i2 * HM + j2] = -t;
    }
    // V rows at or below w: Q U^{-1}; rows above come from L1
    rows_times_upper<NW>(slab, nrows, X, w);
    __syncthreads();
    // outputs: the panel in Ct (S R on and above the diagonal, V below), V
    // (row-major: a warp per row), and Ct's and V^T's columns (a warp per
    // column, consecutive rows on consecutive lanes)
    auto vat = [&](int64_t r, int lr, int c) -> float {
      if (c >= w) return 0.f;
      if (r < w) return c < r ? L1[r * HM + c] : (c == r ? 1.f : 0.f);
      return slab[lr * HM + c];
    };
    for (int lr = warp; lr < nrows; lr += NW) a.V[(r0 + lr) * NB + lane] = vat(r0 + lr, lr, lane);
    for (int c = warp; c < NB; c += NW)
      for (int lr = lane; lr < nrows; lr += 32) {
        const int64_t r = r0 + lr;
        const float v = vat(r, lr, c);
        a.Vt[(int64_t)c * a.ldvt + r] = v;
        if (c < w) a.Ct[(int64_t)c * a.ldt + r] = (r < w && c >= r) ? S[r] * R2[r * HM + c] : v;
      }
    if (rank == 0 && i2 < NB && j2 < NB) {
      Tm[i2 * NB + j2] = (i2 < w && j2 < w) ? Ts[i2 * HM + j2] : 0.f;
      if (i2 == j2 && i2 < w) a.tau[i2] = Ts[i2 * HM + i2];
    }
    cl.sync();
    return;
  }
  // fallback: column-by-column Householder steps on the restored panel
  PanelArgs<float> b = a;
  b.P = slab - r0 * HM;
  b.ld = HM;
  for (int s = 0; s <= w; ++s) {
    ClusterParts<float> parts{slots + ((s + 1) & 1) * PW, slots + (s & 1) * PW};
    panel_step_body<float, NW>(b, s, parts);
    cl.sync();
  }
  __syncthreads();
  for (int c = warp; c < w; c += NW)
    for (int64_t r = r0 + lane; r < r1; r += 32) a.Ct[(int64_t)c * a.ldt + r] = slab[(r - r0) * HM + c];
  // T from V^T V and the reflector scalars (forward accumulation)
  auto vval = [&](int lr, int c) {
    const int64_t r = r0 + lr;
    return c >= w ? 0.f : (r < c ? 0.f : (r == c ? 1.f : slab[lr * HM + c]));
  };
  cl_gram(nrows, vval, Wg, Gp, G, cl);
  if (rank == 0 && warp == 0) {  // CTA 0 wrote the reflector scalars
    for (int k = 0; k < NB; ++k) Ts[k * HM + lane] = 0.f;
    __syncwarp();
    for (int i = 0; i < w; ++i) {
      const float ti = a.tau[i];
      float y = 0.f;
      if (lane < i)
        for (int k = lane; k < i; ++k) y = fmaf(Ts[lane * HM + k], G[k * HM + i], y);
      __syncwarp();
      if (lane < i) Ts[lane * HM + i] = -ti * y;
      if (lane == i) Ts[i * HM + i] = ti;
      __syncwarp();
    }
  }
  __syncthreads();
  if (rank == 0 && i2 < NB && j2 < NB) Tm[i2 * NB + j2] = (i2 < w && j2 < w) ? Ts[i2 * HM + j2] : 0.f;
  cl.sync();
}

// Self-test of the bounded barrier: `nblocks` is one more than the CTAs
// launched, so the barrier never completes and every wait must time out.
__global__ void k_barrier_timeout_probe(GridBar* gb, unsigned nblocks, long long spin_limit) {
  unsigned my_gen = 0;
  grid_sync(gb, nblocks, my_gen, spin_limit);
}


// Z = sum over splits of the V^T V and V^T C partials.
template <class T>
__global__ void k_reduce_z(int w, int64_t nct, const T* __restrict__ pv, int sv, const T* __restrict__ pc, int sc,
                           int64_t ldz, T* __restrict__ Z) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t cols = w + nct;
  if (idx >= (int64_t)w * cols) return;
  int64_t i = idx / cols, c = idx % cols;
  T acc = T(0);
  if (c < w) {
    for (int z = 0; z < sv; ++z) acc += pv[(int64_t)z * NB * NB + i * NB + c];
  } else {
    for (int z = 0; z < sc; ++z) acc += pc[(int64_t)z * NB * ldz + i * ldz + (c - w)];
  }
  Z[i * (NB + ldz) + c] = acc;
}

// T (upper triangular, w x w) from V^T V (first w columns of Z) and tau.
template <class T>
__global__ void k_tfactor(int w, const T* __restrict__ Z, int64_t ldzz, const T* __restrict__ tau, T* __restrict__ Tm) {
  __shared__ T Ts[NB][NB + 1];
  __shared__ T G[NB][NB + 1];
  const int lane = threadIdx.x;
  for (int c = 0; c < NB; ++c) {
    Ts[lane][c] = T(0);
    G[lane][c] = (lane < w && c < w) ? Z[lane * ldzz + c] : T(0);
  }
  __syncwarp();
  for (int i = 0; i < w; ++i) {
    // y[r] = sum_{k=r}^{i-1} T[r,k] * (V^T V)[k, i], r < i
    T y = T(0);
    if (lane < i)
      for (int k = lane; k < i; ++k) y += Ts[lane][k] * G[k][i];
    __syncwarp();
    if (lane < i) Ts[lane][i] = -tau[i] * y;
    if (lane == i) Ts[i][i] = tau[i];
    __syncwarp();
  }
  for (int c = 0; c < NB; ++c) Tm[lane * NB + c] = Ts[lane][c];
}

// One column per thread, one warp per CTA: in FP64 each column's 528 FMAs
// run on the 2-per-clock FP64 pipe, so the columns are spread over as many SMs
// as possible (a 545-column FP64 update: 43 us with 128 threads per CTA).
constexpr int kTtwThreads = 32;
// B'^T[c][i] = (T^T W)[i][c] for i < w, 0 for w <= i < NB; W = columns
// [w, w + nct) of Z.  Row-major nct x NB: the K-major operand of the update.
template <class T>
__global__ void k_ttw(int w, int64_t nct, const T* __restrict__ Z, int64_t ldzz, const T* __restrict__ Tm,
                      T* __restrict__ Bpt) {
  __shared__ T Ts[NB][NB];
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) Ts[e / NB][e % NB] = Tm[e];
  __syncthreads();
  int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= nct) return;
  T wcol[NB];
#pragma unroll
  for (int k = 0; k < NB; ++k) wcol[k] = k < w ? Z[k * ldzz + w + c] : T(0);
  for (int i = 0; i < NB; ++i) {
    T acc = T(0);
#pragma unroll
    for (int k = 0; k < NB; ++k)
      if (k <= i) acc += Ts[k][i] * wcol[k];  // (T^T)[i,k] = T[k,i], nonzero for k <= i
    Bpt[c * NB + i] = i < w ? acc : T(0);
  }
}

template <class T>
__global__ void k_extract_r(int64_t d, const T* __restrict__ Ct, int64_t ldt, int with_rhs, double* __restrict__ R,
                            int64_t ldr, double* __restrict__ qtsb) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= d * d) return;
  int64_t i = idx / d, c = idx % d;
  R[i * ldr + c] = c >= i ? SkiType<T>::to_f64(Ct[c * ldt + i]) : 0.0;
  if (c == 0 && with_rhs && qtsb) qtsb[i] = SkiType<T>::to_f64(Ct[d * ldt + i]);
}

// Ct[c][r] = SA[r][c] through a 32 x 32 shared-memory tile.
template <class T>
__global__ void k_transpose(int64_t m, int64_t ncols, const T* __restrict__ SA, int64_t ld_sa, T* __restrict__ Ct,
                            int64_t ldt) {
  __shared__ T tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32, c0 = (int64_t)blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t r = r0 + k, c = c0 + threadIdx.x;
    tile[k][threadIdx.x] = (r < m && c < ncols) ? SA[r * ld_sa + c] : T(0);
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t c = c0 + k, r = r0 + threadIdx.x;
    if (c < ncols && r < m) Ct[c * ldt + r] = tile[threadIdx.x][k];
  }
}

struct QrWs {
  int64_t ncta_max, splits_max, ldz, ldt;
};

QrWs qr_dims(int64_t m, int64_t ncols) {
  QrWs q;
  q.ncta_max = std::min<int64_t>(1024, ski_cdiv(m, 64));
  q.splits_max = 16;
  q.ldz = ski_round_up(ncols, 4);
  q.ldt = ski_round_up(m, 32);  // 128-byte rows: TMA strides and K offsets stay aligned
  return q;
}

template <class T>
struct QrBufs {
  // V, Vt, Tm alternate between panels (the low-priority update of panel k
  // still reads them while panel k + 1 is factored); pc, Z, Bpt are the
  // high-priority stream's, pc2, Z2, Bpt2 the low-priority stream's
  T *Ct, *P, *V, *V2, *Vt, *Vt2, *partA, *partB, *tau, *pv, *pc, *pc2, *Z, *Z2, *Tm, *Tm2, *Bpt, *Bpt2;
  GridBar* gb;
  int* err;
};

// One carving sequence for the size query and the run.
template <class T>
QrBufs<T> qr_carve(SkiArena& ar, int64_t m, int64_t ncols) {
  const QrWs q = qr_dims(m, ncols);
  QrBufs<T> b;
  b.Ct = ar.take<T>(ncols * q.ldt);
  b.P = ar.take<T>(m * NB);
  b.V = ar.take<T>(m * NB);
  b.V2 = ar.take<T>(m * NB);  // panels alternate: V of panel k is still read by its update
  b.Vt = ar.take<T>(NB * q.ldt);
  b.Vt2 = ar.take<T>(NB * q.ldt);
  b.partA = ar.take<T>(q.ncta_max * PW);
  b.partB = ar.take<T>(q.ncta_max * PW);
  b.tau = ar.take<T>(NB);
  b.pv = ar.take<T>(152 * NB * NB);
  b.pc = ar.take<T>(q.splits_max * NB * q.ldz);
  b.pc2 = ar.take<T>(q.splits_max * NB * q.ldz);
  b.Z = ar.take<T>(NB * (NB + q.ldz));
  b.Z2 = ar.take<T>(NB * (NB + q.ldz));
  b.Tm = ar.take<T>(NB * NB);
  b.Tm2 = ar.take<T>(NB * NB);
  b.Bpt = ar.take<T>(q.ldz * NB);
  b.Bpt2 = ar.take<T>(q.ldz * NB);
  b.gb = ar.take<GridBar>(1);
  b.err = ar.take<int>(1);
  return b;
}

// split3: the FP32 QR's products in three TF32 passes (about FP32 accuracy);
// false: one TF32 pass (SKI_TF32).
template <class T>
ski_status gemm_w(int64_t nct, int64_t mr, const T* Ctr, int64_t ldt, const T* Vt, T* pc, int64_t ldz, int sc,
                  int* err, cudaStream_t st, bool split3);
template <>
ski_status gemm_w<float>(int64_t nct, int64_t mr, const float* Ctr, int64_t ldt, const float* Vt, float* pc,
                         int64_t ldz, int sc, int* err, cudaStream_t st, bool split3) {
  // W^T(c, i) = sum_r Ct[c][r] Vt[i][r] on the tensor cores, stored as W[i][c]
  return ski_gemm_tf32(Ctr, ldt, Vt, ldt, nct, NB, mr, pc, ldz, 2, sc, (int64_t)NB * ldz, err, st, split3);
}
template <>
ski_status gemm_w<double>(int64_t nct, int64_t mr, const double* Ctr, int64_t ldt, const double* Vt, double* pc,
                          int64_t ldz, int sc, int* err, cudaStream_t st, bool) {
  (void)err;
  return ski_gemm_ex<double>(NB, nct, mr, 1.0, Vt, ldt, 1, Ctr, 1, ldt, 0.0, pc, ldz, sc, (int64_t)NB * ldz, st);
}

template <class T>
ski_status gemm_update(int64_t nct, int64_t mr, const T* Bpt, const T* V, T* Ctr, int64_t ldt, int* err,
                       cudaStream_t st, bool split3);
template <>
ski_status gemm_update<float>(int64_t nct, int64_t mr, const float* Bpt, const float* V, float* Ctr, int64_t ldt,
                              int* err, cudaStream_t st, bool split3) {
  // Ct[c][r] -= sum_i B'^T[c][i] V[r][i] on the tensor cores (K = 32)
  return ski_gemm_tf32(Bpt, NB, V, NB, nct, mr, NB, Ctr, ldt, 1, 1, 0, err, st, split3);
}
template <>
ski_status gemm_update<double>(int64_t nct, int64_t mr, const double* Bpt, const double* V, double* Ctr, int64_t ldt,
                               int* err, cudaStream_t st, bool) {
  (void)err;
  return ski_gemm<double>(nct, mr, NB, -1.0, Bpt, NB, 1, V, 1, NB, 1.0, Ctr, ldt, st);
}

// Optional CUDA-event timing of the trailing-update GEMMs (W = V^T C and
// C -= V B'), summed over the panels: the live roofline of the QR's dominant
// kernels.  Events are recorded on the launching stream only.
struct GemmTimer {
  std::vector<cudaEvent_t> ev;
  bool on;
  explicit GemmTimer(bool enable) : on(enable) {}
  ~GemmTimer() {
    for (auto e : ev) cudaEventDestroy(e);
  }
  void mark(cudaStream_t st) {
    if (!on) return;
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) {
      on = false;
      return;
    }
    cudaEventRecord(e, st);
    ev.push_back(e);
  }
  double total_ms() {  // pairs (start, stop); the stream must be synchronised
    double s = 0.0;
    for (size_t i = 0; i + 1 < ev.size(); i += 2) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev[i], ev[i + 1]) == cudaSuccess) s += ms;
    }
    return s;
  }
};

// Look-ahead (two streams): panel k's trailing update is split into the next
// panel's 32 columns (on the high-priority stream, right before that panel)
// and the rest (on the low-priority stream), so panel k + 1 -- latency-bound,
// one barrier per column -- runs while the bulk of update k is in flight, and
// freed SMs go to the panel's CTAs first.  The two streams belong to the host
// thread (created once per thread and device) and join the caller's stream
// at both ends of the factorisation.
struct QrStreams {
  cudaStream_t hi = nullptr, lo = nullptr;
  cudaEvent_t e_start = nullptr, e_upd = nullptr, e_lo = nullptr, e_done = nullptr;
  int dev = -1;
  bool ok = false;
  ~QrStreams() {
    if (e_start) cudaEventDestroy(e_start);
    if (e_upd) cudaEventDestroy(e_upd);
    if (e_lo) cudaEventDestroy(e_lo);
    if (e_done) cudaEventDestroy(e_done);
    if (hi) cudaStreamDestroy(hi);
    if (lo) cudaStreamDestroy(lo);
  }
};

QrStreams* qr_streams() {
  static thread_local QrStreams s[8];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 8) {
    cudaGetLastError();
    return nullptr;
  }
  QrStreams& q = s[dev];
  if (!q.ok && q.dev != dev) {
    q.dev = dev;
    int least = 0, greatest = 0;
    q.ok = cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess &&
           cudaStreamCreateWithPriority(&q.hi, cudaStreamNonBlocking, greatest) == cudaSuccess &&
           cudaStreamCreateWithPriority(&q.lo, cudaStreamNonBlocking, least) == cudaSuccess &&
           cudaEventCreateWithFlags(&q.e_start, cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&q.e_upd, cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&q.e_lo, cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&q.e_done, cudaEventDisableTiming) == cudaSuccess;
    if (!q.ok) cudaGetLastError();
  }
  return q.ok ? &q : nullptr;
}

// cluster panels: 16 CTAs (non-portable size) when the device runs such a
// cluster with the largest slab, else 8.  FP32, and FP64 panels of at most
// kClusterRowsF64 rows whose slabs fit in shared memory (about 12400 rows with
// 16 CTAs).  A tall FP64 panel does its rank-1 updates on the 1/64-rate FP64
// pipe, which 64 SMs (grid-barrier kernel) finish sooner than 16.  But the
// FP64 QR is bound by the trailing update that runs beside the panel, and a
// 16-CTA cluster leaves it 136 SMs instead of 88: the FP64 QR of 8000 x 4001
// took 245.5 ms with cluster panels against 250.3 ms with grid-barrier panels
// above 4096 rows.  A short panel is bound by the per-column synchronisation,
// which the cluster barrier does faster; and 16-CTA clusters run beside the
// other streams' work, where a cooperative grid waits for 64 free SMs.
constexpr int kPanelWarps = 32;  // 16 hid too little of each step's row-loop latency (36.5 -> 32.1 ms at 8000 x 4000)
// FP32 panels: Cholesky QR twice and Householder reconstruction in the
// cluster (two cluster reductions per panel instead of one barrier per
// column), when its work matrices and slab fit in shared memory
constexpr size_t kCholSmem = 200 * 1024;
struct QrSetup {
  bool coop = false, cluster_ok = false, chol_ok = false;
  int CL = 0;
};
template <class T>
const QrSetup& qr_setup() {
  static std::mutex mu;
  static QrSetup su[8];
  static bool have[8] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 8) {
    cudaGetLastError();
    static const QrSetup none;
    return none;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (have[dev]) return su[dev];
  QrSetup& q = su[dev];
  int can = 0;
  q.coop = cudaDeviceGetAttribute(&can, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && can != 0;
  constexpr int CNW = kPanelWarps;
  const size_t big = (size_t)(200 * 1024 + 2 * PW * sizeof(T));
  if (cudaFuncSetAttribute(k_panel_cluster<T, CNW>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
          cudaSuccess &&
      cudaFuncSetAttribute(k_panel_cluster<T, CNW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)big) ==
          cudaSuccess) {
    for (int cand : {16, 8}) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = cand;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3(cand);
      cfg.blockDim = dim3(32 * CNW);
      cfg.dynamicSmemBytes = big;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int nclus = 0;
      if (cudaOccupancyMaxActiveClusters(&nclus, k_panel_cluster<T, CNW>, &cfg) == cudaSuccess && nclus >= 1) {
        q.CL = cand;
        q.cluster_ok = true;
        break;
      }
    }
  }
  if constexpr (sizeof(T) == 4) {
    if (q.cluster_ok &&
        cudaFuncSetAttribute(k_panel_chol<CNW>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
        cudaFuncSetAttribute(k_panel_chol<CNW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCholSmem) ==
            cudaSuccess)
      q.chol_ok = true;
  }
  cudaGetLastError();
  have[dev] = true;
  return q;
}

template <class T>
ski_status qr_impl(int64_t m, int64_t d, int32_t with_rhs, T* B, int64_t ld, double* R, int64_t ldr, double* qtsb,
                   SkiArena& ar, cudaStream_t caller, double* gemm_ms, bool split3) {
  GemmTimer timer(gemm_ms != nullptr);
  // main sequence on the high-priority stream (or the caller's if the
  // auxiliary streams are unavailable), the bulk of each update on the low one
  QrStreams* qs = qr_streams();
  cudaStream_t st = caller, st_lo = caller;
  if (qs) {
    SKI_CUDA_TRY(cudaEventRecord(qs->e_start, caller));
    SKI_CUDA_TRY(cudaStreamWaitEvent(qs->hi, qs->e_start, 0));
    st = qs->hi;
    st_lo = qs->lo;
  }
  bool pending_lo = false;  // an update still running on st_lo
  const int64_t ncols = d + (with_rhs ? 1 : 0);
  const QrWs q = qr_dims(m, ncols);
  QrBufs<T> bf = qr_carve<T>(ar, m, ncols);
  if (!ar.ok() || !bf.err) return SKI_ENOMEM;
  const int64_t ldt = q.ldt;
  // launch setup of this device (cooperative panels, cluster size, the FP32
  // Cholesky panel), queried once per process and device: the attribute and
  // occupancy calls take the driver's process-wide lock, which the host threads
  // of a batch would otherwise meet at every factorisation
  const QrSetup& su = qr_setup<T>();
  const bool coop = su.coop;
  const int64_t max_slab_rows = (200 * 1024) / ((NB + 1) * (int64_t)sizeof(T));
  constexpr int CNW = kPanelWarps;
  const int CL = su.CL;
  // FP32, and FP64 panels of at most kClusterRowsF64 rows, take the cluster kernel
  const bool cluster_ok = su.cluster_ok && (sizeof(T) == 4 || m <= kClusterRowsF64);
  constexpr size_t kCholMats = (size_t)(2 * PW + (10 + GRAM_WARPS) * NB * (NB + 1) + NB) * sizeof(float);
  constexpr size_t kCholSmemMax = kCholSmem;
  const bool chol_ok = sizeof(T) == 4 && cluster_ok && su.chol_ok;
  SKI_CUDA_TRY(cudaMemsetAsync(bf.err, 0, sizeof(int), st));
  SKI_CUDA_TRY(cudaMemsetAsync(bf.gb, 0, sizeof(GridBar), st));
  {
    dim3 grid((unsigned)ski_cdiv(m, 32), (unsigned)ski_cdiv(ncols, 32));
    k_transpose<T><<<grid, dim3(32, 8), 0, st>>>(m, ncols, B, ld, bf.Ct, ldt);
    SKI_LAUNCH_CHECK();
  }
  int timed_out = 0;
  for (int64_t k0 = 0; k0 < d; k0 += NB) {
    const int w = (int)std::min<int64_t>(NB, d - k0);
    const int64_t mr = m - k0;
    // few, fat CTAs: each column step reads every CTA's partials and meets
    // at a grid barrier, so both costs grow with the CTA count
    int ncta = (int)std::min<int64_t>(std::min<int64_t>(q.ncta_max, 64), ski_cdiv(mr, 128));
    // the persistent kernel keeps each CTA's rows in shared memory: one CTA per
    // SM at most, so the slab must fit and the CTAs must fit on the SMs
    const int ncta_coop = (int)std::max<int64_t>(ncta, ski_cdiv(mr, max_slab_rows));
    const bool use_coop = coop && ncta_coop <= 148;
    if (use_coop) ncta = ncta_coop;
    const int64_t rows_per = ski_cdiv(mr, ncta);
    T* Ctp = bf.Ct + k0 * ldt + k0;
    const bool odd = ((k0 / NB) & 1) != 0;
    T* Vk = odd ? bf.V2 : bf.V;
    T* Vtk = odd ? bf.Vt2 : bf.Vt;
    T* Tmk = odd ? bf.Tm2 : bf.Tm;
    PanelArgs<T> pa{bf.P, NB, mr, w, rows_per, ncta, nullptr, nullptr, bf.tau, Vk, Vtk, ldt, Ctp, ldt};
    bool done_panel = false;
    bool t_from_panel = false;  // the panel kernel wrote T (and no V^T V is needed)
    if constexpr (sizeof(T) == 4) {
      const int64_t rp = ski_cdiv(mr, CL);
      const size_t csm = kCholMats + (size_t)rp * (NB + 1) * sizeof(float);
      if (chol_ok && csm <= kCholSmemMax) {
        PanelArgs<T> pc = pa;
        pc.rows_per = rp;
        pc.ncta = CL;
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = CL;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(CL);
        cfg.blockDim = dim3(32 * CNW);
        cfg.dynamicSmemBytes = csm;
        cfg.stream = st;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        SKI_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_panel_chol<CNW>, pc, Tmk));
        SKI_LAUNCH_CHECK();
        done_panel = true;
        t_from_panel = true;
      }
    }
    if (!done_panel && cluster_ok && (sizeof(T) == 4 || mr <= kClusterRowsF64)) {
      // one cluster of CL CTAs: the slab of each must fit in shared memory
      const int64_t rp = ski_cdiv(mr, CL);
      const size_t csm = (size_t)(2 * PW + rp * (NB + 1)) * sizeof(T);
      if (csm <= 200 * 1024) {
        PanelArgs<T> pc = pa;
        pc.rows_per = rp;
        pc.ncta = CL;
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = CL;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(CL);
        cfg.blockDim = dim3(32 * CNW);
        cfg.dynamicSmemBytes = csm;
        cfg.stream = st;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        SKI_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_panel_cluster<T, CNW>, pc));
        SKI_LAUNCH_CHECK();
        done_panel = true;
      }
    }
    if (done_panel) {
    } else if (use_coop) {
      SKI_CUDA_TRY(cudaMemsetAsync(bf.gb, 0, 2 * sizeof(unsigned), st));  // count, gen (keep err)
      long long lim = kSpinLimit;
      void* args[] = {&pa, &bf.partA, &bf.partB, &bf.gb, &lim};
      const size_t smem = (size_t)rows_per * (NB + 1) * sizeof(T);
      if (smem > 48 * 1024)
        SKI_CUDA_TRY(
            cudaFuncSetAttribute(k_panel_coop<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 ski_smem_cap((const void*)k_panel_coop<T>)));
      SKI_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_panel_coop<T>, dim3(ncta), dim3(32 * WARPS), args,
                                               smem, st));
      SKI_LAUNCH_CHECK();
    } else {
      k_panel_copy<T><<<ncta, 32 * WARPS, 0, st>>>(pa, 1);
      SKI_LAUNCH_CHECK();
      for (int s = 0; s <= w; ++s) {
        pa.part_prev = (s & 1) ? bf.partA : bf.partB;
        pa.part_cur = (s & 1) ? bf.partB : bf.partA;
        k_panel_step<T><<<ncta, 32 * WARPS, 0, st>>>(pa, s);
        SKI_LAUNCH_CHECK();
      }
      k_panel_copy<T><<<ncta, 32 * WARPS, 0, st>>>(pa, 0);
      SKI_LAUNCH_CHECK();
    }
    const int64_t nct = ncols - (k0 + w);
    T* Ctr = bf.Ct + (k0 + w) * ldt + k0;  // trailing columns, rows k0..m-1
    // V^T V (split-K over rows, for T) and W = V^T C.  Look-ahead: the next
    // panel's NB columns are updated first, on the high-priority stream, and
    // the rest on the low-priority stream, so that the bulk of the update does
    // not lie between this panel and the next.  FP32 also moves the rest's
    // share of W (and of T^T W) to the low-priority stream; in FP64, where
    // the GEMMs saturate the FP64 pipe and only overlap, W stays whole on the
    // high-priority stream.  Below ~4M updated elements the split costs more
    // than it overlaps.
    const int sv = t_from_panel ? 0 : (int)std::min<int64_t>(152, ski_cdiv(mr, 64));
    if (!t_from_panel)
      SKI_TRY(ski_gemm_ex<T>(NB, NB, mr, T(1), Vtk, ldt, 1, Vtk, 1, ldt, T(0), bf.pv, NB, sv, (int64_t)NB * NB, st));
    constexpr bool split_w = std::is_same<T, float>::value;
    const int64_t nu = (qs && nct > NB && mr * (nct - NB) >= (1ll << 22)) ? NB : nct;
    const int64_t nw = split_w ? nu : nct;
    if (pending_lo) {  // the previous panel's low-priority update wrote the columns W reads
      SKI_CUDA_TRY(cudaStreamWaitEvent(st, qs->e_lo, 0));
      pending_lo = false;
    }
    auto splits_for = [&](int64_t cols) {
      const int64_t tiles = ski_cdiv(cols, 128);
      int sc = (int)std::max<int64_t>(1, std::min<int64_t>(q.splits_max, ski_cdiv(300, tiles)));
      return (int)std::min<int64_t>(sc, ski_cdiv(mr, 128));
    };
    int sca = 1;
    if (nw > 0) {
      sca = splits_for(nw);
      timer.mark(st);
      SKI_TRY(gemm_w<T>(nw, mr, Ctr, ldt, Vtk, bf.pc, q.ldz, sca, bf.err, st, split3));
      timer.mark(st);
    }
    k_reduce_z<T><<<ski_cdiv(w * (w + nw), 256), 256, 0, st>>>(w, nw, bf.pv, sv, bf.pc, sca, q.ldz, bf.Z);
    SKI_LAUNCH_CHECK();
    if (!t_from_panel) {
      k_tfactor<T><<<1, 32, 0, st>>>(w, bf.Z, NB + q.ldz, bf.tau, Tmk);
      SKI_LAUNCH_CHECK();
    }
    if (nw > 0) {
      k_ttw<T><<<ski_cdiv(nw, kTtwThreads), kTtwThreads, 0, st>>>(w, nw, bf.Z, NB + q.ldz, Tmk, bf.Bpt);
      SKI_LAUNCH_CHECK();
    }
    if (nu < nct) {
      // the rest, on the low-priority stream once V, V^T and T (and in FP64
      // T^T W) of this panel exist
      const int64_t nr = nct - nu;
      SKI_CUDA_TRY(cudaEventRecord(qs->e_upd, st));
      SKI_CUDA_TRY(cudaStreamWaitEvent(st_lo, qs->e_upd, 0));
      const T* Bq = bf.Bpt + nu * NB;
      if (split_w) {
        const int scb = splits_for(nr);
        timer.mark(st_lo);
        SKI_TRY(gemm_w<T>(nr, mr, Ctr + nu * ldt, ldt, Vtk, bf.pc2, q.ldz, scb, bf.err, st_lo, split3));
        timer.mark(st_lo);
        k_reduce_z<T><<<ski_cdiv(w * (w + nr), 256), 256, 0, st_lo>>>(w, nr, bf.pv, 0, bf.pc2, scb, q.ldz, bf.Z2);
        SKI_LAUNCH_CHECK();
        k_ttw<T><<<ski_cdiv(nr, kTtwThreads), kTtwThreads, 0, st_lo>>>(w, nr, bf.Z2, NB + q.ldz, Tmk, bf.Bpt2);
        SKI_LAUNCH_CHECK();
        Bq = bf.Bpt2;
      }
      timer.mark(st_lo);
      SKI_TRY(gemm_update<T>(nr, mr, Bq, Vk, Ctr + nu * ldt, ldt, bf.err, st_lo, split3));
      timer.mark(st_lo);
      SKI_CUDA_TRY(cudaEventRecord(qs->e_lo, st_lo));
      pending_lo = true;
    }
    if (nu > 0) {
      timer.mark(st);
      SKI_TRY(gemm_update<T>(nu, mr, bf.Bpt, Vk, Ctr, ldt, bf.err, st, split3));
      timer.mark(st);
    }
  }
  if (pending_lo) SKI_CUDA_TRY(cudaStreamWaitEvent(st, qs->e_lo, 0));
  k_extract_r<T><<<ski_cdiv(d * d, 256), 256, 0, st>>>(d, bf.Ct, ldt, with_rhs, R, ldr, qtsb);
  SKI_LAUNCH_CHECK();
  if (qs) {
    SKI_CUDA_TRY(cudaEventRecord(qs->e_done, st));
    SKI_CUDA_TRY(cudaStreamWaitEvent(caller, qs->e_done, 0));
    st = caller;
  }
  {
    GridBar h;
    int e = 0;
    SKI_CUDA_TRY(cudaMemcpyAsync(&h, bf.gb, sizeof(h), cudaMemcpyDeviceToHost, st));
    SKI_CUDA_TRY(cudaMemcpyAsync(&e, bf.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SKI_CUDA_TRY(cudaStreamSynchronize(st));
    timed_out = h.err || e;
  }
  if (gemm_ms) *gemm_ms = timer.total_ms();
  return timed_out ? SKI_ETIMEOUT : SKI_OK;
}

}  // namespace

size_t ski_qr_ws_bytes(int64_t m, int64_t ncols, int32_t dtype) {
  SkiArena ar{nullptr, 0, 0, true};
  if (dtype == SKI_F64) qr_carve<double>(ar, m, ncols);
  else qr_carve<float>(ar, m, ncols);
  return ar.off;
}

ski_status ski_qr_run(int64_t m, int64_t d, int32_t with_rhs, void* SA, int64_t ld_sa, int32_t dtype, double* R,
                      int64_t ldr, double* qtsb, SkiArena& ar, cudaStream_t st, double* gemm_ms) {
  if (dtype == SKI_F64)
    return qr_impl<double>(m, d, with_rhs, (double*)SA, ld_sa, R, ldr, qtsb, ar, st, gemm_ms, false);
  if (dtype == SKI_F32 || dtype == SKI_TF32)
    return qr_impl<float>(m, d, with_rhs, (float*)SA, ld_sa, R, ldr, qtsb, ar, st, gemm_ms, dtype == SKI_F32);
  return SKI_EINVAL;
}

// Self-test of the bounded grid barrier used by the persistent panel kernel:
// 4 co-resident CTAs wait for a fifth that never arrives; each wait gives up
// after `spin_limit` polls and the error flag must come back set.
ski_status ski_barrier_selftest(long long spin_limit, void* ws, cudaStream_t st) {
  GridBar* gb = (GridBar*)ws;
  SKI_CUDA_TRY(cudaMemsetAsync(gb, 0, sizeof(GridBar), st));
  unsigned nb = 5;
  void* args[] = {&gb, &nb, &spin_limit};
  SKI_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_barrier_timeout_probe, dim3(4), dim3(32), args, 0, st));
  SKI_LAUNCH_CHECK();
  GridBar h;
  SKI_CUDA_TRY(cudaMemcpyAsync(&h, gb, sizeof(h), cudaMemcpyDeviceToHost, st));
  SKI_CUDA_TRY(cudaStreamSynchronize(st));
  return h.err ? SKI_ETIMEOUT : SKI_OK;
}
