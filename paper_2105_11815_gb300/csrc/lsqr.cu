// Step 4 of Algorithm 1: LSQR (Paige & Saunders, ACM TOMS 1982) on
// min ||W delta - r0||, W = A R^{-1}, with the Eq. TC-lsqr stopping test, and
// the FP64 residual / acceptance passes of Steps 3 and 5.
//
// One LSQR iteration is five launches, all device-resident (no host sync):
//   z = M v                      (upper-triangular matvec, M = R^{-1})
//   t = A z - (alpha/beta) t     (fused pass: also accumulates A^T t and ||t||^2
//                                 per CTA, so A is read once per iteration)
//   q = A^T t, beta = ||t||      (fixed-order reduction of the CTA partials)
//   p = M^T q                    (matvec with the stored transpose of M)
//   v, alpha, rotation, y, w     (one CTA; sets `done` on Eq. TC-lsqr)
// u_i is kept unnormalised (t_i = beta_i u_i), so no pass rescales it.  Every
// kernel returns at once when `done` is set, so the host only polls the flag
// every few iterations.
#include "common.cuh"
#include "lsqr_impl.cuh"

namespace {

__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = ski_warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = 0.0;
  const int nw = (blockDim.x + 31) >> 5;
  for (int q = 0; q < nw; ++q) t += sh[q];
  return t;
}

// y = M x (UPPER: M upper triangular, row i uses c >= i) or y = Mt x with Mt
// lower triangular (row c uses i <= c); optionally y += add.  Warp per row.
template <bool UPPER>
__global__ void __launch_bounds__(256) k_trmv(int64_t d, const double* __restrict__ M, int64_t ldm,
                                              const double* __restrict__ x, const double* __restrict__ add,
                                              double* __restrict__ y, const LsqrScalars* __restrict__ sc) {
  if (sc && sc->flag_a) return;
  const int lane = threadIdx.x & 31;
  const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (row >= d) return;
  const int64_t c0 = UPPER ? row : 0, c1 = UPPER ? d : row + 1;
  const double* mr = M + row * ldm;
  double acc = row_dot8(mr, x, c0 + lane, c1);
  acc = ski_warp_sum(acc);
  if (lane == 0) y[row] = add ? add[row] + acc : acc;
}

// Error-free transformations (Knuth's TwoSum; TwoProduct by FMA) and the
// compensated dot product Dot2 of Ogita, Rump & Oishi (SIAM J. Sci. Comput.
// 26, 2005): a sum of products accumulated as an unevaluated pair (s, c)
// whose value s + c is as accurate as if computed in twice the working
// precision.
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  s = a + b;
  const double z = s - a;
  e = (a - (s - z)) + (b - z);
}
__device__ __forceinline__ void dot2_add(double a, double x, double& s, double& c) {
  const double p = a * x;
  const double pe = fma(a, x, -p);
  double t, te;
  two_sum(s, p, t, te);
  s = t;
  c += pe + te;
}
__device__ __forceinline__ void pair_add(double& s, double& c, double s2, double c2) {
  double t, te;
  two_sum(s, s2, t, te);
  s = t;
  c += c2 + te;
}
__device__ __forceinline__ void pair_warp_sum(double& s, double& c) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double s2 = __shfl_xor_sync(0xffffffffu, s, o);
    const double c2 = __shfl_xor_sync(0xffffffffu, c, o);
    pair_add(s, c, s2, c2);
  }
}

// Dense fused pass over A.  Thread tid owns columns tid + k*NT (k < CPT);
// RR rows are processed per step.  t_j = ca (A_j z) + cu u_j + cb b_j.
// COMP (the residual r = b - A z of the acceptance test: ca = -1, cb = 1, no
// u): A_j z is a compensated dot product and r_j = b_j - A_j z is rounded
// once, so r is accurate to the last bit even where b - A z cancels many
// digits (x large along small singular directions), and the FP64 metric
// ||A^T r|| / (||A||_F ||r||) is then a certificate, not a rounding floor.
template <int CPT, int RR, bool COMP>
__global__ void __launch_bounds__(512) k_fused_dense(FusedArgs f) {
  constexpr int NT = 512;
  __shared__ double red[RR][NT / 32];
  __shared__ double redc[COMP ? RR : 1][NT / 32];
  __shared__ double tsh[RR];
  const LsqrScalars* sc = f.sc;
  if (sc && sc->flag_a) return;
  double ca = f.ca, cu = f.cu, cb = f.cb;
  if (f.coef_from_scalars) {
    ca = 1.0;
    cu = -sc->coef;
    cb = 0.0;
  }
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int64_t r0 = (int64_t)blockIdx.x * f.rows_per;
  const int64_t r1 = min(f.n, r0 + f.rows_per);
  double zr[CPT], acc[CPT], aa = 0.0, tt = 0.0;
  int emax = 0;
#pragma unroll
  for (int k = 0; k < CPT; ++k) {
    const int64_t c = tid + (int64_t)k * NT;
    zr[k] = c < f.d ? f.z[c] : 0.0;
    acc[k] = 0.0;
  }
  for (int64_t j0 = r0; j0 < r1; j0 += RR) {
    double a[RR][CPT];
#pragma unroll
    for (int r = 0; r < RR; ++r)
#pragma unroll
      for (int k = 0; k < CPT; ++k) {
        const int64_t c = tid + (int64_t)k * NT;
        a[r][k] = (j0 + r < r1 && c < f.d) ? __ldcs(&f.A[(j0 + r) * f.lda + c]) : 0.0;
      }
    if (f.maxexp) {
#pragma unroll
      for (int r = 0; r < RR; ++r)
#pragma unroll
        for (int k = 0; k < CPT; ++k) emax = max(emax, (int)((__double_as_longlong(a[r][k]) >> 52) & 0x7FF));
    }
    double p[RR], pc[COMP ? RR : 1];
#pragma unroll
    for (int r = 0; r < RR; ++r) {
      double s = 0.0, c = 0.0;
      if (COMP) {
#pragma unroll
        for (int k = 0; k < CPT; ++k) dot2_add(a[r][k], zr[k], s, c);
        pair_warp_sum(s, c);
        pc[COMP ? r : 0] = c;
      } else {
#pragma unroll
        for (int k = 0; k < CPT; ++k) s = fma(a[r][k], zr[k], s);
        s = ski_warp_sum(s);
      }
      if (f.want_aa) {
#pragma unroll
        for (int k = 0; k < CPT; ++k) aa = fma(a[r][k], a[r][k], aa);
      }
      p[r] = s;
    }
    if (lane == 0)
#pragma unroll
      for (int r = 0; r < RR; ++r) {
        red[r][wid] = p[r];
        if (COMP) redc[COMP ? r : 0][wid] = pc[COMP ? r : 0];
      }
    __syncthreads();
    if (tid < RR) {
      const int64_t j = j0 + tid;
      double t = 0.0;
      if (COMP) {
        double s = 0.0, c = 0.0;
#pragma unroll
        for (int q = 0; q < NT / 32; ++q) pair_add(s, c, red[tid][q], redc[COMP ? tid : 0][q]);
        if (j < r1) {
          double h, he;
          two_sum(f.b[j], -s, h, he);
          t = h + (he - c);
          f.t[j] = t;
        }
      } else {
        double dot = 0.0;
#pragma unroll
        for (int q = 0; q < NT / 32; ++q) dot += red[tid][q];
        if (j < r1) {
          t = ca * dot;
          if (f.u) t = fma(cu, f.u[j], t);
          if (f.b) t = fma(cb, f.b[j], t);
          f.t[j] = t;
        }
      }
      tsh[tid] = t;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RR; ++r) {
      const double t = tsh[r];
      if (tid == 0) tt = fma(t, t, tt);
#pragma unroll
      for (int k = 0; k < CPT; ++k) acc[k] = fma(a[r][k], t, acc[k]);
    }
  }
#pragma unroll
  for (int k = 0; k < CPT; ++k) {
    const int64_t c = tid + (int64_t)k * NT;
    if (c < f.d) f.part[(int64_t)blockIdx.x * f.ldp + c] = acc[k];
  }
  __shared__ double sh[NT / 32];
  if (f.want_aa) {
    double s = block_sum(aa, sh);
    if (tid == 0) f.part_aa[blockIdx.x] = s;
  }
  if (tid == 0) f.part_tt[blockIdx.x] = tt;
  if (f.maxexp) {
    emax = __reduce_max_sync(0xffffffffu, emax);
    if (lane == 0) atomicMax(f.maxexp, emax);
  }
}

// CSR pass 1: t_j = ca (A_j z) + cu u_j + cb b_j, warp per row; per-CTA ||t||^2, ||A||_F^2.
__global__ void __launch_bounds__(256) k_csr_rows(FusedArgs f) {
  const LsqrScalars* sc = f.sc;
  if (sc && sc->flag_a) return;
  double ca = f.ca, cu = f.cu, cb = f.cb;
  if (f.coef_from_scalars) {
    ca = 1.0;
    cu = -sc->coef;
    cb = 0.0;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __shared__ double sh_tt[8], sh_aa[8];
  double tt = 0.0, aa = 0.0;
  const int64_t r0 = (int64_t)blockIdx.x * f.rows_per;
  const int64_t r1 = min(f.n, r0 + f.rows_per);
  for (int64_t j = r0 + wid; j < r1; j += 8) {
    double s = 0.0, sa = 0.0, c = 0.0;
    for (int64_t p = f.rowptr[j] + lane; p < f.rowptr[j + 1]; p += 32) {
      const double v = f.val[p];
      if (f.comp)
        dot2_add(v, f.z[f.colidx[p]], s, c);
      else
        s = fma(v, f.z[f.colidx[p]], s);
      sa = fma(v, v, sa);
    }
    if (f.comp)
      pair_warp_sum(s, c);
    else
      s = ski_warp_sum(s);
    if (f.want_aa) aa += ski_warp_sum(sa);
    double t;
    if (f.comp) {
      double h, he;
      two_sum(f.b[j], -s, h, he);
      t = h + (he - c);
    } else {
      t = ca * s;
      if (f.u) t = fma(cu, f.u[j], t);
      if (f.b) t = fma(cb, f.b[j], t);
    }
    if (lane == 0) f.t[j] = t;
    tt = fma(t, t, tt);
  }
  if (lane == 0) {
    sh_tt[wid] = tt;
    sh_aa[wid] = aa;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int q = 0; q < 8; ++q) {
      a += sh_tt[q];
      b += sh_aa[q];
    }
    f.part_tt[blockIdx.x] = a;
    if (f.want_aa) f.part_aa[blockIdx.x] = b;
  }
}

// CSR pass 2: q = A^T t through the CSC copy, warp per column (fixed order).
__global__ void __launch_bounds__(256) k_csc_cols(int64_t d, const int64_t* __restrict__ colptr,
                                                  const int32_t* __restrict__ rowidx, const double* __restrict__ cval,
                                                  const double* __restrict__ t, double* __restrict__ q,
                                                  const LsqrScalars* __restrict__ sc) {
  if (sc && sc->flag_a) return;
  const int lane = threadIdx.x & 31;
  const int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (c >= d) return;
  double s = 0.0;
  for (int64_t p = colptr[c] + lane; p < colptr[c + 1]; p += 32) s = fma(cval[p], t[rowidx[p]], s);
  s = ski_warp_sum(s);
  if (lane == 0) q[c] = s;
}

// q[c] = sum over CTAs of part[blk][c]; CTA 0 also reduces ||t||^2 (and
// ||A||_F^2) into the scalars.
// shard: the row-block form -- ||r||^2 and ||A||_F^2 go to q[d] and q[d+1]
// as this process's partial sums (k_finish_shard derives the scalars after
// the sum over the processes).
__global__ void k_reduce_cols(int nblk, int64_t d, const double* __restrict__ part, int64_t ldp,
                              const double* __restrict__ part_tt, const double* __restrict__ part_aa,
                              double* __restrict__ q, LsqrScalars* __restrict__ sc, int mode, int shard) {
  if (sc->flag_a && mode == 0) return;
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (part && c < d) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * ldp + c];
    q[c] = s;
  }
  if (shard) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      double s = 0.0, a = 0.0;
      for (int b = 0; b < nblk; ++b) s += part_tt[b];
      if (part_aa)
        for (int b = 0; b < nblk; ++b) a += part_aa[b];
      q[d] = s;
      q[d + 1] = a;
    }
    return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part_tt[b];
    sc->beta_new = sqrt(s);  // ||t||: beta of the LSQR step, or ||r|| of a residual pass
    sc->rnorm2 = s;
    if (part_aa) {
      double a = 0.0;
      for (int b = 0; b < nblk; ++b) a += part_aa[b];
      sc->anorm_f2 = a;
    }
  }
}

// ||q|| into sc->atr_norm (one CTA).
__global__ void __launch_bounds__(1024) k_norm(int64_t d, const double* __restrict__ q, LsqrScalars* __restrict__ sc) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t c = threadIdx.x; c < d; c += blockDim.x) s = fma(q[c], q[c], s);
  s = block_sum(s, sh);
  if (threadIdx.x == 0) sc->atr_norm = sqrt(s);
}

// Conjugate gradients on W^T W z = h (adjoint solve), one CTA.  start: r = p
// = h (passed as q), z = 0.  Step: q = W^T W p; alpha = r.r / p.q; z += alpha p;
// r -= alpha q; p = r + (r'.r' / r.r) p; stop when r.r <= tol2 * r0.r0.
__global__ void __launch_bounds__(1024) k_cg(int64_t d, const double* __restrict__ q, double* __restrict__ r,
                                             double* __restrict__ p, double* __restrict__ z,
                                             LsqrScalars* __restrict__ sc, int start) {
  __shared__ double sh[32];
  __shared__ double s_a;
  if (start) {
    double s = 0.0;
    for (int64_t c = threadIdx.x; c < d; c += blockDim.x) {
      const double h = q[c];
      r[c] = h;
      p[c] = h;
      z[c] = 0.0;
      s = fma(h, h, s);
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) {
      sc->cg_rr = s;
      sc->cg_rr0 = s;
      sc->iters = 0;
      sc->flag_a = (s == 0.0) ? 1 : 0;
      sc->conv = sc->flag_a;
    }
    return;
  }
  if (sc->flag_a) return;
  double pq = 0.0;
  for (int64_t c = threadIdx.x; c < d; c += blockDim.x) pq = fma(p[c], q[c], pq);
  pq = block_sum(pq, sh);
  if (threadIdx.x == 0) s_a = pq > 0.0 ? sc->cg_rr / pq : 0.0;
  __syncthreads();
  const double alpha = s_a;
  double rr = 0.0;
  for (int64_t c = threadIdx.x; c < d; c += blockDim.x) {
    z[c] = fma(alpha, p[c], z[c]);
    const double rn = fma(-alpha, q[c], r[c]);
    r[c] = rn;
    rr = fma(rn, rn, rr);
  }
  rr = block_sum(rr, sh);
  const double beta = sc->cg_rr > 0.0 ? rr / sc->cg_rr : 0.0;
  for (int64_t c = threadIdx.x; c < d; c += blockDim.x) p[c] = fma(beta, p[c], r[c]);
  __syncthreads();
  if (threadIdx.x == 0) {
    sc->cg_rr = rr;
    sc->iters += 1;
    const bool conv = rr <= sc->cg_tol2 * sc->cg_rr0 || pq <= 0.0;
    sc->conv = conv ? 1 : 0;
    if (conv || sc->iters >= sc->it_max) sc->flag_a = 1;
  }
}

// dA[j, c] = r_j lam_c - (A lam)_j x_c
__global__ void k_outer(int64_t n, int64_t d, const double* __restrict__ r, const double* __restrict__ lam,
                        const double* __restrict__ al, const double* __restrict__ x, double* __restrict__ dA,
                        int64_t ld) {
  const int64_t j = blockIdx.y;
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n || c >= d) return;
  dA[j * ld + c] = fma(r[j], lam[c], -al[j] * x[c]);
}

template <class T>
__global__ void k_scale(int64_t rows, int64_t cols, T* __restrict__ Y, int64_t ldy, T s) {
  const int64_t j = blockIdx.y;
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j < rows && c < cols) Y[j * ldy + c] *= s;
}

__global__ void k_copy(int64_t n, const double* __restrict__ a, double* __restrict__ b) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = a[i];
}

}  // namespace

// CTAs of a pass over A: one per SM (one wave), and enough that one CTA's rows
// (staged in shared memory by the double-float pass) stay below 16384.
int ski_fused_ctas(int64_t n) {
  const int64_t base = std::min<int64_t>(152, std::max<int64_t>(1, ski_cdiv(n, 16)));
  return (int)std::max<int64_t>(base, ski_cdiv(n, 16384));
}

ski_status ski_fused_launch(const FusedArgs& f0, cudaStream_t st) {
  FusedArgs f = f0;
  if (f.rowptr) {
    if (f.comp && (f.ca != -1.0 || f.cb != 1.0 || f.u || !f.b || f.coef_from_scalars)) return SKI_EINVAL;
    f.rows_per = ski_cdiv(f.n, f.nblk);
    k_csr_rows<<<f.nblk, 256, 0, st>>>(f);
    SKI_LAUNCH_CHECK();
    return SKI_OK;
  }
  f.rows_per = ski_cdiv(f.n, f.nblk);
  const int64_t cpt = ski_cdiv(f.d, 512);
  // the compensated residual is the acceptance pass's alone: r = b - A z
  if (f.comp && (f.ca != -1.0 || f.cb != 1.0 || f.u || !f.b || f.coef_from_scalars)) return SKI_EINVAL;
#define SKI_FUSED_CASE(C, R)                                  \
  if (cpt <= C) {                                             \
    if (f.comp)                                               \
      k_fused_dense<C, R, true><<<f.nblk, 512, 0, st>>>(f);   \
    else                                                      \
      k_fused_dense<C, R, false><<<f.nblk, 512, 0, st>>>(f);  \
    SKI_LAUNCH_CHECK();                                       \
    return SKI_OK;                                            \
  }
  SKI_FUSED_CASE(1, 8)
  SKI_FUSED_CASE(2, 8)
  SKI_FUSED_CASE(4, 4)
  SKI_FUSED_CASE(8, 4)
  SKI_FUSED_CASE(16, 1)
#undef SKI_FUSED_CASE
  return SKI_EINVAL;
}

ski_status ski_trmv_launch(bool upper, int64_t d, const double* M, int64_t ldm, const double* x, const double* add,
                           double* y, const LsqrScalars* sc, cudaStream_t st) {
  const int T = 256;
  const unsigned g = (unsigned)ski_cdiv(d * 32, T);
  if (upper) k_trmv<true><<<g, T, 0, st>>>(d, M, ldm, x, add, y, sc);
  else k_trmv<false><<<g, T, 0, st>>>(d, M, ldm, x, add, y, sc);
  SKI_LAUNCH_CHECK();
  return SKI_OK;
}

ski_status ski_csc_launch(int64_t d, const int64_t* colptr, const int32_t* rowidx, const double* cval,
                          const double* t, double* q, const LsqrScalars* sc, cudaStream_t st) {
  k_csc_cols<<<(unsigned)ski_cdiv(d * 32, 256), 256, 0, st>>>(d, colptr, rowidx, cval, t, q, sc);
  SKI_LAUNCH_CHECK();
  return SKI_OK;
}

ski_status ski_reduce_launch(int nblk, int64_t d, const double* part, int64_t ldp, const double* part_tt,
                             const double* part_aa, double* q, LsqrScalars* sc, int mode, cudaStream_t st,
                             int shard) {
  k_reduce_cols<<<(unsigned)std::max<int64_t>(1, ski_cdiv(d, 256)), 256, 0, st>>>(nblk, d, part, ldp, part_tt, part_aa, q,
                                                                            sc, mode, shard);
  SKI_LAUNCH_CHECK();
  return SKI_OK;
}

namespace {
__global__ void __launch_bounds__(1024) k_norm2(int64_t d, const double* __restrict__ q, const double* __restrict__ x,
                                                LsqrScalars* __restrict__ sc) {
  __shared__ double sh[32];
  double s = 0.0, t = 0.0;
  for (int64_t c = threadIdx.x; c < d; c += blockDim.x) {
    s = fma(q[c], q[c], s);
    if (x) t = fma(x[c], x[c], t);
  }
  s = block_sum(s, sh);
  t = block_sum(t, sh);
  if (threadIdx.x == 0) {
    sc->atr_norm = sqrt(s);
    if (x) sc->xnorm = sqrt(t);
  }
}
}  // namespace

ski_status ski_norm2_launch(int64_t d, const double* q, const double* x, LsqrScalars* sc, cudaStream_t st) {
  k_norm2<<<1, 1024, 0, st>>>(d, q, x, sc);
  SKI_LAUNCH_CHECK();
  return SKI_OK;
}

ski_status ski_norm_launch(int64_t d, const double* q, LsqrScalars* sc, cudaStream_t st) {
  k_norm<<<1, 1024, 0, st>>>(d, q, sc);
  SKI_LAUNCH_CHECK();
  return SKI_OK;
}

ski_status ski_copy_launch(int64_t n, const double* a, double* b, cudaStream_t st) {
  if (n <= 0) return SKI_OK;
  k_copy<<<(unsigned)ski_cdiv(n, 256), 256, 0, st>>>(n, a, b);
  SKI_LAUNCH_CHECK();
  return SKI_OK;
}

ski_status ski_cg_launch(int64_t d, const double* q, double* r, double* p, double* z, LsqrScalars* sc, int start,
                         cudaStream_t st) {
  k_cg<<<1, 1024, 0, st>>>(d, q, r, p, z, sc, start);
  SKI_LAUNCH_CHECK();
  return SKI_OK;
}

ski_status ski_outer_launch(int64_t n, int64_t d, const double* r, const double* lam, const double* al,
                            const double* x, double* dA, int64_t ld_da, cudaStream_t st) {
  for (int64_t j0 = 0; j0 < n; j0 += 65535) {
    const int64_t nr = std::min<int64_t>(65535, n - j0);
    dim3 grid((unsigned)ski_cdiv(d, 256), (unsigned)nr);
    k_outer<<<grid, 256, 0, st>>>(nr, d, r + j0, lam, al + j0, x, dA + j0 * ld_da, ld_da);
    SKI_LAUNCH_CHECK();
  }
  return SKI_OK;
}

ski_status ski_scale_launch(int64_t rows, int64_t cols, double* Y, int64_t ldy, double s, cudaStream_t st) {
  for (int64_t j0 = 0; j0 < rows; j0 += 65535) {
    const int64_t nr = std::min<int64_t>(65535, rows - j0);
    dim3 grid((unsigned)ski_cdiv(cols, 256), (unsigned)nr);
    k_scale<double><<<grid, 256, 0, st>>>(nr, cols, Y + j0 * ldy, ldy, s);
    SKI_LAUNCH_CHECK();
  }
  return SKI_OK;
}

ski_status ski_scale_f32_launch(int64_t rows, int64_t cols, float* Y, int64_t ldy, float s, cudaStream_t st) {
  for (int64_t j0 = 0; j0 < rows; j0 += 65535) {
    const int64_t nr = std::min<int64_t>(65535, rows - j0);
    dim3 grid((unsigned)ski_cdiv(cols, 256), (unsigned)nr);
    k_scale<float><<<grid, 256, 0, st>>>(nr, cols, Y + j0 * ldy, ldy, s);
    SKI_LAUNCH_CHECK();
  }
  return SKI_OK;
}

namespace {
__global__ void k_add_diag(int64_t d, double* __restrict__ R, int64_t ldr, double delta) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < d) R[i * ldr + i] += delta;
}
}  // namespace

ski_status ski_add_diag_launch(int64_t d, double* R, int64_t ldr, double delta, cudaStream_t st) {
  if (d < 1) return SKI_OK;
  k_add_diag<<<(unsigned)ski_cdiv(d, 256), 256, 0, st>>>(d, R, ldr, delta);
  SKI_LAUNCH_CHECK();
  return SKI_OK;
}
