// The LSQR iteration of Step 4 laid out for GB300, whose FP64 pipe issues 2
// DFMA per clock per SM (1/64 of FP32).  A plain FP64 pass over A would be
// bound by those 2 DFMA per element, at 3x the HBM time, so the dense pass
// runs in double-float arithmetic on the FP32 pipe instead:
//
//  * A is copied once per solve into A2 = A * 2^-sA as (hi, lo) float pairs
//    (hi = the leading 24 significant bits, lo = the next 24), 8 bytes per
//    element like FP64: 48 significant bits, scaled so that max|A2| < 1.
//  * products use the error-free transformation p + e = ah * bh (e from an
//    FMA), sums use TwoSum, so every multiply-add keeps ~2^-47 relative
//    accuracy -- far below the 1e-10 acceptance tolerance -- and the only
//    FP64 operations left are per row (t_j) and per column (partials).
//
// One iteration is four launches (no host synchronisation):
//   K2  t = A z - (alpha/beta) t, with per-CTA partials of A^T t and ||t||^2
//   K3  q = A^T t and beta = ||t|| from the partials (fixed order)
//   K4  p = M^T q, v' = p / beta - beta v, per-CTA partials of ||v'||^2
//   K1  alpha = ||v'||, the plane rotation, v = v'/alpha, y and w updates,
//       and z = M v for the next K2; CTA 0 writes the scalars and the
//       Eq. TC-lsqr stop flag.
// Kernels never read a flag written by another CTA of the same launch: K1
// reads flag_b and writes flag_a; K2, K3, K4 read flag_a; K3 copies it to
// flag_b for the next K1.
#include <stdlib.h>

#include <algorithm>

#include "common.cuh"
#include "lsqr_impl.cuh"

namespace {

// ------------------------------------------------ error-free FP32 arithmetic
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (Sh, Sl) += (ah + al) * (bh + bl), dropping al * bl (below 2^-48).
__device__ __forceinline__ void df_mac(float& Sh, float& Sl, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  const float e = __fmaf_rn(ah, bh, -p);
  const float x = __fmaf_rn(ah, bl, __fmul_rn(al, bh));
  float s, err;
  two_sum(Sh, p, s, err);
  Sh = s;
  Sl = __fadd_rn(Sl, __fadd_rn(err, __fadd_rn(e, x)));
}
__device__ __forceinline__ void df_add(float& Sh, float& Sl, float bh, float bl) {
  float s, e;
  two_sum(Sh, bh, s, e);
  Sh = s;
  Sl = __fadd_rn(Sl, __fadd_rn(e, bl));
}
__device__ __forceinline__ void df_warp_sum(float& h, float& l) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, h, o);
    const float ol = __shfl_xor_sync(0xffffffffu, l, o);
    df_add(h, l, oh, ol);
  }
}
// (hi, lo) float pair of x * 2^-s (x FP64): two conversions and one FP64 add.
__device__ __forceinline__ float2 df_split(double x, int s) {
  const double xs = ldexp(x, -s);
  const float h = __double2float_rn(xs);
  const float l = __double2float_rn(xs - (double)h);
  return make_float2(h, l);
}

__device__ __forceinline__ bool flag_set(const volatile int* f) { return *f != 0; }

// A2[j, c] = split(A[j, c] * 2^-sA) using integer operations only: hi keeps
// the top 24 significant bits (exact in FP32), lo the remaining 29 bits
// rounded to 24.  Values below 2^-126 * 2^sA flush to zero.
__global__ void k_split_a(int64_t n, int64_t d, const double* __restrict__ A, int64_t lda, int sA,
                          float2* __restrict__ A2, int64_t ld2, const int32_t* __restrict__ cmap) {
  const int64_t j = blockIdx.y;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < d; c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t src = cmap ? (int64_t)cmap[c] : c;
    const unsigned long long bits = (unsigned long long)__double_as_longlong(A[j * lda + src]);
    const int e = (int)((bits >> 52) & 0x7FF);
    const int es = e - sA;  // biased exponent after scaling by 2^-sA
    float h = 0.f, l = 0.f;
    if (e != 0 && es > 0 && es - 1023 + 127 >= 1) {
      const unsigned long long hb = (bits & 0xFFFFFFFFE0000000ull) - ((unsigned long long)sA << 52);
      h = __double2float_rn(__longlong_as_double((long long)hb));
      const unsigned int low = (unsigned int)(bits & 0x1FFFFFFFull);
      const int le = es - 1075 + 127;  // 2^(es - 1075) as a float exponent field
      if (low != 0 && le >= 1) {
        l = __uint2float_rn(low) * __int_as_float(le << 23);
        if (bits >> 63) l = -l;
      }
    }
    A2[j * ld2 + c] = make_float2(h, l);
  }
}

// K2: double-float fused pass.  Thread tid owns columns tid + k*512 (k < CPT).
// bid: the CTA's row block (blockIdx.x, or a work item's block in the grouped
// form); PF: two row groups in registers, the next one's loads issued before
// this one's reductions (LSQR pass variant 5)
template <int CPT, int RR, bool PF = false>
__device__ __forceinline__ void fused_df_body(const DfArgs& f, int64_t bid) {
  constexpr int NT = 512, NW = NT / 32;
  __shared__ float2 red[RR][NW];
  __shared__ float2 tsh[RR];
  __shared__ int s_zexp;
  LsqrScalars* sc = f.sc;
  if (sc && flag_set(&sc->flag_a)) return;
  const double cu = f.coef_from_scalars ? -sc->coef : f.cu;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  // scale of z: its largest exponent, so that |z * 2^-sz| < 2
  if (tid == 0) s_zexp = -2000;
  __syncthreads();
  int ez = -2000;
#pragma unroll
  for (int k = 0; k < CPT; ++k) {
    const int64_t c = tid + (int64_t)k * NT;
    if (c < f.d) {
      const double zc = f.z[c];
      if (zc != 0.0) ez = max(ez, (int)((__double_as_longlong(zc) >> 52) & 0x7FF) - 1022);
    }
  }
  atomicMax(&s_zexp, ez);
  __syncthreads();
  const int sz = s_zexp == -2000 ? 0 : s_zexp;
  const int st = f.sA + sz;  // t is carried as t * 2^-st
  float zh[CPT], zl[CPT], ah_acc[CPT], al_acc[CPT];
#pragma unroll
  for (int k = 0; k < CPT; ++k) {
    const int64_t c = tid + (int64_t)k * NT;
    const float2 zz = c < f.d ? df_split(f.z[c], sz) : make_float2(0.f, 0.f);
    zh[k] = zz.x;
    zl[k] = zz.y;
    ah_acc[k] = 0.f;
    al_acc[k] = 0.f;
  }
  const int64_t r0 = (int64_t)bid * f.rows_per;
  const int64_t r1 = min(f.n, r0 + f.rows_per);
  // u for this CTA's rows, staged once (off the per-row critical path)
  extern __shared__ double s_u[];
  if (f.u)
    for (int64_t j = r0 + tid; j < r1; j += NT) s_u[j - r0] = f.u[j];
  __syncthreads();
  double tt = 0.0;
  // rows j0 .. j0 + RR - 1 of A2 into registers
  auto load = [&](float2 (&a)[RR][CPT], int64_t j0) {
#pragma unroll
    for (int r = 0; r < RR; ++r)
#pragma unroll
      for (int k = 0; k < CPT; ++k) {
        const int64_t c = tid + (int64_t)k * NT;
        a[r][k] = (j0 + r < r1 && c < f.d) ? __ldcs(&f.A2[(j0 + r) * f.ld2 + c]) : make_float2(0.f, 0.f);
      }
  };
  // one row group: t_j for its rows, then their share of A^T t
  auto process = [&](const float2 (&a)[RR][CPT], int64_t j0) {
#pragma unroll
    for (int r = 0; r < RR; ++r) {
      float h = 0.f, l = 0.f;
#pragma unroll
      for (int k = 0; k < CPT; ++k) df_mac(h, l, a[r][k].x, a[r][k].y, zh[k], zl[k]);
      df_warp_sum(h, l);
      if (lane == 0) red[r][wid] = make_float2(h, l);
    }
    __syncthreads();
    // warp r < RR finishes row j0 + r: tree sum of the 16 warp partials,
    // then t_j in FP64 (one row per warp, all rows in parallel)
    if (wid < RR) {
      const int64_t j = j0 + wid;
      float h = lane < NW ? red[wid][lane].x : 0.f, l = lane < NW ? red[wid][lane].y : 0.f;
#pragma unroll
      for (int o = NW / 2; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, h, o);
        const float ol = __shfl_xor_sync(0xffffffffu, l, o);
        df_add(h, l, oh, ol);
      }
      if (lane == 0) {
        float2 ts = make_float2(0.f, 0.f);
        if (j < r1) {
          double t = ldexp((double)h + (double)l, st);
          if (f.u) t = fma(cu, s_u[j - r0], t);
          f.t[j] = t;
          tt = fma(t, t, tt);
          ts = df_split(t, st);
        }
        tsh[wid] = ts;
      }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RR; ++r) {
      const float2 t = tsh[r];
#pragma unroll
      for (int k = 0; k < CPT; ++k) df_mac(ah_acc[k], al_acc[k], a[r][k].x, a[r][k].y, t.x, t.y);
    }
  };
  if constexpr (!PF) {
    for (int64_t j0 = r0; j0 < r1; j0 += RR) {
      float2 a[RR][CPT];
      load(a, j0);
      process(a, j0);
    }
  } else {
    // two register buffers: the next group's loads are in flight while this
    // group's reductions and barriers run
    float2 a0[RR][CPT], a1[RR][CPT];
    if (r0 < r1) load(a0, r0);
    for (int64_t j0 = r0; j0 < r1; j0 += 2 * RR) {
      if (j0 + RR < r1) load(a1, j0 + RR);
      process(a0, j0);
      if (j0 + RR >= r1) break;
      if (j0 + 2 * RR < r1) load(a0, j0 + 2 * RR);
      process(a1, j0 + RR);
    }
  }
  // partial A^T t of this CTA: (A2 * 2^sA)^T (t2 * 2^st)
#pragma unroll
  for (int k = 0; k < CPT; ++k) {
    const int64_t c = tid + (int64_t)k * NT;
    if (c < f.d) f.part[(int64_t)bid * f.d + c] = ldexp((double)ah_acc[k] + (double)al_acc[k], f.sA + st);
  }
  // ||t||^2: lane 0 of warps < RR hold pieces
  __shared__ double tts[NW];
  if (lane == 0) tts[wid] = tt;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int q = 0; q < RR; ++q) s += tts[q];
    f.part_tt[bid] = s;
  }
}
template <int CPT, int RR>
__global__ void __launch_bounds__(512) k_fused_df(DfArgs f) { fused_df_body<CPT, RR>(f, blockIdx.x); }
template <int CPT, int RR>
__global__ void __launch_bounds__(512) k_fused_df_pf(DfArgs f) { fused_df_body<CPT, RR, true>(f, blockIdx.x); }

// K2, TMA-staged: rows of A2 stream into a shared-memory ring by 1-D bulk
// copies (cp.async.bulk, completion on an mbarrier), one producer thread
// issuing ahead while the 16 warps compute from shared memory -- the loads
// never stall the arithmetic.  Same arithmetic and same result as k_fused_df.
__device__ __forceinline__ uint32_t s_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

template <int CPT, int RR>
__global__ void __launch_bounds__(512, 1) k_fused_df_tma(DfArgs f, int nstage) {
  constexpr int NT = 512, NW = NT / 32;
  constexpr long long kSpin = 1ll << 22;
  __shared__ float2 red[RR][NW];
  __shared__ float2 tsh[RR];
  __shared__ int s_zexp;
  __shared__ double tts[NW];
  __shared__ __align__(8) uint64_t full[4];
  extern __shared__ __align__(128) unsigned char dyn[];
  LsqrScalars* sc = f.sc;
  if (sc && flag_set(&sc->flag_a)) return;
  const double cu = f.coef_from_scalars ? -sc->coef : f.cu;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int64_t r0 = (int64_t)blockIdx.x * f.rows_per;
  const int64_t r1 = min(f.n, r0 + f.rows_per);
  const int64_t rowb = f.ld2 * (int64_t)sizeof(float2);           // bytes per row (multiple of 16)
  float2* ring = reinterpret_cast<float2*>(dyn);                   // [nstage][RR][ld2]
  double* s_u = reinterpret_cast<double*>(dyn + (size_t)nstage * RR * rowb);
  const int64_t ngroups = r1 > r0 ? (r1 - r0 + RR - 1) / RR : 0;
  auto issue = [&](int64_t g) {  // thread 0: bulk copies of group g into stage g % nstage
    const int s = (int)(g % nstage);
    const int64_t j0 = r0 + g * RR;
    const int nr = (int)min((int64_t)RR, r1 - j0);
    const uint32_t bar = s_u32(&full[s]);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                 "r"((uint32_t)(nr * rowb))
                 : "memory");
    for (int r = 0; r < nr; ++r) {
      const uint32_t dst = s_u32(ring + ((size_t)s * RR + r) * f.ld2);
      const float2* src = f.A2 + (j0 + r) * f.ld2;
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       dst),
                   "l"(src), "r"((uint32_t)rowb), "r"(bar)
                   : "memory");
    }
  };
  if (tid == 0) {
    s_zexp = -2000;
    for (int s = 0; s < nstage; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_u32(&full[s])), "r"(1u));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  int64_t issued = 0;  // groups whose copies thread 0 has issued
  if (tid == 0)
    for (; issued < min((int64_t)nstage, ngroups); ++issued) issue(issued);
  if (f.u)
    for (int64_t j = r0 + tid; j < r1; j += NT) s_u[j - r0] = f.u[j];
  int ez = -2000;
#pragma unroll
  for (int k = 0; k < CPT; ++k) {
    const int64_t c = tid + (int64_t)k * NT;
    if (c < f.d) {
      const double zc = f.z[c];
      if (zc != 0.0) ez = max(ez, (int)((__double_as_longlong(zc) >> 52) & 0x7FF) - 1022);
    }
  }
  atomicMax(&s_zexp, ez);
  __syncthreads();
  const int sz = s_zexp == -2000 ? 0 : s_zexp;
  const int st = f.sA + sz;
  float zh[CPT], zl[CPT], ah_acc[CPT], al_acc[CPT];
#pragma unroll
  for (int k = 0; k < CPT; ++k) {
    const int64_t c = tid + (int64_t)k * NT;
    const float2 zz = c < f.d ? df_split(f.z[c], sz) : make_float2(0.f, 0.f);
    zh[k] = zz.x;
    zl[k] = zz.y;
    ah_acc[k] = 0.f;
    al_acc[k] = 0.f;
  }
  double tt = 0.0;
  bool ok = true;
  for (int64_t g = 0; g < ngroups && ok; ++g) {
    const int s = (int)(g % nstage);
    const uint32_t par = (uint32_t)((g / nstage) & 1);
    const int64_t j0 = r0 + g * RR;
    // wait for the group's rows (bounded; the outcome is made CTA-uniform)
    bool got = false;
    for (long long i = 0; i < kSpin; ++i) {
      uint32_t done;
      asm volatile(
          "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(done)
          : "r"(s_u32(&full[s])), "r"(par)
          : "memory");
      if (done) {
        got = true;
        break;
      }
    }
    ok = __syncthreads_and(got) != 0;
    if (!ok) break;
    const float2* rows = ring + (size_t)s * RR * f.ld2;
#pragma unroll
    for (int r = 0; r < RR; ++r) {
      float h = 0.f, l = 0.f;
      if (j0 + r < r1) {
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
          const int64_t c = tid + (int64_t)k * NT;
          if (c < f.d) {
            const float2 a = rows[(size_t)r * f.ld2 + c];
            df_mac(h, l, a.x, a.y, zh[k], zl[k]);
          }
        }
      }
      df_warp_sum(h, l);
      if (lane == 0) red[r][wid] = make_float2(h, l);
    }
    __syncthreads();
    if (wid < RR) {
      const int64_t j = j0 + wid;
      float h = lane < NW ? red[wid][lane].x : 0.f, l = lane < NW ? red[wid][lane].y : 0.f;
#pragma unroll
      for (int o = NW / 2; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, h, o);
        const float ol = __shfl_xor_sync(0xffffffffu, l, o);
        df_add(h, l, oh, ol);
      }
      if (lane == 0) {
        float2 ts = make_float2(0.f, 0.f);
        if (j < r1) {
          double t = ldexp((double)h + (double)l, st);
          if (f.u) t = fma(cu, s_u[j - r0], t);
          f.t[j] = t;
          tt = fma(t, t, tt);
          ts = df_split(t, st);
        }
        tsh[wid] = ts;
      }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RR; ++r) {
      const float2 tv = tsh[r];
      if (j0 + r < r1) {
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
          const int64_t c = tid + (int64_t)k * NT;
          if (c < f.d) {
            const float2 a = rows[(size_t)r * f.ld2 + c];
            df_mac(ah_acc[k], al_acc[k], a.x, a.y, tv.x, tv.y);
          }
        }
      }
    }
    __syncthreads();  // stage s fully consumed before it is refilled
    if (tid == 0 && g + nstage < ngroups) issue(issued++);
  }
  if (!ok) {
    // a bulk copy did not land in time: record it and leave once the copies
    // already issued have completed (bounded wait on each stage's last phase)
    if (tid == 0) {
      atomicExch(&sc->df_err, 1);
      for (int s = 0; s < nstage; ++s) {
        int64_t last = -1;  // last group issued into stage s
        for (int64_t g = s; g < issued; g += nstage) last = g;
        if (last < 0) continue;
        const uint32_t par = (uint32_t)((last / nstage) & 1);
        for (long long i = 0; i < kSpin; ++i) {
          uint32_t done;
          asm volatile(
              "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
              : "=r"(done)
              : "r"(s_u32(&full[s])), "r"(par)
              : "memory");
          if (done) break;
        }
      }
    }
    return;
  }
#pragma unroll
  for (int k = 0; k < CPT; ++k) {
    const int64_t c = tid + (int64_t)k * NT;
    if (c < f.d) f.part[(int64_t)blockIdx.x * f.d + c] = ldexp((double)ah_acc[k] + (double)al_acc[k], f.sA + st);
  }
  if (lane == 0) tts[wid] = tt;
  __syncthreads();
  if (tid == 0) {
    double s2 = 0.0;
    for (int q = 0; q < RR; ++q) s2 += tts[q];
    f.part_tt[blockIdx.x] = s2;
  }
}

// K2, row-per-warp variant: in each group of 16 rows, warp w computes the
// whole dot product of row j0 + w (lanes stride the columns, z staged in
// shared memory), so no CTA barrier sits inside a row; after ONE barrier all
// 512 threads apply the A^T t update of the 16 rows to their own columns,
// re-reading the rows from L1/L2 where the dot phase just brought them.
template <int CPT>
__global__ void __launch_bounds__(512, 1) k_fused_df_rows(DfArgs f) {
  constexpr int NT = 512, NW = NT / 32;
  __shared__ float2 tsh[2][NW];
  __shared__ int s_zexp;
  __shared__ double tts[NW];
  extern __shared__ __align__(128) unsigned char dyn[];
  float2* zs = reinterpret_cast<float2*>(dyn);                            // [ld2]
  double* s_u = reinterpret_cast<double*>(dyn + (size_t)f.ld2 * sizeof(float2));
  LsqrScalars* sc = f.sc;
  if (sc && flag_set(&sc->flag_a)) return;
  const double cu = f.coef_from_scalars ? -sc->coef : f.cu;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int64_t r0 = (int64_t)blockIdx.x * f.rows_per;
  const int64_t r1 = min(f.n, r0 + f.rows_per);
  if (tid == 0) s_zexp = -2000;
  if (f.u)
    for (int64_t j = r0 + tid; j < r1; j += NT) s_u[j - r0] = f.u[j];
  __syncthreads();
  int ez = -2000;
  for (int64_t c = tid; c < f.d; c += NT) {
    const double zc = f.z[c];
    if (zc != 0.0) ez = max(ez, (int)((__double_as_longlong(zc) >> 52) & 0x7FF) - 1022);
  }
  atomicMax(&s_zexp, ez);
  __syncthreads();
  const int sz = s_zexp == -2000 ? 0 : s_zexp;
  const int st = f.sA + sz;
  for (int64_t c = tid; c < f.d; c += NT) zs[c] = df_split(f.z[c], sz);
  float ah_acc[CPT], al_acc[CPT];
#pragma unroll
  for (int k = 0; k < CPT; ++k) {
    ah_acc[k] = 0.f;
    al_acc[k] = 0.f;
  }
  __syncthreads();
  double tt = 0.0;
  int buf = 0;
  for (int64_t j0 = r0; j0 < r1; j0 += NW, buf ^= 1) {
    // dot phase: one row per warp
    const int64_t j = j0 + wid;
    if (j < r1) {
      const float2* row = f.A2 + j * f.ld2;
      float h = 0.f, l = 0.f;
#pragma unroll 4
      for (int64_t c = lane; c < f.d; c += 32) {
        const float2 a = __ldcg(&row[c]);
        const float2 z = zs[c];
        df_mac(h, l, a.x, a.y, z.x, z.y);
      }
      df_warp_sum(h, l);
      if (lane == 0) {
        double t = ldexp((double)h + (double)l, st);
        if (f.u) t = fma(cu, s_u[j - r0], t);
        f.t[j] = t;
        tt = fma(t, t, tt);
        tsh[buf][wid] = df_split(t, st);
      }
    } else if (lane == 0) {
      tsh[buf][wid] = make_float2(0.f, 0.f);
    }
    __syncthreads();
    // update phase: every thread, its columns, the group's rows
    const int nr = (int)min((int64_t)NW, r1 - j0);
    for (int r = 0; r < nr; ++r) {
      const float2 tv = tsh[buf][r];
      const float2* row = f.A2 + (j0 + r) * f.ld2;
#pragma unroll
      for (int k = 0; k < CPT; ++k) {
        const int64_t c = tid + (int64_t)k * NT;
        if (c < f.d) {
          const float2 a = row[c];
          df_mac(ah_acc[k], al_acc[k], a.x, a.y, tv.x, tv.y);
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < CPT; ++k) {
    const int64_t c = tid + (int64_t)k * NT;
    if (c < f.d) f.part[(int64_t)blockIdx.x * f.d + c] = ldexp((double)ah_acc[k] + (double)al_acc[k], f.sA + st);
  }
  if (lane == 0) tts[wid] = tt;
  __syncthreads();
  if (tid == 0) {
    double s2 = 0.0;
    for (int q = 0; q < NW; ++q) s2 += tts[q];
    f.part_tt[blockIdx.x] = s2;
  }
}

// K3: q[c] = sum_b part[b][c] (8 warps share the CTAs, fixed order), beta;
// CTA 0 also copies flag_a to flag_b for the next K1 (also once stopped).
// shard: the row-block form -- q and ||t||^2 (in q[d]) are this process's
// partial sums, to be summed over the processes before k_finish_shard
// derives the scalars; a finished iteration (flag_a) contributes zeros.
__device__ __forceinline__ void reduce_par_body(int nblk, int64_t d, const double* __restrict__ part,
                                                const double* __restrict__ part_tt, double* __restrict__ q,
                                                LsqrScalars* __restrict__ sc, int shard, int64_t bid) {
  __shared__ double sh[8][33];
  const bool skip = sc && flag_set(&sc->flag_a);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (!skip) {
    const int64_t c = (int64_t)bid * 32 + lane;
    double s = 0.0;
    if (part && c < d)
      for (int b = wid; b < nblk; b += 8) s += part[(int64_t)b * d + c];
    sh[wid][lane] = s;
    __syncthreads();
    if (wid == 0) {
      double t = 0.0;
#pragma unroll
      for (int w = 0; w < 8; ++w) t += sh[w][lane];
      if (part && c < d) q[c] = t;
    }
  } else if (shard && part) {
    const int64_t c = (int64_t)bid * 32 + lane;
    if (wid == 0 && c < d) q[c] = 0.0;
  }
  if (shard) {
    if (bid == 0 && wid == 1) {
      double t = 0.0;
      if (!skip) {
        for (int b = lane; b < nblk; b += 32) t += part_tt[b];
        t = ski_warp_sum(t);
      }
      if (lane == 0) q[d] = t;
    }
    return;
  }
  if (bid == 0 && wid == 1 && sc) {
    double t = 0.0;
    if (!skip) {
      for (int b = lane; b < nblk; b += 32) t += part_tt[b];
      t = ski_warp_sum(t);
    }
    if (lane == 0) {
      if (!skip) {
        sc->beta_new = sqrt(t);
        sc->rnorm2 = t;
      }
      sc->flag_b = sc->flag_a;
      // snapshot of the rotation state for the next K1 (see LsqrScalars)
      sc->r_alpha = sc->alpha;
      sc->r_rhobar = sc->rhobar;
      sc->r_phibar = sc->phibar;
      sc->r_anorm2 = sc->anorm2;
      sc->r_iters = sc->iters;
    }
  }
}
__global__ void __launch_bounds__(256) k_reduce_par(int nblk, int64_t d, const double* __restrict__ part,
                                                    const double* __restrict__ part_tt, double* __restrict__ q,
                                                    LsqrScalars* __restrict__ sc, int shard) {
  reduce_par_body(nblk, d, part, part_tt, q, sc, shard, blockIdx.x);
}

// K4: p = M^T q (Mt lower triangular, warp per row), v' = p/beta - beta v
// (start: v' = p/beta), per-CTA partial ||v'||^2.
__device__ __forceinline__ void trmv_lower_vp_body(int64_t d, const double* __restrict__ Mt,
                                                   const double* __restrict__ q, const double* __restrict__ v,
                                                   double* __restrict__ vp, double* __restrict__ part_vv,
                                                   LsqrScalars* __restrict__ sc, int start, int64_t bid) {
  __shared__ double sv[8];
  if (!start && flag_set(&sc->flag_a)) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t row = (int64_t)bid * 8 + wid;
  const double beta = sc->beta_new;
  double vv = 0.0;
  if (row < d) {
    const double* mr = Mt + row * d;
    double acc = row_dot8(mr, q, lane, row + 1);
    acc = ski_warp_sum(acc);
    const double ib = beta > 0.0 ? 1.0 / beta : 0.0;
    double x = acc * ib;
    if (!start) x = fma(-beta, v[row], x);
    if (lane == 0) vp[row] = x;
    vv = x * x;
  }
  if (lane == 0) sv[wid] = vv;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) s += sv[w];
    part_vv[bid] = s;
  }
}
__global__ void __launch_bounds__(256) k_trmv_lower_vp(int64_t d, const double* __restrict__ Mt,
                                                       const double* __restrict__ q, const double* __restrict__ v,
                                                       double* __restrict__ vp, double* __restrict__ part_vv,
                                                       LsqrScalars* __restrict__ sc, int start) {
  trmv_lower_vp_body(d, Mt, q, v, vp, part_vv, sc, start, blockIdx.x);
}

// K1: alpha = ||v'|| from the K4 partials, LSQR rotation, v/y/w updates for
// this CTA's rows, z = M v for the next pass.  Warp per row.
__device__ __forceinline__ void trmv_upper_update_body(int64_t d, const double* __restrict__ M,
                                                       const double* __restrict__ vp, int nvv,
                                                       const double* __restrict__ part_vv, double* __restrict__ v,
                                                       double* __restrict__ w, double* __restrict__ y,
                                                       double* __restrict__ z, LsqrScalars* __restrict__ sc,
                                                       int start, int64_t bid) {
  __shared__ double s_par[4];  // 1/alpha, c1, c2, done
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (!start && flag_set(&sc->flag_b)) return;
  if (wid == 0) {
    double s = 0.0;
    for (int b = lane; b < nvv; b += 32) s += part_vv[b];
    s = ski_warp_sum(s);
    if (lane == 0) {
      const double alpha = sqrt(s);
      const double ia = alpha > 0.0 ? 1.0 / alpha : 0.0;
      const double beta = sc->beta_new;
      double c1 = 0.0, c2 = 0.0;
      int done = 0;
      if (start) {
        done = (alpha * beta == 0.0) ? 1 : 0;
        if (bid == 0) {
          sc->alpha = alpha;
          sc->beta = beta;
          sc->phibar = beta;
          sc->rhobar = alpha;
          sc->anorm2 = 0.0;
          sc->test = 1.0;
          sc->coef = beta > 0.0 ? alpha / beta : 0.0;
          sc->iters = 0;
          sc->conv = done;
          sc->flag_a = done;
          sc->flag_b = done;
        }
      } else {
        // old state from the K3 snapshot: CTA 0 overwrites sc->alpha etc. below
        const double alpha_old = sc->r_alpha, rhobar = sc->r_rhobar, phibar_old = sc->r_phibar;
        const double rho = hypot(rhobar, beta);
        const double cs = rhobar / rho, sn = beta / rho;
        const double theta = sn * alpha;
        const double phi = cs * phibar_old;
        const double phibar = sn * phibar_old;
        c1 = phi / rho;
        c2 = theta / rho;
        const double anorm2 = sc->r_anorm2 + alpha_old * alpha_old + beta * beta;
        const double test = (anorm2 > 0.0 && phibar > 0.0) ? alpha * fabs(cs) / sqrt(anorm2) : 0.0;
        const long long iters = sc->r_iters + 1;
        const bool conv = test <= sc->tau_r || alpha == 0.0 || beta == 0.0;
        done = (conv || iters >= sc->it_max) ? 1 : 0;
        if (bid == 0) {
          sc->anorm2 = anorm2;
          sc->rhobar = -cs * alpha;
          sc->phibar = phibar;
          sc->alpha = alpha;
          sc->beta = beta;
          sc->coef = beta > 0.0 ? alpha / beta : 0.0;
          sc->test = test;
          sc->iters = iters;
          sc->conv = conv ? 1 : 0;
          sc->flag_a = done;
        }
      }
      s_par[0] = ia;
      s_par[1] = c1;
      s_par[2] = c2;
      s_par[3] = done;
    }
  }
  __syncthreads();
  const double ia = s_par[0], c1 = s_par[1], c2 = s_par[2];
  const bool done = s_par[3] != 0.0;
  const int64_t row = (int64_t)bid * 8 + wid;
  if (row >= d) return;
  if (lane == 0) {
    const double vn = vp[row] * ia;
    v[row] = vn;
    if (start) {
      w[row] = vn;
      y[row] = 0.0;
    } else {
      const double wc = w[row];
      y[row] = fma(c1, wc, y[row]);
      w[row] = fma(-c2, wc, vn);
    }
  }
  if (done) return;
  const double* mr = M + row * d;
  double acc = row_dot8(mr, vp, row + lane, d);
  acc = ski_warp_sum(acc);
  if (lane == 0) z[row] = acc * ia;
}
__global__ void __launch_bounds__(256) k_trmv_upper_update(int64_t d, const double* __restrict__ M,
                                                           const double* __restrict__ vp, int nvv,
                                                           const double* __restrict__ part_vv, double* __restrict__ v,
                                                           double* __restrict__ w, double* __restrict__ y,
                                                           double* __restrict__ z, LsqrScalars* __restrict__ sc,
                                                           int start) {
  trmv_upper_update_body(d, M, vp, nvv, part_vv, v, w, y, z, sc, start, blockIdx.x);
}

// ---- grouped form: one launch per kernel for every problem in flight
template <int CPT, int RR, bool PF>
__global__ void __launch_bounds__(512) k_group_df(const LsqrGroupJob* __restrict__ jobs,
                                                  const LsqrGroupItem* __restrict__ items) {
  const LsqrGroupItem it = items[blockIdx.x];
  fused_df_body<CPT, RR, PF>(jobs[it.job].df, it.blk);
}
__global__ void __launch_bounds__(256) k_group_reduce(const LsqrGroupJob* __restrict__ jobs,
                                                      const LsqrGroupItem* __restrict__ items) {
  const LsqrGroupItem it = items[blockIdx.x];
  const LsqrGroupJob& J = jobs[it.job];
  reduce_par_body(J.df.nblk, J.d, J.df.part, J.df.part_tt, J.q, J.df.sc, 0, it.blk);
}
// K4 then K1 need the whole of K4 (part_vv): two launches over the same items
__global__ void __launch_bounds__(256) k_group_trmv_lower(const LsqrGroupJob* __restrict__ jobs,
                                                          const LsqrGroupItem* __restrict__ items) {
  const LsqrGroupItem it = items[blockIdx.x];
  const LsqrGroupJob& J = jobs[it.job];
  trmv_lower_vp_body(J.d, J.Mt, J.q, J.v, J.vp, J.part_vv, J.df.sc, 0, it.blk);
}
__global__ void __launch_bounds__(256) k_group_trmv_upper(const LsqrGroupJob* __restrict__ jobs,
                                                          const LsqrGroupItem* __restrict__ items) {
  const LsqrGroupItem it = items[blockIdx.x];
  const LsqrGroupJob& J = jobs[it.job];
  trmv_upper_update_body(J.d, J.M, J.vp, J.nvv, J.part_vv, J.v, J.w, J.y, J.z, J.df.sc, 0, it.blk);
}
__global__ void k_group_scalars(const LsqrGroupJob* __restrict__ jobs, int njobs, LsqrScalars* __restrict__ out) {
  constexpr int W = sizeof(LsqrScalars) / sizeof(int);
  static_assert(sizeof(LsqrScalars) % sizeof(int) == 0, "LsqrScalars is copied as words");
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)njobs * W;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / W), k = (int)(e % W);
    ((int*)(out + j))[k] = ((const volatile int*)jobs[j].df.sc)[k];
  }
}

}  // namespace

// Classes of the register-blocked pass as ski_fused_df_launch picks it by
// default (the same rows per group, so the same summation order): columns per
// thread 1, 2, 4 with twice the rows, 8 with prefetch, 16
int ski_df_group_class(int64_t d) {
  const int64_t cpt = ski_cdiv(d, 512);
  return cpt <= 1 ? 0 : cpt <= 2 ? 1 : cpt <= 4 ? 2 : cpt <= 8 ? 3 : 4;
}

ski_status ski_group_df_launch(int cls, const LsqrGroupJob* jobs, const LsqrGroupItem* items, int nitems,
                               size_t smem, cudaStream_t st) {
  if (nitems <= 0) return SKI_OK;
  if (smem > 200 * 1024) return SKI_EINVAL;
#define SKI_GDF_CASE(K, C, R, P)                                                                   \
  if (cls == K) {                                                                                  \
    if (smem > 48 * 1024)                                                                          \
      SKI_CUDA_TRY(ski_attr_once((const void*)k_group_df<C, R, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                        [&] { return ski_smem_cap((const void*)k_group_df<C, R, P>); }));          \
    k_group_df<C, R, P><<<(unsigned)nitems, 512, smem, st>>>(jobs, items);                         \
    SKI_LAUNCH_CHECK();                                                                            \
    return SKI_OK;                                                                                 \
  }
  SKI_GDF_CASE(0, 1, 16, false)
  SKI_GDF_CASE(1, 2, 16, false)
  SKI_GDF_CASE(2, 4, 8, false)
  SKI_GDF_CASE(3, 8, 2, true)
  SKI_GDF_CASE(4, 16, 1, false)
#undef SKI_GDF_CASE
  return SKI_EINVAL;
}

ski_status ski_group_reduce_launch(const LsqrGroupJob* jobs, const LsqrGroupItem* items, int nitems,
                                   cudaStream_t st) {
  if (nitems <= 0) return SKI_OK;
  k_group_reduce<<<(unsigned)nitems, 256, 0, st>>>(jobs, items);
  SKI_LAUNCH_CHECK();
  return SKI_OK;
}

ski_status ski_group_trmv_launch(const LsqrGroupJob* jobs, const LsqrGroupItem* items, int nitems,
                                 cudaStream_t st) {
  if (nitems <= 0) return SKI_OK;
  k_group_trmv_lower<<<(unsigned)nitems, 256, 0, st>>>(jobs, items);
  SKI_LAUNCH_CHECK();
  k_group_trmv_upper<<<(unsigned)nitems, 256, 0, st>>>(jobs, items);
  SKI_LAUNCH_CHECK();
  return SKI_OK;
}

ski_status ski_group_scalars_launch(const LsqrGroupJob* jobs, int njobs, LsqrScalars* out, cudaStream_t st) {
  if (njobs <= 0) return SKI_OK;
  k_group_scalars<<<(unsigned)std::min<int64_t>(64, ski_cdiv((int64_t)njobs * 64, 256)), 256, 0, st>>>(jobs, njobs,
                                                                                                      out);
  SKI_LAUNCH_CHECK();
  return SKI_OK;
}

ski_status ski_split_a_launch(int64_t n, int64_t d, const double* A, int64_t lda, int sA, float2* A2, cudaStream_t st,
                              const int32_t* cmap) {
  const int64_t ld2 = ski_a2_ld(d);
  for (int64_t j0 = 0; j0 < n; j0 += 65535) {
    const int64_t nr = std::min<int64_t>(65535, n - j0);
    dim3 grid((unsigned)std::min<int64_t>(ski_cdiv(d, 256), 16), (unsigned)nr);
    k_split_a<<<grid, 256, 0, st>>>(nr, d, A + j0 * lda, lda, sA, A2 + j0 * ld2, ld2, cmap);
    SKI_LAUNCH_CHECK();
  }
  return SKI_OK;
}

bool ski_df_supported(int64_t d) { return d <= SKI_DENSE_DMAX; }

int64_t ski_a2_ld(int64_t d) { return ski_round_up(d, 2); }  // rows 16-byte aligned

// Variant of the LSQR pass (DfArgs.variant, from ski_opts.lsqr_pass): the
// register-blocked kernel (k_fused_df, 0 and 1) measured fastest at
// 50000 x 4000 (0.55 ms per iteration against 0.68 for the TMA-staged ring (2)
// and 0.75 for row per warp (3)); the autotuner times them per shape.
ski_status ski_fused_df_launch(const DfArgs& f0, cudaStream_t st) {
  DfArgs f = f0;
  f.ld2 = ski_a2_ld(f.d);
  f.rows_per = ski_cdiv(f.n, f.nblk);
  const int64_t cpt = ski_cdiv(f.d, 512);
  // row-per-warp variant (z and u staged in shared memory)
  {
    const size_t sm = (size_t)f.ld2 * sizeof(float2) + (size_t)f.rows_per * sizeof(double);
    if (sm <= 200 * 1024 && f.variant == 3) {
#define SKI_DFR_CASE(C)                                                                                  \
      if (cpt <= C) {                                                                                    \
        SKI_CUDA_TRY(ski_attr_once((const void*)k_fused_df_rows<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                                          [&] { return ski_smem_cap((const void*)k_fused_df_rows<C>); }));               \
        k_fused_df_rows<C><<<f.nblk, 512, sm, st>>>(f);                                                  \
        SKI_LAUNCH_CHECK();                                                                              \
        return SKI_OK;                                                                                   \
      }
      SKI_DFR_CASE(1)
      SKI_DFR_CASE(2)
      SKI_DFR_CASE(4)
      SKI_DFR_CASE(8)
#undef SKI_DFR_CASE
    }
  }
  // TMA-staged variant: nstage x RR rows of A2 in shared memory
  if (f.variant == 2) {
    const size_t rowb = (size_t)f.ld2 * sizeof(float2);
    const size_t ub = (size_t)f.rows_per * sizeof(double);
    const size_t budget = 200 * 1024;
#define SKI_DFT_CASE(C, R)                                                                            \
    if (cpt <= C) {                                                                                   \
      for (int ns = 3; ns >= 2; --ns) {                                                               \
        const size_t sm = (size_t)ns * R * rowb + ub;                                                 \
        if (sm <= budget) {                                                                           \
          SKI_CUDA_TRY(ski_attr_once((const void*)k_fused_df_tma<C, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                            [&] { return ski_smem_cap((const void*)k_fused_df_tma<C, R>); }));        \
          k_fused_df_tma<C, R><<<f.nblk, 512, sm, st>>>(f, ns);                                       \
          SKI_LAUNCH_CHECK();                                                                         \
          return SKI_OK;                                                                              \
        }                                                                                             \
      }                                                                                               \
    }
    SKI_DFT_CASE(1, 8)
    SKI_DFT_CASE(2, 4)
    SKI_DFT_CASE(4, 4)
    SKI_DFT_CASE(8, 2)
#undef SKI_DFT_CASE
  }
  const size_t smem = (size_t)f.rows_per * sizeof(double);
  if (smem > 200 * 1024) return SKI_EINVAL;
#define SKI_DF_CASE(C, R)                                                                        \
  if (cpt <= C) {                                                                                \
    if (smem > 48 * 1024)                                                                        \
      SKI_CUDA_TRY(ski_attr_once((const void*)k_fused_df<C, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                        [&] { return ski_smem_cap((const void*)k_fused_df<C, R>); }));           \
    k_fused_df<C, R><<<f.nblk, 512, smem, st>>>(f);                                              \
    SKI_LAUNCH_CHECK();                                                                          \
    return SKI_OK;                                                                               \
  }
  // variant 5: prefetching form (two register buffers of RR rows); the auto
  // choice for d in (2048, 4096], where it was measured fastest (LSQR stage of
  // 50000 x 4000: 33.3 -> 32.1 ms; 200000 x 4000: 111.2 -> 108.1 ms)
  if (f.variant == 5 || (f.variant == 0 && cpt > 4 && cpt <= 8)) {
#define SKI_DFP_CASE(C, R)                                                                       \
    if (cpt <= C) {                                                                              \
      if (smem > 48 * 1024)                                                                      \
        SKI_CUDA_TRY(ski_attr_once((const void*)k_fused_df_pf<C, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                          [&] { return ski_smem_cap((const void*)k_fused_df_pf<C, R>); }));      \
      k_fused_df_pf<C, R><<<f.nblk, 512, smem, st>>>(f);                                         \
      SKI_LAUNCH_CHECK();                                                                        \
      return SKI_OK;                                                                             \
    }
    SKI_DFP_CASE(1, 8)
    SKI_DFP_CASE(2, 4)
    SKI_DFP_CASE(4, 2)
    SKI_DFP_CASE(8, 2)
#undef SKI_DFP_CASE
  }
  // auto: twice the rows per row group for d <= 2048, where it was measured
  // faster (LSQR stage of 50000 x 2000: 26.0 -> 19.5 ms; 30000 x 1000: 10.1 ->
  // 9.7 ms)
  if (f.variant == 4 || (f.variant == 0 && cpt <= 4)) {  // twice the rows between the two barriers of a row group
    SKI_DF_CASE(1, 16)
    SKI_DF_CASE(2, 16)
    SKI_DF_CASE(4, 8)
    SKI_DF_CASE(8, 4)
  }
  SKI_DF_CASE(1, 8)
  SKI_DF_CASE(2, 8)
  SKI_DF_CASE(4, 4)
  SKI_DF_CASE(8, 2)
  SKI_DF_CASE(16, 1)
#undef SKI_DF_CASE
  return SKI_EINVAL;
}

ski_status ski_reduce_par_launch(int nblk, int64_t d, const double* part, const double* part_tt, double* q,
                                 LsqrScalars* sc, cudaStream_t st, int shard) {
  k_reduce_par<<<(unsigned)std::max<int64_t>(1, ski_cdiv(d, 32)), 256, 0, st>>>(nblk, d, part, part_tt, q, sc, shard);
  SKI_LAUNCH_CHECK();
  return SKI_OK;
}

namespace {
// After the sum over the processes of a row-block form's partials q[0..d),
// q[d] = ||t||^2 (and q[d+1] = ||A||_F^2 of a residual pass): the scalars
// k_reduce_par (mode 0) or k_reduce_cols (mode 2) derive from them.
__global__ void k_finish_shard(const double* __restrict__ q, int64_t d, LsqrScalars* __restrict__ sc, int mode,
                               int want_aa) {
  if (threadIdx.x != 0) return;
  if (mode == 0) {
    if (!flag_set(&sc->flag_a)) {
      sc->beta_new = sqrt(q[d]);
      sc->rnorm2 = q[d];
    }
    sc->flag_b = sc->flag_a;
    sc->r_alpha = sc->alpha;
    sc->r_rhobar = sc->rhobar;
    sc->r_phibar = sc->phibar;
    sc->r_anorm2 = sc->anorm2;
    sc->r_iters = sc->iters;
  } else {
    sc->beta_new = sqrt(q[d]);
    sc->rnorm2 = q[d];
    if (want_aa) sc->anorm_f2 = q[d + 1];
  }
}
}  // namespace

ski_status ski_finish_shard_launch(const double* q, int64_t d, LsqrScalars* sc, int mode, int want_aa,
                                   cudaStream_t st) {
  k_finish_shard<<<1, 32, 0, st>>>(q, d, sc, mode, want_aa);
  SKI_LAUNCH_CHECK();
  return SKI_OK;
}

int ski_vv_blocks(int64_t d) { return (int)ski_cdiv(d, 8); }

ski_status ski_trmv_lower_vp_launch(int64_t d, const double* Mt, const double* q, const double* v, double* vp,
                                    double* part_vv, LsqrScalars* sc, int start, cudaStream_t st) {
  k_trmv_lower_vp<<<(unsigned)ski_vv_blocks(d), 256, 0, st>>>(d, Mt, q, v, vp, part_vv, sc, start);
  SKI_LAUNCH_CHECK();
  return SKI_OK;
}

ski_status ski_trmv_upper_update_launch(int64_t d, const double* M, const double* vp, const double* part_vv,
                                        double* v, double* w, double* y, double* z, LsqrScalars* sc, int start,
                                        cudaStream_t st) {
  k_trmv_upper_update<<<(unsigned)ski_vv_blocks(d), 256, 0, st>>>(d, M, vp, ski_vv_blocks(d), part_vv, v, w, y, z,
                                                                    sc, start);
  SKI_LAUNCH_CHECK();
  return SKI_OK;
}
