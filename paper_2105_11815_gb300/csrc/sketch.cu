// Step 1 of Algorithm 1: the s-hashing sketch [S A | S b] (Def. 5).
//
// S is never formed.  For every column j of S (row j of A) the s rows it
// hits are drawn from the counter hash (hash.cuh).  The sketch is computed as
// a deterministic gather: the (row j, nonzero k) pairs are bucketed by their
// target row i of SA (count, scan, fill, canonical sort inside each bucket),
// then row i of SA is formed from the rows of A listed in bucket i.
//
// FP64 output: every output element is accumulated in exact int64 block
// fixed point (FxAcc, common.cuh) -- integer adds on the INT32 pipe instead
// of FP64 adds, which on GB300 would cost more than the HBM traffic.
// FP32 / BF16 output: FP32 accumulation of FP64 loads converted to FP32.
#include "common.cuh"
#include "hash.cuh"
#include "sketch_impl.cuh"

// ------------------------------------------------------------ hash tables
template <int SMAX>
__global__ void k_hash_table(uint64_t kb, uint64_t ks, int s, uint64_t m, int64_t n, int replace, int32_t* idx,
                             int8_t* sign) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n) return;
  int32_t rows[SMAX];
  int neg[SMAX];
  ski_column<SMAX>(kb, ks, s, m, (uint64_t)j, replace, rows, neg);
  for (int k = 0; k < s; ++k) {
    idx[j * s + k] = rows[k];
    sign[j * s + k] = neg[k] ? (int8_t)-1 : (int8_t)1;
  }
}

__global__ void k_premix_signs(uint64_t kd, int64_t n, int8_t* D) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j < n) D[j] = ski_premix_neg(kd, (uint64_t)j) ? (int8_t)-1 : (int8_t)1;
}

// Count pass: draw the column, store its (row, sign) pairs, count per bucket.
template <int SMAX>
__global__ void k_bucket_count(uint64_t kb, uint64_t ks, int s, uint64_t m, int64_t n, int replace, int64_t row0,
                               int32_t* __restrict__ pair_row, uint8_t* __restrict__ pair_neg,
                               int32_t* __restrict__ counts) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n) return;
  int32_t rows[SMAX];
  int neg[SMAX];
  // the draw of column row0 + j of S: a row block of a larger A keeps its rows' columns of S
  ski_column<SMAX>(kb, ks, s, m, (uint64_t)(row0 + j), replace, rows, neg);
  for (int k = 0; k < s; ++k) {
    pair_row[j * s + k] = rows[k];
    pair_neg[j * s + k] = (uint8_t)neg[k];
    atomicAdd(&counts[rows[k]], 1);
  }
}

// Exclusive scan of counts[0..m) into offsets[0..m], one CTA of 1024 threads.
__global__ void k_scan_counts(const int32_t* __restrict__ counts, int64_t m, int64_t* __restrict__ offsets) {
  __shared__ int64_t warp_tot[32];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t base = 0; base < m; base += blockDim.x) {
    int64_t i = base + threadIdx.x;
    int64_t v = i < m ? counts[i] : 0;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int64_t w = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      warp_tot[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    int64_t before = carry + (wid ? warp_tot[wid - 1] : 0) + x - v;
    if (i < m) offsets[i] = before;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = before + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) offsets[m] = carry;
}

// Fill pass: entry = (j << 1) | neg, placed at offsets[row] + cursor.
__global__ void k_bucket_fill(int s, int64_t n, const int32_t* __restrict__ pair_row,
                              const uint8_t* __restrict__ pair_neg, const int64_t* __restrict__ offsets,
                              int32_t* __restrict__ cursor, uint32_t* __restrict__ list) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n * s) return;
  int32_t r = pair_row[p];
  int32_t pos = atomicAdd(&cursor[r], 1);
  list[offsets[r] + pos] = ((uint32_t)(p / s) << 1) | (uint32_t)pair_neg[p];
}

// Canonical order inside each bucket (ascending entry), so that the sketch is
// bit-reproducible whatever order the fill's atomics took.  One warp per
// bucket: rank sort, O(K^2 / 32) per bucket.  Entries are distinct for
// s-hashing; the variant can repeat one (same j and sign twice), and equal
// entries take consecutive ranks in list order (they are interchangeable).
__global__ void k_bucket_sort(int64_t m, const int64_t* __restrict__ offsets, const uint32_t* __restrict__ list_in,
                              uint32_t* __restrict__ list_out) {
  int64_t bkt = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (bkt >= m) return;
  int64_t lo = offsets[bkt], hi = offsets[bkt + 1];
  int64_t K = hi - lo;
  for (int64_t a = lane; a < K; a += 32) {
    uint32_t v = list_in[lo + a];
    int64_t rank = 0;
    for (int64_t c = 0; c < K; ++c) {
      const uint32_t w = list_in[lo + c];
      rank += (w < v) | ((w == v) & (c < a));
    }
    list_out[lo + rank] = v;
  }
}

// ------------------------------------------------------------ dense gather
// Lean exact accumulator for the gather: block exponent E only ever rises
// (a rare branch), every addend costs ~20 integer instructions.  The
// caller bounds |S| by calling renorm() every 4 addends (each < 2^55).
struct FxGather {
  long long S;
  int E;  // biased exponent field of the largest addend so far (>= 1)
  bool bad;
  __device__ __forceinline__ void init() { S = 0; E = 1; bad = false; }
  __device__ __forceinline__ void add(double v, unsigned neg) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned hi = (unsigned)(b >> 32);
    int e = (int)((hi >> 20) & 0x7FF);
    if (e > E) {
      if (e == 0x7FF) bad = true;
      const int sh = e - E;
      S = sh > 62 ? (S < 0 ? -1 : 0) : (S >> sh);
      E = e;
    }
    const unsigned long long M = (b & 0xFFFFFFFFFFFFFull) | (e ? (1ull << 52) : 0ull);
    const int sh = E - (e ? e : 1);
    const long long q = sh > 63 ? 0ll : (long long)((M << FX_LIFT) >> sh);
    const long long mask = -(long long)((hi >> 31) ^ neg);
    S += (q ^ mask) - mask;
  }
  __device__ __forceinline__ void renorm() {
    if (S >= (1ll << 60) || S <= -(1ll << 60)) {
      S >>= 4;
      E += 4;
    }
  }
};

__device__ __forceinline__ double fxg_scaled(const FxGather& a, long long c, int e) {
  if (a.bad) return __longlong_as_double(0x7FF8000000000000ll);
  const long long Sp = (long long)(((__int128)a.S * (__int128)c) >> 62);
  return fx_to_double(Sp, a.E, e);
}

// Row i of SA, columns c0 + k*128 (k < 4): sum over the bucket's entries
// (j, neg) of (-1)^neg * X[j, c] (X = [A | b]), times `scale`.
template <class TOUT>
__global__ void __launch_bounds__(128) k_sketch_dense_f64acc(
    const double* __restrict__ A, int64_t lda, int64_t nrows, int64_t d, const double* __restrict__ b,
    const int64_t* __restrict__ offsets, const uint32_t* __restrict__ list, long long scale_c, int scale_e,
    TOUT* __restrict__ SA, int64_t ld_sa, int64_t m) {
  constexpr int CPT = 4, BPC = 4;  // columns per thread, buckets per CTA
  const int64_t ncols = d + (b != nullptr);
  const int64_t cb = (int64_t)blockIdx.y * (CPT * 128) + threadIdx.x;
  const int64_t cfirst = (int64_t)blockIdx.y * (CPT * 128);
  const int64_t ccount = max((int64_t)0, min((int64_t)(CPT * 128), d - cfirst));
  const int64_t i0 = (int64_t)blockIdx.x * BPC;
  // bulk L2 prefetch of this CTA's column chunk of every row of bucket i
  auto prefetch = [&](int64_t i) {
    if (i >= m || ccount == 0) return;
    const int64_t lo = offsets[i], hi = offsets[i + 1];
    for (int64_t e = lo + threadIdx.x / 8; e < hi; e += 16) {
      const int64_t j = list[e] >> 1;
      ski_l2_prefetch_range(A + j * lda + cfirst, (size_t)ccount * sizeof(double), threadIdx.x & 7, 8);
    }
  };
  prefetch(i0);
  for (int bi = 0; bi < BPC; ++bi) {
    const int64_t i = i0 + bi;
    if (i >= m) break;
    prefetch(i + 1);
    const int64_t lo = offsets[i], hi = offsets[i + 1];
    FxGather acc[CPT];
#pragma unroll
    for (int k = 0; k < CPT; ++k) acc[k].init();
    int64_t e = lo;
    for (; e + 4 <= hi; e += 4) {
      uint32_t en[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) en[u] = __ldg(&list[e + u]);
      double v[4][CPT];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t j = en[u] >> 1;
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
          const int64_t c = cb + k * 128;
          v[u][k] = c < d ? __ldcs(&A[j * lda + c]) : (c == d && b ? __ldg(&b[j]) : 0.0);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int k = 0; k < CPT; ++k) acc[k].add(v[u][k], en[u] & 1u);
#pragma unroll
      for (int k = 0; k < CPT; ++k) acc[k].renorm();
    }
    for (; e < hi; ++e) {
      const uint32_t en = __ldg(&list[e]);
      const int64_t j = en >> 1;
#pragma unroll
      for (int k = 0; k < CPT; ++k) {
        const int64_t c = cb + k * 128;
        const double v = c < d ? __ldcs(&A[j * lda + c]) : (c == d && b ? __ldg(&b[j]) : 0.0);
        acc[k].add(v, en & 1u);
      }
    }
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
      const int64_t c = cb + k * 128;
      if (c < ncols) SA[i * ld_sa + c] = SkiType<TOUT>::from(fxg_scaled(acc[k], scale_c, scale_e));
    }
  }
  (void)nrows;
}

template <class TOUT>
__global__ void __launch_bounds__(128) k_sketch_dense_f32acc(
    const double* __restrict__ A, int64_t lda, int64_t d, const double* __restrict__ b,
    const int64_t* __restrict__ offsets, const uint32_t* __restrict__ list, float scale,
    TOUT* __restrict__ SA, int64_t ld_sa) {
  const int64_t i = blockIdx.x;
  const int64_t ncols = d + (b != nullptr);
  const int64_t c0 = (int64_t)blockIdx.y * (2 * blockDim.x) + threadIdx.x;
  const int64_t c1 = c0 + blockDim.x;
  const int64_t lo = offsets[i], hi = offsets[i + 1];
  float s0 = 0.f, s1 = 0.f;
  for (int64_t e = lo; e < hi; ++e) {
    uint32_t en = __ldg(&list[e]);
    int64_t j = en >> 1;
    float v0 = c0 < d ? (float)__ldcs(&A[j * lda + c0]) : (c0 == d && b ? (float)__ldg(&b[j]) : 0.f);
    float v1 = c1 < d ? (float)__ldcs(&A[j * lda + c1]) : (c1 == d && b ? (float)__ldg(&b[j]) : 0.f);
    if (en & 1) { v0 = -v0; v1 = -v1; }
    s0 += v0;
    s1 += v1;
  }
  if (c0 < ncols) SA[i * ld_sa + c0] = SkiType<TOUT>::from((double)(s0 * scale));
  if (c1 < ncols) SA[i * ld_sa + c1] = SkiType<TOUT>::from((double)(s1 * scale));
}

// Same gather reading an FP32 matrix Y (the FP32 premix output).
template <class TOUT>
__global__ void __launch_bounds__(128) k_sketch_dense_f32in(
    const float* __restrict__ Y, int64_t ldy, int64_t ncols, const int64_t* __restrict__ offsets,
    const uint32_t* __restrict__ list, float scale, TOUT* __restrict__ SA, int64_t ld_sa) {
  const int64_t i = blockIdx.x;
  const int64_t c0 = (int64_t)blockIdx.y * (2 * blockDim.x) + threadIdx.x;
  const int64_t c1 = c0 + blockDim.x;
  const int64_t lo = offsets[i], hi = offsets[i + 1];
  float s0 = 0.f, s1 = 0.f;
  for (int64_t e = lo; e < hi; ++e) {
    uint32_t en = __ldg(&list[e]);
    int64_t j = en >> 1;
    float v0 = c0 < ncols ? __ldcs(&Y[j * ldy + c0]) : 0.f;
    float v1 = c1 < ncols ? __ldcs(&Y[j * ldy + c1]) : 0.f;
    if (en & 1) { v0 = -v0; v1 = -v1; }
    s0 += v0;
    s1 += v1;
  }
  if (c0 < ncols) SA[i * ld_sa + c0] = SkiType<TOUT>::from((double)(s0 * scale));
  if (c1 < ncols) SA[i * ld_sa + c1] = SkiType<TOUT>::from((double)(s1 * scale));
}

// Exact sum of block-fixed-point addends q * 2^x (|q| < 2^62, x per addend)
// with an adaptive block exponent, as FxGather but without an FP64 decode:
// each addend gives up its 4 low bits for headroom, a larger x shifts the
// running sum down once, and |S| >= 2^61 coarsens the block by 2^4.
struct FxQ {
  long long S;
  int E;
  __device__ __forceinline__ void init() { S = 0; E = -(1 << 30); }
  __device__ __forceinline__ void add(long long q, int x, unsigned neg) {
    if (q == 0) return;
    q >>= 4;
    x += 4;
    if (x > E) {
      const int sh = x - E;
      S = sh > 62 ? (S < 0 ? -1 : 0) : (S >> sh);
      E = x;
    }
    const int sh = E - x;
    const long long v = sh > 62 ? (q < 0 ? -1 : 0) : (q >> sh);
    S += neg ? -v : v;
  }
  __device__ __forceinline__ void renorm() {
    if (S >= (1ll << 61) || S <= -(1ll << 61)) {
      S >>= 4;
      E += 4;
    }
  }
};

// scale * S * 2^(E - yshift) with scale = c * 2^(-62 - e)
__device__ __forceinline__ double fxq_scaled(const FxQ& a, long long c, int e, int yshift) {
  if (a.S == 0) return 0.0;
  const long long Sp = (long long)(((__int128)a.S * (__int128)c) >> 62);
  return fx_i64_to_double(Sp, a.E - yshift - e);
}

// Hash gather over the premix output in block-fixed-point form (SkiPremixQ):
// the layout and work split of k_sketch_dense_f64acc (4 buckets per CTA, 4
// columns per thread, bulk L2 prefetch of the next bucket's rows).
__global__ void __launch_bounds__(128) k_sketch_q_f64acc(
    const long long* __restrict__ Q, int64_t ldq, const int16_t* __restrict__ X, int64_t ldx, int lo, int nb,
    int yshift, int64_t ncols, const int64_t* __restrict__ offsets, const uint32_t* __restrict__ list,
    long long scale_c, int scale_e, double* __restrict__ SA, int64_t ld_sa, int64_t m) {
  constexpr int CPT = 4, BPC = 4;
  const int64_t cb = (int64_t)blockIdx.y * (CPT * 128) + threadIdx.x;
  const int64_t cfirst = (int64_t)blockIdx.y * (CPT * 128);
  const int64_t ccount = max((int64_t)0, min((int64_t)(CPT * 128), ncols - cfirst));
  const int64_t i0 = (int64_t)blockIdx.x * BPC;
  const int64_t lomask = (1ll << lo) - 1;
  auto tile_of = [&](int64_t j) { return ((j >> (lo + nb)) << lo) | (j & lomask); };
  auto prefetch = [&](int64_t i) {
    if (i >= m || ccount == 0) return;
    const int64_t lo_e = offsets[i], hi_e = offsets[i + 1];
    for (int64_t e = lo_e + threadIdx.x / 8; e < hi_e; e += 16) {
      const int64_t j = list[e] >> 1;
      ski_l2_prefetch_range(Q + j * ldq + cfirst, (size_t)ccount * sizeof(long long), threadIdx.x & 7, 8);
    }
  };
  prefetch(i0);
  for (int bi = 0; bi < BPC; ++bi) {
    const int64_t i = i0 + bi;
    if (i >= m) break;
    prefetch(i + 1);
    const int64_t lo_e = offsets[i], hi_e = offsets[i + 1];
    FxQ acc[CPT];
#pragma unroll
    for (int k = 0; k < CPT; ++k) acc[k].init();
    int64_t e = lo_e;
    for (; e + 4 <= hi_e; e += 4) {
      uint32_t en[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) en[u] = __ldg(&list[e + u]);
      long long v[4][CPT];
      int x[4][CPT];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t j = en[u] >> 1;
        const int64_t tj = tile_of(j);
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
          const int64_t c = cb + k * 128;
          const bool ok = c < ncols;
          v[u][k] = ok ? __ldcs(&Q[j * ldq + c]) : 0ll;
          x[u][k] = ok ? (int)__ldg(&X[tj * ldx + c]) : 0;
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int k = 0; k < CPT; ++k) acc[k].add(v[u][k], x[u][k], en[u] & 1u);
#pragma unroll
      for (int k = 0; k < CPT; ++k) acc[k].renorm();
    }
    for (; e < hi_e; ++e) {
      const uint32_t en = __ldg(&list[e]);
      const int64_t j = en >> 1;
      const int64_t tj = tile_of(j);
#pragma unroll
      for (int k = 0; k < CPT; ++k) {
        const int64_t c = cb + k * 128;
        if (c < ncols) acc[k].add(__ldcs(&Q[j * ldq + c]), (int)__ldg(&X[tj * ldx + c]), en & 1u);
      }
#pragma unroll
      for (int k = 0; k < CPT; ++k) acc[k].renorm();
    }
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
      const int64_t c = cb + k * 128;
      if (c < ncols) SA[i * ld_sa + c] = fxq_scaled(acc[k], scale_c, scale_e, yshift);
    }
  }
}

// Exact sum of column-aligned addends (|q| < 2^55, one exponent per column):
// plain int64 adds; |S| >= 2^61 coarsens the sum by 2^4 (later addends are
// shifted to match), so any number of addends is safe.
struct FxA {
  long long S;
  int E;
  __device__ __forceinline__ void init() { S = 0; E = 0; }
  __device__ __forceinline__ void add(long long q, unsigned neg) {
    const long long v = q >> E;
    S += neg ? -v : v;
  }
  __device__ __forceinline__ void renorm() {
    if (S >= (1ll << 61) || S <= -(1ll << 61)) {
      S >>= 4;
      E += 4;
    }
  }
};

// Column c of SA (m rows) := NaN where nf[c] is set, or everywhere when *err
// is (a bounded wait of the premix gave up: the sketch is incomplete, and the
// asynchronous entry points report it through SA).
__global__ void __launch_bounds__(256) k_poison_columns(double* __restrict__ SA, int64_t ld_sa, int64_t m,
                                                        int64_t ncols, const int* __restrict__ nf,
                                                        const int* __restrict__ err) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncols || !(nf[c] || (err && *err))) return;
  for (int64_t i = 0; i < m; ++i) SA[i * ld_sa + c] = __longlong_as_double(0x7FF8000000000000ll);
}

// Hash gather over the column-aligned premix output (SkiPremixQ with ecol):
// the layout and work split of k_sketch_dense_f64acc, with 8 addends per
// renormalisation check and no per-addend exponent.
__global__ void __launch_bounds__(128) k_sketch_qa_f64acc(
    const long long* __restrict__ Q, int64_t ldq, const int* __restrict__ ecol, int headroom, int yshift,
    int64_t ncols, const int64_t* __restrict__ offsets, const uint32_t* __restrict__ list, long long scale_c,
    int scale_e, double* __restrict__ SA, int64_t ld_sa, int64_t m) {
  constexpr int CPT = 4, BPC = 4, U = 8;
  const int64_t cb = (int64_t)blockIdx.y * (CPT * 128) + threadIdx.x;
  const int64_t cfirst = (int64_t)blockIdx.y * (CPT * 128);
  const int64_t ccount = max((int64_t)0, min((int64_t)(CPT * 128), ncols - cfirst));
  const int64_t i0 = (int64_t)blockIdx.x * BPC;
  auto prefetch = [&](int64_t i) {
    if (i >= m || ccount == 0) return;
    const int64_t lo_e = offsets[i], hi_e = offsets[i + 1];
    for (int64_t e = lo_e + threadIdx.x / 8; e < hi_e; e += 16) {
      const int64_t j = list[e] >> 1;
      ski_l2_prefetch_range(Q + j * ldq + cfirst, (size_t)ccount * sizeof(long long), threadIdx.x & 7, 8);
    }
  };
  int ec[CPT];
#pragma unroll
  for (int k = 0; k < CPT; ++k) {
    const int64_t c = cb + k * 128;
    ec[k] = c < ncols ? __ldg(&ecol[c]) : 0;
  }
  prefetch(i0);
  for (int bi = 0; bi < BPC; ++bi) {
    const int64_t i = i0 + bi;
    if (i >= m) break;
    prefetch(i + 1);
    const int64_t lo_e = offsets[i], hi_e = offsets[i + 1];
    FxA acc[CPT];
#pragma unroll
    for (int k = 0; k < CPT; ++k) acc[k].init();
    int64_t e = lo_e;
    for (; e + U <= hi_e; e += U) {
      uint32_t en[U];
#pragma unroll
      for (int u = 0; u < U; ++u) en[u] = __ldg(&list[e + u]);
      long long v[U][CPT];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t j = en[u] >> 1;
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
          const int64_t c = cb + k * 128;
          v[u][k] = c < ncols ? __ldcs(&Q[j * ldq + c]) : 0ll;
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int k = 0; k < CPT; ++k) acc[k].add(v[u][k], en[u] & 1u);
#pragma unroll
      for (int k = 0; k < CPT; ++k) acc[k].renorm();
    }
    for (; e < hi_e; ++e) {
      const uint32_t en = __ldg(&list[e]);
      const int64_t j = en >> 1;
#pragma unroll
      for (int k = 0; k < CPT; ++k) {
        const int64_t c = cb + k * 128;
        if (c < ncols) acc[k].add(__ldcs(&Q[j * ldq + c]), en & 1u);
      }
    }
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
      const int64_t c = cb + k * 128;
      if (c < ncols) {
        double r = 0.0;
        if (acc[k].S != 0) {
          const long long Sp = (long long)(((__int128)acc[k].S * (__int128)scale_c) >> 62);
          r = fx_i64_to_double(Sp, acc[k].E + ec[k] + headroom - yshift - scale_e);
        }
        SA[i * ld_sa + c] = r;
      }
    }
  }
}

// Gather of a narrow column slab (ncols <= 32 * CPT) of the premix output:
// warp w of the CTA owns bucket blockIdx.x * 8 + w, lane l its columns
// l + 32 k.  The slab of Y was written just before by the premix and is still
// in L2, so rows are read with default caching.
template <int CPT, class TOUT>
__global__ void __launch_bounds__(256) k_sketch_slab_f64acc(
    const double* __restrict__ Y, int64_t ldy, int64_t ncols, const int64_t* __restrict__ offsets,
    const uint32_t* __restrict__ list, long long scale_c, int scale_e, TOUT* __restrict__ SA, int64_t ld_sa,
    int64_t m) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (i >= m) return;
  const int64_t lo = offsets[i], hi = offsets[i + 1];
  FxGather acc[CPT];
#pragma unroll
  for (int k = 0; k < CPT; ++k) acc[k].init();
  int64_t e = lo;
  for (; e + 4 <= hi; e += 4) {
    uint32_t en[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) en[u] = __ldg(&list[e + u]);
    double v[4][CPT];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const double* row = Y + (int64_t)(en[u] >> 1) * ldy;
#pragma unroll
      for (int k = 0; k < CPT; ++k) {
        const int64_t c = lane + 32 * k;
        v[u][k] = c < ncols ? __ldg(&row[c]) : 0.0;
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int k = 0; k < CPT; ++k) acc[k].add(v[u][k], en[u] & 1u);
#pragma unroll
    for (int k = 0; k < CPT; ++k) acc[k].renorm();
  }
  for (; e < hi; ++e) {
    const uint32_t en = __ldg(&list[e]);
    const double* row = Y + (int64_t)(en >> 1) * ldy;
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
      const int64_t c = lane + 32 * k;
      acc[k].add(c < ncols ? __ldg(&row[c]) : 0.0, en & 1u);
    }
  }
#pragma unroll
  for (int k = 0; k < CPT; ++k) {
    const int64_t c = lane + 32 * k;
    if (c < ncols) SA[i * ld_sa + c] = SkiType<TOUT>::from(fxg_scaled(acc[k], scale_c, scale_e));
  }
}

template <int CPT, class TOUT>
__global__ void __launch_bounds__(256) k_sketch_slab_f32in(
    const float* __restrict__ Y, int64_t ldy, int64_t ncols, const int64_t* __restrict__ offsets,
    const uint32_t* __restrict__ list, float scale, TOUT* __restrict__ SA, int64_t ld_sa, int64_t m) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (i >= m) return;
  const int64_t lo = offsets[i], hi = offsets[i + 1];
  float s[CPT];
#pragma unroll
  for (int k = 0; k < CPT; ++k) s[k] = 0.f;
  for (int64_t e = lo; e < hi; ++e) {
    const uint32_t en = __ldg(&list[e]);
    const float* row = Y + (int64_t)(en >> 1) * ldy;
    const float sg = (en & 1u) ? -1.f : 1.f;
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
      const int64_t c = lane + 32 * k;
      s[k] += c < ncols ? sg * __ldg(&row[c]) : 0.f;
    }
  }
#pragma unroll
  for (int k = 0; k < CPT; ++k) {
    const int64_t c = lane + 32 * k;
    if (c < ncols) SA[i * ld_sa + c] = SkiType<TOUT>::from((double)(s[k] * scale));
  }
}

// ------------------------------------------------------------ CSR gather
// Row i of SA for a CSR A: SA is zeroed first (a bandwidth-bound memset of the
// dense m x (d+1) output, the dominant traffic), then warp i scatters the
// nonzeros of bucket i's rows into row i of SA, one source row after another
// (__syncwarp between rows orders the read-modify-writes), so the summation
// order is fixed and no atomics are needed.  Column indices within one CSR
// row must be distinct.  Each SA entry receives few addends (about
// s * nnz / (m d) on average), so FP32 / BF16 outputs are accumulated in place.
template <class TOUT>
__global__ void __launch_bounds__(256) k_sketch_csr(
    const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colidx, const double* __restrict__ val,
    int64_t d, const double* __restrict__ b, const int64_t* __restrict__ offsets,
    const uint32_t* __restrict__ list, double scale, TOUT* __restrict__ SA, int64_t ld_sa, int64_t m) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (i >= m) return;
  TOUT* out = SA + i * ld_sa;
  const int64_t lo = offsets[i], hi = offsets[i + 1];
  double bacc = 0.0;
  for (int64_t e = lo; e < hi; ++e) {
    const uint32_t en = __ldg(&list[e]);
    const int64_t j = en >> 1;
    const double sg = (en & 1u) ? -scale : scale;
    const int64_t p0 = __ldg(&rowptr[j]), p1 = __ldg(&rowptr[j + 1]);
    for (int64_t p = p0 + lane; p < p1; p += 32) {
      const int32_t c = __ldg(&colidx[p]);
      const double v = sg * __ldg(&val[p]);
      out[c] = SkiType<TOUT>::from(SkiType<TOUT>::to_f64(out[c]) + v);
    }
    if (b && lane == 0) bacc += sg * __ldg(&b[j]);
    __syncwarp();
  }
  if (b && lane == 0) out[d] = SkiType<TOUT>::from(bacc);
}

// ------------------------------------------------------------ host side
static void scale_fixed(double scale, long long* c, int* e) {
  // scale = c * 2^(-62 - e) with c in [2^61, 2^62): the integer multiplier of fx_scaled.
  int ex;
  double f = frexp(scale, &ex);  // scale = f * 2^ex, f in [0.5, 1)
  *c = (long long)ldexp(f, 62);
  *e = -ex;
}

size_t ski_bucket_ws_bytes(int64_t nrows, int32_t s, int64_t m) {
  SkiArena ar{nullptr, 0, 0, true};
  ar.take<int32_t>(nrows * s);
  ar.take<uint8_t>(nrows * s);
  ar.take<int32_t>(m);
  ar.take<int32_t>(m);
  ar.take<int64_t>(m + 1);
  ar.take<uint32_t>(nrows * s);
  ar.take<uint32_t>(nrows * s);
  return ar.off;
}

ski_status ski_build_buckets(uint64_t seed, int32_t s, int32_t replace, int64_t m, int64_t nrows, SkiArena& ar,
                             cudaStream_t st, SkiBuckets* out, int64_t row0) {
  int32_t* pair_row = ar.take<int32_t>(nrows * s);
  uint8_t* pair_neg = ar.take<uint8_t>(nrows * s);
  int32_t* counts = ar.take<int32_t>(m);
  int32_t* cursor = ar.take<int32_t>(m);
  int64_t* offsets = ar.take<int64_t>(m + 1);
  uint32_t* tmp = ar.take<uint32_t>(nrows * s);
  uint32_t* list = ar.take<uint32_t>(nrows * s);
  if (!ar.ok() || !list) return SKI_ENOMEM;
  uint64_t kb = ski_tag_base(seed, SKI_TAG_BUCKET), ks = ski_tag_base(seed, SKI_TAG_SIGN);
  SKI_CUDA_TRY(cudaMemsetAsync(counts, 0, m * sizeof(int32_t), st));
  SKI_CUDA_TRY(cudaMemsetAsync(cursor, 0, m * sizeof(int32_t), st));
  const int T = 256;
  if (nrows > 0) {
    if (s <= 4)
      k_bucket_count<4><<<ski_cdiv(nrows, T), T, 0, st>>>(kb, ks, s, m, nrows, replace, row0, pair_row, pair_neg,
                                                           counts);
    else
      k_bucket_count<64><<<ski_cdiv(nrows, T), T, 0, st>>>(kb, ks, s, m, nrows, replace, row0, pair_row, pair_neg,
                                                            counts);
    SKI_LAUNCH_CHECK();
  }
  k_scan_counts<<<1, 1024, 0, st>>>(counts, m, offsets);
  SKI_LAUNCH_CHECK();
  if (nrows > 0) {
    k_bucket_fill<<<ski_cdiv(nrows * s, T), T, 0, st>>>(s, nrows, pair_row, pair_neg, offsets, cursor, tmp);
    SKI_LAUNCH_CHECK();
    k_bucket_sort<<<ski_cdiv(m * 32, T), T, 0, st>>>(m, offsets, tmp, list);
    SKI_LAUNCH_CHECK();
  }
  out->offsets = offsets;
  out->list = list;
  out->m = m;
  return SKI_OK;
}

ski_status ski_gather_dense(const double* A, int64_t lda, int64_t nrows, int64_t d, const double* b,
                            const SkiBuckets& bk, double scale, int32_t out_dtype, void* SA, int64_t ld_sa,
                            cudaStream_t st) {
  const int T = 128;
  const int64_t ncols = d + (b != nullptr);
  dim3 grid((unsigned)bk.m, (unsigned)ski_cdiv(ncols, 2 * T));
  if (out_dtype == SKI_F64) {
    long long c;
    int e;
    scale_fixed(scale, &c, &e);
    dim3 grid64((unsigned)ski_cdiv(bk.m, 4), (unsigned)ski_cdiv(ncols, 4 * T));
    k_sketch_dense_f64acc<double><<<grid64, T, 0, st>>>(A, lda, nrows, d, b, bk.offsets, bk.list, c, e,
                                                       (double*)SA, ld_sa, bk.m);
  } else if (out_dtype == SKI_F32) {
    k_sketch_dense_f32acc<float><<<grid, T, 0, st>>>(A, lda, d, b, bk.offsets, bk.list, (float)scale,
                                                     (float*)SA, ld_sa);
  } else {
    k_sketch_dense_f32acc<__nv_bfloat16><<<grid, T, 0, st>>>(A, lda, d, b, bk.offsets, bk.list, (float)scale,
                                                             (__nv_bfloat16*)SA, ld_sa);
  }
  SKI_LAUNCH_CHECK();
  return SKI_OK;
}

ski_status ski_gather_dense_f32in(const float* Y, int64_t ldy, int64_t ncols, const SkiBuckets& bk,
                                  double scale, int32_t out_dtype, void* SA, int64_t ld_sa, cudaStream_t st) {
  const int T = 128;
  dim3 grid((unsigned)bk.m, (unsigned)ski_cdiv(ncols, 2 * T));
  if (out_dtype == SKI_F32)
    k_sketch_dense_f32in<float><<<grid, T, 0, st>>>(Y, ldy, ncols, bk.offsets, bk.list, (float)scale,
                                                    (float*)SA, ld_sa);
  else
    k_sketch_dense_f32in<__nv_bfloat16><<<grid, T, 0, st>>>(Y, ldy, ncols, bk.offsets, bk.list, (float)scale,
                                                            (__nv_bfloat16*)SA, ld_sa);
  SKI_LAUNCH_CHECK();
  return SKI_OK;
}

ski_status ski_gather_q(const SkiPremixQ& y, int64_t ncols, const SkiBuckets& bk, double scale, double* SA,
                        int64_t ld_sa, cudaStream_t st) {
  long long c;
  int e;
  scale_fixed(scale, &c, &e);
  dim3 grid((unsigned)ski_cdiv(bk.m, 4), (unsigned)ski_cdiv(ncols, 4 * 128));
  if (!y.X)
    k_sketch_qa_f64acc<<<grid, 128, 0, st>>>(y.Q, y.ldq, y.ecol, y.headroom, y.yshift, ncols, bk.offsets, bk.list, c,
                                              e, SA, ld_sa, bk.m);
  else
    k_sketch_q_f64acc<<<grid, 128, 0, st>>>(y.Q, y.ldq, y.X, y.ldx, y.lo, y.nb, y.yshift, ncols, bk.offsets, bk.list,
                                             c, e, SA, ld_sa, bk.m);
  SKI_LAUNCH_CHECK();
  // the integer path cannot carry a NaN or Inf: columns flagged by the premix become NaN
  k_poison_columns<<<(unsigned)ski_cdiv(ncols, 256), 256, 0, st>>>(SA, ld_sa, bk.m, ncols, y.nonfinite, y.err);
  SKI_LAUNCH_CHECK();
  return SKI_OK;
}

ski_status ski_gather_slab(const void* Y, int32_t y_dtype, int64_t ldy, int64_t ncols, const SkiBuckets& bk,
                           double scale, int32_t out_dtype, void* SA, int64_t ld_sa, cudaStream_t st) {
  if (ncols < 1 || ncols > 128) return SKI_EINVAL;
  const int cpt = (int)ski_cdiv(ncols, 32);
  const unsigned grid = (unsigned)ski_cdiv(bk.m, 8);
  if (y_dtype == SKI_F64) {
    if (out_dtype != SKI_F64) return SKI_EINVAL;
    long long c;
    int e;
    scale_fixed(scale, &c, &e);
    const double* y = (const double*)Y;
    double* sa = (double*)SA;
    switch (cpt) {
      case 1: k_sketch_slab_f64acc<1, double><<<grid, 256, 0, st>>>(y, ldy, ncols, bk.offsets, bk.list, c, e, sa, ld_sa, bk.m); break;
      case 2: k_sketch_slab_f64acc<2, double><<<grid, 256, 0, st>>>(y, ldy, ncols, bk.offsets, bk.list, c, e, sa, ld_sa, bk.m); break;
      case 3: k_sketch_slab_f64acc<3, double><<<grid, 256, 0, st>>>(y, ldy, ncols, bk.offsets, bk.list, c, e, sa, ld_sa, bk.m); break;
      default: k_sketch_slab_f64acc<4, double><<<grid, 256, 0, st>>>(y, ldy, ncols, bk.offsets, bk.list, c, e, sa, ld_sa, bk.m); break;
    }
  } else {
    const float* y = (const float*)Y;
    const float sc = (float)scale;
#define SKI_SLAB32(CP)                                                                                       \
  if (out_dtype == SKI_F32)                                                                                  \
    k_sketch_slab_f32in<CP, float><<<grid, 256, 0, st>>>(y, ldy, ncols, bk.offsets, bk.list, sc, (float*)SA, \
                                                         ld_sa, bk.m);                                       \
  else                                                                                                       \
    k_sketch_slab_f32in<CP, __nv_bfloat16><<<grid, 256, 0, st>>>(y, ldy, ncols, bk.offsets, bk.list, sc,    \
                                                                 (__nv_bfloat16*)SA, ld_sa, bk.m);
    switch (cpt) {
      case 1: SKI_SLAB32(1) break;
      case 2: SKI_SLAB32(2) break;
      case 3: SKI_SLAB32(3) break;
      default: SKI_SLAB32(4) break;
    }
#undef SKI_SLAB32
  }
  SKI_LAUNCH_CHECK();
  return SKI_OK;
}

ski_status ski_gather_csr(const ski_matrix* A, const double* b, const SkiBuckets& bk, double scale,
                          int32_t out_dtype, void* SA, int64_t ld_sa, cudaStream_t st) {
  const size_t esz = out_dtype == SKI_F64 ? 8 : (out_dtype == SKI_F32 ? 4 : 2);
  SKI_CUDA_TRY(cudaMemsetAsync(SA, 0, (size_t)bk.m * (size_t)ld_sa * esz, st));
  const unsigned grid = (unsigned)ski_cdiv(bk.m, 8);
  if (out_dtype == SKI_F64)
    k_sketch_csr<double><<<grid, 256, 0, st>>>(A->rowptr, A->colidx, A->val, A->d, b, bk.offsets, bk.list, scale,
                                               (double*)SA, ld_sa, bk.m);
  else if (out_dtype == SKI_F32)
    k_sketch_csr<float><<<grid, 256, 0, st>>>(A->rowptr, A->colidx, A->val, A->d, b, bk.offsets, bk.list, scale,
                                              (float*)SA, ld_sa, bk.m);
  else
    k_sketch_csr<__nv_bfloat16><<<grid, 256, 0, st>>>(A->rowptr, A->colidx, A->val, A->d, b, bk.offsets, bk.list,
                                                      scale, (__nv_bfloat16*)SA, ld_sa, bk.m);
  SKI_LAUNCH_CHECK();
  return SKI_OK;
}

static ski_status hash_indices(uint64_t seed, int32_t s, int replace, int64_t m, int64_t n, int32_t* idx,
                               int8_t* sign, void* stream) {
  if (s < 1 || m < (replace ? 1 : s) || m >= (1ll << 31) || n < 0 || s > 64) return SKI_EINVAL;
  if (n == 0) return SKI_OK;
  if (!idx || !sign) return SKI_EINVAL;
  uint64_t kb = ski_tag_base(seed, SKI_TAG_BUCKET), ks = ski_tag_base(seed, SKI_TAG_SIGN);
  const int T = 256;
  if (s <= 4)
    k_hash_table<4><<<ski_cdiv(n, T), T, 0, ski_stream(stream)>>>(kb, ks, s, (uint64_t)m, n, replace, idx, sign);
  else
    k_hash_table<64><<<ski_cdiv(n, T), T, 0, ski_stream(stream)>>>(kb, ks, s, (uint64_t)m, n, replace, idx, sign);
  SKI_LAUNCH_CHECK();
  return SKI_OK;
}

extern "C" ski_status ski_hash_indices(uint64_t seed, int32_t s, int64_t m, int64_t n, int32_t* idx,
                                       int8_t* sign, void* stream) {
  return hash_indices(seed, s, 0, m, n, idx, sign, stream);
}

extern "C" ski_status ski_hash_variant_indices(uint64_t seed, int32_t s, int64_t m, int64_t n, int32_t* idx,
                                               int8_t* sign, void* stream) {
  return hash_indices(seed, s, 1, m, n, idx, sign, stream);
}

extern "C" ski_status ski_premix_signs(uint64_t seed, int64_t n, int8_t* D, void* stream) {
  if (n < 0) return SKI_EINVAL;
  if (n == 0) return SKI_OK;
  if (!D) return SKI_EINVAL;
  const int T = 256;
  k_premix_signs<<<ski_cdiv(n, T), T, 0, ski_stream(stream)>>>(ski_tag_base(seed, SKI_TAG_PREMIX), n, D);
  SKI_LAUNCH_CHECK();
  return SKI_OK;
}
