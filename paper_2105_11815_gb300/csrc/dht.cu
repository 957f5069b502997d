// Randomised discrete Hartley premix F D (Section 6, Eq. HR-DHT) and the
// row-sampling sketch S_s of Eq. SR-DHT, for dense A.
//
// F is the normalised DHT of length N >= n applied to [D A; 0] down every
// column: (F x)_k = N^{-1/2} sum_j x_j cas(2 pi j k / N), cas = cos + sin.
// N = n when the prime factors of n are all at most 13 (every size of the
// paper's experiments); ski_dht_length gives the smallest such N >= n, to
// which [D A; 0] is zero-padded otherwise.  For real x,
// F x = N^{-1/2} (Re X - Im X) with X the DFT, X_k = sum_j x_j e^{-2 pi i jk/N},
// computed by a self-sorting (Stockham) mixed-radix FFT along the row index,
// every column at once.  A pass of radix R and span Ns (the product of the
// radices before it) takes, for each j < N / R, the rows j + r N / R
// (r < R), multiplies row r by e^{-2 pi i r (j mod Ns) / (Ns R)}, applies the
// R-point DFT, and writes its outputs to rows (j div Ns) Ns R + (j mod Ns) +
// r Ns.  Passes alternate between two complex (re, im) planes; the first
// reads D [A | b] straight from A and b, the last writes N^{-1/2} (re - im).
// Radices: 4 and 2 as butterflies, the odd primes 3 .. 13 as direct R-point
// DFTs.  One thread per (j, column): a warp reads and writes 32 neighbouring
// columns of a row (256 bytes in FP64).  Arithmetic in FP64, or FP32 for an
// FP32 or BF16 sketch.
#include <math.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "hash.cuh"
#include "sketch_impl.cuh"

namespace {

template <class T>
struct DhtPassArgs {
  int64_t N, ncols, Ns;
  // first pass: x = D [A | b] (rows >= n are zero)
  const double* A;
  int64_t lda, n, d;
  const double* b;
  const int8_t* D;
  // later passes: the complex planes of the previous one
  const T* xr;
  const T* xi;
  int64_t ldx;
  // output: complex planes, or (last pass) Y = scale (re - im)
  T* yr;
  T* yi;
  int64_t ldy;
  T* Y;
  int64_t ldY;
  T scale;
  // e^{-2 pi i t / N}, t < N
  const T* twr;
  const T* twi;
};

template <class T, int R>
__device__ __forceinline__ void dft_small(T (&vr)[R], T (&vi)[R], const DhtPassArgs<T>& a) {
  if constexpr (R == 2) {
    const T r0 = vr[0] + vr[1], i0 = vi[0] + vi[1];
    vr[1] = vr[0] - vr[1];
    vi[1] = vi[0] - vi[1];
    vr[0] = r0;
    vi[0] = i0;
  } else if constexpr (R == 4) {
    // e^{-2 pi i / 4} = -i: X1 = (a0 - a2) - i (a1 - a3), X3 = (a0 - a2) + i (a1 - a3)
    const T s0r = vr[0] + vr[2], s0i = vi[0] + vi[2], d0r = vr[0] - vr[2], d0i = vi[0] - vi[2];
    const T s1r = vr[1] + vr[3], s1i = vi[1] + vi[3], d1r = vr[1] - vr[3], d1i = vi[1] - vi[3];
    vr[0] = s0r + s1r;
    vi[0] = s0i + s1i;
    vr[2] = s0r - s1r;
    vi[2] = s0i - s1i;
    vr[1] = d0r + d1i;
    vi[1] = d0i - d1r;
    vr[3] = d0r - d1i;
    vi[3] = d0i + d1r;
  } else if constexpr (R > 1) {
    // direct: X_q = sum_r v_r w^{(q r) mod R}, w = e^{-2 pi i / R} = twiddle N / R
    const int64_t st = a.N / R;
    T wr[R], wi[R];
#pragma unroll
    for (int t = 0; t < R; ++t) {
      wr[t] = a.twr[t * st];
      wi[t] = a.twi[t * st];
    }
    T orr[R], oi[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      T sr = vr[0], si = vi[0];
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const int t = (q * r) % R;
        sr = fma(vr[r], wr[t], fma(-vi[r], wi[t], sr));
        si = fma(vr[r], wi[t], fma(vi[r], wr[t], si));
      }
      orr[q] = sr;
      oi[q] = si;
    }
#pragma unroll
    for (int q = 0; q < R; ++q) {
      vr[q] = orr[q];
      vi[q] = oi[q];
    }
  }
}

template <class T, int R, int IN, int OUT>
__global__ void __launch_bounds__(256) k_dht_pass(DhtPassArgs<T> a) {
  const int64_t c = (int64_t)blockIdx.y * 32 + threadIdx.x;
  const int64_t j = (int64_t)blockIdx.x * 8 + threadIdx.y;
  const int64_t M = a.N / R;
  if (c >= a.ncols || j >= M) return;
  T vr[R], vi[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t row = j + r * M;
    if (IN == 0) {
      double x = 0.0;
      if (row < a.n) {
        x = c < a.d ? a.A[row * a.lda + c] : a.b[row];
        if (a.D[row] < 0) x = -x;
      }
      vr[r] = (T)x;
      vi[r] = T(0);
    } else {
      vr[r] = a.xr[row * a.ldx + c];
      vi[r] = a.xi[row * a.ldx + c];
    }
  }
  const int64_t k = j % a.Ns;
  if (k != 0) {
    const int64_t step = k * (a.N / (a.Ns * R));  // r * step < N for r < R
#pragma unroll
    for (int r = 1; r < R; ++r) {
      const int64_t t = r * step;
      const T wr = a.twr[t], wi = a.twi[t];
      const T xr = vr[r], xi = vi[r];
      vr[r] = fma(xr, wr, -xi * wi);
      vi[r] = fma(xr, wi, xi * wr);
    }
  }
  dft_small<T, R>(vr, vi, a);
  const int64_t base = (j / a.Ns) * a.Ns * R + k;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t row = base + r * a.Ns;
    if (OUT == 0) {
      a.yr[row * a.ldy + c] = vr[r];
      a.yi[row * a.ldy + c] = vi[r];
    } else {
      a.Y[row * a.ldY + c] = a.scale * (vr[r] - vi[r]);
    }
  }
}

// e^{-2 pi i t / N} for t < N, from sincospi of the reduced angle
// -2 t / N in (-1, 1].
template <class T>
__global__ void k_dht_twiddles(int64_t N, T* __restrict__ twr, T* __restrict__ twi) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= N) return;
  const int64_t tt = 2 * t > N ? t - N : t;  // same root, |angle| <= 1
  double s, c;
  sincospi(-2.0 * (double)tt / (double)N, &s, &c);
  twr[t] = (T)c;
  twi[t] = (T)s;
}

// Row i of the sketch = row c_i of X (the premixed Y, or [A | b] itself),
// c_i = high word of key(SAMPLE, i, 0, 0) * nrows (Eq. SR-DHT: one 1 per row
// of S_s, in a column drawn uniformly with replacement).
template <class TIN, class TOUT>
__global__ void k_sample_rows(uint64_t kb, int64_t m, int64_t nrows, const TIN* __restrict__ X, int64_t ldx,
                              int64_t dx, const double* __restrict__ b, int64_t ncols, TOUT* __restrict__ SA,
                              int64_t ld_sa) {
  const int64_t c = (int64_t)blockIdx.y * 128 + threadIdx.x;
  const int64_t i = blockIdx.x;
  if (c >= ncols || i >= m) return;
  const int64_t row = (int64_t)__umul64hi(ski_key(kb, (uint64_t)i, 0u, 0u), (uint64_t)nrows);
  const double v = c < dx ? (double)X[row * ldx + c] : b[row];
  SA[i * ld_sa + c] = SkiType<TOUT>::from(v);
}

bool smooth13(int64_t N) {
  if (N < 1) return false;
  for (int64_t p : {2, 3, 5, 7, 11, 13})
    while (N % p == 0) N /= p;
  return N == 1;
}

std::vector<int> dht_radices(int64_t N) {
  std::vector<int> rs;
  while (N % 4 == 0) {
    rs.push_back(4);
    N /= 4;
  }
  while (N % 2 == 0) {
    rs.push_back(2);
    N /= 2;
  }
  for (int p : {3, 5, 7, 11, 13})
    while (N % p == 0) {
      rs.push_back(p);
      N /= p;
    }
  return rs;
}

template <class T, int R>
ski_status launch_pass(int in, int out, const DhtPassArgs<T>& a, cudaStream_t st) {
  const int64_t M = a.N / R;
  dim3 grid((unsigned)ski_cdiv(M, 8), (unsigned)ski_cdiv(a.ncols, 32));
  dim3 block(32, 8);
  if (in == 0 && out == 0) k_dht_pass<T, R, 0, 0><<<grid, block, 0, st>>>(a);
  else if (in == 0) k_dht_pass<T, R, 0, 1><<<grid, block, 0, st>>>(a);
  else if (out == 0) k_dht_pass<T, R, 1, 0><<<grid, block, 0, st>>>(a);
  else k_dht_pass<T, R, 1, 1><<<grid, block, 0, st>>>(a);
  SKI_LAUNCH_CHECK();
  return SKI_OK;
}

template <class T>
ski_status launch_any(int R, int in, int out, const DhtPassArgs<T>& a, cudaStream_t st) {
  switch (R) {
    case 1: return launch_pass<T, 1>(in, out, a, st);
    case 2: return launch_pass<T, 2>(in, out, a, st);
    case 3: return launch_pass<T, 3>(in, out, a, st);
    case 4: return launch_pass<T, 4>(in, out, a, st);
    case 5: return launch_pass<T, 5>(in, out, a, st);
    case 7: return launch_pass<T, 7>(in, out, a, st);
    case 11: return launch_pass<T, 11>(in, out, a, st);
    case 13: return launch_pass<T, 13>(in, out, a, st);
    default: return SKI_EINVAL;
  }
}

template <class T>
ski_status dht_run(const double* A, int64_t lda, int64_t n, int64_t d, const double* b, uint64_t seed, int64_t N,
                   T* Y, int64_t ldY, SkiArena& ar, cudaStream_t st) {
  const int64_t ncols = d + (b ? 1 : 0);
  const int64_t ldc = ski_round_up(std::max<int64_t>(ncols, 1), 4);
  int8_t* D = ar.take<int8_t>(ski_round_up(std::max<int64_t>(n, 1), 256));
  T* twr = ar.take<T>(N);
  T* twi = ar.take<T>(N);
  T* p[4];
  for (auto& q : p) q = ar.take<T>(N * ldc);
  if (!ar.ok() || !p[3]) return SKI_ENOMEM;
  SKI_TRY(ski_premix_signs(seed, n, D, st));
  k_dht_twiddles<T><<<(unsigned)ski_cdiv(N, 256), 256, 0, st>>>(N, twr, twi);
  SKI_LAUNCH_CHECK();
  std::vector<int> rs = dht_radices(N);
  if (rs.empty()) rs.push_back(1);  // N = 1: the identity, one copy pass
  DhtPassArgs<T> a{};
  a.N = N;
  a.ncols = ncols;
  a.A = A;
  a.lda = lda;
  a.n = n;
  a.d = d;
  a.b = b;
  a.D = D;
  a.twr = twr;
  a.twi = twi;
  a.Y = Y;
  a.ldY = ldY;
  a.scale = (T)(1.0 / sqrt((double)N));
  a.ldx = a.ldy = ldc;
  int64_t Ns = 1;
  for (size_t q = 0; q < rs.size(); ++q) {
    const int in = q == 0 ? 0 : 1, out = q + 1 == rs.size() ? 1 : 0;
    a.Ns = Ns;
    a.xr = p[(q + 1) & 1 ? 0 : 2];  // previous pass's output planes
    a.xi = p[(q + 1) & 1 ? 1 : 3];
    a.yr = p[q & 1 ? 0 : 2];
    a.yi = p[q & 1 ? 1 : 3];
    SKI_TRY(launch_any<T>(rs[q], in, out, a, st));
    Ns *= rs[q];
  }
  return SKI_OK;
}

}  // namespace

bool ski_dht_length_ok(int64_t N) { return smooth13(N); }

int64_t ski_dht_length(int64_t n) {
  int64_t N = std::max<int64_t>(n, 1);
  while (!smooth13(N)) ++N;
  return N;
}

size_t ski_dht_ws_bytes(int64_t n, int64_t ncols, int64_t N, int32_t dtype) {
  SkiArena ar{nullptr, 0, 0, true};
  const int64_t ldc = ski_round_up(std::max<int64_t>(ncols, 1), 4);
  const size_t ts = dtype == SKI_F64 ? sizeof(double) : sizeof(float);
  // the takes of dht_run, one by one (each is aligned)
  ar.take<int8_t>(ski_round_up(std::max<int64_t>(n, 1), 256));
  for (int q = 0; q < 2; ++q) ar.take<char>(N * ts);
  for (int q = 0; q < 4; ++q) ar.take<char>(N * ldc * ts);
  return ar.off;
}

ski_status ski_dht_premix(const double* A, int64_t lda, int64_t n, int64_t d, const double* b, uint64_t seed,
                          int64_t N, int32_t dtype, void* Y, int64_t ldY, SkiArena& ar, cudaStream_t st) {
  if (N < std::max<int64_t>(n, 1) || !smooth13(N) || ldY < d + (b ? 1 : 0)) return SKI_EINVAL;
  if (N * ski_round_up(d + 2, 4) >= (1ll << 40)) return SKI_EINVAL;
  if (dtype == SKI_F64) return dht_run<double>(A, lda, n, d, b, seed, N, (double*)Y, ldY, ar, st);
  if (dtype == SKI_F32) return dht_run<float>(A, lda, n, d, b, seed, N, (float*)Y, ldY, ar, st);
  return SKI_EINVAL;
}

ski_status ski_sample_rows(uint64_t seed, int64_t m, int64_t nrows, const void* X, int32_t x_dtype, int64_t ldx,
                           int64_t dx, const double* b, int32_t out_dtype, void* SA, int64_t ld_sa, cudaStream_t st) {
  const int64_t ncols = dx + (b ? 1 : 0);
  if (m <= 0 || ncols <= 0) return SKI_OK;
  if (nrows < 1 || m >= (1ll << 31) || ncols > 128ll * 65535) return SKI_EINVAL;
  const uint64_t kb = ski_tag_base(seed, SKI_TAG_SAMPLE);
  dim3 grid((unsigned)m, (unsigned)ski_cdiv(ncols, 128));
  auto go = [&](auto tin, auto tout) {
    using TI = decltype(tin);
    using TO = decltype(tout);
    k_sample_rows<TI, TO><<<grid, 128, 0, st>>>(kb, m, nrows, (const TI*)X, ldx, dx, b, ncols, (TO*)SA, ld_sa);
  };
  if (x_dtype == SKI_F64) {
    if (out_dtype == SKI_F64) go(double{}, double{});
    else if (out_dtype == SKI_F32) go(double{}, float{});
    else go(double{}, __nv_bfloat16{});
  } else {
    if (out_dtype == SKI_F64) go(float{}, double{});
    else if (out_dtype == SKI_F32) go(float{}, float{});
    else go(float{}, __nv_bfloat16{});
  }
  SKI_LAUNCH_CHECK();
  return SKI_OK;
}
