// Shared helpers of the Ski-LLS CUDA library: status handling, workspace
// carving, warp reductions and the exact int64 block-fixed-point arithmetic
// that replaces FP64 adds on GB300 (whose FP64 pipe runs at 1/64 of FP32).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stddef.h>
#include <algorithm>
#include <mutex>
#include <set>
#include <tuple>
#include "../../include/skills.h"

#define SKI_CUDA_TRY(expr)                                   \
  do {                                                       \
    cudaError_t e_ = (expr);                                 \
    if (e_ != cudaSuccess) { ski_note_cuda_error(e_); return SKI_ECUDA; } \
  } while (0)

#define SKI_TRY(expr)                                        \
  do {                                                       \
    ski_status s_ = (expr);                                  \
    if (s_ != SKI_OK) return s_;                             \
  } while (0)

// Every kernel launch of the library is followed by exactly one
// SKI_LAUNCH_CHECK, which also counts it (ski_launch_count()).
#define SKI_LAUNCH_CHECK()               \
  do {                                   \
    ski_count_launch();                  \
    SKI_CUDA_TRY(cudaGetLastError());    \
  } while (0)

void ski_note_cuda_error(cudaError_t e);
void ski_count_launch();

static inline cudaStream_t ski_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// The dynamic shared-memory cap given to a kernel whose launch size varies:
// the device's opt-in maximum less the kernel's static shared memory.  A cap
// only permits, so one constant per kernel keeps concurrent host threads from
// lowering it under each other's in-flight launches (a per-launch cap races).
// cudaFuncSetAttribute(fn, attr, value()) once per (device, kernel, attribute)
// and call site: every caller passes the same value for a given kernel, so
// later calls, from any host thread, skip the driver (whose calls serialise
// the threads that launch the problems of a batch).
template <class F>
inline cudaError_t ski_attr_once(const void* fn, cudaFuncAttribute attr, F value) {
  static std::mutex mu;
  static std::set<std::tuple<int, const void*, int>> done;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return cudaGetLastError();
  const auto key = std::make_tuple(dev, fn, (int)attr);
  {
    std::lock_guard<std::mutex> lk(mu);
    if (done.count(key)) return cudaSuccess;
  }
  const cudaError_t e = cudaFuncSetAttribute(fn, attr, value());
  if (e == cudaSuccess) {
    std::lock_guard<std::mutex> lk(mu);
    done.insert(key);
  }
  return e;
}

static inline int ski_smem_cap(const void* fn) {
  int dev = 0, optin = 0;
  cudaFuncAttributes a;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaFuncGetAttributes(&a, fn) != cudaSuccess) {
    cudaGetLastError();
    return 48 * 1024;
  }
  return optin - (int)a.sharedSizeBytes;
}

static inline int64_t ski_cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
static inline int64_t ski_round_up(int64_t a, int64_t b) { return ski_cdiv(a, b) * b; }

// Bump allocator over the caller workspace.  Every carve is 256-byte aligned.
struct SkiArena {
  char* base;
  size_t cap;
  size_t off;
  bool dry;  // size query only
  template <class T>
  T* take(size_t count) {
    size_t bytes = ski_round_up((int64_t)(count * sizeof(T)), 256);
    size_t o = off;
    off += bytes;
    if (dry || off > cap) return nullptr;
    return reinterpret_cast<T*>(base + o);
  }
  bool ok() const { return dry || off <= cap; }
};

// One lane's share of a row dot product: sum over c = c0, c0 + 32, ... < c1
// of m[c] x[c], with eight independent accumulators so that eight loads of
// the row are in flight per lane (one chain left the pass latency-bound)
__device__ __forceinline__ double row_dot8(const double* __restrict__ m, const double* __restrict__ x, int64_t c0,
                                           int64_t c1) {
  double a[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  int64_t c = c0;
  for (; c + 7 * 32 < c1; c += 8 * 32) {
    double mv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) mv[u] = __ldcs(&m[c + 32 * u]);
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u] = fma(mv[u], x[c + 32 * u], a[u]);
  }
  for (; c < c1; c += 32) a[0] = fma(__ldcs(&m[c]), x[c], a[0]);
  return ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
}

// ----------------------------------------------------------------- device
__device__ __forceinline__ double ski_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float ski_warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Bulk prefetch of [p, p + bytes) into L2 (TMA unit, no registers or shared
// memory involved).  p and bytes must be multiples of 16; callers pass only
// ranges inside their buffers.
__device__ __forceinline__ void ski_l2_prefetch(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Prefetch the 16-byte-aligned interior of [p, p + bytes) in chunks of 4 KB,
// chunk i issued by the calling thread when i % nthreads == tid.
__device__ __forceinline__ void ski_l2_prefetch_range(const void* p, size_t bytes, int tid, int nthreads) {
  uintptr_t a = ((uintptr_t)p + 15) & ~(uintptr_t)15;
  uintptr_t e = ((uintptr_t)p + bytes) & ~(uintptr_t)15;
  for (uintptr_t c = a + (uintptr_t)tid * 4096; c < e; c += (uintptr_t)nthreads * 4096) {
    const uintptr_t n = (e - c) < 4096 ? (e - c) : 4096;
    ski_l2_prefetch((const void*)c, (unsigned)n);
  }
}

template <class T> struct SkiType;
template <> struct SkiType<double> {
  static constexpr int id = SKI_F64;
  __device__ __forceinline__ static double from(double v) { return v; }
  __device__ __forceinline__ static double to_f64(double v) { return v; }
};
template <> struct SkiType<float> {
  static constexpr int id = SKI_F32;
  __device__ __forceinline__ static float from(double v) { return (float)v; }
  __device__ __forceinline__ static double to_f64(float v) { return (double)v; }
};
template <> struct SkiType<__nv_bfloat16> {
  static constexpr int id = SKI_BF16;
  __device__ __forceinline__ static __nv_bfloat16 from(double v) { return __float2bfloat16((float)v); }
  __device__ __forceinline__ static double to_f64(__nv_bfloat16 v) { return (double)__bfloat162float(v); }
};

// ------------------------------------------- int64 block fixed point (FP64)
// A double v = (-1)^s * M * 2^(e - 1075) with M the 53-bit significand
// (implicit bit included; e the biased exponent field, subnormals use e = 1).
// Values that share a block exponent E are summed exactly as integers
// q = (M << FX_LIFT) >> (E - e): only bits below 2^(E - 1075 - FX_LIFT) are
// dropped, i.e. each term is truncated by less than 2^-54 of the largest one,
// and the integer sum itself is exact and order-independent.  The result is
// as accurate as FP64 additions, deterministic, and runs on the INT32 pipe
// (128 lanes/SM) instead of GB300's FP64 pipe (2 DFMA/clk/SM).
#define FX_LIFT 2

__device__ __forceinline__ int fx_exp(double v) {
  int e = (int)((__double_as_longlong(v) >> 52) & 0x7FF);
  return e == 0 ? 1 : e;
}

// q(v) relative to block exponent E >= fx_exp(v); sign applied; neg flips.
__device__ __forceinline__ long long fx_quant(double v, int E, bool neg) {
  unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  int e = (int)((bits >> 52) & 0x7FF);
  unsigned long long M = (bits & 0xFFFFFFFFFFFFFull) | (e ? (1ull << 52) : 0ull);
  int sh = E - (e ? e : 1);
  unsigned long long q = sh > 63 ? 0ull : ((M << FX_LIFT) >> sh);
  bool negative = ((bits >> 63) != 0) != neg;
  return negative ? -(long long)q : (long long)q;
}

// Out-of-range tail of fx_i64_to_double (kept out of line so that the FP64
// instructions it needs are never issued, predicated, on the fast path).
static __device__ __noinline__ double fx_i64_to_double_slow(long long S, int X) { return ldexp(__ll2double_rn(S), X); }

// The double nearest to S * 2^X (round to nearest even), using integer
// operations only: on GB300 the int64 -> FP64 conversion instruction runs on
// the 1/64-rate FP64 pipe.  |S| < 2^63.
__device__ __forceinline__ double fx_i64_to_double(long long S, int X) {
  if (S == 0) return 0.0;
  const unsigned long long sign = S < 0 ? (1ull << 63) : 0ull;
  unsigned long long u = S < 0 ? (unsigned long long)(-S) : (unsigned long long)S;
  const int lz = __clzll(u);
  u <<= lz;  // leading one at bit 63
  unsigned long long m = u >> 11;
  const unsigned long long rem = u & 0x7FFull;
  m += (rem > 0x400ull || (rem == 0x400ull && (m & 1ull))) ? 1ull : 0ull;
  int e = 63 - lz + X;  // S * 2^X = m * 2^(e - 52)
  if (m >> 53) {
    m >>= 1;
    e += 1;
  }
  const int be = e + 1023;
  if (be < 1 || be > 2046) return fx_i64_to_double_slow(S, X);  // subnormal or overflow: rare
  return __longlong_as_double((long long)(sign | ((unsigned long long)be << 52) | (m & 0xFFFFFFFFFFFFFull)));
}

// The double nearest to S * 2^(E - 1075 - FX_LIFT - extra).
__device__ __forceinline__ double fx_to_double(long long S, int E, int extra = 0) {
  return fx_i64_to_double(S, E - 1075 - FX_LIFT - extra);
}

// Running exact sum with an adaptive block exponent: a larger addend raises
// the exponent and truncates the running sum's low bits once.
// Every addend is below 2^(53 + FX_LIFT) = 2^55 in units of the block; the
// block is coarsened by 2^6 whenever |S| has reached 2^61 before an add, so
// |S| < 2^62 for any number of addends.  NaN/Inf make value() NaN.
struct FxAcc {
  long long S;
  int E;
  bool bad;
  __device__ __forceinline__ void init() { S = 0; E = 1; bad = false; }
  __device__ __forceinline__ void add(double v, bool neg) {
    int e = (int)((__double_as_longlong(v) >> 52) & 0x7FF);
    if (e == 0x7FF) { bad = true; return; }
    e = e ? e : 1;
    if (e > E) {
      int sh = e - E;
      S = sh > 63 ? (S < 0 ? -1 : 0) : (S >> sh);
      E = e;
    }
    if (S >= (1ll << 61) || S <= -(1ll << 61)) { S >>= 6; E += 6; }
    S += fx_quant(v, E, neg);
  }
  __device__ __forceinline__ double value(int extra = 0) const {
    return bad ? __longlong_as_double(0x7FF8000000000000ll) : fx_to_double(S, E, extra);
  }
};

// Grid-wide barrier of a persistent kernel (all CTAs co-resident by the
// cooperative launch).  Every wait is bounded: after `spin_limit` polls
// the CTA sets gb->err and all CTAs leave at their next barrier.
struct GridBar {
  unsigned count, gen;
  int err, pad;
};

__device__ __forceinline__ bool grid_sync(GridBar* gb, unsigned nblocks, unsigned& my_gen, long long spin_limit) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned g = my_gen;
    __threadfence();
    const unsigned arrived = atomicAdd(&gb->count, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(&gb->count, 0u);
      __threadfence();
      atomicAdd(&gb->gen, 1u);
    } else {
      long long spins = 0;
      while (*(volatile unsigned*)&gb->gen == g) {
        if (++spins > spin_limit || *(volatile int*)&gb->err) {
          atomicExch(&gb->err, 1);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = *(volatile int*)&gb->err == 0;
  }
  ++my_gen;
  __syncthreads();
  return s_ok != 0;
}
