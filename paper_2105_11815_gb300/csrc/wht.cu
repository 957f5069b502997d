// Randomised Walsh-Hadamard premix H D (Def. 8) for dense A.
//
// Y = H D [A b; 0]: rows scaled by D_jj, zero-padded to n_pad = 2^L rows and
// transformed along the row index by the Sylvester-order Walsh-Hadamard
// matrix.  The transform is L butterfly levels (rows i and i + 2^l replaced
// by sum and difference); they are split into passes of at most 9 levels.
// One pass stages a tile of 2^nb rows (row index bits [lo, lo+nb)) by 32
// columns: each thread holds 2^RB rows of one column in registers and does
// RB levels there, the tile is exchanged once through shared memory, and the
// remaining GB = nb - RB levels are again done in registers.  Every global
// access is a 32-column (256 B) coalesced row segment.
//
// FP64: the butterflies run on int64 block-fixed-point values (each tile
// column shares one power-of-two exponent, stored beside the intermediate),
// i.e. exact integer adds with headroom for the nb levels of growth -- on
// GB300 the FP64 pipe (2 adds/clk/SM) could not keep up with HBM here.
// FP32: plain FP32 butterflies.
#include <stdlib.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "hash.cuh"
#include "sketch_impl.cuh"

namespace {

constexpr int CT = 32;

__device__ __forceinline__ int64_t tile_base(int64_t tile, int lo, int nb) {
  int64_t low = tile & ((1ll << lo) - 1);
  int64_t hi = tile >> lo;
  return (hi << (lo + nb)) | low;
}
__device__ __forceinline__ int64_t tile_of_row(int64_t row, int lo, int nb) {
  return ((row >> (lo + nb)) << lo) | (row & ((1ll << lo) - 1));
}

struct FxIn {
  // IN == 0: FP64 source
  const double* A;
  int64_t lda, n, d;
  const double* b;
  const int8_t* D;
  int* err;  // bounded-wait error flag of the TMA-fed first pass (nullptr: not used)
  // IN == 1: previous pass
  const long long* Q;
  const int16_t* X;
  int64_t ldq, ldx, nvalid;
  int lo_p, nb_p;
  const int* nf;  // per-column nonfinite flags of the first pass
};
struct FxOut {
  long long* Q;
  int16_t* X;
  int64_t ldq, ldx;
  double* Y;
  int64_t ldy;
  int yshift;
  int* nf;          // per column: set when the column holds a NaN or Inf
  int* nf_any;      // TMA-fed first pass: set when any column does (then a scan sets nf)
  const int* ecol;  // OUT == 2: per-column exponent all tiles are aligned to
};

// OUT == 2 (last pass feeding the hash gather): values are stored as
// q >> (ecol[c] - X + kAlignHeadroom), i.e. in units of 2^(ecol[c] + headroom)
// shared by the whole column, so the gather sums them with plain int64 adds;
// outputs below 2^(ecol[c] + 62) become < 2^55, leaving room for 2^6 addends
// between renorms.
constexpr int kAlignHeadroom = 7;
constexpr int kZeroTile = -32768;  // exponent of an all-zero tile column

// CW: columns per tile (32, or 16 for twice the CTAs per SM where the pass is
// latency-bound).
template <int RB, int GB, int IN, int OUT, int CW = CT>
// off32: every per-thread offset below ((R - 1) * stride) fits in 32 bits, so
// the row loops index with 32-bit offsets (address math on the FMA pipe; the
// integer ALU pipe is the pass's bound).
__global__ void __launch_bounds__(CW << GB, (GB >= 4 && RB <= 4) ? (CW == 16 ? 4 : 2) : 1) k_wht_fx(int lo, int64_t n_pad, int64_t ncols, FxIn in, FxOut out, int colx, int off32) {
  constexpr int R = 1 << RB, G = 1 << GB, NB = RB + GB;
  extern __shared__ long long sq[];            // [R*G][CW]
  __shared__ int sx[G][CW];
  const int c = threadIdx.x & (CW - 1), g = threadIdx.x / CW;
  // colx: column tiles along x, so that the CTAs resident together read
  // neighbouring segments of the same rows (DRAM page locality)
  const int64_t tile = colx ? blockIdx.y : blockIdx.x;
  const int64_t base = tile_base(tile, lo, NB);
  if (IN == 0 && OUT == 0 && lo == 0 && base >= in.n) return;  // whole tile in the zero padding
  const int64_t col = (int64_t)(colx ? blockIdx.x : blockIdx.y) * CW + c;
  const bool cok = col < ncols;
  long long q[R];
  int xsrc[IN == 1 ? R : 1];
  int emax = -100000;
  // input rows of this thread: in0 + t 2^(GB + lo), t < R; the first tv exist
  const int64_t in0 = base + ((int64_t)g << lo);
  const int64_t nin = IN == 0 ? in.n : in.nvalid;
  const int tv = (!cok || in0 >= nin) ? 0 : (int)min((int64_t)R, ((nin - in0 - 1) >> (GB + lo)) + 1);
  if (IN == 0) {
    // A[row][col] (or b[row] for col == d) and D[row]
    const bool isb = col >= in.d;
    const double* ap = isb ? in.b + in0 : in.A + (tv ? in0 * in.lda + col : 0);
    const int64_t as = isb ? ((int64_t)1 << (GB + lo)) : (in.lda << (GB + lo));
    const int8_t* dp = in.D + in0;
    auto ld = [&](auto o, auto full) {
      using O = decltype(o);
#pragma unroll
      for (int t = 0; t < R; ++t) {
        long long bits = 0;
        if (decltype(full)::value || t < tv) {
          bits = __double_as_longlong(ap[(O)t * (O)as]);
          if (dp[(O)t << (GB + lo)] < 0) bits ^= (1ll << 63);  // D_jj = -1: flip the sign bit (no FP64 op)
        }
        const int e = (int)((bits >> 52) & 0x7FF);
        emax = max(emax, e ? e : 1);
        q[t] = bits;
      }
    };
    if (off32) {
      if (tv == R) ld(uint32_t{}, std::true_type{});
      else ld(uint32_t{}, std::false_type{});
    } else {
      ld(int64_t{}, std::false_type{});
    }
  } else {
    // Q[row][col] and the previous pass's exponent of row's tile, which is
    // tile_of_row(in0) + t 2^(GB + lo_p) (the passes' row bits are adjacent)
    const long long* qp = in.Q + (tv ? in0 * in.ldq + col : 0);
    const int16_t* xp = in.X + (tv ? tile_of_row(in0, in.lo_p, in.nb_p) * in.ldx + col : 0);
    const int64_t qs = in.ldq << (GB + lo), xst = in.ldx << (GB + in.lo_p);
    auto ld = [&](auto o, auto full) {
      using O = decltype(o);
#pragma unroll
      for (int t = 0; t < R; ++t) {
        long long v = 0;
        int xs = kZeroTile;
        if (decltype(full)::value || t < tv) {
          v = qp[(O)t * (O)qs];
          xs = xp[(O)t * (O)xst];
        }
        q[t] = v;
        xsrc[t] = xs;  // a zero in a nonzero tile may raise E: harmless, the column unit caps Xq
        emax = max(emax, xs);
      }
    };
    if (off32) {
      if (tv == R) ld(uint32_t{}, std::true_type{});
      else ld(uint32_t{}, std::false_type{});
    } else {
      ld(int64_t{}, std::false_type{});
    }
  }
  sx[g][c] = emax;
  __syncthreads();
  int E = sx[0][c];
#pragma unroll
  for (int gg = 1; gg < G; ++gg) E = max(E, sx[gg][c]);
  // a NaN or Inf in the tile column: the largest exponent field is all ones
  if (IN == 0 && g == 0 && cok && E == 0x7FF && out.nf) atomicOr(&out.nf[col], 1);
  // OUT == 1: a column with a NaN or Inf becomes NaN.  With one pass (IN == 0)
  // the tile is the whole column and E its largest exponent field.
  bool colbad = false;
  if (OUT == 1) colbad = IN == 0 ? (E == 0x7FF) : (cok && in.nf && in.nf[col] != 0);
  // ... and every column when a bounded wait of an earlier pass gave up
  if (OUT == 1 && IN == 1 && in.err && *in.err) colbad = true;
  int X;  // value = q * 2^X after quantisation
  if (IN == 0) {
    constexpr int LIFT = 9 - NB;  // |q| < 2^(62 - NB) before the NB levels
#pragma unroll
    for (int t = 0; t < R; ++t) {
      unsigned long long bits = (unsigned long long)q[t];
      int e = (int)((bits >> 52) & 0x7FF);
      unsigned long long M = (bits & 0xFFFFFFFFFFFFFull) | (e ? (1ull << 52) : 0ull);
      int sh = E - (e ? e : 1);
      unsigned long long mq = sh > 63 ? 0ull : ((M << LIFT) >> sh);
      q[t] = (bits >> 63) ? -(long long)mq : (long long)mq;
    }
    X = E - 1075 - LIFT;
  } else {
    const bool zero = E == -32768;  // all-zero tile column
    if (zero) E = 0;
    // units 2^Xq: NB bits of headroom for the levels, or (OUT == 2) at most
    // the column's output unit 2^(ecol + headroom) -- the family bound keeps
    // every partial sum below 2^(ecol + 62) -- so the output shift is >= 0
    int Xq = E + NB;
    if (OUT == 2 && cok && !zero) Xq = min(Xq, out.ecol[col] + kAlignHeadroom);
#pragma unroll
    for (int t = 0; t < R; ++t) q[t] >>= min(Xq - xsrc[IN == 1 ? t : 0], 63);  // >= 0; absent rows hold 0
    X = zero ? kZeroTile : Xq;
  }
  // RB levels in registers: row bits [GB, GB+RB) of the tile index
#pragma unroll
  for (int h = 1; h < R; h <<= 1) {
#pragma unroll
    for (int t = 0; t < R; ++t) {
      if (!(t & h)) {
        long long u = q[t], w = q[t + h];
        q[t] = u + w;
        q[t + h] = u - w;
      }
    }
  }
#pragma unroll
  for (int t = 0; t < R; ++t) sq[(g + (t << GB)) * CW + c] = q[t];
  __syncthreads();
#pragma unroll
  for (int t = 0; t < R; ++t) q[t] = sq[((g << RB) + t) * CW + c];
  // GB levels in registers: row bits [0, GB)
#pragma unroll
  for (int h = 1; h < G; h <<= 1) {
#pragma unroll
    for (int t = 0; t < R; ++t) {
      if (!(t & h)) {
        long long u = q[t], w = q[t + h];
        q[t] = u + w;
        q[t + h] = u - w;
      }
    }
  }
  if (!cok) return;
  // output rows of this thread: out0 + t 2^lo, t < R; the first to exist
  const int64_t out0 = base + ((int64_t)(g << RB) << lo);
  const int to = out0 >= n_pad ? 0 : (int)min((int64_t)R, ((n_pad - out0 - 1) >> lo) + 1);
  if (OUT == 0 || OUT == 2) {
    if (OUT == 2) {  // to units of 2^(ecol + headroom); X <= ecol + headroom
      const int ash = max(0, min(63, out.ecol[col] - X + kAlignHeadroom));
#pragma unroll
      for (int t = 0; t < R; ++t) q[t] >>= ash;
    }
    long long* op = out.Q + (to ? out0 * out.ldq + col : 0);
    const int64_t os = out.ldq << lo;
    auto st = [&](auto o, auto full) {
      using O = decltype(o);
#pragma unroll
      for (int t = 0; t < R; ++t)
        if (decltype(full)::value || t < to) op[(O)t * (O)os] = q[t];
    };
    if (off32) {
      if (to == R) st(uint32_t{}, std::true_type{});
      else st(uint32_t{}, std::false_type{});
    } else {
      st(int64_t{}, std::false_type{});
    }
  } else {
#pragma unroll
    for (int t = 0; t < R; ++t) {
      const int64_t row = out0 + ((int64_t)t << lo);
      if (t < to)
        out.Y[row * out.ldy + col] = colbad ? __longlong_as_double(0x7FF8000000000000ll)
                                            : fx_to_double(q[t], X - out.yshift + 1075 + FX_LIFT, 0);
    }
  }
  if (OUT == 0 && g == 0) out.X[tile * out.ldx + col] = (int16_t)X;
}

// ecol[c]: an exponent with every output of the next (last) pass in column c
// below 2^(ecol[c] + 62).  An output of that pass sums one row from each of
// 2^nb tiles of the previous pass -- the tiles t = f + k 2^lo_p of one family
// f (the row's bits below lo_p) -- and tile t's values are below
// 2^(X[t][c] + 62).  So 2^ecol[c] = max over families of the sum of 2^X[t][c]
// bounds them; rounded up to a power of two in exact integer arithmetic
// (units of 2^-30 relative to the largest X, tiny terms counted as one unit;
// at most 2^24 tiles).  The plain max + nb bound would give up nb bits where
// one tile dominates a column (a coherent row of A).
// CTA: 32 columns x 8 lanes over the tiles (one family) or the families.
__global__ void __launch_bounds__(256) k_colmax_exp(int64_t ncols, const int16_t* __restrict__ X, int64_t ldx,
                                                    int64_t ntiles, int lo_p, int* __restrict__ ecol) {
  constexpr int LN = 8, FRAC = 30;
  __shared__ int se[LN][32];
  __shared__ unsigned long long ss[LN][32];
  const int cl = threadIdx.x & 31, r = threadIdx.x >> 5;
  const int64_t c = (int64_t)blockIdx.x * 32 + cl;
  const bool ok = c < ncols;
  int e = kZeroTile;
  if (ok)
    for (int64_t tt = r; tt < ntiles; tt += LN) e = max(e, (int)X[tt * ldx + c]);
  se[r][cl] = e;
  __syncthreads();
#pragma unroll
  for (int k = 0; k < LN; ++k) e = max(e, se[k][cl]);
  const int64_t fam = 1ll << lo_p;
  auto term = [&](int x) -> unsigned long long {
    if (x == kZeroTile) return 0ull;
    const int sh = x - e + FRAC;  // <= FRAC
    return sh > 0 ? (1ull << sh) : 1ull;
  };
  unsigned long long v = 0;
  if (ok && e != kZeroTile) {
    if (fam == 1) {  // one family: partial sums over strided tiles
      for (int64_t tt = r; tt < ntiles; tt += LN) v += term(X[tt * ldx + c]);
    } else {  // several: whole families per lane
      for (int64_t f = r; f < fam && f < ntiles; f += LN) {
        unsigned long long s = 0;
        for (int64_t tt = f; tt < ntiles; tt += fam) s += term(X[tt * ldx + c]);
        v = max(v, s);
      }
    }
  }
  ss[r][cl] = v;
  __syncthreads();
  if (r != 0 || !ok) return;
  unsigned long long best = 0;
#pragma unroll
  for (int k = 0; k < LN; ++k) best = fam == 1 ? best + ss[k][cl] : max(best, ss[k][cl]);
  // all-zero column: every output is 0.  Else sum of 2^(X - e) <= best 2^-FRAC
  // < 2^(bitlen(best) - FRAC)
  ecol[c] = e == kZeroTile ? 0 : e + (64 - __clzll((long long)best)) - FRAC;
}

// ---- first pass fed by the tensor memory accelerator
// Row bits 0..7, FP64 A in, int64 tile out: the arithmetic and output of
// k_wht_fx<4, 4, 0, 0, 16>.  A persistent CTA walks its tiles u = blockIdx.x,
// + gridDim.x, ... (column tile fastest) through a 3-stage ring of 256-row x
// 16-column boxes of A (and the tile's 256 signs of D) that TMA fills ahead,
// so the loads of the next two tiles are in flight while the current one is
// transformed; each stage also serves as its tile's exchange buffer.  The
// one-tile-per-CTA kernel idles HBM while it transforms and stores.
constexpr int P1_CW = 16, P1_ROWS = 256, P1_STAGES = 3;
constexpr long long kP1Spin = 1ll << 24;
struct P1Smem {
  long long tile[P1_STAGES][P1_ROWS * P1_CW];  // 32 KB per stage
  int8_t dseg[P1_STAGES][P1_ROWS];
  int sx[16][P1_CW];
  uint64_t full[P1_STAGES];
  int ok;
};

__device__ __forceinline__ uint32_t p1_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ bool p1_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__global__ void __launch_bounds__(256, 2) k_wht_p1_tma(const __grid_constant__ CUtensorMap ta, FxIn in, FxOut out,
                                                       int64_t n_pad, int64_t ncols, int64_t nct, int64_t ntotal,
                                                       int* err) {
  constexpr int RB = 4, GB = 4, R = 1 << RB, G = 1 << GB, NB = RB + GB, CW = P1_CW, S = P1_STAGES;
  extern __shared__ unsigned char p1_raw[];
  P1Smem& sm = *reinterpret_cast<P1Smem*>(((uintptr_t)p1_raw + 127) & ~(uintptr_t)127);
  const int c = threadIdx.x & (CW - 1), g = threadIdx.x / CW;
  const int64_t gstride = gridDim.x;
  const int64_t u0 = blockIdx.x;
  const int64_t mine = u0 < ntotal ? (ntotal - u0 + gstride - 1) / gstride : 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(p1_u32(&sm.full[s])), "r"(1u));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // thread 0: the k-th tile of this CTA into stage k % S
  auto issue = [&](int64_t k) {
    const int64_t u = u0 + k * gstride;
    const int s = (int)(k % S);
    const int64_t base = (u / nct) * P1_ROWS;
    const uint32_t bar = p1_u32(&sm.full[s]);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                 "r"((uint32_t)(P1_ROWS * CW * sizeof(long long) + P1_ROWS))
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            p1_u32(sm.tile[s])),
        "l"((uint64_t)&ta), "r"((int)((u % nct) * CW)), "r"((int)base), "r"(bar)
        : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     p1_u32(sm.dseg[s])),
                 "l"(in.D + base), "r"((uint32_t)P1_ROWS), "r"(bar)
                 : "memory");
  };
  int64_t issued = 0;
  if (threadIdx.x == 0)
    for (; issued < mine && issued < S; ++issued) issue(issued);
  bool bad = false;
  int64_t k = 0;
  for (; k < mine; ++k) {
    const int s = (int)(k % S);
    const uint32_t ph = (uint32_t)(k / S) & 1u;
    const int64_t u = u0 + k * gstride;
    const int64_t tile = u / nct;
    const int64_t base = tile * P1_ROWS;
    const int64_t col = (u % nct) * CW + c;
    const bool cok = col < ncols;
    if (threadIdx.x == 0) {
      bool got = false;
      for (long long i = 0; i < kP1Spin; ++i)
        if (p1_try(p1_u32(&sm.full[s]), ph)) {
          got = true;
          break;
        }
      if (!got) atomicExch(err, 1);
      sm.ok = got ? 1 : 0;
    }
    __syncthreads();
    if (!sm.ok) break;
    long long q[R];
    int emax = -100000;
    if (col < in.d) {  // A: zero outside it (TMA fill)
#pragma unroll
      for (int t = 0; t < R; ++t) {
        const int rl = g + (t << GB);
        long long bits = sm.tile[s][rl * CW + c];
        bits ^= (long long)((unsigned long long)(sm.dseg[s][rl] < 0) << 63);  // D_jj = -1: flip the sign bit
        const int e = (int)((bits >> 52) & 0x7FF);
        bad |= (e == 0x7FF);
        emax = max(emax, e ? e : 1);
        q[t] = bits;
      }
    } else {  // b (column d), or nothing
      const bool isb = col == in.d && in.b;
#pragma unroll
      for (int t = 0; t < R; ++t) {
        const int rl = g + (t << GB);
        long long bits = (isb && base + rl < in.n) ? __double_as_longlong(in.b[base + rl]) : 0ll;
        bits ^= (long long)((unsigned long long)(sm.dseg[s][rl] < 0) << 63);
        const int e = (int)((bits >> 52) & 0x7FF);
        bad |= (e == 0x7FF);
        emax = max(emax, e ? e : 1);
        q[t] = bits;
      }
    }
    sm.sx[g][c] = emax;
    __syncthreads();
    int E = sm.sx[0][c];
#pragma unroll
    for (int gg = 1; gg < G; ++gg) E = max(E, sm.sx[gg][c]);
    constexpr int LIFT = 9 - NB;
#pragma unroll
    for (int t = 0; t < R; ++t) {
      const unsigned long long bits = (unsigned long long)q[t];
      const int e = (int)((bits >> 52) & 0x7FF);
      const unsigned long long M = (bits & 0xFFFFFFFFFFFFFull) | (e ? (1ull << 52) : 0ull);
      const unsigned long long mq = (M << LIFT) >> min(E - (e ? e : 1), 63);  // 0 for shifts >= 63
      q[t] = (bits >> 63) ? -(long long)mq : (long long)mq;
    }
    const int X = E - 1075 - LIFT;
#pragma unroll
    for (int h = 1; h < R; h <<= 1)
#pragma unroll
      for (int t = 0; t < R; ++t)
        if (!(t & h)) {
          const long long a = q[t], b = q[t + h];
          q[t] = a + b;
          q[t + h] = a - b;
        }
#pragma unroll
    for (int t = 0; t < R; ++t) sm.tile[s][(g + (t << GB)) * CW + c] = q[t];
    __syncthreads();
#pragma unroll
    for (int t = 0; t < R; ++t) q[t] = sm.tile[s][((g << RB) + t) * CW + c];
#pragma unroll
    for (int h = 1; h < G; h <<= 1)
#pragma unroll
      for (int t = 0; t < R; ++t)
        if (!(t & h)) {
          const long long a = q[t], b = q[t + h];
          q[t] = a + b;
          q[t + h] = a - b;
        }
    __syncthreads();  // stage s is free again
    if (threadIdx.x == 0 && issued < mine) issue(issued++);
    if (cok) {
      // rows base + (g << RB) + t: all below round_up(n, 256) <= n_pad
      long long* op = out.Q + (base + (g << RB)) * out.ldq + col;
#pragma unroll
      for (int t = 0; t < R; ++t) op[(uint32_t)t * (uint32_t)out.ldq] = q[t];
      if (g == 0) out.X[tile * out.ldx + col] = (int16_t)X;
    }
  }
  if (threadIdx.x == 0) {
    // after a timeout: let the copies still in flight land before leaving
    for (int64_t kk = k; kk < issued; ++kk) {
      const uint32_t bar = p1_u32(&sm.full[kk % S]);
      const uint32_t ph = (uint32_t)(kk / S) & 1u;
      for (long long i = 0; i < kP1Spin && !p1_try(bar, ph); ++i) {
      }
    }
  }
  if (bad && out.nf_any) atomicOr(out.nf_any, 1);
}

// After the TMA-fed pass, only if it met a NaN or Inf: nf[c] for every
// column c of [A b] that holds one.
__global__ void __launch_bounds__(256) k_column_nonfinite(const double* __restrict__ A, int64_t lda, int64_t n,
                                                          int64_t d, const double* __restrict__ b, int64_t ncols,
                                                          const int* __restrict__ any, int* __restrict__ nf) {
  if (*any == 0) return;
  for (int64_t j = blockIdx.x; j < n; j += gridDim.x)
    for (int64_t c = threadIdx.x; c < ncols; c += blockDim.x) {
      const long long bits = __double_as_longlong(c < d ? A[j * lda + c] : b[j]);
      if (((bits >> 52) & 0x7FF) == 0x7FF) atomicOr(&nf[c], 1);
    }
}

template <class TOUT>
struct F32Out {
  float* Q;
  int64_t ldq;
  TOUT* Y;
  int64_t ldy;
  float yscale;
};

template <int RB, int GB, int IN, int OUT, class TOUT>
__global__ void __launch_bounds__(CT << GB) k_wht_f32(int lo, int64_t n_pad, int64_t ncols, FxIn in,
                                                       const float* Qin, int64_t ldqin, F32Out<TOUT> out, int colx) {
  constexpr int R = 1 << RB, G = 1 << GB, NB = RB + GB;
  extern __shared__ float sf[];
  const int c = threadIdx.x & (CT - 1), g = threadIdx.x / CT;
  const int64_t tile = colx ? blockIdx.y : blockIdx.x;
  const int64_t base = tile_base(tile, lo, NB);
  if (IN == 0 && OUT == 0 && lo == 0 && base >= in.n) return;
  const int64_t col = (int64_t)(colx ? blockIdx.x : blockIdx.y) * CT + c;
  const bool cok = col < ncols;
  float q[R];
#pragma unroll
  for (int t = 0; t < R; ++t) {
    const int64_t row = base + ((int64_t)(g + (t << GB)) << lo);
    float v = 0.f;
    if (IN == 0) {
      if (cok && row < in.n) {
        v = (float)(col < in.d ? in.A[row * in.lda + col] : in.b[row]);
        if (in.D[row] < 0) v = -v;
      }
    } else {
      if (cok && row < in.nvalid) v = Qin[row * ldqin + col];
    }
    q[t] = v;
  }
#pragma unroll
  for (int h = 1; h < R; h <<= 1)
#pragma unroll
    for (int t = 0; t < R; ++t)
      if (!(t & h)) {
        float u = q[t], w = q[t + h];
        q[t] = u + w;
        q[t + h] = u - w;
      }
#pragma unroll
  for (int t = 0; t < R; ++t) sf[(g + (t << GB)) * CT + c] = q[t];
  __syncthreads();
#pragma unroll
  for (int t = 0; t < R; ++t) q[t] = sf[((g << RB) + t) * CT + c];
#pragma unroll
  for (int h = 1; h < G; h <<= 1)
#pragma unroll
    for (int t = 0; t < R; ++t)
      if (!(t & h)) {
        float u = q[t], w = q[t + h];
        q[t] = u + w;
        q[t + h] = u - w;
      }
  if (!cok) return;
#pragma unroll
  for (int t = 0; t < R; ++t) {
    const int64_t row = base + ((int64_t)((g << RB) + t) << lo);
    if (row >= n_pad) continue;
    if (OUT == 0) out.Q[row * out.ldq + col] = q[t];
    else out.Y[row * out.ldy + col] = SkiType<TOUT>::from((double)(q[t] * out.yscale));
  }
}

int ilog2(int64_t v) {
  int l = 0;
  while ((1ll << l) < v) ++l;
  return l;
}

void plan_passes(int L, int* nbs, int* np) {
  if (L == 0) {
    nbs[0] = 1;
    *np = 1;
    return;
  }
  int P = (L + 8) / 9;
  for (int p = 0; p < P; ++p) nbs[p] = L / P + (p < L % P ? 1 : 0);
  *np = P;
}

// Whether a k_wht_fx launch may index rows with 32-bit offsets: (R - 1)
// times each per-row stride (elements) below 2^32.
bool fx_off32(int IN, int RB, int GB, int lo, const FxIn& in, const FxOut& out) {
  const int64_t R1 = (1ll << RB) - 1;
  int64_t s = 0;
  if (IN == 0) s = std::max(in.lda << (GB + lo), (int64_t)1 << (GB + lo));
  else s = std::max(in.ldq << (GB + lo), in.ldx << (GB + in.lo_p));
  s = std::max(s, out.ldq << lo);
  return R1 * s < (1ll << 32) - 1;
}

template <int IN, int OUT>
ski_status launch_fx(int nb, int lo, int64_t n_pad, int64_t ncols, const FxIn& in, const FxOut& out,
                     cudaStream_t st) {
  const int GB = nb / 2, RB = nb - GB;
  const int64_t ntiles = n_pad >> nb > 0 ? (n_pad >> nb) : 1;
  const int colx = ntiles <= 65535 ? 1 : 0;
  dim3 grid = colx ? dim3((unsigned)ski_cdiv(ncols, CT), (unsigned)ntiles)
                   : dim3((unsigned)ntiles, (unsigned)ski_cdiv(ncols, CT));
  const size_t smem = (size_t)(1 << nb) * CT * sizeof(long long);
  const int threads = CT << GB;
  // the first pass (FP64 in) is latency-bound: fed by TMA when A's layout
  // allows a tensor map (row stride a multiple of 16 bytes), else 16-column
  // tiles at four CTAs per SM
  if (IN == 0 && OUT == 0 && RB == 4 && GB == 4 && lo == 0 && in.err && 15 * out.ldq < (1ll << 32)) {
    CUtensorMap ta;
    if (ski_tmap_f64_2d(&ta, in.A, in.n, in.d, in.lda, P1_ROWS, P1_CW)) {
      const int64_t nct = ski_cdiv(ncols, P1_CW);
      const int64_t ntotal = ski_cdiv(in.n, (int64_t)P1_ROWS) * nct;
      int sms = 0, dev = 0;
      SKI_CUDA_TRY(cudaGetDevice(&dev));
      SKI_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
      const size_t sm1 = sizeof(P1Smem) + 128;
      SKI_CUDA_TRY(cudaFuncSetAttribute(k_wht_p1_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1));
      const unsigned grid1 = (unsigned)std::min<int64_t>(ntotal, 2ll * sms);
      if (ntotal > 0) k_wht_p1_tma<<<grid1, 256, sm1, st>>>(ta, in, out, n_pad, ncols, nct, ntotal, in.err);
      SKI_LAUNCH_CHECK();
      if (out.nf && out.nf_any && in.n > 0) {
        k_column_nonfinite<<<(unsigned)(2 * sms), 256, 0, st>>>(in.A, in.lda, in.n, in.d, in.b, ncols, out.nf_any,
                                                                 out.nf);
        SKI_LAUNCH_CHECK();
      }
      return SKI_OK;
    }
  }
  if (IN == 0 && RB == 4 && GB == 4 && lo == 0) {
    constexpr int CW = 16;
    auto kfn = k_wht_fx<4, 4, IN, OUT, CW>;
    const size_t sm16 = (size_t)(1 << nb) * CW * sizeof(long long);
    dim3 g16 = colx ? dim3((unsigned)ski_cdiv(ncols, CW), (unsigned)ntiles)
                    : dim3((unsigned)ntiles, (unsigned)ski_cdiv(ncols, CW));
    if (sm16 > 48 * 1024)
      SKI_CUDA_TRY(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm16));
    kfn<<<g16, CW << 4, sm16, st>>>(lo, n_pad, ncols, in, out, colx, fx_off32(IN, 4, 4, lo, in, out) ? 1 : 0);
    SKI_LAUNCH_CHECK();
    return SKI_OK;
  }
#define SKI_FX_CASE(rb, gb)                                                                      \
  if (RB == rb && GB == gb) {                                                                    \
    auto kfn = k_wht_fx<rb, gb, IN, OUT>;                                                        \
    if (smem > 48 * 1024)                                                                        \
      SKI_CUDA_TRY(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
    kfn<<<grid, threads, smem, st>>>(lo, n_pad, ncols, in, out, colx, fx_off32(IN, rb, gb, lo, in, out) ? 1 : 0); \
    SKI_LAUNCH_CHECK();                                                                          \
    return SKI_OK;                                                                               \
  }
  SKI_FX_CASE(1, 0) SKI_FX_CASE(1, 1) SKI_FX_CASE(2, 1) SKI_FX_CASE(2, 2) SKI_FX_CASE(3, 2)
  SKI_FX_CASE(3, 3) SKI_FX_CASE(4, 3) SKI_FX_CASE(4, 4) SKI_FX_CASE(5, 4)
#undef SKI_FX_CASE
  return SKI_EINVAL;
}

template <int IN, int OUT, class TOUT>
ski_status launch_f32(int nb, int lo, int64_t n_pad, int64_t ncols, const FxIn& in, const float* Qin,
                      int64_t ldqin, const F32Out<TOUT>& out, cudaStream_t st) {
  const int GB = nb / 2, RB = nb - GB;
  const int64_t ntiles = n_pad >> nb > 0 ? (n_pad >> nb) : 1;
  const int colx = ntiles <= 65535 ? 1 : 0;
  dim3 grid = colx ? dim3((unsigned)ski_cdiv(ncols, CT), (unsigned)ntiles)
                   : dim3((unsigned)ntiles, (unsigned)ski_cdiv(ncols, CT));
  const size_t smem = (size_t)(1 << nb) * CT * sizeof(float);
  const int threads = CT << GB;
#define SKI_F32_CASE(rb, gb)                                                                     \
  if (RB == rb && GB == gb) {                                                                    \
    auto kfn = k_wht_f32<rb, gb, IN, OUT, TOUT>;                                                 \
    if (smem > 48 * 1024)                                                                        \
      SKI_CUDA_TRY(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
    kfn<<<grid, threads, smem, st>>>(lo, n_pad, ncols, in, Qin, ldqin, out, colx);               \
    SKI_LAUNCH_CHECK();                                                                          \
    return SKI_OK;                                                                               \
  }
  SKI_F32_CASE(1, 0) SKI_F32_CASE(1, 1) SKI_F32_CASE(2, 1) SKI_F32_CASE(2, 2) SKI_F32_CASE(3, 2)
  SKI_F32_CASE(3, 3) SKI_F32_CASE(4, 3) SKI_F32_CASE(4, 4) SKI_F32_CASE(5, 4)
#undef SKI_F32_CASE
  return SKI_EINVAL;
}

// Tiles of the pass with the fewest row bits: rows of a per-tile exponent plane.
int64_t fx_max_tiles(int64_t n_pad) {
  int nbs[8], np = 0;
  plan_passes(ilog2(n_pad), nbs, &np);
  int nbmin = nbs[0];
  for (int p = 1; p < np; ++p) nbmin = std::min(nbmin, nbs[p]);
  return std::max<int64_t>(1, n_pad >> nbmin);
}

}  // namespace

size_t ski_premix_ws_bytes(int64_t n, int64_t ncols, int64_t n_pad, int32_t dtype) {
  SkiArena ar{nullptr, 0, 0, true};
  const int64_t ldq = ski_round_up(ncols, CT);
  ar.take<int8_t>(ski_round_up(n, 256));
  ar.take<int>(ldq + 1);
  ar.take<int>(1);
  if (dtype == SKI_F64) {
    ar.take<long long>(n_pad * ldq);
    ar.take<long long>(n_pad * ldq);
    ar.take<int16_t>(fx_max_tiles(n_pad) * ldq);
    ar.take<int16_t>(fx_max_tiles(n_pad) * ldq);
    ar.take<int>(ldq);
  } else {
    ar.take<float>(n_pad * ldq);
    ar.take<float>(n_pad * ldq);
  }
  return ar.off;
}

ski_status ski_premix_plan(int64_t n, int64_t ncols_max, int64_t n_pad, int32_t dtype, uint64_t seed, SkiArena& ar,
                           cudaStream_t st, SkiPremixPlan* pp, int* err_flag) {
  SkiPremixPlan& P = *pp;
  P.n = n;
  P.n_pad = n_pad;
  P.dtype = dtype;
  P.ldq = ski_round_up(ncols_max, CT);
  P.D = ar.take<int8_t>(ski_round_up(n, 256));  // padded: the TMA pass copies 256 signs per tile
  P.nonfinite = ar.take<int>(P.ldq + 1);  // per column, then the any-column flag
  int* own_err = ar.take<int>(1);
  P.err = err_flag ? err_flag : own_err;
  P.L = ilog2(n_pad);
  plan_passes(P.L, P.nbs, &P.P);
  P.residual_scale = (P.L & 1) ? 0.70710678118654752440 : 1.0;
  P.yshift = P.L / 2;
  if (dtype == SKI_F64) {
    P.Qa = ar.take<long long>(n_pad * P.ldq);
    P.Qb = ar.take<long long>(n_pad * P.ldq);
    P.Xa = ar.take<int16_t>(fx_max_tiles(n_pad) * P.ldq);
    P.Xb = ar.take<int16_t>(fx_max_tiles(n_pad) * P.ldq);
    P.ecol = ar.take<int>(P.ldq);
  } else {
    P.Qa = ar.take<float>(n_pad * P.ldq);
    P.Qb = ar.take<float>(n_pad * P.ldq);
    P.Xa = P.Xb = nullptr;
    P.ecol = nullptr;
  }
  if (!ar.ok() || !P.Qb) return SKI_ENOMEM;
  SKI_TRY(ski_premix_signs(seed, n, P.D, st));
  if (ski_round_up(n, 256) > n) SKI_CUDA_TRY(cudaMemsetAsync(P.D + n, 0, ski_round_up(n, 256) - n, st));
  SKI_CUDA_TRY(cudaMemsetAsync(P.nonfinite, 0, (P.ldq + 1) * sizeof(int), st));
  if (!err_flag) SKI_CUDA_TRY(cudaMemsetAsync(P.err, 0, sizeof(int), st));
  return SKI_OK;
}

namespace {
// FP64 passes; qfinal: the last pass also writes block-fixed-point int64
// values and per-(tile, column) exponents instead of FP64 Y, described in *qo.
ski_status premix_fx_passes(const SkiPremixPlan& P, const FxIn& in, int64_t ncols, void* Y, int64_t ldy, bool qfinal,
                            SkiPremixQ* qo, cudaStream_t st) {
  const int64_t n = P.n, n_pad = P.n_pad, ldq = P.ldq;
  long long* Qa = (long long*)P.Qa;
  long long* Qb = (long long*)P.Qb;
  // per-column flags of this call's columns (a slab reuses the plan)
  SKI_CUDA_TRY(cudaMemsetAsync(P.nonfinite, 0, (ldq + 1) * sizeof(int), st));
  int lo = 0;
  int64_t nvalid = n;
  long long* Qin = nullptr;
  int16_t* Xin = nullptr;
  int lo_p = 0, nb_p = 0;
  for (int p = 0; p < P.P; ++p) {
    const int nb = P.nbs[p];
    const bool last = p == P.P - 1;
    const bool to_y = last && !qfinal;
    const bool aligned = last && qfinal && p > 0;  // column-aligned int64 for the gather
    long long* Qo = (p & 1) ? Qb : Qa;
    int16_t* Xo = (p & 1) ? P.Xb : P.Xa;
    FxOut out{};
    out.Q = Qo; out.X = Xo; out.ldq = ldq; out.ldx = ldq; out.Y = (double*)Y; out.ldy = ldy;
    out.yshift = P.yshift; out.nf = P.nonfinite; out.nf_any = P.nonfinite + ldq; out.ecol = P.ecol;
    FxIn cur = in;
    cur.Q = Qin; cur.X = Xin; cur.ldq = ldq; cur.ldx = ldq; cur.nvalid = nvalid; cur.lo_p = lo_p; cur.nb_p = nb_p;
    cur.nf = P.nonfinite;
    if (aligned) {
      // exponent bound of every tile of the last pass, per column, from the
      // previous pass's exponents (its tiles that hold rows below nvalid)
      const int64_t ntp = ski_cdiv(nvalid, 1ll << nb_p) << lo_p;
      k_colmax_exp<<<(unsigned)ski_cdiv(ncols, 32), 256, 0, st>>>(ncols, Xin, ldq, std::min<int64_t>(ntp, n_pad >> nb_p),
                                                                  lo_p, P.ecol);
      SKI_LAUNCH_CHECK();
    }
    ski_status s;
    if (p == 0) s = to_y ? launch_fx<0, 1>(nb, lo, n_pad, ncols, cur, out, st) : launch_fx<0, 0>(nb, lo, n_pad, ncols, cur, out, st);
    else if (aligned) s = launch_fx<1, 2>(nb, lo, n_pad, ncols, cur, out, st);
    else s = to_y ? launch_fx<1, 1>(nb, lo, n_pad, ncols, cur, out, st) : launch_fx<1, 0>(nb, lo, n_pad, ncols, cur, out, st);
    if (s != SKI_OK) return s;
    if (last && qfinal) {
      qo->Q = Qo;
      qo->nonfinite = P.nonfinite;
      qo->err = P.err;
      qo->X = aligned ? nullptr : Xo;
      qo->ecol = aligned ? P.ecol : nullptr;
      qo->headroom = kAlignHeadroom;
      qo->ldq = ldq;
      qo->ldx = ldq;
      qo->lo = lo;
      qo->nb = nb;
      qo->yshift = P.yshift;
    }
    nvalid = (p == 0) ? ski_round_up(n, 1ll << nb) : n_pad;
    if (nvalid > n_pad) nvalid = n_pad;
    Qin = Qo; Xin = Xo; lo_p = lo; nb_p = nb;
    lo += nb;
  }
  return SKI_OK;
}
}  // namespace

ski_status ski_premix_cols_q(const SkiPremixPlan& P, const double* A, int64_t lda, int64_t d, const double* b,
                             SkiPremixQ* qo, cudaStream_t st) {
  const int64_t ncols = d + (b != nullptr);
  if (ncols > P.ldq || P.dtype != SKI_F64) return SKI_EINVAL;
  FxIn in{};
  in.A = A; in.lda = lda; in.n = P.n; in.d = d; in.b = b; in.D = P.D; in.err = P.err;
  return premix_fx_passes(P, in, ncols, nullptr, 0, true, qo, st);
}

ski_status ski_premix_cols(const SkiPremixPlan& P, const double* A, int64_t lda, int64_t d, const double* b, void* Y,
                           int64_t ldy, cudaStream_t st) {
  const int64_t ncols = d + (b != nullptr);
  if (ncols > P.ldq) return SKI_EINVAL;
  const int64_t n = P.n, n_pad = P.n_pad, ldq = P.ldq;
  FxIn in{};
  in.A = A; in.lda = lda; in.n = n; in.d = d; in.b = b; in.D = P.D; in.err = P.err;
  if (P.dtype == SKI_F64) {
    SKI_TRY(premix_fx_passes(P, in, ncols, Y, ldy, false, nullptr, st));
  } else {
    float* Qa = (float*)P.Qa;
    float* Qb = (float*)P.Qb;
    int lo = 0;
    int64_t nvalid = n;
    const float* Qin = nullptr;
    const float yscale = ldexpf(1.0f, -P.yshift);
    for (int p = 0; p < P.P; ++p) {
      const int nb = P.nbs[p];
      const bool last = p == P.P - 1;
      float* Qo = (p & 1) ? Qb : Qa;
      FxIn cur = in;
      cur.nvalid = nvalid;
      ski_status s;
      if (P.dtype == SKI_F32) {
        F32Out<float> out{Qo, ldq, (float*)Y, ldy, yscale};
        if (p == 0) s = last ? launch_f32<0, 1, float>(nb, lo, n_pad, ncols, cur, Qin, ldq, out, st)
                             : launch_f32<0, 0, float>(nb, lo, n_pad, ncols, cur, Qin, ldq, out, st);
        else s = last ? launch_f32<1, 1, float>(nb, lo, n_pad, ncols, cur, Qin, ldq, out, st)
                      : launch_f32<1, 0, float>(nb, lo, n_pad, ncols, cur, Qin, ldq, out, st);
      } else {
        F32Out<__nv_bfloat16> out{Qo, ldq, (__nv_bfloat16*)Y, ldy, yscale};
        if (p == 0) s = last ? launch_f32<0, 1, __nv_bfloat16>(nb, lo, n_pad, ncols, cur, Qin, ldq, out, st)
                             : launch_f32<0, 0, __nv_bfloat16>(nb, lo, n_pad, ncols, cur, Qin, ldq, out, st);
        else s = last ? launch_f32<1, 1, __nv_bfloat16>(nb, lo, n_pad, ncols, cur, Qin, ldq, out, st)
                      : launch_f32<1, 0, __nv_bfloat16>(nb, lo, n_pad, ncols, cur, Qin, ldq, out, st);
      }
      if (s != SKI_OK) return s;
      nvalid = (p == 0) ? ski_round_up(n, 1ll << nb) : n_pad;
      if (nvalid > n_pad) nvalid = n_pad;
      Qin = Qo;
      lo += nb;
    }
  }
  return SKI_OK;
}

ski_status ski_premix_run(const double* A, int64_t lda, int64_t n, int64_t d, const double* b, uint64_t seed,
                          int64_t n_pad, int32_t dtype, void* Y, int64_t ldy, SkiArena& ar, cudaStream_t st,
                          double* residual_scale) {
  SkiPremixPlan P;
  SKI_TRY(ski_premix_plan(n, d + (b != nullptr), n_pad, dtype, seed, ar, st, &P));
  *residual_scale = P.residual_scale;
  return ski_premix_cols(P, A, lda, d, b, Y, ldy, st);
}
