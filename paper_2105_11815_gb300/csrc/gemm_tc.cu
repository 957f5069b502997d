// Tensor-core GEMM for the FP32 QR trailing update (Algorithm 1, Step 2):
// D[M x N] = A[M x K] * B[N x K]^T with A and B K-major FP32 in global
// memory, multiplied as TF32 by tcgen05.mma with the FP32 accumulator in
// tensor memory, and stored (or subtracted) to a row-major C.
//
// Precision: one TF32 pass keeps 11 significant bits of each operand (unit
// roundoff 2^-11).  The split form (SPLIT) writes each operand tile as
// x = hi + lo with hi = x rounded to TF32 and lo = (x - hi) rounded to TF32,
// and accumulates lo*hi + hi*lo + hi*hi (the lo*lo term, below 2^-22 |a||b|,
// is dropped): about FP32 accuracy from three tensor-core passes.
//
// One CTA computes one BM x BN tile (BM = 128 rows = 128 TMEM lanes, BN up to
// 256 TMEM columns), K in steps of BK = 32 FP32 (128 bytes, one 128-byte
// swizzle row).  Four warps:
//   warp 0, lane 0   TMA producer: 2-D tensor-map copies of the A and B
//                    tiles into a STAGES-deep shared-memory ring (128B swizzle)
//   warp 1           allocates TMEM; lane 0 issues 4 tcgen05.mma per stage
//                    (K = 8 each) and commits each stage back to the producer
//   warps 2, 3       (SPLIT only) split each landed stage into hi and lo
//                    tiles in place, then release it to the MMA issuer
//   warps 0..3       epilogue: tcgen05.ld of their 32 TMEM lanes, store to C
// Every mbarrier wait is bounded: after kSpinLimit polls the CTA raises the
// error flag, drains its outstanding copies (again bounded), frees its TMEM
// and returns.
#include <cuda.h>

#include "common.cuh"
#include "sketch_impl.cuh"

namespace {

constexpr int BM = 128, BK = 32, NTHR = 128;
constexpr long long kSpinLimit = 1ll << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait; false (and the error flag set) when it gave up.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err) {
  for (long long i = 0; i < kSpinLimit; ++i) {
    if (mbar_try(bar, parity)) return true;
    if ((i & 1023) == 1023 && *(volatile int*)err) return false;
  }
  atomicExch(err, 1);
  return false;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
          "r"(dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor, K-major operand in the 128-byte swizzle
// canonical layout: 8-row groups 1024 bytes apart (stride byte offset),
// descriptor version 1, layout type 2 (128B swizzle).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor of kind::tf32: D = F32, A = B = TF32, both K-major.
__host__ __device__ constexpr uint32_t tf32_idesc(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
// Instruction descriptor of kind::f16: D = F32, A = B = F16, both K-major.
__host__ __device__ constexpr uint32_t f16_idesc(int m, int n) {
  return (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

template <int BN, int STAGES, bool SPLIT>
struct TcSmem {
  float A[STAGES][BM * BK];  // 16 KB per stage
  float B[STAGES][BN * BK];  // BN * 128 bytes per stage
  float Alo[SPLIT ? STAGES : 1][SPLIT ? BM * BK : 256];  // lo parts (SPLIT), same swizzled layout
  float Blo[SPLIT ? STAGES : 1][SPLIT ? BN * BK : 256];
  float stage[4][32][33];     // epilogue staging, one 32 x 32 block per warp
  uint64_t full[STAGES], conv[STAGES], empty[STAGES], done;
  uint32_t tmem;
};

// x -> (hi, lo): hi = x rounded to TF32 (low 13 mantissa bits cleared after
// rounding), lo = x - hi (exact) rounded to TF32.  In place for hi.
__device__ __forceinline__ void tf32_split(float* hi_tile, float* lo_tile, int count, int t, int nt) {
  float4* h4 = reinterpret_cast<float4*>(hi_tile);
  float4* l4 = reinterpret_cast<float4*>(lo_tile);
  for (int i = t; i < count / 4; i += nt) {
    const float4 x = h4[i];
    float xs[4] = {x.x, x.y, x.z, x.w}, hs[4], ls[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float h = __uint_as_float((__float_as_uint(xs[k]) + 0x1000u) & 0xFFFFE000u);
      const float l = __fsub_rn(xs[k], h);
      hs[k] = h;
      ls[k] = __uint_as_float((__float_as_uint(l) + 0x1000u) & 0xFFFFE000u);
    }
    h4[i] = make_float4(hs[0], hs[1], hs[2], hs[3]);
    l4[i] = make_float4(ls[0], ls[1], ls[2], ls[3]);
  }
}

// mode 0: C[m * ldc + n] = D; mode 1: C[m * ldc + n] -= D; mode 2: C[n * ldc + m] = D;
// mode 3 (F16 only): C64[m * ldc + n] += scale64 * D (FP64).
// mode | 4: only the tiles that meet the upper triangle (some m <= n).
// F16: operands FP16 (a stage is 64 of them per row, the same 128 bytes),
// multiplied by kind::f16 (K = 16 per instruction), read through 3-D tensor
// maps over a stack of matrices: the accumulator sums A[pr.a[p]] B[pr.b[p]]^T
// over the pr.n pairs p (K each); else FP32 as TF32.
template <int BN, int STAGES, bool SPLIT, bool F16 = false>
__global__ void __launch_bounds__(NTHR, 1) k_gemm_tc(const __grid_constant__ CUtensorMap ta,
                                                      const __grid_constant__ CUtensorMap tb, int M, int N, int K,
                                                      int kchunk, float* __restrict__ C, int64_t ldc,
                                                      int64_t c_zstride, int mode, int* err,
                                                      double* __restrict__ C64, double scale64, TcPairs pr) {
  static_assert(!(F16 && SPLIT), "the split form is for FP32 operands");
  constexpr int BKE = F16 ? 2 * BK : BK;  // K elements per stage
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  TcSmem<BN, STAGES, SPLIT>& sm = *reinterpret_cast<TcSmem<BN, STAGES, SPLIT>*>(
      (void*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  const int nkp = kend > kbeg ? (kend - kbeg + BKE - 1) / BKE : 0;  // K steps of one pair
  const int nk = F16 ? nkp * pr.n : nkp;
  C += (int64_t)blockIdx.z * c_zstride;
  if ((mode & 4) && m0 >= n0 + BN) return;  // the whole tile is below the diagonal (CTA-uniform)
  mode &= 3;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&sm.full[s]), 1);
      mbar_init(smem_u32(&sm.conv[s]), 64);
      mbar_init(smem_u32(&sm.empty[s]), 1);
    }
    mbar_init(smem_u32(&sm.done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm.tmem)),
                 "r"(BN < 32 ? 32 : BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = sm.tmem;

  if (warp == 0 && lane == 0) {
    // TMA producer
    const uint32_t bytes = (uint32_t)(BM + BN) * BK * sizeof(float);
    int issued = 0;
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % STAGES;
      const uint32_t ph = (uint32_t)(kt / STAGES) & 1u;
      if (!mbar_wait(smem_u32(&sm.empty[s]), ph ^ 1u, err)) break;
      mbar_expect_tx(smem_u32(&sm.full[s]), bytes);
      if constexpr (F16) {
        const int p = kt / nkp, kx = kbeg + (kt - p * nkp) * BKE;
        tma_load_3d(smem_u32(sm.A[s]), &ta, kx, m0, pr.a[p], smem_u32(&sm.full[s]));
        tma_load_3d(smem_u32(sm.B[s]), &tb, kx, n0, pr.b[p], smem_u32(&sm.full[s]));
      } else {
        const int kx = kbeg + kt * BKE;
        tma_load_2d(smem_u32(sm.A[s]), &ta, kx, m0, smem_u32(&sm.full[s]));
        tma_load_2d(smem_u32(sm.B[s]), &tb, kx, n0, smem_u32(&sm.full[s]));
      }
      ++issued;
    }
    if (issued < nk) {
      // error: drain the copies already in flight before leaving (bounded)
      for (int kt = (issued > STAGES ? issued - STAGES : 0); kt < issued; ++kt) {
        const uint32_t bar = smem_u32(&sm.full[kt % STAGES]);
        const uint32_t ph = (uint32_t)(kt / STAGES) & 1u;
        for (long long i = 0; i < kSpinLimit && !mbar_try(bar, ph); ++i) {
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    constexpr uint32_t idesc = F16 ? f16_idesc(BM, BN) : tf32_idesc(BM, BN);
    bool ok = true;
    for (int kt = 0; kt < nk && ok; ++kt) {
      const int s = kt % STAGES;
      const uint32_t ph = (uint32_t)(kt / STAGES) & 1u;
      if (!mbar_wait(smem_u32(SPLIT ? &sm.conv[s] : &sm.full[s]), ph, err)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t abase = smem_u32(sm.A[s]), bbase = smem_u32(sm.B[s]);
#pragma unroll
      for (int kk = 0; kk < BK / 8; ++kk) {
        const uint64_t ad = sw128_desc(abase + kk * 32);
        const uint64_t bd = sw128_desc(bbase + kk * 32);
        uint32_t acc = (kt | kk) ? 1u : 0u;
        if (SPLIT) {
          const uint64_t adl = sw128_desc(smem_u32(sm.Alo[s]) + kk * 32);
          const uint64_t bdl = sw128_desc(smem_u32(sm.Blo[s]) + kk * 32);
          asm volatile(
              "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
              "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
              "l"(adl), "l"(bd), "r"(idesc), "r"(acc));
          asm volatile(
              "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
              "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
              "l"(ad), "l"(bdl), "r"(idesc), "r"(1u));
          acc = 1u;
        }
        if constexpr (F16)
          asm volatile(
              "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
        else
          asm volatile(
              "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
              "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&sm.empty[s]))
                   : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(&sm.done))
                 : "memory");
  } else if (SPLIT && warp >= 2) {
    // split each landed stage into hi (in place) and lo tiles
    const int ct = threadIdx.x - 64;
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % STAGES;
      const uint32_t ph = (uint32_t)(kt / STAGES) & 1u;
      if (!mbar_wait(smem_u32(&sm.full[s]), ph, err)) break;
      tf32_split(sm.A[s], sm.Alo[s], BM * BK, ct, 64);
      tf32_split(sm.B[s], sm.Blo[s], BN * BK, ct, 64);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(smem_u32(&sm.conv[s]));
    }
  }
  __syncwarp();
  // epilogue: warp w owns TMEM lanes (rows) 32w .. 32w + 31
  bool have = nk > 0 && mbar_wait(smem_u32(&sm.done), 0u, err);
  have = __all_sync(0xffffffffu, have && !*(volatile int*)err);  // warp-uniform for tcgen05.ld
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int row = m0 + warp * 32 + lane;
  if (have) {
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 32) {
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
          "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
            "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
            "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (mode == 2) {
        // transposed store: consecutive lanes (rows) are consecutive addresses
        if (row < M)
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int col = n0 + c0 + j;
            if (col < N) C[(int64_t)col * ldc + row] = __uint_as_float(v[j]);
          }
      } else {
        // row-major C: stage the warp's 32 x 32 block in shared memory so that
        // each store instruction covers 32 consecutive columns of one row
        float(*st)[33] = sm.stage[warp];
#pragma unroll
        for (int j = 0; j < 32; ++j) st[lane][j] = __uint_as_float(v[j]);
        __syncwarp();
        const int col = n0 + c0 + lane;
        const bool cok = col < N;
        if (F16 && mode == 3) {
          double cv[32];
#pragma unroll
          for (int rr = 0; rr < 32; ++rr) {
            const int r = m0 + warp * 32 + rr;
            cv[rr] = (r < M && cok) ? C64[(int64_t)r * ldc + col] : 0.0;
          }
#pragma unroll
          for (int rr = 0; rr < 32; ++rr) {
            const int r = m0 + warp * 32 + rr;
            if (r < M && cok) C64[(int64_t)r * ldc + col] = fma(scale64, (double)st[rr][lane], cv[rr]);
          }
        } else if (mode == 1) {
          // all 32 rows' loads in flight before the first use
          float cv[32];
#pragma unroll
          for (int rr = 0; rr < 32; ++rr) {
            const int r = m0 + warp * 32 + rr;
            cv[rr] = (r < M && cok) ? C[(int64_t)r * ldc + col] : 0.f;
          }
#pragma unroll
          for (int rr = 0; rr < 32; ++rr) {
            const int r = m0 + warp * 32 + rr;
            if (r < M && cok) C[(int64_t)r * ldc + col] = cv[rr] - st[rr][lane];
          }
        } else {
#pragma unroll
          for (int rr = 0; rr < 32; ++rr) {
            const int r = m0 + warp * 32 + rr;
            if (r < M && cok) C[(int64_t)r * ldc + col] = st[rr][lane];
          }
        }
        __syncwarp();
      }
    }
  } else if (nk == 0 && row < M) {
    for (int j = 0; j < BN; ++j) {
      const int col = n0 + j;
      if (col < N) {
        if (mode == 0) C[(int64_t)row * ldc + col] = 0.f;
        else if (mode == 2) C[(int64_t)col * ldc + row] = 0.f;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN < 32 ? 32 : BN));
  }
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Resolved once per process (thread-safe static initialisation).
EncodeTiled encoder() {
  static const EncodeTiled fn = []() -> EncodeTiled {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return (EncodeTiled)p;
    cudaGetLastError();
    return nullptr;
  }();
  return fn;
}

// 2-D FP32 tensor map over a row-major (rows x cols) matrix with row stride
// ld elements; box = box_rows x 32 columns, 128-byte swizzle.
bool make_map(CUtensorMap* map, const float* base, int64_t rows, int64_t cols, int64_t ld, int box_rows) {
  EncodeTiled fn = encoder();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * sizeof(float))};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)base, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 3-D FP16 tensor map over a stack of ns row-major (rows x cols) matrices,
// row stride ld elements, matrix stride mstride elements; box = box_rows x 64
// columns (128 bytes) of one matrix, 128-byte swizzle; reads outside fill
// with zeros.
bool make_map_f16_3d(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld, int64_t mstride,
                     int ns, int box_rows) {
  EncodeTiled fn = encoder();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)ns};
  cuuint64_t strides[2] = {(cuuint64_t)(ld * 2), (cuuint64_t)(mstride * 2)};
  cuuint32_t box[3] = {(cuuint32_t)(2 * BK), (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, (void*)base, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// 2-D FP64 tensor map over a row-major rows x cols matrix (row stride ld
// elements, a multiple of 2), box = box_rows x box_cols, no swizzle, zero
// fill outside the matrix.  False when the CUDA driver's cuTensorMapEncodeTiled is missing or
// the encoding is refused.
bool ski_tmap_f64_2d(CUtensorMap* map, const double* base, int64_t rows, int64_t cols, int64_t ld, int box_rows,
                     int box_cols) {
  EncodeTiled fn = encoder();
  if (!fn || (ld & 1) || ((uintptr_t)base & 15)) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * sizeof(double))};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  const bool ok = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, (void*)base, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  cudaGetLastError();
  return ok;
}

namespace {

template <int BN, int STAGES, bool SPLIT>
ski_status launch(const float* A, int64_t lda, const float* B, int64_t ldb, int M, int N, int K, float* C,
                  int64_t ldc, int mode, int splits, int64_t c_zstride, int* err, cudaStream_t st) {
  CUtensorMap ta, tb;
  if (!make_map(&ta, A, M, K, lda, BM) || !make_map(&tb, B, N, K, ldb, BN)) return SKI_ECUDA;
  const size_t smem = sizeof(TcSmem<BN, STAGES, SPLIT>) + 1024;
  static_assert(sizeof(TcSmem<BN, STAGES, SPLIT>) + 1024 <= 227 * 1024, "shared memory");
  SKI_CUDA_TRY(ski_attr_once((const void*)k_gemm_tc<BN, STAGES, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              [&] { return (int)smem; }));
  const int kchunk = (int)ski_round_up(ski_cdiv(K, splits), BK);
  dim3 grid((unsigned)ski_cdiv(M, BM), (unsigned)ski_cdiv(N, BN), (unsigned)splits);
  k_gemm_tc<BN, STAGES, SPLIT><<<grid, NTHR, smem, st>>>(ta, tb, M, N, K, kchunk, C, ldc, c_zstride, mode, err,
                                                          nullptr, 0.0, TcPairs{});
  SKI_LAUNCH_CHECK();
  return SKI_OK;
}

template <bool SPLIT>
ski_status dispatch(const float* A, int64_t lda, const float* B, int64_t ldb, int M, int N, int K, float* C,
                    int64_t ldc, int mode, int splits, int64_t c_zstride, int* err, cudaStream_t st) {
  // deep K (the V^T C products): 4-stage ring; K <= 64 (the rank-32 update):
  // 2 stages, leaving room for two CTAs (and their TMEM) per SM.  The split
  // form doubles the tiles, so its 256-wide tiles keep 2 stages.
  const bool shallow = ski_cdiv(K, splits) <= 2 * BK;
  if (N <= 32)
    return shallow ? launch<32, 2, SPLIT>(A, lda, B, ldb, M, N, K, C, ldc, mode, splits, c_zstride, err, st)
                   : launch<32, 4, SPLIT>(A, lda, B, ldb, M, N, K, C, ldc, mode, splits, c_zstride, err, st);
  if (N <= 64) return launch<64, 4, SPLIT>(A, lda, B, ldb, M, N, K, C, ldc, mode, splits, c_zstride, err, st);
  if (shallow || SPLIT)
    return launch<256, 2, SPLIT>(A, lda, B, ldb, M, N, K, C, ldc, mode, splits, c_zstride, err, st);
  return launch<256, SPLIT ? 2 : 4, SPLIT>(A, lda, B, ldb, M, N, K, C, ldc, mode, splits, c_zstride, err, st);
}

}  // namespace

// D = A B^T (TF32 tensor cores, FP32 accumulate).  A: M x K, B: N x K, both
// row-major (K contiguous) with row strides lda, ldb that are multiples of 4
// and 16-byte aligned bases.  mode 0 stores C = D, 1 subtracts C -= D, 2
// stores the transpose; mode | 4 computes only the tiles that meet the upper
// triangle of C (for a symmetric product whose lower part is not used).  splits > 1 splits K, writing partials at
// C + z * c_zstride (modes 0 and 2 only).
ski_status ski_gemm_tf32(const float* A, int64_t lda, const float* B, int64_t ldb, int64_t M, int64_t N, int64_t K,
                         float* C, int64_t ldc, int mode, int splits, int64_t c_zstride, int* err, cudaStream_t st,
                         bool split3) {
  if (M <= 0 || N <= 0) return SKI_OK;
  if ((lda & 3) || (ldb & 3) || ((uintptr_t)A & 15) || ((uintptr_t)B & 15)) return SKI_EINVAL;
  if (M > INT32_MAX || N > INT32_MAX || K > INT32_MAX) return SKI_EINVAL;
  if (split3)
    return dispatch<true>(A, lda, B, ldb, (int)M, (int)N, (int)K, C, ldc, mode, splits, c_zstride, err, st);
  return dispatch<false>(A, lda, B, ldb, (int)M, (int)N, (int)K, C, ldc, mode, splits, c_zstride, err, st);
}

// C64 += scale * sum over the pairs p of S[pr.a[p]] S[pr.b[p]]^T, S a stack
// of ns FP16 matrices (rows x K each, row-major and K-contiguous; row stride
// lds, a multiple of 8; matrix stride sstride; 16-byte aligned base),
// multiplied on the tensor cores (kind::f16) with one FP32 accumulator for
// all the pairs, then scaled and added to the FP64 C64 (rows x rows) in the
// epilogue.  The accumulation is exact when the operands are integers and
// every partial sum stays below 2^24 in magnitude.  upper: only the tiles
// that meet the upper triangle.
ski_status ski_gemm_f16_pairs_f64acc(const void* S, int64_t lds, int64_t sstride, int ns, int64_t rows, int64_t K,
                                     const TcPairs& pr, double* C64, int64_t ldc, double scale, bool upper, int* err,
                                     cudaStream_t st) {
  if (rows <= 0 || pr.n <= 0) return SKI_OK;
  if (pr.n > kTcMaxPairs || ns < 1) return SKI_EINVAL;
  for (int p = 0; p < pr.n; ++p)
    if (pr.a[p] < 0 || pr.a[p] >= ns || pr.b[p] < 0 || pr.b[p] >= ns) return SKI_EINVAL;
  if ((lds & 7) || (sstride & 7) || ((uintptr_t)S & 15)) return SKI_EINVAL;
  if (rows > INT32_MAX || K > INT32_MAX) return SKI_EINVAL;
  constexpr int BNF = 256, STF = 4;
  CUtensorMap ta, tb;
  if (!make_map_f16_3d(&ta, S, rows, K, lds, sstride, ns, BM) || !make_map_f16_3d(&tb, S, rows, K, lds, sstride, ns, BNF))
    return SKI_ECUDA;
  const size_t smem = sizeof(TcSmem<BNF, STF, false>) + 1024;
  static_assert(sizeof(TcSmem<BNF, STF, false>) + 1024 <= 227 * 1024, "shared memory");
  SKI_CUDA_TRY(ski_attr_once((const void*)k_gemm_tc<BNF, STF, false, true>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, [&] { return (int)smem; }));
  dim3 grid((unsigned)ski_cdiv(rows, BM), (unsigned)ski_cdiv(rows, BNF), 1);
  k_gemm_tc<BNF, STF, false, true><<<grid, NTHR, smem, st>>>(ta, tb, (int)rows, (int)rows, (int)K,
                                                              (int)ski_round_up(K, 2 * BK), nullptr, ldc, 0,
                                                              3 | (upper ? 4 : 0), err, C64, scale, pr);
  SKI_LAUNCH_CHECK();
  return SKI_OK;
}

extern "C" ski_status ski_gemm_tc_f32(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda, const float* B,
                                      int64_t ldb, float* C, int64_t ldc, int32_t subtract, int32_t passes, void* ws,
                                      size_t ws_bytes, void* stream) {
  if (M < 0 || N < 0 || K < 0 || !A || !B || !C || !ws || ws_bytes < sizeof(int)) return SKI_EINVAL;
  if (passes != 1 && passes != 3) return SKI_EINVAL;
  if (lda < K || ldb < K || ldc < N) return SKI_EINVAL;
  cudaStream_t st = ski_stream(stream);
  int* err = (int*)ws;
  SKI_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
  SKI_TRY(ski_gemm_tf32(A, lda, B, ldb, M, N, K, C, ldc, subtract ? 1 : 0, 1, 0, err, st, passes == 3));
  int h = 0;
  SKI_CUDA_TRY(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  SKI_CUDA_TRY(cudaStreamSynchronize(st));
  return h ? SKI_ETIMEOUT : SKI_OK;
}
