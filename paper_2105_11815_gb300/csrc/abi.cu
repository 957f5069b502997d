// C ABI of the library (include/skills.h): argument checks, workspace
// planning and the stage order of Algorithm 1.  Every arithmetic step runs in
// the kernels of the other translation units; this file only sequences them.
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "hash.cuh"
#include "lsqr_impl.cuh"
#include "sketch_impl.cuh"

#include <atomic>

static thread_local cudaError_t g_last_cuda = cudaSuccess;
static std::atomic<long long> g_launches{0};
void ski_note_cuda_error(cudaError_t e) { g_last_cuda = e; }
static thread_local long long t_launches = 0;  // this thread's launches (graph recording)
void ski_count_launch() {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  ++t_launches;
}
static void ski_count_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

extern "C" int64_t ski_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

extern "C" void ski_opts_default(ski_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->seed = 0;
  o->s = 1;
  o->m = 0;
  o->premix = 0;
  o->n_pad = 0;
  o->sketch_dtype = SKI_F64;
  o->qr_dtype = SKI_F64;
  o->tau_a = 1e-8;
  o->tau_r = 1e-6;
  o->tol = 0.0;
  o->rcond = 1e-12;
  o->perturb = 0.0;
  o->it_max = 10000;
}

extern "C" const char* ski_status_string(int32_t st) {
  switch (st) {
    case SKI_OK: return "SKI_OK";
    case SKI_EINVAL: return "SKI_EINVAL: invalid argument";
    case SKI_ENOMEM: return "SKI_ENOMEM: workspace too small";
    case SKI_ECUDA: return "SKI_ECUDA: CUDA call failed";
    case SKI_ENONFINITE: return "SKI_ENONFINITE: NaN or Inf encountered";
    case SKI_ESINGULAR: return "SKI_ESINGULAR: R fails the rank rule";
    case SKI_ENOCONV: return "SKI_ENOCONV: iteration limit reached";
    case SKI_ETIMEOUT: return "SKI_ETIMEOUT: bounded device wait expired";
    default: return "unknown ski_status";
  }
}

extern "C" int32_t ski_version(void) { return 100; }

extern "C" int32_t ski_last_cuda_error(void) { return (int32_t)g_last_cuda; }

namespace {
int64_t mixed_lsqr_budget(int64_t m, int64_t d, double tau_r);
}
extern "C" int64_t ski_mixed_lsqr_budget(int64_t m, int64_t d, double tau_r) { return mixed_lsqr_budget(m, d, tau_r); }

// ------------------------------------------------------------ validation
static bool pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }
static int64_t next_pow2(int64_t v) {
  int64_t p = 1;
  while (p < v) p <<= 1;
  return p;
}
static bool dtype_ok(int32_t t) { return t == SKI_F64 || t == SKI_F32 || t == SKI_BF16; }
static size_t dtype_size(int32_t t) { return t == SKI_F64 ? 8 : ((t == SKI_F32 || t == SKI_TF32) ? 4 : 2); }
// storage type of a QR precision: TF32 factors FP32 data
static int32_t qr_storage(int32_t t) { return t == SKI_F64 ? SKI_F64 : SKI_F32; }

static ski_status check_matrix(const ski_matrix* A) {
  if (!A) return SKI_EINVAL;
  if (A->n < 1 || A->d < 1) return SKI_EINVAL;
  if (A->kind == SKI_DENSE) {
    if (!A->val || A->ld < A->d) return SKI_EINVAL;
  } else if (A->kind == SKI_CSR) {
    if (!A->rowptr || !A->colidx || A->nnz < 0 || (A->nnz > 0 && !A->val)) return SKI_EINVAL;
    if (A->n >= (1ll << 31) || A->d >= (1ll << 31)) return SKI_EINVAL;
  } else {
    return SKI_EINVAL;
  }
  return SKI_OK;
}

static bool launch_opts_ok(const ski_opts* o) {
  return o->lsqr_pass >= 0 && o->lsqr_pass <= 5 && o->lsqr_ctas >= 0 && (o->graphs == 0 || o->graphs == 1) &&
         (o->batch_lsqr == 0 || o->batch_lsqr == 1);
}

static ski_status check_sketch_opts(const ski_matrix* A, const ski_opts* o) {
  if (!o) return SKI_EINVAL;
  if (o->hash_kind < 0 || o->hash_kind > 2) return SKI_EINVAL;
  if (o->s < 1 || o->s > 64 || o->m < (o->hash_kind ? 1 : o->s) || o->m >= (1ll << 31)) return SKI_EINVAL;
  // the sampling sketch S_s (Eq. SR-DHT): one 1 per row, dense A, no s, and
  // with the Hartley premix or none
  if (o->hash_kind == 2 && (o->s != 1 || A->kind != SKI_DENSE || o->premix == 1 || o->row_offset != 0))
    return SKI_EINVAL;
  if (o->premix_slab < 0 || o->streams < 0) return SKI_EINVAL;
  if (!launch_opts_ok(o)) return SKI_EINVAL;
  if (!dtype_ok(o->sketch_dtype)) return SKI_EINVAL;
  if (o->premix < 0 || o->premix > 2) return SKI_EINVAL;
  if (o->premix) {
    if (A->kind != SKI_DENSE) return SKI_EINVAL;
    if (o->premix == 1 && o->n_pad != 0 && (!pow2(o->n_pad) || o->n_pad < A->n)) return SKI_EINVAL;
    if (o->premix == 2 && o->n_pad != 0 && (!ski_dht_length_ok(o->n_pad) || o->n_pad < A->n)) return SKI_EINVAL;
    if (o->row_offset != 0) return SKI_EINVAL;  // the premix mixes every row of A: no row block premixes alone
  }
  if (o->row_offset < 0 || o->row_offset + A->n >= (1ll << 62)) return SKI_EINVAL;
  const int64_t rows = o->premix == 2 ? (o->n_pad ? o->n_pad : ski_dht_length(A->n))
                       : o->premix ? (o->n_pad ? o->n_pad : next_pow2(A->n)) : A->n;
  if (rows * (int64_t)o->s >= (1ll << 31) || rows >= (1ll << 31)) return SKI_EINVAL;
  return SKI_OK;
}

// CTAs of the LSQR passes (row tiles of ceil(n / ctas) rows): the option, or
// the default; at least n / 16384 (the register-blocked pass keeps a tile's
// row values in shared memory), at most n and 65535.
static int lsqr_ctas(int64_t n, const ski_opts* o) {
  if (!o || o->lsqr_ctas <= 0) return ski_fused_ctas(n);
  int64_t c = std::min<int64_t>({(int64_t)o->lsqr_ctas, std::max<int64_t>(1, n), 65535});
  return (int)std::max<int64_t>(c, ski_cdiv(n, 16384));
}

// Rows of the premixed matrix: n_pad, else the next power of two (Def. 8)
// or the DHT length (Eq. HR-DHT: n itself when its prime factors are <= 13).
static int64_t eff_npad(const ski_matrix* A, const ski_opts* o) {
  if (o->premix == 2) return o->n_pad ? o->n_pad : ski_dht_length(A->n);
  return o->premix ? (o->n_pad ? o->n_pad : next_pow2(A->n)) : 0;
}

// ------------------------------------------------------------ sketch stage
// Columns per premix slab.  With o->premix_slab = w > 0 (a multiple of 32, at
// most 128) the premix and the hash gather run slab by slab over the columns:
// the pass-1 intermediate and Y of one slab (n_pad rows each) can stay in the
// 126 MiB L2 (w = 64 at n_pad = 65536), so only A is read from HBM and only
// [SA | Sb] written.  0 (the default) transforms all columns at once: at
// 50000 x 4000 the 63 slabs' 189 launches, each too small to hide its load
// latency, took 4.6 ms against 3.1 ms for the full-width passes.
static int64_t premix_slab_cols(int64_t n_pad, int64_t ncols, int32_t pdt, int32_t fixed) {
  (void)n_pad;
  (void)pdt;
  const int64_t full = ski_round_up(ncols, 32);
  if (fixed <= 0) return full;
  const int64_t w = std::min<int64_t>(128, std::max<int64_t>(32, fixed / 32 * 32));
  return std::min<int64_t>(w, full);
}

// The FP64 premix over all columns at once leaves its output as int64 planes
// with per-tile exponents, which the FP64 hash gather reads directly.
static bool premix_q_path(int32_t pdt, int64_t ncols, int64_t w, const ski_opts* o) {
  return pdt == SKI_F64 && o->sketch_dtype == SKI_F64 && w >= ncols && (w > 128 || o->premix_slab <= 0);
}

// Scratch layout: [bucket lists][premix Y slab][premix intermediates]
static size_t sketch_scratch_bytes(const ski_matrix* A, int32_t with_b, const ski_opts* o, int64_t* ldy_out) {
  const int64_t ncols = A->d + (with_b ? 1 : 0);
  const int64_t rows = o->premix ? eff_npad(A, o) : A->n;
  SkiArena ar{nullptr, 0, 0, true};
  // (the sampling sketch needs no bucket lists: one aligned block keeps the
  // size query nonzero, 0 being its error value)
  ar.take<char>(o->hash_kind != 2 ? ski_bucket_ws_bytes(rows, o->s, o->m) : 1);
  int64_t ldy = 0;
  if (o->premix == 2) {
    const int32_t pdt = o->sketch_dtype == SKI_F64 ? SKI_F64 : SKI_F32;
    ldy = ski_round_up(ncols, 4);
    ar.take<char>(dtype_size(pdt) * rows * ldy);
    ar.take<char>(ski_dht_ws_bytes(A->n, ncols, rows, pdt));
  } else if (o->premix) {
    const int32_t pdt = o->sketch_dtype == SKI_F64 ? SKI_F64 : SKI_F32;
    ldy = premix_slab_cols(rows, ncols, pdt, o->premix_slab);
    // the full-width FP64 premix hands its int64 planes to the gather: no Y
    if (!premix_q_path(pdt, ncols, ldy, o)) ar.take<char>(dtype_size(pdt) * rows * ldy);
    ar.take<char>(ski_premix_ws_bytes(A->n, ldy, rows, pdt));
  }
  if (ldy_out) *ldy_out = ldy;
  return ar.off;
}

static ski_status sketch_run(const ski_matrix* A, const double* b, const ski_opts* o, void* SA, int64_t ld_sa,
                             char* scratch, size_t scratch_bytes, cudaStream_t st, cudaEvent_t e_bk = nullptr,
                             cudaEvent_t e_pm = nullptr, int* err_flag = nullptr) {
  const int64_t ncols = A->d + (b ? 1 : 0);
  const int64_t rows = o->premix ? eff_npad(A, o) : A->n;
  SkiArena ar{scratch, scratch_bytes, 0, false};
  const bool sample = o->hash_kind == 2;
  SkiBuckets bk{};
  if (sample) {
    ar.take<char>(1);
  } else {
    const size_t bkb = ski_bucket_ws_bytes(rows, o->s, o->m);
    char* bkws = ar.take<char>(bkb);
    if (!ar.ok() || !bkws) return SKI_ENOMEM;
    SkiArena bar{bkws, bkb, 0, false};
    SKI_TRY(ski_build_buckets(o->seed, o->s, o->hash_kind, o->m, rows, bar, st, &bk, o->row_offset));
  }
  if (e_bk) SKI_CUDA_TRY(cudaEventRecord(e_bk, st));
  const double inv_sqrt_s = 1.0 / sqrt((double)o->s);
  if (o->premix == 2) {
    // Hartley premix F D into Y, then the s-hashing gather or the sampling
    const int32_t pdt = o->sketch_dtype == SKI_F64 ? SKI_F64 : SKI_F32;
    const int64_t ldy = ski_round_up(ncols, 4);
    void* Y = ar.take<char>(dtype_size(pdt) * rows * ldy);
    const size_t dwb = ski_dht_ws_bytes(A->n, ncols, rows, pdt);
    char* dws = ar.take<char>(dwb);
    if (!ar.ok() || !dws) return SKI_ENOMEM;
    SkiArena dar{dws, dwb, 0, false};
    SKI_TRY(ski_dht_premix(A->val, A->ld, A->n, A->d, b, o->seed, rows, pdt, Y, ldy, dar, st));
    if (e_pm) SKI_CUDA_TRY(cudaEventRecord(e_pm, st));
    if (sample) return ski_sample_rows(o->seed, o->m, rows, Y, pdt, ldy, ncols, nullptr, o->sketch_dtype, SA, ld_sa, st);
    if (pdt == SKI_F64)
      return ski_gather_dense((const double*)Y, ldy, rows, ncols, nullptr, bk, inv_sqrt_s, SKI_F64, SA, ld_sa, st);
    return ski_gather_dense_f32in((const float*)Y, ldy, ncols, bk, inv_sqrt_s, o->sketch_dtype, SA, ld_sa, st);
  }
  if (!o->premix) {
    if (sample) {
      if (e_pm) SKI_CUDA_TRY(cudaEventRecord(e_pm, st));
      return ski_sample_rows(o->seed, o->m, A->n, A->val, SKI_F64, A->ld, A->d, b, o->sketch_dtype, SA, ld_sa, st);
    }
    if (e_pm) SKI_CUDA_TRY(cudaEventRecord(e_pm, st));
    if (A->kind == SKI_DENSE)
      return ski_gather_dense(A->val, A->ld, A->n, A->d, b, bk, inv_sqrt_s, o->sketch_dtype, SA, ld_sa, st);
    return ski_gather_csr(A, b, bk, inv_sqrt_s, o->sketch_dtype, SA, ld_sa, st);
  }
  const int32_t pdt = o->sketch_dtype == SKI_F64 ? SKI_F64 : SKI_F32;
  if (pdt == SKI_F64 && o->sketch_dtype != SKI_F64) return SKI_EINVAL;
  const int64_t w = premix_slab_cols(rows, ncols, pdt, o->premix_slab);
  const bool qpath = premix_q_path(pdt, ncols, w, o);
  void* Y = qpath ? nullptr : ar.take<char>(dtype_size(pdt) * rows * w);
  const size_t pwb = ski_premix_ws_bytes(A->n, w, rows, pdt);
  char* pws = ar.take<char>(pwb);
  if (!ar.ok() || !pws) return SKI_ENOMEM;
  SkiArena par{pws, pwb, 0, false};
  SkiPremixPlan plan;
  SKI_TRY(ski_premix_plan(A->n, w, rows, pdt, o->seed, par, st, &plan, err_flag));
  const double scale = plan.residual_scale * inv_sqrt_s;
  if (qpath) {
    // all columns at once, FP64: premix into block-fixed-point planes, then
    // the hash gather straight from them
    SkiPremixQ yq;
    SKI_TRY(ski_premix_cols_q(plan, A->val, A->ld, A->d, b, &yq, st));
    if (e_pm) SKI_CUDA_TRY(cudaEventRecord(e_pm, st));
    return ski_gather_q(yq, ncols, bk, scale, (double*)SA, ld_sa, st);
  }
  if (w >= ncols && (w > 128 || o->premix_slab <= 0)) {
    // all columns at once: premix into Y, then the full-width hash gather
    SKI_TRY(ski_premix_cols(plan, A->val, A->ld, A->d, b, Y, w, st));
    if (e_pm) SKI_CUDA_TRY(cudaEventRecord(e_pm, st));
    if (pdt == SKI_F64)
      return ski_gather_dense((const double*)Y, w, rows, ncols, nullptr, bk, scale, SKI_F64, SA, ld_sa, st);
    return ski_gather_dense_f32in((const float*)Y, w, ncols, bk, scale, o->sketch_dtype, SA, ld_sa, st);
  }
  // column slabs: premix then hash-gather each slab while it is in L2
  const size_t osz = dtype_size(o->sketch_dtype);
  for (int64_t c0 = 0; c0 < ncols; c0 += w) {
    const int64_t cw = std::min<int64_t>(w, ncols - c0);
    const int64_t da = std::max<int64_t>(0, std::min<int64_t>(cw, A->d - c0));  // columns of A in the slab
    const double* bs = (b && c0 + cw > A->d) ? b : nullptr;                      // b is column d
    SKI_TRY(ski_premix_cols(plan, A->val + std::min<int64_t>(c0, A->d), A->ld, da, bs, Y, w, st));
    SKI_TRY(ski_gather_slab(Y, pdt, w, cw, bk, scale, o->sketch_dtype, (char*)SA + c0 * osz, ld_sa, st));
  }
  if (e_pm) SKI_CUDA_TRY(cudaEventRecord(e_pm, st));
  return SKI_OK;
}

extern "C" size_t ski_sketch_workspace_size(const ski_matrix* A, int32_t with_b, const ski_opts* o) {
  if (check_matrix(A) != SKI_OK || check_sketch_opts(A, o) != SKI_OK) return 0;
  return sketch_scratch_bytes(A, with_b, o, nullptr);
}

extern "C" ski_status ski_sketch_hash(const ski_matrix* A, const double* b, const ski_opts* o, void* SA,
                                      int64_t ld_sa, void* ws, size_t ws_bytes, void* stream) {
  SKI_TRY(check_matrix(A));
  SKI_TRY(check_sketch_opts(A, o));
  if (!SA || ld_sa < A->d + (b ? 1 : 0)) return SKI_EINVAL;
  const size_t need = sketch_scratch_bytes(A, b != nullptr, o, nullptr);
  if (ws_bytes < need || (!ws && need)) return SKI_ENOMEM;
  return sketch_run(A, b, o, SA, ld_sa, (char*)ws, ws_bytes, ski_stream(stream));
}

extern "C" size_t ski_premix_workspace_size(const ski_matrix* A, int32_t with_b, const ski_opts* o) {
  if (check_matrix(A) != SKI_OK || !o || A->kind != SKI_DENSE) return 0;
  const int32_t pdt = o->sketch_dtype == SKI_F64 ? SKI_F64 : SKI_F32;
  if (o->premix == 2) {
    const int64_t rows = eff_npad(A, o);
    if (!ski_dht_length_ok(rows) || rows < A->n) return 0;
    return ski_dht_ws_bytes(A->n, A->d + (with_b ? 1 : 0), rows, pdt);
  }
  const int64_t rows = o->n_pad ? o->n_pad : next_pow2(A->n);
  return ski_premix_ws_bytes(A->n, A->d + (with_b ? 1 : 0), rows, pdt);
}

extern "C" ski_status ski_premix(const ski_matrix* A, const double* b, const ski_opts* o, void* Y, int64_t ld_y,
                                 void* ws, size_t ws_bytes, void* stream) {
  SKI_TRY(check_matrix(A));
  if (!o || A->kind != SKI_DENSE || !Y) return SKI_EINVAL;
  if (o->sketch_dtype != SKI_F64 && o->sketch_dtype != SKI_F32) return SKI_EINVAL;
  if (o->premix == 2) {  // the Hartley premix F D of Eq. HR-DHT
    const int64_t rows = eff_npad(A, o);
    const int64_t ncols = A->d + (b ? 1 : 0);
    if (!ski_dht_length_ok(rows) || rows < A->n || ld_y < ncols) return SKI_EINVAL;
    const size_t need = ski_dht_ws_bytes(A->n, ncols, rows, o->sketch_dtype);
    if (ws_bytes < need || !ws) return SKI_ENOMEM;
    SkiArena ar{(char*)ws, ws_bytes, 0, false};
    return ski_dht_premix(A->val, A->ld, A->n, A->d, b, o->seed, rows, o->sketch_dtype, Y, ld_y, ar,
                          ski_stream(stream));
  }
  const int64_t rows = o->n_pad ? o->n_pad : next_pow2(A->n);
  if (!pow2(rows) || rows < A->n) return SKI_EINVAL;
  const int64_t ncols = A->d + (b ? 1 : 0);
  if (ld_y < ncols) return SKI_EINVAL;
  const size_t need = ski_premix_ws_bytes(A->n, ncols, rows, o->sketch_dtype);
  if (ws_bytes < need || !ws) return SKI_ENOMEM;
  SkiArena ar{(char*)ws, ws_bytes, 0, false};
  double resid;
  cudaStream_t st = ski_stream(stream);
  SKI_TRY(ski_premix_run(A->val, A->ld, A->n, A->d, b, o->seed, rows, o->sketch_dtype, Y, ld_y, ar, st, &resid));
  if (resid != 1.0) {  // odd log2(n_pad): the last factor 2^{-1/2} of n_pad^{-1/2}
    if (o->sketch_dtype == SKI_F64) return ski_scale_launch(rows, ncols, (double*)Y, ld_y, resid, st);
    return ski_scale_f32_launch(rows, ncols, (float*)Y, ld_y, (float)resid, st);
  }
  return SKI_OK;
}

// ------------------------------------------------------------ QR stage
extern "C" size_t ski_precondition_workspace_size(int64_t m, int64_t d, int32_t with_rhs, int32_t sa_dtype) {
  if (m < d || d < 1) return 0;
  return ski_qr_ws_bytes(m, d + (with_rhs ? 1 : 0), qr_storage(sa_dtype));
}

static ski_status rank_from_diag(int64_t d, const double* R, int64_t ldr, double rcond, cudaStream_t st, int32_t* rank,
                                 bool* nonfinite, double* ratio = nullptr) {
  std::vector<double> diag(d);
  // strided gather of the diagonal: d small copies would be slow; copy rows' diagonal via 2D memcpy
  SKI_CUDA_TRY(cudaMemcpy2DAsync(diag.data(), sizeof(double), R, (ldr + 1) * sizeof(double), sizeof(double), d,
                                 cudaMemcpyDeviceToHost, st));
  SKI_CUDA_TRY(cudaStreamSynchronize(st));
  *nonfinite = false;
  int32_t p = 0;
  const double r11 = fabs(diag[0]);
  for (int64_t q = 0; q < d; ++q) {
    if (!isfinite(diag[q])) *nonfinite = true;
  }
  if (r11 > 0) {
    while (p < d && fabs(diag[p]) >= rcond * r11) ++p;
  }
  *rank = p;
  if (ratio) {
    double mx = 0.0, mn = INFINITY;
    for (int64_t q = 0; q < d; ++q) {
      mx = std::max(mx, fabs(diag[q]));
      mn = std::min(mn, fabs(diag[q]));
    }
    *ratio = mn > 0.0 ? mx / mn : INFINITY;
  }
  return SKI_OK;
}

extern "C" ski_status ski_precondition(int64_t m, int64_t d, int32_t with_rhs, void* SA, int64_t ld_sa,
                                       int32_t sa_dtype, double* R, int64_t ldr, double* qtsb, int32_t* rank,
                                       const ski_opts* o, void* ws, size_t ws_bytes, void* stream) {
  if (d < 1 || m < d || !SA || !R || ldr < d || ld_sa < d + (with_rhs ? 1 : 0)) return SKI_EINVAL;
  if (sa_dtype != SKI_F64 && sa_dtype != SKI_F32 && sa_dtype != SKI_TF32) return SKI_EINVAL;
  const size_t need = ski_qr_ws_bytes(m, d + (with_rhs ? 1 : 0), qr_storage(sa_dtype));
  if (ws_bytes < need || !ws) return SKI_ENOMEM;
  cudaStream_t st = ski_stream(stream);
  SkiArena ar{(char*)ws, ws_bytes, 0, false};
  SKI_TRY(ski_qr_run(m, d, with_rhs, SA, ld_sa, sa_dtype, R, ldr, with_rhs ? qtsb : nullptr, ar, st));
  if (rank) {
    bool nf;
    SKI_TRY(rank_from_diag(d, R, ldr, o ? o->rcond : 1e-12, st, rank, &nf));
    if (nf) return SKI_ENONFINITE;
  }
  return SKI_OK;
}

extern "C" size_t ski_trinv_workspace_size(int64_t d, int32_t dtype) {
  if (d < 1) return 0;
  return ski_trinv_ws_bytes(d, dtype);
}

extern "C" ski_status ski_trinv(int64_t d, const double* R, int64_t ldr, double* M, double* Mt, int64_t ldm,
                                int32_t dtype, double perturb, void* ws, size_t ws_bytes, void* stream) {
  if (d < 1 || !R || !M || ldr < d || ldm < d) return SKI_EINVAL;
  if (dtype != SKI_F64 && dtype != SKI_F32) return SKI_EINVAL;
  const size_t need = ski_trinv_ws_bytes(d, dtype);
  if (ws_bytes < need || !ws) return SKI_ENOMEM;
  SkiArena ar{(char*)ws, ws_bytes, 0, false};
  return ski_trinv_run(d, R, ldr, M, Mt, ldm, dtype, perturb, ar, ski_stream(stream));
}

// ------------------------------------------------------------ solve
namespace {

// The sum over the processes of a row-block solve (ski_solve_rowblock), or
// none for a whole A.
struct ShardHook {
  ski_allreduce_fn fn;
  void* ctx;
  ski_status sum(void* buf, int64_t count, int32_t dtype, cudaStream_t st) const {
    return fn(buf, count, dtype, ctx, (void*)st);
  }
};

struct SolvePlan {
  int64_t n, d, m, ncols, ld_sa, ldq_sa;
  const ShardHook* sh;  // row-block form: partial sums are summed over the processes
  int64_t dl;        // unknowns of Steps 3-5: d, or p after the column-pivoted QR
  bool pivoted;      // Step 2 took the column-pivoted QR (rank-revealing form)
  int32_t* piv;      // [d] the column of A at each pivoted position (p used)
  double* xfull;     // [d] an iterate in A's column order (zero outside V1)
  int32_t qr_dt;    // storage of the QR (F64 or F32)
  int32_t qr_prec;  // its precision (F64, F32 or TF32)
  int nblk;
  int lsqr_pass;  // variant of the dense LSQR pass (ski_opts.lsqr_pass)
  bool csr;
  // persistent
  double *R, *qtsb, *M, *Mt, *xs, *t, *v, *w, *y, *z, *p, *q, *part, *part_tt, *part_aa;
  LsqrScalars* sc;
  int* perr;  // bounded-wait flag of the premix (read after Step 2)
  double *vp, *part_vv;
  float2* A2;  // double-float copy of a dense A for the LSQR passes
  int sA;
  int64_t *colptr;
  int32_t* rowidx;
  double* cval;
  // phase region
  char* region;
  size_t region_bytes;
  void* SA;
  void* SAq;  // QR input (SA itself, or an FP32 copy of a BF16 sketch)
  char* stage;
  size_t stage_bytes;
  char* csc_tmp;
  size_t csc_tmp_bytes;
};

// Mixed form: LSQR iterations allowed with an FP32 / TF32 preconditioner
// before Steps 1-2 are redone in FP64.  Theorem 10 bounds the iterations with
// an eps-subspace embedding by (log 2 + |log tau_r|) / |log eps|, and a hashing
// sketch of m = gamma d rows embeds with eps ~ gamma^(-1/2) (m = O(d / eps^2)).
// The budget is 2.2 times that bound with eps = sqrt(d / m), and at least 150.
// At m = 2d and tau_r = 1e-10 the two coincide (an FP64-preconditioned solve
// of the dense test set takes 58 there).  A fixed 150 made every mixed solve
// with m < 1.4 d refactor in FP64 although its FP32 factor preconditioned as
// well as the FP64 one: 197 iterations against 192 at m = 1.2 d.
int64_t mixed_lsqr_budget(int64_t m, int64_t d, double tau_r) {
  constexpr double kFloor = 150.0, kCap = 4000.0;
  if (!(tau_r > 0.0 && tau_r < 1.0) || d < 1) return (int64_t)kFloor;
  if (m <= d) return (int64_t)kCap;
  const double bound = (log(2.0) - log(tau_r)) / (0.5 * log((double)m / (double)d));
  return (int64_t)std::max(kFloor, std::min(kCap, ceil(2.2 * bound)));
}
// Largest max|r_ii| / min|r_ii| of an FP32 (TF32) factor kept as the
// preconditioner: kappa(SA) u must stay well below 1 for R^{-1} to
// precondition, with u the coarser of the factorisation's unit roundoff
// (~2^-22 for the three-pass products, 2^-11 for one) and the sketch's
// (2^-9 for a BF16 SA).
// The ratio underestimates kappa: at 200000 x 4000, kappa = 1e6 it was 5.9e4
// (FP32 factor kept, 60 LSQR iterations), at kappa = 1e10 the FP32 factor's
// ratio saturated at 3.2e6 (FP64: 3.7e8).  A BF16 sketch at kappa = 1e6
// spent the 150-iteration LSQR budget before refactoring (553 ms against
// 412 ms for FP64); on the i.i.d. dense test set (ratio 1.5) it matched FP32.
double mixed_ratio_limit(int32_t qr_dtype, int32_t sketch_dtype) {
  double lim = qr_dtype == SKI_TF32 ? 0x1p7 : 0x1p19;
  if (sketch_dtype == SKI_BF16) lim = std::min(lim, 0x1p5);
  return lim;
}
// After >= 24 iterations, the Eq. TC-lsqr estimate extrapolated geometrically
// (test_k ~ rho^k from test_0 = 1) predicts more than the budget: the FP32
// preconditioner is too weak, so stop early instead of spending the budget.
bool weak_preconditioner(double test, long long iters, double tau_r, int64_t budget) {
  if (iters < 24 || !(tau_r > 0.0) || !(tau_r < 1.0)) return false;
  if (!(test < 1.0)) return true;
  if (test <= tau_r) return false;
  return (double)iters * log(tau_r) / log(test) > (double)budget;
}

// Bytes of the phase region for the sketch / QR / trinv precisions of o.
// Step 2 from the Gram matrix SA^T SA (factorization 2): of a sparse SA for
// CSR A (FP64), of the dense sketch for dense A (any QR precision)
bool gram_path(const ski_matrix* A, const ski_opts* o) {
  if (o->factorization != 2) return false;
  if (A->kind == SKI_CSR) return o->qr_dtype == SKI_F64 && o->sketch_dtype == SKI_F64;
  return true;
}
size_t gram_stage_bytes(const ski_matrix* A, const ski_opts* o) {
  if (!gram_path(A, o)) return 0;
  if (A->kind == SKI_CSR) return ski_gram_ws_bytes(A->n, A->d, A->nnz, o->s, o->m);
  return ski_gram_dense_ws_bytes(o->m, A->d, o->qr_dtype);
}
// Largest max_j sqrt(g_jj) / r_jj (g_jj = |SA_j|^2; a lower bound on the
// condition number of SA with unit columns) of a factor from the Gram matrix
// kept as the preconditioner: its relative error grows like kappa^2 u, with
// kappa that of the column-scaled SA (the Cholesky is invariant under
// power-of-two column scales), so the limit is about u^{-1/2} / 8 of the
// Gram's precision; past it Step 2 is redone by the Householder QR in the
// same precision.
double gram_ratio_limit(int32_t qr_prec) { return qr_prec == SKI_F64 ? 0x1p23 : 0x1p9; }

size_t region_need(const ski_matrix* A, const ski_opts* o) {
  const int64_t d = A->d, m = o->m, ncols = d + 1, ld_sa = ski_round_up(ncols, 4);
  const int32_t qdt = qr_storage(o->qr_dtype);
  const size_t sa_bytes = ski_round_up((int64_t)(dtype_size(o->sketch_dtype) * m * ld_sa), 256);
  const bool copy_q = dtype_size(o->sketch_dtype) != dtype_size(qdt) || o->sketch_dtype == SKI_BF16;
  const size_t saq_bytes = copy_q ? ski_round_up((int64_t)(dtype_size(qdt) * m * ld_sa), 256) : 0;
  const size_t stage = std::max({sketch_scratch_bytes(A, 1, o, nullptr), ski_qr_ws_bytes(m, ncols, qdt),
                                  gram_stage_bytes(A, o)});
  return std::max(sa_bytes + saq_bytes + stage, ski_trinv_ws_bytes(d, qdt));
}

// Points SA, SAq (the QR input), the stage scratch and the precisions at the
// region for the sketch / QR precisions of o.
void carve_region(const ski_matrix* A, const ski_opts* o, SolvePlan* P) {
  const int64_t d = A->d, m = o->m, ncols = d + 1;
  P->qr_dt = qr_storage(o->qr_dtype);
  P->qr_prec = o->qr_dtype;
  const size_t sa_bytes = ski_round_up((int64_t)(dtype_size(o->sketch_dtype) * m * P->ld_sa), 256);
  const bool copy_q = dtype_size(o->sketch_dtype) != dtype_size(P->qr_dt) || o->sketch_dtype == SKI_BF16;
  const size_t saq_bytes = copy_q ? ski_round_up((int64_t)(dtype_size(P->qr_dt) * m * P->ld_sa), 256) : 0;
  P->SA = P->region;
  P->SAq = copy_q ? (void*)(P->region + sa_bytes) : P->SA;
  P->stage = P->region + sa_bytes + saq_bytes;
  P->stage_bytes = std::max({sketch_scratch_bytes(A, 1, o, nullptr), ski_qr_ws_bytes(m, ncols, P->qr_dt),
                             gram_stage_bytes(A, o)});
  (void)d;
}

size_t plan_solve(const ski_matrix* A, const ski_opts* o, char* base, size_t cap, SolvePlan* P) {
  SkiArena ar{base, cap, 0, base == nullptr};
  const int64_t n = A->n, d = A->d, m = o->m, ncols = d + 1;
  P->n = n;
  P->d = d;
  P->m = m;
  P->ncols = ncols;
  P->csr = A->kind == SKI_CSR;
  P->qr_dt = qr_storage(o->qr_dtype);
  P->qr_prec = o->qr_dtype;
  P->ld_sa = ski_round_up(ncols, 4);
  P->nblk = lsqr_ctas(n, o);
  P->lsqr_pass = o->lsqr_pass;
  P->dl = d;
  P->pivoted = false;
  P->R = ar.take<double>(d * d);
  P->qtsb = ar.take<double>(d);
  P->piv = ar.take<int32_t>(d);
  P->xfull = ar.take<double>(d);
  P->M = ar.take<double>(d * d);
  P->Mt = ar.take<double>(d * d);
  P->xs = ar.take<double>(d);
  P->t = ar.take<double>(n);
  P->v = ar.take<double>(d);
  P->w = ar.take<double>(d);
  P->y = ar.take<double>(d);
  P->z = ar.take<double>(d);
  P->p = ar.take<double>(d);
  P->q = ar.take<double>(d + 2);  // + ||t||^2, ||A||_F^2 of the row-block form
  P->part = ar.take<double>((int64_t)P->nblk * d);
  P->part_tt = ar.take<double>(P->nblk);
  P->part_aa = ar.take<double>(P->nblk);
  P->sc = ar.take<LsqrScalars>(1);
  P->perr = ar.take<int>(1);
  P->vp = ar.take<double>(d);
  P->part_vv = ar.take<double>(ski_vv_blocks(d));
  P->A2 = P->csr ? nullptr : ar.take<float2>(n * ski_a2_ld(d));
  if (P->csr) {
    P->colptr = ar.take<int64_t>(d + 1);
    P->rowidx = ar.take<int32_t>(A->nnz);
    P->cval = ar.take<double>(A->nnz);
  } else {
    P->colptr = nullptr;
    P->rowidx = nullptr;
    P->cval = nullptr;
  }
  // phase region: max(SA [+ QR copy] + max(sketch scratch, QR ws), trinv ws, csc tmp),
  // for the requested precisions and, when the QR is not FP64, for the FP64
  // refactorisation the solve falls back to (see ski_solve)
  ski_opts o64 = *o;
  o64.sketch_dtype = SKI_F64;
  o64.qr_dtype = SKI_F64;
  const size_t cscw = P->csr ? ski_csc_ws_bytes(n, d, A->nnz) : 0;
  P->region_bytes = std::max(region_need(A, o), cscw);
  if (!P->csr && o->factorization == 1) P->region_bytes = std::max(P->region_bytes, ski_cpqr_ws_bytes(d));
  if (o->qr_dtype != SKI_F64) P->region_bytes = std::max(P->region_bytes, region_need(A, &o64));
  P->region = ar.take<char>(P->region_bytes);
  if (P->region) {
    carve_region(A, o, P);
    P->csc_tmp = P->region;
    P->csc_tmp_bytes = cscw;
  }
  return ar.off;
}

template <class TI, class TO>
__global__ void k_convert(int64_t count, const TI* __restrict__ a, TO* __restrict__ b) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < count) b[i] = SkiType<TO>::from(SkiType<TI>::to_f64(a[i]));
}

struct Events {
  cudaEvent_t e[8];
  bool ok;
  Events() : ok(true) {
    for (auto& x : e) {
      if (cudaEventCreate(&x) != cudaSuccess) ok = false;
    }
  }
  ~Events() {
    for (auto& x : e) cudaEventDestroy(x);
  }
  float ms(int a, int b) {
    float v = 0.f;
    if (cudaEventElapsedTime(&v, e[a], e[b]) != cudaSuccess) return 0.f;
    return v;
  }
};

// A fixed sequence of launches (a chunk of LSQR or CG iterations, whose
// kernels stop themselves through the device stop flag) recorded once per
// solve as a CUDA graph and replayed: one launch per chunk instead of 30-40.
// Recorded on a private stream in thread-local capture mode, so other host
// threads (the batched workers) are unaffected; the graph is launched on the
// solve's own stream.  Disabled or failed: the launches are enqueued directly.
// Chunk graphs are used when opts.graphs = 1: they saved 0.6 ms of 36 ms of
// LSQR on one 50000 x 4000 solve, but recording and instantiating a graph per
// solve cost more than the launches it saved on the ragged batch of small
// problems (45 against 57 problems/s), so direct launches are the default.
struct ChunkGraph {
  explicit ChunkGraph(bool on) : failed(!on) {}
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool failed;
  long long nkern = 0;  // kernels per replay (counted as launches when they run)
  ~ChunkGraph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
  }
  template <class F>
  ski_status run(cudaStream_t st, F&& enqueue) {
    if (!exec && !failed) {
      bool ok = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) == cudaSuccess &&
                cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (ok) {
        const long long before = t_launches;
        const ski_status s = enqueue(cap);
        nkern = t_launches - before;
        ski_count_launches(-nkern);  // recorded, not run
        cudaGraph_t g = nullptr;
        ok = cudaStreamEndCapture(cap, &g) == cudaSuccess && s == SKI_OK && g;
        graph = g;
        ok = ok && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
      }
      if (!ok) {
        failed = true;
        cudaGetLastError();
      }
    }
    if (exec) {
      SKI_CUDA_TRY(cudaGraphLaunch(exec, st));
      ski_count_launches(nkern);
      return SKI_OK;
    }
    return enqueue(st);
  }
};

// r = b - A x (into P.t), q = A^T r, ||r||^2 (and ||A||_F^2 when want_aa) into scalars.
// comp: r by compensated dot products (the acceptance test of Step 5).
ski_status residual_pass(const ski_matrix* A, const double* b, const double* x, SolvePlan& P, bool want_aa,
                         cudaStream_t st, bool comp = false) {
  FusedArgs f{};
  f.comp = comp ? 1 : 0;
  f.maxexp = (want_aa && A->kind == SKI_DENSE) ? &P.sc->amax_exp : nullptr;
  f.A = A->kind == SKI_DENSE ? A->val : nullptr;
  f.lda = A->ld;
  f.rowptr = A->kind == SKI_CSR ? A->rowptr : nullptr;
  f.colidx = A->colidx;
  f.val = A->val;
  f.n = P.n;
  f.d = P.d;
  f.z = x;
  f.u = nullptr;
  f.b = b;
  f.ca = -1.0;
  f.cu = 0.0;
  f.cb = 1.0;
  f.coef_from_scalars = 0;
  f.t = P.t;
  f.part = P.part;
  f.ldp = P.d;
  f.part_tt = P.part_tt;
  f.part_aa = P.part_aa;
  f.want_aa = want_aa ? 1 : 0;
  f.nblk = P.nblk;
  f.sc = nullptr;
  SKI_TRY(ski_fused_launch(f, st));
  const int shard = P.sh ? 1 : 0;
  if (P.csr) {
    SKI_TRY(ski_csc_launch(P.d, P.colptr, P.rowidx, P.cval, P.t, P.q, nullptr, st));
    SKI_TRY(ski_reduce_launch(P.nblk, P.d, nullptr, P.d, P.part_tt, want_aa ? P.part_aa : nullptr, P.q, P.sc, 2, st,
                              shard));
  } else {
    SKI_TRY(ski_reduce_launch(P.nblk, P.d, P.part, P.d, P.part_tt, want_aa ? P.part_aa : nullptr, P.q, P.sc, 2, st,
                              shard));
  }
  if (P.sh) {  // A^T r, ||r||^2, ||A||_F^2 of the whole A
    SKI_TRY(P.sh->sum(P.q, P.d + 2, SKI_F64, st));
    SKI_TRY(ski_finish_shard_launch(P.q, P.d, P.sc, 2, want_aa ? 1 : 0, st));
  }
  return SKI_OK;
}

// One LSQR iteration (lsqr_df.cu): K2 pass over A, K3 reduction (q, beta),
// K4 p = M^T q and v', K1 rotation, v / y / w and z = M v.
ski_status lsqr_iteration(const ski_matrix* A, SolvePlan& P, cudaStream_t st) {
  if (P.csr) {
    FusedArgs f{};
    f.rowptr = A->rowptr;
    f.colidx = A->colidx;
    f.val = A->val;
    f.n = P.n;
    f.d = P.d;
    f.z = P.z;
    f.u = P.t;
    f.coef_from_scalars = 1;
    f.t = P.t;
    f.part_tt = P.part_tt;
    f.nblk = P.nblk;
    f.sc = P.sc;
    SKI_TRY(ski_fused_launch(f, st));
    SKI_TRY(ski_csc_launch(P.d, P.colptr, P.rowidx, P.cval, P.t, P.q, P.sc, st));
    SKI_TRY(ski_reduce_par_launch(P.nblk, P.d, nullptr, P.part_tt, P.q, P.sc, st, P.sh ? 1 : 0));
  } else {
    DfArgs f{};
    f.A2 = P.A2;
    f.n = P.n;
    f.d = P.dl;
    f.sA = P.sA;
    f.z = P.z;
    f.u = P.t;
    f.coef_from_scalars = 1;
    f.t = P.t;
    f.part = P.part;
    f.part_tt = P.part_tt;
    f.nblk = P.nblk;
    f.sc = P.sc;
    f.variant = P.lsqr_pass;
    SKI_TRY(ski_fused_df_launch(f, st));
    SKI_TRY(ski_reduce_par_launch(P.nblk, P.dl, P.part, P.part_tt, P.q, P.sc, st, P.sh ? 1 : 0));
  }
  if (P.sh) {  // q = A^T t and ||t||^2 of the whole A
    SKI_TRY(P.sh->sum(P.q, P.dl + 1, SKI_F64, st));
    SKI_TRY(ski_finish_shard_launch(P.q, P.dl, P.sc, 0, 0, st));
  }
  SKI_TRY(ski_trmv_lower_vp_launch(P.dl, P.Mt, P.q, P.v, P.vp, P.part_vv, P.sc, 0, st));
  SKI_TRY(ski_trmv_upper_update_launch(P.dl, P.M, P.vp, P.part_vv, P.v, P.w, P.y, P.z, P.sc, 0, st));
  return SKI_OK;
}

ski_status read_scalars(const SolvePlan& P, LsqrScalars* h, cudaStream_t st) {
  SKI_CUDA_TRY(cudaMemcpyAsync(h, P.sc, sizeof(LsqrScalars), cudaMemcpyDeviceToHost, st));
  SKI_CUDA_TRY(cudaStreamSynchronize(st));
  return SKI_OK;
}

}  // namespace

extern "C" size_t ski_solve_workspace_size(const ski_matrix* A, const ski_opts* o) {
  if (check_matrix(A) != SKI_OK || check_sketch_opts(A, o) != SKI_OK) return 0;
  SolvePlan P;
  return plan_solve(A, o, nullptr, 0, &P);
}

static ski_status solve_impl(const ski_matrix* A, const double* b, const ski_opts* o, double* x, double* R_out,
                             ski_info* info, void* ws, size_t ws_bytes, void* stream, const ShardHook* sh,
                             LsqrGroupHook* gh = nullptr) {
  if (info) {
    memset(info, 0, sizeof(*info));
    info->status = SKI_EINVAL;
  }
  SKI_TRY(check_matrix(A));
  SKI_TRY(check_sketch_opts(A, o));
  if (!b || !x) return SKI_EINVAL;
  if (!sh && o->row_offset != 0) return SKI_EINVAL;  // a solve of a whole A
  if (sh && o->premix) return SKI_EINVAL;             // H D mixes every row: no row block premixes alone
  if (o->m < A->d || (!sh && A->n < A->d)) return SKI_EINVAL;
  if (o->qr_dtype != SKI_F64 && o->qr_dtype != SKI_F32 && o->qr_dtype != SKI_TF32) return SKI_EINVAL;
  if (A->kind == SKI_DENSE && A->d > SKI_DENSE_DMAX) return SKI_EINVAL;
  if (o->it_max < 0) return SKI_EINVAL;
  if (o->factorization < 0 || o->factorization > 2) return SKI_EINVAL;
  SolvePlan P;
  const size_t need = plan_solve(A, o, nullptr, 0, &P);
  if (ws_bytes < need || !ws) {
    if (info) info->status = SKI_ENOMEM;
    return SKI_ENOMEM;
  }
  plan_solve(A, o, (char*)ws, ws_bytes, &P);
  P.sh = sh;
  cudaStream_t st = ski_stream(stream);
  Events ev;
  if (!ev.ok) return SKI_ECUDA;
  const int64_t d = P.d;
  ski_status result = SKI_OK;
  LsqrScalars hs;
  memset(&hs, 0, sizeof(hs));
  hs.tau_r = o->tau_r;
  hs.it_max = o->it_max;
  hs.amax_exp = 0;

  double qr_gemm_ms = 0.0;
  float ms_sk = 0.f, ms_qr = 0.f, ms_ti = 0.f, ms_pm = 0.f, ms_ga = 0.f;
  int32_t rank = 0;
  double rdiag_ratio = 0.0;
  // R^{-1} is only the preconditioner (Theorem 10: any fixed M close to R^{-1}
  // serves, and x is accepted by the FP64 test), so an FP64 factor whose
  // diagonal ratio allows FP32 (the limit the mixed form applies to an FP32
  // factor: kappa(R) 2^-24 stays small) is inverted in FP32 -- with CUDA-core
  // FP32 products, about 10x faster than on the FP64 pipe.  Like the mixed
  // factor it is guarded by the LSQR budget; after any fallback M is FP64.
  bool inv64_only = false;
  int32_t inv_dt = SKI_F64;
  // Step 2's rank-revealing form (column-pivoted QR), dense A only
  const bool pivot_ok = o->factorization == 1 && !P.csr;
  bool need_pivot = false;
  bool perturbed = false;  // R + perturb I replaced R (the perturbed back-solve)
  bool gram_used = false;  // Step 2 took the Cholesky factor of the sketch's Gram matrix
  double gram_eq = INFINITY;  // its column-scaled diagonal ratio
  // Steps 1-2 and R^{-1} in the precisions of `of`
  auto factor = [&](const ski_opts* of) -> ski_status {
    carve_region(A, of, &P);
    perturbed = false;
    Events fe;
    if (!fe.ok) return SKI_ECUDA;
    SKI_CUDA_TRY(cudaMemsetAsync(P.perr, 0, sizeof(int), st));
    SKI_CUDA_TRY(cudaEventRecord(fe.e[0], st));
    // Step 1: sketch [SA | Sb] (a row block's partial sketch, summed over the processes)
    SKI_TRY(sketch_run(A, b, of, P.SA, P.ld_sa, P.stage, P.stage_bytes, st, fe.e[5], fe.e[6], P.perr));
    if (P.sh) SKI_TRY(P.sh->sum(P.SA, P.m * P.ld_sa, of->sketch_dtype, st));
    SKI_CUDA_TRY(cudaEventRecord(fe.e[1], st));
    // Step 2: QR of [SA | Sb] in qr_dtype
    if (P.SAq != P.SA) {
      const int64_t cnt = P.m * P.ld_sa;
      const unsigned g = (unsigned)ski_cdiv(cnt, 256);
      if (of->sketch_dtype == SKI_BF16)
        k_convert<__nv_bfloat16, float><<<g, 256, 0, st>>>(cnt, (const __nv_bfloat16*)P.SA, (float*)P.SAq);
      else if (of->sketch_dtype == SKI_F32)
        k_convert<float, double><<<g, 256, 0, st>>>(cnt, (const float*)P.SA, (double*)P.SAq);
      else
        k_convert<double, float><<<g, 256, 0, st>>>(cnt, (const double*)P.SA, (float*)P.SAq);
      SKI_LAUNCH_CHECK();
    }
    double gm = 0.0;
    {
      // factorization 2 (CSR A, FP64): R from the Cholesky factor of the
      // sparse sketch's Gram matrix, else (or when that breaks down) the
      // Householder QR of the dense [SA | Sb]
      bool done = false;
      gram_used = false;
      if (gram_path(A, of) && !P.sh) {
        SkiArena gar{P.stage, P.stage_bytes, 0, false};
        if (P.csr)
          SKI_TRY(ski_gram_chol_run(A, of->seed, of->s, of->hash_kind, P.m, (const double*)P.SA + d, P.ld_sa, P.R,
                                    d, P.qtsb, &done, &gram_eq, gar, st));
        else
          SKI_TRY(ski_gram_dense_run(P.SAq, P.ld_sa, P.m, d, P.qr_prec, P.R, d, P.qtsb, &done, &gram_eq, gar, st,
                                     info ? &gm : nullptr));
        gram_used = done;
      }
      SkiArena qar{P.stage, P.stage_bytes, 0, false};
      if (!done)
        SKI_TRY(ski_qr_run(P.m, d, 1, P.SAq, P.ld_sa, P.qr_prec, P.R, d, P.qtsb, qar, st, info ? &gm : nullptr));
    }
    qr_gemm_ms += gm;
    SKI_CUDA_TRY(cudaEventRecord(fe.e[2], st));
    bool nonfinite = false;
    SKI_TRY(rank_from_diag(d, P.R, d, o->rcond, st, &rank, &nonfinite, &rdiag_ratio));
    if (gram_used && (nonfinite || rank < d || !(gram_eq <= gram_ratio_limit(P.qr_prec)))) {
      // too ill-conditioned for the Gram matrix's precision: Householder QR
      gram_used = false;
      SkiArena qar{P.stage, P.stage_bytes, 0, false};
      SKI_TRY(ski_qr_run(P.m, d, 1, P.SAq, P.ld_sa, P.qr_prec, P.R, d, P.qtsb, qar, st, info ? &gm : nullptr));
      SKI_TRY(rank_from_diag(d, P.R, d, o->rcond, st, &rank, &nonfinite, &rdiag_ratio));
    }
    int perr = 0;
    SKI_CUDA_TRY(cudaMemcpyAsync(&perr, P.perr, sizeof(int), cudaMemcpyDeviceToHost, st));
    SKI_CUDA_TRY(cudaStreamSynchronize(st));
    if (perr) return SKI_ETIMEOUT;
    if (nonfinite) return SKI_ENONFINITE;
    if (rank < d && pivot_ok) {
      // the column-pivoted QR of R replaces this factor (after R_out is taken)
      need_pivot = true;
      ms_sk += fe.ms(0, 1);
      ms_qr += fe.ms(1, 2);
      ms_pm += fe.ms(5, 6);
      ms_ga += fe.ms(6, 1);
      return SKI_OK;
    }
    need_pivot = false;
    if (rank < d && o->perturb <= 0.0) return SKI_ESINGULAR;
    // R^{-1} (explicit, and its transpose)
    inv_dt = P.qr_dt;
    if (inv_dt == SKI_F64 && !inv64_only && rank == d &&
        rdiag_ratio <= mixed_ratio_limit(SKI_F32, SKI_F64))
      inv_dt = SKI_F32;
    {
      SkiArena tar{P.region, P.region_bytes, 0, false};
      if (rank < d) {
        // the perturbed back-solve (Ski-LLS-sparse): every division by r_ii
        // becomes one by r_ii + perturb, i.e. the factor is R + perturb I.
        // The diagonal is changed in place so that the inverse, the Step 3
        // refinement against the factor and R_out all use the same matrix.
        SKI_TRY(ski_add_diag_launch(d, P.R, d, o->perturb, st));
        perturbed = true;
      }
      SKI_TRY(ski_trinv_run(d, P.R, d, P.M, P.Mt, d, inv_dt, 0.0, tar, st));
    }
    SKI_CUDA_TRY(cudaEventRecord(fe.e[3], st));
    SKI_CUDA_TRY(cudaEventSynchronize(fe.e[3]));
    ms_sk += fe.ms(0, 1);
    ms_qr += fe.ms(1, 2);
    ms_ti += fe.ms(2, 3);
    ms_pm += fe.ms(5, 6);
    ms_ga += fe.ms(6, 1);
    return SKI_OK;
  };
  // The mixed form factors in FP32 (or TF32); R only has to precondition
  // (Theorem 10), which fails once kappa(SA) times the factorisation's unit
  // roundoff nears 1.  |r_11| ... |r_dd| bound kappa(R) from below: past the
  // limit of mixed_ratio_limit() -- or when the FP32 factor fails the rank
  // rule, or its LSQR run exhausts a budget (below) -- Steps 1-2 are redone
  // in FP64 and the solve continues from there.
  const bool mixed = o->qr_dtype != SKI_F64;
  ski_opts o64 = *o;
  o64.sketch_dtype = SKI_F64;
  o64.qr_dtype = SKI_F64;
  int32_t fell_back = 0;
  SKI_CUDA_TRY(cudaEventRecord(ev.e[0], st));
  ski_status fs = factor(o);
  const double ratio_first = rdiag_ratio;
  if (mixed && (fs == SKI_ESINGULAR || fs == SKI_ENONFINITE ||
                (fs == SKI_OK && !(rdiag_ratio <= mixed_ratio_limit(o->qr_dtype, o->sketch_dtype))))) {
    fell_back = 1;
    inv64_only = true;
    fs = factor(&o64);
  }
  if (info) {
    info->rank = rank;
    info->rdiag_ratio = ratio_first;
    info->qr_fallback = fell_back;
  }
  if (fs != SKI_OK) {
    if (info) info->status = fs;
    return fs;
  }
  if (R_out) SKI_CUDA_TRY(cudaMemcpyAsync(R_out, P.R, d * d * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (need_pivot) {
    // Step 2, rank-revealing: the column-pivoted QR of [R | Q^T Sb] gives the
    // pivots V, R11 (p x p, rows of stride d in P.R) and Q1^T Sb (P.qtsb);
    // Steps 3-5 then run on the p unknowns of W = A V1 R11^{-1}
    Events pe;
    if (!pe.ok) return SKI_ECUDA;
    SKI_CUDA_TRY(cudaEventRecord(pe.e[0], st));
    int32_t p2 = 0;
    {
      SkiArena car{P.region, P.region_bytes, 0, false};
      const ski_status cs = ski_cpqr_run(d, P.R, d, P.qtsb, o->rcond, P.R, d, P.qtsb, P.piv, &p2, car, st);
      if (cs != SKI_OK) {
        if (info) info->status = cs;
        return cs;
      }
    }
    SKI_CUDA_TRY(cudaEventRecord(pe.e[1], st));
    if (p2 < 1) {
      if (info) info->status = SKI_ESINGULAR;
      return SKI_ESINGULAR;
    }
    {
      SkiArena tar{P.region, P.region_bytes, 0, false};
      SKI_TRY(ski_trinv_run(p2, P.R, d, P.M, P.Mt, p2, SKI_F64, 0.0, tar, st));
    }
    SKI_CUDA_TRY(cudaEventRecord(pe.e[2], st));
    SKI_CUDA_TRY(cudaEventSynchronize(pe.e[2]));
    ms_qr += pe.ms(0, 1);
    ms_ti += pe.ms(1, 2);
    inv_dt = SKI_F64;
    rank = p2;
    P.dl = p2;
    P.pivoted = true;
    if (info) {
      info->rank = rank;
      info->pivoted = 1;
    }
  }
  const int64_t dl = P.dl;
  if (P.csr) {
    SkiArena car{P.csc_tmp, P.region_bytes, 0, false};
    SKI_TRY(ski_csc_build(A, P.colptr, P.rowidx, P.cval, car, st));
  }
  SKI_CUDA_TRY(cudaEventRecord(ev.e[3], st));
  // Step 3: x_s = R^{-1} Q^T Sb and its residual
  SKI_TRY(ski_trmv_launch(true, dl, P.M, dl, P.qtsb, nullptr, P.xs, nullptr, st));
  if ((inv_dt == SKI_F32 && P.qr_dt == SKI_F64) || perturbed) {
    // M is R^{-1} to FP32 accuracy: two steps of refinement against the FP64
    // R, x_s += M (Q^T Sb - R x_s), give x_s to FP64 accuracy (the error
    // squares each step), so that a consistent system still exits at Step 3.
    // The same holds for the perturbed factor R + perturb I, whose explicit
    // inverse loses about kappa u against a back-substitution (kappa ~
    // |r_11| / perturb): the refined x_s is as accurate as the back-solve's.
    // The LSQR vectors are free here: v = -x_s, w = the step's residual.
    for (int it = 0; it < 2; ++it) {
      SKI_TRY(ski_copy_launch(d, P.xs, P.v, st));
      SKI_TRY(ski_scale_launch(1, d, P.v, d, -1.0, st));
      SKI_TRY(ski_trmv_launch(true, d, P.R, d, P.v, P.qtsb, P.w, nullptr, st));
      SKI_TRY(ski_trmv_launch(true, d, P.M, d, P.w, P.xs, P.vp, nullptr, st));
      SKI_TRY(ski_copy_launch(d, P.vp, P.xs, st));
    }
  }
  SKI_CUDA_TRY(cudaMemcpyAsync(P.sc, &hs, sizeof(hs), cudaMemcpyHostToDevice, st));
  if (P.pivoted) {
    SKI_TRY(ski_scatter_launch(d, dl, P.piv, P.xs, P.xfull, st));
    SKI_TRY(residual_pass(A, b, P.xfull, P, true, st));
  } else {
    SKI_TRY(residual_pass(A, b, P.xs, P, true, st));
  }
  SKI_TRY(read_scalars(P, &hs, st));
  const double anorm_f = sqrt(hs.anorm_f2);
  if (!isfinite(hs.rnorm2) || !isfinite(hs.anorm_f2)) {
    if (info) info->status = SKI_ENONFINITE;
    return SKI_ENONFINITE;
  }
  if (!P.csr) {
    // A2 = A * 2^-sA with max|A2| < 1, in (hi, lo) float pairs
    P.sA = hs.amax_exp > 0 ? hs.amax_exp - 1022 : 0;
    SKI_TRY(ski_split_a_launch(P.n, dl, A->val, A->ld, P.sA, P.A2, st, P.pivoted ? P.piv : nullptr));
  }
  int64_t iters_total = 0;
  int restarts = 0;
  ChunkGraph lsqr_graph(o->graphs == 1 && !sh);  // the row-block sums are host calls: no capture
  double metric = 0.0, lsqr_test = 0.0;
  bool early = false;
  // The acceptance metric ||A^T r|| / (||A||_F ||r||) of x from the residual
  // pass just run, whose r = b - A x is plain FP64.  Its rounding is about
  // sqrt(d) u |A| |x| per entry of r (at most sqrt(d) u ||A||_F ||x|| in
  // norm), and A^T of such noise, nearly orthogonal to range(A) for n >> d, is
  // about ||A||_F / sqrt(n) times it.  When that estimate (times 16) could
  // decide the test -- x large along small singular directions, where the
  // plain value is itself noise at the level of tol -- the pass is redone
  // with the compensated residual, which the metric then certifies.  The
  // row-block form always takes the compensated pass.
  auto acceptance = [&](const double* xv, double* mout) -> ski_status {
    SKI_TRY(ski_norm2_launch(d, P.q, xv, P.sc, st));
    SKI_TRY(read_scalars(P, &hs, st));
    if (!isfinite(hs.rnorm2) || !isfinite(hs.atr_norm)) return SKI_ENONFINITE;
    double mtr = hs.rnorm2 > 0 ? hs.atr_norm / (anorm_f * sqrt(hs.rnorm2)) : 0.0;
    if (o->tol > 0.0 && hs.rnorm2 > 0) {
      const double noise = 16.0 * sqrt((double)d) * 0x1p-53 * anorm_f * hs.xnorm / (sqrt((double)P.n) * sqrt(hs.rnorm2));
      if (P.sh || !(fabs(mtr - o->tol) > noise)) {
        SKI_TRY(residual_pass(A, b, xv, P, false, st, true));
        SKI_TRY(ski_norm_launch(d, P.q, P.sc, st));
        SKI_TRY(read_scalars(P, &hs, st));
        if (!isfinite(hs.rnorm2) || !isfinite(hs.atr_norm)) return SKI_ENONFINITE;
        mtr = hs.rnorm2 > 0 ? hs.atr_norm / (anorm_f * sqrt(hs.rnorm2)) : 0.0;
      }
    }
    *mout = mtr;
    return SKI_OK;
  };
  if (sqrt(hs.rnorm2) <= o->tau_a) {
    early = true;
    if (P.pivoted)
      SKI_TRY(ski_scatter_launch(d, dl, P.piv, P.xs, x, st));
    else
      SKI_TRY(ski_copy_launch(d, P.xs, x, st));
    // P.q holds A^T r of x from Step 3's residual pass
    const ski_status as = acceptance(x, &metric);
    if (as != SKI_OK) {
      if (info) info->status = as;
      return as;
    }
  } else {
    // Step 4: LSQR from y_0 = Q^T Sb (x_s), restarted from the current x while
    // the FP64 acceptance metric is above tol.
    for (;;) {
      // start: beta_1 u_1 = r (in P.t), alpha_1 v_1 = M^T A^T u_1
      LsqrScalars init = hs;
      init.iters = 0;
      init.it_max = o->it_max - iters_total;
      const int64_t budget = mixed_lsqr_budget(o->m, d, o->tau_r);
      const bool inv32 = !mixed && inv_dt == SKI_F32;
      const bool budgeted = (mixed || inv32) && !fell_back && init.it_max > budget;
      if (budgeted) init.it_max = budget;
      init.flag_a = 0;
      init.flag_b = 0;
      init.conv = 0;
      init.tau_r = o->tau_r;
      SKI_CUDA_TRY(cudaMemcpyAsync(P.sc, &init, sizeof(init), cudaMemcpyHostToDevice, st));
      // A^T r of the residual pass is in A's column order: V1^T picks the pivots
      if (P.pivoted) SKI_TRY(ski_gather_launch(dl, P.piv, P.q, P.p, st));
      SKI_TRY(ski_trmv_lower_vp_launch(dl, P.Mt, P.pivoted ? P.p : P.q, P.v, P.vp, P.part_vv, P.sc, 1, st));
      SKI_TRY(ski_trmv_upper_update_launch(dl, P.M, P.vp, P.part_vv, P.v, P.w, P.y, P.z, P.sc, 1, st));
      const int CHUNK = 8;
      int64_t polled = 0;
      const bool grouped = gh && !P.csr && !sh;
      if (grouped) {  // Step 4 on the batch's grouped launches
        LsqrGroupTask task{};
        DfArgs& f = task.job.df;
        f.A2 = P.A2;
        f.n = P.n;
        f.d = dl;
        f.ld2 = ski_a2_ld(dl);
        f.sA = P.sA;
        f.z = P.z;
        f.u = P.t;
        f.coef_from_scalars = 1;
        f.t = P.t;
        f.part = P.part;
        f.part_tt = P.part_tt;
        f.nblk = P.nblk;
        f.rows_per = ski_cdiv(P.n, (int64_t)P.nblk);
        f.sc = P.sc;
        task.job.d = dl;
        task.job.q = P.q;
        task.job.Mt = P.Mt;
        task.job.M = P.M;
        task.job.v = P.v;
        task.job.vp = P.vp;
        task.job.part_vv = P.part_vv;
        task.job.w = P.w;
        task.job.y = P.y;
        task.job.z = P.z;
        task.job.nvv = ski_vv_blocks(dl);
        task.cls = ski_df_group_class(dl);
        task.smem = (size_t)f.rows_per * sizeof(double);
        task.st = st;
        task.it_max = o->it_max;
        task.chunk = CHUNK;
        task.budgeted = budgeted;
        task.budget = budget;
        task.tau_r = o->tau_r;
        SKI_TRY(gh->run(task));
        hs = task.hs;
      }
      while (!grouped) {
        SKI_TRY(lsqr_graph.run(st, [&](cudaStream_t s) -> ski_status {
          for (int k = 0; k < CHUNK; ++k) SKI_TRY(lsqr_iteration(A, P, s));
          return SKI_OK;
        }));
        polled += CHUNK;
        SKI_TRY(read_scalars(P, &hs, st));
        if (hs.flag_a) break;
        if (polled > o->it_max + CHUNK) break;
        if (budgeted && weak_preconditioner(hs.test, hs.iters, o->tau_r, budget)) break;
      }
      iters_total += hs.iters;
      lsqr_test = hs.test;
      if (hs.df_err) {
        result = SKI_ETIMEOUT;
        break;
      }
      // Step 5: x = x_s + R^{-1} delta (x = V1 (x_s + R11^{-1} delta) when pivoted)
      if (P.pivoted) {
        SKI_TRY(ski_trmv_launch(true, dl, P.M, dl, P.y, P.xs, P.p, nullptr, st));
        SKI_TRY(ski_scatter_launch(d, dl, P.piv, P.p, x, st));
      } else {
        SKI_TRY(ski_trmv_launch(true, d, P.M, d, P.y, P.xs, x, nullptr, st));
      }
      SKI_TRY(residual_pass(A, b, x, P, false, st));
      const ski_status as = acceptance(x, &metric);
      if (as == SKI_ENONFINITE) {
        result = SKI_ENONFINITE;
        break;
      }
      SKI_TRY(as);
      const bool lsqr_ok = hs.conv != 0;
      if (o->tol > 0.0 ? metric <= o->tol : lsqr_ok) break;
      if (budgeted && !lsqr_ok && inv32) {
        // the FP32 inverse of the FP64 factor is too inaccurate: form it in
        // FP64 and continue from x
        fell_back = 3;
        inv64_only = true;
        Events te;
        if (!te.ok) return SKI_ECUDA;
        SKI_CUDA_TRY(cudaEventRecord(te.e[0], st));
        {
          SkiArena tar{P.region, P.region_bytes, 0, false};
          SKI_TRY(ski_trinv_run(d, P.R, d, P.M, P.Mt, d, SKI_F64, 0.0, tar, st));
        }
        inv_dt = SKI_F64;
        SKI_CUDA_TRY(cudaEventRecord(te.e[1], st));
        SKI_CUDA_TRY(cudaEventSynchronize(te.e[1]));
        ms_ti += te.ms(0, 1);
        if (info) info->qr_fallback = fell_back;
        SKI_TRY(ski_copy_launch(d, x, P.xs, st));  // P.t = r, P.q = A^T r from the pass above
        continue;
      }
      if (budgeted && !lsqr_ok) {
        // the FP32 preconditioner is too weak: refactor in FP64, continue from x
        fell_back = 2;
        inv64_only = true;
        SKI_TRY(factor(&o64));
        if (info) {
          info->rank = rank;
          info->qr_fallback = fell_back;
        }
        if (R_out) SKI_CUDA_TRY(cudaMemcpyAsync(R_out, P.R, d * d * sizeof(double), cudaMemcpyDeviceToDevice, st));
        SKI_TRY(ski_copy_launch(d, x, P.xs, st));  // P.t = r, P.q = A^T r from the pass above
        continue;
      }
      if (iters_total >= o->it_max || restarts >= 8) {
        result = SKI_ENOCONV;
        break;
      }
      ++restarts;
      // warm restart from x; P.t = r, P.q = A^T r
      if (P.pivoted)
        SKI_TRY(ski_gather_launch(dl, P.piv, x, P.xs, st));
      else
        SKI_TRY(ski_copy_launch(d, x, P.xs, st));
    }
  }
  SKI_CUDA_TRY(cudaEventRecord(ev.e[4], st));
  SKI_CUDA_TRY(cudaEventSynchronize(ev.e[4]));
  if (info) {
    info->iters = iters_total;
    info->restarts = restarts;
    info->early_exit = early ? 1 : 0;
    info->metric = metric;
    info->resid_norm = sqrt(hs.rnorm2);
    info->anorm_f = anorm_f;
    info->lsqr_test = lsqr_test;
    info->ms_sketch = ms_sk;
    info->ms_qr = ms_qr;
    info->ms_trinv = ms_ti;
    info->ms_lsqr = ev.ms(3, 4);
    info->ms_total = ev.ms(0, 4);
    info->ms_premix = ms_pm;
    info->ms_gather = ms_ga;
    info->qr_fallback = fell_back;
    info->inv_dtype = inv_dt;
    info->ms_qr_gemm = (float)qr_gemm_ms;
    info->pivoted = P.pivoted ? 1 : 0;
    info->gram = gram_used ? 1 : 0;
    info->status = result;
  }
  return result;
}

extern "C" ski_status ski_solve(const ski_matrix* A, const double* b, const ski_opts* o, double* x, double* R_out,
                                ski_info* info, void* ws, size_t ws_bytes, void* stream) {
  return solve_impl(A, b, o, x, R_out, info, ws, ws_bytes, stream, nullptr);
}

ski_status ski_solve_grouped(const ski_matrix* A, const double* b, const ski_opts* o, double* x, double* R_out,
                             ski_info* info, void* ws, size_t ws_bytes, void* stream, LsqrGroupHook* hook) {
  return solve_impl(A, b, o, x, R_out, info, ws, ws_bytes, stream, nullptr, hook);
}

bool ski_weak_preconditioner(double test, long long iters, double tau_r, int64_t budget) {
  return weak_preconditioner(test, iters, tau_r, budget);
}

int ski_lsqr_ctas(int64_t n, const ski_opts* o) { return lsqr_ctas(n, o); }

extern "C" ski_status ski_solve_rowblock(const ski_matrix* A, const double* b, const ski_opts* o, double* x,
                                         double* R_out, ski_info* info, void* ws, size_t ws_bytes, void* stream,
                                         ski_allreduce_fn allreduce, void* ctx) {
  if (!allreduce) return SKI_EINVAL;
  ShardHook h{allreduce, ctx};
  return solve_impl(A, b, o, x, R_out, info, ws, ws_bytes, stream, &h);
}

// ------------------------------------------------------------ adjoint
namespace {
struct AdjPlan {
  double *M, *Mt, *t, *rres, *h, *r, *p, *z, *zz, *q, *lam, *part, *part_tt;
  float2* A2;
  LsqrScalars* sc;
  char* tw;
  size_t tw_bytes;
  int nblk;
  int lsqr_pass;  // variant of the dense LSQR pass (ski_opts.lsqr_pass)
};
size_t plan_adjoint(const ski_matrix* A, const ski_opts* o, char* base, size_t cap, AdjPlan* P) {
  SkiArena ar{base, cap, 0, base == nullptr};
  const int64_t n = A->n, d = A->d;
  P->nblk = lsqr_ctas(n, o);
  P->lsqr_pass = o ? o->lsqr_pass : 0;
  P->M = ar.take<double>(d * d);
  P->Mt = ar.take<double>(d * d);
  P->t = ar.take<double>(n);
  P->rres = ar.take<double>(n);
  P->h = ar.take<double>(d);
  P->r = ar.take<double>(d);
  P->p = ar.take<double>(d);
  P->z = ar.take<double>(d);
  P->zz = ar.take<double>(d);
  P->q = ar.take<double>(d);
  P->lam = ar.take<double>(d);
  P->part = ar.take<double>((int64_t)P->nblk * d);
  P->part_tt = ar.take<double>(P->nblk);
  P->sc = ar.take<LsqrScalars>(1);
  P->A2 = ar.take<float2>(n * ski_a2_ld(d));
  P->tw_bytes = ski_trinv_ws_bytes(d, SKI_F64);
  P->tw = ar.take<char>(P->tw_bytes);
  return ar.off;
}

FusedArgs dense_pass(const ski_matrix* A, const AdjPlan& P, const double* z, double ca, const double* bvec,
                     double cb, double* t, const LsqrScalars* sc) {
  FusedArgs f{};
  f.A = A->val;
  f.lda = A->ld;
  f.n = A->n;
  f.d = A->d;
  f.z = z;
  f.b = bvec;
  f.ca = ca;
  f.cb = cb;
  f.t = t;
  f.part = P.part;
  f.ldp = A->d;
  f.part_tt = P.part_tt;
  f.nblk = P.nblk;
  f.sc = sc;
  return f;
}
}  // namespace

extern "C" size_t ski_solve_adjoint_workspace_size(const ski_matrix* A, const ski_opts* o) {
  if (check_matrix(A) != SKI_OK || A->kind != SKI_DENSE) return 0;
  AdjPlan P;
  return plan_adjoint(A, o, nullptr, 0, &P);
}

// Backward pass (see include/skills.h).  The CG products W^T W p = M^T A^T A M p
// use the double-float pass over the (hi, lo) copy of A, as the forward LSQR
// does (the FP64 pipe cannot keep up with HBM, see lsqr_df.cu); the residual r,
// db = A lambda and dA stay in FP64.
extern "C" ski_status ski_solve_adjoint(const ski_matrix* A, const double* b, const double* x, const double* R,
                                        int64_t ldr, const double* g, double* dA, int64_t ld_da, double* db,
                                        const ski_opts* o, ski_info* info, void* ws, size_t ws_bytes, void* stream) {
  if (info) {
    memset(info, 0, sizeof(*info));
    info->status = SKI_EINVAL;
  }
  SKI_TRY(check_matrix(A));
  if (A->kind != SKI_DENSE || A->d > SKI_DENSE_DMAX || !o || !b || !x || !R || !g || !db || ldr < A->d ||
      !launch_opts_ok(o))
    return SKI_EINVAL;
  if (dA && ld_da < A->d) return SKI_EINVAL;
  AdjPlan P;
  const size_t need = plan_adjoint(A, o, nullptr, 0, &P);
  if (ws_bytes < need || !ws) return SKI_ENOMEM;
  plan_adjoint(A, o, (char*)ws, ws_bytes, &P);
  cudaStream_t st = ski_stream(stream);
  const int64_t d = A->d, n = A->n;
  {
    SkiArena tar{P.tw, P.tw_bytes, 0, false};
    SKI_TRY(ski_trinv_run(d, R, ldr, P.M, P.Mt, d, SKI_F64, 0.0, tar, st));
  }
  LsqrScalars hs;
  memset(&hs, 0, sizeof(hs));
  hs.it_max = o->it_max > 0 ? o->it_max : 1000;
  hs.cg_tol2 = o->tau_r * o->tau_r;
  SKI_CUDA_TRY(cudaMemcpyAsync(P.sc, &hs, sizeof(hs), cudaMemcpyHostToDevice, st));
  // r = b - A x in FP64, with the largest exponent of A for the (hi, lo) split
  {
    FusedArgs f = dense_pass(A, P, x, -1.0, b, 1.0, P.rres, nullptr);
    f.maxexp = &P.sc->amax_exp;
    SKI_TRY(ski_fused_launch(f, st));
  }
  SKI_CUDA_TRY(cudaMemcpyAsync(&hs, P.sc, sizeof(hs), cudaMemcpyDeviceToHost, st));
  SKI_CUDA_TRY(cudaStreamSynchronize(st));
  const int sA = hs.amax_exp > 0 ? hs.amax_exp - 1022 : 0;
  SKI_TRY(ski_split_a_launch(n, d, A->val, A->ld, sA, P.A2, st));
  // h = R^{-T} g; CG on W^T W z = h
  SKI_TRY(ski_trmv_launch(false, d, P.Mt, d, g, nullptr, P.h, nullptr, st));
  SKI_TRY(ski_cg_launch(d, P.h, P.r, P.p, P.z, P.sc, 1, st));
  DfArgs f{};
  f.A2 = P.A2;
  f.n = n;
  f.d = d;
  f.sA = sA;
  f.z = P.zz;
  f.u = nullptr;
  f.cu = 0.0;
  f.coef_from_scalars = 0;
  f.t = P.t;
  f.part = P.part;
  f.part_tt = P.part_tt;
  f.nblk = P.nblk;
  f.sc = P.sc;
  f.variant = P.lsqr_pass;
  int64_t polled = 0;
  ChunkGraph cg_graph(o->graphs == 1);
  for (;;) {
    SKI_TRY(cg_graph.run(st, [&](cudaStream_t s) -> ski_status {
      for (int k = 0; k < 8; ++k) {
        SKI_TRY(ski_trmv_launch(true, d, P.M, d, P.p, nullptr, P.zz, P.sc, s));
        SKI_TRY(ski_fused_df_launch(f, s));
        SKI_TRY(ski_reduce_par_launch(P.nblk, d, P.part, P.part_tt, P.q, P.sc, s));
        SKI_TRY(ski_trmv_launch(false, d, P.Mt, d, P.q, nullptr, P.zz, P.sc, s));
        SKI_TRY(ski_cg_launch(d, P.zz, P.r, P.p, P.z, P.sc, 0, s));
      }
      return SKI_OK;
    }));
    SKI_CUDA_TRY(cudaMemcpyAsync(&hs, P.sc, sizeof(hs), cudaMemcpyDeviceToHost, st));
    SKI_CUDA_TRY(cudaStreamSynchronize(st));
    polled += 8;
    if (hs.flag_a || hs.df_err || polled > hs.it_max + 16) break;
  }
  // lambda = R^{-1} z; db = A lambda; dA = r lambda^T - (A lambda) x^T
  SKI_TRY(ski_trmv_launch(true, d, P.M, d, P.z, nullptr, P.lam, nullptr, st));
  SKI_TRY(ski_fused_launch(dense_pass(A, P, P.lam, 1.0, nullptr, 0.0, db, nullptr), st));
  if (dA) SKI_TRY(ski_outer_launch(n, d, P.rres, P.lam, db, x, dA, ld_da, st));
  SKI_CUDA_TRY(cudaStreamSynchronize(st));
  const ski_status res = hs.df_err ? SKI_ETIMEOUT : (hs.conv ? SKI_OK : SKI_ENOCONV);
  if (info) {
    info->iters = hs.iters;
    info->status = res;
    info->lsqr_test = hs.cg_rr0 > 0 ? sqrt(hs.cg_rr / hs.cg_rr0) : 0.0;
  }
  return res;
}

extern "C" ski_status ski_selftest_wait_timeout(int64_t spin_limit, void* ws, size_t ws_bytes, void* stream) {
  if (spin_limit < 1 || !ws || ws_bytes < 16) return SKI_EINVAL;
  return ski_barrier_selftest(spin_limit, ws, ski_stream(stream));
}
