// Device-resident LSQR state and launch helpers (lsqr.cu) used by the C ABI.
#pragma once
#include "common.cuh"

// Largest d the dense fused pass handles (512 threads x 16 columns each).
#define SKI_DENSE_DMAX 8192

struct LsqrScalars {
  double alpha, beta, beta_new, rhobar, phibar, anorm2, test, coef;
  double tau_r;
  double rnorm2, anorm_f2, atr_norm;
  double cg_rr, cg_rr0, cg_tol2;  // conjugate gradients of the adjoint solve
  long long iters, it_max;
  int flag_a, flag_b;  // stop flags (see lsqr_df.cu for who writes which)
  int conv;
  int amax_exp;  // largest biased exponent field of A (from the first residual pass)
  int df_err;    // a staged copy of the LSQR pass timed out
  // the rotation state as the LSQR step kernel (K1) reads it: a copy of
  // alpha, rhobar, phibar, anorm2, iters taken by K3 before every K1, so that
  // CTA 0 of K1 can write the new state while its other CTAs still read the old
  double r_alpha, r_rhobar, r_phibar, r_anorm2;
  long long r_iters;
  double xnorm;  // ||x|| of the last acceptance check (its rounding-noise estimate)
};

struct FusedArgs {
  // dense A (row-major) or CSR A
  const double* A;
  int64_t lda;
  const int64_t* rowptr;
  const int32_t* colidx;
  const double* val;
  int64_t n, d;
  // t = ca * (A z) + cu * u + cb * b ; coefficients from scalars when coef_from_scalars
  const double* z;
  const double* u;
  const double* b;
  double ca, cu, cb;
  int coef_from_scalars;
  double* t;
  // per-CTA partials: A^T t (dense only), ||t||^2, ||A||_F^2
  double* part;
  int64_t ldp;
  double* part_tt;
  double* part_aa;
  int want_aa;
  int nblk;
  int64_t rows_per;
  const LsqrScalars* sc;
  int* maxexp;  // when set: atomicMax of the biased exponent fields of A
  int comp;     // compensated residual r = b - A z (Dot2; ca = -1, cb = 1, no u)
};

// Double-float dense pass (lsqr_df.cu): t = A z + cu u with A held as
// A2 = A * 2^-sA in (hi, lo) float pairs.
struct DfArgs {
  const float2* A2;
  int64_t n, d, ld2;  // ld2: row stride of A2 (even, so rows are 16-byte aligned)
  int sA;
  const double* z;
  const double* u;
  double cu;
  int coef_from_scalars;
  double* t;
  double* part;     // [nblk][d] partial A^T t
  double* part_tt;  // [nblk] partial ||t||^2
  int nblk;
  int64_t rows_per;
  LsqrScalars* sc;
  int variant;  // 0, 1: register-blocked rows; 2: TMA-staged row ring; 3: row per warp;
                // 4: register-blocked, twice the rows; 5: register-blocked with prefetch
};

// A2 = the (hi, lo) split of A * 2^-sA; with cmap, column c of A2 is column
// cmap[c] of A (d columns in all)
ski_status ski_split_a_launch(int64_t n, int64_t d, const double* A, int64_t lda, int sA, float2* A2,
                              cudaStream_t st, const int32_t* cmap = nullptr);
bool ski_df_supported(int64_t d);
int64_t ski_a2_ld(int64_t d);
ski_status ski_fused_df_launch(const DfArgs& f, cudaStream_t st);
// shard = 1: the row-block form (q and q[d] = ||t||^2 are partial sums; see
// ski_finish_shard_launch)
ski_status ski_reduce_par_launch(int nblk, int64_t d, const double* part, const double* part_tt, double* q,
                                 LsqrScalars* sc, cudaStream_t st, int shard = 0);
// After q[0..d] (and q[d+1]) were summed over the processes of a row-block
// solve: the scalars of an LSQR step (mode 0) or of a residual pass (mode 2)
// ||q|| into sc->atr_norm and, when x is given, ||x|| into sc->xnorm (one launch)
ski_status ski_norm2_launch(int64_t d, const double* q, const double* x, LsqrScalars* sc, cudaStream_t st);
ski_status ski_finish_shard_launch(const double* q, int64_t d, LsqrScalars* sc, int mode, int want_aa,
                                   cudaStream_t st);
int ski_vv_blocks(int64_t d);
ski_status ski_trmv_lower_vp_launch(int64_t d, const double* Mt, const double* q, const double* v, double* vp,
                                    double* part_vv, LsqrScalars* sc, int start, cudaStream_t st);
ski_status ski_trmv_upper_update_launch(int64_t d, const double* M, const double* vp, const double* part_vv,
                                        double* v, double* w, double* y, double* z, LsqrScalars* sc, int start,
                                        cudaStream_t st);

// ---- grouped LSQR iterations (ski_solve_batched): the four kernels of one
// iteration (K2 pass, K3 reduction, K4 and K1 triangular products) each run
// once for every problem in flight, over a list of (problem, block) work
// items; a finished problem's items return at once (its flags).
struct LsqrGroupJob {
  DfArgs df;  // K2 of this problem (ld2 and rows_per set)
  int64_t d;  // unknowns
  double* q;
  const double* Mt;
  const double* M;
  double *v, *vp, *part_vv, *w, *y, *z;
  int nvv;  // K4 blocks (ski_vv_blocks(d))
};
struct LsqrGroupItem {
  int32_t job, blk;
};
// K2 template class of the register-blocked pass for d unknowns (0 .. 4)
int ski_df_group_class(int64_t d);
constexpr int kDfGroupClasses = 5;
// items[0 .. nitems): K2 blocks of jobs of class cls; smem: largest rows_per * 8
ski_status ski_group_df_launch(int cls, const LsqrGroupJob* jobs, const LsqrGroupItem* items, int nitems,
                               size_t smem, cudaStream_t st);
// items: (job, 32-column block) for K3, (job, 8-row block) for K4 and K1
ski_status ski_group_reduce_launch(const LsqrGroupJob* jobs, const LsqrGroupItem* items, int nitems,
                                   cudaStream_t st);
ski_status ski_group_trmv_launch(const LsqrGroupJob* jobs, const LsqrGroupItem* items, int nitems,
                                 cudaStream_t st);
// out[j] = *jobs[j].df.sc
ski_status ski_group_scalars_launch(const LsqrGroupJob* jobs, int njobs, LsqrScalars* out, cudaStream_t st);

// A problem's Step 4 handed to a batch-wide executor (batch.cu): the
// solve fills the task after the LSQR start kernels are queued on st and
// blocks in run() until the executor has iterated the problem to its stop,
// with the single-problem loop's rules: flag_a, polled > it_max + chunk, or
// (budgeted) the weak-preconditioner rule.
struct LsqrGroupTask {
  LsqrGroupJob job;
  int cls;      // ski_df_group_class(job.d)
  size_t smem;  // job.df.rows_per * 8
  cudaStream_t st;
  int64_t it_max;
  int chunk;
  bool budgeted;
  int64_t budget;
  double tau_r;
  LsqrScalars hs;  // out: the scalars when the loop stopped
};
class LsqrGroupHook {
 public:
  virtual ski_status run(LsqrGroupTask& task) = 0;

 protected:
  ~LsqrGroupHook() = default;
};
// ski_solve with Step 4 of a dense problem run by hook (nullptr: ski_solve)
ski_status ski_solve_grouped(const ski_matrix* A, const double* b, const ski_opts* o, double* x, double* R_out,
                             ski_info* info, void* ws, size_t ws_bytes, void* stream, LsqrGroupHook* hook);
bool ski_weak_preconditioner(double test, long long iters, double tau_r, int64_t budget);
int ski_lsqr_ctas(int64_t n, const ski_opts* o);

int ski_fused_ctas(int64_t n);
ski_status ski_fused_launch(const FusedArgs& f, cudaStream_t st);
ski_status ski_trmv_launch(bool upper, int64_t d, const double* M, int64_t ldm, const double* x, const double* add,
                           double* y, const LsqrScalars* sc, cudaStream_t st);
ski_status ski_csc_launch(int64_t d, const int64_t* colptr, const int32_t* rowidx, const double* cval,
                          const double* t, double* q, const LsqrScalars* sc, cudaStream_t st);
ski_status ski_reduce_launch(int nblk, int64_t d, const double* part, int64_t ldp, const double* part_tt,
                             const double* part_aa, double* q, LsqrScalars* sc, int mode, cudaStream_t st,
                             int shard = 0);

ski_status ski_norm_launch(int64_t d, const double* q, LsqrScalars* sc, cudaStream_t st);
ski_status ski_copy_launch(int64_t n, const double* a, double* b, cudaStream_t st);
ski_status ski_cg_launch(int64_t d, const double* q, double* r, double* p, double* z, LsqrScalars* sc, int start,
                         cudaStream_t st);
ski_status ski_outer_launch(int64_t n, int64_t d, const double* r, const double* lam, const double* al,
                            const double* x, double* dA, int64_t ld_da, cudaStream_t st);
ski_status ski_scale_launch(int64_t rows, int64_t cols, double* Y, int64_t ldy, double s, cudaStream_t st);
// R[i][i] += delta for i < d (R row-major, ldr)
ski_status ski_add_diag_launch(int64_t d, double* R, int64_t ldr, double delta, cudaStream_t st);
ski_status ski_scale_f32_launch(int64_t rows, int64_t cols, float* Y, int64_t ldy, float s, cudaStream_t st);

// csc.cu: deterministic CSR -> CSC transpose (row indices ascending per column).
size_t ski_csc_ws_bytes(int64_t n, int64_t d, int64_t nnz);
ski_status ski_csc_build(const ski_matrix* A, int64_t* colptr, int32_t* rowidx, double* cval, SkiArena& ar,
                         cudaStream_t st);
