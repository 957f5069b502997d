/*
 * skills.h -- C ABI of the GB300 (sm_103a) Ski-LLS hot path.
 *
 * The library solves the linear least-squares problem min_x ||A x - b||_2
 * (Eq. LLS-statement; A is n x d, n >= d) by Algorithm 1 of Cartis, Fiala &
 * Shao, "Hashing embeddings of optimal dimension, with applications to linear
 * least squares" (arXiv 2105.11815):
 *   Step 1  sketch: SA = S A and Sb = S b with S an s-hashing matrix (Def. 5),
 *           optionally after the randomised Walsh-Hadamard premix H D (Def. 8);
 *   Step 2  factor SA = Q R (Householder QR; plain QR since SA has full rank);
 *   Step 3  x_s = R^{-1} Q^T Sb, accepted when ||A x_s - b|| <= tau_a;
 *   Step 4  LSQR on min ||W y - b|| with W = A R^{-1}, stopped by Eq. TC-lsqr;
 *   Step 5  x = R^{-1} y.
 *
 * Conventions for every entry point:
 *   - Pointers named as device pointers must be device memory of the current
 *     CUDA device; the caller owns all memory and the library frees nothing.
 *   - Scratch memory is caller-provided (`ws`, `ws_bytes`); each entry point
 *     that needs it has a *_workspace_size query.  A too-small workspace
 *     returns SKI_ENOMEM before any launch.  Workspace base pointers must be
 *     256-byte aligned (cudaMalloc / the PyTorch allocator give this).
 *   - Work is enqueued on `stream` (a cudaStream_t, NULL = legacy default).
 *     Entry points documented as synchronous synchronise that stream before
 *     returning.
 *   - Argument errors are detected on the host before any launch and return
 *     SKI_EINVAL.  CUDA launch/runtime errors return SKI_ECUDA.  No exception
 *     crosses the ABI.
 *   - Dense matrices are row-major with an explicit leading dimension (row
 *     stride, in elements).  Element counts are int64.
 */
#ifndef SKILLS_H
#define SKILLS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SKI_OK = 0,
  SKI_EINVAL = 1,      /* bad argument (detected on the host, nothing launched)   */
  SKI_ENOMEM = 2,      /* caller workspace smaller than the *_workspace_size query */
  SKI_ECUDA = 3,       /* a CUDA call failed                                       */
  SKI_ENONFINITE = 4,  /* NaN/Inf met in the sketch, the factor or the residual    */
  SKI_ESINGULAR = 5,   /* numerical rank of R below d under the rcond rule         */
  SKI_ENOCONV = 6,     /* it_max LSQR iterations without meeting the tolerance     */
  SKI_ETIMEOUT = 7     /* a bounded device-side wait gave up                       */
} ski_status;

/* SKI_TF32 is a QR precision only (qr_dtype, ski_precondition's sa_dtype): FP32
 * storage with the trailing-update products in one TF32 tensor-core pass (11
 * significant bits), where SKI_F32 takes three passes (about FP32 accuracy). */
typedef enum { SKI_F64 = 0, SKI_F32 = 1, SKI_BF16 = 2, SKI_TF32 = 3 } ski_dtype;
typedef enum { SKI_DENSE = 0, SKI_CSR = 1 } ski_kind;
/* The sketching matrix: s-hashing (Def. 5), the s-hashing variant (Def. 7), or
 * the sampling matrix S_s of Eq. SR-DHT (one 1 per row, in a column drawn
 * uniformly with replacement). */
typedef enum { SKI_S_HASHING = 0, SKI_S_HASHING_VARIANT = 1, SKI_SAMPLING = 2 } ski_hash_kind;

/* The data matrix A (n x d).  Values are FP64 in both layouts. */
typedef struct {
  int32_t kind;           /* SKI_DENSE or SKI_CSR                                      */
  int32_t pad_;
  int64_t n, d;           /* rows, columns; n >= 1, d >= 1                             */
  int64_t ld;             /* SKI_DENSE: row stride in elements, ld >= d                */
  const double* val;      /* device. SKI_DENSE: n x d row-major. SKI_CSR: [nnz] values */
  const int64_t* rowptr;  /* SKI_CSR: device [n+1], rowptr[0] = 0, non-decreasing      */
  const int32_t* colidx;  /* SKI_CSR: device [nnz], each in [0, d), distinct in a row  */
  int64_t nnz;            /* SKI_CSR: number of stored entries                        */
} ski_matrix;

/* Parameters of Algorithm 1 (names as in the paper's Section 6). */
typedef struct {
  uint64_t seed;          /* draws S (Def. 5) and D (Def. 8) through the counter hash  */
  int32_t s;              /* nonzeros per column of S, 1 <= s <= m                     */
  int32_t premix;         /* 1: S = S_h H D (Def. 8); 2: S = S_h F D, F the normalised */
                          /* discrete Hartley transform (Eq. HR-DHT); dense A only;    */
                          /* 0: S = S_h                                                */
  int64_t m;              /* sketch rows, d <= m < 2^31                                */
  int64_t n_pad;          /* premix height N >= n: premix 1 a power of two (0: the     */
                          /* next); premix 2 an integer whose prime factors are all    */
                          /* <= 13 ([D A; 0] zero-padded to N rows; 0: the smallest    */
                          /* such N >= n, n itself when n is one)                      */
  int32_t sketch_dtype;   /* ski_dtype of the premix, the sketch and its output SA     */
  int32_t qr_dtype;       /* QR of SA: SKI_F64, SKI_F32 (tensor-core products in three  */
                          /* TF32 passes) or SKI_TF32 (one); R kept in FP64.  R^{-1} is */
                          /* formed in FP32 unless the FP64 form is needed (inv_dtype) */
  double tau_a;           /* Step 3: accept x_s when ||A x_s - b|| <= tau_a            */
  double tau_r;           /* Step 4: LSQR tolerance of Eq. TC-lsqr                     */
  double tol;             /* acceptance: ||A^T r|| / (||A||_F ||r||) <= tol, 0 = off   */
  double rcond;           /* rank rule: |r_qq| >= rcond |r_11| for all q               */
  double perturb;         /* > 0: divide by r_ii + perturb when R fails the rank rule  */
  int64_t it_max;         /* Step 4 iteration cap                                       */
  int32_t streams;        /* batched entry points: problems in flight, each on its own */
                          /* stream and workspace slice; 0 = min(nprob, 8), max 32      */
  int32_t premix_slab;    /* premix + hash run in column slabs of this many columns     */
                          /* (a multiple of 32, <= 128) kept in L2; 0 = auto            */
  /* Launch parameters of Steps 4-5 (the result is the same up to rounding; the
     Python autotuner times them per problem shape and caches the fastest):    */
  int32_t lsqr_pass;      /* dense LSQR pass over A: 0 = auto (4 for d <= 2048, 5 for  */
                          /* 2048 < d <= 4096, else 1), 1 = register-                   */
                          /* blocked rows, 2 = TMA-staged row ring, 3 = row per warp,   */
                          /* 4 = register-blocked with twice the rows per row group,    */
                          /* 5 = register-blocked with the next row group's loads       */
                          /* issued before this group's reductions (d <= 4096)          */
  int32_t lsqr_ctas;      /* CTAs of that pass, i.e. row tiles of ceil(n / ctas) rows; */
                          /* 0 = auto (min(152, n / 16)); raised to n / 16384 at least  */
  int32_t graphs;         /* 1: each chunk of 8 LSQR (or CG) iterations is recorded    */
                          /* once per solve as a CUDA graph and replayed; 0: launched   */
  int32_t hash_kind;      /* ski_hash_kind of S_h: 0 = s-hashing (Def. 5: s distinct    */
                          /* rows per column), 1 = the s-hashing variant (Def. 7: s     */
                          /* rows drawn with replacement, coinciding entries add),      */
                          /* 2 = sampling S_s (Eq. SR-DHT: row i of SA is row c_i of    */
                          /* the (premixed) [A | b]; s = 1, dense A, premix 0 or 2)     */
  int32_t factorization;  /* Step 2 when R fails the rank rule (Remark (i)):            */
                          /* 0 = SKI_ESINGULAR, or the perturbed back-solve when        */
                          /* perturb > 0; 1 = column-pivoted QR (SA V = Q R with        */
                          /* R = [R11 R12; 0 0], R11 p x p), Steps 3-5 on W = A V1      */
                          /* R11^{-1}; dense A only (CSR keeps the behaviour of 0);     */
                          /* 2 = R the Cholesky factor of SA^T SA (R^T R = SA^T SA,     */
                          /* positive diagonal) and Q^T Sb = R^{-T} SA^T Sb: for CSR A  */
                          /* (FP64 factor) from a sparse SA kept in CSR (Section 6),    */
                          /* for dense A from the dense sketch in the QR precision;     */
                          /* the Householder QR when the Cholesky breaks down or       */
                          /* max_j |SA_j| / r_jj passes 2^23 (FP64) / 2^9 (FP32);       */
                          /* then as 0                                                  */
  int32_t batch_lsqr;     /* ski_solve_batched, dense problems: 0 = each problem's own  */
                          /* Step 4 launches on its stream; 1 = Step 4 of all problems  */
                          /* in flight grouped, one launch per kernel of an iteration   */
                          /* over (problem, block) work items (same results)            */
  int64_t row_offset;     /* A holds rows [row_offset, row_offset + n) of a larger      */
                          /* matrix: the sketch entry points draw the columns of S for */
                          /* those global rows, so the sketches of row blocks sum to   */
                          /* the sketch of the whole (row-block sharding); 0 for a     */
                          /* whole A; premix and the solve entry points need 0         */
} ski_opts;

/* Result record of a solve (host memory). */
typedef struct {
  int64_t iters;          /* LSQR iterations (Step 4), summed over restarts          */
  int32_t restarts;       /* LSQR restarts made to meet `tol`                        */
  int32_t rank;           /* numerical rank p of R under the rcond rule              */
  int32_t early_exit;     /* 1 when Step 3 accepted x_s                               */
  int32_t status;         /* ski_status of the solve                                  */
  double metric;          /* ||A^T r|| / (||A||_F ||r||), r = b - A x, FP64          */
  double resid_norm;      /* ||b - A x||_2                                            */
  double anorm_f;         /* ||A||_F                                                  */
  double lsqr_test;       /* last Eq. TC-lsqr estimate                                */
  float ms_sketch, ms_qr, ms_trinv, ms_lsqr, ms_total;  /* stage times, CUDA events */
  float ms_premix, ms_gather;  /* inside ms_sketch: the H D premix and the hash gather */
  float ms_qr_gemm;            /* inside ms_qr: the trailing-update GEMMs, summed     */
                               /* (Step 2 from the Gram matrix: its product SA^T SA)  */
  int32_t qr_fallback;         /* mixed form: 0 kept the FP32/TF32 factor; 1 redid     */
                               /* Steps 1-2 in FP64 (ratio or rank), 2 after its LSQR  */
                               /* run exhausted, or was predicted to exceed, a budget  */
                               /* (ski_mixed_lsqr_budget).  FP64 factor: 3 when its    */
                               /* FP32 inverse met that budget and was redone in FP64  */
  int32_t inv_dtype;           /* precision M = R^{-1} was formed in at the end:        */
                               /* SKI_F32 when max|r_ii|/min|r_ii| <= 2^19 (the FP32   */
                               /* factor's limit) and no fallback, else SKI_F64; the   */
                               /* preconditioner is applied in FP64 either way         */
  double rdiag_ratio;          /* max |r_ii| / min |r_ii| of the first factor (the     */
                               /* requested precision; it decides the fallback)        */
  int32_t pivoted;             /* 1 when Step 2 took the column-pivoted QR: rank is   */
                               /* then p of R11, and x is zero outside V1's columns    */
  int32_t gram;                /* 1 when R came from the Cholesky factor of the sparse */
                               /* sketch's Gram matrix (factorization 2)              */
} ski_info;

/* Defaults of Ski-LLS-dense (Section 6): m = 0 (caller must set), s = 1,
 * tau_a = 1e-8, tau_r = 1e-6, it_max = 1e4, rcond = 1e-12; here also
 * tol = 0, perturb = 0, premix = 0, FP64 sketch and QR. */
void ski_opts_default(ski_opts* o);

/* Human-readable name of a ski_status.  Never NULL. */
const char* ski_status_string(int32_t status);

/* ABI version (major * 100 + minor). */
int32_t ski_version(void);

/* cudaError_t code of the last CUDA call that failed in this host thread
 * (the cause behind a SKI_ECUDA), 0 when none has failed. */
int32_t ski_last_cuda_error(void);

/* Number of CUDA kernels this library has launched in the process so far
 * (all threads).  Diagnostic: lets a caller count the kernels of a region. */
int64_t ski_launch_count(void);

/* LSQR iterations the mixed form (qr_dtype or sketch_dtype not SKI_F64) runs
 * with its FP32 / TF32 factor before Steps 1-2 are redone in FP64 (reported as
 * ski_info.qr_fallback = 2), and an FP64 factor with its inverse formed in FP32
 * runs before that inverse is redone in FP64 (qr_fallback = 3).  Theorem 10 bounds the iterations with an
 * eps-subspace embedding by (log 2 + |log tau_r|) / |log eps|; a hashing sketch
 * of m rows for d columns embeds with eps ~ sqrt(d / m) (m = O(d / eps^2)).
 * The budget is ceil(2.2 * that bound) at eps = sqrt(d / m), at least 150 and
 * at most 4000; 150 when tau_r is not in (0, 1) or d < 1, 4000 when m <= d.
 * Host only: launches nothing. */
int64_t ski_mixed_lsqr_budget(int64_t m, int64_t d, double tau_r);

/*
 * ski_selftest_wait_timeout -- checks the library's bounded device-side wait
 * (the grid barrier of the persistent QR panel kernel) on the GPU without a
 * fault: 4 co-resident CTAs wait for a fifth that never arrives, each poll
 * loop gives up after spin_limit polls (~64 ns each) and sets an error flag.
 * Returns SKI_ETIMEOUT when the wait timed out as designed (the expected
 * result), SKI_OK if it did not.  ws: device scratch of >= 16 bytes.
 * Synchronous.
 */
ski_status ski_selftest_wait_timeout(int64_t spin_limit, void* ws, size_t ws_bytes, void* stream);

/*
 * ski_hash_indices -- the nonzeros of the s-hashing matrix S (Def. 5).
 * Column j < n of S (multiplying row j of A) holds sign[j*s+k] / sqrt(s) in row
 * idx[j*s+k], k < s; the s rows are distinct (drawn without replacement).
 * The draw is a counter hash: with sm() the SplitMix64 output function
 * (Steele, Lea & Flood 2014) and key(tag, j, k, t) =
 * sm(sm(sm(seed ^ tag << 56) ^ j) ^ (k << 32 | t)) modulo 2^64, nonzero k takes
 * row floor(key(0xB1, j, k, t) * m / 2^64) for the first retry t = 0, 1, ...
 * whose row differs from those of nonzeros 0..k-1, and sign -1 exactly when
 * the top bit of key(0x5A, j, k, 0) is set.  D of Def. 8 uses key(0xD3, j, 0, 0).
 *   idx  device int32 [n*s], sign device int8 [n*s] (+1 / -1).
 * Asynchronous.  Errors: SKI_EINVAL unless 1 <= s <= min(m, 64), m < 2^31
 * and n >= 0.
 */
ski_status ski_hash_indices(uint64_t seed, int32_t s, int64_t m, int64_t n,
                            int32_t* idx, int8_t* sign, void* stream);

/*
 * ski_hash_variant_indices -- the draws of the s-hashing variant T (Def. 7).
 * Column j < n of T adds sign[j*s+k] / sqrt(s) to row idx[j*s+k] for each
 * k < s; the s rows are drawn with replacement, so two draws may name the same
 * row, whose entry is then their sum (0 or +-2/sqrt(s) when s >= 2).  Draw k
 * is the retry-0 draw of ski_hash_indices: row floor(key(0xB1, j, k, 0) * m /
 * 2^64), sign from key(0x5A, j, k, 0).  Wherever the s rows of a column of T
 * are distinct, that column equals the column of the s-hashing matrix with
 * the same seed; with s = 1 the two are the same 1-hashing matrix.  Setting
 * ski_opts.hash_kind = 1 sketches with T (Lemma 5: T = (S1 + ... + Ss) / sqrt(s)
 * for independent 1-hashing matrices Sk).
 *   idx  device int32 [n*s], sign device int8 [n*s] (+1 / -1).
 * Asynchronous.  Errors: SKI_EINVAL unless 1 <= s <= 64, 1 <= m < 2^31 and
 * n >= 0.
 */
ski_status ski_hash_variant_indices(uint64_t seed, int32_t s, int64_t m, int64_t n,
                                    int32_t* idx, int8_t* sign, void* stream);

/*
 * ski_premix_signs -- the diagonal of D in the HRHT premix (Def. 8), D[j] in
 * {+1, -1} for j < n.  D: device int8 [n].  Asynchronous.
 */
ski_status ski_premix_signs(uint64_t seed, int64_t n, int8_t* D, void* stream);

/*
 * ski_premix -- Y = H D [A b ; 0] for the n_pad x n_pad normalised
 * Walsh-Hadamard matrix H_ij = n_pad^{-1/2} (-1)^{<(i-1)_2,(j-1)_2>} (Def. 8),
 * or, with o->premix = 2, Y = F D [A b ; 0] for the N x N normalised discrete
 * Hartley matrix F_ij = N^{-1/2} cas(2 pi i j / N), cas = cos + sin
 * (Section 6, Eq. HR-DHT; N = o->n_pad or the default length described at
 * ski_opts.n_pad), computed by a mixed-radix FFT in the sketch precision.
 * A dense FP64 n x d; b device FP64 [n] or NULL.  Y: device, n_pad (N) rows of
 * d (+1 when b != NULL) columns, row stride ld_y, element type o->sketch_dtype
 * (FP64 or FP32).  Asynchronous.  Uses o->seed, o->premix and o->n_pad.
 * Walsh-Hadamard: a NaN or Inf in a column of [A b] makes that column of Y
 * NaN (FP64 also when a bounded wait of the first pass gave up: then all of
 * Y); Hartley: it spreads through the FFT of that column.
 */
size_t ski_premix_workspace_size(const ski_matrix* A, int32_t with_b, const ski_opts* o);
ski_status ski_premix(const ski_matrix* A, const double* b, const ski_opts* o,
                      void* Y, int64_t ld_y, void* ws, size_t ws_bytes, void* stream);

/*
 * ski_sketch_hash -- Step 1 of Algorithm 1: [SA | Sb] with S the s-hashing
 * matrix (Def. 5), or S = S_h H D (Def. 8) when o->premix = 1, or
 * S = S_h F D (Eq. HR-DHT) when o->premix = 2; with o->hash_kind = 2 the
 * sampling S_s takes the place of S_h (Eq. SR-DHT).
 *   SA  device, m rows, row stride ld_sa, element type o->sketch_dtype;
 *       columns 0..d-1 receive S A and, when b != NULL, column d receives S b.
 *       ld_sa >= d + (b != NULL).
 * Row i of SA is the sum over the rows j hashed to i of sign/sqrt(s) * A[j,:],
 * formed per output element in a fixed order (deterministic, bit-reproducible
 * for a given seed).  Asynchronous.  With the FP64 premix, a NaN or Inf in a
 * column of [A b] makes that column of SA NaN, and a bounded wait of the
 * premix that gave up makes all of SA NaN (ski_solve returns SKI_ETIMEOUT).
 */
size_t ski_sketch_workspace_size(const ski_matrix* A, int32_t with_b, const ski_opts* o);
ski_status ski_sketch_hash(const ski_matrix* A, const double* b, const ski_opts* o,
                           void* SA, int64_t ld_sa, void* ws, size_t ws_bytes, void* stream);

/*
 * ski_sketch_hash_noalloc -- ski_sketch_hash for callers that cannot allocate
 * device memory (no cudaMalloc of their own, no workspace to pass).  The
 * paper has no counterpart.
 *   Same arguments and result as ski_sketch_hash without `ws`/`ws_bytes`; the
 *   bucket-list scratch lives in one 4 MiB __device__ array inside this
 *   library, held by every GPU that loads it until the process exits.
 *   Limits: o->premix = 0 (the premix needs O(n_pad * d) scratch), rows * s
 *   <= 262144 and m <= 32768; beyond them SKI_EINVAL, with nothing launched.
 *   Allocates nothing (no cudaMalloc/cudaFree, no allocating library call).
 *   Each call looks up the array's device address on the current device; the
 *   first call on a device may load the module there, so make that first
 *   call before any stream capture.  Every
 *   call reuses the same array, so calls that overlap on the GPU race: the
 *   caller must serialise them.  Asynchronous.
 */
ski_status ski_sketch_hash_noalloc(const ski_matrix* A, const double* b, const ski_opts* o,
                                   void* SA, int64_t ld_sa, void* stream);

/*
 * ski_precondition -- Step 2 of Algorithm 1: Householder QR of SA (m x d,
 * d <= m), applying every reflector also to column d when with_rhs = 1 so that
 * column d becomes Q^T Sb.
 *   SA     device, m x (d + with_rhs), row stride ld_sa, element type sa_dtype
 *          (FP64, or FP32 for SKI_F32 and SKI_TF32, which differ in the
 *          tensor-core passes of the trailing update); overwritten.
 *   R      device FP64 d x d (row stride ldr): the upper triangle receives R,
 *          the strict lower triangle is set to zero.
 *   qtsb   device FP64 [d] or NULL: receives (Q^T Sb)[0..d-1] (with_rhs = 1).
 *   rank   host int32 or NULL: numerical rank under o->rcond (synchronises).
 * The factorisation runs in sa_dtype; R is returned in FP64.  Asynchronous
 * unless rank != NULL.
 */
size_t ski_precondition_workspace_size(int64_t m, int64_t d, int32_t with_rhs, int32_t sa_dtype);
ski_status ski_precondition(int64_t m, int64_t d, int32_t with_rhs, void* SA, int64_t ld_sa,
                            int32_t sa_dtype, double* R, int64_t ldr, double* qtsb,
                            int32_t* rank, const ski_opts* o, void* ws, size_t ws_bytes,
                            void* stream);

/*
 * ski_gemm_tc_f32 -- C = A B^T (subtract = 0) or C -= A B^T (subtract = 1)
 * on the TF32 tensor cores with FP32 accumulation: the kernel of the FP32
 * trailing update of Step 2, exposed for testing and reuse.  A: M x K,
 * B: N x K, C: M x N, all device FP32 row-major; lda and ldb multiples of 4
 * with 16-byte aligned bases (SKI_EINVAL otherwise).  passes = 1: products
 * of the operands rounded to TF32 (11 significant bits); passes = 3: each
 * operand split as hi + lo (both TF32) and lo*hi + hi*lo + hi*hi accumulated
 * (error about 2^-21 |a||b| per product).  ws: device scratch >= 4 bytes (an
 * error flag).  Synchronous; SKI_ETIMEOUT if a bounded wait gave up.
 */
ski_status ski_gemm_tc_f32(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda, const float* B,
                           int64_t ldb, float* C, int64_t ldc, int32_t subtract, int32_t passes, void* ws,
                           size_t ws_bytes, void* stream);

/*
 * ski_trinv -- M = R^{-1} for an upper-triangular d x d R (FP64, row stride
 * ldr), written to M (FP64, row stride ldm; strict lower triangle zero) and
 * its transpose to Mt (row stride ldm) when Mt != NULL.  Computed in dtype
 * (FP64 or FP32) and returned in FP64.  When perturb > 0 every diagonal
 * r_ii is replaced by r_ii + perturb (the perturbed back-solve of Ski-LLS-sparse).
 * The library applies R^{-1} as this explicit triangular matrix instead of a
 * back-substitution (Remark (iii) only asks that no inverse of SA is formed).
 */
size_t ski_trinv_workspace_size(int64_t d, int32_t dtype);
ski_status ski_trinv(int64_t d, const double* R, int64_t ldr, double* M, double* Mt, int64_t ldm,
                     int32_t dtype, double perturb, void* ws, size_t ws_bytes, void* stream);

/*
 * ski_solve -- Algorithm 1 end to end.  x: device FP64 [d].  info: host, may
 * be NULL.  R_out: device FP64 d x d (row stride d) or NULL, receives R (for a
 * later ski_solve_adjoint): the plain QR factor of SA, with perturb added to
 * its diagonal when the perturbed back-solve was taken.  With
 * o->factorization = 1 and a sketch that fails the rank rule, Step 2 takes the
 * column-pivoted QR: info->pivoted = 1, info->rank = p, and x is zero outside
 * the p pivoted columns (the basic solution of Theorem 8).  With o->tol > 0
 * the acceptance metric ||A^T r|| / (||A||_F ||r||) is formed from the plain
 * FP64 r = b - A x, and again from r by compensated (twice-working-precision)
 * dot products whenever the plain value's estimated rounding noise could
 * decide the test (x large along small singular directions), so that it
 * certifies x.  Synchronous.  Returns SKI_ESINGULAR when R fails the rank rule with
 * o->perturb = 0 and o->factorization = 0, SKI_ENOCONV when it_max is reached
 * before the tolerances (x then holds the last iterate), SKI_ENONFINITE on
 * NaN/Inf.
 */
size_t ski_solve_workspace_size(const ski_matrix* A, const ski_opts* o);

/*
 * The sum over the processes of a row-block solve: replace the `count`
 * elements of type `dtype` (ski_dtype) at the device address `buf` by their
 * sum over all processes, in the order of `stream` (e.g. an NCCL all-reduce
 * enqueued on it, or a synchronise-copy-add-copy); every process must see the
 * same sum.  Returns SKI_OK, or a status that ends the solve.
 */
typedef ski_status (*ski_allreduce_fn)(void* buf, int64_t count, int32_t dtype, void* ctx, void* stream);

/*
 * ski_solve_rowblock -- Algorithm 1 on A split by rows over processes (one
 * GPU each).  The paper solves on one machine; this is the data-parallel form
 * of the same computation.  This process holds rows [o->row_offset,
 * o->row_offset + A->n) of the whole A and the same rows of b; x (device FP64
 * [d]) receives the whole solution on every process.
 *   Step 1: each process sketches its rows with the columns of S of its
 *     global rows, and one sum of [SA | Sb] (m x ld_sa) gives every process
 *     S A = sum over row blocks of S[:, rows] A[rows, :] (Def. 5); Steps 2-3
 *     then run on every process on the same sketch.
 *   Step 4: every LSQR iteration sums A^T t (d) and ||t||^2 over the
 *     processes; the residual passes of Steps 3 and 5 sum A^T r, ||r||^2 and
 *     ||A||_F^2.  All other work is local or repeated on every process.
 * Same options, workspace query (ski_solve_workspace_size of the local
 * block), statuses and report as ski_solve, except: o->premix must be 0 (H D
 * mixes every row of A), A->n may be below d, graph replay is off, and
 * `allreduce` is called with the same sequence of buffers on every process
 * (a collective).  Synchronous.  SKI_EINVAL when allreduce is NULL.
 */
ski_status ski_solve_rowblock(const ski_matrix* A, const double* b, const ski_opts* o, double* x,
                              double* R_out, ski_info* info, void* ws, size_t ws_bytes, void* stream,
                              ski_allreduce_fn allreduce, void* ctx);
ski_status ski_solve(const ski_matrix* A, const double* b, const ski_opts* o, double* x,
                     double* R_out, ski_info* info, void* ws, size_t ws_bytes, void* stream);

/*
 * ski_solve_batched -- nprob independent problems (ragged n_i, d_i), each
 * solved as ski_solve with the same options except m_i = ceil(gamma * d_i)
 * when o->m <= 0 (gamma = -o->m / 1000, e.g. m = -2000 for gamma = 2) and
 * seed_i = o->seed + i.  Not in the paper, which solves one problem: this is
 * the throughput form for many small problems.  A, b, x, R_out, info are host
 * arrays of nprob entries (R_out may be NULL, or hold NULL entries); b[i],
 * x[i], R_out[i] are device pointers.  W = o->streams problems (0: min(nprob,
 * 8)) are solved at once, each by a host worker on its own non-blocking
 * stream, largest problems first; work already queued on `stream` comes
 * first and `stream` is ordered after all of it.  A problem's results do not
 * depend on W or on which worker ran it.  The workspace holds W slices of the
 * largest single-problem workspace: ski_solve_batched_workspace_size gives
 * its size.  Synchronous.  Every problem is attempted unless a CUDA call
 * fails (SKI_ECUDA stops the batch); returns the status of the
 * lowest-numbered problem that did not return SKI_OK, else SKI_OK.
 * SKI_EINVAL for o->streams < 0 or an invalid problem.
 */
size_t ski_solve_batched_workspace_size(int32_t nprob, const ski_matrix* A, const ski_opts* o);
ski_status ski_solve_batched(int32_t nprob, const ski_matrix* A, const double* const* b,
                             const ski_opts* o, double* const* x, double* const* R_out,
                             ski_info* info, void* ws, size_t ws_bytes, void* stream);

/*
 * ski_solve_adjoint -- backward pass of x = argmin ||A x - b|| for an upstream
 * gradient g = dL/dx.  Solves (A^T A) lambda = g by conjugate gradients on the
 * R-preconditioned normal equations (W^T W z = R^{-T} g, lambda = R^{-1} z,
 * W = A R^{-1}, R from the forward solve), then forms
 *   db = A lambda          (device FP64 [n])
 *   dA = r lambda^T - (A lambda) x^T,  r = b - A x   (device FP64 n x d, row
 *        stride ld_da; skipped when dA == NULL).
 * Dense A only.  Stops when ||W^T W z - R^{-T} g|| <= o->tau_r ||R^{-T} g|| or
 * after o->it_max iterations (SKI_ENOCONV).  Synchronous.
 */
size_t ski_solve_adjoint_workspace_size(const ski_matrix* A, const ski_opts* o);
ski_status ski_solve_adjoint(const ski_matrix* A, const double* b, const double* x,
                             const double* R, int64_t ldr, const double* g, double* dA,
                             int64_t ld_da, double* db, const ski_opts* o, ski_info* info,
                             void* ws, size_t ws_bytes, void* stream);

/*
 * ski_solve_adjoint_batched -- ski_solve_adjoint for nprob independent dense
 * problems, W = o->streams at once as in ski_solve_batched (same stream
 * ordering, workspace slicing and status rule).  Host arrays of nprob device
 * pointers: b[i] [n_i], x[i] [d_i], R[i] (d_i x d_i, row stride d_i), g[i]
 * [d_i], db[i] [n_i], dA[i] (n_i x d_i, row stride d_i; dA may be NULL, or
 * hold NULL entries, to skip dA).  Synchronous.
 */
size_t ski_solve_adjoint_batched_workspace_size(int32_t nprob, const ski_matrix* A, const ski_opts* o);
ski_status ski_solve_adjoint_batched(int32_t nprob, const ski_matrix* A, const double* const* b,
                                     const double* const* x, const double* const* R,
                                     const double* const* g, double* const* dA, double* const* db,
                                     const ski_opts* o, ski_info* info, void* ws, size_t ws_bytes,
                                     void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SKILLS_H */
