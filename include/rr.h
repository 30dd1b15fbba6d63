/*
 * rr.h -- C ABI of the GB300 orthogonalization-free Rayleigh-Ritz library.
 *
 * Method: arXiv 2505.00281, "Mixed Precision Orthogonalization-Free
 * Projection Methods for Eigenvalue and Singular Value Problems".
 *   - Algorithm 1 (multi-step subspace iteration) coupled with the RR output
 *     as the next start block (Sec. 2),
 *   - Algorithm 3 (OFRR for eigenvalue problems: B = U^T A U, M = U^T U,
 *     B Y = M Y Lambda, U~ = U Y),
 *   - Algorithm 5 (OFRR for the SVD: the 2x2 block pencil, positive
 *     eigenvalues, lift sqrt(2) U Y, sqrt(2) V Z; theorem of Sec. 3.2),
 *   - Algorithm 8 (Hessenberg process for a block, the inner-product-free
 *     basis step; equal to row-pivoted LU, Sec. 4.2.2),
 *   - the mixed-precision map of Sec. 4.2 (Fig. 4): low-precision basis and
 *     products (BF16, or FP8-E4M3 with power-of-two scales), higher-precision
 *     projection, FP64 small solve.
 * Beyond the paper: a refinement phase to FP64-level residuals, batched
 * solves with tuned launch parameters, and the kernels of a learned start
 * block (its network's convolutions, loss gradient and optimiser).
 *
 * Conventions for every entry point:
 *   - All matrices are column-major ("Fortran", Sec. 5.1) with an explicit
 *     leading dimension unless the entry's comment gives another layout (the
 *     row-major blocks of rr_chebyshev_step_rows and rr_quantize_e4m3, the
 *     NCHW images of the convolution kernels); all matrix pointers are DEVICE
 *     pointers unless the comment says "host".
 *   - The caller owns every buffer.  The library allocates no device memory:
 *     scratch space is the caller's workspace (see rr_workspace_size).
 *   - Calls are asynchronous on `stream` (a cudaStream_t passed as void*;
 *     NULL = the legacy default stream) except where a comment says the call
 *     synchronises.  The solvers (rr_eig, rr_svd, rr_batch_svd) synchronise
 *     the stream to read convergence counts and return only when done.
 *   - Errors are returned as rr_status; nothing aborts or throws across the
 *     ABI.  RR_ERR_ARG: invalid sizes/pointers (nothing launched).
 *     RR_ERR_WORKSPACE: the workspace is missing, too small or not 256-byte
 *     aligned (nothing launched).  RR_ERR_NAN (solvers): every wanted
 *     residual is NaN after a projection, as when the operator holds a NaN
 *     or infinity (outputs undefined).
 *     RR_ERR_CUDA: a CUDA launch or runtime call failed (rr_last_error()
 *     returns its text).  RR_ERR_TIMEOUT: a device-side bounded wait gave up
 *     (the kernel returned early; outputs are undefined).
 */
#ifndef RR_H_
#define RR_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { RR_F64 = 0, RR_F32 = 1, RR_BF16 = 2, RR_E4M3 = 3, RR_F16 = 4 } rr_dtype;
/* (RR_F16: storage of the comparator basis builders only, rr_basis_builder.) */

typedef enum {
  RR_OK = 0,
  RR_ERR_ARG = 1,
  RR_ERR_CUDA = 2,
  RR_ERR_NOT_SPD = 3,
  RR_ERR_NO_CONV = 4,
  RR_ERR_TIMEOUT = 5,
  RR_ERR_WORKSPACE = 6,
  RR_ERR_NAN = 7
} rr_status;

enum { RR_DENSE = 0, RR_CSR = 1, RR_KERNEL = 2 };
enum { RR_LARGEST = 0, RR_SMALLEST = 1 };
enum { RR_POWER = 0, RR_CHEBYSHEV = 1 };
enum { RR_MGS_L = 0, RR_MGS_R = 1, RR_CGS = 2, RR_CGS2 = 3, RR_HESS_L = 4, RR_HESS_R = 5 };

/* The operator A.
 *   RR_DENSE:  m x n FP64, column-major, leading dimension ld >= m.
 *   RR_CSR:    square n x n (m == n), FP32 values, int32 row_ptr[n+1] and
 *              col_idx[nnz] (sorted within rows), symmetric (used by rr_eig).
 *   RR_KERNEL: the Gaussian kernel matrix of Sec. 2 / Sec. 5's kernel-matrix
 *              experiments, never stored (matrix-free):
 *              A(i, j) = f (exp(-|x_i - y_j|^2 / (2 l^2)) + s [i == j]),
 *              with (f, l, s) = kparams; values = the m points x_i (m x d
 *              FP64, column-major, ld >= m), points_y = the n points y_j
 *              (n x d, ld n) or NULL for the square symmetric operator over
 *              the x_i alone (the shift s applies only then); nnz = d
 *              (1 .. 8); dtype RR_F64.
 * All pointers are device pointers.  The library never writes to them. */
typedef struct {
  int32_t kind;
  int32_t dtype;
  int64_t m, n, ld, nnz;
  const void* values;
  const int32_t* row_ptr;
  const int32_t* col_idx;
  const double* points_y;  /* RR_KERNEL only */
  double kparams[3];       /* RR_KERNEL only: f, l, s */
} rr_operator;

/* Solver parameters (Algorithm 1 inputs A, k, m, iter; Sec. 4.2 precisions). */
typedef struct {
  int32_t k;             /* wanted pairs (k <= block)                                */
  int32_t block;         /* block size b (b <= 335, and b <= 167 with refinement)    */
  int32_t filter;        /* RR_POWER (products per sweep) or RR_CHEBYSHEV            */
  int32_t degree;        /* power: products per sweep (Alg. 1 "iter"); Chebyshev: d  */
  int32_t max_sweeps;    /* projections (Alg. 1 "m"), counting both phases           */
  int32_t which;         /* RR_LARGEST or RR_SMALLEST (RR_SMALLEST needs Chebyshev)  */
  int32_t basis;         /* RR_F64, RR_F32 or RR_BF16: storage of the basis and of
                            the operator copy the filter products use                */
  int32_t hessenberg;    /* 1: Algorithm 8 after each product; 0: inf-norm scaling   */
  int32_t refine;        /* 1: after `phase1_sweeps` projections, refine with FP64-
                            accurate residuals and low-precision corrections         */
  int32_t phase1_sweeps; /* projections of the plain (paper) phase before refining   */
  double tol;            /* relative residual target (Sec. 5.2.2)                    */
  double bounds[2];      /* Chebyshev: spectral bounds (lo, up); lo >= up -> computed */
  const double* v0;      /* n x block FP64 start block (device), e.g. U(0,1); NULL:
                            drawn U(0,1) on the device from `seed` (Alg. 1's random
                            start block, Sec. 5.2)                                   */
  int32_t profile;       /* 1: time every stage with CUDA events (rr_info.stage_ms)  */
  double hess_tol;       /* Algorithm 8's column-skip tolerance, relative to the
                            column's inf-norm; <= 0: 4 b eps of the arithmetic that
                            runs the process (Sec. 5.2 sets it from the machine
                            epsilon)                                                 */
  uint64_t seed;         /* start block generator seed when v0 is NULL (counter-
                            based splitmix64 stream, the one rr_batch_svd uses)      */
  int32_t refine_degree; /* SVD: products of the correction recurrence per
                            refinement sweep (0: degree)                             */
} rr_params;

typedef struct {
  int32_t n_converged;   /* wanted pairs with residual <= tol                        */
  int32_t sweeps;        /* projections performed                                    */
  int32_t refine_sweeps; /* of which in the refinement phase                         */
  int32_t cols_dropped;  /* basis columns the whitening dropped at the last projection
                            (columns Alg. 8 skipped are zero and counted here)       */
  double max_res;        /* largest residual among the k wanted pairs                */
  double res_history[64];/* max residual of the wanted pairs after each projection   */
  double stage_ms[8];    /* with params.profile: device time per stage (see below)   */
  int32_t stage_calls[8];/* number of timed calls per stage                          */
  double cond_G_est;     /* estimate of cond_2 of the Gram matrix (Alg. 3's M, Alg. 5's
                            larger of U^T U, V^T V) whitened at the last projection:
                            max_i G_ii * max_i (G^-1)_ii, with G^-1 = W W^T from the
                            whitener; a lower bound within a factor b^2 of cond_2    */
  double cond_history[64];/* cond_G_est after each projection                        */
  double tc_bytes;       /* with params.profile: algorithmic bytes of the launches
                            timed in stage_ms[RR_KERNEL_TC]                          */
  int32_t polish_sweeps; /* SVD refinement sweeps run as the FP64 polish (the
                            method's sweep in FP64-accurate arithmetic from the Ritz
                            vectors, taken when the corrections stop contracting the
                            residual, and as a batched problem's last two sweeps)    */
  double tc_role_ms[2];   /* with params.profile: stage_ms[RR_KERNEL_TC] split by the
                            launch's role: [0] low-precision products (filter,
                            split corrections, E4M3), [1] FP64-emulation passes
                            (FP64-accurate products, Grams, lifts)                  */
  double tc_role_bytes[2];/* algorithmic bytes of those launches (as tc_bytes)        */
  double tc_role_flops[2];/* algorithmic flops: 2 M N K per product formed (per slice
                            pair of an emulation pass)                              */
} rr_info;

/* Stages of rr_info.stage_ms: */
enum {
  RR_STAGE_LOWP_PRODUCT = 0, /* low-precision block products (filter, corrections)   */
  RR_STAGE_F64_PRODUCT = 1,  /* FP64-accurate products with A (residuals)            */
  RR_STAGE_HESSENBERG = 2,   /* Algorithm 8                                          */
  RR_STAGE_GRAM = 3,         /* projection products G, H / B                         */
  RR_STAGE_PENCIL = 4,       /* small FP64 pencil solve                              */
  RR_STAGE_LIFT = 5,         /* Ritz lift                                            */
  RR_STAGE_OTHER = 6,        /* casts, scaling, residual norms, projections          */
  RR_KERNEL_TC = 7           /* not a stage: every launch of the tensor-core product
                                kernel, in whichever stage it ran (filter products,
                                corrections, FP64-emulation passes); its algorithmic
                                bytes (operands read once, output written once) are
                                in rr_info.tc_bytes                                  */
};

/* Number of kernels this library has launched in this process so far. */
uint64_t rr_kernel_launches(void);

/* Text of the last RR_ERR_CUDA (thread-local, static storage). */
const char* rr_last_error(void);

/* Failure detection (every device-side wait of the library is bounded):
 * runs one of the library's waits where nothing can ever release it and
 * returns what the kernel reported.  mode 0: the grid barrier of the
 * cooperative kernels (Hessenberg, block Jacobi), entered by one CTA of a
 * grid that counts two; mode 1: the mbarrier wait of the tensor-core
 * kernels on a barrier nothing arrives on.  The wait gives up after
 * limit_ns (1 .. 1e10), records RR_ERR_TIMEOUT and the kernel returns, so
 * the expected result is RR_ERR_TIMEOUT with the context still usable.
 * scratch: 16 bytes of device memory (16-byte aligned), zeroed by the call.
 * Synchronises `stream`.  The paper has no counterpart. */
rr_status rr_wait_selftest(int32_t mode, int64_t limit_ns, void* scratch, void* stream);

/* ---------------------------------------------------------------------------
 * Solvers
 * ------------------------------------------------------------------------- */

/* Bytes of device workspace rr_eig (svd = 0) or rr_svd (svd = 1) needs.
 * The workspace must start on a 256-byte boundary (as cudaMalloc's blocks do;
 * RR_ERR_WORKSPACE otherwise). */
size_t rr_workspace_size(const rr_operator* A, const rr_params* p, int svd);

/* Wanted eigenpairs of a symmetric operator (dense n x n or CSR).
 * theta: k FP64 (device), ordered by `which`; X: n x k FP64 (device, ld n),
 * unit 2-norm columns, sign fixed so the largest-|.| entry is positive.
 * Returns RR_ERR_NO_CONV (outputs filled with the best pairs) when fewer than
 * k pairs reached tol within max_sweeps.  Synchronises `stream`. */
rr_status rr_eig(const rr_operator* A, const rr_params* p, double* theta, double* X,
                 void* ws, size_t ws_bytes, rr_info* info, void* stream);

/* Largest k singular triplets of a dense m x n operator (m >= n) (Alg. 5).
 * sigma: k FP64 descending; U: m x k; V: n x k (device, FP64, unit columns,
 * sign fixed so the largest-|.| entry of v is positive).  Synchronises. */
rr_status rr_svd(const rr_operator* A, const rr_params* p, double* sigma, double* U,
                 double* V, void* ws, size_t ws_bytes, rr_info* info, void* stream);

/* Launch parameters of the batched SVD (chosen per size class by the
 * package's autotuner): branches = concurrent graph branches (1..64, default
 * 16), max_splits = upper bound on the K splits of each tensor-core product
 * (0 = as many as fill the GPU, the single-problem choice), order = 0 (as
 * given) or 1 (largest m n first), fixed_sweeps = 0 (default: each problem
 * stops at tol under device-side loop control) or 1 (every problem runs
 * max_sweeps sweeps, keeping the triplets it reached tol with). */
typedef struct {
  int32_t branches;
  int32_t max_splits;
  int32_t order;
  int32_t fixed_sweeps;
} rr_batch_tuning;

/* Bytes of device workspace rr_batch_svd needs for `count` operators. */
size_t rr_batch_workspace_size(int32_t count, const rr_operator* A, const rr_params* p);

/* `count` independent rr_svd problems (host arrays of operators and of device
 * output pointers).  One parameter set for all (p->v0 is ignored; each problem
 * draws its start block from U(0,1) with a counter-based generator seeded by
 * `seed` + problem index).  per_problem (host, count entries) and info (host,
 * count entries) receive each problem's status and counts.  The batch runs
 * as captured CUDA graphs launched in order on `stream` (one graph per 16
 * problems; with fixed_sweeps one per up to 4096 problem-sweeps), the host
 * capturing the next graph while the GPU runs the earlier ones.  A problem's
 * first sweep is captured as plain
 * graph nodes and its later sweeps run inside WHILE graph nodes: after each
 * sweep a kernel checks the k wanted residuals against tol and the sweep
 * count against max_sweeps and sets the node's condition, so every problem
 * stops on the GPU as soon as it converges (info[i].sweeps = the sweeps it
 * ran).  With the mixed-precision refinement, a problem whose correction
 * sweeps stop contracting its residual (largest wanted residual above 0.3
 * times the previous sweep's), or that reaches the last two of max_sweeps,
 * continues with FP64 polish sweeps (the correction sweep in FP64-accurate
 * arithmetic).  Synchronises. */
rr_status rr_batch_svd(int32_t count, const rr_operator* A, const rr_params* p, uint64_t seed,
                       double* const* sigma, double* const* U, double* const* V,
                       void* ws, size_t ws_bytes, rr_status* per_problem, rr_info* info,
                       void* stream);
/* rr_batch_svd with explicit launch parameters (NULL: the defaults above);
 * RR_ERR_ARG for parameters out of range. */
rr_status rr_batch_svd_tuned(int32_t count, const rr_operator* A, const rr_params* p, uint64_t seed,
                             double* const* sigma, double* const* U, double* const* V, void* ws,
                             size_t ws_bytes, const rr_batch_tuning* tuning, rr_status* per_problem,
                             rr_info* info, void* stream);

/* ---------------------------------------------------------------------------
 * Stage entry points (the hot-path steps, callable on their own)
 * ------------------------------------------------------------------------- */

/* Start block and casts (Sec. 5.2: U(0,1) in FP64 cast to the working
 * precision; Sec. 2: column scaling).  Y(:,j) = X(:,j) / ||X(:,j)||_inf cast to
 * `dtype` (RR_F64, RR_F32 or RR_BF16); zero columns stay zero.  scale (device,
 * cols FP64, required) receives the inf-norms. */
rr_status rr_colscale_cast(int64_t rows, int64_t cols, const double* X, int64_t ldx,
                           int32_t dtype, void* Y, int64_t ldy, double* scale, void* stream);

/* Cast a dense FP64 m x n operator to `dtype` (RR_F32 or RR_BF16), writing the
 * column-major copy (ld m) to out_col and, if out_row != NULL, the row-major
 * copy (element (i,j) at out_row[i*n + j]) used as the K-major operand of
 * A * V.  `workspace` unused; one pass over A. */
rr_status rr_cast_operator(int64_t m, int64_t n, const double* A, int64_t lda, int32_t dtype,
                           void* out_col, void* out_row, void* stream);

/* Split BF16 copy of a dense FP64 m x n operator, for the FP32-accurate
 * correction products of the refinement phase: hi = bf16(A) and
 * lo = bf16(A - hi), both rounded to nearest even (A - hi is exact in FP64),
 * so hi + lo carries about 16 significant bits of A.  Each of hi_col / lo_col
 * (column-major, ld m) and hi_row / lo_row (row-major: element (i,j) at
 * [i*n + j], the K-major operand of A * V) may be NULL.  One pass over A.
 * RR_ERR_ARG: m, n < 0, lda < m, or A NULL. */
rr_status rr_split_operator(int64_t m, int64_t n, const double* A, int64_t lda, void* hi_col,
                            void* hi_row, void* lo_col, void* lo_row, void* stream);

/* Ritz lift (Alg. 3 "U~ = U Y"; Alg. 5 lifts both sides), FP64 result:
 *   X (n x b, ld ldx) = S1 (n x p1, ld ld1) Y(0:p1, :) + S2 (n x p2, ld ld2) Y(p1:p1+p2, :)
 * with Y FP64 (p1+p2) x b (ld ldy), all column-major; S1, S2 of type t1, t2
 * (RR_F64, RR_F32 or RR_BF16); S2 may be NULL (p2 ignored).  FP64-accurate:
 * when p1+p2 is a multiple of 8 and at most 512, b <= 256 and ws holds
 * rr_lift_workspace_size(n, b, p1+p2) bytes, the product runs on the BF16
 * tensor cores through error-free 6-bit slices of both operands (per-entry
 * error below (p1+p2) 2^-47 max_k|S(i,k)| max_k|Y(k,j)|); otherwise in FP64
 * arithmetic.  RR_ERR_ARG: negative sizes, p1 < 1, b < 1, bad type or NULL
 * pointers. */
size_t rr_lift_workspace_size(int64_t n, int64_t b, int64_t K);
rr_status rr_lift(int64_t n, int64_t b, int32_t t1, const void* S1, int64_t ld1, int64_t p1,
                  int32_t t2, const void* S2, int64_t ld2, int64_t p2, const double* Y, int64_t ldy,
                  double* X, int64_t ldx, void* ws, size_t ws_bytes, void* stream);

/* Low-precision block product (Eq. of Sec. 2, X_iter = A X; Fig. 4 "W = AV"):
 * C (M x N, FP32, ld ldc) = A_k^T * B + coef[j] * R(:,j)
 * where A_k is the K x M operand stored K-contiguous (element (kk,i) at
 * A_k[kk + i*lda]) and B is K x N column-major, both of `dtype` (RR_BF16 or
 * RR_F32), FP32 accumulation.  R (M x N FP64, ld ldr) and coef (N FP64) may
 * be NULL (no added term).  This one shape serves both W = A V (A_k = the
 * row-major copy of A) and Z = A^T W (A_k = the column-major copy). */
rr_status rr_gemm_lowp(int32_t dtype, int64_t M, int64_t N, int64_t K, const void* A_k,
                       int64_t lda, const void* B, int64_t ldb, float* C, int64_t ldc,
                       const double* R, int64_t ldr, const double* coef, void* stream);

/* Split-BF16 block product (the correction recurrence of the refinement phase;
 * Sec. 4.2's BF16 tensor-core products with each operand carried as the BF16
 * rounding of a wider value plus its BF16 residual):
 *   C (M x N, FP32) = A_hi^T B_hi + A_lo^T B_hi + A_hi^T B_lo  [+ coef[j] R(:,j)]
 * (the lo.lo term, of relative size u_bf16^2, is dropped).  Layouts as for
 * rr_gemm_lowp: A_hi, A_lo K x M K-contiguous (ld lda), B_hi, B_lo K x N
 * column-major (ld ldb), all BF16; one tcgen05 launch accumulating the three
 * K ranges in FP32.  Tensor cores only: RR_ERR_ARG unless N <= 256, lda and
 * ldb are multiples of 8 and every base pointer is 16-byte aligned. */
rr_status rr_gemm_lowp_split(int64_t M, int64_t N, int64_t K, const void* A_hi, const void* A_lo,
                             int64_t lda, const void* B_hi, const void* B_lo, int64_t ldb, float* C,
                             int64_t ldc, const double* R, int64_t ldr, const double* coef, void* stream);

/* FP64 product C = op(A) * B (+ C if accumulate), op(A) = A (trans = 0, A is/* FP64 product C = op(A) * B (+ C if accumulate), op(A) = A (trans = 0, A is
 * M x K, ld lda) or A^T (trans = 1, A is K x M).  B is K x N FP64 (ld ldb).
 * Used for the FP64-accurate residual products and by the all-FP64 mode. */
rr_status rr_gemm_f64(int32_t trans, int64_t M, int64_t N, int64_t K, const double* A,
                      int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc,
                      int32_t accumulate, void* stream);

/* FP64-accurate product C = op(A) B on the BF16 tensor cores (error-free
 * fixed-point slicing): op(A) as in rr_gemm_f64, A and B FP64, C FP64.
 * Rows of A (trans = 0) or columns of A (trans = 1) and columns of B are
 * scaled by powers of two and split into `slices` (1..10) integer BF16
 * slices of 6 bits; every slice product is exact in the FP32 tensor-core
 * accumulator (K-chunks of at most 4096), and is scaled and summed in FP64.
 * With 8 slices the result agrees with FP64 arithmetic to about 2^-54 of
 * |op(A)| |B|.  N <= 256; the row strides of op(A)'s K-major copy (m and n)
 * must be multiples of 8.  Needs rr_gemm_f64_emulated_workspace_size bytes
 * (it holds the slices of A and B). */
size_t rr_gemm_f64_emulated_workspace_size(int32_t trans, int64_t M, int64_t N, int64_t K,
                                           int32_t slices);
rr_status rr_gemm_f64_emulated(int32_t trans, int64_t M, int64_t N, int64_t K, const double* A,
                               int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc,
                               int32_t slices, void* ws, size_t ws_bytes, void* stream);

/* Algorithm 8, right-looking Hessenberg process on an n x k block (Sec. 4.2.2).
 * W (FP32 if arith == RR_F32, FP64 if RR_F64; ld ldw) is overwritten by the
 * process; the result is also written to Q (dtype qtype: RR_BF16, RR_F32 or
 * RR_F64; ld ldq; may alias W when the types match).  Skipped columns (pivot
 * magnitude below tol * the column's entry inf-norm) are set to zero instead
 * of being compacted.  piv (k int32, device): pivot row per column, -1 if
 * skipped.  tol <= 0 selects 4*k*eps(arith).  Argmax ties resolve to the
 * smallest row index.  Arithmetic is IEEE with separately rounded multiply
 * and subtract (no FMA contraction), so results are reproducible bit for bit.
 * Needs rr_hessenberg_workspace_size(n, k, arith) bytes of workspace.
 * Runs as one cooperative launch with one grid barrier per column. */
size_t rr_hessenberg_workspace_size(int64_t n, int64_t k, int32_t arith);
rr_status rr_hessenberg(int32_t arith, int64_t n, int64_t k, void* W, int64_t ldw,
                        int32_t qtype, void* Q, int64_t ldq, int32_t* piv, double tol,
                        void* ws, size_t ws_bytes, void* stream);

/* Blocked (level-3) form of the same process (the panel form of Algorithm 8
 * that Table 1's "Block" row and the closing future-work passage of Sec. 4.2
 * point to), FP32 arithmetic: columns in panels of `panel` (1..32); each
 * panel is factored by the right-looking process on its columns only (skip
 * thresholds from the column inf-norms on entry to the whole process), then
 * the trailing columns take the panel at once: weights by forward
 * substitution with the panel's unit lower triangle at its pivot rows, then
 * T -= L_panel W.  Every entry sees the same separately rounded operations in
 * the same order as in rr_hessenberg, so W, Q and piv equal its results bit
 * for bit; the trailing columns are streamed once per panel instead of once
 * per column.  rr_hessenberg takes this path by itself (panel 16) when a
 * CTA's share of rows of all k columns does not fit its shared memory.
 * W: n x k FP32 (ld ldw, overwritten); Q: qtype RR_F32, RR_BF16 or RR_F64;
 * n < 2^24.  Workspace: rr_hessenberg_workspace_size(n, k, RR_F32).
 * RR_ERR_ARG: bad sizes, panel out of range, null pointers. */
rr_status rr_hessenberg_blocked(int64_t n, int64_t k, float* W, int64_t ldw, int32_t qtype, void* Q,
                                int64_t ldq, int32_t* piv, double tol, int32_t panel, void* ws,
                                size_t ws_bytes, void* stream);

/* Krylov-Hessenberg process (Sec. 4.1, Alg. 7) on a CSR operator (FP32
 * values, as rr_csr_spmm): a basis V (n x k, column-major, ld ldv) of
 * K_k(A, v) with no inner products.  Each new vector A v_j is reduced at the
 * pivot rows of the earlier vectors (h_ij = its entry at pi_i after the
 * first i-1 subtractions, subtracted in order i = 1..j) and scaled so that
 * its largest-magnitude entry (first index on ties) is 1.  arith RR_F64 or
 * RR_F32: the arithmetic and storage of V and AV; each step a separately
 * rounded multiply and subtract.  Outputs: V; AV (n x k, ld ldv) the raw
 * products A v_j (column j before the reduction); H (k x k FP64,
 * column-major) with H(i, j) = h_ij for i <= j and H(j+1, j) the pivot value
 * (Alg. 7's upper Hessenberg matrix; column k-1 unused); piv (k int32) the
 * pivot rows.  v: n FP64 start vector (device).  Workspace:
 * rr_krylov_hessenberg_workspace_size(n, k, arith).  RR_ERR_ARG: k < 1 or
 * k > n, null pointers, bad arith. */
size_t rr_krylov_hessenberg_workspace_size(int64_t n, int32_t k, int32_t arith);
rr_status rr_krylov_hessenberg(int32_t arith, int64_t n, int32_t k, const int32_t* row_ptr,
                               const int32_t* col_idx, const float* values, const double* v, void* V,
                               void* AV, int64_t ldv, double* H, int32_t* piv, void* ws,
                               size_t ws_bytes, void* stream);

/* Largest eigenpairs of a symmetric CSR operator by the Krylov-Hessenberg
 * basis with OFRR (Alg. 7 + Alg. 3; the sparse experiment of Sec. 5.2.2):
 * restarts + 1 cycles, each building the m-dimensional basis of K_m(A, v)
 * (arith RR_F64 or RR_F32) and solving (V^T A V) y = theta (V^T V) y with
 * FP64-accurate projection products; the next cycle restarts from the single
 * Ritz vector of the largest Ritz value.  Outputs (device): theta (k FP64,
 * descending), X (n x k FP64, ld n, unit columns, sign fixed so the
 * largest-|.| entry is positive), res (k FP64: |A x - theta x|_2 / |theta|).
 * v0: n FP64 start vector.  2 <= m <= min(n, 335), 1 <= k <= m.  Workspace
 * rr_krylov_workspace_size(n, m, k, arith) (256-byte aligned).  Does not
 * synchronise. */
size_t rr_krylov_workspace_size(int64_t n, int32_t m, int32_t k, int32_t arith);
rr_status rr_krylov_eig(const rr_operator* A, int32_t m, int32_t restarts, int32_t k, int32_t arith,
                        const double* v0, double* theta, double* X, double* res, void* ws,
                        size_t ws_bytes, void* stream);

/* The basis builders the paper compares (Sec. 4, Table 1; timed in Table 3)
 * on an n x k block W (column-major, ld ldw), overwritten with the basis Q:
 *   RR_MGS_L  modified Gram-Schmidt, left-looking, no re-orthogonalisation;
 *   RR_MGS_R  modified Gram-Schmidt, right-looking;
 *   RR_CGS    classical Gram-Schmidt; RR_CGS2 with one re-orthogonalisation;
 *   RR_HESS_L Hessenberg process, left-looking (no column skip);
 *   RR_HESS_R Hessenberg process, right-looking (Algorithm 8, rr_hessenberg).
 * storage RR_F64 (FP64 arithmetic), RR_F32 or RR_F16 (FP32 arithmetic).
 * R (k x k FP64, column-major, may be NULL): the Gram-Schmidt methods'
 * triangular factor (W = Q R).  piv (k int32, the Hessenberg methods,
 * required there): pivot rows.  Workspace: rr_basis_builder_workspace_size.
 * RR_ERR_ARG: bad method, storage or sizes (k <= n, k <= 4096). */
size_t rr_basis_builder_workspace_size(int32_t method, int32_t storage, int64_t n, int64_t k);
rr_status rr_basis_builder(int32_t method, int32_t storage, int64_t n, int64_t k, void* W, int64_t ldw,
                           double* R, int32_t* piv, void* ws, size_t ws_bytes, void* stream);

/* Projection products (Alg. 3: B = U^T A U, M = U^T U; Alg. 5: U^T A V,
 * U^T U, V^T V): G (p x q FP64, ld ldg) = X^T Y (+ G if accumulate) for tall
 * X (n x p) and Y (n x q) of types xtype/ytype (RR_F64, RR_F32, RR_BF16).
 * FP64-accurate: when n >= 64 and n % 8 == 0 the products run on the tensor
 * cores (in column chunks of at most 128 of Y) from 8 column-scaled 6-bit
 * slices of each operand with
 * exact FP32 sums over 4096-long K chunks (error per entry below
 * 2^-47 n max|X(:,i)| max|Y(:,j)|); otherwise FP64 accumulation on the CUDA
 * cores.  Needs rr_gram_workspace_size(n, p, q) bytes (slices and
 * deterministic split-K partials, reduced in a fixed order). */
size_t rr_gram_workspace_size(int64_t n, int64_t p, int64_t q);
rr_status rr_gram(int64_t n, int64_t p, int64_t q, int32_t xtype, const void* X, int64_t ldx,
                  int32_t ytype, const void* Y, int64_t ldy, double* G, int64_t ldg,
                  int32_t accumulate, void* ws, size_t ws_bytes, void* stream);

/* rr_gram without a workspace argument, for callers that cannot allocate
 * device memory: code that runs where the allocator may not be called (for
 * example a thread that must not block, or a host framework that owns every
 * device allocation and hands this library only its operands), or that has
 * no buffer to spare for scratch.  The paper has no counterpart; it is a
 * deployment convenience.  Same operands and result as rr_gram.  The
 * split-K partial sums go to a 2 MiB array of FP64 compiled into the library
 * (262144 doubles per GPU, held by every GPU that loads the library until the
 * process exits), so p * q must not exceed 262144 (RR_ERR_ARG otherwise);
 * the number of row chunks shrinks to fit.  The first call on each device
 * (in each context) looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * With lazy module loading (the CUDA default) that lookup is also what
 * loads the library's module on the device and commits the 2 MiB: the
 * driver allocates it then, and the call can fail with RR_ERR_CUDA when the
 * device is out of memory.  Callers that must not touch the allocator later
 * should make one warm-up call at start-up, e.g. p = q = 1, n = 0 and
 * accumulate = 1 (it launches nothing and leaves G as it is).  The cached address is keyed by device and context, so
 * after a device reset the next call looks it up again.  All calls share
 * the one array: calls whose executions overlap on the GPU (different
 * streams, or concurrent graph branches) race and give wrong results.
 * Invalid dtypes return RR_ERR_ARG as in rr_gram, even for empty sizes.
 * Allocates nothing itself. */
rr_status rr_gram_noalloc(int64_t n, int64_t p, int64_t q, int32_t xtype, const void* X,
                          int64_t ldx, int32_t ytype, const void* Y, int64_t ldy, double* G,
                          int64_t ldg, int32_t accumulate, void* stream);

/* Small projected problems, FP64 (Alg. 3: B Y = M Y Lambda; Alg. 5).
 * rr_pencil_eig: H, G (b x b, ld b) symmetric, G positive semidefinite.
 *   theta (b) ascending; Y (b x b) with Y^T G Y = I on the kept part.
 *   Whitening by Cholesky with column dropping (a pivot with L_jj^2 <=
 *   64 u64 max_i G_ii drops column j); dropped directions get theta = NaN and
 *   a zero column of Y, sorted last.  dropped (host int*, may be NULL).
 * rr_pencil_svd: B (b1 x b2, ld b1), Gu (b1 x b1), Gv (b2 x b2).
 *   s (min(b1,b2)) descending, Y (b1 x r), Z (b2 x r) with sqrt(2)-scaled
 *   normalisation already applied: U~ = U Y, V~ = V Z are orthonormal
 *   (theorem of Sec. 3.2).  Solved as the whitened SVD of
 *   Lu^-1 B Lv^-T by one-sided Jacobi (equivalent to the positive half of
 *   the 2x2 block pencil).
 * Sizes up to 335 x 335 (RR_ERR_ARG above).
 * Both need rr_pencil_workspace_size(b1, b2) bytes of workspace and
 * synchronise nothing (dropped counts are read only when dropped != NULL,
 * which synchronises). */
size_t rr_pencil_workspace_size(int64_t b1, int64_t b2);
rr_status rr_pencil_eig(int64_t b, const double* H, const double* G, double* theta, double* Y,
                        void* ws, size_t ws_bytes, int32_t* dropped, void* stream);
rr_status rr_pencil_svd(int64_t b1, int64_t b2, const double* B, const double* Gu,
                        const double* Gv, double* s, double* Y, double* Z, void* ws,
                        size_t ws_bytes, int32_t* dropped, void* stream);

/* Matrix-free product with a kernel operator (RR_KERNEL):
 *   Y (rows x b) = op(A) X (+ coef_j R(:, j)),  op(A) = A (trans = 0, rows = m)
 *   or A^T (trans = 1, rows = n); X (cols x b, xtype RR_BF16 / RR_F32 /
 *   RR_F64, ld ldx), Y of otype RR_F32 or RR_F64 (ld ldy), R FP64 and coef
 *   (b FP64) may be NULL.  Every entry of A is evaluated where it is used
 *   (one exponential, d differences) and never stored; FP32 evaluation and
 *   accumulation when xtype and otype are 32-bit or narrower, FP64 when
 *   either is RR_F64.  RR_ERR_ARG: not a valid RR_KERNEL operator, bad sizes
 *   or types. */
rr_status rr_kernel_apply(int32_t trans, const rr_operator* A, int64_t b, int32_t xtype, const void* X,
                          int64_t ldx, int32_t otype, void* Y, int64_t ldy, const double* R, int64_t ldr,
                          const double* coef, void* stream);

/* Sparse block product (a CSR operator applied to a block; Sec. 5.1 CSR):
 * Y (n x b, FP32 out, ld ldy) = A X with A CSR FP32, X (n x b, dtype xtype
 * RR_BF16/RR_F32/RR_F64, ld ldx).  FP32 accumulation (FP64 when xtype is F64,
 * then Y must be FP64: pass ytype RR_F64). */
rr_status rr_csr_spmm(int64_t n, int64_t b, const int32_t* row_ptr, const int32_t* col_idx,
                      const float* values, int32_t xtype, const void* X, int64_t ldx,
                      int32_t ytype, void* Y, int64_t ldy, void* stream);

/* One step of the scaled Chebyshev three-term recurrence (the chebfsi filter
 * the paper cites in Sec. 2), fused with the CSR product:
 *   Y_next(:,j) = alpha (A - c I) Y_cur(:,j) - beta * bc_j * Y_prev(:,j)
 *                 + gamma_j * R(:,j)
 * with A CSR FP32, Y_cur/Y_prev of dtype ytype (RR_BF16/RR_F32/RR_F64,
 * ld ld), FP32 accumulation (FP64 when ytype is RR_F64).  Y_next is written
 * as out_type (ytype or RR_F32; ld ld_next).  Y_prev may be NULL (first step).
 * bc (beta_col) may be NULL (bc_j = 1); R (FP64, ld ldr) and gamma may be
 * NULL (no added term).  b <= 3072 (RR_ERR_ARG above). */
rr_status rr_chebyshev_step(int64_t n, int64_t b, const int32_t* row_ptr,
                            const int32_t* col_idx, const float* values, int32_t ytype,
                            const void* Y_cur, const void* Y_prev, int64_t ld, double alpha,
                            double c, double beta, const double* beta_col, const double* R,
                            int64_t ldr, const double* gamma, int32_t out_type, void* Y_next,
                            int64_t ld_next, void* stream);

/* The same step on row-major blocks (element (i, j) at Y[i * ldr + j]), the
 * layout of the eigensolver's plain Chebyshev filter: one 16-byte gather per
 * neighbour row and 16 / sizeof(ytype) columns.  Y_next = alpha (A - c I)
 * Y_cur - beta Y_prev (Y_prev may be NULL).  (ytype, out_type) is one of
 * (RR_BF16, RR_BF16), (RR_BF16, RR_F32), (RR_F32, RR_F32), (RR_F64, RR_F64).
 * Columns are processed in vectors of 16 / sizeof(ytype): the row strides
 * ldr, ldr_next must be at least b rounded up to that width, multiples of 16
 * bytes, and the pointers 16-byte aligned (RR_ERR_ARG otherwise); pad
 * columns up to the rounded width are read and written like the others.
 * At most 256 vectors per row (b <= 2048 BF16, 1024 FP32, 512 FP64). */
rr_status rr_chebyshev_step_rows(int64_t n, int64_t b, const int32_t* row_ptr,
                                 const int32_t* col_idx, const float* values, int32_t ytype,
                                 const void* Y_cur, const void* Y_prev, int64_t ldr, double alpha,
                                 double c, double beta, int32_t out_type, void* Y_next,
                                 int64_t ldr_next, void* stream);

/* FP8-E4M3 operands and their block product (the FP8 storage option of the
 * precision map, Sec. 4.2 / Fig. 4, with FP32 accumulation).
 * rr_quantize_e4m3: X (rows x cols FP64, column-major, ld ldx) -> Q (E4M3
 *   bytes).  by_rows = 0: one scale per column, Q column-major (ldq >= rows);
 *   by_rows = 1: one scale per row, Q row-major, Q[i * ldq + j] (ldq >= cols).
 *   Each scale is the power of two 2^e, the largest with max|x| 2^e <= 448
 *   (e clamped to [-126, 126]; an all-zero line gets 2^0), applied exactly;
 *   Q = e4m3_rn(fp32_rn(x 2^e)), round to nearest even, saturating at 448.
 *   inv_scale (cols or rows FP32) receives 2^-e.  scratch: 8 max(rows, cols)
 *   bytes of device memory.
 * rr_gemm_e4m3: C (M x N FP32, column-major) = diag(a_scale) A_k^T B
 *   diag(b_scale), A_k (K x M) and B (K x N) E4M3 with K contiguous (ld in
 *   elements: multiples of 16, bases 16-byte aligned), N <= 256; tcgen05
 *   kind::f8f6f4 on the tensor cores, FP32 accumulation.  For W = A V: A_k is
 *   A quantised by rows (row-major), B the block V quantised by columns.
 * Errors: RR_ERR_ARG for bad sizes, strides, alignment or null pointers. */
rr_status rr_quantize_e4m3(int64_t rows, int64_t cols, const double* X, int64_t ldx, int32_t by_rows,
                           void* Q, int64_t ldq, float* inv_scale, void* scratch, void* stream);
rr_status rr_gemm_e4m3(int64_t M, int64_t N, int64_t K, const void* A_k, int64_t lda,
                       const float* a_scale, const void* B, int64_t ldb, const float* b_scale, float* C,
                       int64_t ldc, void* stream);

/* Learned warm start (the start block V of Alg. 1, which the paper draws at
 * random, proposed instead by a small convolutional network of the operator's
 * potential and trained on converged Ritz vectors).  All FP32, NCHW layout on
 * the device: x[n, c, i, j] at ((n*C + c)*H + i)*W + j, so one image with C
 * channels is an (H*W) x C column-major block.  Pointers are device pointers
 * owned by the caller; every call is asynchronous on `stream`.
 *
 * rr_conv3x3_forward: y (N, O, H, W) = correlation of x (N, C, H, W) with
 *   w (O, C, 3, 3), zero padding 1, plus bias b (O), plus the image `add`
 *   (O, H, W per sample, samples add_nstride floats apart; NULL: nothing
 *   added); relu != 0 clamps the sum at 0.
 * rr_conv3x3_backward: given g = dL/dy, ADDS dL/dw to dw (O, C, 3, 3) and
 *   dL/db to db (O) (zero them first), and writes dL/dx to dx (N, C, H, W)
 *   unless dx is NULL.
 * rr_relu_mask: g[e] = 0 wherever act[e] <= 0 (the ReLU derivative taken at
 *   the layer's output).
 * rr_procrustes_grad: net output `out` (n x k, column-major, ld n) scaled by
 *   `scale` gives V; with R = U W^T (U, W k x k FP64 column-major, from the
 *   SVD of V^T V*), writes grad = scale * 2 (V R - V*) R^T (dL/d out) and
 *   ADDS |V R - V*|_F^2 to *loss (FP64).  k <= 64.
 * rr_adam: one Adam update of `count` parameters at step t >= 1 (moments m,
 *   v updated in place, bias corrections 1 - b1^t, 1 - b2^t).
 * rr_net_block: V[:, 0:k] (FP64, ld ldv >= n) = scale * out (n x k FP32,
 *   ld n): the network output as the leading columns of a start block.
 * Errors: RR_ERR_ARG for negative sizes, null pointers or k out of range;
 * empty sizes return RR_OK without a launch. */
rr_status rr_conv3x3_forward(int32_t N, int32_t C, int32_t H, int32_t W, int32_t O, const float* x,
                             const float* w, const float* b, const float* add, int64_t add_nstride,
                             int32_t relu, float* y, void* stream);
rr_status rr_conv3x3_backward(int32_t N, int32_t C, int32_t H, int32_t W, int32_t O, const float* x,
                              const float* w, const float* g, float* dx, float* dw, float* db,
                              void* stream);
rr_status rr_relu_mask(int64_t count, float* g, const float* act, void* stream);
rr_status rr_procrustes_grad(int64_t n, int32_t k, const float* out, const double* Vstar,
                             const double* U, const double* Wm, float scale, float* grad,
                             double* loss, void* stream);
rr_status rr_adam(int64_t count, float* p, const float* g, float* m, float* v, float lr, float b1,
                  float b2, float eps, int32_t t, void* stream);
rr_status rr_net_block(int64_t n, int32_t k, const float* out, float scale, double* V, int64_t ldv,
                       void* stream);

#ifdef __cplusplus
}
#endif
#endif /* RR_H_ */
