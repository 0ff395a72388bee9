/*
 * chfsi.h -- C ABI of the GB300 (sm_103a) Chebyshev-filtered subspace iteration library.
 *
 * The library implements the filter and closure of ChFSI as given in Algorithm 1
 * (Sec. 3.4) of "GPU acceleration of the Tucker-tensor based Kohn-Sham DFT"
 * (arXiv 2110.15853): the degree-m scaled Chebyshev filter (step 1), the
 * orthonormalisation (step 2), the subspace projection (step 3), the dense
 * eigensolve (step 4) and the rotation (step 5), plus the spectral bounds the
 * algorithm takes as input and the reverse-mode derivative of the filter.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Matrix and vector pointers are DEVICE pointers owned by the caller; the
 *   library never frees or retains them.  Dense blocks (X, Y, Psi, dY, dX) are
 *   row-major N x n_cols with an explicit leading dimension ld >= n_cols
 *   (element (i, j) at p[i * ld + j]); each block must start on a 16-byte boundary.
 *   Only columns 0 .. n_cols-1 of a row are read or written, so a block may be a
 *   column view of a wider array.  An output block must not overlap any input.
 * - Scalars a, b, a0 are the paper's eps_ub^w (upper bound of the wanted
 *   spectrum), eps_ub^uw (upper bound of the unwanted spectrum) and eps_0 (lower
 *   bound of the wanted spectrum).  a0 < a < b is required (if a0 lies in [a, b]
 *   the scaled Chebyshev value T_m(tau) can vanish and the sigma recurrence
 *   divides by zero).
 * - Work is queued on `stream` (a cudaStream_t; NULL = the legacy default
 *   stream) and returns before it finishes, unless stated otherwise.  Scratch
 *   comes from the caller's workspace `ws` of `ws_bytes` bytes (256-byte aligned),
 *   sized by the matching *_workspace_size call; nothing is allocated on these
 *   paths.  The first 256 bytes of every workspace hold a device status word that
 *   kernels set when they meet a non-finite value, an out-of-range column index or
 *   a non-positive Cholesky pivot; chfsi_read_status() synchronises the stream and
 *   returns it.
 * - Every call returns an int status (CHFSI_OK = 0 or a CHFSI_ERR_* code below);
 *   argument errors are detected on the host before anything is queued.
 * - Calls that share a workspace must not overlap on the GPU.
 */
#ifndef CHFSI_H
#define CHFSI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status codes */
#define CHFSI_OK 0
#define CHFSI_ERR_ARG 1         /* bad pointer, size, leading dimension or alignment      */
#define CHFSI_ERR_BOUNDS 2      /* not a0 < a < b, or a bound is not finite              */
#define CHFSI_ERR_PATTERN 3     /* bad CSR/BSR pattern (device found a column out of range) */
#define CHFSI_ERR_CHOL 4        /* Gram matrix not positive definite (Cholesky pivot <= 0) */
#define CHFSI_ERR_NONFINITE 5   /* a kernel produced or read a NaN / Inf                 */
#define CHFSI_ERR_CUDA 6        /* a CUDA runtime call failed                            */
#define CHFSI_ERR_TIMEOUT 7     /* a bounded device wait gave up                         */
#define CHFSI_ERR_NOMEM 8       /* workspace smaller than the *_workspace_size answer    */
#define CHFSI_ERR_UNSUPPORTED 9 /* combination not implemented (e.g. a precision on BSR) */

/* Text for a status code (static storage, never NULL). */
const char* chfsi_status_string(int status);

/* Library version as major*10000 + minor*100 + patch. */
int chfsi_version(void);

/* ------------------------------------------------------------------ operator H */
#define CHFSI_CSR 0
#define CHFSI_BSR 1
#define CHFSI_HYBRID 2   /* both layouts of one operator, rows in the blocked order (see below) */
#define CHFSI_SPLIT 3    /* dense diagonal blocks + CSR of the rest (Sec. 4.1-4.2, see below) */

/*
 * Sparse symmetric H (the projected Kohn-Sham Hamiltonian H^L of Sec. 3.3,
 * Eq. "localized standard ks problem") in CSR: row_ptr[n_rows + 1] (int64,
 * row_ptr[0] = 0, non-decreasing, row_ptr[n_rows] = nnz), col[nnz] (int32 in
 * [0, n_rows)), val[nnz] (double).  The filter never assumes symmetry; the
 * backward pass uses H in place of H^T and so requires it (pattern and values).
 */
typedef struct {
    int64_t n_rows;
    int64_t nnz;
    const int64_t* row_ptr;
    const int32_t* col;
    const double* val;
} chfsi_csr;

/*
 * Blocked CSR with dense bdim x bdim blocks (bdim = 64: 4 x 4 x 4 sub-cubes of
 * the tensor-index grid).  brow_ptr[n_block_rows + 1] (int32), bcol[n_blocks]
 * (int32 block column), val[n_blocks * bdim * bdim] (double, each block row-major).
 * Rows of X and Y are in the same blocked order as H's rows.
 */
typedef struct {
    int64_t n_block_rows;
    int64_t n_blocks;
    int32_t bdim;
    const int32_t* brow_ptr;
    const int32_t* bcol;
    const double* val;
} chfsi_bsr;

/*
 * The paper's split storage of a row-partitioned H (Sec. 4.1-4.2: the dense diagonal
 * block H^{L(D)}_k and the sparse off-diagonal part H^{L(OD)}_k of each row block):
 * rows in consecutive blocks of `block` rows; diagonal block k (rows and columns
 * k*block .. (k+1)*block - 1) is stored dense, every entry outside the diagonal
 * blocks in the CSR `off` over all n_rows rows with global column indices (an entry
 * inside a diagonal block must not appear in `off`).  block is a multiple of 128 and
 * at most 8192; diag holds ceil(n_rows / block) blocks of block x block doubles, each
 * row-major, stacked (rows and columns past n_rows zero).  The filter runs the dense
 * blocks on the BF16 tensor cores by Ozaki slices (see chfsi_ozaki_gemm) and the
 * sparse part with the CSR kernel, FP64 schedule only.
 */
typedef struct {
    int64_t n_rows;
    int32_t block;
    const double* diag;
    chfsi_csr off;
} chfsi_split;

/*
 * kind = CHFSI_CSR uses `csr`, CHFSI_BSR uses `bsr`, CHFSI_SPLIT uses `split`.
 * CHFSI_HYBRID carries the same operator in both layouts with the CSR rows in the
 * blocked order: FP64 and FP32 steps (and the backward pass, the Lanczos bounds and
 * the projection) use the CSR kernels, BF16-operand steps use the BSR blocks on the
 * tensor cores.  CHFSI_SPLIT is accepted by the filter (FP64 schedule) only.
 */
typedef struct {
    int32_t kind;      /* CHFSI_CSR, CHFSI_BSR, CHFSI_HYBRID or CHFSI_SPLIT */
    chfsi_csr csr;
    chfsi_bsr bsr;
    chfsi_split split;
} chfsi_matrix;

/* ------------------------------------------------------------------ precision schedule */
#define CHFSI_F64 0           /* FP64 storage and FP64 arithmetic                      */
#define CHFSI_F32 1           /* FP32 storage, FP32 FMA, FP64-computed coefficients    */
#define CHFSI_BF16_F32ACC 2   /* BF16 copy of Y_k as the product operand, FP32 accumulate,
                                 FP32 storage of the iterates                           */
#define CHFSI_F32X2 3         /* two-float: values as hi + lo FP32 pairs (about 48 bits),
                                 FP32-pipe arithmetic with error-free transformations;
                                 CSR layout (CHFSI_CSR or CHFSI_HYBRID) only            */
#define CHFSI_F64_OZAKI 4     /* FP64-accurate products on the BF16 tensor cores: FP64
                                 values split into seven 8-bit slices, exact integer
                                 accumulation (see chfsi_ozaki_gemm).  In the closure
                                 (chfsi_rayleigh_ritz_ex) its dense products; in a filter
                                 schedule the FP64 steps of a BSR or hybrid operator, its
                                 64 x 64 blocks as Ozaki products (rows of at most 128
                                 blocks), FP64 iterates and recurrence                   */
#define CHFSI_F40_OZAKI 5     /* filter schedules only, wherever CHFSI_F64_OZAKI steps may
                                 run: the same step with the first five of the seven
                                 slices of each operand (40-bit operands, truncated) and
                                 the 15 slice pairs of weight 2^-48 and above, each term
                                 within about 2^-40 of its row scales (2^16 finer than
                                 FP32) for about half the tensor-core work; FP64 iterates
                                 and recurrence.  Not in the paper: a precision knob of
                                 this library, for the early steps of a schedule whose
                                 last steps are CHFSI_F64_OZAKI                          */

/*
 * Per-step precision of the filter: step_prec[k-1] is the precision of the step
 * that produces Y_k (k = 1..m).  Low-precision steps (CHFSI_F32, CHFSI_BF16_F32ACC,
 * CHFSI_F32X2, one kind) must form a prefix; the steps after it are all CHFSI_F64, or
 * all Ozaki steps (CHFSI_F64_OZAKI and CHFSI_F40_OZAKI in any order; both keep FP64
 * iterates).  The two iterates carried across the switch are widened exactly.  A NULL
 * schedule (or step_prec == NULL) means every step in FP64.
 */
typedef struct {
    int32_t m;
    const int32_t* step_prec;
} chfsi_schedule;

/* ------------------------------------------------------------------ filter (Algorithm 1, step 1) */

/* Bytes of workspace chfsi_filter needs for this operator, n_cols, m and schedule. */
int chfsi_filter_workspace_size(const chfsi_matrix* H, int64_t n_cols, int32_t m,
                                const chfsi_schedule* sched, size_t* bytes);

/*
 * Y = Y_m, the scaled Chebyshev filter of Algorithm 1 step 1 (Sec. 3.4):
 *   e = (b - a)/2, c = (b + a)/2, sigma_1 = e/(a0 - c), gamma = 2/sigma_1,
 *   Y_1 = (sigma_1/e)(H X - c X),
 *   Y_{k+1} = (2 sigma_{k+1}/e)(H Y_k - c Y_k) - sigma_k sigma_{k+1} Y_{k-1},
 *   sigma_{k+1} = 1/(gamma - sigma_k),
 * returning the newest iterate Y_m (the paper's X~ after the loop).
 * X: N x n_cols (ldx), read only.  Y: N x n_cols (ldy), written.  m >= 1.
 * sched: NULL for all-FP64, else a schedule with sched->m == m.
 * A CSR operator over more than 512 columns is filtered in column slabs of 512
 * (all m steps per slab; the columns are independent), so the workspace holds one
 * slab's iterates.
 * Errors: CHFSI_ERR_ARG, CHFSI_ERR_BOUNDS, CHFSI_ERR_NOMEM, CHFSI_ERR_UNSUPPORTED
 * (e.g. CHFSI_F64_OZAKI steps without BSR blocks or with a block row of more than
 * 128 blocks; checking the latter copies the block-row pointers to the host and
 * synchronises `stream` once), CHFSI_ERR_CUDA (launch failure).  Device-side findings
 * (non-finite output, column out of range) go to the workspace status word.
 */
int chfsi_filter(const chfsi_matrix* H, const double* X, int64_t ldx, double* Y, int64_t ldy,
                 int64_t n_cols, int32_t m, double a, double b, double a0,
                 const chfsi_schedule* sched, void* ws, size_t ws_bytes, void* stream);

/*
 * chfsi_filter without a caller workspace, for callers that cannot allocate
 * device memory (a host whose own allocator owns the whole device, and which
 * must not call cudaMalloc/cudaFree or pass scratch pointers).  The paper has no
 * counterpart; this is a deployment convenience.
 *
 * Same arguments and result as chfsi_filter minus ws/ws_bytes.  The scratch is a
 * 16 MiB array in the library's device memory (held by every GPU that loads the
 * library until the process exits).  Problems whose chfsi_filter_workspace_size
 * exceeds 16 MiB are rejected with CHFSI_ERR_NOMEM (FP64 schedule on a CSR
 * operator: about 2 * N * round_up(min(n_cols, 512), 8) * 8 bytes, e.g. N = 8000
 * with 64 columns fits).
 * The first call on each device looks up the array's device address (with that
 * device current) and keeps it until the process exits; make that first call
 * before any stream capture.  A device reset between calls is not supported (the
 * kept address would be stale).  Nothing is allocated.  All calls share the one
 * array: calls that overlap on the GPU (other streams, other threads) race and
 * must be serialised by the caller.  The array holds the filter's device status
 * word, cleared at the start of each call; read it with
 * chfsi_filter_noalloc_read_status after the call.
 */
int chfsi_filter_noalloc(const chfsi_matrix* H, const double* X, int64_t ldx, double* Y,
                         int64_t ldy, int64_t n_cols, int32_t m, double a, double b, double a0,
                         const chfsi_schedule* sched, void* stream);

/*
 * Companion of chfsi_filter_noalloc on the current device: synchronises `stream`
 * and returns the status word that the last chfsi_filter_noalloc call's kernels
 * left in the static array, mapped like chfsi_read_status (CHFSI_ERR_PATTERN for a
 * column index out of range, CHFSI_ERR_NONFINITE for a NaN or Inf read or
 * produced, CHFSI_OK if clean), and clears it.  The paper has no counterpart.
 */
int chfsi_filter_noalloc_read_status(void* stream);

/* ------------------------------------------------------------------ adjoint of the filter */

int chfsi_filter_backward_workspace_size(const chfsi_matrix* H, int64_t n_cols, int32_t m,
                                         int32_t ckpt_stride, size_t* bytes);

/*
 * Reverse-mode derivative of chfsi_filter (all-FP64 schedule) for a loss L with
 * dL/dY_m = dY.  Writing the filter as Y_1 = alpha_1 (H - c) Y_0 and
 * Y_k = alpha_k (H - c) Y_{k-1} - beta_k Y_{k-2} (alpha_1 = sigma_1/e,
 * alpha_k = 2 sigma_k/e, beta_k = sigma_{k-1} sigma_k, Y_0 = X):
 *   Ybar_m = dY,  Ybar_{k-1} = alpha_k (H - c) Ybar_k - beta_{k+1} Ybar_{k+1},
 *   dX = Ybar_0,
 *   dH_val[p] = sum_{k=1..m} alpha_k <Ybar_k[row p, :], Y_{k-1}[col p, :]>
 * for every stored entry p of H (the unconstrained per-entry gradient).  Uses H
 * for H^T (H must be symmetric; the paper's Eq. "transpose_equal" is the same
 * fact).  Forward iterates are kept only every ckpt_stride steps (as pairs
 * Y_{s-1}, Y_s; 0 selects ceil(sqrt(m))) and the rest are recomputed per segment.
 * dH_val may be NULL (then only dX).  Needs the CSR layout (CHFSI_CSR or CHFSI_HYBRID).
 * More than 512 columns are swept in column slabs of 512 (dX's columns are
 * independent; each slab adds its part of dH_val), so the workspace holds one slab.
 */
int chfsi_filter_backward(const chfsi_matrix* H, const double* X, int64_t ldx,
                          const double* dY, int64_t lddy, double* dX, int64_t lddx,
                          double* dH_val, int64_t n_cols, int32_t m, double a, double b,
                          double a0, int32_t ckpt_stride, void* ws, size_t ws_bytes,
                          void* stream);

int chfsi_filter_backward_ex_workspace_size(const chfsi_matrix* H, int64_t n_cols, int32_t m,
                                            int32_t ckpt_stride, int32_t precision, size_t* bytes);

/*
 * chfsi_filter_backward with a choice of arithmetic for the whole reverse sweep
 * (forward replay, reverse recurrence and the dH products): precision =
 * CHFSI_F64 (the same as chfsi_filter_backward) or CHFSI_F32X2 (two-float hi/lo
 * FP32 pairs on the FP32 pipe, about 48 significant bits; dH accumulates in FP64).
 * Same arguments, layout requirements and errors as chfsi_filter_backward.
 */
int chfsi_filter_backward_ex(const chfsi_matrix* H, const double* X, int64_t ldx,
                             const double* dY, int64_t lddy, double* dX, int64_t lddx,
                             double* dH_val, int64_t n_cols, int32_t m, double a, double b,
                             double a0, int32_t ckpt_stride, int32_t precision, void* ws,
                             size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------ closure (Algorithm 1, steps 2-5) */

int chfsi_rayleigh_ritz_workspace_size(const chfsi_matrix* H, int64_t n_cols,
                                       int32_t cholqr_passes, size_t* bytes);

/*
 * Steps 2-5 of Algorithm 1 in FP64 on the GPU:
 *   2. X_F = Orth(Y) by Cholesky-QR: S = Y^T Y, S = R^T R, X_F = Y R^-1
 *      (cholqr_passes = 2 repeats it on X_F: CholQR2);
 *   3. H_F = X_F^T (H X_F);
 *   4. H_F Q = Q Lambda (ascending eigenvalues), by the library's dense eigensolver
 *      (the algorithm of chfsi_eigh, which synchronises `stream` once per merge of
 *      its divide and conquer);
 *   5. Psi = X_F Q.
 * With cholqr_passes = 2 the second pass's X_F = X1 R2^-1 is not formed: steps 3 and 5
 * use H_F = R2^-T (X1^T H X1) R2^-1 and Psi = X1 (R2^-1 Q), the same quantities in exact
 * arithmetic (n x n products in place of one N x n product).
 * Y: N x n_cols (ldy), read only.  Psi: N x n_cols (ldpsi), written.
 * ritz: device array of n_cols doubles, written ascending.  n_cols <= N.
 * Synchronises `stream` before returning (it reads the status word); returns
 * CHFSI_ERR_CHOL if a Cholesky pivot was not positive, CHFSI_ERR_NONFINITE if a
 * non-finite value was met, CHFSI_ERR_CUDA if a launch failed.
 */
int chfsi_rayleigh_ritz(const chfsi_matrix* H, const double* Y, int64_t ldy, int64_t n_cols,
                        double* Psi, int64_t ldpsi, double* ritz, int32_t cholqr_passes,
                        void* ws, size_t ws_bytes, void* stream);

int chfsi_rayleigh_ritz_ex_workspace_size(const chfsi_matrix* H, int64_t n_cols,
                                          int32_t cholqr_passes, int32_t precision, size_t* bytes);

/*
 * chfsi_rayleigh_ritz with a choice of arithmetic for the three large products
 * (Gram / projection A^T B over N, X_F = Y R^-1, Psi = X_F Q) and H X_F:
 * precision = CHFSI_F64 (the same as chfsi_rayleigh_ritz), CHFSI_F32X2
 * (two-float products on the FP32 pipe, about 48 significant bits; needs the CSR
 * layout) or CHFSI_F64_OZAKI (the dense products as chfsi_ozaki_gemm on the BF16
 * tensor cores, about 48 significant bits of the row scales; H X_F in two-float
 * arithmetic on a CSR operator, in FP64 on a BSR one).  The Cholesky
 * factorisation, the triangular inverse and the eigensolve stay FP64 in all
 * three.  Same arguments, errors and synchronisation as chfsi_rayleigh_ritz.
 */
int chfsi_rayleigh_ritz_ex(const chfsi_matrix* H, const double* Y, int64_t ldy, int64_t n_cols,
                           double* Psi, int64_t ldpsi, double* ritz, int32_t cholqr_passes,
                           int32_t precision, void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------ FP64-accurate dense products */

#define CHFSI_OP_TN 0              /* C = A^T B: A is K x M (lda), B is K x Nc (ldb)          */
#define CHFSI_OP_NN 1              /* C = A B:   A is M x K (lda), B is K x Nc (ldb)          */
#define CHFSI_GEMM_SYMMETRIC 1     /* TN, M == Nc, C known to be symmetric (Y^T Y, X^T H X):
                                      the 128 x 128 tiles on and above the diagonal are
                                      computed, the others mirrored                          */
#define CHFSI_GEMM_B_UPPER 2       /* NN, B upper triangular (B[k][j] = 0 for k > j)          */

int chfsi_ozaki_gemm_workspace_size(int32_t op, int64_t M, int64_t Nc, int64_t K, int32_t flags,
                                    size_t* bytes);

/*
 * The closure's dense FP64 products (Algorithm 1 steps 2, 3 and 5: S = Y^T Y,
 * X_F = Y R^-1, H_F = X_F^T (H X_F), Psi = X_F Q) on the BF16 tensor cores, by
 * Ozaki-scheme splitting: each row of the K-major operands (A^T or A, and B^T) is
 * scaled by a power of two and rounded to a 56-bit fixed-point number held as seven
 * balanced 8-bit digits, each digit slice exact in BF16; the 28 slice products
 * with digit weights down to 2^-64 run as tcgen05 MMAs, one FP32 accumulator per digit
 * level, each drained before its sums pass 2^24 units, so that the accumulation is
 * exact (integer multiples, whatever the tensor cores' rounding) and ends in two
 * 64-bit integers per element.  The only errors are the 56-bit rounding of the inputs
 * and the dropped slice pairs: |C_ij - (A_hat B_hat^T)_ij| is below K 2^-50 times the
 * product of the two rows' largest magnitudes (errors of random sign make it about
 * sqrt(K) times that in practice).  Row-major blocks with leading dimensions; C
 * must not overlap A or B.  The workspace (chfsi_ozaki_gemm_workspace_size) holds
 * the status word, the slices (14 bytes per operand element) and the split-K
 * partial tiles.  A non-finite input sets CHFSI_ERR_NONFINITE in the status word.
 * Errors: CHFSI_ERR_ARG, CHFSI_ERR_NOMEM, CHFSI_ERR_UNSUPPORTED (K above 2^21 in
 * the TN form, above 8192 in the NN form), CHFSI_ERR_CUDA.  No counterpart in the paper, which runs these products with
 * FP64 cuBLAS (Sec. 4.3).
 */
int chfsi_ozaki_gemm(int32_t op, const double* A, int64_t lda, const double* B, int64_t ldb, double* C,
                     int64_t ldc, int64_t M, int64_t Nc, int64_t K, int32_t flags, void* ws,
                     size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------ dense symmetric eigensolver */

int chfsi_eigh_workspace_size(int64_t n, size_t* bytes);

/*
 * A = Q diag(w) Q^T for a symmetric n x n A (row-major, lda, both triangles stored),
 * the dense eigenproblem of Algorithm 1 step 4 (Sec. 3.4), in FP64 on the GPU:
 * Householder tridiagonalisation, divide and conquer on the tridiagonal matrix
 * (deflation, secular equation by bracketed rational-model steps, eigenvector weights recomputed from the
 * roots), back-transformation in panels of 64 reflectors.  w: n doubles, ascending.
 * Q: n x n (ldq), Q[k * ldq + i] = component k of the eigenvector of w[i].  A is
 * overwritten.  Q must not overlap A.  The call synchronises `stream` once per merge
 * of the divide and conquer.  Workspace (chfsi_eigh_workspace_size): the status word
 * and about 3 n^2 + 200 n doubles.  Errors: CHFSI_ERR_ARG, CHFSI_ERR_NOMEM,
 * CHFSI_ERR_UNSUPPORTED (n above 65535), CHFSI_ERR_CUDA.
 */
int chfsi_eigh(double* A, int64_t lda, int64_t n, double* w, double* Q, int64_t ldq, void* ws,
               size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------ spectral bounds */

int chfsi_lanczos_workspace_size(const chfsi_matrix* H, int32_t steps, size_t* bytes);

/*
 * The bounds (a, b, a0) = (eps_ub^w, eps_ub^uw, eps_0) that Algorithm 1 takes as
 * input (Sec. 3.4 does not say how they are found).  k = min(steps, N) steps of
 * Lanczos with full re-orthogonalisation from the start vector v0 (N doubles on
 * the device, need not be normalised; the caller draws it), then
 *   a0 = smallest eigenvalue of the tridiagonal T_k,
 *   b  = largest eigenvalue of T_k + |beta_k| (residual norm),
 *   a  = a0 + (b - a0) (n_wanted / N)^(2/3).
 * Breakdown (beta_j <= 1e-12 times the largest |alpha_i| + beta_{i-1} so far)
 * stops early with a zero residual.  a, b, a0 are HOST pointers; the call
 * synchronises `stream`.  1 <= n_wanted < N.  Needs the CSR layout (CHFSI_CSR or CHFSI_HYBRID).
 */
int chfsi_lanczos_bounds(const chfsi_matrix* H, int32_t steps, const double* v0,
                         int64_t n_wanted, double* a, double* b, double* a0, void* ws,
                         size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------ utilities */

/* Synchronise `stream` and return the workspace status word as a CHFSI_* code
 * (CHFSI_OK if clean); clears the word.  */
int chfsi_read_status(void* ws, void* stream);

/* Clear the workspace status word (queued on `stream`). */
int chfsi_clear_status(void* ws, void* stream);

/*
 * Measured FMA throughput (FLOP/s, two per fused multiply-add) of the current
 * device's FP64 (precision = CHFSI_F64: the DFMA pipe) or FP32 (CHFSI_F32: the
 * FFMA pipe), from a register-resident loop of independent multiply-adds over
 * 8 blocks of 256 threads per SM, timed with CUDA events on `stream` after one
 * untimed launch (the fastest of three timed launches of about 70 ms of FP64 work
 * each).  Synchronises `stream`.  The denominator of the roofline
 * fraction of the arithmetic-bound filter steps.  Diagnostics only: the paper
 * has no counterpart.  Errors: CHFSI_ERR_ARG (bad precision or NULL output),
 * CHFSI_ERR_CUDA.
 */
int chfsi_measure_pipe_peak(int32_t precision, double* flops_per_second, void* stream);

/* Number of kernels this library has launched in this process (all devices, all
 * threads).
 * Diagnostics only: the paper has no counterpart. */
unsigned long long chfsi_kernel_launches(void);

/*
 * Limit, in nanoseconds, of the mbarrier waits in which one role of a tensor-core
 * kernel (chfsi_filter's BF16 steps on a BSR or hybrid operator, chfsi_ozaki_gemm and
 * the products that use it) waits on another: a copy producer on a free stage, the
 * MMA issuer on a loaded stage or a drained accumulator, the epilogue on a finished
 * accumulator.  A wait that runs out makes its CTA stop, wait for its own copies and
 * MMAs in flight (those waits keep a fixed 1 s bound), free its tensor memory and exit;
 * the call's status word then holds CHFSI_ERR_TIMEOUT and its outputs are undefined.
 * 0 restores the default of 1 s.  Process-wide, read at each launch; meant for tests
 * of that abort path (a limit of a few nanoseconds makes the first wait that does not
 * succeed at once run out).  Diagnostics only: the paper has no counterpart.
 * Returns CHFSI_OK.
 */
int chfsi_set_pipeline_wait_limit(uint64_t ns);

#ifdef __cplusplus
}
#endif
#endif /* CHFSI_H */
