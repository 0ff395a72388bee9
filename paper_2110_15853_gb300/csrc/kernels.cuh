// Internal launcher declarations shared by the chfsi C-ABI implementation.
#pragma once

#include "common.cuh"

namespace chfsi {

// Limit, in ns, of the waits of one role of a tensor-core kernel on another: 1 s, or
// the shorter value set by chfsi_set_pipeline_wait_limit (tests of the abort path).
uint64_t pipeline_wait_ns();

enum class Buf { F64, F32, BF16, F32X2 };
enum class StepMath { F64, F32, BF16 };

// CSR operator on the device; val_t says whether val points at the caller's FP64
// values or a converted FP32 copy (low-precision steps).
struct CsrDev {
    int64_t N;
    int64_t nnz;
    const int64_t* row_ptr;
    const int32_t* col;
    const void* val;
    Buf val_t;
};

// BSR operator on the device (dense bdim x bdim blocks, bdim = 64).
struct BsrDev {
    int64_t nbr;        // block rows
    int64_t nblocks;
    int bdim;
    const int32_t* brow_ptr;
    const int32_t* bcol;
    const void* val;
    Buf val_t;
};

// Buffers of one filter step: Y_out = alpha (H Y_gather - c Y_cur) - beta Y_prev.
// gather and cur are the same iterate (gather may be its BF16 shadow).
struct StepIO {
    const void* gather; Buf gather_t; int64_t ldg;
    const void* cur;    Buf cur_t;    int64_t ldc;
    const void* prev;   Buf prev_t;   int64_t ldp;   // prev == nullptr: no beta term
    void* out;          Buf out_t;    int64_t ldo;
    void* shadow;       int64_t lds;                 // BF16 copy of the output, or nullptr
    const double* addend; int64_t lda;               // FP64 steps: added to H Y_gather (nullptr: none)
};

int csr_step(const CsrDev& h, StepMath math, int64_t n, const StepIO& io, double alpha, double c,
             double beta, bool vec, unsigned* status, cudaStream_t s);

int bsr_step(const BsrDev& h, StepMath math, int64_t n, const StepIO& io, double alpha, double c,
             double beta, unsigned* status, cudaStream_t s);

// Tensor-core (tcgen05) BF16-operand BSR step; h.val holds BF16 blocks, the BF16
// iterate copies ysh_in / ysh_out are block-major [N/64][n][64].
int bsr_step_tc(const BsrDev& h, int64_t n, const void* ysh_in, const float* Yc, int64_t ldc, const float* Yp,
                int64_t ldp, float* Yo, int64_t ldo, void* ysh_out, double alpha, double c, double beta,
                unsigned* status, cudaStream_t s);
int bsr_values_to_bf16(const double* src, void* dst, int64_t count, cudaStream_t s);

// Two-float blocks (a value is hi + lo, two FP32 numbers, 8 bytes per element).
// Iterate blocks (N x n, leading dimension ld in elements, even) use the pair-split
// layout: the 16 bytes of columns 2t and 2t + 1 of a row hold {hi_2t, hi_2t+1, lo_2t,
// lo_2t+1}, so one 16-byte load gives both lanes of a packed FP32x2 operand.  CSR
// values and small n x n matrices use the pair layout ({hi, lo} per element, float2).
// csr_step_f32x2: h.val in the pair layout, Y blocks pair-split.
int csr_step_f32x2(const CsrDev& h, int64_t n, const void* Yc, int64_t ldc, const void* Yp, int64_t ldp, void* Yo,
                   int64_t ldo, double alpha, double c, double beta, unsigned* status, cudaStream_t s);
// FP64 <-> two-float; split selects the pair-split layout for the two-float side.
int to_f32x2(const double* src, int64_t lds, void* dst, int64_t ldd, int64_t rows, int64_t n, bool split,
             cudaStream_t s);
int from_f32x2(const void* src, int64_t lds, double* dst, int64_t ldd, int64_t rows, int64_t n, bool split,
               cudaStream_t s);
// Two-float dense products: S = A^T B (FP64 result, split-K partials in FP64), A and B
// pair-split N x n blocks; C = A B with A a pair-split N x n block, B an n x n matrix in
// the pair layout, C pair-split two-float or FP64.
int gemm_tn_f32x2(const void* A, int64_t lda, const void* B, int64_t ldb, int64_t K, int64_t n, double* S,
                  int64_t lds, bool symmetric, double* part, int splits, cudaStream_t s);
int gemm_nn_f32x2(const void* A, int64_t lda, const void* B, int64_t ldb, void* C, int64_t ldc, bool c_f64,
                  int64_t M, int64_t n, bool b_upper, cudaStream_t s);
int transpose_to_bf16(const double* src, int64_t lds, void* dst, int64_t N, int64_t n, cudaStream_t s);

// Element-wise conversions (row-major blocks with leading dimensions): columns
// [0, width) of each output row are written, [n, width) as zeros (n <= width <= ldd);
// internal buffers pass width = ldd, caller blocks width = n.
int convert_block(const void* src, Buf src_t, int64_t lds, void* dst, Buf dst_t, int64_t ldd,
                  int64_t rows, int64_t n, int64_t width, cudaStream_t s);
int convert_values(const double* src, void* dst, Buf dst_t, int64_t count, bool round_bf16,
                   cudaStream_t s);

// Dense FP64 kernels of the closure (all row-major).
// S (n x n, lds) = A^T B with A, B: K x n (lda, ldb).  part: split-K scratch of
// splits * n * n doubles; symmetric = compute the upper triangle and mirror it.
int gemm_tn(const double* A, int64_t lda, const double* B, int64_t ldb, int64_t K, int64_t n,
            double* S, int64_t lds, bool symmetric, double* part, int splits, cudaStream_t s);
int gemm_tn_splits(int64_t K, int64_t n);
// C (M x n, ldc) = A (M x n, lda) * B (n x n, ldb); b_upper: B is upper triangular.
int gemm_nn(const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc,
            int64_t M, int64_t n, bool b_upper, cudaStream_t s);
// C (M x Nc, ldc) = alpha op(A) B (+ C when accumulate), op(A) = A (M x K, lda) or, when
// a_t, the transpose of A stored K x M; B: K x Nc (ldb).  FP64 on the DFMA pipe.
int gemm_general(const double* A, int64_t lda, bool a_t, const double* B, int64_t ldb, double* C, int64_t ldc,
                 int64_t M, int64_t Nc, int64_t K, double alpha, bool accumulate, cudaStream_t s);
// In place: upper Cholesky S = R^T R (R in the upper triangle, lower zeroed).
// With oz_ws and scratch (at least (n - 64)^2 doubles) the trailing updates of 256 rows
// and more run as Ozaki products on the tensor cores.
int cholesky_upper(double* S, int64_t n, int64_t lds, unsigned* status, cudaStream_t s, void* oz_ws = nullptr,
                   size_t oz_bytes = 0, double* scratch = nullptr);
// Rinv (n x n) = R^-1 for upper-triangular R (column per warp, n <= 20480).
int tri_inverse_upper(const double* R, int64_t ldr, double* Rinv, int64_t ldi, int64_t n,
                      cudaStream_t s);
// The same by halves with products for the off-diagonal blocks (Ozaki products when oz_ws
// is given); tmp: at least ceil(n/2) x ceil(n/2) doubles (ldt >= n / 2 + 64).
int tri_inverse_upper_blocked(const double* R, int64_t ldr, double* X, int64_t ldx, int64_t n, double* tmp,
                              int64_t ldt, void* oz_ws, size_t oz_bytes, unsigned* status, cudaStream_t s);
// B = A^T (n x n).
int transpose(const double* A, int64_t lda, double* B, int64_t ldb, int64_t n, cudaStream_t s);
// S = (S + S^T)/2 in place.
int symmetrize(double* S, int64_t n, int64_t lds, cudaStream_t s);

// Lanczos (K steps, full re-orthogonalisation) writing bounds to dev_out[3] = {a, b, a0}.
int lanczos_run(const CsrDev& h, int steps, const double* v0, int64_t n_wanted, double* V,
                double* w, double* part, double* scal, double* dev_out, unsigned* status,
                cudaStream_t s);
size_t lanczos_part_count(int64_t N, int steps);

// Sampled dense-dense product on H's pattern: dH[p] += alpha <Ybar[row p,:], Yprev[col p,:]>.
int sddmm_accumulate(const CsrDev& h, int64_t n, const double* Ybar, int64_t ldb,
                     const double* Yprev, int64_t ldp, double alpha, double* dH, cudaStream_t s);

// Two-float variant of sddmm_accumulate on pair-split blocks; ld in elements (even), n even
// or padded with zero columns.
int sddmm_accumulate_f32x2(const CsrDev& h, int64_t n, const void* Ybar, int64_t ldb, const void* Yprev,
                           int64_t ldp, double alpha, double* dH, cudaStream_t s);

int fill_zero(void* p, size_t bytes, cudaStream_t s);

// Hand-written dense symmetric eigensolver (eigh.cu): A (n x n, lda, both triangles)
// = Q diag(w) Q^T with w ascending and Q[k][i] (ldq) component k of eigenvector i.
// A is overwritten.  Scratch from ws (eigh_workspace_bytes).
size_t eigh_workspace_bytes(int64_t n);
int eigh(double* A, int64_t lda, int64_t n, double* w, double* Q, int64_t ldq, void* ws, size_t ws_bytes,
         unsigned* status, cudaStream_t s);

// FP64-accurate products on the BF16 tensor cores (Ozaki-scheme slices, dense_ozaki.cu).
// tn form: C (M x Nc) = A^T B with A: K x M (lda), B: K x Nc (ldb); symmetric: the
// product is known to be symmetric (M == Nc), only the upper tiles are computed.
// nn form: C (M x Nc) = A B with A: M x K (lda), B: K x Nc (ldb); b_upper: B is upper
// triangular.  Scratch from ws (ozaki_workspace_bytes; same = the tn form's A is B).
size_t ozaki_workspace_bytes(bool tn_form, int64_t M, int64_t Nc, int64_t K, bool same);
int ozaki_gemm_tn(const double* A, int64_t lda, const double* B, int64_t ldb, int64_t K, int64_t M, int64_t Nc,
                  double* C, int64_t ldc, bool symmetric, void* ws, size_t ws_bytes, unsigned* status,
                  cudaStream_t s);
int ozaki_gemm_nn(const double* A, int64_t lda, const double* B, int64_t ldb, int64_t M, int64_t K, int64_t Nc,
                  double* C, int64_t ldc, bool b_upper, void* ws, size_t ws_bytes, unsigned* status,
                  cudaStream_t s);
// Block-diagonal product of the split layout: T[kB + i][j] = sum_l D_k[i][l] Y[kB + l][j]
// for every diagonal block k (B x B, row-major, stacked; B a multiple of 128, at most
// 8192).  ozaki_blockdiag_prepare slices the blocks once; ozaki_blockdiag_apply slices
// Y and runs the batched product.  Both use the same workspace (ozaki_blockdiag_bytes).
// FP64-accurate BSR filter step with H's 64 x 64 blocks as Ozaki products on the tensor
// cores: Y_out = alpha (H Y_cur - c Y_cur) - beta Y_prev (Y_prev may be null), FP64
// iterates.  ozaki_bsr_prepare slices H once (rows of at most 128 blocks);
// ozaki_bsr_step slices Y_cur and runs the step.  Both use one workspace (ozaki_bsr_bytes).
// slices = 7: FP64-accurate; slices = 5: the 40-bit step (five digits per operand, the
// 15 slice pairs of weight 2^-48 and above).
size_t ozaki_bsr_bytes(int64_t nbr, int64_t nblocks, int64_t n);
int ozaki_bsr_prepare(const BsrDev& h, int64_t n, void* ws, size_t ws_bytes, unsigned* status, cudaStream_t s);
int ozaki_bsr_step(const BsrDev& h, int64_t n, const double* Yc, int64_t ldc, const double* Yp, int64_t ldp,
                   double* Yo, int64_t ldo, double alpha, double c, double beta, void* ws, size_t ws_bytes,
                   unsigned* status, cudaStream_t s, int slices = 7);
size_t ozaki_blockdiag_bytes(int64_t N, int B, int64_t n);
int ozaki_blockdiag_prepare(const double* diag, int64_t N, int B, int64_t n, void* ws, size_t ws_bytes,
                            unsigned* status, cudaStream_t s);
int ozaki_blockdiag_apply(const double* Y, int64_t ldy, int64_t N, int B, int64_t n, double* T, int64_t ldt,
                          void* ws, size_t ws_bytes, unsigned* status, cudaStream_t s);

}  // namespace chfsi
