// C ABI of the chfsi library: argument validation, workspace layout, the
// per-step schedule of the Chebyshev filter, the adjoint with checkpointing, the
// Rayleigh-Ritz closure and the Lanczos bounds.  Host code here only orders
// kernels on the caller's stream; every arithmetic step runs on the GPU.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <functional>
#include <cstring>
#include <mutex>
#include <vector>


#include "common.cuh"
#include "kernels.cuh"

using namespace chfsi;

namespace {
std::atomic<unsigned long long> g_launches{0};
}

void chfsi::note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

namespace {
constexpr uint64_t kPipelineWaitNs = 1000000000ull;
std::atomic<uint64_t> g_pipeline_wait_ns{kPipelineWaitNs};
}  // namespace

uint64_t chfsi::pipeline_wait_ns() { return g_pipeline_wait_ns.load(std::memory_order_relaxed); }

namespace {

constexpr int kVersion = 10000;   // 1.0.0

inline cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

inline int64_t pad8(int64_t n) { return (n + 7) / 8 * 8; }

// A CSR filter over more than kSlab states runs slab by slab (all m steps on kSlab
// states, then the next kSlab): the columns are independent, and a 512-state slab of
// the iterate gathered by a window of neighbouring rows stays resident in L2 where the
// full width would not.  BSR and hybrid operators keep the full width (the tensor-core
// step's BF16 copy is block-major over all states).
constexpr int64_t kSlab = 512;
inline int64_t filter_slab(const chfsi_matrix* H, int64_t n) {
    return ((H->kind == CHFSI_CSR || H->kind == CHFSI_SPLIT) && n > kSlab) ? kSlab : n;
}

int check_csr(const chfsi_csr& c) {
    if (c.n_rows <= 0 || c.nnz < 0 || c.nnz > INT64_C(0x7fffffffffff)) return CHFSI_ERR_ARG;
    if (c.n_rows > INT32_MAX) return CHFSI_ERR_ARG;
    if (!c.row_ptr || (c.nnz > 0 && (!c.col || !c.val))) return CHFSI_ERR_ARG;
    return CHFSI_OK;
}

int check_bsr(const chfsi_bsr& b) {
    if (b.bdim != 64 || b.n_block_rows <= 0 || b.n_blocks < 0) return CHFSI_ERR_ARG;
    if (!b.brow_ptr || (b.n_blocks > 0 && (!b.bcol || !b.val))) return CHFSI_ERR_ARG;
    if (b.n_block_rows * 64 > INT32_MAX) return CHFSI_ERR_ARG;
    return CHFSI_OK;
}

inline bool has_csr(const chfsi_matrix* H) { return H->kind == CHFSI_CSR || H->kind == CHFSI_HYBRID; }
inline bool has_bsr(const chfsi_matrix* H) { return H->kind == CHFSI_BSR || H->kind == CHFSI_HYBRID; }

int check_split(const chfsi_split& sp) {
    int rc = check_csr(sp.off);
    if (rc) return rc;
    if (sp.n_rows != sp.off.n_rows || !sp.diag) return CHFSI_ERR_ARG;
    if (sp.block <= 0 || sp.block % 128 || sp.block > 8192) return CHFSI_ERR_UNSUPPORTED;
    return CHFSI_OK;
}

int rows_of(const chfsi_matrix* H, int64_t* N) {
    if (!H) return CHFSI_ERR_ARG;
    if (H->kind == CHFSI_SPLIT) {
        const int rc = check_split(H->split);
        if (rc) return rc;
        *N = H->split.n_rows;
        return CHFSI_OK;
    }
    if (H->kind != CHFSI_CSR && H->kind != CHFSI_BSR && H->kind != CHFSI_HYBRID) return CHFSI_ERR_ARG;
    int rc;
    if (has_csr(H) && (rc = check_csr(H->csr))) return rc;
    if (has_bsr(H) && (rc = check_bsr(H->bsr))) return rc;
    if (H->kind == CHFSI_HYBRID && H->csr.n_rows != H->bsr.n_block_rows * H->bsr.bdim) return CHFSI_ERR_ARG;
    *N = has_csr(H) ? H->csr.n_rows : H->bsr.n_block_rows * H->bsr.bdim;
    return CHFSI_OK;
}

int64_t bsr_values(const chfsi_matrix* H) { return H->bsr.n_blocks * (int64_t)H->bsr.bdim * H->bsr.bdim; }

inline int split_block(const chfsi_matrix* H) { return H->kind == CHFSI_SPLIT ? H->split.block : 0; }

// Values of H converted for the low-precision steps (FP32 copy for CUDA-core
// steps, BF16 blocks for tensor-core steps): size of the larger candidate.
// Entries of the low-precision copy of H's values (a BSR copy is followed by one zero
// block, the tensor-core step's stand-in for a block missing from a block-row pair).
int64_t low_values(const chfsi_matrix* H) {
    int64_t v = 0;
    if (has_csr(H)) v = H->csr.nnz;
    if (has_bsr(H)) {
        const int64_t b = bsr_values(H) + (int64_t)H->bsr.bdim * H->bsr.bdim;
        if (b > v) v = b;
    }
    return v;
}

int check_bounds(double a, double b, double a0) {
    if (!std::isfinite(a) || !std::isfinite(b) || !std::isfinite(a0)) return CHFSI_ERR_BOUNDS;
    if (!(a0 < a) || !(a < b)) return CHFSI_ERR_BOUNDS;
    return CHFSI_OK;
}

int check_block(const void* p, int64_t ld, int64_t n) {
    if (!p || ld < n || !aligned16(p)) return CHFSI_ERR_ARG;
    return CHFSI_OK;
}

// Coefficients of Y_k = alpha_k (H - c) Y_{k-1} - beta_k Y_{k-2} from the sigma
// recurrence of Algorithm 1 (alpha_1 = sigma_1/e, alpha_k = 2 sigma_k/e,
// beta_k = sigma_{k-1} sigma_k), computed in FP64 on the host.
void coefficients(int m, double a, double b, double a0, std::vector<double>& alpha, std::vector<double>& beta,
                  double& c) {
    const double e = (b - a) / 2.0;
    c = (b + a) / 2.0;
    double sigma = e / (a0 - c);
    const double sigma1 = sigma;
    const double gamma = 2.0 / sigma1;
    alpha.assign(m + 2, 0.0);
    beta.assign(m + 2, 0.0);
    alpha[1] = sigma1 / e;
    for (int k = 2; k <= m + 1; k++) {
        const double sigma2 = 1.0 / (gamma - sigma);
        alpha[k] = 2.0 * sigma2 / e;
        beta[k] = sigma * sigma2;
        sigma = sigma2;
    }
}

// Low-precision prefix length of a schedule (validated) and the kind of its FP64
// tail: plain FP64 steps, or Ozaki steps (CHFSI_F64_OZAKI, with CHFSI_F40_OZAKI steps
// anywhere among them; tail kind CHFSI_F64_OZAKI), one kind for the whole tail.
int schedule_prefix(const chfsi_schedule* sched, int m, int* L, int* low_kind, int* tail_kind) {
    *L = 0;
    *low_kind = CHFSI_F64;
    *tail_kind = CHFSI_F64;
    if (!sched || !sched->step_prec) return CHFSI_OK;
    if (sched->m != m) return CHFSI_ERR_ARG;
    auto is_oz = [](int p) { return p == CHFSI_F64_OZAKI || p == CHFSI_F40_OZAKI; };
    auto is_tail = [&](int p) { return p == CHFSI_F64 || is_oz(p); };
    int k = 0;
    while (k < m && !is_tail(sched->step_prec[k])) {
        int p = sched->step_prec[k];
        if (p != CHFSI_F32 && p != CHFSI_BF16_F32ACC && p != CHFSI_F32X2) return CHFSI_ERR_ARG;
        if (k > 0 && p != *low_kind) return CHFSI_ERR_ARG;
        *low_kind = p;
        k++;
    }
    if (k < m) *tail_kind = is_oz(sched->step_prec[k]) ? CHFSI_F64_OZAKI : CHFSI_F64;
    for (int r = k; r < m; r++) {
        const int p = sched->step_prec[r];
        if (*tail_kind == CHFSI_F64_OZAKI ? !is_oz(p) : p != CHFSI_F64) return CHFSI_ERR_ARG;
    }
    *L = k;
    return CHFSI_OK;
}

// Whether every block row of a 64 x 64 BSR operator has at most 128 blocks (8192
// columns), the K one Ozaki work item accumulates exactly; copies the block-row
// pointers to the host and synchronises `s`.
int bsr_rows_fit_ozaki(const chfsi_matrix* H, cudaStream_t s, bool* fit) {
    *fit = false;
    if (!has_bsr(H) || H->bsr.bdim != 64) return CHFSI_OK;
    std::vector<int32_t> bp((size_t)H->bsr.n_block_rows + 1);
    CHFSI_CUDA_TRY(cudaMemcpyAsync(bp.data(), H->bsr.brow_ptr, sizeof(int32_t) * bp.size(), cudaMemcpyDeviceToHost, s));
    CHFSI_CUDA_TRY(cudaStreamSynchronize(s));
    for (size_t r = 0; r + 1 < bp.size(); r++)
        if (bp[r + 1] - bp[r] > 128) return CHFSI_OK;
    *fit = true;
    return CHFSI_OK;
}

// Scratch of the Ozaki BSR steps (0 when the schedule has none).
size_t ozaki_tail_bytes(const chfsi_matrix* H, int64_t n, int m, int L, int tail) {
    if (tail != CHFSI_F64_OZAKI || L >= m || !has_bsr(H)) return 0;
    return ozaki_bsr_bytes(H->bsr.n_block_rows, H->bsr.n_blocks, n);
}

struct FilterLayout {
    double* W[2] = {nullptr, nullptr};
    double* T = nullptr;               // split layout: the dense-block product of a step
    unsigned char* bd = nullptr;       // split layout: scratch of the block-diagonal product
    size_t bd_bytes = 0;
    void* hlow = nullptr;
    float* F[3] = {nullptr, nullptr, nullptr};
    __nv_bfloat16* S[2] = {nullptr, nullptr};
    float2* D[3] = {nullptr, nullptr, nullptr};   // two-float iterates
    unsigned char* oz = nullptr;       // Ozaki BSR steps: slices of H and of Y_cur
    size_t oz_bytes = 0;
};

template <typename A>
void filter_layout(A& ar, int64_t N, int64_t n, int m, int L, int low_kind, int64_t nvals, FilterLayout* out,
                   int split_block = 0, size_t oz_bytes = 0) {
    const int64_t ldw = pad8(n);
    FilterLayout fl;
    ar.template take<unsigned char>(kStatusBytes);
    if (m >= 2) {
        fl.W[0] = ar.template take<double>((size_t)(N * ldw));
        fl.W[1] = ar.template take<double>((size_t)(N * ldw));
    }
    if (split_block > 0) {
        fl.T = ar.template take<double>((size_t)(N * ldw));
        fl.bd_bytes = ozaki_blockdiag_bytes(N, split_block, n);
        fl.bd = ar.template take<unsigned char>(fl.bd_bytes);
    }
    if (oz_bytes) {
        fl.oz_bytes = oz_bytes;
        fl.oz = ar.template take<unsigned char>(oz_bytes);
    }
    if (L > 0 && low_kind == CHFSI_F32X2) {
        fl.hlow = ar.template take<float2>((size_t)nvals);
        for (int i = 0; i < 3; i++) fl.D[i] = ar.template take<float2>((size_t)(N * ldw));
    } else if (L > 0) {
        fl.hlow = ar.template take<float>((size_t)nvals);
        for (int i = 0; i < 3; i++) fl.F[i] = ar.template take<float>((size_t)(N * ldw));
        if (low_kind == CHFSI_BF16_F32ACC)
            for (int i = 0; i < 2; i++) fl.S[i] = ar.template take<__nv_bfloat16>((size_t)(N * ldw));
    }
    if (out) *out = fl;
}

struct SizeOnly {
    size_t used = 0;
    template <typename T>
    T* take(size_t count) {
        used = align_up(used) + align_up(count * sizeof(T));
        return nullptr;
    }
};

// FP64 and FP32 steps run on the CSR operator when one is given (CHFSI_CSR or
// CHFSI_HYBRID), otherwise on the BSR blocks with the CUDA-core kernel.
int run_step(const chfsi_matrix* H, const CsrDev& csr, const BsrDev& bsr, StepMath math, int64_t n,
             const StepIO& io, double alpha, double c, double beta, bool vec, unsigned* st, cudaStream_t s) {
    if (has_csr(H)) return csr_step(csr, math, n, io, alpha, c, beta, vec, st, s);
    return bsr_step(bsr, math, n, io, alpha, c, beta, st, s);
}

void make_devs(const chfsi_matrix* H, const void* csr_val, const void* bsr_val, Buf vt, CsrDev* csr, BsrDev* bsr) {
    if (has_csr(H)) *csr = CsrDev{H->csr.n_rows, H->csr.nnz, H->csr.row_ptr, H->csr.col, csr_val, vt};
    if (has_bsr(H))
        *bsr = BsrDev{H->bsr.n_block_rows, H->bsr.n_blocks, H->bsr.bdim, H->bsr.brow_ptr, H->bsr.bcol, bsr_val, vt};
}

}  // namespace

// Exported entry points (C linkage comes from the declarations in chfsi.h).

const char* chfsi_status_string(int st) {
    switch (st) {
        case CHFSI_OK: return "ok";
        case CHFSI_ERR_ARG: return "invalid argument (pointer, size, leading dimension or alignment)";
        case CHFSI_ERR_BOUNDS: return "spectral bounds must be finite with a0 < a < b";
        case CHFSI_ERR_PATTERN: return "invalid sparsity pattern (index out of range)";
        case CHFSI_ERR_CHOL: return "Cholesky-QR failed: Gram matrix not positive definite";
        case CHFSI_ERR_NONFINITE: return "non-finite value produced or read";
        case CHFSI_ERR_CUDA: return "CUDA runtime error";
        case CHFSI_ERR_TIMEOUT: return "bounded device wait timed out";
        case CHFSI_ERR_NOMEM: return "workspace too small";
        case CHFSI_ERR_UNSUPPORTED: return "unsupported combination of layout and precision";
        default: return "unknown status";
    }
}

int chfsi_version(void) { return kVersion; }

unsigned long long chfsi_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int chfsi_set_pipeline_wait_limit(uint64_t ns) {
    g_pipeline_wait_ns.store(ns == 0 ? kPipelineWaitNs : ns, std::memory_order_relaxed);
    return CHFSI_OK;
}

int chfsi_clear_status(void* ws, void* stream) {
    if (!ws) return CHFSI_ERR_ARG;
    CHFSI_CUDA_TRY(cudaMemsetAsync(ws, 0, sizeof(unsigned), as_stream(stream)));
    return CHFSI_OK;
}

int chfsi_read_status(void* ws, void* stream) {
    if (!ws) return CHFSI_ERR_ARG;
    unsigned word = 0;
    CHFSI_CUDA_TRY(cudaStreamSynchronize(as_stream(stream)));
    CHFSI_CUDA_TRY(cudaMemcpy(&word, ws, sizeof(unsigned), cudaMemcpyDeviceToHost));
    CHFSI_CUDA_TRY(cudaMemset(ws, 0, sizeof(unsigned)));
    if (word & DEV_PATTERN) return CHFSI_ERR_PATTERN;
    if (word & DEV_CHOL) return CHFSI_ERR_CHOL;
    if (word & DEV_TIMEOUT) return CHFSI_ERR_TIMEOUT;
    if (word & DEV_NONFINITE) return CHFSI_ERR_NONFINITE;
    return CHFSI_OK;
}

// ------------------------------------------------------------------ filter

int chfsi_filter_workspace_size(const chfsi_matrix* H, int64_t n_cols, int32_t m, const chfsi_schedule* sched,
                                size_t* bytes) {
    if (!bytes) return CHFSI_ERR_ARG;
    int64_t N = 0;
    int rc = rows_of(H, &N);
    if (rc) return rc;
    if (n_cols < 0 || m < 1) return CHFSI_ERR_ARG;
    int L = 0, low = 0, tail = 0;
    rc = schedule_prefix(sched, m, &L, &low, &tail);
    if (rc) return rc;
    if (H->kind == CHFSI_SPLIT && L > 0) return CHFSI_ERR_UNSUPPORTED;
    if (tail == CHFSI_F64_OZAKI && L < m && !has_bsr(H)) return CHFSI_ERR_UNSUPPORTED;
    const int64_t slab = filter_slab(H, n_cols);
    SizeOnly sz;
    filter_layout(sz, N, slab, m, L, low, low_values(H), nullptr, split_block(H), ozaki_tail_bytes(H, slab, m, L, tail));
    *bytes = sz.used;
    return CHFSI_OK;
}

namespace {

// Everything a slab of the filter needs besides its columns.
struct FilterRun {
    const chfsi_matrix* H;
    int64_t N;
    int m, L, low, tail;
    const int32_t* prec;      // the schedule's per-step precisions, or nullptr (all FP64)
    const std::vector<double>* al;
    const std::vector<double>* be;
    double c;
    CsrDev csr64, csrlo;
    BsrDev bsr64, bsrlo;
    FilterLayout fl;
    int64_t ldw;
    unsigned* st;
    cudaStream_t s;
};

// All m steps on n columns: X and Y point at the slab's first column; the internal
// buffers of fl are slab-sized with leading dimension ldw.
int filter_columns(const FilterRun& R, const double* X, int64_t ldx, double* Y, int64_t ldy, int64_t n) {
    const chfsi_matrix* H = R.H;
    const FilterLayout& fl = R.fl;
    const int64_t N = R.N, ldw = R.ldw;
    const int m = R.m, L = R.L, low = R.low;
    const std::vector<double>& al = *R.al;
    const std::vector<double>& be = *R.be;
    const double c = R.c;
    unsigned* st = R.st;
    cudaStream_t s = R.s;
    int rc = CHFSI_OK;
    const bool vec = (n % 2 == 0) && (ldx % 2 == 0) && (ldy % 2 == 0);

    // FP64 iterate k lives in cyc[(m - k) % 3], so that Y_m lands in Y.
    double* cyc[3] = {Y, fl.W[0], fl.W[1]};
    int64_t cyc_ld[3] = {ldy, ldw, ldw};
    auto f64_buf = [&](int k) { return cyc[(m - k) % 3]; };
    auto f64_ld = [&](int k) { return cyc_ld[(m - k) % 3]; };

    bool widened = false;   // low-precision Y_L, Y_{L-1} already widened into their FP64 slots
    if (L > 0 && low == CHFSI_F32X2) {
        const CsrDev h2{H->csr.n_rows, H->csr.nnz, H->csr.row_ptr, H->csr.col, fl.hlow, Buf::F32X2};
        if ((rc = to_f32x2(X, ldx, fl.D[0], ldw, N, n, true, s))) return rc;
        for (int k = 1; k <= L; k++) {
            const void* prev = k >= 2 ? fl.D[(k - 2) % 3] : nullptr;
            rc = csr_step_f32x2(h2, n, fl.D[(k - 1) % 3], ldw, prev, ldw, fl.D[k % 3], ldw, al[k], c,
                                k >= 2 ? be[k] : 0.0, st, s);
            if (rc) return rc;
        }
        if (L == m) return from_f32x2(fl.D[m % 3], ldw, Y, ldy, N, n, true, s);
        if ((rc = from_f32x2(fl.D[L % 3], ldw, f64_buf(L), f64_ld(L), N, n, true, s))) return rc;
        if (L >= 2 && (rc = from_f32x2(fl.D[(L - 1) % 3], ldw, f64_buf(L - 1), f64_ld(L - 1), N, n, true, s))) return rc;
        widened = true;
    } else if (L > 0 && has_bsr(H) && low == CHFSI_BF16_F32ACC) {
        // tensor-core path: BF16 blocks, block-major BF16 iterate copies
        if ((rc = convert_block(X, Buf::F64, ldx, fl.F[0], Buf::F32, ldw, N, n, ldw, s))) return rc;
        if ((rc = transpose_to_bf16(X, ldx, fl.S[0], N, n, s))) return rc;
        for (int k = 1; k <= L; k++) {
            const float* prev = k >= 2 ? fl.F[(k - 2) % 3] : nullptr;
            rc = bsr_step_tc(R.bsrlo, n, fl.S[(k - 1) % 2], fl.F[(k - 1) % 3], ldw, prev, ldw, fl.F[k % 3], ldw,
                             fl.S[k % 2], al[k], c, k >= 2 ? be[k] : 0.0, st, s);
            if (rc) return rc;
        }
        if (L == m) return convert_block(fl.F[m % 3], Buf::F32, ldw, Y, Buf::F64, ldy, N, n, n, s);
    } else if (L > 0) {
        const bool bf = low == CHFSI_BF16_F32ACC;
        if ((rc = convert_block(X, Buf::F64, ldx, fl.F[0], Buf::F32, ldw, N, n, ldw, s))) return rc;
        if (bf && (rc = convert_block(X, Buf::F64, ldx, fl.S[0], Buf::BF16, ldw, N, n, ldw, s))) return rc;
        const StepMath lm = bf ? StepMath::BF16 : StepMath::F32;
        for (int k = 1; k <= L; k++) {
            StepIO io{};
            io.cur = fl.F[(k - 1) % 3]; io.cur_t = Buf::F32; io.ldc = ldw;
            if (bf) { io.gather = fl.S[(k - 1) % 2]; io.gather_t = Buf::BF16; }
            else { io.gather = io.cur; io.gather_t = Buf::F32; }
            io.ldg = ldw;
            if (k >= 2) { io.prev = fl.F[(k - 2) % 3]; io.prev_t = Buf::F32; io.ldp = ldw; }
            io.out = fl.F[k % 3]; io.out_t = Buf::F32; io.ldo = ldw;
            if (bf) { io.shadow = fl.S[k % 2]; io.lds = ldw; }
            rc = run_step(H, R.csrlo, R.bsrlo, lm, n, io, al[k], c, k >= 2 ? be[k] : 0.0, true, st, s);
            if (rc) return rc;
        }
        if (L == m)   // no FP64 step: widen the last iterate into Y
            return convert_block(fl.F[m % 3], Buf::F32, ldw, Y, Buf::F64, ldy, N, n, n, s);
    }

    const bool oz_tail = R.tail == CHFSI_F64_OZAKI;
    if (oz_tail && L > 0 && L < m && !widened) {
        // the Ozaki steps read FP64 iterates: widen Y_L and Y_{L-1} (exact)
        if ((rc = convert_block(fl.F[L % 3], Buf::F32, ldw, f64_buf(L), Buf::F64, f64_ld(L), N, n, n, s))) return rc;
        if (L >= 2 && (rc = convert_block(fl.F[(L - 1) % 3], Buf::F32, ldw, f64_buf(L - 1), Buf::F64, f64_ld(L - 1), N,
                                          n, n, s)))
            return rc;
        widened = true;
    }
    for (int k = L + 1; k <= m; k++) {
        StepIO io{};
        // Y_{k-1}
        if (k - 1 == 0) { io.cur = X; io.cur_t = Buf::F64; io.ldc = ldx; }
        else if (k - 1 <= L && !widened) { io.cur = fl.F[(k - 1) % 3]; io.cur_t = Buf::F32; io.ldc = ldw; }
        else { io.cur = f64_buf(k - 1); io.cur_t = Buf::F64; io.ldc = f64_ld(k - 1); }
        io.gather = io.cur; io.gather_t = io.cur_t; io.ldg = io.ldc;
        // Y_{k-2}
        if (k >= 2) {
            if (k - 2 == 0) { io.prev = X; io.prev_t = Buf::F64; io.ldp = ldx; }
            else if (k - 2 <= L && !widened) { io.prev = fl.F[(k - 2) % 3]; io.prev_t = Buf::F32; io.ldp = ldw; }
            else { io.prev = f64_buf(k - 2); io.prev_t = Buf::F64; io.ldp = f64_ld(k - 2); }
        }
        io.out = f64_buf(k); io.out_t = Buf::F64; io.ldo = f64_ld(k);
        if (oz_tail) {
            // H's blocks as Ozaki products on the tensor cores, FP64 recurrence
            const int slices = R.prec && R.prec[k - 1] == CHFSI_F40_OZAKI ? 5 : 7;
            rc = ozaki_bsr_step(R.bsr64, n, static_cast<const double*>(io.cur), io.ldc,
                                static_cast<const double*>(io.prev), io.ldp, static_cast<double*>(io.out), io.ldo,
                                al[k], c, k >= 2 ? be[k] : 0.0, fl.oz, fl.oz_bytes, st, s, slices);
        } else if (H->kind == CHFSI_SPLIT) {
            // dense diagonal blocks on the tensor cores, then the sparse rest with that sum added
            rc = ozaki_blockdiag_apply(static_cast<const double*>(io.cur), io.ldc, N, H->split.block, n, fl.T, ldw,
                                       fl.bd, fl.bd_bytes, st, s);
            if (rc) return rc;
            io.addend = fl.T;
            io.lda = ldw;
            rc = csr_step(R.csr64, StepMath::F64, n, io, al[k], c, k >= 2 ? be[k] : 0.0, vec, st, s);
        } else {
            rc = run_step(H, R.csr64, R.bsr64, StepMath::F64, n, io, al[k], c, k >= 2 ? be[k] : 0.0, vec, st, s);
        }
        if (rc) return rc;
    }
    return CHFSI_OK;
}

}  // namespace

int chfsi_filter(const chfsi_matrix* H, const double* X, int64_t ldx, double* Y, int64_t ldy, int64_t n_cols,
                 int32_t m, double a, double b, double a0, const chfsi_schedule* sched, void* ws, size_t ws_bytes,
                 void* stream) {
    int64_t N = 0;
    int rc = rows_of(H, &N);
    if (rc) return rc;
    if (n_cols < 0 || m < 1) return CHFSI_ERR_ARG;
    if ((rc = check_bounds(a, b, a0))) return rc;
    if (n_cols == 0) return CHFSI_OK;
    if ((rc = check_block(X, ldx, n_cols)) || (rc = check_block(Y, ldy, n_cols))) return rc;
    if (X == Y) return CHFSI_ERR_ARG;
    int L = 0, low = 0, tail = 0;
    if ((rc = schedule_prefix(sched, m, &L, &low, &tail))) return rc;
    if (!ws || !aligned16(ws)) return CHFSI_ERR_ARG;
    const int64_t slab = filter_slab(H, n_cols);
    if (H->kind == CHFSI_SPLIT && L > 0) return CHFSI_ERR_UNSUPPORTED;
    const bool oz_tail = tail == CHFSI_F64_OZAKI && L < m;
    if (oz_tail && (!has_bsr(H) || H->bsr.bdim != 64)) return CHFSI_ERR_UNSUPPORTED;
    const size_t oz_bytes = ozaki_tail_bytes(H, slab, m, L, tail);
    SizeOnly sz;
    filter_layout(sz, N, slab, m, L, low, low_values(H), nullptr, split_block(H), oz_bytes);
    if (ws_bytes < sz.used) return CHFSI_ERR_NOMEM;
    if (L > 0 && low == CHFSI_F32X2 && !has_csr(H)) return CHFSI_ERR_UNSUPPORTED;
    if (oz_tail) {
        // an Ozaki work item holds one block row: at most 128 blocks (8192 columns) per row
        bool fit = false;
        if ((rc = bsr_rows_fit_ozaki(H, as_stream(stream), &fit))) return rc;
        if (!fit) return CHFSI_ERR_UNSUPPORTED;
    }

    std::vector<double> al, be;
    FilterRun R{};
    R.H = H;
    R.N = N;
    R.m = m;
    R.L = L;
    R.low = low;
    R.tail = tail;
    R.prec = sched ? sched->step_prec : nullptr;
    R.al = &al;
    R.be = &be;
    R.ldw = pad8(slab);
    R.s = as_stream(stream);
    R.st = status_word(ws);
    Arena ar(ws, ws_bytes);
    filter_layout(ar, N, slab, m, L, low, low_values(H), &R.fl, split_block(H), oz_bytes);
    coefficients(m, a, b, a0, al, be, R.c);
    CHFSI_CUDA_TRY(cudaMemsetAsync(R.st, 0, sizeof(unsigned), R.s));
    make_devs(H, H->csr.val, H->bsr.val, Buf::F64, &R.csr64, &R.bsr64);
    if (oz_tail && (rc = ozaki_bsr_prepare(R.bsr64, slab, R.fl.oz, R.fl.oz_bytes, R.st, R.s))) return rc;
    if (H->kind == CHFSI_SPLIT) {
        // the off-diagonal part through the CSR kernel; the dense blocks sliced once
        const chfsi_csr& o = H->split.off;
        R.csr64 = CsrDev{o.n_rows, o.nnz, o.row_ptr, o.col, o.val, Buf::F64};
        if ((rc = ozaki_blockdiag_prepare(H->split.diag, N, H->split.block, slab, R.fl.bd, R.fl.bd_bytes, R.st,
                                          R.s)))
            return rc;
    }

    // low-precision copies of H's values, once for all slabs
    cudaStream_t s = R.s;
    if (L > 0 && low == CHFSI_F32X2) {
        rc = to_f32x2(H->csr.val, 1, R.fl.hlow, 1, H->csr.nnz, 1, false, s);
    } else if (L > 0 && has_bsr(H) && low == CHFSI_BF16_F32ACC) {
        rc = bsr_values_to_bf16(H->bsr.val, R.fl.hlow, bsr_values(H), s);
        make_devs(H, nullptr, R.fl.hlow, Buf::BF16, &R.csrlo, &R.bsrlo);
    } else if (L > 0) {
        const bool bf = low == CHFSI_BF16_F32ACC;
        if (has_csr(H)) rc = convert_values(H->csr.val, R.fl.hlow, Buf::F32, H->csr.nnz, bf, s);
        else rc = convert_values(H->bsr.val, R.fl.hlow, Buf::F32, bsr_values(H), bf, s);
        make_devs(H, R.fl.hlow, R.fl.hlow, Buf::F32, &R.csrlo, &R.bsrlo);
    }
    if (rc) return rc;

    for (int64_t j0 = 0; j0 < n_cols; j0 += slab) {
        const int64_t ns = std::min(slab, n_cols - j0);
        if ((rc = filter_columns(R, X + j0, ldx, Y + j0, ldy, ns))) return rc;
    }
    return CHFSI_OK;
}

// ------------------------------------------------------------------ adjoint

namespace {

struct BackLayout {
    int S = 1, nseg = 1;
    std::vector<double*> ck;      // checkpoint blocks: 2 per segment i >= 1
    std::vector<double*> seg;     // S - 1 replay blocks
    double* A[3] = {nullptr, nullptr, nullptr};
    // two-float run: hi/lo copies of X and dY, Ybar_0, and H's values
    void *X2 = nullptr, *G2 = nullptr, *D0 = nullptr, *H2 = nullptr;
};

// Every block holds 8-byte elements (FP64, or a float2 hi/lo pair), N x round_up(n, 8).
template <typename Ar>
void back_layout(Ar& ar, int64_t N, int64_t n, int m, int stride, int precision, int64_t nnz, BackLayout* out) {
    BackLayout bl;
    bl.S = stride > 0 ? stride : (int)std::ceil(std::sqrt((double)m));
    if (bl.S < 1) bl.S = 1;
    if (bl.S > m) bl.S = m;
    bl.nseg = (m + bl.S - 1) / bl.S;
    const int64_t ldw = pad8(n);
    ar.template take<unsigned char>(kStatusBytes);
    for (int i = 1; i < bl.nseg; i++) {
        bl.ck.push_back(ar.template take<double>((size_t)(N * ldw)));
        bl.ck.push_back(ar.template take<double>((size_t)(N * ldw)));
    }
    for (int i = 1; i < bl.S; i++) bl.seg.push_back(ar.template take<double>((size_t)(N * ldw)));
    for (int i = 0; i < 3; i++) bl.A[i] = ar.template take<double>((size_t)(N * ldw));
    if (precision == CHFSI_F32X2) {
        bl.X2 = ar.template take<double>((size_t)(N * ldw));
        bl.G2 = ar.template take<double>((size_t)(N * ldw));
        bl.D0 = ar.template take<double>((size_t)(N * ldw));
        bl.H2 = ar.template take<double>((size_t)(nnz > 0 ? nnz : 1));
    }
    if (out) *out = bl;
}

// One filter-form step on 8-byte blocks: out = alpha (H cur - c cur) - beta prev.
using BackStep = std::function<int(const void* cur, int64_t ldc, const void* prev, int64_t ldp, void* out,
                                   int64_t ldo, double alpha, double beta)>;
// dH[p] += alpha <Ybar[row p, :], Yprev[col p, :]>.
using BackSddmm = std::function<int(const void* ybar, int64_t ldb, const void* yprev, int64_t ldp, double alpha)>;

// Checkpointed reverse sweep shared by both arithmetics (see chfsi.h).
int backward_sweep(int m, const BackLayout& bl, int64_t ldw, const std::vector<double>& al,
                   const std::vector<double>& be, const void* X, int64_t ldx, const void* dY, int64_t lddy, void* dX,
                   int64_t lddx, bool want_dH, const BackStep& step, const BackSddmm& sddmm) {
    const int S = bl.S;
    int rc;
    // Forward pass to the last checkpoint.  Checkpoint pair of segment i >= 1:
    // Y_{iS-1} -> ck[2(i-1)], Y_{iS} -> ck[2(i-1)+1]; other iterates rotate in A[].
    auto ck_slot = [&](int k) -> void* {
        for (int i = 1; i < bl.nseg; i++) {
            if (k == i * S - 1) return bl.ck[2 * (i - 1)];
            if (k == i * S) return bl.ck[2 * (i - 1) + 1];
        }
        return nullptr;
    };
    std::vector<const void*> fptr(m + 1, nullptr);
    std::vector<int64_t> fld(m + 1, ldw);
    fptr[0] = X;
    fld[0] = ldx;
    const int k_last = (bl.nseg - 1) * S;
    for (int k = 1; k <= k_last; k++) {
        void* out = ck_slot(k);
        if (!out) out = bl.A[k % 3];
        const void* prev = k >= 2 ? fptr[k - 2] : nullptr;
        if ((rc = step(fptr[k - 1], fld[k - 1], prev, k >= 2 ? fld[k - 2] : 0, out, ldw, al[k],
                       k >= 2 ? be[k] : 0.0)))
            return rc;
        fptr[k] = out;
        fld[k] = ldw;
    }

    // Adjoint iterates: Ybar_m = dY; Ybar_j for 1 <= j < m in A[j % 3]; Ybar_0 = dX.
    auto bar_ptr = [&](int j) -> void* { return j == 0 ? dX : (void*)bl.A[j % 3]; };
    auto bar_ld = [&](int j) -> int64_t { return j == m ? lddy : (j == 0 ? lddx : ldw); };
    auto bar_cptr = [&](int j) -> const void* { return j == m ? dY : (const void*)bar_ptr(j); };

    for (int i = bl.nseg - 1; i >= 0; i--) {
        const int s0 = i * S;
        const int e0 = (s0 + S < m) ? s0 + S : m;
        // replay Y_{s0+1} .. Y_{e0-1} from the checkpoint pair (Y_{s0-1}, Y_{s0}), which the
        // forward pass stored in dedicated slots (fptr[0] = X); rotating buffers are not read
        std::vector<const void*> yp(e0 - s0, nullptr);
        std::vector<int64_t> yl(e0 - s0, ldw);
        const void* prevp = (s0 == 0) ? nullptr : fptr[s0 - 1];
        const int64_t prevl = (s0 == 0) ? ldw : fld[s0 - 1];
        yp[0] = fptr[s0];
        yl[0] = fld[s0];
        for (int k = s0 + 1; k <= e0 - 1; k++) {
            void* out = bl.seg[k - s0 - 1];
            const void* pp = (k - 2 - s0 >= 0) ? yp[k - 2 - s0] : prevp;
            const int64_t pl = (k - 2 - s0 >= 0) ? yl[k - 2 - s0] : prevl;
            if ((rc = step(yp[k - 1 - s0], yl[k - 1 - s0], k >= 2 ? pp : nullptr, pl, out, ldw, al[k],
                           k >= 2 ? be[k] : 0.0)))
                return rc;
            yp[k - s0] = out;
        }
        // reverse steps k = e0 .. s0+1
        for (int k = e0; k >= s0 + 1; k--) {
            if (want_dH && (rc = sddmm(bar_cptr(k), bar_ld(k), yp[k - 1 - s0], yl[k - 1 - s0], al[k]))) return rc;
            const void* prev = k + 1 <= m ? bar_cptr(k + 1) : nullptr;
            if ((rc = step(bar_cptr(k), bar_ld(k), prev, k + 1 <= m ? bar_ld(k + 1) : 0, bar_ptr(k - 1),
                           bar_ld(k - 1), al[k], k + 1 <= m ? be[k + 1] : 0.0)))
                return rc;
        }
    }
    return CHFSI_OK;
}

// The reverse sweep reads only the CSR, so it runs in column slabs whatever the layout:
// dX's columns are independent and dH sums over all columns (each slab adds its part).
inline int64_t backward_slab(int64_t n) { return n > kSlab ? kSlab : n; }

int backward_check(const chfsi_matrix* H, int64_t n_cols, int32_t m, int32_t ckpt_stride, int32_t precision,
                   int64_t* N) {
    int rc = rows_of(H, N);
    if (rc) return rc;
    if (!has_csr(H)) return CHFSI_ERR_UNSUPPORTED;
    if (n_cols < 0 || m < 1 || ckpt_stride < 0) return CHFSI_ERR_ARG;
    if (precision != CHFSI_F64 && precision != CHFSI_F32X2) return CHFSI_ERR_ARG;
    return CHFSI_OK;
}

}  // namespace

int chfsi_filter_backward_ex_workspace_size(const chfsi_matrix* H, int64_t n_cols, int32_t m, int32_t ckpt_stride,
                                            int32_t precision, size_t* bytes) {
    if (!bytes) return CHFSI_ERR_ARG;
    int64_t N = 0;
    int rc = backward_check(H, n_cols, m, ckpt_stride, precision, &N);
    if (rc) return rc;
    SizeOnly sz;
    back_layout(sz, N, backward_slab(n_cols), m, ckpt_stride, precision, H->csr.nnz, nullptr);
    *bytes = sz.used;
    return CHFSI_OK;
}

int chfsi_filter_backward_workspace_size(const chfsi_matrix* H, int64_t n_cols, int32_t m, int32_t ckpt_stride,
                                         size_t* bytes) {
    return chfsi_filter_backward_ex_workspace_size(H, n_cols, m, ckpt_stride, CHFSI_F64, bytes);
}

int chfsi_filter_backward_ex(const chfsi_matrix* H, const double* X, int64_t ldx, const double* dY, int64_t lddy,
                             double* dX, int64_t lddx, double* dH_val, int64_t n_cols, int32_t m, double a, double b,
                             double a0, int32_t ckpt_stride, int32_t precision, void* ws, size_t ws_bytes,
                             void* stream) {
    int64_t N = 0;
    int rc = backward_check(H, n_cols, m, ckpt_stride, precision, &N);
    if (rc) return rc;
    if ((rc = check_bounds(a, b, a0))) return rc;
    cudaStream_t s = as_stream(stream);
    if (n_cols == 0) {
        if (dH_val) return fill_zero(dH_val, sizeof(double) * (size_t)H->csr.nnz, s);
        return CHFSI_OK;
    }
    if ((rc = check_block(X, ldx, n_cols)) || (rc = check_block(dY, lddy, n_cols)) ||
        (rc = check_block(dX, lddx, n_cols)))
        return rc;
    if (dX == X || dX == dY) return CHFSI_ERR_ARG;
    if (!ws || !aligned16(ws)) return CHFSI_ERR_ARG;
    const int64_t slab = backward_slab(n_cols);
    SizeOnly sz;
    back_layout(sz, N, slab, m, ckpt_stride, precision, H->csr.nnz, nullptr);
    if (ws_bytes < sz.used) return CHFSI_ERR_NOMEM;
    Arena ar(ws, ws_bytes);
    BackLayout bl;
    back_layout(ar, N, slab, m, ckpt_stride, precision, H->csr.nnz, &bl);
    unsigned* st = status_word(ws);
    CHFSI_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(unsigned), s));

    std::vector<double> al, be;
    double c = 0.0;
    coefficients(m, a, b, a0, al, be, c);
    const int64_t ldw = pad8(slab);
    if (dH_val && (rc = fill_zero(dH_val, sizeof(double) * (size_t)H->csr.nnz, s))) return rc;
    if (precision == CHFSI_F32X2 && (rc = to_f32x2(H->csr.val, 1, bl.H2, 1, H->csr.nnz, 1, false, s))) return rc;

    for (int64_t j0 = 0; j0 < n_cols; j0 += slab) {
        const int64_t n = std::min(slab, n_cols - j0);
        const double* Xs = X + j0;
        const double* dYs = dY + j0;
        double* dXs = dX + j0;
        if (precision == CHFSI_F64) {
            const bool vec = (n % 2 == 0) && (ldx % 2 == 0) && (lddy % 2 == 0) && (lddx % 2 == 0);
            const CsrDev h{H->csr.n_rows, H->csr.nnz, H->csr.row_ptr, H->csr.col, H->csr.val, Buf::F64};
            BackStep step = [&](const void* cur, int64_t ldc, const void* prev, int64_t ldp, void* out,
                                int64_t ldo, double alpha, double beta) {
                StepIO io{};
                io.cur = cur; io.cur_t = Buf::F64; io.ldc = ldc;
                io.gather = cur; io.gather_t = Buf::F64; io.ldg = ldc;
                if (prev) { io.prev = prev; io.prev_t = Buf::F64; io.ldp = ldp; }
                io.out = out; io.out_t = Buf::F64; io.ldo = ldo;
                return csr_step(h, StepMath::F64, n, io, alpha, c, beta, vec, st, s);
            };
            BackSddmm sddmm = [&](const void* yb, int64_t ldb, const void* ypv, int64_t ldp, double alpha) {
                return sddmm_accumulate(h, n, static_cast<const double*>(yb), ldb, static_cast<const double*>(ypv),
                                        ldp, alpha, dH_val, s);
            };
            rc = backward_sweep(m, bl, ldw, al, be, Xs, ldx, dYs, lddy, dXs, lddx, dH_val != nullptr, step, sddmm);
            if (rc) return rc;
            continue;
        }
        // two-float: hi/lo copies of the slab of X and dY; Ybar_0 widened into dX at the end
        if ((rc = to_f32x2(Xs, ldx, bl.X2, ldw, N, n, true, s))) return rc;
        if ((rc = to_f32x2(dYs, lddy, bl.G2, ldw, N, n, true, s))) return rc;
        const CsrDev h2{H->csr.n_rows, H->csr.nnz, H->csr.row_ptr, H->csr.col, bl.H2, Buf::F32X2};
        BackStep step = [&](const void* cur, int64_t ldc, const void* prev, int64_t ldp, void* out, int64_t ldo,
                            double alpha, double beta) {
            return csr_step_f32x2(h2, n, cur, ldc, prev, prev ? ldp : 0, out, ldo, alpha, c, beta, st, s);
        };
        BackSddmm sddmm = [&](const void* yb, int64_t ldb, const void* ypv, int64_t ldp, double alpha) {
            return sddmm_accumulate_f32x2(h2, n, yb, ldb, ypv, ldp, alpha, dH_val, s);
        };
        if ((rc = backward_sweep(m, bl, ldw, al, be, bl.X2, ldw, bl.G2, ldw, bl.D0, ldw, dH_val != nullptr, step,
                                 sddmm)))
            return rc;
        if ((rc = from_f32x2(bl.D0, ldw, dXs, lddx, N, n, true, s))) return rc;
    }
    return CHFSI_OK;
}

int chfsi_filter_backward(const chfsi_matrix* H, const double* X, int64_t ldx, const double* dY, int64_t lddy,
                          double* dX, int64_t lddx, double* dH_val, int64_t n_cols, int32_t m, double a, double b,
                          double a0, int32_t ckpt_stride, void* ws, size_t ws_bytes, void* stream) {
    return chfsi_filter_backward_ex(H, X, ldx, dY, lddy, dX, lddx, dH_val, n_cols, m, a, b, a0, ckpt_stride,
                                    CHFSI_F64, ws, ws_bytes, stream);
}

// ------------------------------------------------------------------ Rayleigh-Ritz

namespace {

struct RRLayout {
    double *S = nullptr, *part = nullptr, *XF = nullptr, *T = nullptr, *Rinv = nullptr, *Q = nullptr;
    unsigned char* eig = nullptr;    // scratch of the dense eigensolver
    size_t eig_bytes = 0;
    int splits = 1;
    // two-float closure
    float2 *Y2 = nullptr, *B2[2] = {nullptr, nullptr}, *HX2 = nullptr, *R2 = nullptr, *Q2 = nullptr, *H2 = nullptr;
    // Ozaki closure: scratch of the tensor-core products, reused by the two-float H X_F
    unsigned char* oz = nullptr;
    size_t oz_bytes = 0;
};

// Scratch of the Ozaki closure: the largest of its four products and of the
// two-float H X_F (two pair-split N x ldw blocks and H's values as pairs).
size_t rr_ozaki_bytes(int64_t N, int64_t n, int64_t nnz, bool csr) {
    size_t b = ozaki_workspace_bytes(true, n, n, N, true);
    b = std::max(b, ozaki_workspace_bytes(false, N, n, n, false));
    b = std::max(b, ozaki_workspace_bytes(true, n, n, N, false));
    if (csr) {
        Sizer sz;
        sz.take<float2>((size_t)(N * pad8(n)));
        sz.take<float2>((size_t)(N * pad8(n)));
        sz.take<float2>((size_t)(nnz > 0 ? nnz : 1));
        b = std::max(b, sz.used);
    }
    return b;
}

// Scratch of the Ozaki closure's H X_F as an Ozaki BSR step (operators with 64 x 64
// blocks), 0 otherwise.
size_t rr_bsr_ozaki_bytes(const chfsi_matrix* H, int64_t n, int precision) {
    if (precision != CHFSI_F64_OZAKI || !has_bsr(H) || H->bsr.bdim != 64) return 0;
    return ozaki_bsr_bytes(H->bsr.n_block_rows, H->bsr.n_blocks, n);
}

template <typename Ar>
void rr_layout(Ar& ar, int64_t N, int64_t n, int precision, int64_t nnz, bool csr, size_t bsr_oz, RRLayout* out) {
    RRLayout rl;
    const int64_t ldw = pad8(n);
    rl.splits = gemm_tn_splits(N, n);
    ar.template take<unsigned char>(kStatusBytes);
    rl.S = ar.template take<double>((size_t)(n * n));
    rl.part = ar.template take<double>((size_t)(rl.splits * n * n));
    rl.Rinv = ar.template take<double>((size_t)(n * n));
    rl.Q = ar.template take<double>((size_t)(n * n));
    rl.eig_bytes = eigh_workspace_bytes(n);
    rl.eig = ar.template take<unsigned char>(rl.eig_bytes);
    if (precision == CHFSI_F32X2) {
        rl.Y2 = ar.template take<float2>((size_t)(N * ldw));
        rl.B2[0] = ar.template take<float2>((size_t)(N * ldw));
        rl.B2[1] = ar.template take<float2>((size_t)(N * ldw));
        rl.R2 = ar.template take<float2>((size_t)(n * n));
        rl.Q2 = ar.template take<float2>((size_t)(n * n));
        rl.H2 = ar.template take<float2>((size_t)(nnz > 0 ? nnz : 1));
    } else {
        rl.XF = ar.template take<double>((size_t)(N * ldw));
        rl.T = ar.template take<double>((size_t)(N * ldw));
    }
    if (precision == CHFSI_F64_OZAKI) {
        rl.oz_bytes = std::max(rr_ozaki_bytes(N, n, nnz, csr), bsr_oz);
        rl.oz = ar.template take<unsigned char>(rl.oz_bytes);
    }
    if (out) *out = rl;
}

int rr_check(const chfsi_matrix* H, int64_t n_cols, int32_t cholqr_passes, int32_t precision, int64_t* N) {
    int rc = rows_of(H, N);
    if (rc) return rc;
    if (H->kind == CHFSI_SPLIT) return CHFSI_ERR_UNSUPPORTED;
    if (n_cols < 1 || n_cols > *N || (cholqr_passes != 1 && cholqr_passes != 2)) return CHFSI_ERR_ARG;
    if (precision != CHFSI_F64 && precision != CHFSI_F32X2 && precision != CHFSI_F64_OZAKI) return CHFSI_ERR_ARG;
    if (precision == CHFSI_F32X2 && !has_csr(H)) return CHFSI_ERR_UNSUPPORTED;
    return CHFSI_OK;
}

// Step 4 (eigensolve, the library's divide-and-conquer solver) and the status read-back
// shared by all precisions.  Q[k][i] = component k of the eigenvector of ritz[i].
int rr_eig(const RRLayout& rl, int64_t n, double* ritz, unsigned* st, cudaStream_t s) {
    return eigh(rl.S, n, n, ritz, rl.Q, n, rl.eig, rl.eig_bytes, st, s);
}

int rr_finish(const RRLayout& rl, unsigned* st, cudaStream_t s) {
    (void)rl;
    CHFSI_CUDA_TRY(cudaStreamSynchronize(s));
    unsigned word = 0;
    CHFSI_CUDA_TRY(cudaMemcpy(&word, st, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (word & DEV_PATTERN) return CHFSI_ERR_PATTERN;
    if (word & DEV_CHOL) return CHFSI_ERR_CHOL;
    if (word & DEV_NONFINITE) return CHFSI_ERR_NONFINITE;
    return CHFSI_OK;
}

// CholQR2 without the last product: with X1 the first pass's basis and X1^T X1 = R2^T R2,
// X_F = X1 R2^-1 is not formed.  Its projection is R2^-T (X1^T H X1) R2^-1 and its Ritz
// vectors are X1 (R2^-1 Q): in exact arithmetic the same quantities (Algorithm 1 steps
// 2, 3, 5), for n x n x n products in place of one N x n x n product.  rr_fold_projection
// takes P = X1^T H X1 in rl.S and leaves H_F there (T = P R2^-1 in rl.Q, then R2^-T T,
// symmetric); rr_fold_vectors leaves G = R2^-1 Q in rl.part.  Ozaki products when oz,
// FP64 otherwise.
int rr_fold_projection(const RRLayout& rl, int64_t n, bool oz, unsigned* st, cudaStream_t s) {
    int rc;
    if (oz) {
        if ((rc = ozaki_gemm_nn(rl.S, n, rl.Rinv, n, n, n, n, rl.Q, n, true, rl.oz, rl.oz_bytes, st, s))) return rc;
        if ((rc = ozaki_gemm_tn(rl.Rinv, n, rl.Q, n, n, n, n, rl.S, n, true, rl.oz, rl.oz_bytes, st, s))) return rc;
    } else {
        if ((rc = gemm_general(rl.S, n, false, rl.Rinv, n, rl.Q, n, n, n, n, 1.0, false, s))) return rc;
        if ((rc = gemm_general(rl.Rinv, n, true, rl.Q, n, rl.S, n, n, n, n, 1.0, false, s))) return rc;
    }
    return symmetrize(rl.S, n, n, s);
}

int rr_fold_vectors(const RRLayout& rl, int64_t n, bool oz, unsigned* st, cudaStream_t s) {
    if (oz) return ozaki_gemm_nn(rl.Rinv, n, rl.Q, n, n, n, n, rl.part, n, false, rl.oz, rl.oz_bytes, st, s);
    return gemm_general(rl.Rinv, n, false, rl.Q, n, rl.part, n, n, n, n, 1.0, false, s);
}

// Steps 2, 3 and 5 with two-float products (Cholesky, triangular inverse and the
// eigensolve stay FP64).
int rr_run_f32x2(const chfsi_matrix* H, const double* Y, int64_t ldy, int64_t N, int64_t n, double* Psi,
                 int64_t ldpsi, double* ritz, int passes, const RRLayout& rl, unsigned* st, cudaStream_t s) {
    const int64_t ldw = pad8(n);
    int rc;
    if ((rc = to_f32x2(Y, ldy, rl.Y2, ldw, N, n, true, s))) return rc;
    const float2* cur = rl.Y2;
    int which = 0;
    const bool fold = passes == 2;
    for (int pass = 0; pass < passes; pass++) {
        if ((rc = gemm_tn_f32x2(cur, ldw, cur, ldw, N, n, rl.S, n, true, rl.part, rl.splits, s))) return rc;
        if ((rc = cholesky_upper(rl.S, n, n, st, s))) return rc;
        if ((rc = tri_inverse_upper_blocked(rl.S, n, rl.Rinv, n, n, rl.Q, n, nullptr, 0, st, s))) return rc;
        if (fold && pass == passes - 1) break;   // X_F = X1 R2^-1 is not formed
        if ((rc = to_f32x2(rl.Rinv, n, rl.R2, n, n, n, false, s))) return rc;
        float2* out = rl.B2[which];
        if ((rc = gemm_nn_f32x2(cur, ldw, rl.R2, n, out, ldw, false, N, n, true, s))) return rc;
        cur = out;
        which ^= 1;
    }
    const float2* XF = cur;
    float2* HXF = rl.B2[which];
    if ((rc = to_f32x2(H->csr.val, 1, rl.H2, 1, H->csr.nnz, 1, false, s))) return rc;
    const CsrDev h2{H->csr.n_rows, H->csr.nnz, H->csr.row_ptr, H->csr.col, rl.H2, Buf::F32X2};
    if ((rc = csr_step_f32x2(h2, n, XF, ldw, nullptr, 0, HXF, ldw, 1.0, 0.0, 0.0, st, s))) return rc;
    // H_F is symmetric: only the tiles on and above the diagonal are computed, the others
    // mirrored, and the diagonal tiles averaged with their transposes
    if ((rc = gemm_tn_f32x2(XF, ldw, HXF, ldw, N, n, rl.S, n, true, rl.part, rl.splits, s))) return rc;
    if ((rc = symmetrize(rl.S, n, n, s))) return rc;
    if (fold && (rc = rr_fold_projection(rl, n, false, st, s))) return rc;
    if ((rc = rr_eig(rl, n, ritz, st, s))) return rc;
    if (fold && (rc = rr_fold_vectors(rl, n, false, st, s))) return rc;
    if ((rc = to_f32x2(fold ? rl.part : rl.Q, n, rl.Q2, n, n, n, false, s))) return rc;
    if ((rc = gemm_nn_f32x2(XF, ldw, rl.Q2, n, Psi, ldpsi, true, N, n, false, s))) return rc;
    return rr_finish(rl, st, s);
}

// Steps 2, 3 and 5 with the dense products on the tensor cores (Ozaki slices) and
// H X_F in two-float arithmetic (FP64 on a BSR-only operator); the Cholesky
// factorisation, the triangular inverse and the eigensolve stay FP64.
int rr_run_ozaki(const chfsi_matrix* H, const double* Y, int64_t ldy, int64_t N, int64_t n, double* Psi,
                 int64_t ldpsi, double* ritz, int passes, bool bsr_hx, const RRLayout& rl, unsigned* st,
                 cudaStream_t s) {
    const int64_t ldw = pad8(n);
    int rc;
    const double* cur = Y;
    int64_t cur_ld = ldy;
    double* bufs[2] = {rl.XF, rl.T};
    int which = 0;
    const bool fold = passes == 2;
    for (int pass = 0; pass < passes; pass++) {
        if ((rc = ozaki_gemm_tn(cur, cur_ld, cur, cur_ld, N, n, n, rl.S, n, true, rl.oz, rl.oz_bytes, st, s)))
            return rc;
        if ((rc = cholesky_upper(rl.S, n, n, st, s, rl.oz, rl.oz_bytes, rl.Q))) return rc;
        if ((rc = tri_inverse_upper_blocked(rl.S, n, rl.Rinv, n, n, rl.Q, n, rl.oz, rl.oz_bytes, st, s)))
            return rc;
        if (fold && pass == passes - 1) break;   // X_F = X1 R2^-1 is not formed
        double* out = bufs[which];
        if ((rc = ozaki_gemm_nn(cur, cur_ld, rl.Rinv, n, N, n, n, out, ldw, true, rl.oz, rl.oz_bytes, st, s)))
            return rc;
        cur = out;
        cur_ld = ldw;
        which ^= 1;
    }
    double* XF = const_cast<double*>(cur);
    double* HXF = bufs[which];
    if (bsr_hx) {
        // H's 64 x 64 blocks as Ozaki products (the BSR step with alpha = 1, c = 0)
        CsrDev csr{};
        BsrDev bsr{};
        make_devs(H, H->csr.val, H->bsr.val, Buf::F64, &csr, &bsr);
        if ((rc = ozaki_bsr_prepare(bsr, n, rl.oz, rl.oz_bytes, st, s))) return rc;
        if ((rc = ozaki_bsr_step(bsr, n, XF, ldw, nullptr, 0, HXF, ldw, 1.0, 0.0, 0.0, rl.oz, rl.oz_bytes, st, s)))
            return rc;
    } else if (has_csr(H)) {
        Arena ar(rl.oz, rl.oz_bytes);
        float2* X2 = ar.take<float2>((size_t)(N * ldw));
        float2* HX2 = ar.take<float2>((size_t)(N * ldw));
        float2* H2 = ar.take<float2>((size_t)(H->csr.nnz > 0 ? H->csr.nnz : 1));
        if ((rc = to_f32x2(XF, ldw, X2, ldw, N, n, true, s))) return rc;
        if ((rc = to_f32x2(H->csr.val, 1, H2, 1, H->csr.nnz, 1, false, s))) return rc;
        const CsrDev h2{H->csr.n_rows, H->csr.nnz, H->csr.row_ptr, H->csr.col, H2, Buf::F32X2};
        if ((rc = csr_step_f32x2(h2, n, X2, ldw, nullptr, 0, HX2, ldw, 1.0, 0.0, 0.0, st, s))) return rc;
        if ((rc = from_f32x2(HX2, ldw, HXF, ldw, N, n, true, s))) return rc;
    } else {
        CsrDev csr{};
        BsrDev bsr{};
        make_devs(H, H->csr.val, H->bsr.val, Buf::F64, &csr, &bsr);
        StepIO io{};
        io.cur = XF; io.cur_t = Buf::F64; io.ldc = ldw;
        io.gather = XF; io.gather_t = Buf::F64; io.ldg = ldw;
        io.out = HXF; io.out_t = Buf::F64; io.ldo = ldw;
        if ((rc = run_step(H, csr, bsr, StepMath::F64, n, io, 1.0, 0.0, 0.0, n % 2 == 0, st, s))) return rc;
    }
    // H_F is symmetric: the tiles on and above the diagonal, mirrored, the diagonal
    // tiles averaged with their transposes
    if ((rc = ozaki_gemm_tn(XF, ldw, HXF, ldw, N, n, n, rl.S, n, true, rl.oz, rl.oz_bytes, st, s))) return rc;
    if ((rc = symmetrize(rl.S, n, n, s))) return rc;
    if (fold && (rc = rr_fold_projection(rl, n, true, st, s))) return rc;
    if ((rc = rr_eig(rl, n, ritz, st, s))) return rc;
    if (fold && (rc = rr_fold_vectors(rl, n, true, st, s))) return rc;
    if ((rc = ozaki_gemm_nn(XF, ldw, fold ? rl.part : rl.Q, n, N, n, n, Psi, ldpsi, false, rl.oz, rl.oz_bytes, st,
                            s)))
        return rc;
    return rr_finish(rl, st, s);
}

}  // namespace

int chfsi_rayleigh_ritz_ex_workspace_size(const chfsi_matrix* H, int64_t n_cols, int32_t cholqr_passes,
                                          int32_t precision, size_t* bytes) {
    if (!bytes) return CHFSI_ERR_ARG;
    int64_t N = 0;
    int rc = rr_check(H, n_cols, cholqr_passes, precision, &N);
    if (rc) return rc;
    SizeOnly sz;
    rr_layout(sz, N, n_cols, precision, has_csr(H) ? H->csr.nnz : 0, has_csr(H), rr_bsr_ozaki_bytes(H, n_cols, precision),
              nullptr);
    *bytes = sz.used;
    return CHFSI_OK;
}

int chfsi_rayleigh_ritz_workspace_size(const chfsi_matrix* H, int64_t n_cols, int32_t cholqr_passes, size_t* bytes) {
    return chfsi_rayleigh_ritz_ex_workspace_size(H, n_cols, cholqr_passes, CHFSI_F64, bytes);
}

int chfsi_rayleigh_ritz_ex(const chfsi_matrix* H, const double* Y, int64_t ldy, int64_t n_cols, double* Psi,
                           int64_t ldpsi, double* ritz, int32_t cholqr_passes, int32_t precision, void* ws,
                           size_t ws_bytes, void* stream) {
    int64_t N = 0;
    int rc = rr_check(H, n_cols, cholqr_passes, precision, &N);
    if (rc) return rc;
    if ((rc = check_block(Y, ldy, n_cols)) || (rc = check_block(Psi, ldpsi, n_cols))) return rc;
    if (!ritz || Psi == Y) return CHFSI_ERR_ARG;
    if (!ws || !aligned16(ws)) return CHFSI_ERR_ARG;
    const int64_t nnz = has_csr(H) ? H->csr.nnz : 0;
    SizeOnly sz;
    const size_t bsr_oz = rr_bsr_ozaki_bytes(H, n_cols, precision);
    rr_layout(sz, N, n_cols, precision, nnz, has_csr(H), bsr_oz, nullptr);
    if (ws_bytes < sz.used) return CHFSI_ERR_NOMEM;
    Arena ar(ws, ws_bytes);
    RRLayout rl;
    rr_layout(ar, N, n_cols, precision, nnz, has_csr(H), bsr_oz, &rl);
    cudaStream_t s = as_stream(stream);
    unsigned* st = status_word(ws);
    CHFSI_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(unsigned), s));
    const int64_t n = n_cols, ldw = pad8(n);
    if (precision == CHFSI_F32X2) return rr_run_f32x2(H, Y, ldy, N, n, Psi, ldpsi, ritz, cholqr_passes, rl, st, s);
    if (precision == CHFSI_F64_OZAKI) {
        bool bsr_hx = false;
        if (bsr_oz && (rc = bsr_rows_fit_ozaki(H, s, &bsr_hx))) return rc;
        return rr_run_ozaki(H, Y, ldy, N, n, Psi, ldpsi, ritz, cholqr_passes, bsr_hx, rl, st, s);
    }

    // step 2: X_F = Y R^-1 with S = Y^T Y = R^T R (repeated on X_F for CholQR2, whose last
    // product is folded into steps 3 and 5)
    const double* cur = Y;
    int64_t cur_ld = ldy;
    double* bufs[2] = {rl.XF, rl.T};
    int which = 0;
    const bool fold = cholqr_passes == 2;
    for (int pass = 0; pass < cholqr_passes; pass++) {
        if ((rc = gemm_tn(cur, cur_ld, cur, cur_ld, N, n, rl.S, n, true, rl.part, rl.splits, s))) return rc;
        if ((rc = cholesky_upper(rl.S, n, n, st, s))) return rc;
        if ((rc = tri_inverse_upper_blocked(rl.S, n, rl.Rinv, n, n, rl.Q, n, nullptr, 0, st, s))) return rc;
        if (fold && pass == cholqr_passes - 1) break;   // X_F = X1 R2^-1 is not formed
        double* out = bufs[which];
        if ((rc = gemm_nn(cur, cur_ld, rl.Rinv, n, out, ldw, N, n, true, s))) return rc;
        cur = out;
        cur_ld = ldw;
        which ^= 1;
    }
    double* XF = const_cast<double*>(cur);
    double* HXF = bufs[which];
    // step 3: H_F = X_F^T (H X_F)
    {
        CsrDev csr{};
        BsrDev bsr{};
        make_devs(H, H->csr.val, H->bsr.val, Buf::F64, &csr, &bsr);
        StepIO io{};
        io.cur = XF; io.cur_t = Buf::F64; io.ldc = ldw;
        io.gather = XF; io.gather_t = Buf::F64; io.ldg = ldw;
        io.out = HXF; io.out_t = Buf::F64; io.ldo = ldw;
        if ((rc = run_step(H, csr, bsr, StepMath::F64, n, io, 1.0, 0.0, 0.0, n % 2 == 0, st, s))) return rc;
    }
    // H_F is symmetric: only the tiles on and above the diagonal are computed, the others
    // mirrored, and the diagonal tiles averaged with their transposes
    if ((rc = gemm_tn(XF, ldw, HXF, ldw, N, n, rl.S, n, true, rl.part, rl.splits, s))) return rc;
    if ((rc = symmetrize(rl.S, n, n, s))) return rc;
    if (fold && (rc = rr_fold_projection(rl, n, false, st, s))) return rc;
    // step 4: H_F Q = Q Lambda
    if ((rc = rr_eig(rl, n, ritz, st, s))) return rc;
    // step 5: Psi = X_F Q (= X1 (R2^-1 Q) after CholQR2)
    if (fold && (rc = rr_fold_vectors(rl, n, false, st, s))) return rc;
    if ((rc = gemm_nn(XF, ldw, fold ? rl.part : rl.Q, n, Psi, ldpsi, N, n, false, s))) return rc;
    return rr_finish(rl, st, s);
}

int chfsi_rayleigh_ritz(const chfsi_matrix* H, const double* Y, int64_t ldy, int64_t n_cols, double* Psi,
                        int64_t ldpsi, double* ritz, int32_t cholqr_passes, void* ws, size_t ws_bytes, void* stream) {
    return chfsi_rayleigh_ritz_ex(H, Y, ldy, n_cols, Psi, ldpsi, ritz, cholqr_passes, CHFSI_F64, ws, ws_bytes,
                                  stream);
}

// ------------------------------------------------------------------ Lanczos bounds

int chfsi_lanczos_workspace_size(const chfsi_matrix* H, int32_t steps, size_t* bytes) {
    if (!bytes) return CHFSI_ERR_ARG;
    int64_t N = 0;
    int rc = rows_of(H, &N);
    if (rc) return rc;
    if (!has_csr(H)) return CHFSI_ERR_UNSUPPORTED;
    if (steps < 1 || steps > 64) return CHFSI_ERR_ARG;
    SizeOnly sz;
    sz.take<unsigned char>(kStatusBytes);
    sz.take<double>((size_t)((steps + 1) * N));
    sz.take<double>((size_t)N);
    sz.take<double>(lanczos_part_count(N, steps));
    sz.take<double>(512);
    sz.take<double>(4);
    *bytes = sz.used;
    return CHFSI_OK;
}

int chfsi_lanczos_bounds(const chfsi_matrix* H, int32_t steps, const double* v0, int64_t n_wanted, double* a,
                         double* b, double* a0, void* ws, size_t ws_bytes, void* stream) {
    int64_t N = 0;
    int rc = rows_of(H, &N);
    if (rc) return rc;
    if (!has_csr(H)) return CHFSI_ERR_UNSUPPORTED;
    if (steps < 1 || steps > 64 || !v0 || !a || !b || !a0 || n_wanted < 1 || n_wanted >= N) return CHFSI_ERR_ARG;
    if (!ws || !aligned16(ws)) return CHFSI_ERR_ARG;
    size_t need = 0;
    if ((rc = chfsi_lanczos_workspace_size(H, steps, &need))) return rc;
    if (ws_bytes < need) return CHFSI_ERR_NOMEM;
    Arena ar(ws, ws_bytes);
    ar.take<unsigned char>(kStatusBytes);
    double* V = ar.take<double>((size_t)((steps + 1) * N));
    double* w = ar.take<double>((size_t)N);
    double* part = ar.take<double>(lanczos_part_count(N, steps));
    double* scal = ar.take<double>(512);
    double* out = ar.take<double>(4);
    cudaStream_t s = as_stream(stream);
    unsigned* st = status_word(ws);
    CHFSI_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(unsigned), s));
    CsrDev h{H->csr.n_rows, H->csr.nnz, H->csr.row_ptr, H->csr.col, H->csr.val, Buf::F64};
    if ((rc = lanczos_run(h, steps, v0, n_wanted, V, w, part, scal, out, st, s))) return rc;
    double host[3];
    CHFSI_CUDA_TRY(cudaMemcpyAsync(host, out, sizeof(host), cudaMemcpyDeviceToHost, s));
    CHFSI_CUDA_TRY(cudaStreamSynchronize(s));
    unsigned word = 0;
    CHFSI_CUDA_TRY(cudaMemcpy(&word, st, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (word & DEV_PATTERN) return CHFSI_ERR_PATTERN;
    if (!std::isfinite(host[0]) || !std::isfinite(host[1]) || !std::isfinite(host[2])) return CHFSI_ERR_NONFINITE;
    *a = host[0];
    *b = host[1];
    *a0 = host[2];
    return CHFSI_OK;
}
