// Dense FP64 kernels of the ChFSI closure (Algorithm 1 steps 2-5, Sec. 3.4):
// Gram / projection products A^T B with a deterministic split-K reduction over
// the long dimension N, the product with an n x n matrix (X_F = Y R^-1,
// Psi = X_F Q), a blocked right-looking Cholesky S = R^T R, the inverse of the
// upper-triangular factor, and small element-wise helpers.
//
// FP64 on this part runs on the DFMA pipe (about 1.2 TFLOP/s for the whole GPU),
// so the tiles are sized for DFMA issue, not for bandwidth: 64 x 64 output tiles,
// 256 threads, 4 x 4 outputs per thread with stride-16 row/column ownership so
// that shared-memory reads are conflict-free and global stores coalesce.
#include "common.cuh"
#include "kernels.cuh"

namespace chfsi {

namespace {

constexpr int TB = 64;   // output tile edge
constexpr int BK = 16;   // reduction chunk

struct GemmArgs {
    const double* A; int64_t lda; bool a_t;   // a_t: A stored K x M, element (i,k) = A[k*lda+i]
    const double* B; int64_t ldb;             // B stored K x Nc, element (k,j) = B[k*ldb+j]
    double* C; int64_t ldc;
    int64_t M, Nc, K;
    double alpha;
    bool accumulate;                          // C = C + alpha*AB (else C = alpha*AB)
    bool upper_tiles;                         // only tiles with tile_row <= tile_col
    bool b_upper;                             // B upper triangular: k <= j
    int splits;
    double* part;                             // splits x M x Nc partials, or nullptr
};

__global__ void __launch_bounds__(256) gemm_kernel(GemmArgs g) {
    __shared__ double As[BK][TB + 1];
    __shared__ double Bs[BK][TB];
    const int bi = blockIdx.y, bj = blockIdx.x, z = blockIdx.z;
    if (g.upper_tiles && bi > bj) return;
    const int64_t i0 = (int64_t)bi * TB, j0 = (int64_t)bj * TB;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;

    int64_t kc = (g.K + g.splits - 1) / g.splits;
    kc = (kc + BK - 1) / BK * BK;
    int64_t k_begin = (int64_t)z * kc;
    int64_t k_end = k_begin + kc < g.K ? k_begin + kc : g.K;
    if (g.b_upper) {
        int64_t lim = j0 + TB;
        if (k_end > lim) k_end = lim;
    }

    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 4; b++) acc[a][b] = 0.0;

    for (int64_t k0 = k_begin; k0 < k_end; k0 += BK) {
        // stage A chunk as As[k][i] and B chunk as Bs[k][j]
        for (int e = threadIdx.x; e < BK * TB; e += 256) {
            int kk, ii;
            double va = 0.0;
            if (g.a_t) {
                kk = e / TB; ii = e % TB;                     // coalesced along i
                int64_t k = k0 + kk, i = i0 + ii;
                if (k < k_end && i < g.M) va = g.A[k * g.lda + i];
            } else {
                ii = e / BK; kk = e % BK;                     // coalesced along k
                int64_t k = k0 + kk, i = i0 + ii;
                if (k < k_end && i < g.M) va = g.A[i * g.lda + k];
            }
            As[kk][ii] = va;
            int kb = e / TB, jb = e % TB;
            int64_t k = k0 + kb, j = j0 + jb;
            Bs[kb][jb] = (k < k_end && j < g.Nc) ? g.B[k * g.ldb + j] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk++) {
            double av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; a++) av[a] = As[kk][ty + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; b++) bv[b] = Bs[kk][tx + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; a++)
#pragma unroll
                for (int b = 0; b < 4; b++) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
        }
        __syncthreads();
    }

#pragma unroll
    for (int a = 0; a < 4; a++) {
        int64_t i = i0 + ty + 16 * a;
        if (i >= g.M) continue;
#pragma unroll
        for (int b = 0; b < 4; b++) {
            int64_t j = j0 + tx + 16 * b;
            if (j >= g.Nc) continue;
            if (g.part) {
                g.part[((int64_t)z * g.M + i) * g.Nc + j] = g.alpha * acc[a][b];
            } else {
                double v = g.alpha * acc[a][b];
                if (g.accumulate) v += g.C[i * g.ldc + j];
                g.C[i * g.ldc + j] = v;
            }
        }
    }
}

// C[i][j] = sum_z part[z][i][j] in split order; with `mirror`, tiles below the
// diagonal take the transposed upper-tile sum.
__global__ void reduce_parts_kernel(const double* __restrict__ part, int splits, int64_t M, int64_t Nc,
                                    double* C, int64_t ldc, bool mirror) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= M * Nc) return;
    int64_t i = idx / Nc, j = idx % Nc;
    int64_t si = i, sj = j;
    if (mirror && (i / TB) > (j / TB)) { si = j; sj = i; }
    double s = 0.0;
    for (int z = 0; z < splits; z++) s += part[((int64_t)z * M + si) * Nc + sj];
    C[i * ldc + j] = s;
}

int run_gemm(const GemmArgs& g, cudaStream_t s) {
    if (g.M <= 0 || g.Nc <= 0) return CHFSI_OK;
    dim3 grid((unsigned)((g.Nc + TB - 1) / TB), (unsigned)((g.M + TB - 1) / TB), (unsigned)g.splits);
    gemm_kernel<<<grid, 256, 0, s>>>(g);
    CHFSI_LAUNCH_CHECK();
    return CHFSI_OK;
}

// ---------------------------------------------------------------- Cholesky

constexpr int NB = 64;

// Unblocked upper Cholesky of the nb x nb diagonal block at S[k0][k0] (in place).
__global__ void __launch_bounds__(256) chol_diag_kernel(double* S, int64_t lds, int64_t k0, int nb,
                                                        unsigned* status) {
    __shared__ double A[NB][NB + 1];
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        int i = e / nb, j = e % nb;
        A[i][j] = S[(k0 + i) * lds + k0 + j];
    }
    __syncthreads();
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int k = 0; k < nb; k++) {
        if (threadIdx.x == 0) {
            double p = A[k][k];
            if (!(p > 0.0) || !isfinite(p)) { bad = 1; p = 1.0; }
            A[k][k] = sqrt(p);
        }
        __syncthreads();
        double d = A[k][k];
        for (int j = k + 1 + threadIdx.x; j < nb; j += blockDim.x) A[k][j] /= d;
        __syncthreads();
        const int m = nb - k - 1;
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            int i = k + 1 + e / m, j = k + 1 + e % m;
            if (j >= i) A[i][j] -= A[k][i] * A[k][j];
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        int i = e / nb, j = e % nb;
        S[(k0 + i) * lds + k0 + j] = (j >= i) ? A[i][j] : 0.0;
    }
    if (threadIdx.x == 0 && bad) raise_status(status, DEV_CHOL);
}

// Panel: R[k0:k0+nb, j] = R_kk^-T S[k0:k0+nb, j] for j >= k0+nb (forward substitution).
__global__ void __launch_bounds__(64) chol_panel_kernel(double* S, int64_t lds, int64_t n, int64_t k0,
                                                        int nb) {
    __shared__ double R[NB][NB + 1];
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        int i = e / nb, j = e % nb;
        R[i][j] = S[(k0 + i) * lds + k0 + j];
    }
    __syncthreads();
    int64_t j = k0 + nb + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double z[NB];
#pragma unroll 1
    for (int i = 0; i < nb; i++) {
        double v = S[(k0 + i) * lds + j];
        for (int l = 0; l < i; l++) v -= R[l][i] * z[l];
        z[i] = v / R[i][i];
    }
    for (int i = 0; i < nb; i++) S[(k0 + i) * lds + j] = z[i];
}

__global__ void zero_lower_kernel(double* S, int64_t lds, int64_t n) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * n) return;
    int64_t i = idx / n, j = idx % n;
    if (j < i) S[i * lds + j] = 0.0;
}

// ---------------------------------------------------------------- triangular inverse

// Column j of R^-1 by back substitution, one warp per column:
//   z_j = 1/R_jj,  z_i = -(sum_{l=i+1..j} R_il z_l)/R_ii  for i = j-1..0.
__global__ void tri_inv_kernel(const double* __restrict__ R, int64_t ldr, double* Rinv, int64_t ldi,
                               int64_t n, int warps_per_block) {
    extern __shared__ double zs[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * warps_per_block + warp;
    if (j >= n) return;
    double* z = zs + (int64_t)warp * n;
    for (int64_t i = lane; i <= j; i += 32) z[i] = 0.0;
    __syncwarp();
    if (lane == 0) z[j] = 1.0 / R[j * ldr + j];
    __syncwarp();
    for (int64_t i = j - 1; i >= 0; i--) {
        double s = 0.0;
        for (int64_t l = i + 1 + lane; l <= j; l += 32) s = fma(R[i * ldr + l], z[l], s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) z[i] = -s / R[i * ldr + i];
        __syncwarp();
    }
    for (int64_t i = lane; i < n; i += 32) Rinv[i * ldi + j] = (i <= j) ? z[i] : 0.0;
}

__global__ void transpose_kernel(const double* __restrict__ A, int64_t lda, double* B, int64_t ldb, int64_t n) {
    __shared__ double t[32][33];
    int64_t bx = (int64_t)blockIdx.x * 32, by = (int64_t)blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        int64_t i = by + k, j = bx + threadIdx.x;
        if (i < n && j < n) t[k][threadIdx.x] = A[i * lda + j];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        int64_t i = bx + k, j = by + threadIdx.x;
        if (i < n && j < n) B[i * ldb + j] = t[threadIdx.x][k];
    }
}

__global__ void symmetrize_kernel(double* S, int64_t lds, int64_t n) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * n) return;
    int64_t i = idx / n, j = idx % n;
    if (j <= i) return;
    double v = 0.5 * (S[i * lds + j] + S[j * lds + i]);
    S[i * lds + j] = v;
    S[j * lds + i] = v;
}

// ---------------------------------------------------------------- conversions

template <typename TS, typename TD>
__global__ void convert_kernel(const TS* __restrict__ src, int64_t lds, TD* dst, int64_t ldd, int64_t rows,
                               int64_t n, int64_t width) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * width) return;
    const int64_t i = idx / width, j = idx % width;
    float fv;
    double dv;
    if (j < n) {
        if constexpr (std::is_same<TS, __nv_bfloat16>::value) { fv = __bfloat162float(src[i * lds + j]); dv = fv; }
        else { dv = (double)src[i * lds + j]; fv = (float)src[i * lds + j]; }
    } else {
        dv = 0.0; fv = 0.0f;
    }
    if constexpr (std::is_same<TD, double>::value) dst[i * ldd + j] = dv;
    else if constexpr (std::is_same<TD, float>::value) dst[i * ldd + j] = fv;
    else dst[i * ldd + j] = __float2bfloat16_rn(fv);
}

template <typename TS, typename TD>
int launch_convert(const void* src, int64_t lds, void* dst, int64_t ldd, int64_t rows, int64_t n, int64_t width,
                   cudaStream_t s) {
    int64_t total = rows * width;
    if (total <= 0) return CHFSI_OK;
    convert_kernel<TS, TD><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(
        static_cast<const TS*>(src), lds, static_cast<TD*>(dst), ldd, rows, n, width);
    CHFSI_LAUNCH_CHECK();
    return CHFSI_OK;
}

__global__ void convert_values_kernel(const double* __restrict__ src, float* dst, int64_t count, bool bf) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    float f = (float)src[i];
    if (bf) f = __bfloat162float(__float2bfloat16_rn(f));
    dst[i] = f;
}

}  // namespace

int gemm_tn_splits(int64_t K, int64_t n) {
    int64_t tiles = ((n + TB - 1) / TB);
    tiles = tiles * (tiles + 1) / 2;
    int64_t want = (4 * 152 + tiles - 1) / tiles;        // about four CTAs per SM
    int64_t maxs = (K + 2047) / 2048;                    // keep >= 2048 rows per split
    int64_t s = want < maxs ? want : maxs;
    if (s < 1) s = 1;
    if (s > 64) s = 64;
    return (int)s;
}

int gemm_tn(const double* A, int64_t lda, const double* B, int64_t ldb, int64_t K, int64_t n, double* S,
            int64_t lds, bool symmetric, double* part, int splits, cudaStream_t s) {
    if (n <= 0) return CHFSI_OK;
    GemmArgs g{A, lda, true, B, ldb, S, lds, n, n, K, 1.0, false, symmetric, false, splits, part};
    int rc = run_gemm(g, s);
    if (rc) return rc;
    int64_t total = n * n;
    reduce_parts_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(part, splits, n, n, S, lds, symmetric);
    CHFSI_LAUNCH_CHECK();
    return CHFSI_OK;
}

int gemm_nn(const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc, int64_t M,
            int64_t n, bool b_upper, cudaStream_t s) {
    GemmArgs g{A, lda, false, B, ldb, C, ldc, M, n, n, 1.0, false, false, b_upper, 1, nullptr};
    return run_gemm(g, s);
}

int gemm_general(const double* A, int64_t lda, bool a_t, const double* B, int64_t ldb, double* C, int64_t ldc,
                 int64_t M, int64_t Nc, int64_t K, double alpha, bool accumulate, cudaStream_t s) {
    if (M <= 0 || Nc <= 0) return CHFSI_OK;
    GemmArgs g{A, lda, a_t, B, ldb, C, ldc, M, Nc, K, alpha, accumulate, false, false, 1, nullptr};
    return run_gemm(g, s);
}

namespace {

// Z -= D on the upper triangle of a rows x rows block (D dense, leading dimension rows).
__global__ void sub_upper_kernel(double* Z, int64_t ldz, const double* __restrict__ D, int64_t rows) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * rows) return;
    const int64_t i = idx / rows, c = idx % rows;
    if (c >= i) Z[i * ldz + c] -= D[idx];
}

constexpr int64_t kCholOzakiMin = 256;   // trailing blocks from this size on as Ozaki products

}  // namespace

int cholesky_upper(double* S, int64_t n, int64_t lds, unsigned* status, cudaStream_t s, void* oz_ws, size_t oz_bytes,
                   double* scratch) {
    for (int64_t k0 = 0; k0 < n; k0 += NB) {
        int nb = (int)((n - k0) < NB ? (n - k0) : NB);
        chol_diag_kernel<<<1, 256, 0, s>>>(S, lds, k0, nb, status);
        CHFSI_LAUNCH_CHECK();
        int64_t rest = n - k0 - nb;
        if (rest <= 0) break;
        chol_panel_kernel<<<(unsigned)((rest + 63) / 64), 64, 0, s>>>(S, lds, n, k0, nb);
        CHFSI_LAUNCH_CHECK();
        // trailing update S22 -= R12^T R12 (upper tiles): an Ozaki product on the tensor
        // cores into the scratch block when one is given, else FP64 on the DFMA pipe
        const double* R12 = S + k0 * lds + (k0 + nb);
        double* S22 = S + (k0 + nb) * lds + (k0 + nb);
        int rc;
        if (oz_ws && scratch && rest >= kCholOzakiMin &&
            oz_bytes >= ozaki_workspace_bytes(true, rest, rest, nb, true)) {
            if ((rc = ozaki_gemm_tn(R12, lds, R12, lds, nb, rest, rest, scratch, rest, true, oz_ws, oz_bytes, status,
                                    s)))
                return rc;
            sub_upper_kernel<<<(unsigned)((rest * rest + 255) / 256), 256, 0, s>>>(S22, lds, scratch, rest);
            CHFSI_LAUNCH_CHECK();
            continue;
        }
        GemmArgs g{R12, lds, true, R12, lds, S22, lds, rest, rest, nb, -1.0, true, true, false, 1, nullptr};
        if ((rc = run_gemm(g, s))) return rc;
    }
    int64_t total = n * n;
    zero_lower_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(S, lds, n);
    CHFSI_LAUNCH_CHECK();
    return CHFSI_OK;
}

int tri_inverse_upper(const double* R, int64_t ldr, double* Rinv, int64_t ldi, int64_t n, cudaStream_t s) {
    if (n <= 0) return CHFSI_OK;
    int wpb = (int)((160 * 1024) / (n * 8));
    if (wpb > 8) wpb = 8;
    if (wpb < 1) return CHFSI_ERR_UNSUPPORTED;            // n > 20480
    size_t smem = (size_t)wpb * n * 8;
    if (smem > 48 * 1024)
        CHFSI_CUDA_TRY(cudaFuncSetAttribute(tri_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    tri_inv_kernel<<<(unsigned)((n + wpb - 1) / wpb), 32 * wpb, smem, s>>>(R, ldr, Rinv, ldi, n, wpb);
    CHFSI_LAUNCH_CHECK();
    return CHFSI_OK;
}

namespace {

__global__ void negate_block_kernel(double* X, int64_t ldx, int64_t rows, int64_t cols) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * cols) return;
    X[(idx / cols) * ldx + idx % cols] = -X[(idx / cols) * ldx + idx % cols];
}

constexpr int64_t kTriInvLeaf = 1024;   // the column-per-warp kernel below this size

}  // namespace

// R^-1 of an upper-triangular R by halves: with R = [R11 R12; 0 R22],
// R^-1 = [X11, -X11 R12 X22; 0, X22] (X11 = R11^-1, X22 = R22^-1, both recursively), the
// off-diagonal block from two products (T = R12 X22 into `tmp`, then X11 T) -- Ozaki
// products on the tensor cores when oz_ws is given and the depth fits (<= 8192), FP64
// products otherwise; blocks of at most kTriInvLeaf columns by back substitution.
int tri_inverse_upper_blocked(const double* R, int64_t ldr, double* X, int64_t ldx, int64_t n, double* tmp,
                              int64_t ldt, void* oz_ws, size_t oz_bytes, unsigned* status, cudaStream_t s) {
    if (n <= kTriInvLeaf) return tri_inverse_upper(R, ldr, X, ldx, n, s);
    const int64_t h = (n / 2 + 63) / 64 * 64, r = n - h;
    int rc;
    if ((rc = tri_inverse_upper_blocked(R, ldr, X, ldx, h, tmp, ldt, oz_ws, oz_bytes, status, s))) return rc;
    if ((rc = tri_inverse_upper_blocked(R + h * ldr + h, ldr, X + h * ldx + h, ldx, r, tmp, ldt, oz_ws, oz_bytes, status,
                                        s)))
        return rc;
    CHFSI_CUDA_TRY(cudaMemset2DAsync(X + h * ldx, sizeof(double) * (size_t)ldx, 0, sizeof(double) * (size_t)h,
                                     (size_t)r, s));
    const double* R12 = R + h;
    const double* X22 = X + h * ldx + h;
    double* X12 = X + h;
    if (oz_ws && r <= 8192 && h <= 8192 && oz_bytes >= ozaki_workspace_bytes(false, h, r, r, false)) {
        if ((rc = ozaki_gemm_nn(R12, ldr, X22, ldx, h, r, r, tmp, ldt, true, oz_ws, oz_bytes, status, s))) return rc;
        if ((rc = ozaki_gemm_nn(X, ldx, tmp, ldt, h, h, r, X12, ldx, false, oz_ws, oz_bytes, status, s))) return rc;
        negate_block_kernel<<<(unsigned)((h * r + 255) / 256), 256, 0, s>>>(X12, ldx, h, r);
        CHFSI_LAUNCH_CHECK();
        return CHFSI_OK;
    }
    if ((rc = gemm_general(R12, ldr, false, X22, ldx, tmp, ldt, h, r, r, 1.0, false, s))) return rc;
    return gemm_general(X, ldx, false, tmp, ldt, X12, ldx, h, r, h, -1.0, false, s);
}

int transpose(const double* A, int64_t lda, double* B, int64_t ldb, int64_t n, cudaStream_t s) {
    if (n <= 0) return CHFSI_OK;
    dim3 grid((unsigned)((n + 31) / 32), (unsigned)((n + 31) / 32));
    transpose_kernel<<<grid, dim3(32, 8), 0, s>>>(A, lda, B, ldb, n);
    CHFSI_LAUNCH_CHECK();
    return CHFSI_OK;
}

int symmetrize(double* S, int64_t n, int64_t lds, cudaStream_t s) {
    int64_t total = n * n;
    if (total <= 0) return CHFSI_OK;
    symmetrize_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(S, lds, n);
    CHFSI_LAUNCH_CHECK();
    return CHFSI_OK;
}

int convert_block(const void* src, Buf st, int64_t lds, void* dst, Buf dt, int64_t ldd, int64_t rows, int64_t n,
                  int64_t width, cudaStream_t s) {
    if (width < n || width > ldd) return CHFSI_ERR_ARG;
    if (st == Buf::F64 && dt == Buf::F32) return launch_convert<double, float>(src, lds, dst, ldd, rows, n, width, s);
    if (st == Buf::F64 && dt == Buf::BF16)
        return launch_convert<double, __nv_bfloat16>(src, lds, dst, ldd, rows, n, width, s);
    if (st == Buf::F32 && dt == Buf::F64) return launch_convert<float, double>(src, lds, dst, ldd, rows, n, width, s);
    if (st == Buf::F32 && dt == Buf::BF16)
        return launch_convert<float, __nv_bfloat16>(src, lds, dst, ldd, rows, n, width, s);
    if (st == Buf::F64 && dt == Buf::F64) return launch_convert<double, double>(src, lds, dst, ldd, rows, n, width, s);
    if (st == Buf::F32 && dt == Buf::F32) return launch_convert<float, float>(src, lds, dst, ldd, rows, n, width, s);
    return CHFSI_ERR_UNSUPPORTED;
}

int convert_values(const double* src, void* dst, Buf dt, int64_t count, bool round_bf16, cudaStream_t s) {
    if (dt != Buf::F32) return CHFSI_ERR_UNSUPPORTED;
    if (count <= 0) return CHFSI_OK;
    convert_values_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(src, static_cast<float*>(dst), count,
                                                                          round_bf16);
    CHFSI_LAUNCH_CHECK();
    return CHFSI_OK;
}

int fill_zero(void* p, size_t bytes, cudaStream_t s) {
    if (!bytes) return CHFSI_OK;
    CHFSI_CUDA_TRY(cudaMemsetAsync(p, 0, bytes, s));
    return CHFSI_OK;
}

}  // namespace chfsi
