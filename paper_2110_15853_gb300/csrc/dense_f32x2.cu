// Dense products of the ChFSI closure (Algorithm 1 steps 2-5, Sec. 3.4) in
// two-float arithmetic on the FP32 pipe: Gram / projection products A^T B with a
// split-K reduction over the long dimension N (partials in FP64, summed in a fixed
// order), and products with an n x n matrix (X_F = Y R^-1, Psi = X_F Q).
//
// Same tiling as the FP64 kernels (64 x 64 output tile, 256 threads, 4 x 4 outputs
// per thread with stride-16 ownership, 16-deep shared-memory chunks), with hi/lo
// pairs in shared memory.  Each multiply-add is about 12 FP32 operations, and with
// 8 pair loads per 16 multiply-adds the kernel is bound by the FP32 pipe.
#include "common.cuh"
#include "kernels.cuh"
#include "twofloat.cuh"

namespace chfsi {

namespace {

constexpr int TB = 64;
constexpr int BK = 16;
constexpr int kRenorm = 8;

enum class Out { Part, F64, F32X2 };

struct Gemm2Args {
    const float2* A; int64_t lda; bool a_t;   // a_t: A stored K x M (element (i,k) = A[k*lda+i])
    const float2* B; int64_t ldb;             // B stored K x Nc
    void* C; int64_t ldc;                     // double or float2 output (Out::F64 / Out::F32X2)
    double* part;                             // splits x M x Nc FP64 partials (Out::Part)
    int64_t M, Nc, K;
    bool upper_tiles;                         // only tiles with tile_row <= tile_col
    bool b_upper;                             // B upper triangular
    int splits;
};

template <Out kOut>
__global__ void __launch_bounds__(256) gemm_f32x2_kernel(Gemm2Args g) {
    __shared__ float2 As[BK][TB + 1];
    __shared__ float2 Bs[BK][TB];
    const int bi = blockIdx.y, bj = blockIdx.x, z = blockIdx.z;
    if (g.upper_tiles && bi > bj) return;
    const int64_t i0 = (int64_t)bi * TB, j0 = (int64_t)bj * TB;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;

    int64_t kc = (g.K + g.splits - 1) / g.splits;
    kc = (kc + BK - 1) / BK * BK;
    const int64_t k_begin = (int64_t)z * kc;
    int64_t k_end = k_begin + kc < g.K ? k_begin + kc : g.K;
    if (g.b_upper && k_end > j0 + TB) k_end = j0 + TB;

    float sh[4][4], sl[4][4];
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 4; b++) sh[a][b] = sl[a][b] = 0.f;

    const float2 zero = make_float2(0.f, 0.f);
    for (int64_t k0 = k_begin; k0 < k_end; k0 += BK) {
        for (int e = threadIdx.x; e < BK * TB; e += 256) {
            int kk, ii;
            float2 va = zero;
            if (g.a_t) {
                kk = e / TB; ii = e % TB;
                const int64_t k = k0 + kk, i = i0 + ii;
                if (k < k_end && i < g.M) va = g.A[k * g.lda + i];
            } else {
                ii = e / BK; kk = e % BK;
                const int64_t k = k0 + kk, i = i0 + ii;
                if (k < k_end && i < g.M) va = g.A[i * g.lda + k];
            }
            As[kk][ii] = va;
            const int kb = e / TB, jb = e % TB;
            const int64_t k = k0 + kb, j = j0 + jb;
            Bs[kb][jb] = (k < k_end && j < g.Nc) ? g.B[k * g.ldb + j] : zero;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk++) {
            float2 av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; a++) av[a] = As[kk][ty + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; b++) bv[b] = Bs[kk][tx + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; a++)
#pragma unroll
                for (int b = 0; b < 4; b++) df_madd(av[a].x, av[a].y, bv[b].x, bv[b].y, sh[a][b], sl[a][b]);
            if ((kk & (kRenorm - 1)) == kRenorm - 1) {
#pragma unroll
                for (int a = 0; a < 4; a++)
#pragma unroll
                    for (int b = 0; b < 4; b++) {
                        const DF t = fast_norm(sh[a][b], sl[a][b]);
                        sh[a][b] = t.hi;
                        sl[a][b] = t.lo;
                    }
            }
        }
        __syncthreads();
    }

#pragma unroll
    for (int a = 0; a < 4; a++) {
        const int64_t i = i0 + ty + 16 * a;
        if (i >= g.M) continue;
#pragma unroll
        for (int b = 0; b < 4; b++) {
            const int64_t j = j0 + tx + 16 * b;
            if (j >= g.Nc) continue;
            const DF v = fast_norm(sh[a][b], sl[a][b]);
            if constexpr (kOut == Out::Part) {
                g.part[((int64_t)z * g.M + i) * g.Nc + j] = (double)v.hi + (double)v.lo;
            } else if constexpr (kOut == Out::F64) {
                static_cast<double*>(g.C)[i * g.ldc + j] = (double)v.hi + (double)v.lo;
            } else {
                static_cast<float2*>(g.C)[i * g.ldc + j] = make_float2(v.hi, v.lo);
            }
        }
    }
}

template <Out kOut>
int run(const Gemm2Args& g, cudaStream_t s) {
    if (g.M <= 0 || g.Nc <= 0) return CHFSI_OK;
    dim3 grid((unsigned)((g.Nc + TB - 1) / TB), (unsigned)((g.M + TB - 1) / TB), (unsigned)g.splits);
    gemm_f32x2_kernel<kOut><<<grid, 256, 0, s>>>(g);
    CHFSI_LAUNCH_CHECK();
    return CHFSI_OK;
}

// C[i][j] = sum_z part[z][i][j] (fixed order); mirrored below the diagonal tiles.
__global__ void reduce_parts2_kernel(const double* __restrict__ part, int splits, int64_t n, double* C,
                                     int64_t ldc, bool mirror) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * n) return;
    const int64_t i = idx / n, j = idx % n;
    int64_t si = i, sj = j;
    if (mirror && (i / TB) > (j / TB)) { si = j; sj = i; }
    double s = 0.0;
    for (int z = 0; z < splits; z++) s += part[((int64_t)z * n + si) * n + sj];
    C[i * ldc + j] = s;
}

}  // namespace

int gemm_tn_f32x2(const void* A, int64_t lda, const void* B, int64_t ldb, int64_t K, int64_t n, double* S,
                  int64_t lds, bool symmetric, double* part, int splits, cudaStream_t s) {
    if (n <= 0) return CHFSI_OK;
    Gemm2Args g{static_cast<const float2*>(A), lda, true, static_cast<const float2*>(B), ldb, nullptr, 0, part,
                n, n, K, symmetric, false, splits};
    int rc = run<Out::Part>(g, s);
    if (rc) return rc;
    reduce_parts2_kernel<<<(unsigned)((n * n + 255) / 256), 256, 0, s>>>(part, splits, n, S, lds, symmetric);
    CHFSI_LAUNCH_CHECK();
    return CHFSI_OK;
}

int gemm_nn_f32x2(const void* A, int64_t lda, const void* B, int64_t ldb, void* C, int64_t ldc, bool c_f64,
                  int64_t M, int64_t n, bool b_upper, cudaStream_t s) {
    Gemm2Args g{static_cast<const float2*>(A), lda, false, static_cast<const float2*>(B), ldb, C, ldc, nullptr,
                M, n, n, false, b_upper, 1};
    return c_f64 ? run<Out::F64>(g, s) : run<Out::F32X2>(g, s);
}

}  // namespace chfsi
