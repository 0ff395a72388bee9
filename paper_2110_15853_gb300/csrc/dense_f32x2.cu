// Dense products of the ChFSI closure (Algorithm 1 steps 2-5, Sec. 3.4) in
// two-float arithmetic on the FP32 pipe: Gram / projection products A^T B with a
// split-K reduction over the long dimension N (partials in FP64, summed in a fixed
// order), and products with an n x n matrix (X_F = Y R^-1, Psi = X_F Q).
//
// Same tiling as the FP64 kernels (64 x 64 output tile, 256 threads, 4 x 4 outputs
// per thread, 16-deep shared-memory chunks).  The products run on the packed FP32
// instructions (two lanes per instruction): a thread owns the column pairs
// (32 P + 2 tx, 32 P + 2 tx + 1), P = 0, 1, one register pair each, so a two-float
// multiply-add of two outputs is 12 packed instructions.  Shared memory holds the
// operands already in packed form -- B as {hi, hi', lo, lo'} for a column pair (the
// pair-split layout of the iterate blocks), A as {hi, hi, -hi, -hi} and {lo, lo} --
// so that no register shuffling is needed.
#include "common.cuh"
#include "kernels.cuh"
#include "twofloat.cuh"

namespace chfsi {

namespace {

constexpr int TB = 64;
constexpr int BK = 16;
constexpr int kRenorm = 8;

enum class Out { Part, F64, F32X2 };

// Element (i, j) of a two-float block with leading dimension ld: pair-split layout
// (hi at float 2 (i ld + (j & ~1)) + (j & 1), lo two floats on) or pair layout.
__device__ __forceinline__ float2 load_el(const float2* P, int64_t ld, int64_t i, int64_t j, bool split) {
    if (!split) return P[i * ld + j];
    const float* f = reinterpret_cast<const float*>(P) + 2 * (i * ld + (j & ~(int64_t)1)) + (j & 1);
    return make_float2(f[0], f[2]);
}

struct Gemm2Args {
    const float2* A; int64_t lda; bool a_t;   // pair-split; a_t: A stored K x M (element (i,k) at row k)
    const float2* B; int64_t ldb; bool b_split;  // B stored K x Nc
    void* C; int64_t ldc;                     // FP64 or pair-split two-float output (Out::F64 / Out::F32X2)
    double* part;                             // splits x M x Nc FP64 partials (Out::Part)
    int64_t M, Nc, K;
    bool upper_tiles;                         // only tiles with tile_row <= tile_col
    bool b_upper;                             // B upper triangular
    int splits;
};

template <Out kOut>
__global__ void __launch_bounds__(256) gemm_f32x2_kernel(Gemm2Args g) {
    // As4[k][i] = {hi, hi, -hi, -hi} and Asl[k][i] = {lo, lo} of A(i, k);
    // Bs4[k][P][t] = {hi, hi', lo, lo'} of B(k, 32 P + 2 t) and B(k, 32 P + 2 t + 1).
    __shared__ float4 As4[BK][TB];
    __shared__ float2 Asl[BK][TB];
    __shared__ float4 Bs4[BK][2][16];
    const int bi = blockIdx.y, bj = blockIdx.x, z = blockIdx.z;
    if (g.upper_tiles && bi > bj) return;
    const int64_t i0 = (int64_t)bi * TB, j0 = (int64_t)bj * TB;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;

    int64_t kc = (g.K + g.splits - 1) / g.splits;
    kc = (kc + BK - 1) / BK * BK;
    const int64_t k_begin = (int64_t)z * kc;
    int64_t k_end = k_begin + kc < g.K ? k_begin + kc : g.K;
    if (g.b_upper && k_end > j0 + TB) k_end = j0 + TB;

    // acc[a][P]: row ty + 16 a, columns (32 P + 2 tx, 32 P + 2 tx + 1) in the two lanes
    F2 sh[4][2], sl[4][2];
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int q = 0; q < 2; q++) sh[a][q] = sl[a][q] = 0ull;

    const float2 zero = make_float2(0.f, 0.f);
    for (int64_t k0 = k_begin; k0 < k_end; k0 += BK) {
        for (int e = threadIdx.x; e < BK * TB; e += 256) {
            int kk, ii;
            float2 va = zero;
            if (g.a_t) {
                kk = e / TB; ii = e % TB;
                const int64_t k = k0 + kk, i = i0 + ii;
                if (k < k_end && i < g.M) va = load_el(g.A, g.lda, k, i, true);
            } else {
                ii = e / BK; kk = e % BK;
                const int64_t k = k0 + kk, i = i0 + ii;
                if (k < k_end && i < g.M) va = load_el(g.A, g.lda, i, k, true);
            }
            As4[kk][ii] = make_float4(va.x, va.x, -va.x, -va.x);
            Asl[kk][ii] = make_float2(va.y, va.y);
            const int kb = e / TB, jb = e % TB;
            const int64_t k = k0 + kb, j = j0 + jb;
            const float2 vb = (k < k_end && j < g.Nc) ? load_el(g.B, g.ldb, k, j, g.b_split) : zero;
            float* bp = reinterpret_cast<float*>(&Bs4[kb][jb >> 5][(jb & 31) >> 1]);
            const int h = jb & 1;
            bp[h] = vb.x;
            bp[2 + h] = vb.y;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk++) {
            F2 yh[2], yl[2];
#pragma unroll
            for (int q = 0; q < 2; q++) {
                const float4 b4 = Bs4[kk][q][tx];
                yh[q] = pk2(b4.x, b4.y);
                yl[q] = pk2(b4.z, b4.w);
            }
#pragma unroll
            for (int a = 0; a < 4; a++) {
                const float4 a4 = As4[kk][ty + 16 * a];
                const float2 a2 = Asl[kk][ty + 16 * a];
                const F2 hh2 = pk2(a4.x, a4.y), nhh2 = pk2(a4.z, a4.w), hl2 = pk2(a2.x, a2.y);
#pragma unroll
                for (int q = 0; q < 2; q++) df_madd2(hh2, nhh2, hl2, yh[q], yl[q], sh[a][q], sl[a][q]);
            }
            if ((kk & (kRenorm - 1)) == kRenorm - 1) {
#pragma unroll
                for (int a = 0; a < 4; a++)
#pragma unroll
                    for (int q = 0; q < 2; q++) fast_norm2(sh[a][q], sl[a][q]);
            }
        }
        __syncthreads();
    }

#pragma unroll
    for (int a = 0; a < 4; a++) {
        const int64_t i = i0 + ty + 16 * a;
        if (i >= g.M) continue;
#pragma unroll
        for (int q = 0; q < 2; q++) {
            float hs[2], ls[2];
            upk2(sh[a][q], hs[0], hs[1]);
            upk2(sl[a][q], ls[0], ls[1]);
            const int64_t jp = j0 + 32 * q + 2 * tx;
            DF v[2];
#pragma unroll
            for (int h = 0; h < 2; h++) v[h] = fast_norm(hs[h], ls[h]);
            if constexpr (kOut == Out::F32X2) {
                float* f = static_cast<float*>(g.C) + 2 * (i * g.ldc + jp);
                if (jp + 1 < g.Nc) {
                    *reinterpret_cast<float4*>(f) = make_float4(v[0].hi, v[1].hi, v[0].lo, v[1].lo);
                } else if (jp < g.Nc) {
                    f[0] = v[0].hi;
                    f[2] = v[0].lo;
                }
            } else {
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const int64_t j = jp + h;
                    if (j >= g.Nc) continue;
                    if constexpr (kOut == Out::Part) {
                        g.part[((int64_t)z * g.M + i) * g.Nc + j] = (double)v[h].hi + (double)v[h].lo;
                    } else {
                        static_cast<double*>(g.C)[i * g.ldc + j] = (double)v[h].hi + (double)v[h].lo;
                    }
                }
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
    if ((lda % 2) || (ldb % 2)) return CHFSI_ERR_UNSUPPORTED;
    Gemm2Args g{static_cast<const float2*>(A), lda, true, static_cast<const float2*>(B), ldb, true, nullptr, 0,
                part, n, n, K, symmetric, false, splits};
    int rc = run<Out::Part>(g, s);
    if (rc) return rc;
    reduce_parts2_kernel<<<(unsigned)((n * n + 255) / 256), 256, 0, s>>>(part, splits, n, S, lds, symmetric);
    CHFSI_LAUNCH_CHECK();
    return CHFSI_OK;
}

int gemm_nn_f32x2(const void* A, int64_t lda, const void* B, int64_t ldb, void* C, int64_t ldc, bool c_f64,
                  int64_t M, int64_t n, bool b_upper, cudaStream_t s) {
    if ((lda % 2) || (!c_f64 && (ldc % 2))) return CHFSI_ERR_UNSUPPORTED;
    Gemm2Args g{static_cast<const float2*>(A), lda, false, static_cast<const float2*>(B), ldb, false, C, ldc,
                nullptr, M, n, n, false, b_upper, 1};
    return c_f64 ? run<Out::F64>(g, s) : run<Out::F32X2>(g, s);
}

}  // namespace chfsi
