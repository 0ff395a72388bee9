// Sampled dense-dense product of the filter's adjoint: for every stored entry p
// of H (row r, column q),
//     dH[p] += alpha_k * <Ybar_k[r, :], Y_{k-1}[q, :]>
// which is the H-gradient of step k of Algorithm 1 (Sec. 3.4) written as
// Y_k = alpha_k (H - c) Y_{k-1} - beta_k Y_{k-2}.  One warp per row: the lanes
// split the columns, each entry's dot product is reduced across the warp with a
// fixed shuffle tree, so every dH[p] is owned by one warp (no atomics) and the
// result is reproducible.  Ybar_k[r, :] is re-read per entry from L1.
#include "common.cuh"
#include "kernels.cuh"

namespace chfsi {

namespace {

constexpr int kWarps = 8;

template <int V>
__global__ void __launch_bounds__(kWarps * 32)
sddmm_kernel(int64_t N, const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col, int64_t nnz,
             int64_t n, const double* __restrict__ Yb, int64_t ldb, const double* __restrict__ Yp, int64_t ldp,
             double alpha, double* __restrict__ dH) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * kWarps + warp;
    if (r >= N) return;
    int64_t b = row_ptr[r], e = row_ptr[r + 1];
    if (b < 0) b = 0;
    if (e > nnz) e = nnz;
    const double* yb = Yb + r * ldb;
    for (int64_t p = b; p < e; p++) {
        const int32_t q = col[p];
        double s = 0.0;
        if (q >= 0 && (int64_t)q < N) {
            const double* yp = Yp + (int64_t)q * ldp;
            if constexpr (V == 2) {
                for (int64_t j = (int64_t)lane * 2; j < n; j += 64) {
                    double2 x = __ldg(reinterpret_cast<const double2*>(yb + j));
                    double2 y = __ldg(reinterpret_cast<const double2*>(yp + j));
                    s = fma(x.x, y.x, s);
                    s = fma(x.y, y.y, s);
                }
            } else {
                for (int64_t j = lane; j < n; j += 32) s = fma(__ldg(yb + j), __ldg(yp + j), s);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) dH[p] = fma(alpha, s, dH[p]);
    }
}

}  // namespace

int sddmm_accumulate(const CsrDev& h, int64_t n, const double* Ybar, int64_t ldb, const double* Yprev,
                     int64_t ldp, double alpha, double* dH, cudaStream_t s) {
    if (h.N <= 0 || n <= 0) return CHFSI_OK;
    const unsigned blocks = (unsigned)((h.N + kWarps - 1) / kWarps);
    const bool vec = (n % 2 == 0) && (ldb % 2 == 0) && (ldp % 2 == 0) &&
                     ((reinterpret_cast<uintptr_t>(Ybar) | reinterpret_cast<uintptr_t>(Yprev)) % 16 == 0);
    if (vec)
        sddmm_kernel<2><<<blocks, kWarps * 32, 0, s>>>(h.N, h.row_ptr, h.col, h.nnz, n, Ybar, ldb, Yprev, ldp,
                                                       alpha, dH);
    else
        sddmm_kernel<1><<<blocks, kWarps * 32, 0, s>>>(h.N, h.row_ptr, h.col, h.nnz, n, Ybar, ldb, Yprev, ldp,
                                                       alpha, dH);
    CHFSI_LAUNCH_CHECK();
    return CHFSI_OK;
}

}  // namespace chfsi

// ---------------------------------------------------------------- two-float SDDMM
#include "twofloat.cuh"

namespace chfsi {

namespace {

constexpr int kRenorm = 8;  // renormalise the two-float accumulators every kRenorm terms

// dH[p] += alpha * <Ybar[row p, :], Yprev[col p, :]> with both blocks two-float in the
// pair-split layout: per-lane two-float dot products on the packed FP32x2 instructions
// (even and odd states in the two lanes), a fixed shuffle tree of two-float adds, and
// one FP64 multiply-add into dH[p] per entry (one warp per row, no atomics).
__global__ void __launch_bounds__(256)
sddmm_f32x2_kernel(int64_t N, const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col, int64_t nnz,
                   int64_t n, const float2* __restrict__ Yb, int64_t ldb, const float2* __restrict__ Yp, int64_t ldp,
                   double alpha, double* __restrict__ dH) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * 8 + warp;
    if (r >= N) return;
    int64_t b = row_ptr[r], e = row_ptr[r + 1];
    if (b < 0) b = 0;
    if (e > nnz) e = nnz;
    const float2* yb = Yb + r * ldb;
    for (int64_t p = b; p < e; p++) {
        const int32_t q = col[p];
        F2 sh2 = 0ull, sl2 = 0ull;
        if (q >= 0 && (int64_t)q < N) {
            const float2* yp = Yp + (int64_t)q * ldp;
            const F2 minus1 = pk2(-1.f, -1.f);
            int t = 0;
            for (int64_t j = (int64_t)lane * 2; j < n; j += 64) {
                const float4 x = __ldg(reinterpret_cast<const float4*>(yb + j));
                const float4 y = __ldg(reinterpret_cast<const float4*>(yp + j));
                const F2 xh2 = pk2(x.x, x.y);
                df_madd2(xh2, mul2(xh2, minus1), pk2(x.z, x.w), pk2(y.x, y.y), pk2(y.z, y.w), sh2, sl2);
                if ((++t & (kRenorm - 1)) == 0) fast_norm2(sh2, sl2);
            }
        }
        fast_norm2(sh2, sl2);
        float h0, h1, l0, l1;
        upk2(sh2, h0, h1);
        upk2(sl2, l0, l1);
        DF acc = df_add(DF{h0, l0}, DF{h1, l1});
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            DF other;
            other.hi = __shfl_xor_sync(0xffffffffu, acc.hi, o);
            other.lo = __shfl_xor_sync(0xffffffffu, acc.lo, o);
            acc = df_add(acc, other);
        }
        if (lane == 0) dH[p] = fma(alpha, (double)acc.hi + (double)acc.lo, dH[p]);
    }
}

}  // namespace

int sddmm_accumulate_f32x2(const CsrDev& h, int64_t n, const void* Ybar, int64_t ldb, const void* Yprev,
                           int64_t ldp, double alpha, double* dH, cudaStream_t s) {
    if (h.N <= 0 || n <= 0) return CHFSI_OK;
    if ((ldb % 2) || (ldp % 2)) return CHFSI_ERR_UNSUPPORTED;
    sddmm_f32x2_kernel<<<(unsigned)((h.N + 7) / 8), 256, 0, s>>>(h.N, h.row_ptr, h.col, h.nnz, n,
                                                                  static_cast<const float2*>(Ybar), ldb,
                                                                  static_cast<const float2*>(Yprev), ldp, alpha, dH);
    CHFSI_LAUNCH_CHECK();
    return CHFSI_OK;
}

}  // namespace chfsi
