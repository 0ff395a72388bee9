// Sampled dense-dense product of the filter's adjoint: for every stored entry p
// of H (row r, column q),
//     dH[p] += alpha_k * <Ybar_k[r, :], Y_{k-1}[q, :]>
// which is the H-gradient of step k of Algorithm 1 (Sec. 3.4) written as
// Y_k = alpha_k (H - c) Y_{k-1} - beta_k Y_{k-2}.  One warp per row: the lanes
// split the columns and take the row's entries four at a time, so each load of
// Ybar_k[r, :] serves four dot products.  The four partial sums are reduced across
// the warp by a fixed transposed shuffle tree (lanes trade halves of their sums at
// the first two levels, then reduce one sum), 6 shuffle-adds per four entries
// instead of 20; every dH[p] is owned by one warp (no atomics) and the result is
// reproducible.
#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"

namespace chfsi {

namespace {

constexpr int kWarps = 8;

constexpr int kGroup = 4;   // entries per pass

// Sum of v over the 32 lanes for entry (lane >> 3) of a group of four, given each
// lane's partial sums v[0..3]: at xor 16 a lane keeps two of its sums and adds its
// partner's matching two, at xor 8 one, then a plain tree over the last 8 lanes.
// Lanes 0, 8, 16 and 24 end with the totals of entries 0, 1, 2 and 3.
template <typename T, typename Add, typename Shfl>
__device__ __forceinline__ T transpose_reduce4(const T (&v)[kGroup], int lane, Add add, Shfl shfl) {
    const bool b4 = lane & 16, b3 = lane & 8;
    const T keep0 = b4 ? v[2] : v[0], keep1 = b4 ? v[3] : v[1];
    const T send0 = b4 ? v[0] : v[2], send1 = b4 ? v[1] : v[3];
    const T t0 = add(keep0, shfl(send0, 16)), t1 = add(keep1, shfl(send1, 16));
    T u = add(b3 ? t1 : t0, shfl(b3 ? t0 : t1, 8));
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) u = add(u, shfl(u, o));
    return u;
}

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
    for (int64_t pb = b; pb < e; pb += kGroup) {
        const double* yp[kGroup];
        bool ok[kGroup];
#pragma unroll
        for (int g = 0; g < kGroup; g++) {
            const int64_t p = pb + g;
            const int32_t q = p < e ? col[p] : -1;
            ok[g] = q >= 0 && (int64_t)q < N;
            yp[g] = Yp + (ok[g] ? (int64_t)q : 0) * ldp;
        }
        double s[kGroup] = {0.0, 0.0, 0.0, 0.0};
        if constexpr (V == 2) {
            for (int64_t j = (int64_t)lane * 2; j < n; j += 64) {
                const double2 x = __ldg(reinterpret_cast<const double2*>(yb + j));
#pragma unroll
                for (int g = 0; g < kGroup; g++) {
                    if (!ok[g]) continue;
                    const double2 y = __ldg(reinterpret_cast<const double2*>(yp[g] + j));
                    s[g] = fma(x.x, y.x, s[g]);
                    s[g] = fma(x.y, y.y, s[g]);
                }
            }
        } else {
            for (int64_t j = lane; j < n; j += 32) {
                const double x = __ldg(yb + j);
#pragma unroll
                for (int g = 0; g < kGroup; g++)
                    if (ok[g]) s[g] = fma(x, __ldg(yp[g] + j), s[g]);
            }
        }
        const double tot = transpose_reduce4(
            s, lane, [](double x, double y) { return x + y; },
            [](double x, int o) { return __shfl_xor_sync(0xffffffffu, x, o); });
        const int64_t p = pb + (lane >> 3);
        if ((lane & 7) == 0 && p < e) dH[p] = fma(alpha, tot, dH[p]);
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
// (even and odd states in the two lanes), four entries per pass as in sddmm_kernel, the
// transposed shuffle tree on two-float sums, and one FP64 multiply-add into dH[p] per
// entry (one warp per row, no atomics).
__global__ void __launch_bounds__(256, 2)
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
    constexpr unsigned long long kSigns = 0x8000000080000000ull;   // negates both lanes (ALU, not FMA)
    for (int64_t pb = b; pb < e; pb += kGroup) {
        const float2* yp[kGroup];
        bool ok[kGroup];
#pragma unroll
        for (int g = 0; g < kGroup; g++) {
            const int64_t p = pb + g;
            const int32_t q = p < e ? col[p] : -1;
            ok[g] = q >= 0 && (int64_t)q < N;
            yp[g] = Yp + (ok[g] ? (int64_t)q : 0) * ldp;
        }
        F2 sh2[kGroup], sl2[kGroup];
#pragma unroll
        for (int g = 0; g < kGroup; g++) sh2[g] = sl2[g] = 0ull;
        // A group of four valid entries (the common case) runs a loop without per-entry
        // checks.
        auto pass = [&](auto all_tag) {
            constexpr bool kAll = decltype(all_tag)::value;
            int t = 0;
            for (int64_t j = (int64_t)lane * 2; j < n; j += 64) {
                const float4 x = __ldg(reinterpret_cast<const float4*>(yb + j));
                float4 y[kGroup];
#pragma unroll
                for (int g = 0; g < kGroup; g++)
                    y[g] = (kAll || ok[g]) ? __ldg(reinterpret_cast<const float4*>(yp[g] + j))
                                           : make_float4(0.f, 0.f, 0.f, 0.f);
                const F2 xh2 = pk2(x.x, x.y), nxh2 = xh2 ^ kSigns, xl2 = pk2(x.z, x.w);
#pragma unroll
                for (int g = 0; g < kGroup; g++)
                    df_madd2(xh2, nxh2, xl2, pk2(y[g].x, y[g].y), pk2(y[g].z, y[g].w), sh2[g], sl2[g]);
                if ((++t & (kRenorm - 1)) == 0) {
#pragma unroll
                    for (int g = 0; g < kGroup; g++) fast_norm2(sh2[g], sl2[g]);
                }
            }
        };
        if (ok[0] && ok[1] && ok[2] && ok[3]) pass(std::true_type{});
        else pass(std::false_type{});
        DF v[kGroup];
#pragma unroll
        for (int g = 0; g < kGroup; g++) {
            fast_norm2(sh2[g], sl2[g]);
            float h0, h1, l0, l1;
            upk2(sh2[g], h0, h1);
            upk2(sl2[g], l0, l1);
            v[g] = df_add(DF{h0, l0}, DF{h1, l1});
        }
        const DF tot = transpose_reduce4(
            v, lane, [](DF x, DF y) { return df_add(x, y); },
            [](DF x, int o) {
                return DF{__shfl_xor_sync(0xffffffffu, x.hi, o), __shfl_xor_sync(0xffffffffu, x.lo, o)};
            });
        const int64_t p = pb + (lane >> 3);
        if ((lane & 7) == 0 && p < e) dH[p] = fma(alpha, (double)tot.hi + (double)tot.lo, dH[p]);
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
