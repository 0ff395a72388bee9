// Fused CSR filter step in two-float arithmetic (Algorithm 1 step 1, Sec. 3.4):
//
//     Y_out = alpha (H Y_cur - c Y_cur) - beta Y_prev
//
// with every value held as an unevaluated sum hi + lo of two FP32 numbers
// (|lo| <= ulp(hi)/2, about 48 significant bits) and every operation done on the
// FP32 pipe with error-free transformations: the exact product error of
// hi*hi comes from one FMA (TwoProduct), sums use Knuth's TwoSum (Dekker 1971;
// Knuth, TAOCP vol. 2, 4.2.2).  GB300 runs 64 FP32 operations per FP64 one, so
// the 12 FP32 operations of a two-float multiply-add (6 packed FP32x2 instructions
// per state, two states per instruction) still run several times faster than the
// FP64 DFMA pipe, at FP64-level accuracy for the filter.
//
// Layout and staging follow the FP64 CSR step: one CTA per 8 consecutive rows,
// the CTA's CSR slice (hi/lo value pairs and column indices) staged once in
// shared memory by cp.async and reused for every column chunk; a lane owns two
// consecutive states, and the iterate blocks are in the pair-split layout (the 16
// bytes of states 2t, 2t+1 hold {hi, hi', lo, lo'}), so one 16-byte load per
// gathered row gives both register pairs of the packed FP32x2 multiply-add.
// Column indices are range-checked while staging.  The packed instructions are
// inline PTX with explicit rounding (add/sub/mul/fma.rn.f32x2), which the compiler
// cannot contract, so the error-free transformations stay exact.
#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"
#include "twofloat.cuh"

namespace chfsi {

namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kCapMax = 6144;       // staged entries per CTA (8 rows x up to 768 entries)
constexpr int kRenorm = 8;          // renormalise the accumulator every kRenorm terms

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
}

// Y blocks row-major in the pair-split layout with leading dimension ld (in elements,
// even).  Each lane owns 2 consecutive states (one float4); U chunks per pass.
template <int U>
__global__ void __launch_bounds__(kThreads, (U >= 4 ? 2 : 3))
csr_step_f32x2_kernel(int64_t N, const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                      const float2* __restrict__ val, int64_t nnz, int64_t n, const float2* __restrict__ Yc,
                      int64_t ldc, const float2* __restrict__ Yp, int64_t ldp, float2* __restrict__ Yo, int64_t ldo,
                      double alpha, double c, double beta, int cap, unsigned* status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* s_val = reinterpret_cast<float2*>(smem_raw);
    int32_t* s_col = reinterpret_cast<int32_t*>(smem_raw + sizeof(float2) * (size_t)cap);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r0 = (int64_t)blockIdx.x * kWarps;
    const int64_t r_end = (r0 + kWarps < N) ? r0 + kWarps : N;
    auto clampp = [&](int64_t p) { return p < 0 ? (int64_t)0 : (p > nnz ? nnz : p); };
    const int64_t p_lo = clampp(row_ptr[r0]);
    const int64_t p_hi = clampp(row_ptr[r_end]);
    const int64_t cnt = p_hi > p_lo ? p_hi - p_lo : 0;
    const bool staged = cnt <= cap;
    bool bad = false;
    if (staged) {
        for (int64_t q = threadIdx.x; q < cnt; q += kThreads) {
            cp_async8(s_val + q, val + p_lo + q);
            cp_async4(s_col + q, col + p_lo + q);
        }
        asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
        __syncthreads();
        for (int64_t q = threadIdx.x; q < cnt; q += kThreads) {
            if (s_col[q] < 0 || (int64_t)s_col[q] >= N) {
                s_col[q] = 0;
                s_val[q] = make_float2(0.f, 0.f);
                bad = true;
            }
        }
        __syncthreads();
    }

    const DF A = df_from_double(alpha), Cs = df_from_double(c), B = df_from_double(beta);
    const int64_t r = r0 + warp;
    if (r < r_end) {
        int64_t rb = clampp(row_ptr[r]), re = clampp(row_ptr[r + 1]);
        if (re < rb) { re = rb; bad = true; }
        if (rb < p_lo || re > p_hi) { rb = re = p_lo; bad = true; }
        const float2* hv = staged ? s_val + (rb - p_lo) : val + rb;
        const int32_t* hc = staged ? s_col + (rb - p_lo) : col + rb;
        const int len = (int)(re - rb);
        bool nonfinite = false;

        for (int64_t jbase = 0; jbase < n; jbase += 64 * U) {
            // Packed accumulators: lane 0 of sh2[u]/sl2[u] is state j0 + 64 u, lane 1 the next.
            F2 sh2[U], sl2[U];
            bool on[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                on[u] = jbase + (int64_t)(u * 32 + lane) * 2 < n;
                sh2[u] = sl2[u] = 0ull;
            }
            const int64_t j0 = jbase + (int64_t)lane * 2;
            // Register pipeline with two alternating buffers: the gathers of entry q+1
            // are in flight while entry q is accumulated (no register copies).  The
            // common case -- a staged row slice and a full chunk -- is compiled as its own
            // loop with no per-entry checks; otherwise a bad column index (unstaged rows
            // only) becomes a zero entry on row 0 and chunks past n read zeros.
            const bool full = jbase + 64 * U <= n;
            auto pass = [&](auto fast_tag) {
                constexpr bool kFast = decltype(fast_tag)::value;
                auto fetch = [&](int q, float4 (&y)[U], float2& h) {
                    int32_t cj = hc[q];
                    h = hv[q];
                    if (!kFast && !staged && (cj < 0 || (int64_t)cj >= N)) {
                        bad = true;
                        cj = 0;
                        h = make_float2(0.f, 0.f);
                    }
                    const float2* src = Yc + (int64_t)cj * ldc + j0;
#pragma unroll
                    for (int u = 0; u < U; u++)
                        y[u] = (kFast || on[u]) ? __ldg(reinterpret_cast<const float4*>(src + u * 64))
                                                : make_float4(0.f, 0.f, 0.f, 0.f);
                };
                auto accumulate = [&](const float4 (&y)[U], float2 h) {
                    const F2 hh2 = pk2(h.x, h.x), nhh2 = hh2 ^ 0x8000000080000000ull, hl2 = pk2(h.y, h.y);
#pragma unroll
                    for (int u = 0; u < U; u++)
                        df_madd2(hh2, nhh2, hl2, pk2(y[u].x, y[u].y), pk2(y[u].z, y[u].w), sh2[u], sl2[u]);
                };
                auto renorm = [&]() {
#pragma unroll
                    for (int u = 0; u < U; u++) fast_norm2(sh2[u], sl2[u]);
                };
                float4 ya[U], yb[U];
                float2 ha = make_float2(0.f, 0.f), hb = make_float2(0.f, 0.f);
                if (len > 0) fetch(0, ya, ha);
                int q = 0;
                for (; q + 1 < len; q += 2) {
                    fetch(q + 1, yb, hb);
                    accumulate(ya, ha);
                    if (q + 2 < len) fetch(q + 2, ya, ha);
                    accumulate(yb, hb);
                    if ((q & (kRenorm - 1)) == kRenorm - 2) renorm();
                }
                if (q < len) accumulate(ya, ha);
            };
            if (staged && full) pass(std::true_type{});
            else pass(std::false_type{});
#pragma unroll
            for (int u = 0; u < U; u++) {
                if (!on[u]) continue;
                const int64_t j = j0 + u * 64;
                const float4 yc = *reinterpret_cast<const float4*>(Yc + r * ldc + j);
                float4 yp = make_float4(0.f, 0.f, 0.f, 0.f);
                if (Yp) yp = *reinterpret_cast<const float4*>(Yp + r * ldp + j);
                float sh[2], sl[2];
                upk2(sh2[u], sh[0], sh[1]);
                upk2(sl2[u], sl[0], sl[1]);
                DF o[2];
#pragma unroll
                for (int v = 0; v < 2; v++) {
                    const DF acc{sh[v], sl[v]};
                    const DF ycur = v == 0 ? DF{yc.x, yc.z} : DF{yc.y, yc.w};
                    DF t = df_add(acc, df_neg(df_mul(Cs, ycur)));
                    t = df_mul(A, t);
                    if (Yp) {
                        const DF yprev = v == 0 ? DF{yp.x, yp.z} : DF{yp.y, yp.w};
                        t = df_add(t, df_neg(df_mul(B, yprev)));
                    }
                    nonfinite |= !isfinite(t.hi);
                    o[v] = t;
                }
                *reinterpret_cast<float4*>(Yo + r * ldo + j) = make_float4(o[0].hi, o[1].hi, o[0].lo, o[1].lo);
            }
        }
        if (__any_sync(0xffffffffu, nonfinite) && lane == 0) raise_status(status, DEV_NONFINITE);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) raise_status(status, DEV_PATTERN);
}

// Element (i, j) of a two-float block: {hi, lo} at [i*ld + j] (pair layout), or, in
// the pair-split layout, hi at float 2 (i*ld + (j & ~1)) + (j & 1) and lo two floats on.
__device__ __forceinline__ int64_t split_hi_index(int64_t i, int64_t ld, int64_t j) {
    return 2 * (i * ld + (j & ~(int64_t)1)) + (j & 1);
}

__global__ void to_f32x2_kernel(const double* __restrict__ src, int64_t lds, float2* dst, int64_t ldd, int64_t rows,
                                int64_t n, bool split) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * ldd) return;
    const int64_t i = idx / ldd, j = idx % ldd;
    DF v{0.f, 0.f};
    if (j < n) v = df_from_double(src[i * lds + j]);
    if (split) {
        float* f = reinterpret_cast<float*>(dst) + split_hi_index(i, ldd, j);
        f[0] = v.hi;
        f[2] = v.lo;
    } else {
        dst[idx] = make_float2(v.hi, v.lo);
    }
}

__global__ void from_f32x2_kernel(const float2* __restrict__ src, int64_t lds, double* dst, int64_t ldd, int64_t rows,
                                  int64_t n, bool split) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * n) return;
    const int64_t i = idx / n, j = idx % n;
    float2 v;
    if (split) {
        const float* f = reinterpret_cast<const float*>(src) + split_hi_index(i, lds, j);
        v = make_float2(f[0], f[2]);
    } else {
        v = src[i * lds + j];
    }
    dst[i * ldd + j] = (double)v.x + (double)v.y;
}

}  // namespace

int to_f32x2(const double* src, int64_t lds, void* dst, int64_t ldd, int64_t rows, int64_t n, bool split,
             cudaStream_t s) {
    const int64_t total = rows * ldd;
    if (total <= 0) return CHFSI_OK;
    if (split && (ldd % 2)) return CHFSI_ERR_UNSUPPORTED;
    to_f32x2_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(src, lds, static_cast<float2*>(dst), ldd, rows,
                                                                    n, split);
    CHFSI_LAUNCH_CHECK();
    return CHFSI_OK;
}

int from_f32x2(const void* src, int64_t lds, double* dst, int64_t ldd, int64_t rows, int64_t n, bool split,
               cudaStream_t s) {
    const int64_t total = rows * n;
    if (total <= 0) return CHFSI_OK;
    if (split && (lds % 2)) return CHFSI_ERR_UNSUPPORTED;
    from_f32x2_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(static_cast<const float2*>(src), lds, dst, ldd,
                                                                      rows, n, split);
    CHFSI_LAUNCH_CHECK();
    return CHFSI_OK;
}

int csr_step_f32x2(const CsrDev& h, int64_t n, const void* Yc, int64_t ldc, const void* Yp, int64_t ldp, void* Yo,
                   int64_t ldo, double alpha, double c, double beta, unsigned* status, cudaStream_t s) {
    if (n <= 0 || h.N <= 0) return CHFSI_OK;
    if (h.val_t != Buf::F32X2 || (ldc % 2) || (ldp % 2) || (ldo % 2)) return CHFSI_ERR_UNSUPPORTED;
    // stage 8 rows of a typical length (1.25 x the mean, so that several CTAs fit per SM);
    // longer row blocks read their entries from global memory instead
    const int64_t mean = (h.nnz + h.N - 1) / h.N;
    int64_t cap = (kWarps * mean * 5 / 4 + 127) / 128 * 128;
    if (cap < 256) cap = 256;
    if (cap > kCapMax) cap = kCapMax;
    const size_t smem = (sizeof(float2) + sizeof(int32_t)) * (size_t)cap;
    static bool attr[kMaxDevices] = {};
    const int dev = current_device();
    if (dev < 0) return CHFSI_ERR_CUDA;
    if (!attr[dev]) {
        CHFSI_CUDA_TRY(cudaFuncSetAttribute(csr_step_f32x2_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)((sizeof(float2) + sizeof(int32_t)) * kCapMax)));
        CHFSI_CUDA_TRY(cudaFuncSetAttribute(csr_step_f32x2_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)((sizeof(float2) + sizeof(int32_t)) * kCapMax)));
        attr[dev] = true;
    }
    const int64_t blocks = (h.N + kWarps - 1) / kWarps;
    // 4 chunks of 64 states per pass when n fills them, else 2
    if (n >= 256)
        csr_step_f32x2_kernel<4><<<(unsigned)blocks, kThreads, smem, s>>>(
            h.N, h.row_ptr, h.col, static_cast<const float2*>(h.val), h.nnz, n, static_cast<const float2*>(Yc), ldc,
            static_cast<const float2*>(Yp), ldp, static_cast<float2*>(Yo), ldo, alpha, c, beta, (int)cap, status);
    else
        csr_step_f32x2_kernel<2><<<(unsigned)blocks, kThreads, smem, s>>>(
            h.N, h.row_ptr, h.col, static_cast<const float2*>(h.val), h.nnz, n, static_cast<const float2*>(Yc), ldc,
            static_cast<const float2*>(Yp), ldp, static_cast<float2*>(Yo), ldo, alpha, c, beta, (int)cap, status);
    CHFSI_LAUNCH_CHECK();
    return CHFSI_OK;
}

}  // namespace chfsi
