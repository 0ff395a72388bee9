// Fused CSR filter step (Algorithm 1, step 1, Sec. 3.4):
//
//     Y_out = alpha * (H * Y_cur - c * Y_cur) - beta * Y_prev
//
// (FP64 steps may add a precomputed block Y_add to H * Y_cur: the dense-diagonal-block
// product of the split layout, Sec. 4.1-4.2, with H the off-diagonal part.)
//
// one launch per Chebyshev step, so Y_prev, Y_cur and Y_out each make one HBM pass
// per step (the gathers of H * Y_cur hit L1/L2: the rows a warp gathers are the
// 3-D grid neighbours of its own row).  The same kernel with alpha = 1, c = 0,
// beta = 0 is the plain product H X of the subspace projection (step 3), and with
// (alpha_k, beta_{k+1}) on the adjoint iterates it is the reverse recurrence.
//
// Layout: one CTA owns kWarps consecutive rows (one warp per row).  The CTA's
// slice of the CSR arrays (values and column indices, contiguous because the rows
// are consecutive) is staged once into shared memory with cp.async and reused for
// every column chunk of the row.  Lanes own V consecutive columns (vector loads:
// double2 for FP64, float4 for FP32, 4 x bf16 for the BF16 operand); a chunk is
// 32 * V * U columns.  Accumulation order over a row's entries is the stored order.
// Every column index is range-checked while staging; a bad one is replaced by a
// zero entry and reported in the status word, so no access leaves the buffers.
#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"

namespace chfsi {

namespace {

constexpr int kWarps = 8;            // rows (warps) per CTA
constexpr int kThreads = kWarps * 32;

template <typename A, typename T> __device__ __forceinline__ A cvt(T x);
template <> __device__ __forceinline__ double cvt<double, double>(double x) { return x; }
template <> __device__ __forceinline__ double cvt<double, float>(float x) { return (double)x; }
template <> __device__ __forceinline__ float cvt<float, float>(float x) { return x; }
template <> __device__ __forceinline__ float cvt<float, __nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }

// Read V consecutive elements (aligned to V * sizeof(T)) through the read-only path.
template <typename A, typename T, int V>
__device__ __forceinline__ void ldv(const T* __restrict__ p, A (&o)[V]) {
    if constexpr (std::is_same<T, double>::value && V % 2 == 0) {
#pragma unroll
        for (int i = 0; i < V; i += 2) {
            double2 t = __ldg(reinterpret_cast<const double2*>(p + i));
            o[i] = cvt<A>(t.x); o[i + 1] = cvt<A>(t.y);
        }
    } else if constexpr (std::is_same<T, float>::value && V % 4 == 0) {
#pragma unroll
        for (int i = 0; i < V; i += 4) {
            float4 t = __ldg(reinterpret_cast<const float4*>(p + i));
            o[i] = cvt<A>(t.x); o[i + 1] = cvt<A>(t.y); o[i + 2] = cvt<A>(t.z); o[i + 3] = cvt<A>(t.w);
        }
    } else if constexpr (std::is_same<T, float>::value && V % 2 == 0) {
#pragma unroll
        for (int i = 0; i < V; i += 2) {
            float2 t = __ldg(reinterpret_cast<const float2*>(p + i));
            o[i] = cvt<A>(t.x); o[i + 1] = cvt<A>(t.y);
        }
    } else if constexpr (std::is_same<T, __nv_bfloat16>::value && V % 4 == 0) {
#pragma unroll
        for (int i = 0; i < V; i += 4) {
            uint2 t = __ldg(reinterpret_cast<const uint2*>(p + i));
            __nv_bfloat162 lo = *reinterpret_cast<__nv_bfloat162*>(&t.x);
            __nv_bfloat162 hi = *reinterpret_cast<__nv_bfloat162*>(&t.y);
            float2 a = __bfloat1622float2(lo), b = __bfloat1622float2(hi);
            o[i] = cvt<A>(a.x); o[i + 1] = cvt<A>(a.y); o[i + 2] = cvt<A>(b.x); o[i + 3] = cvt<A>(b.y);
        }
    } else {
#pragma unroll
        for (int i = 0; i < V; i++) o[i] = cvt<A>(p[i]);
    }
}

template <typename A, typename T, int V>
__device__ __forceinline__ void stv(T* p, const A (&v)[V]) {
    if constexpr (std::is_same<T, double>::value && V % 2 == 0) {
#pragma unroll
        for (int i = 0; i < V; i += 2)
            *reinterpret_cast<double2*>(p + i) = make_double2((double)v[i], (double)v[i + 1]);
    } else if constexpr (std::is_same<T, float>::value && V % 4 == 0) {
#pragma unroll
        for (int i = 0; i < V; i += 4)
            *reinterpret_cast<float4*>(p + i) = make_float4((float)v[i], (float)v[i + 1], (float)v[i + 2], (float)v[i + 3]);
    } else if constexpr (std::is_same<T, __nv_bfloat16>::value && V % 4 == 0) {
#pragma unroll
        for (int i = 0; i < V; i += 4) {
            __nv_bfloat162 lo = __floats2bfloat162_rn((float)v[i], (float)v[i + 1]);
            __nv_bfloat162 hi = __floats2bfloat162_rn((float)v[i + 2], (float)v[i + 3]);
            uint2 t;
            t.x = *reinterpret_cast<unsigned*>(&lo);
            t.y = *reinterpret_cast<unsigned*>(&hi);
            *reinterpret_cast<uint2*>(p + i) = t;
        }
    } else {
#pragma unroll
        for (int i = 0; i < V; i++) {
            if constexpr (std::is_same<T, __nv_bfloat16>::value) p[i] = __float2bfloat16_rn((float)v[i]);
            else p[i] = (T)v[i];
        }
    }
}

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Gathered operand of one chunk: converted values, or for the BF16 operand the raw
// bf16 pairs, which the mixed-precision FMA (fma.rn.f32.bf16: BF16 x BF16 product,
// FP32 addend) consumes without a conversion instruction.
template <typename ACC, typename TG, int V>
struct Gathered {
    ACC v[V];
    __device__ __forceinline__ void load(const TG* p) { ldv<ACC, TG, V>(p, v); }
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int i = 0; i < V; i++) v[i] = (ACC)0;
    }
    __device__ __forceinline__ void madd(ACC h, ACC (&acc)[V]) const {
#pragma unroll
        for (int i = 0; i < V; i++) acc[i] = fma(h, v[i], acc[i]);
    }
};

template <int V>
struct Gathered<float, __nv_bfloat16, V> {
    static_assert(V % 4 == 0, "BF16 operand chunks are 4-element vectors");
    uint32_t w[V / 2];
    __device__ __forceinline__ void load(const __nv_bfloat16* p) {
#pragma unroll
        for (int i = 0; i < V; i += 4) {
            const uint2 t = __ldg(reinterpret_cast<const uint2*>(p + i));
            w[i / 2] = t.x;
            w[i / 2 + 1] = t.y;
        }
    }
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int i = 0; i < V / 2; i++) w[i] = 0u;
    }
    // h must be exactly representable in BF16 (the BF16 schedule rounds H once).
    __device__ __forceinline__ void madd(float h, float (&acc)[V]) const {
        const __nv_bfloat16 hb = __float2bfloat16_rn(h);
        const unsigned short hbits = *reinterpret_cast<const unsigned short*>(&hb);
#pragma unroll
        for (int i = 0; i < V / 2; i++) {
            unsigned short lo, hi;
            asm("mov.b32 {%0, %1}, %2;" : "=h"(lo), "=h"(hi) : "r"(w[i]));
            asm("fma.rn.f32.bf16 %0, %1, %2, %0;" : "+f"(acc[2 * i]) : "h"(hbits), "h"(lo));
            asm("fma.rn.f32.bf16 %0, %1, %2, %0;" : "+f"(acc[2 * i + 1]) : "h"(hbits), "h"(hi));
        }
    }
};

// Resident CTAs per SM the register budget of a low-precision step is sized for: the
// FP32 and BF16-operand steps are bound by gather latency, so they take fewer chunks
// per pass (U) for more resident warps.  (The FP64 step, bound by the FP64 pipe, has
// no bound.)
template <typename TG, int U>
constexpr int lp_min_blocks() { return 3; }

template <typename TH>
__device__ __forceinline__ void stage_entry(TH* sv, int32_t* sc, const TH* val, const int32_t* col,
                                            int64_t p) {
    if constexpr (sizeof(TH) == 8) cp_async8(sv, val + p);
    else cp_async4(sv, val + p);
    cp_async4(sc, col + p);
}

// ACC: arithmetic type; TH: stored H value type; TG: gathered operand (Y_cur or
// its BF16 shadow); TC: own-row Y_cur (for the -c Y_cur term); TP: Y_prev; TO:
// output; TS: optional BF16 shadow of the output (void-like when !kShadow).
template <typename ACC, typename TH, typename TG, typename TC, typename TP, typename TO, int V, int U,
          bool kShadow>
__device__ __forceinline__ void
csr_step_body(int64_t N, const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
              const TH* __restrict__ val, int64_t nnz, int64_t n,
              const TG* __restrict__ Yg, int64_t ldg, const TC* __restrict__ Yc, int64_t ldc,
              const TP* __restrict__ Yp, int64_t ldp, TO* __restrict__ Yo, int64_t ldo,
              __nv_bfloat16* __restrict__ Ys, int64_t lds, const double* __restrict__ Ya, int64_t lda,
              ACC alpha, ACC c, ACC beta, int cap, unsigned* status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TH* s_val = reinterpret_cast<TH*>(smem_raw);
    int32_t* s_col = reinterpret_cast<int32_t*>(smem_raw + sizeof(TH) * (size_t)cap);

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
        for (int64_t q = threadIdx.x; q < cnt; q += kThreads) stage_entry(s_val + q, s_col + q, val, col, p_lo + q);
        cp_async_wait_all();
        __syncthreads();
        for (int64_t q = threadIdx.x; q < cnt; q += kThreads) {
            if ((uint64_t)(uint32_t)s_col[q] >= (uint64_t)N || s_col[q] < 0) {
                s_col[q] = 0;
                s_val[q] = (TH)0;
                bad = true;
            }
        }
        __syncthreads();
    }

    const int64_t r = r0 + warp;
    if (r < r_end) {
        int64_t rb = clampp(row_ptr[r]), re = clampp(row_ptr[r + 1]);
        if (re < rb) { re = rb; bad = true; }
        if (rb < p_lo || re > p_hi) { rb = re = p_lo; bad = true; }
        const TH* hv = staged ? s_val + (rb - p_lo) : val + rb;
        const int32_t* hc = staged ? s_col + (rb - p_lo) : col + rb;
        const int len = (int)(re - rb);
        bool nonfinite = false;

        for (int64_t jbase = 0; jbase < n; jbase += 32 * V * U) {
            ACC acc[U][V];
            bool on[U];
            const int64_t j0 = jbase + (int64_t)lane * V;
#pragma unroll
            for (int u = 0; u < U; u++) {
                on[u] = jbase + (int64_t)(u * 32 + lane) * V < n;
#pragma unroll
                for (int v = 0; v < V; v++) acc[u][v] = (ACC)0;
                if constexpr (std::is_same<ACC, double>::value) {
                    if (Ya && on[u]) ldv<double, double, V>(Ya + r * lda + j0 + u * 32 * V, acc[u]);
                }
            }
            // Register pipeline with two alternating buffers: the gathers of entry q+1
            // are in flight while entry q is accumulated.  Full chunks take a
            // predicate-free path; a bad column index (unstaged rows only) becomes a
            // zero entry on row 0.  In the low-precision steps the common case (a
            // staged slice and a full chunk) is compiled as its own loop with no
            // per-entry checks; the FP64 step, bound by its pipe, keeps one loop.
            const bool full = jbase + 32 * V * U <= n;
            using G = Gathered<ACC, TG, V>;
            auto pass = [&](auto fast_tag) {
                constexpr bool kFast = decltype(fast_tag)::value;
                auto fetch = [&](int q, G (&y)[U], ACC& h) {
                    int32_t cj = hc[q];
                    h = cvt<ACC>(hv[q]);
                    if (!kFast && !staged && (cj < 0 || (int64_t)cj >= N)) { bad = true; cj = 0; h = (ACC)0; }
                    const TG* src = Yg + (int64_t)cj * ldg + j0;
#pragma unroll
                    for (int u = 0; u < U; u++) {
                        if (kFast || full || on[u]) y[u].load(src + u * 32 * V);
                        else y[u].zero();
                    }
                };
                auto accumulate = [&](const G (&y)[U], ACC h) {
#pragma unroll
                    for (int u = 0; u < U; u++) y[u].madd(h, acc[u]);
                };
                G ya[U], yb[U];
                ACC ha = (ACC)0, hb = (ACC)0;
                if (len > 0) fetch(0, ya, ha);
                int q = 0;
                for (; q + 1 < len; q += 2) {
                    fetch(q + 1, yb, hb);
                    accumulate(ya, ha);
                    if (q + 2 < len) fetch(q + 2, ya, ha);
                    accumulate(yb, hb);
                }
                if (q < len) accumulate(ya, ha);
            };
            if constexpr (std::is_same<ACC, double>::value) {
                pass(std::false_type{});
            } else {
                if (staged && full) pass(std::true_type{});
                else pass(std::false_type{});
            }
#pragma unroll
            for (int u = 0; u < U; u++) {
                if (!on[u]) continue;
                const int64_t j = j0 + u * 32 * V;
                ACC yc[V], out[V];
                ldv<ACC, TC, V>(Yc + r * ldc + j, yc);
                if (Yp) {
                    ACC yp[V];
                    ldv<ACC, TP, V>(Yp + r * ldp + j, yp);
#pragma unroll
                    for (int v = 0; v < V; v++) out[v] = fma(-beta, yp[v], alpha * fma(-c, yc[v], acc[u][v]));
                } else {
#pragma unroll
                    for (int v = 0; v < V; v++) out[v] = alpha * fma(-c, yc[v], acc[u][v]);
                }
#pragma unroll
                for (int v = 0; v < V; v++) nonfinite |= !isfinite(out[v]);
                stv<ACC, TO, V>(Yo + r * ldo + j, out);
                if constexpr (kShadow) stv<ACC, __nv_bfloat16, V>(Ys + r * lds + j, out);
            }
        }
        if (__any_sync(0xffffffffu, nonfinite) && lane == 0) raise_status(status, DEV_NONFINITE);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) raise_status(status, DEV_PATTERN);
}

#define CSR_STEP_PARAMS                                                                                         \
    int64_t N, const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,                           \
        const TH *__restrict__ val, int64_t nnz, int64_t n, const TG *__restrict__ Yg, int64_t ldg,           \
        const TC *__restrict__ Yc, int64_t ldc, const TP *__restrict__ Yp, int64_t ldp, TO *__restrict__ Yo, \
        int64_t ldo, __nv_bfloat16 *__restrict__ Ys, int64_t lds, const double *__restrict__ Ya, int64_t lda,   \
        ACC alpha, ACC c, ACC beta, int cap, unsigned *status
#define CSR_STEP_ARGS \
    N, row_ptr, col, val, nnz, n, Yg, ldg, Yc, ldc, Yp, ldp, Yo, ldo, Ys, lds, Ya, lda, alpha, c, beta, cap, status

// FP64 step (and FP64 steps reading FP32 iterates).
template <typename ACC, typename TH, typename TG, typename TC, typename TP, typename TO, int V, int U,
          bool kShadow>
__global__ void __launch_bounds__(kThreads) csr_step_kernel(CSR_STEP_PARAMS) {
    csr_step_body<ACC, TH, TG, TC, TP, TO, V, U, kShadow>(CSR_STEP_ARGS);
}

// FP32 and BF16-operand steps.
template <typename ACC, typename TH, typename TG, typename TC, typename TP, typename TO, int V, int U,
          bool kShadow>
__global__ void __launch_bounds__(kThreads, lp_min_blocks<TG, U>()) csr_step_lp_kernel(CSR_STEP_PARAMS) {
    csr_step_body<ACC, TH, TG, TC, TP, TO, V, U, kShadow>(CSR_STEP_ARGS);
}

#undef CSR_STEP_PARAMS
#undef CSR_STEP_ARGS

template <typename ACC, typename TH, typename TG, typename TC, typename TP, typename TO, int V, int U,
          bool kShadow>
int launch(const CsrDev& h, const void* hval, int64_t n, const StepIO& io, double alpha, double c,
           double beta, unsigned* status, cudaStream_t s) {
    constexpr int kCapMax = 6144;   // staged entries per CTA (8 rows x up to 768 entries)
    // The low-precision steps stage 8 rows of a typical length (1.25 x the mean, longer
    // row blocks read their entries from global memory), so that shared memory leaves
    // L1 room for the gathers at their higher occupancy.
    int cap = kCapMax;
    if (!std::is_same<ACC, double>::value) {
        const int64_t mean = (h.nnz + h.N - 1) / h.N;
        int64_t want = (kWarps * mean * 5 / 4 + 127) / 128 * 128;
        cap = (int)(want < 256 ? 256 : (want > kCapMax ? kCapMax : want));
    }
    const size_t smem = (sizeof(TH) + sizeof(int32_t)) * (size_t)cap;
    const size_t smem_max = (sizeof(TH) + sizeof(int32_t)) * (size_t)kCapMax;
    auto kern = [] {
        if constexpr (std::is_same<ACC, double>::value) return csr_step_kernel<ACC, TH, TG, TC, TP, TO, V, U, kShadow>;
        else return csr_step_lp_kernel<ACC, TH, TG, TC, TP, TO, V, U, kShadow>;
    }();
    static bool attr_set[kMaxDevices] = {};   // per instantiation and device
    const int dev = current_device();
    if (dev < 0) return CHFSI_ERR_CUDA;
    if (!attr_set[dev]) {
        CHFSI_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max));
        attr_set[dev] = true;
    }
    const int64_t blocks = (h.N + kWarps - 1) / kWarps;
    kern<<<(unsigned)blocks, kThreads, smem, s>>>(
        h.N, h.row_ptr, h.col, static_cast<const TH*>(hval), h.nnz, n,
        static_cast<const TG*>(io.gather), io.ldg, static_cast<const TC*>(io.cur), io.ldc,
        static_cast<const TP*>(io.prev), io.ldp, static_cast<TO*>(io.out), io.ldo,
        static_cast<__nv_bfloat16*>(io.shadow), io.lds, std::is_same<ACC, double>::value ? io.addend : nullptr,
        io.lda, (ACC)alpha, (ACC)c, (ACC)beta, cap, status);
    CHFSI_LAUNCH_CHECK();
    return CHFSI_OK;
}

}  // namespace

// Dispatch on the buffer types of one step.  f64 math steps run in FP64 with any
// mix of FP64/FP32 inputs (the first FP64 steps after a low-precision prefix read
// FP32 iterates, widened exactly); f32 steps run FP32 FMA; bf16 steps gather the
// BF16 shadow and write FP32 plus a fresh shadow.
int csr_step(const CsrDev& h, StepMath math, int64_t n, const StepIO& io, double alpha, double c,
             double beta, bool vec, unsigned* status, cudaStream_t s) {
    if (n <= 0 || h.N <= 0) return CHFSI_OK;
    const Buf g = io.gather_t, cu = io.cur_t, p = io.prev ? io.prev_t : io.cur_t, o = io.out_t;
    if (math == StepMath::F64) {
        if (h.val_t != Buf::F64) return CHFSI_ERR_UNSUPPORTED;
        if (g == Buf::F64 && cu == Buf::F64 && p == Buf::F64 && o == Buf::F64) {
            if (vec) return launch<double, double, double, double, double, double, 2, 1, false>(h, h.val, n, io, alpha, c, beta, status, s);
            return launch<double, double, double, double, double, double, 1, 1, false>(h, h.val, n, io, alpha, c, beta, status, s);
        }
        if (g == Buf::F64 && cu == Buf::F64 && p == Buf::F32 && o == Buf::F64) {
            if (vec) return launch<double, double, double, double, float, double, 2, 1, false>(h, h.val, n, io, alpha, c, beta, status, s);
            return launch<double, double, double, double, float, double, 1, 1, false>(h, h.val, n, io, alpha, c, beta, status, s);
        }
        if (g == Buf::F32 && cu == Buf::F32 && p == Buf::F32 && o == Buf::F64) {
            if (vec) return launch<double, double, float, float, float, double, 2, 1, false>(h, h.val, n, io, alpha, c, beta, status, s);
            return launch<double, double, float, float, float, double, 1, 1, false>(h, h.val, n, io, alpha, c, beta, status, s);
        }
        if (g == Buf::F32 && cu == Buf::F32 && p == Buf::F64 && o == Buf::F64) {
            if (vec) return launch<double, double, float, float, double, double, 2, 1, false>(h, h.val, n, io, alpha, c, beta, status, s);
            return launch<double, double, float, float, double, double, 1, 1, false>(h, h.val, n, io, alpha, c, beta, status, s);
        }
        return CHFSI_ERR_UNSUPPORTED;
    }
    if (h.val_t != Buf::F32) return CHFSI_ERR_UNSUPPORTED;
    if (math == StepMath::F32) {
        if (g == Buf::F32 && cu == Buf::F32 && p == Buf::F32 && o == Buf::F32)
            return launch<float, float, float, float, float, float, 4, 2, false>(h, h.val, n, io, alpha, c, beta, status, s);
        return CHFSI_ERR_UNSUPPORTED;
    }
    // BF16 operand, FP32 accumulate
    if (g == Buf::BF16 && cu == Buf::F32 && p == Buf::F32 && o == Buf::F32 && io.shadow)
        return launch<float, float, __nv_bfloat16, float, float, float, 4, 4, true>(h, h.val, n, io, alpha, c, beta, status, s);
    return CHFSI_ERR_UNSUPPORTED;
}

}  // namespace chfsi
