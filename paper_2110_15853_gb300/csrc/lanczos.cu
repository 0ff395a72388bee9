// Spectral bounds for Algorithm 1 (Sec. 3.4 takes eps_0, eps_ub^w, eps_ub^uw as
// inputs without saying how they are found): k-step Lanczos with full
// re-orthogonalisation on the GPU, then the extreme eigenvalues of the k x k
// tridiagonal T_k by Sturm-sequence bisection in a one-thread kernel.
//
// Every scalar (alpha_j, beta_j, the re-orthogonalisation coefficients, the stop
// flag) stays in device memory, so the k steps queue without host round trips.
// Every reduction uses a fixed partition and a fixed combination order, so the
// result is bitwise reproducible run to run.
#include "common.cuh"
#include "kernels.cuh"

namespace chfsi {

namespace {

constexpr int kRowsPerBlock = 8;     // SpMV: one warp per row
constexpr int kChunk = 2048;         // vector kernels: rows per block
constexpr int kMaxSteps = 64;

// scal layout
enum {
    S_ALPHA = 0,                 // [kMaxSteps]
    S_BETA = kMaxSteps,          // [kMaxSteps]
    S_H = 2 * kMaxSteps,         // [kMaxSteps + 1] re-orthogonalisation coefficients
    S_K = 3 * kMaxSteps + 1,     // number of completed steps (as double)
    S_STOP = S_K + 1,            // 1.0 after breakdown
    S_SCALE = S_STOP + 1,        // running max |alpha_i| + beta_{i-1}
    S_TOTAL = S_SCALE + 1,
};

__device__ __forceinline__ double block_sum(double v, double* red) {
    // fixed-shape tree over the block (blockDim.x = 256)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
    return t;   // valid on thread 0
}

// w = H v ; part[b] = sum over the block's rows of v[r] w[r]
__global__ void __launch_bounds__(256) spmv_dot_kernel(int64_t N, const int64_t* __restrict__ row_ptr,
                                                       const int32_t* __restrict__ col,
                                                       const double* __restrict__ val, int64_t nnz,
                                                       const double* __restrict__ v, double* w, double* part,
                                                       const double* scal, unsigned* status) {
    if (scal[S_STOP] != 0.0) return;
    __shared__ double rowdot[kRowsPerBlock];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * kRowsPerBlock + warp;
    double d = 0.0;
    if (r < N) {
        int64_t b = row_ptr[r], e = row_ptr[r + 1];
        if (b < 0) b = 0;
        if (e > nnz) e = nnz;
        double s = 0.0;
        bool bad = false;
        for (int64_t p = b + lane; p < e; p += 32) {
            int32_t c = col[p];
            if (c < 0 || (int64_t)c >= N) { bad = true; continue; }
            s = fma(val[p], v[c], s);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (__any_sync(0xffffffffu, bad) && lane == 0) raise_status(status, DEV_PATTERN);
        if (lane == 0) {
            w[r] = s;
            d = v[r] * s;
        }
    }
    if (lane == 0) rowdot[warp] = d;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < kRowsPerBlock; i++) t += rowdot[i];
        part[blockIdx.x] = t;
    }
}

// out[idx] = sum_b part[b * stride + idx], one block per idx, fixed order.
__global__ void __launch_bounds__(256) finalize_kernel(const double* part, int64_t nparts, int64_t stride,
                                                       double* out, int mode, int j, double* scal) {
    if (scal[S_STOP] != 0.0) return;
    __shared__ double red[8];
    const int idx = blockIdx.x;
    double s = 0.0;
    for (int64_t b = threadIdx.x; b < nparts; b += blockDim.x) s += part[b * stride + idx];
    double t = block_sum(s, red);
    if (threadIdx.x != 0) return;
    if (mode == 0) {                 // alpha_j
        out[idx] = t;
    } else if (mode == 1) {          // re-orthogonalisation coefficients h_i
        out[idx] = t;
    } else {                         // beta_j = |w|, breakdown test
        double beta = sqrt(t);
        double al = scal[S_ALPHA + j];
        double scale = scal[S_SCALE];
        double cand = fabs(al) + (j > 0 ? scal[S_BETA + j - 1] : 0.0);
        if (cand > scale) scale = cand;
        scal[S_SCALE] = scale;
        scal[S_K] = (double)(j + 1);
        if (beta <= 1e-12 * scale) {
            scal[S_BETA + j] = 0.0;
            scal[S_STOP] = 1.0;
        } else {
            scal[S_BETA + j] = beta;
        }
    }
}

// w -= alpha_j v_j + beta_{j-1} v_{j-1}; part[b*(j+1) + i] = <V_i, w> over the block's rows
__global__ void __launch_bounds__(256) three_term_dots_kernel(int64_t N, double* w, const double* V, int j,
                                                              double* part, const double* scal) {
    if (scal[S_STOP] != 0.0) return;
    __shared__ double red[8];
    const int64_t r0 = (int64_t)blockIdx.x * kChunk;
    const int64_t r1 = r0 + kChunk < N ? r0 + kChunk : N;
    const double al = scal[S_ALPHA + j];
    const double bp = j > 0 ? scal[S_BETA + j - 1] : 0.0;
    const double* vj = V + (int64_t)j * N;
    const double* vjm = j > 0 ? V + (int64_t)(j - 1) * N : nullptr;
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        double x = w[r] - al * vj[r];
        if (vjm) x -= bp * vjm[r];
        w[r] = x;
    }
    __syncthreads();
    for (int i = 0; i <= j; i++) {
        const double* vi = V + (int64_t)i * N;
        double s = 0.0;
        for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) s = fma(vi[r], w[r], s);
        double t = block_sum(s, red);
        if (threadIdx.x == 0) part[(int64_t)blockIdx.x * (j + 1) + i] = t;
    }
}

// w -= sum_i h_i V_i ; part[b] = |w|^2 over the block's rows
__global__ void __launch_bounds__(256) reorth_norm_kernel(int64_t N, double* w, const double* V, int j,
                                                          double* part, const double* scal) {
    if (scal[S_STOP] != 0.0) return;
    __shared__ double red[8];
    const int64_t r0 = (int64_t)blockIdx.x * kChunk;
    const int64_t r1 = r0 + kChunk < N ? r0 + kChunk : N;
    double s = 0.0;
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        double x = w[r];
        for (int i = 0; i <= j; i++) x -= scal[S_H + i] * V[(int64_t)i * N + r];
        w[r] = x;
        s = fma(x, x, s);
    }
    double t = block_sum(s, red);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// v_{j+1} = w / beta_j
__global__ void scale_next_kernel(int64_t N, const double* w, double* V, int j, const double* scal) {
    if (scal[S_STOP] != 0.0) return;
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    V[(int64_t)(j + 1) * N + r] = w[r] / scal[S_BETA + j];
}

// v_0 = v0 / |v0| (norm from part sums, fixed order)
__global__ void __launch_bounds__(256) sq_part_kernel(int64_t N, const double* v, double* part) {
    __shared__ double red[8];
    const int64_t r0 = (int64_t)blockIdx.x * kChunk;
    const int64_t r1 = r0 + kChunk < N ? r0 + kChunk : N;
    double s = 0.0;
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) s = fma(v[r], v[r], s);
    double t = block_sum(s, red);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void __launch_bounds__(256) norm0_kernel(int64_t N, const double* v0, double* V, const double* part,
                                                    int64_t nparts, double* scal) {
    __shared__ double red[8];
    __shared__ double nrm;
    double s = 0.0;
    for (int64_t b = threadIdx.x; b < nparts; b += blockDim.x) s += part[b];
    double t = block_sum(s, red);
    if (threadIdx.x == 0) {
        nrm = sqrt(t);
        for (int i = 0; i < S_TOTAL; i++) scal[i] = 0.0;
        if (!(nrm > 0.0) || !isfinite(nrm)) scal[S_STOP] = 2.0;   // unusable start vector
    }
    __syncthreads();
    if (scal[S_STOP] != 0.0) return;
    for (int64_t r = threadIdx.x; r < N; r += blockDim.x) V[r] = v0[r] / nrm;
}

// Number of eigenvalues of the symmetric tridiagonal (d, e) that are < x.
__device__ int sturm_count(const double* d, const double* e, int k, double x) {
    int cnt = 0;
    double q = d[0] - x;
    const double tiny = 1e-300;
    if (q == 0.0) q = -tiny;
    if (q < 0.0) cnt++;
    for (int i = 1; i < k; i++) {
        q = (d[i] - x) - e[i - 1] * e[i - 1] / q;
        if (q == 0.0) q = -tiny;
        if (q < 0.0) cnt++;
    }
    return cnt;
}

// The point of (a, b) where the Sturm count reaches `target` (the target-th smallest
// eigenvalue of T_k), by multisection on one warp: each lane counts at one of 32
// equally spaced interior points, and the bracket shrinks to the interval between the
// last point below the target and the first at or above it (a factor 33 per round, where
// bisection gives 2).  Every lane ends with the same bracket.
__device__ double sturm_edge(const double* d, const double* e, int k, double a, double b, int target) {
    const int lane = threadIdx.x & 31;
    for (int it = 0; it < 64; it++) {
        const double h = (b - a) / 33.0;
        const double x = a + h * (double)(lane + 1);
        const bool ge = !(x < b) || sturm_count(d, e, k, x) >= target;
        const unsigned mask = __ballot_sync(0xffffffffu, ge);
        double na, nb;
        if (mask == 0) {
            na = __shfl_sync(0xffffffffu, x, 31);
            nb = b;
        } else {
            const int f = __ffs(mask) - 1;
            nb = __shfl_sync(0xffffffffu, x, f);
            const double xl = __shfl_sync(0xffffffffu, x, f > 0 ? f - 1 : 0);
            na = f > 0 ? xl : a;
        }
        if (!(na > a) && !(nb < b)) break;   // the bracket is at rounding resolution
        a = na > a ? na : a;
        b = nb < b ? nb : b;
    }
    return 0.5 * (a + b);
}

// Smallest and largest eigenvalue of T_k by multisection (one warp), then the bounds.
__global__ void bounds_kernel(const double* scal, int64_t N, int64_t n_wanted, double* out) {
    if (blockIdx.x != 0 || threadIdx.x >= 32) return;
    if (scal[S_STOP] == 2.0) {
        if (threadIdx.x == 0) out[0] = out[1] = out[2] = nan("");
        return;
    }
    int k = (int)scal[S_K];
    const double* d = scal + S_ALPHA;
    const double* e = scal + S_BETA;
    double lo = d[0], hi = d[0];
    for (int i = 0; i < k; i++) {
        double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < k ? fabs(e[i]) : 0.0);
        lo = fmin(lo, d[i] - r);
        hi = fmax(hi, d[i] + r);
    }
    double span = hi - lo;
    lo -= 1e-12 * (span + 1.0);
    hi += 1e-12 * (span + 1.0);
    const double theta_min = sturm_edge(d, e, k, lo, hi, 1);
    const double theta_max = sturm_edge(d, e, k, lo, hi, k);
    if (threadIdx.x != 0) return;
    const double resid = fabs(e[k - 1]);
    const double a0 = theta_min;
    const double bb = theta_max + resid;
    const double aa = a0 + (bb - a0) * pow((double)n_wanted / (double)N, 2.0 / 3.0);
    out[0] = aa;
    out[1] = bb;
    out[2] = a0;
}

}  // namespace

size_t lanczos_part_count(int64_t N, int steps) {
    int64_t spmv_blocks = (N + kRowsPerBlock - 1) / kRowsPerBlock;
    int64_t chunks = (N + kChunk - 1) / kChunk;
    int64_t a = chunks * (steps + 1);
    return (size_t)(spmv_blocks > a ? spmv_blocks : a) + S_TOTAL;
}

int lanczos_run(const CsrDev& h, int steps, const double* v0, int64_t n_wanted, double* V, double* w,
                double* part, double* scal, double* dev_out, unsigned* status, cudaStream_t s) {
    const int64_t N = h.N;
    int k = steps < N ? steps : (int)N;
    if (k < 1 || k > kMaxSteps) return CHFSI_ERR_ARG;
    const double* val = static_cast<const double*>(h.val);
    const int64_t chunks = (N + kChunk - 1) / kChunk;
    const int64_t spmv_blocks = (N + kRowsPerBlock - 1) / kRowsPerBlock;

    sq_part_kernel<<<(unsigned)chunks, 256, 0, s>>>(N, v0, part);
    CHFSI_LAUNCH_CHECK();
    norm0_kernel<<<1, 256, 0, s>>>(N, v0, V, part, chunks, scal);
    CHFSI_LAUNCH_CHECK();
    for (int j = 0; j < k; j++) {
        const double* vj = V + (int64_t)j * N;
        spmv_dot_kernel<<<(unsigned)spmv_blocks, 256, 0, s>>>(N, h.row_ptr, h.col, val, h.nnz, vj, w, part,
                                                              scal, status);
        CHFSI_LAUNCH_CHECK();
        finalize_kernel<<<1, 256, 0, s>>>(part, spmv_blocks, 1, scal + S_ALPHA + j, 0, j, scal);
        CHFSI_LAUNCH_CHECK();
        three_term_dots_kernel<<<(unsigned)chunks, 256, 0, s>>>(N, w, V, j, part, scal);
        CHFSI_LAUNCH_CHECK();
        finalize_kernel<<<j + 1, 256, 0, s>>>(part, chunks, j + 1, scal + S_H, 1, j, scal);
        CHFSI_LAUNCH_CHECK();
        reorth_norm_kernel<<<(unsigned)chunks, 256, 0, s>>>(N, w, V, j, part, scal);
        CHFSI_LAUNCH_CHECK();
        finalize_kernel<<<1, 256, 0, s>>>(part, chunks, 1, nullptr, 2, j, scal);
        CHFSI_LAUNCH_CHECK();
        scale_next_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(N, w, V, j, scal);
        CHFSI_LAUNCH_CHECK();
    }
    bounds_kernel<<<1, 32, 0, s>>>(scal, N, n_wanted, dev_out);
    CHFSI_LAUNCH_CHECK();
    return CHFSI_OK;
}

}  // namespace chfsi
