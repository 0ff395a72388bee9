// Dense symmetric eigensolver of the Rayleigh-Ritz step (Algorithm 1 step 4, Sec. 3.4:
// H_F Q = Q Lambda), FP64, written for the GPU:
//   1. Householder tridiagonalisation  A = Q_H T Q_H^T, one reflector per column
//      (reflector of row j, symmetric matrix-vector product with the trailing block,
//      symmetric rank-2 update);
//   2. divide and conquer on T (Cuppen's splitting T = diag(T1, T2) + rho u u^T):
//      leaves of 32 rows by parallel-ordered Jacobi in shared memory; each merge
//      deflates (small components of z, nearly equal poles rotated together), finds
//      the roots of the secular equation 1 + rho sum z_j^2 / (d_j - lambda) (one warp
//      per root, bracketed steps of a two-pole rational model from the nearer pole), recomputes z
//      from the roots (the
//      Gu-Eisenstat formula, so that the eigenvectors come out orthogonal), and
//      multiplies the subproblem vectors by the eigenvectors of D + rho z z^T;
//   3. back-transformation Q = Q_H Q_T in panels of 64 reflectors (compact WY form
//      I - V T V^T, three matrix products per panel).
// Everything runs in this library's kernels (FP64 on the DFMA pipe); the host only
// orders the launches.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace chfsi {

namespace {

constexpr double kEps = 2.220446049250313e-16;
constexpr int kLeaf = 32;
constexpr int kPanel = 64;
constexpr int kSecularSmem = 6144;   // poles and weights staged in shared memory up to this size

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block (blockDim.x a multiple of 32, at most 1024); every thread gets it.
__device__ double block_sum(double v) {
    __shared__ double part[32];
    __shared__ double total;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) part[w] = v;
    __syncthreads();
    if (w == 0) {
        double t = lane < (int)(blockDim.x >> 5) ? part[lane] : 0.0;
        t = warp_sum(t);
        if (lane == 0) total = t;
    }
    __syncthreads();
    return total;
}

// ------------------------------------------------------------------ 1. tridiagonalisation

// Column j takes two launches.  The product kernel forms the reflector of row j
// (columns j+1 .. n-1 of the symmetric A): H = I - tau v v^T with v_0 = 1 maps
// x = A[j][j+1:] to beta e_1, every block recomputing beta, tau and the scale of v
// from x_0 and sum_{i>=1} x_i^2; it computes p = tau A22 v (A22 = A[j+1:, j+1:], one
// warp per row) and p . v.  The update kernel applies A22 -= v w^T + w v^T with
// w = p - (tau/2)(p . v) v, stores v in A's row j (not read again by the reduction),
// and sums the squares of the next reflector's row, A[j+1][j+3:].  The two sums are
// reduced in block order by the last block to finish (a completion counter, no
// waiting), so the results do not depend on the blocks' timing.
constexpr int kPanel32 = 32;   // columns per panel of the blocked tridiagonalisation

struct TriScalars {
    double sumsq;            // sum_{i>=1} x_i^2 of the current reflector's row
    double dot;              // p . v of the current column (blocked: (tau / 2) p . v)
    unsigned cnt_a, cnt_b;   // completion counters of the two kernels
    double c12[2 * kPanel32];   // blocked: W_t . v (t < i), then V_t . v
    double scale;               // blocked: v_q = scale x_q (q >= 1) of the current reflector
};

// Sum of the nparts partial sums written by the other blocks (called by the whole block
// that finished last): strided per thread, then the block reduction, so the order of
// the additions is fixed.
__device__ double last_block_sum(const double* part, unsigned nparts) {
    __threadfence();
    const volatile double* pp = part;
    double t = 0.0;
    for (unsigned b = threadIdx.x; b < nparts; b += blockDim.x) t += pp[b];
    return block_sum(t);
}

__device__ __forceinline__ void reflector(double x0, double sumsq, double& beta, double& t, double& scale) {
    if (sumsq == 0.0) {
        beta = x0;
        t = 0.0;
        scale = 0.0;
    } else {
        const double nrm = sqrt(x0 * x0 + sumsq);
        beta = x0 >= 0.0 ? -nrm : nrm;
        t = (beta - x0) / beta;
        scale = 1.0 / (x0 - beta);
    }
}

// Sum of squares of A[0][2:] (the first reflector's row past its leading entry).  One block.
__global__ void tri_init_kernel(const double* A, int64_t n, TriScalars* tri) {
    double s = 0.0;
    for (int64_t c = 2 + threadIdx.x; c < n; c += blockDim.x) s = fma(A[c], A[c], s);
    s = block_sum(s);
    if (threadIdx.x == 0) {
        tri->sumsq = s;
        tri->cnt_a = tri->cnt_b = 0;
    }
}

constexpr int kTriRows = 8;     // rows (one warp each) per block of the product kernel
constexpr int kTriUnroll = 8;   // loads in flight per lane in the product kernel

__global__ void __launch_bounds__(32 * kTriRows) tri_product_kernel(const double* __restrict__ A, int64_t lda,
                                                                    int64_t n, int64_t j, TriScalars* tri,
                                                                    double* part, double* d, double* e, double* tau,
                                                                    double* vbuf, double* pbuf) {
    const int64_t m = n - j - 1;
    const double* x = A + j * lda + j + 1;
    double beta, t, scale;
    reflector(x[0], tri->sumsq, beta, t, scale);
    auto v_at = [&](int64_t i) { return i == 0 ? 1.0 : x[i] * scale; };
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * kTriRows + warp;
    double pv = 0.0;
    if (r < m) {
        // eight independent partial sums per lane (eight loads in flight), combined in a
        // fixed order
        const double* row = A + (j + 1 + r) * lda + j + 1;
        double acc[kTriUnroll];
#pragma unroll
        for (int q = 0; q < kTriUnroll; q++) acc[q] = 0.0;
        int64_t i = lane;
        for (; i + 32 * (kTriUnroll - 1) < m; i += 32 * kTriUnroll) {
            double rv[kTriUnroll];
#pragma unroll
            for (int q = 0; q < kTriUnroll; q++) rv[q] = row[i + 32 * q];
#pragma unroll
            for (int q = 0; q < kTriUnroll; q++) acc[q] = fma(rv[q], v_at(i + 32 * q), acc[q]);
        }
        for (; i < m; i += 32) acc[0] = fma(row[i], v_at(i), acc[0]);
#pragma unroll
        for (int w = kTriUnroll / 2; w > 0; w /= 2)
#pragma unroll
            for (int q = 0; q < w; q++) acc[q] += acc[q + w];
        const double pr = t * warp_sum(acc[0]);
        if (lane == 0) pbuf[r] = pr;
        pv = pr * v_at(r);
    }
    if (blockIdx.x == 0)
        for (int64_t i = threadIdx.x; i < m; i += blockDim.x) vbuf[i] = v_at(i);
    __shared__ double wpart[kTriRows];
    __shared__ bool last;
    if (lane == 0) wpart[warp] = pv;
    __syncthreads();
    if (threadIdx.x == 0) {
        double bs = 0.0;
        for (int w = 0; w < kTriRows; w++) bs += wpart[w];
        part[blockIdx.x] = bs;
        __threadfence();
        last = atomicAdd(&tri->cnt_a, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {   // the last block to finish reduces the partial sums (fixed order)
        const double tot = last_block_sum(part, gridDim.x);
        if (threadIdx.x == 0) {
            tri->dot = tot;
            tri->cnt_a = 0;
            d[j] = A[j * lda + j];
            e[j] = beta;
            tau[j] = t;
        }
    }
}

constexpr int kTriUpdRows = 16;  // rows of A22 per thread of the update kernel

__global__ void __launch_bounds__(256) tri_update_kernel(double* A, int64_t lda, int64_t n, int64_t j,
                                                         TriScalars* tri, double* part,
                                                         const double* __restrict__ tau,
                                                         const double* __restrict__ vbuf,
                                                         const double* __restrict__ pbuf) {
    const int64_t m = n - j - 1;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.y * kTriUpdRows;
    const double K = 0.5 * tau[j] * tri->dot;
    double sq = 0.0;
    if (c < m) {
        const double vc = vbuf[c];
        const double wc = pbuf[c] - K * vc;
        const int64_t nr = m - r0 < kTriUpdRows ? m - r0 : kTriUpdRows;
        double* a = A + (j + 1 + r0) * lda + j + 1 + c;
        double cur[kTriUpdRows];
#pragma unroll
        for (int q = 0; q < kTriUpdRows; q++)
            if (q < nr) cur[q] = a[q * lda];          // the rows' loads all in flight
#pragma unroll
        for (int q = 0; q < kTriUpdRows; q++) {
            if (q >= nr) break;
            const double vr = vbuf[r0 + q];
            const double wr = pbuf[r0 + q] - K * vr;
            const double v = cur[q] - (vr * wc + wr * vc);
            a[q * lda] = v;
            if (r0 + q == 0) {
                if (c >= 2) sq = v * v;                // the next reflector's row past its leading entry
                A[j * lda + j + 1 + c] = vc;           // v kept in row j for the back-transformation
            }
        }
    }
    if (blockIdx.y == 0) {   // block-uniform: the blocks of the first rows sum the next reflector's squares
        __shared__ bool last;
        const double bs = block_sum(sq);
        if (threadIdx.x == 0) {
            part[blockIdx.x] = bs;
            __threadfence();
            last = atomicAdd(&tri->cnt_b, 1u) == gridDim.x - 1;
        }
        __syncthreads();
        if (last) {
            const double tot = last_block_sum(part, gridDim.x);
            if (threadIdx.x == 0) {
                tri->sumsq = tot;
                tri->cnt_b = 0;
            }
        }
    }
}

// ---- blocked tridiagonalisation (n >= kBlockedMinN)
// A panel reduces kPanel32 columns j0 .. j0 + 31 against the trailing matrix as it stood at
// the panel's start (A0); the reflectors v_t and the vectors w_t of the panel's columns
// are kept as rows of PV = [V; W; V] (length n each, zero left of their column), so that
// the matrix current at column j is A0 - sum_t (v_t w_t^T + w_t v_t^T).  Per column
// j = j0 + i: the row kernel brings row j up to date (and writes the previous column's
// v, w rows of PV); the product kernel forms y = A0[j+1:, j+1:] v (the only pass over the
// trailing matrix) and the dots W_t . v, V_t . v; the p kernel corrects
// p = tau (y - V (W^T v) - W (V^T v)) and stores v in A's row j.  After the panel the
// trailing matrix takes A -= V^T W + W^T V in one product of depth 2 * 32.

// Writes rows i of V, W (both copies of V) for the column jc whose v and p are in vbuf and
// pbuf and whose (tau / 2) p . v is kw: v_c, and w_c = p_c - kw v_c, for c in [c0, n).
__device__ __forceinline__ void blk_store_vw(double* PV, int64_t n, int i, int64_t c, const double* vbuf,
                                             const double* pbuf, double kw, double* vo, double* wo) {
    const double v = vbuf[c];
    const double w = pbuf[c] - kw * v;
    PV[(int64_t)i * n + c] = v;
    PV[(int64_t)(kPanel32 + i) * n + c] = w;
    PV[(int64_t)(2 * kPanel32 + i) * n + c] = v;
    *vo = v;
    *wo = w;
}

// Row j = j0 + i brought up to date over columns c in [j, n):
// a_c = A0[j][c] - sum_{t < i} (V_t[j] W_t[c] + W_t[j] V_t[c]); for i >= 1 the previous
// column's rows of V and W are formed from vbuf, pbuf, tri->dot (and written).  The sum of
// squares of a_c for c >= j + 2 (the next reflector's row past x_0) goes to tri->sumsq.
// A block takes 32 columns; its 8 groups of 32 threads share the terms t < i - 1 (t = g,
// g + 8, ...: all loads of a thread in flight at once) and group 0 adds their sums in order.
constexpr int kColGroups = 8, kGroupCols = 32;

__global__ void __launch_bounds__(kColGroups * kGroupCols) blk_row_kernel(double* A, int64_t lda, int64_t n,
                                                                          int64_t j, int i, double* PV,
                                                                          TriScalars* tri, double* part,
                                                                          const double* __restrict__ vbuf,
                                                                          const double* __restrict__ pbuf) {
    __shared__ double cv[kPanel32], cw[kPanel32];
    __shared__ double red[kColGroups][kGroupCols];
    const double kw = tri->dot;
    if (threadIdx.x < i) {
        const int t = threadIdx.x;
        if (t == i - 1) {   // the previous column's entries at row j, from its vbuf / pbuf
            cv[t] = vbuf[j];
            cw[t] = pbuf[j] - kw * vbuf[j];
        } else {
            cv[t] = PV[(int64_t)t * n + j];
            cw[t] = PV[(int64_t)(kPanel32 + t) * n + j];
        }
    }
    __syncthreads();
    const int cl = threadIdx.x % kGroupCols, g = threadIdx.x / kGroupCols;
    const int64_t c = j + (int64_t)blockIdx.x * kGroupCols + cl;
    double acc = 0.0;
    if (c < n) {
        const double* __restrict__ Vr = PV;
        const double* __restrict__ Wr = PV + (int64_t)kPanel32 * n;
        double vt[kPanel32 / kColGroups], wt[kPanel32 / kColGroups];
#pragma unroll
        for (int u = 0; u < kPanel32 / kColGroups; u++) {
            const int t = g + kColGroups * u;
            const bool in = t < i - 1;
            vt[u] = in ? Vr[(int64_t)t * n + c] : 0.0;
            wt[u] = in ? Wr[(int64_t)t * n + c] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kPanel32 / kColGroups; u++) {
            const int t = g + kColGroups * u;
            if (t < i - 1) acc += cv[t] * wt[u] + cw[t] * vt[u];
        }
    }
    red[g][cl] = acc;
    __syncthreads();
    double sq = 0.0;
    if (g == 0 && c < n) {
        double sum = 0.0;
#pragma unroll
        for (int h = 0; h < kColGroups; h++) sum += red[h][cl];
        double a = A[j * lda + c] - sum;
        if (i >= 1) {
            double vt, wt;
            blk_store_vw(PV, n, i - 1, c, vbuf, pbuf, kw, &vt, &wt);
            a -= cv[i - 1] * wt + cw[i - 1] * vt;
        }
        A[j * lda + c] = a;
        if (c >= j + 2) sq = a * a;
    }
    __shared__ bool last;
    const double bs = block_sum(sq);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = bs;
        __threadfence();
        last = atomicAdd(&tri->cnt_b, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
        const double tot = last_block_sum(part, gridDim.x);
        if (threadIdx.x == 0) {
            tri->sumsq = tot;
            tri->cnt_b = 0;
        }
    }
}

// The rows i of V and W for the panel's last column jc (before the trailing update):
// c in [jc + 1, n).
__global__ void blk_finish_kernel(double* PV, int64_t n, int64_t jc, int i, const TriScalars* tri,
                                  const double* __restrict__ vbuf, const double* __restrict__ pbuf) {
    const int64_t c = jc + 1 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    double v, w;
    blk_store_vw(PV, n, i, c, vbuf, pbuf, tri->dot, &v, &w);
}

// y = A0[j+1:, j+1:] v (one warp per row, blocks 0 .. nsymv-1) for the reflector of row j
// (formed in every block from x_0 and tri->sumsq, as in the unblocked product), and in
// blocks 0 .. 2i - 1 (first, so that they overlap the rows) the dots W_t . v (t < i) and
// V_t . v.  The FP64 pipe, not
// memory, bounds this pass on GB300 (one multiply-add per 8-byte entry is above the
// ridge), so v is not formed per entry: with v = scale x except v_0 = 1,
// y_r = scale (sum_q A[r][q] x_q - beta A[r][0]) (1 - scale x_0 = -scale beta), one FMA an
// entry with x read straight from A's row j; when sum_{q>=1} x_q^2 = 0 (scale = 0, v = e_0)
// y_r = A[r][0].  Block 0 also writes d[j], e[j], tau[j] and the scale of v.
constexpr int kBlkRows = 4;   // rows (one warp each) per block of the blocked product

__global__ void __launch_bounds__(32 * kBlkRows) blk_product_kernel(const double* __restrict__ A, int64_t lda,
                                                                    int64_t n, int64_t j, int i,
                                                                    const double* __restrict__ PV, TriScalars* tri,
                                                                    double* d, double* e, double* tau,
                                                                    double* ybuf) {
    const int64_t m = n - j - 1;
    const double* x = A + j * lda + j + 1;
    double beta, t, scale;
    reflector(x[0], tri->sumsq, beta, t, scale);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        d[j] = A[j * lda + j];
        e[j] = beta;
        tau[j] = t;
        tri->scale = scale;
    }
    if ((int)blockIdx.x < 2 * i) {   // block-uniform: one dot product per block
        auto v_at = [&](int64_t q) { return q == 0 ? 1.0 : x[q] * scale; };
        const int tp = (int)blockIdx.x;
        const double* row = tp < i ? PV + (int64_t)(kPanel32 + tp) * n : PV + (int64_t)(tp - i) * n;
        double acc = 0.0;
        for (int64_t q = threadIdx.x; q < m; q += blockDim.x) acc = fma(row[j + 1 + q], v_at(q), acc);
        acc = block_sum(acc);
        if (threadIdx.x == 0) tri->c12[tp] = acc;
        return;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r = (int64_t)(blockIdx.x - 2 * i) * kBlkRows + warp;
    if (r < m) {
        const double* arow = A + (j + 1 + r) * lda + j + 1;
        if (scale == 0.0) {
            if (lane == 0) ybuf[j + 1 + r] = arow[0];
        } else {
            // 16-byte loads of the row and of x (two entries a lane) after one peeled entry
            // when the segment does not start on a 16-byte boundary (A's rows and row j
            // share the alignment when lda is even)
            const bool pair_ok = (lda % 2) == 0;
            const int64_t head = (reinterpret_cast<uintptr_t>(arow) & 15u) ? 1 : 0;
            double acc[kTriUnroll];
#pragma unroll
            for (int q = 0; q < kTriUnroll; q++) acc[q] = 0.0;
            if (pair_ok) {
                const int64_t m2 = (m - head) / 2;
                const double2* a2 = reinterpret_cast<const double2*>(arow + head);
                const double2* x2 = reinterpret_cast<const double2*>(x + head);
                if (head && lane == 0) acc[0] = arow[0] * x[0];
                int64_t q0 = lane;
                for (; q0 + 32 * (kTriUnroll - 1) < m2; q0 += 32 * kTriUnroll) {
                    double2 rv[kTriUnroll], xv[kTriUnroll];
#pragma unroll
                    for (int q = 0; q < kTriUnroll; q++) {
                        rv[q] = a2[q0 + 32 * q];
                        xv[q] = x2[q0 + 32 * q];
                    }
#pragma unroll
                    for (int q = 0; q < kTriUnroll; q++) {
                        acc[q] = fma(rv[q].x, xv[q].x, acc[q]);
                        acc[q] = fma(rv[q].y, xv[q].y, acc[q]);
                    }
                }
                for (; q0 < m2; q0 += 32) {
                    const double2 rv = a2[q0], xv = x2[q0];
                    acc[0] = fma(rv.x, xv.x, acc[0]);
                    acc[0] = fma(rv.y, xv.y, acc[0]);
                }
                if (((m - head) & 1) && lane == 0) acc[1] = fma(arow[m - 1], x[m - 1], acc[1]);
            } else {
                for (int64_t q = lane; q < m; q += 32) acc[0] = fma(arow[q], x[q], acc[0]);
            }
#pragma unroll
            for (int w = kTriUnroll / 2; w > 0; w /= 2)
#pragma unroll
                for (int q = 0; q < w; q++) acc[q] += acc[q + w];
            const double y = warp_sum(acc[0]);
            if (lane == 0) ybuf[j + 1 + r] = scale * fma(-beta, arow[0], y);
        }
    }
}

// p = tau (y - sum_t (V_t W_t . v + W_t V_t . v)) over rows r in [j+1, n), v (from x and
// the scale) stored in vbuf and in A's row j for the back-transformation, and (tau / 2) p . v
// to tri->dot (reduced in a fixed order by the last block to finish).  A block takes 32
// rows; its 8 groups share the terms t < i as in the row kernel.
__global__ void __launch_bounds__(kColGroups * kGroupCols) blk_p_kernel(double* A, int64_t lda, int64_t n, int64_t j,
                                                                        int i, const double* __restrict__ PV,
                                                                        TriScalars* tri, double* part,
                                                                        const double* __restrict__ tau, double* vbuf,
                                                                        const double* __restrict__ ybuf, double* pbuf) {
    __shared__ double c1[kPanel32], c2[kPanel32];
    __shared__ double red[kColGroups][kGroupCols];
    if (threadIdx.x < kPanel32) {
        c1[threadIdx.x] = (int)threadIdx.x < i ? tri->c12[threadIdx.x] : 0.0;
        c2[threadIdx.x] = (int)threadIdx.x < i ? tri->c12[i + threadIdx.x] : 0.0;
    }
    __syncthreads();
    const int rl = threadIdx.x % kGroupCols, g = threadIdx.x / kGroupCols;
    const int64_t r = j + 1 + (int64_t)blockIdx.x * kGroupCols + rl;
    double acc = 0.0;
    if (r < n) {
        double vt[kPanel32 / kColGroups], wt[kPanel32 / kColGroups];
#pragma unroll
        for (int u = 0; u < kPanel32 / kColGroups; u++) {
            const int t = g + kColGroups * u;
            const bool in = t < i;
            vt[u] = in ? PV[(int64_t)t * n + r] : 0.0;
            wt[u] = in ? PV[(int64_t)(kPanel32 + t) * n + r] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kPanel32 / kColGroups; u++) {
            const int t = g + kColGroups * u;
            if (t < i) acc += vt[u] * c1[t] + wt[u] * c2[t];
        }
    }
    red[g][rl] = acc;
    __syncthreads();
    const double tj = tau[j];
    double pv = 0.0;
    if (g == 0 && r < n) {
        double sum = 0.0;
#pragma unroll
        for (int h = 0; h < kColGroups; h++) sum += red[h][rl];
        const double pr = tj * (ybuf[r] - sum);
        pbuf[r] = pr;
        const double v = r == j + 1 ? 1.0 : A[j * lda + r] * tri->scale;   // x_r read, then v_r stored
        vbuf[r] = v;
        pv = pr * v;
        A[j * lda + r] = v;
    }
    __shared__ bool last;
    const double bs = block_sum(pv);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = bs;
        __threadfence();
        last = atomicAdd(&tri->cnt_a, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
        const double tot = last_block_sum(part, gridDim.x);
        if (threadIdx.x == 0) {
            tri->dot = 0.5 * tj * tot;
            tri->cnt_a = 0;
        }
    }
}

// The last 2 x 2 (or 1 x 1) block of T.
__global__ void tridiag_tail_kernel(const double* A, int64_t lda, int64_t n, double* d, double* e, double* tau) {
    if (threadIdx.x != 0) return;
    if (n >= 2) {
        d[n - 2] = A[(n - 2) * lda + n - 2];
        e[n - 2] = A[(n - 2) * lda + n - 1];
        tau[n - 2] = 0.0;
    }
    d[n - 1] = A[(n - 1) * lda + n - 1];
}

// ------------------------------------------------------------------ 2. divide and conquer

// Cuppen's splitting at every leaf boundary m: d[m-1] and d[m] lose rho = e[m-1];
// the original off-diagonal is kept in ebak.
__global__ void dc_split_kernel(int64_t n, double* d, const double* e, double* ebak) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n - 1) ebak[i] = e[i];
    const int64_t m = (i + 1) * kLeaf;   // boundary number i
    if (m < n) {
        const double rho = e[m - 1];
        d[m - 1] -= rho;
        d[m] -= rho;
    }
}

// Leaf eigenproblems by parallel (round-robin ordered) Jacobi; one block per leaf.
// Writes ascending eigenvalues to w[l ..] and the eigenvectors into the diagonal block
// Q[l.., l..] (the rest of Q is zero).
__global__ void __launch_bounds__(256) dc_leaf_kernel(int64_t n, const double* d, const double* e, double* w,
                                                      double* Q, int64_t ldq) {
    __shared__ double A[kLeaf][kLeaf + 1];
    __shared__ double V[kLeaf][kLeaf + 1];
    __shared__ double rc[kLeaf / 2], rs[kLeaf / 2];
    __shared__ int rp[kLeaf / 2], rq[kLeaf / 2];
    __shared__ int rank[kLeaf];
    const int64_t l = (int64_t)blockIdx.x * kLeaf;
    const int s = (int)((n - l) < kLeaf ? (n - l) : kLeaf);
    for (int idx = threadIdx.x; idx < kLeaf * kLeaf; idx += blockDim.x) {
        const int i = idx / kLeaf, j = idx % kLeaf;
        double v = 0.0;
        if (i < s && j < s) {
            if (i == j) v = d[l + i];
            else if (j == i + 1) v = e[l + i];
            else if (i == j + 1) v = e[l + j];
        }
        A[i][j] = v;
        V[i][j] = i == j ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int sweep = 0; sweep < 20; sweep++) {
        double o = 0.0, t2 = 0.0;
        for (int idx = threadIdx.x; idx < kLeaf * kLeaf; idx += blockDim.x) {
            const int i = idx / kLeaf, j = idx % kLeaf;
            const double a2 = A[i][j] * A[i][j];
            t2 += a2;
            if (i != j) o += a2;
        }
        o = block_sum(o);
        t2 = block_sum(t2);
        if (o <= 1e-30 * t2 || o == 0.0) break;   // off-diagonal below about 1e-15 |A|
        for (int round = 0; round < kLeaf - 1; round++) {
            // pairs of this round: players 0 .. kLeaf-1, player 0 fixed, the others rotating
            if (threadIdx.x < kLeaf / 2) {
                const int k = threadIdx.x;
                auto player = [&](int pos) { return pos == 0 ? 0 : ((pos - 1 + round) % (kLeaf - 1)) + 1; };
                int p = player(k), q = player(kLeaf - 1 - k);
                if (p > q) { const int t = p; p = q; q = t; }
                const double apq = A[p][q];
                double c = 1.0, sn = 0.0;
                if (apq != 0.0 && fabs(apq) > 1e-300) {
                    const double theta = (A[q][q] - A[p][p]) / (2.0 * apq);
                    const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                    c = 1.0 / sqrt(t * t + 1.0);
                    sn = t * c;
                }
                rp[k] = p; rq[k] = q; rc[k] = c; rs[k] = sn;
            }
            __syncthreads();
            // rows p, q of A (rotations of one round touch disjoint rows)
            for (int idx = threadIdx.x; idx < (kLeaf / 2) * kLeaf; idx += blockDim.x) {
                const int k = idx / kLeaf, col = idx % kLeaf;
                const int p = rp[k], q = rq[k];
                const double c = rc[k], sn = rs[k];
                const double ap = A[p][col], aq = A[q][col];
                A[p][col] = c * ap - sn * aq;
                A[q][col] = sn * ap + c * aq;
            }
            __syncthreads();
            // columns p, q of A and of V
            for (int idx = threadIdx.x; idx < (kLeaf / 2) * kLeaf; idx += blockDim.x) {
                const int k = idx / kLeaf, row = idx % kLeaf;
                const int p = rp[k], q = rq[k];
                const double c = rc[k], sn = rs[k];
                const double ap = A[row][p], aq = A[row][q];
                A[row][p] = c * ap - sn * aq;
                A[row][q] = sn * ap + c * aq;
                const double vp = V[row][p], vq = V[row][q];
                V[row][p] = c * vp - sn * vq;
                V[row][q] = sn * vp + c * vq;
            }
            __syncthreads();
        }
    }
    // ascending order of the s real eigenvalues (the padding rows never mix with them)
    if (threadIdx.x < s) {
        const int i = threadIdx.x;
        const double li = A[i][i];
        int r = 0;
        for (int j = 0; j < s; j++) {
            const double lj = A[j][j];
            r += (lj < li) || (lj == li && j < i);
        }
        rank[i] = r;
    }
    __syncthreads();
    if (threadIdx.x < s) w[l + rank[threadIdx.x]] = A[threadIdx.x][threadIdx.x];
    for (int idx = threadIdx.x; idx < s * s; idx += blockDim.x) {
        const int r = idx / s, i = idx % s;
        Q[(l + r) * ldq + l + rank[i]] = V[r][i];
    }
}

// Per-merge scratch (device arrays of n, or of n x n for the matrices).
struct MergeBufs {
    double *D, *z, *Dnd, *znd, *tau_r, *zhat, *norm, *val, *rot_c, *rot_s, *par;
    int *perm, *defl, *ndidx, *pos, *org, *rot_a, *rot_b, *rank;
    double *G, *U, *Gn;
};

// par[] = {rho_hat, sign, k_nd, nrot}.
// Merge preparation: z from the boundary rows, signs, the sorted poles, deflation with
// the Givens rotations of nearly equal poles.  One block (the scans on thread 0).
__global__ void __launch_bounds__(1024) dc_merge_prep_kernel(int64_t l, int64_t m, int64_t r, const double* w,
                                                             const double* Q, int64_t ldq, const double* ebak,
                                                             MergeBufs b) {
    const int64_t n1 = m - l, k = r - l;
    const double rho0 = ebak[m - 1];
    const double sg = rho0 >= 0.0 ? 1.0 : -1.0;
    double zz = 0.0;
    for (int64_t p = threadIdx.x; p < k; p += blockDim.x) {
        const double zp = p < n1 ? Q[(m - 1) * ldq + l + p] : Q[m * ldq + m + (p - n1)];
        b.z[p] = zp;
        b.D[p] = sg * w[l + p];
        zz += zp * zp;
    }
    zz = block_sum(zz);
    __syncthreads();
    if (threadIdx.x == 0) {
        const double rho_hat = fabs(rho0) * zz;
        const double zs = 1.0 / sqrt(zz > 0.0 ? zz : 1.0);
        // merge the two sorted halves (ascending when sg > 0, descending otherwise)
        int64_t i = 0, j = 0, o = 0;
        auto at1 = [&](int64_t t) { return sg > 0.0 ? t : n1 - 1 - t; };
        auto at2 = [&](int64_t t) { return sg > 0.0 ? n1 + t : k - 1 - t; };
        while (i < n1 || j < k - n1) {
            if (j >= k - n1 || (i < n1 && b.D[at1(i)] <= b.D[at2(j)])) b.perm[o++] = (int)at1(i++);
            else b.perm[o++] = (int)at2(j++);
        }
        double dmax = 0.0;
        for (int64_t p = 0; p < k; p++) {
            const int q = b.perm[p];
            b.val[p] = b.D[q];                 // sorted poles (modified by the rotations below)
            b.tau_r[p] = b.z[q] * zs;          // sorted, normalised z (temporarily)
            dmax = fmax(dmax, fabs(b.val[p]));
        }
        const double tol = 8.0 * kEps * fmax(dmax, rho_hat);
        int nrot = 0;
        int64_t last = -1;
        for (int64_t p = 0; p < k; p++) {
            b.defl[p] = fabs(rho_hat * b.tau_r[p]) <= tol;
            if (b.defl[p]) continue;
            if (last >= 0 && fabs(b.val[p] - b.val[last]) <= tol) {
                const double zl = b.tau_r[last], zp = b.tau_r[p];
                const double rr = hypot(zl, zp), c = zp / rr, s = -zl / rr;
                const double dl = b.val[last], dp = b.val[p];
                b.val[last] = c * c * dl + s * s * dp;
                b.val[p] = s * s * dl + c * c * dp;
                b.tau_r[p] = rr;
                b.tau_r[last] = 0.0;
                b.defl[last] = 1;
                b.rot_a[nrot] = (int)last;
                b.rot_b[nrot] = (int)p;
                b.rot_c[nrot] = c;
                b.rot_s[nrot] = s;
                nrot++;
            }
            last = p;
        }
        int64_t kn = 0;
        for (int64_t p = 0; p < k; p++) {
            if (!b.defl[p]) {
                b.ndidx[kn] = (int)p;
                b.pos[p] = (int)kn;
                b.Dnd[kn] = b.val[p];
                b.znd[kn] = b.tau_r[p];
                kn++;
            } else {
                b.pos[p] = -1;
            }
        }
        b.par[0] = rho_hat;
        b.par[1] = sg;
        b.par[2] = (double)kn;
        b.par[3] = (double)nrot;
    }
}

// The deflation rotations on the block's columns (column p of the sorted problem is
// block column perm[p]); one thread per row applies them in order.
__global__ void dc_rotate_kernel(int64_t l, int64_t k, double* Q, int64_t ldq, MergeBufs b) {
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= k) return;
    const int nrot = (int)b.par[3];
    double* q = Q + (l + row) * ldq + l;
    for (int t = 0; t < nrot; t++) {
        const int a = b.perm[b.rot_a[t]], c2 = b.perm[b.rot_b[t]];
        const double c = b.rot_c[t], s = b.rot_s[t];
        const double qa = q[a], qb = q[c2];
        q[a] = c * qa + s * qb;
        q[c2] = -s * qa + c * qb;
    }
}

constexpr int kRootWarps = 8;        // roots (one warp each) per block of the secular-equation kernels

__device__ __forceinline__ double warp_prod(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v *= __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Roots of 1 + rho sum_j z_j^2 / (d_j - lambda) (rho > 0, d ascending, sum z^2 <= 1):
// root i lies in (d_i, d_{i+1}), the last in (d_k, d_k + rho).  One warp per root, the
// lanes sharing the sum over the poles (the xor-butterfly sums leave the same value in
// every lane, so the warp's control flow stays uniform).  Each root is found in
// tau = lambda - d_org, measured from the nearer pole d_org, so that the differences
// d_j - lambda = (d_j - d_org) - tau keep their relative accuracy.  Steps to the zero
// of a rational model with the two neighbouring poles (constant plus one pole term for
// each side, fitted to the value and slope of each side's sum: the interpolation
// behind the classical secular-equation solvers of Bunch, Nielsen and Sorensen and of
// R.-C. Li), kept inside a bracket [lo, hi] with g(lo) < 0 < g(hi) by a bisection step
// whenever the model's step would leave it.
__global__ void __launch_bounds__(32 * kRootWarps) dc_secular_kernel(MergeBufs b, int cap) {
    extern __shared__ double sh[];
    const int k = (int)b.par[2];
    const double rho = b.par[0];
    const bool staged = k <= cap;   // cap: poles the dynamic shared memory was sized for
    double* Ds = sh;
    double* z2 = sh + (staged ? k : 0);
    if (staged) {
        for (int j = threadIdx.x; j < k; j += blockDim.x) {
            Ds[j] = b.Dnd[j];
            z2[j] = b.znd[j] * b.znd[j];
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * kRootWarps + (threadIdx.x >> 5);
    if (i >= k) return;
    auto Dj = [&](int j) { return staged ? Ds[j] : b.Dnd[j]; };
    auto Zj = [&](int j) { return staged ? z2[j] : b.znd[j] * b.znd[j]; };
    const double d_i = Dj(i);
    const double gap = (i + 1 < k) ? Dj(i + 1) - d_i : rho;
    // g at the midpoint decides which pole is nearer
    const double mid = d_i + 0.5 * gap;
    double fm = 0.0;
    for (int j = lane; j < k; j += 32) fm += Zj(j) / (Dj(j) - mid);
    fm = 1.0 + rho * warp_sum(fm);
    int org;
    double lo, hi;
    if (i + 1 == k) {
        org = i;
        if (fm < 0.0) { lo = 0.5 * gap; hi = gap; }
        else { lo = 0.0; hi = 0.5 * gap; }
    } else if (fm >= 0.0) {
        org = i; lo = 0.0; hi = 0.5 * gap;
    } else {
        org = i + 1; lo = -0.5 * gap; hi = 0.0;
    }
    const double dorg = Dj(org);
    const bool last = i + 1 == k;
    double t = 0.5 * (lo + hi);
    for (int it = 0; it < 200; it++) {
        // g = 1 + psi + phi (poles j <= i and j > i) and the derivatives of both parts
        double psi = 0.0, phi = 0.0, dpsi = 0.0, dphi = 0.0;
        for (int j = lane; j < k; j += 32) {
            const double r = 1.0 / ((Dj(j) - dorg) - t);
            const double q = Zj(j) * r;
            if (j <= i) {
                psi += q;
                dpsi = fma(q, r, dpsi);
            } else {
                phi += q;
                dphi = fma(q, r, dphi);
            }
        }
        psi = rho * warp_sum(psi);
        phi = rho * warp_sum(phi);
        dpsi = rho * warp_sum(dpsi);
        dphi = rho * warp_sum(dphi);
        const double g = 1.0 + psi + phi;
        if (g == 0.0) break;
        if (g > 0.0) hi = t;
        else lo = t;
        // the step to the zero of the model c + s / (Di - eta) + S / (Dn - eta), which has
        // the poles d_i and d_{i+1} and matches g and g' at tau (the last root: d_i only);
        // of its two zeros the one nearer tau
        const double Di = (d_i - dorg) - t;
        const double s = Di * Di * dpsi;
        double eta = 0.0;
        bool have = false;
        if (last) {
            const double c = g - s / Di;
            if (c != 0.0) {
                eta = Di + s / c;
                have = true;
            }
        } else {
            const double Dn = (Dj(i + 1) - dorg) - t;
            const double S = Dn * Dn * dphi;
            const double c = g - s / Di - S / Dn;
            const double qa = c, qb = -(c * (Di + Dn) + s + S), qc = c * Di * Dn + s * Dn + S * Di;
            if (qa == 0.0) {
                if (qb != 0.0) {
                    eta = -qc / qb;
                    have = true;
                }
            } else {
                const double disc = qb * qb - 4.0 * qa * qc;
                if (disc >= 0.0) {
                    const double qq = -0.5 * (qb + copysign(sqrt(disc), qb));
                    const double e1 = qq / qa, e2 = qq != 0.0 ? qc / qq : e1;
                    eta = fabs(e1) <= fabs(e2) ? e1 : e2;
                    have = true;
                }
            }
        }
        have = have && isfinite(eta);
        if (have && fabs(eta) <= 2.0 * kEps * fabs(t)) break;   // converged
        double tn = have ? t + eta : 0.5 * (lo + hi);
        if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);        // a bisection step instead
        const bool done = fabs(tn - t) <= 2.0 * kEps * fabs(tn) || hi - lo <= 2.0 * kEps * fmax(fabs(lo), fabs(hi));
        t = tn;
        if (done) break;
    }
    if (lane == 0) {
        b.org[i] = org;
        b.tau_r[i] = t;
    }
}

// Recomputed weights zhat_i^2 = prod_j (lambda_j - d_i) / (rho prod_{j != i} (d_j - d_i))
// (sign of the original z_i); one warp per i, each lane a strided part of the product.
// By interlacing, every partial product of the ratios stays between the bounds of the
// telescoping products, far from overflow.
__global__ void __launch_bounds__(32 * kRootWarps) dc_lowner_kernel(MergeBufs b) {
    const int k = (int)b.par[2];
    const double rho = b.par[0];
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * kRootWarps + (threadIdx.x >> 5);
    if (i >= k) return;
    const double di = b.Dnd[i];
    double prod = 1.0;
    for (int j = lane; j < k; j += 32) {
        const double lmd = (b.Dnd[b.org[j]] - di) + b.tau_r[j];   // lambda_j - d_i
        prod *= (j == i) ? lmd / rho : lmd / (b.Dnd[j] - di);
    }
    prod = warp_prod(prod);
    if (lane == 0) {
        const double zh = sqrt(fabs(prod));
        b.zhat[i] = b.znd[i] >= 0.0 ? zh : -zh;
    }
}

// Norms of the eigenvectors u_i = (zhat_j / (d_j - lambda_i))_j; one warp per i.
__global__ void __launch_bounds__(32 * kRootWarps) dc_norm_kernel(MergeBufs b) {
    const int k = (int)b.par[2];
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * kRootWarps + (threadIdx.x >> 5);
    if (i >= k) return;
    const double dorg = b.Dnd[b.org[i]], t = b.tau_r[i];
    double s = 0.0;
    for (int j = lane; j < k; j += 32) {
        const double q = b.zhat[j] / ((b.Dnd[j] - dorg) - t);
        s = fma(q, q, s);
    }
    s = warp_sum(s);
    if (lane == 0) b.norm[i] = sqrt(s);
}

// U[j][i] = zhat_j / (d_j - lambda_i) / |u_i|  (k_nd x k_nd, row-major).
__global__ void dc_build_u_kernel(MergeBufs b) {
    const int k = (int)b.par[2];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= k || j >= k) return;
    b.U[(int64_t)j * k + i] = b.zhat[j] / ((b.Dnd[j] - b.Dnd[b.org[i]]) - b.tau_r[i]) / b.norm[i];
}

// G[row][c] = block column perm[ndidx[c]] of Q.
__global__ void dc_gather_kernel(int64_t l, int64_t k, const double* Q, int64_t ldq, MergeBufs b) {
    const int kn = (int)b.par[2];
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t row = blockIdx.y;
    if (c >= kn || row >= k) return;
    b.G[row * kn + c] = Q[(l + row) * ldq + l + b.perm[b.ndidx[c]]];
}

// Final eigenvalues of the merged problem (sign restored) and their ascending ranks.
__global__ void dc_rank_kernel(int64_t k, MergeBufs b) {
    const double sg = b.par[1];
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < k; p += (int64_t)gridDim.x * blockDim.x) {
        const int q = b.pos[p];
        b.D[p] = sg * (q < 0 ? b.val[p] : b.Dnd[b.org[q]] + b.tau_r[q]);
    }
}

// Ascending rank of each merged eigenvalue (ties by index); one warp per value.
__global__ void __launch_bounds__(32 * kRootWarps) dc_rank2_kernel(int64_t k, MergeBufs b) {
    const int lane = threadIdx.x & 31;
    const int64_t p = (int64_t)blockIdx.x * kRootWarps + (threadIdx.x >> 5);
    if (p >= k) return;
    const double vp = b.D[p];
    int r = 0;
    for (int64_t q = lane; q < k; q += 32) {
        const double vq = b.D[q];
        r += (vq < vp) || (vq == vp && q < p);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    if (lane == 0) b.rank[p] = r;
}

// Writes the merged eigenvalues w[l + rank] and the block's new columns into F
// (k x k): deflated columns from Q, the others from Gn = G U.
__global__ void dc_scatter_kernel(int64_t l, int64_t k, const double* Q, int64_t ldq, double* w, double* F,
                                  MergeBufs b) {
    const int kn = (int)b.par[2];
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t row = blockIdx.y;
    if (p >= k || row >= k) return;
    const int dst = b.rank[p];
    const int q = b.pos[p];
    F[row * k + dst] = q < 0 ? Q[(l + row) * ldq + l + b.perm[p]] : b.Gn[row * kn + q];
    if (row == 0) w[l + dst] = b.D[p];
}

__global__ void copy_block_kernel(const double* F, int64_t k, double* Q, int64_t ldq, int64_t l) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t row = blockIdx.y;
    if (c >= k || row >= k) return;
    Q[(l + row) * ldq + l + c] = F[row * k + c];
}

// ------------------------------------------------------------------ 3. back-transformation

// Vp[t][i] = component j0 + 1 + i of reflector j0 + t (rows j0 + 1 .. n - 1), zero above its 1.
__global__ void panel_v_kernel(const double* A, int64_t lda, int64_t n, int64_t j0, int nb, double* Vp) {
    const int64_t mr = n - j0 - 1;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int t = blockIdx.y;
    if (i >= mr || t >= nb) return;
    const int64_t j = j0 + t, row = j0 + 1 + i;
    double v = 0.0;
    if (row == j + 1) v = 1.0;
    else if (row > j + 1) v = A[j * lda + row];
    Vp[t * mr + i] = v;
}

// Gv[s][t] = Vp[s] . Vp[t] (s <= t), one block per pair.
__global__ void panel_gram_kernel(const double* Vp, int64_t mr, int nb, double* Gv) {
    const int s = blockIdx.x, t = blockIdx.y;
    if (s > t) return;
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < mr; i += blockDim.x) acc = fma(Vp[s * mr + i], Vp[t * mr + i], acc);
    acc = block_sum(acc);
    if (threadIdx.x == 0) Gv[s * nb + t] = acc;
}

// T of H_j0 ... H_{j0+nb-1} = I - V T V^T (upper triangular, forward accumulation):
// T[t][t] = tau_t, T[0:t, t] = -tau_t T[0:t, 0:t] Gv[0:t, t].  One block.
__global__ void panel_t_kernel(const double* Gv, const double* tau, int64_t j0, int nb, double* T) {
    for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) T[idx] = 0.0;
    __syncthreads();
    for (int t = 0; t < nb; t++) {
        const double tt = tau[j0 + t];
        if (threadIdx.x < t) {
            const int s = threadIdx.x;
            double acc = 0.0;
            for (int u = s; u < t; u++) acc = fma(T[s * nb + u], Gv[u * nb + t], acc);
            T[s * nb + t] = -tt * acc;
        }
        if (threadIdx.x == 0) T[t * nb + t] = tt;
        __syncthreads();
    }
}

// ------------------------------------------------------------------ workspace

inline int64_t round8(int64_t x) { return (x + 7) / 8 * 8; }

// Products of the merges (G U) and of the back-transformation run as Ozaki products on
// the tensor cores for 256 <= n <= 8192 (the NN form takes inner dimensions up to
// 8192), otherwise as FP64 products on the DFMA pipe (small n: a few tiles, where the
// slicing passes would cost more than they save).
constexpr int64_t kOzakiMinN = 256, kOzakiMaxN = 8192;
constexpr int64_t kBlockedMinN = 2048;   // the blocked tridiagonalisation from this n on

struct EighBufs {
    double *d, *e, *tau, *ebak, *vbuf, *pbuf, *part_a, *part_b;
    double *PV, *ybuf;      // blocked tridiagonalisation: [V; W; V] of a panel, y = A0 v
    TriScalars* tri;
    MergeBufs mb;
    double *Vp, *Gv, *T, *W1, *W2;
    unsigned char* oz;      // Ozaki product scratch (nullptr for n > kOzakiMaxN)
    size_t oz_bytes;
};

size_t eigh_ozaki_bytes(int64_t n) {
    if (n < kOzakiMinN || n > kOzakiMaxN) return 0;
    return std::max({ozaki_workspace_bytes(false, n, n, n, false), ozaki_workspace_bytes(false, kPanel, n, n, false),
                     ozaki_workspace_bytes(true, n, n, kPanel, false)});
}

template <typename Ar>
void eigh_layout(Ar& ar, int64_t n, EighBufs* out) {
    EighBufs u{};
    u.d = ar.template take<double>(n);
    u.e = ar.template take<double>(n);
    u.tau = ar.template take<double>(n);
    u.ebak = ar.template take<double>(n);
    u.vbuf = ar.template take<double>(n);
    u.pbuf = ar.template take<double>(n);
    u.part_a = ar.template take<double>((size_t)(n / kTriRows + 1));
    u.part_b = ar.template take<double>((size_t)(n / 32 + 1));
    u.tri = ar.template take<TriScalars>(1);
    u.PV = ar.template take<double>((size_t)(3 * kPanel32) * n);
    u.ybuf = ar.template take<double>(n);
    MergeBufs& b = u.mb;
    b.D = ar.template take<double>(n);
    b.z = ar.template take<double>(n);
    b.Dnd = ar.template take<double>(n);
    b.znd = ar.template take<double>(n);
    b.tau_r = ar.template take<double>(n);
    b.zhat = ar.template take<double>(n);
    b.norm = ar.template take<double>(n);
    b.val = ar.template take<double>(n);
    b.rot_c = ar.template take<double>(n);
    b.rot_s = ar.template take<double>(n);
    b.par = ar.template take<double>(8);
    b.perm = ar.template take<int>(n);
    b.defl = ar.template take<int>(n);
    b.ndidx = ar.template take<int>(n);
    b.pos = ar.template take<int>(n);
    b.org = ar.template take<int>(n);
    b.rot_a = ar.template take<int>(n);
    b.rot_b = ar.template take<int>(n);
    b.rank = ar.template take<int>(n);
    b.G = ar.template take<double>((size_t)n * n);
    b.U = ar.template take<double>((size_t)n * n);
    b.Gn = ar.template take<double>((size_t)n * n);
    u.Vp = ar.template take<double>((size_t)kPanel * n);
    u.Gv = ar.template take<double>((size_t)kPanel * kPanel);
    u.T = ar.template take<double>((size_t)kPanel * kPanel);
    u.W1 = ar.template take<double>((size_t)kPanel * n);
    u.W2 = ar.template take<double>((size_t)kPanel * n);
    u.oz_bytes = eigh_ozaki_bytes(n);
    u.oz = u.oz_bytes ? ar.template take<unsigned char>(u.oz_bytes) : nullptr;
    if (out) *out = u;
}

// Z[i][c] -= D[i][c] (rows x cols; Z with leading dimension ldz, D dense).
__global__ void sub_block_kernel(double* Z, int64_t ldz, const double* __restrict__ D, int64_t rows, int64_t cols) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * cols) return;
    const int64_t i = idx / cols, c = idx % cols;
    Z[i * ldz + c] -= D[idx];
}

struct CountOnly {
    Sizer s;
    template <typename T>
    T* take(size_t n) {
        s.take<T>(n);
        return nullptr;
    }
};

}  // namespace

size_t eigh_workspace_bytes(int64_t n) {
    CountOnly ar;
    eigh_layout(ar, n > 0 ? n : 1, nullptr);
    return ar.s.used;
}

int eigh(double* A, int64_t lda, int64_t n, double* w, double* Q, int64_t ldq, void* ws, size_t ws_bytes,
         unsigned* status, cudaStream_t s) {
    if (n <= 0) return CHFSI_OK;
    if (ws_bytes < eigh_workspace_bytes(n)) return CHFSI_ERR_NOMEM;
    Arena ar(ws, ws_bytes);
    EighBufs u;
    eigh_layout(ar, n, &u);
    double *d = u.d, *e = u.e, *tau = u.tau, *ebak = u.ebak, *Vp = u.Vp, *Gv = u.Gv, *T = u.T, *W1 = u.W1,
           *W2 = u.W2;
    MergeBufs& mb = u.mb;
    const bool oz = u.oz != nullptr;

    // 1. tridiagonalisation: blocked for large n (one pass over the trailing matrix per
    // column plus one product per panel), else two launches per column
    if (n >= kBlockedMinN) {
        CHFSI_CUDA_TRY(cudaMemsetAsync(u.tri, 0, sizeof(TriScalars), s));
        for (int64_t j0 = 0; j0 + 2 < n; j0 += kPanel32) {
            const int nc = (int)std::min<int64_t>(kPanel32, (n - 2) - j0);
            if (nc < kPanel32)   // rows nc .. 31 of V and W take part in the trailing product
                CHFSI_CUDA_TRY(cudaMemsetAsync(u.PV, 0, sizeof(double) * (size_t)(3 * kPanel32) * n, s));
            for (int i = 0; i < nc; i++) {
                const int64_t j = j0 + i, m = n - j - 1;
                blk_row_kernel<<<(unsigned)((n - j + kGroupCols - 1) / kGroupCols), kColGroups * kGroupCols, 0, s>>>(
                    A, lda, n, j, i, u.PV, u.tri, u.part_b, u.vbuf, u.pbuf);
                CHFSI_LAUNCH_CHECK();
                const unsigned nrowb = (unsigned)((m + kBlkRows - 1) / kBlkRows);
                blk_product_kernel<<<nrowb + 2 * i, 32 * kBlkRows, 0, s>>>(A, lda, n, j, i, u.PV, u.tri, d, e, tau,
                                                                          u.ybuf);
                CHFSI_LAUNCH_CHECK();
                blk_p_kernel<<<(unsigned)((m + kGroupCols - 1) / kGroupCols), kColGroups * kGroupCols, 0, s>>>(
                    A, lda, n, j, i, u.PV, u.tri, u.part_a, tau, u.vbuf, u.ybuf, u.pbuf);
                CHFSI_LAUNCH_CHECK();
            }
            const int64_t jl = j0 + nc - 1, jn = j0 + nc, mp = n - jn;
            blk_finish_kernel<<<(unsigned)((n - jl - 1 + 255) / 256), 256, 0, s>>>(u.PV, n, jl, nc - 1, u.tri, u.vbuf,
                                                                                   u.pbuf);
            CHFSI_LAUNCH_CHECK();
            // trailing matrix: A[jn:, jn:] -= V^T W + W^T V over the panel's rows of PV
            const double* Vop = u.PV + jn;
            const double* Wop = u.PV + (int64_t)kPanel32 * n + jn;
            double* C22 = A + jn * lda + jn;
            int rc;
            if (oz && mp >= kOzakiMinN) {
                if ((rc = ozaki_gemm_tn(Vop, n, Wop, n, 2 * kPanel32, mp, mp, mb.G, mp, true, u.oz, u.oz_bytes, status,
                                        s)))
                    return rc;
                sub_block_kernel<<<(unsigned)((mp * mp + 255) / 256), 256, 0, s>>>(C22, lda, mb.G, mp, mp);
                CHFSI_LAUNCH_CHECK();
            } else if ((rc = gemm_general(Vop, n, true, Wop, n, C22, lda, mp, mp, 2 * kPanel32, -1.0, true, s))) {
                return rc;
            }
        }
    } else if (n >= 3) {
        tri_init_kernel<<<1, 1024, 0, s>>>(A, n, u.tri);
        CHFSI_LAUNCH_CHECK();
    }
    for (int64_t j = 0; n < kBlockedMinN && j + 2 < n; j++) {
        const int64_t m = n - j - 1;
        tri_product_kernel<<<(unsigned)((m + kTriRows - 1) / kTriRows), 32 * kTriRows, 0, s>>>(
            A, lda, n, j, u.tri, u.part_a, d, e, tau, u.vbuf, u.pbuf);
        CHFSI_LAUNCH_CHECK();
        tri_update_kernel<<<dim3((unsigned)((m + 255) / 256), (unsigned)((m + kTriUpdRows - 1) / kTriUpdRows)), 256, 0,
                            s>>>(A, lda, n, j, u.tri, u.part_b, tau, u.vbuf, u.pbuf);
        CHFSI_LAUNCH_CHECK();
    }
    tridiag_tail_kernel<<<1, 32, 0, s>>>(A, lda, n, d, e, tau);
    CHFSI_LAUNCH_CHECK();

    // 2. divide and conquer on (d, e): Q starts as the leaf eigenvectors
    CHFSI_CUDA_TRY(cudaMemset2DAsync(Q, sizeof(double) * (size_t)ldq, 0, sizeof(double) * (size_t)n, (size_t)n, s));
    dc_split_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, d, e, ebak);
    CHFSI_LAUNCH_CHECK();
    const int64_t nleaf = (n + kLeaf - 1) / kLeaf;
    dc_leaf_kernel<<<(unsigned)nleaf, 256, 0, s>>>(n, d, e, w, Q, ldq);
    CHFSI_LAUNCH_CHECK();
    std::vector<int64_t> bounds;
    for (int64_t i = 0; i <= nleaf; i++) bounds.push_back(std::min(i * kLeaf, n));
    while (bounds.size() > 2) {
        std::vector<int64_t> next;
        next.push_back(bounds[0]);
        for (size_t i = 0; i + 2 < bounds.size(); i += 2) {
            const int64_t l = bounds[i], m = bounds[i + 1], r = bounds[i + 2];
            const int64_t k = r - l;
            dc_merge_prep_kernel<<<1, 1024, 0, s>>>(l, m, r, w, Q, ldq, ebak, mb);
            CHFSI_LAUNCH_CHECK();
            dc_rotate_kernel<<<(unsigned)((k + 255) / 256), 256, 0, s>>>(l, k, Q, ldq, mb);
            CHFSI_LAUNCH_CHECK();
            const size_t sh = k <= kSecularSmem ? 2 * sizeof(double) * (size_t)k : 0;
            if (sh > 48 * 1024) {
                static bool attr[kMaxDevices] = {};
                const int dev = current_device();
                if (dev < 0) return CHFSI_ERR_CUDA;
                if (!attr[dev]) {
                    CHFSI_CUDA_TRY(cudaFuncSetAttribute(dc_secular_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                        (int)(2 * sizeof(double) * kSecularSmem)));
                    attr[dev] = true;
                }
            }
            // the non-deflated count is only known on the device: size the grids for k
            const unsigned root_blocks = (unsigned)((k + kRootWarps - 1) / kRootWarps);
            dc_secular_kernel<<<root_blocks, 32 * kRootWarps, sh, s>>>(mb, sh ? (int)k : 0);
            CHFSI_LAUNCH_CHECK();
            dc_lowner_kernel<<<root_blocks, 32 * kRootWarps, 0, s>>>(mb);
            CHFSI_LAUNCH_CHECK();
            dc_norm_kernel<<<root_blocks, 32 * kRootWarps, 0, s>>>(mb);
            CHFSI_LAUNCH_CHECK();
            dc_build_u_kernel<<<dim3((unsigned)((k + 255) / 256), (unsigned)k), 256, 0, s>>>(mb);
            CHFSI_LAUNCH_CHECK();
            dc_gather_kernel<<<dim3((unsigned)((k + 255) / 256), (unsigned)k), 256, 0, s>>>(l, k, Q, ldq, mb);
            CHFSI_LAUNCH_CHECK();
            // Gn (k x kn) = G (k x kn) U (kn x kn); kn <= k is read on the device, so the
            // product runs at the full size k with G, U and Gn laid out for kn: a host copy
            // of kn keeps the shapes exact
            double kn_d = 0.0;
            CHFSI_CUDA_TRY(cudaMemcpyAsync(&kn_d, mb.par + 2, sizeof(double), cudaMemcpyDeviceToHost, s));
            CHFSI_CUDA_TRY(cudaStreamSynchronize(s));
            const int64_t kn = (int64_t)kn_d;
            int rc = oz ? ozaki_gemm_nn(mb.G, kn, mb.U, kn, k, kn, kn, mb.Gn, kn, false, u.oz, u.oz_bytes, status, s)
                        : gemm_general(mb.G, kn, false, mb.U, kn, mb.Gn, kn, k, kn, kn, 1.0, false, s);
            if (rc) return rc;
            dc_rank_kernel<<<(unsigned)((k + 255) / 256), 256, 0, s>>>(k, mb);
            CHFSI_LAUNCH_CHECK();
            dc_rank2_kernel<<<root_blocks, 32 * kRootWarps, 0, s>>>(k, mb);
            CHFSI_LAUNCH_CHECK();
            dc_scatter_kernel<<<dim3((unsigned)((k + 255) / 256), (unsigned)k), 256, 0, s>>>(l, k, Q, ldq, w, mb.U,
                                                                                          mb);
            CHFSI_LAUNCH_CHECK();
            copy_block_kernel<<<dim3((unsigned)((k + 255) / 256), (unsigned)k), 256, 0, s>>>(mb.U, k, Q, ldq, l);
            CHFSI_LAUNCH_CHECK();
            next.push_back(r);
        }
        if (bounds.size() % 2 == 0) next.push_back(bounds.back());   // an unpaired last block carries over
        bounds.swap(next);
    }

    // 3. back-transformation Q = H_0 H_1 ... H_{n-3} Q, panels from the last
    const int64_t nref = n - 2;   // reflectors j = 0 .. n - 3
    for (int64_t j0 = ((nref - 1) / kPanel) * kPanel; nref > 0 && j0 >= 0; j0 -= kPanel) {
        const int nb = (int)std::min<int64_t>(kPanel, nref - j0);
        const int64_t mr = n - j0 - 1;
        panel_v_kernel<<<dim3((unsigned)((mr + 255) / 256), (unsigned)nb), 256, 0, s>>>(A, lda, n, j0, nb, Vp);
        CHFSI_LAUNCH_CHECK();
        panel_gram_kernel<<<dim3((unsigned)nb, (unsigned)nb), 256, 0, s>>>(Vp, mr, nb, Gv);
        CHFSI_LAUNCH_CHECK();
        panel_t_kernel<<<1, 128, 0, s>>>(Gv, tau, j0, nb, T);
        CHFSI_LAUNCH_CHECK();
        double* ZR = Q + (j0 + 1) * ldq;
        int rc;
        if (oz) {
            // W1 = V^T Z, W2 = T W1 (small, DFMA), Z -= V W2 through a product block
            if ((rc = ozaki_gemm_nn(Vp, mr, ZR, ldq, nb, mr, n, W1, n, false, u.oz, u.oz_bytes, status, s))) return rc;
            if ((rc = gemm_general(T, nb, false, W1, n, W2, n, nb, n, nb, 1.0, false, s))) return rc;
            if ((rc = ozaki_gemm_tn(Vp, mr, W2, n, nb, mr, n, mb.G, n, false, u.oz, u.oz_bytes, status, s))) return rc;
            sub_block_kernel<<<(unsigned)((mr * n + 255) / 256), 256, 0, s>>>(ZR, ldq, mb.G, mr, n);
            CHFSI_LAUNCH_CHECK();
        } else {
            if ((rc = gemm_general(Vp, mr, false, ZR, ldq, W1, n, nb, n, mr, 1.0, false, s))) return rc;
            if ((rc = gemm_general(T, nb, false, W1, n, W2, n, nb, n, nb, 1.0, false, s))) return rc;
            if ((rc = gemm_general(Vp, mr, true, W2, n, ZR, ldq, mr, n, nb, -1.0, true, s))) return rc;
        }
    }
    return CHFSI_OK;
}

}  // namespace chfsi

int chfsi_eigh_workspace_size(int64_t n, size_t* bytes) {
    if (!bytes || n < 0) return CHFSI_ERR_ARG;
    *bytes = chfsi::align_up(chfsi::kStatusBytes) + chfsi::eigh_workspace_bytes(n);
    return CHFSI_OK;
}

int chfsi_eigh(double* A, int64_t lda, int64_t n, double* w, double* Q, int64_t ldq, void* ws, size_t ws_bytes,
               void* stream) {
    if (n < 0 || (n > 0 && (!A || !w || !Q || lda < n || ldq < n))) return CHFSI_ERR_ARG;
    if (n == 0) return CHFSI_OK;
    if (n > 65535) return CHFSI_ERR_UNSUPPORTED;   // one grid row per matrix row in several launches
    size_t need = 0;
    int rc = chfsi_eigh_workspace_size(n, &need);
    if (rc) return rc;
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u)) return CHFSI_ERR_ARG;
    if (ws_bytes < need) return CHFSI_ERR_NOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned* st = chfsi::status_word(ws);
    CHFSI_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(unsigned), s));
    char* rest = static_cast<char*>(ws) + chfsi::align_up(chfsi::kStatusBytes);
    return chfsi::eigh(A, lda, n, w, Q, ldq, rest, ws_bytes - chfsi::align_up(chfsi::kStatusBytes), st, s);
}
