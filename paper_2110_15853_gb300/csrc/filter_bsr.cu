// Fused BSR filter step (Algorithm 1, step 1, Sec. 3.4) on dense 64 x 64 blocks:
//
//     Y_out[R] = alpha * (sum_{(R,C)} H_RC Y_cur[C] - c Y_cur[R]) - beta Y_prev[R]
//
// for block row R (64 grid points of one 4 x 4 x 4 sub-cube) and a 64-column tile.
// This is the paper's "dense near the diagonal" treatment of H (Sec. 4.2 splits H
// into dense and sparse parts for the same reason) taken to a blocked layout: each
// CTA is a small dense GEMM chain over the <= 27 neighbouring blocks, with the
// recurrence fused into the epilogue.  CUDA-core FMA version (FP64 DFMA or FP32
// FFMA): 256 threads, 4 x 4 outputs per thread, operands staged in shared memory in
// 16-deep chunks.  The blocks are dense, so the zero entries inside them are
// executed too (7-42% fill on the Kronecker-banded operators).
#include "common.cuh"
#include "kernels.cuh"

namespace chfsi {

namespace {

constexpr int TB = 64;
constexpr int BK = 16;

template <typename ACC, typename TH, typename TG, typename TC, typename TP, typename TO>
__global__ void __launch_bounds__(256)
bsr_step_kernel(int64_t nbr, const int32_t* __restrict__ brow_ptr, const int32_t* __restrict__ bcol,
                const TH* __restrict__ val, int64_t nblocks, int64_t n, const TG* __restrict__ Yg, int64_t ldg,
                const TC* __restrict__ Yc, int64_t ldc, const TP* __restrict__ Yp, int64_t ldp, TO* __restrict__ Yo,
                int64_t ldo, ACC alpha, ACC c, ACC beta, unsigned* status) {
    __shared__ ACC Hs[BK][TB + 1];   // Hs[k][i] = H_block[i][k0 + k]
    __shared__ ACC Ys[BK][TB];       // Ys[k][j] = Y[C*64 + k0 + k][j0 + j]
    const int64_t R = blockIdx.y;
    const int64_t j0 = (int64_t)blockIdx.x * TB;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    int64_t qb = brow_ptr[R], qe = brow_ptr[R + 1];
    bool bad = false;
    if (qb < 0) { qb = 0; bad = true; }
    if (qe > nblocks) { qe = nblocks; bad = true; }

    ACC acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 4; b++) acc[a][b] = (ACC)0;

    for (int64_t q = qb; q < qe; q++) {
        const int32_t C = bcol[q];
        if (C < 0 || (int64_t)C >= nbr) { bad = true; continue; }
        const TH* hb = val + q * (int64_t)(TB * TB);
        const TG* yb = Yg + (int64_t)C * TB * ldg;
        for (int k0 = 0; k0 < TB; k0 += BK) {
            for (int e = threadIdx.x; e < BK * TB; e += 256) {
                int ii = e / BK, kk = e % BK;
                Hs[kk][ii] = (ACC)hb[ii * TB + k0 + kk];
                int kb = e / TB, jb = e % TB;
                int64_t j = j0 + jb;
                Ys[kb][jb] = (j < n) ? (ACC)yb[(int64_t)(k0 + kb) * ldg + j] : (ACC)0;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < BK; kk++) {
                ACC av[4], bv[4];
#pragma unroll
                for (int a = 0; a < 4; a++) av[a] = Hs[kk][ty + 16 * a];
#pragma unroll
                for (int b = 0; b < 4; b++) bv[b] = Ys[kk][tx + 16 * b];
#pragma unroll
                for (int a = 0; a < 4; a++)
#pragma unroll
                    for (int b = 0; b < 4; b++) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
            }
            __syncthreads();
        }
    }

    bool nonfinite = false;
#pragma unroll
    for (int a = 0; a < 4; a++) {
        const int64_t i = R * TB + ty + 16 * a;
#pragma unroll
        for (int b = 0; b < 4; b++) {
            const int64_t j = j0 + tx + 16 * b;
            if (j >= n) continue;
            ACC yc = (ACC)Yc[i * ldc + j];
            ACC out = alpha * fma(-c, yc, acc[a][b]);
            if (Yp) out = fma(-beta, (ACC)Yp[i * ldp + j], out);
            nonfinite |= !isfinite(out);
            Yo[i * ldo + j] = (TO)out;
        }
    }
    if (__syncthreads_or(nonfinite) && threadIdx.x == 0) raise_status(status, DEV_NONFINITE);
    if (bad && threadIdx.x == 0) raise_status(status, DEV_PATTERN);
}

template <typename ACC, typename TH, typename TG, typename TC, typename TP, typename TO>
int launch(const BsrDev& h, int64_t n, const StepIO& io, double alpha, double c, double beta, unsigned* status,
           cudaStream_t s) {
    dim3 grid((unsigned)((n + TB - 1) / TB), (unsigned)h.nbr);
    bsr_step_kernel<ACC, TH, TG, TC, TP, TO><<<grid, 256, 0, s>>>(
        h.nbr, h.brow_ptr, h.bcol, static_cast<const TH*>(h.val), h.nblocks, n, static_cast<const TG*>(io.gather),
        io.ldg, static_cast<const TC*>(io.cur), io.ldc, static_cast<const TP*>(io.prev), io.ldp,
        static_cast<TO*>(io.out), io.ldo, (ACC)alpha, (ACC)c, (ACC)beta, status);
    CHFSI_LAUNCH_CHECK();
    return CHFSI_OK;
}

}  // namespace

int bsr_step(const BsrDev& h, StepMath math, int64_t n, const StepIO& io, double alpha, double c, double beta,
             unsigned* status, cudaStream_t s) {
    if (n <= 0 || h.nbr <= 0) return CHFSI_OK;
    if (h.bdim != TB) return CHFSI_ERR_UNSUPPORTED;
    const Buf g = io.gather_t, cu = io.cur_t, p = io.prev ? io.prev_t : io.cur_t, o = io.out_t;
    if (math == StepMath::F64) {
        if (h.val_t != Buf::F64) return CHFSI_ERR_UNSUPPORTED;
        if (g == Buf::F64 && cu == Buf::F64 && p == Buf::F64 && o == Buf::F64)
            return launch<double, double, double, double, double, double>(h, n, io, alpha, c, beta, status, s);
        if (g == Buf::F64 && cu == Buf::F64 && p == Buf::F32 && o == Buf::F64)
            return launch<double, double, double, double, float, double>(h, n, io, alpha, c, beta, status, s);
        if (g == Buf::F32 && cu == Buf::F32 && p == Buf::F32 && o == Buf::F64)
            return launch<double, double, float, float, float, double>(h, n, io, alpha, c, beta, status, s);
        if (g == Buf::F32 && cu == Buf::F32 && p == Buf::F64 && o == Buf::F64)
            return launch<double, double, float, float, double, double>(h, n, io, alpha, c, beta, status, s);
        return CHFSI_ERR_UNSUPPORTED;
    }
    if (math == StepMath::F32) {
        if (h.val_t != Buf::F32) return CHFSI_ERR_UNSUPPORTED;
        if (g == Buf::F32 && cu == Buf::F32 && p == Buf::F32 && o == Buf::F32)
            return launch<float, float, float, float, float, float>(h, n, io, alpha, c, beta, status, s);
        return CHFSI_ERR_UNSUPPORTED;
    }
    return CHFSI_ERR_UNSUPPORTED;   // BF16 operands on BSR: tensor-core kernel
}

}  // namespace chfsi
