// Pipe-peak probe: the FMA throughput of this GPU's FP64 (DFMA) or FP32 (FFMA)
// pipe, measured with a register-resident loop of independent fused multiply-adds
// and timed with CUDA events on the caller's stream.  It is the denominator of the
// roofline fraction of the FP64 and FP32 filter steps (those steps are bound by the
// arithmetic pipe, not by HBM), measured in the same process and at the same
// clocks as the kernels it is compared with.  Diagnostics only: the paper has no
// counterpart.
#include "common.cuh"
#include "kernels.cuh"

namespace chfsi {

namespace {

constexpr int kChains = 8;        // independent FMA chains per thread
constexpr int kIters = 16384;     // loop trips per chain (about 70 ms of DFMA work per launch)
constexpr int kTimed = 3;         // timed launches; the fastest counts
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;

// Written only if a result equals an impossible value, so that the compiler keeps
// every FMA; no allocation is needed for it.
__device__ double g_probe_sink;

// Each chain multiplies and adds its own registers: with one operand register shared
// by every chain the DFMA issue rate measured about 16% lower on GB300.
template <typename T>
__global__ void __launch_bounds__(kThreads) fma_loop_kernel(T seed) {
    T a[kChains], b[kChains];
    const T x = seed + (T)threadIdx.x * (T)1e-7;
#pragma unroll
    for (int c = 0; c < kChains; c++) {
        a[c] = x + (T)c;
        b[c] = (T)0.999999 - (T)c * (T)1e-9;
    }
#pragma unroll 4
    for (int i = 0; i < kIters; i++) {
#pragma unroll
        for (int c = 0; c < kChains; c++) a[c] = fma(a[c], b[c], b[c]);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; c++) s += a[c];
    if (s == (T)-12345.0) g_probe_sink = (double)s;
}

template <typename T>
int run_probe(double* flops_per_s, cudaStream_t s) {
    int dev = current_device();
    if (dev < 0) return CHFSI_ERR_CUDA;
    int sms = 0;
    CHFSI_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const unsigned grid = (unsigned)(sms * kBlocksPerSm);
    cudaEvent_t e0, e1;
    CHFSI_CUDA_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return CHFSI_ERR_CUDA;
    }
    int rc = CHFSI_OK;
    float best = 0.0f;
    // one untimed launch (clocks ramp, code loaded), then kTimed timed ones
    for (int rep = 0; rep <= kTimed && rc == CHFSI_OK; rep++) {
        if (rep >= 1 && cudaEventRecord(e0, s) != cudaSuccess) rc = CHFSI_ERR_CUDA;
        fma_loop_kernel<T><<<grid, kThreads, 0, s>>>((T)1.0);
        note_launch();
        if (cudaGetLastError() != cudaSuccess) rc = CHFSI_ERR_CUDA;
        if (rep == 0 || rc != CHFSI_OK) continue;
        float ms = 0.0f;
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
            rc = CHFSI_ERR_CUDA;
        else if (ms > 0.0f && (best == 0.0f || ms < best))
            best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != CHFSI_OK) return rc;
    if (!(best > 0.0f)) return CHFSI_ERR_CUDA;
    const float ms = best;
    const double flops = 2.0 * kChains * (double)kIters * kThreads * (double)grid;
    *flops_per_s = flops / (ms * 1e-3);
    return CHFSI_OK;
}

}  // namespace

}  // namespace chfsi

int chfsi_measure_pipe_peak(int32_t precision, double* flops_per_second, void* stream) {
    if (!flops_per_second) return CHFSI_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (precision == CHFSI_F64) return chfsi::run_probe<double>(flops_per_second, s);
    if (precision == CHFSI_F32) return chfsi::run_probe<float>(flops_per_second, s);
    return CHFSI_ERR_ARG;
}
