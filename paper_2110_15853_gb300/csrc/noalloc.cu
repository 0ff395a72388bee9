// chfsi_filter_noalloc: the Chebyshev filter for callers that cannot allocate
// device memory.
//
// Some hosts own all device memory through their own allocator -- a DFT code with
// a pre-sized device pool, or a framework whose caching allocator must stay the
// only one -- and must not call cudaMalloc/cudaFree (those calls synchronise the
// device and fragment the pool) nor hand this library a workspace.  For them the
// filter's scratch (the status word and the two FP64 iterate buffers of the
// three-term recurrence) lives in the file-scope device array below, which every
// GPU that loads the library holds until the process exits.  The caller still
// passes X and Y.
//
// The array's name is only a host-side stand-in in host code, so the device
// address is looked up once per device with cudaGetSymbolAddress (with that device
// current) and cached until the process exits; that lookup happens on the first
// call made on each device.  A device reset (cudaDeviceReset, or a primary context
// torn down and created again) reloads the module and makes the cached address
// stale, so it is not supported between calls.  Every call then runs the regular
// chfsi_filter with the array as its workspace; the status word that the filter's
// kernels set (non-finite values, column indices out of range) sits in the
// array's first bytes and chfsi_filter_noalloc_read_status reads it back.
#include <mutex>

#include "common.cuh"

namespace {

constexpr size_t kNoallocScratchBytes = size_t(16) << 20;   // 16 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (looked up once).
int scratch_address(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CHFSI_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return CHFSI_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return CHFSI_OK;
}

}  // namespace

int chfsi_filter_noalloc(const chfsi_matrix* H, const double* X, int64_t ldx, double* Y, int64_t ldy,
                         int64_t n_cols, int32_t m, double a, double b, double a0, const chfsi_schedule* sched,
                         void* stream) {
    size_t need = 0;
    int rc = chfsi_filter_workspace_size(H, n_cols, m, sched, &need);
    if (rc != CHFSI_OK) return rc;
    if (need > kNoallocScratchBytes) return CHFSI_ERR_NOMEM;   // problem larger than the static scratch
    void* ws = nullptr;
    if ((rc = scratch_address(&ws)) != CHFSI_OK) return rc;
    // chfsi_filter clears the status word at the start of the call; the iterate
    // buffers need no clearing (every element read is written first).
    return chfsi_filter(H, X, ldx, Y, ldy, n_cols, m, a, b, a0, sched, ws, kNoallocScratchBytes, stream);
}

int chfsi_filter_noalloc_read_status(void* stream) {
    void* ws = nullptr;
    const int rc = scratch_address(&ws);
    if (rc != CHFSI_OK) return rc;
    return chfsi_read_status(ws, stream);
}
