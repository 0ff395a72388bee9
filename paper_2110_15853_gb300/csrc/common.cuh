// Shared device/host helpers of the chfsi library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stddef.h>

#include "chfsi.h"

namespace chfsi {

// Bits of the device status word kept in the first 256 bytes of every workspace.
enum : unsigned {
    DEV_NONFINITE = 1u << 0,
    DEV_PATTERN = 1u << 1,
    DEV_CHOL = 1u << 2,
    DEV_TIMEOUT = 1u << 3,
};

constexpr size_t kStatusBytes = 256;
constexpr size_t kAlign = 256;

inline size_t align_up(size_t x, size_t a = kAlign) { return (x + a - 1) / a * a; }

// Carves a caller-provided workspace into aligned sub-buffers.
struct Arena {
    char* base;
    size_t cap;
    size_t used;
    Arena(void* p, size_t bytes) : base(static_cast<char*>(p)), cap(bytes), used(0) {}
    template <typename T>
    T* take(size_t count) {
        size_t off = align_up(used);
        used = off + align_up(count * sizeof(T));
        if (!base) return nullptr;
        return reinterpret_cast<T*>(base + off);
    }
    bool ok() const { return used <= cap; }
};

// Size-only twin of Arena.
struct Sizer {
    size_t used = 0;
    template <typename T>
    void take(size_t count) { used = align_up(used) + align_up(count * sizeof(T)); }
};

inline unsigned* status_word(void* ws) { return static_cast<unsigned*>(ws); }

// Kernel attributes (dynamic shared memory limits) are set once per device.
constexpr int kMaxDevices = 64;
inline int current_device() {
    int d = -1;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices) return -1;
    return d;
}

__device__ __forceinline__ void raise_status(unsigned* st, unsigned bits) {
    if (st) atomicOr(st, bits);
}

template <typename T> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float2; };

__device__ __forceinline__ bool finite_d(double x) { return isfinite(x); }

}  // namespace chfsi

#define CHFSI_CUDA_TRY(expr)                                   \
    do {                                                       \
        cudaError_t _e = (expr);                               \
        if (_e != cudaSuccess) return CHFSI_ERR_CUDA;          \
    } while (0)

namespace chfsi {
// Counts kernel launches issued by the library (diagnostics; see chfsi_kernel_launches).
void note_launch();
}

// Every kernel launch in the library is followed by exactly one CHFSI_LAUNCH_CHECK.
#define CHFSI_LAUNCH_CHECK()                                   \
    do {                                                       \
        ::chfsi::note_launch();                                \
        cudaError_t _e = cudaGetLastError();                   \
        if (_e != cudaSuccess) return CHFSI_ERR_CUDA;          \
    } while (0)
