// Helpers shared by the library's 5th-generation tensor-core kernels (sm_103a):
// mbarrier waits with a time limit, TMA tile loads, tcgen05 commit and shared-memory
// matrix descriptors, and the host-side tensor-map encoder.
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace chfsi {
namespace tc {

__device__ __forceinline__ uint32_t sa(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtime() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Limit of the waits that drain a CTA's own copies and MMAs before it exits: they
// end by themselves once the hardware finishes, so they keep this bound whatever the
// pipeline limit (chfsi_set_pipeline_wait_limit) is.
constexpr uint64_t kDrainNs = 1000000000ull;

// Wait for the phase of `parity` on an mbarrier for at most `limit_ns`; false on
// timeout.  The clock is read every 1024 polls so that a completed phase is seen at
// once; limits below a millisecond (the short limits of the abort-path tests) read
// it at every poll.
__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity, uint64_t limit_ns) {
    const uint32_t mask = limit_ns < 1000000ull ? 0u : 1023u;
    uint64_t t0 = 0;
    for (uint32_t polls = 1;; polls++) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done) : "r"(addr), "r"(parity) : "memory");
        if (done) return true;
        if ((polls & mask) == 0) {
            const uint64_t now = gtime();
            if (t0 == 0) t0 = now;
            else if (now - t0 > limit_ns) return false;
        }
    }
}

__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(sa(b)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(sa(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(sa(b)), "r"(bytes) : "memory");
}
// Arrive on the mbarrier once every tcgen05 operation this thread issued before has completed.
__device__ __forceinline__ void umma_commit(uint64_t* b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(sa(b))
                 : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        :: "r"(dst), "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar) : "memory");
}

// UMMA shared-memory descriptor of a K-major operand tile written by TMA with a
// 128-byte (rows of 64 BF16, 8-row atoms of 1024 B), 64-byte (rows of 32 BF16, atoms of
// 512 B) or 32-byte (rows of 16 BF16, atoms of 256 B) swizzle.
__device__ __forceinline__ uint64_t desc_kmajor(uint32_t addr, int swizzle_bytes) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);                      // start address
    d |= (uint64_t)1 << 16;                                      // leading byte offset (unused when swizzled)
    d |= (uint64_t)((8 * swizzle_bytes) >> 4) << 32;             // stride byte offset: one 8-row atom
    d |= (uint64_t)1 << 46;                                      // descriptor version
    const uint64_t layout = swizzle_bytes == 128 ? 2 : (swizzle_bytes == 64 ? 4 : 6);
    d |= layout << 61;                                           // swizzle mode
    return d;
}

// tcgen05.mma kind::f16 instruction descriptor: BF16 x BF16 -> FP32, A and B K-major,
// M x N tile.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// 2-D BF16 tensor map over a row-major [rows x cols] array with a [box_rows x box_cols]
// box and the given swizzle (box_cols * 2 bytes must equal the swizzle width: 32, 64 or
// 128 bytes).
inline int make_map_bf16(CUtensorMap* map, const void* base, int64_t cols, int64_t rows, int box_cols, int box_rows,
                         CUtensorMapSwizzle swizzle) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return CHFSI_ERR_CUDA;
    if ((reinterpret_cast<uintptr_t>(base) & 15u) || ((cols * 2) % 16)) return CHFSI_ERR_ARG;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? CHFSI_OK : CHFSI_ERR_CUDA;
}

inline int sm_count() {
    static int cache[kMaxDevices] = {};
    const int dev = current_device();
    if (dev < 0) return 0;
    if (!cache[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        cache[dev] = v;
    }
    return cache[dev];
}

}  // namespace tc
}  // namespace chfsi
