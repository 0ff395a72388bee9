// BSR filter step on the 5th-generation tensor cores (tcgen05, BF16 operands,
// FP32 accumulation in tensor memory), for the low-precision prefix of the
// filter schedule (Algorithm 1 step 1, Sec. 3.4; the dense-block treatment of H
// follows the dense diagonal blocks of Sec. 4.1-4.2):
//
//     Y_out[R] = alpha (sum_{(R,C)} H_RC Y_cur[C] - c Y_cur[R]) - beta Y_prev[R]
//
// computed transposed, so that both MMA operands are K-major.  A work item is a pair
// of block rows (R0 = 2p, R1 = 2p + 1; 128 grid points) and a span of 256 states, two
// tiles of 128 states j:
//     D_u[j][i] = sum_C sum_k Ysh^T[j][C*64 + k] * [H_R0C; H_R1C][i][k]   (M = 128, N = 128, K = 64/block)
// over the merged block columns C of the two rows (a block missing from one row is a
// zero block).  Ysh^T is the BF16 copy of Y_cur, stored block-major as [N/64][n][64]
// so that the 128 x 64 operand tile of block column C and a state tile is one
// contiguous 16 KB read.  Pairing the rows doubles the work of every MMA instruction
// (with one 64-row block per MMA the single issuing thread limited the step), and the
// two state tiles of an item share each stage's pair of H blocks, so that a stage
// moves 48 KB into shared memory for the work that took 64 KB in two stages of one
// tile.  The epilogue reads D from TMEM, applies the recurrence in FP32 against the
// FP32 iterates and writes Y_out (FP32, row-major) plus its BF16 block-major copy for
// the next step.
//
// Persistent, warp-specialised CTA (one per SM), looping over work items with the
// state spans fastest (a pair's H blocks are then shared through L2 by its spans):
//   warp 0, lane 0 : TMA producer of the MMA operands -- per merged block column, the
//                    two 128B-swizzled Ysh^T tiles and the two H blocks into a 4-stage
//                    ring, with per-stage flags (first / last / empty item) for the issuer;
//   warp 1         : owns the TMEM allocation (all 512 columns: two items of two
//                    128-column FP32 accumulators); lane 0 issues the MMAs;
//   warp 2, lane 0 : TMA producer of each item's FP32 Y_cur / Y_prev epilogue tiles,
//                    8 rows x 256 states at a time into a two-deep ring;
//   warps 3-6      : epilogue (warp w reads TMEM lanes 32*(w%4)..+31) of one item
//                    while the MMAs of the next one run.
// Every mbarrier wait is bounded on %globaltimer.  A wait of one role on another
// (a stage, an accumulator, an epilogue chunk) gives up after the pipeline limit
// (1 s, shorter only when a test sets chfsi_set_pipeline_wait_limit); the CTA then
// flags DEV_TIMEOUT, stops issuing work, waits for its own copies and MMAs in flight
// (those drains keep a fixed 1 s bound: they end as soon as the hardware does), frees
// TMEM and exits.
#include <cuda.h>

#include "common.cuh"
#include "kernels.cuh"
#include "tcgen05.cuh"

namespace chfsi {

namespace {

// Block rows per work item.  Two double the work per MMA instruction over one; four
// (N = 256, both 256-column accumulators filling TMEM) measured slower at 40^3 with
// 1024 states (0.345 against 0.333 ms per step): 54 merged block columns per quad
// carry 50% zero blocks and the ring holds only 4 of its 48 KB stages.
constexpr int kRowsPerItem = 2;
// State tiles per work item: the tiles of an item share every stage's H blocks, so a
// stage carries kTiles operand tiles and one pair of H blocks.  Two tiles (4 stages of
// 48 KB, TMEM full) measured 0.277 ms per step at 40^3 with 1024 states against 0.333
// ms for one (6 stages of 32 KB).
constexpr int kTiles = 2;
constexpr int kTileJ = 128;                       // states per MMA (M)
constexpr int kItemJ = kTiles * kTileJ;           // states per work item
constexpr int kBlk = 64;                          // block edge (K per block; rows per block row)
constexpr int kRowsN = kRowsPerItem * kBlk;       // rows per item (MMA N)
constexpr int kATile = kTileJ * kBlk * 2;         // 16 KB
constexpr int kBTile = kRowsN * kBlk * 2;         // one H block per row of the item
constexpr int kStageBytes = kTiles * kATile + kBTile;
constexpr int kStages = (192 * 1024) / kStageBytes;
constexpr int kEpiRows = kTiles == 1 ? 16 : 8;    // rows per epilogue chunk
constexpr int kEpiChunks = kRowsN / kEpiRows;     // chunks per item
constexpr int kEpiTile = kEpiRows * kItemJ * 4;   // 8 KB: kEpiRows rows x kItemJ states FP32
constexpr int kEpiSlot = 2 * kEpiTile;            // Y_cur + Y_prev chunk
constexpr int kSmemBytes = kStages * kStageBytes + 2 * kEpiSlot + 1024;
constexpr int kThreads = 224;
constexpr uint32_t kAccCols = kTiles * kRowsN;    // TMEM columns of one item's accumulators
constexpr uint32_t kTmemCols = 2 * kAccCols;      // two items in flight
static_assert(kTmemCols <= 512 && kEpiRows % 8 == 0 && kBlk % kEpiRows == 0, "tile shape");
static_assert(kSmemBytes + 1024 <= 227 * 1024, "shared memory per CTA (with the static barriers)");
// per-stage flags written by the operand producer for the MMA issuer
constexpr int kFirst = 1, kLast = 2, kEmptyItem = 4;
using namespace tc;

// Instruction descriptor: kind::f16, BF16 x BF16 -> FP32, both K-major, M = 128 states, N = 128 rows.
constexpr uint32_t kIdesc = idesc_bf16(kTileJ, kRowsN);

// kEpiRows consecutive accumulator columns of this warp's 32 TMEM lanes (one per lane).
__device__ __forceinline__ void tmem_ld_chunk(uint32_t taddr, uint32_t (&r)[kEpiRows]) {
    static_assert(kEpiRows == 8 || kEpiRows == 16, "epilogue chunk of 8 or 16 rows");
    if constexpr (kEpiRows == 16) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
            "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
              "=r"(r[15])
            : "r"(taddr));
    } else {
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                       "=r"(r[7])
                     : "r"(taddr));
    }
}

__global__ void __launch_bounds__(kThreads, 1)
bsr_tc_kernel(const __grid_constant__ CUtensorMap tmY, const __grid_constant__ CUtensorMap tmH,
              const __grid_constant__ CUtensorMap tmYc, const __grid_constant__ CUtensorMap tmYp, int has_prev,
              int64_t nbr, const int32_t* __restrict__ brow_ptr, const int32_t* __restrict__ bcol, int64_t nblocks,
              int64_t N, int64_t n, int64_t nspans, float* __restrict__ Yo, int64_t ldo,
              // the BF16 block table holds a zero block at index nblocks (the missing block of a pair)
              __nv_bfloat16* __restrict__ Ysh_out, float alpha, float c, float beta, uint64_t wait_ns,
              unsigned* status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* stages = smem;                                   // kStages x (A | B), 1024-aligned
    unsigned char* epi = smem + kStages * kStageBytes;              // 2 x (Y_cur chunk | Y_prev chunk)
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages], tfull[2], tempty[2], efull[2], eempty[2];
    __shared__ int stage_flags[kStages];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ngroups = (nbr + kRowsPerItem - 1) / kRowsPerItem;
    const int64_t total = ngroups * nspans;   // work items: (block-row group, span of kItemJ states)
    bool bad = false;
    // state tiles of span sp that hold states < n (the last span may hold fewer than kTiles)
    auto tiles_of = [&](int64_t sp) -> int {
        const int64_t left = (n - sp * kItemJ + kTileJ - 1) / kTileJ;
        return left < kTiles ? (int)left : kTiles;
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 4);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&efull[b], 1);
            mbar_init(&eempty[b], 4);
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
        asm volatile("fence.proxy.async.shared::cta;");
        abort_flag = 0;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(sa(&tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_slot;
    volatile int* abort_v = &abort_flag;

    // block range of a block row, clamped to the stored blocks (empty past the last row)
    auto blocks_of = [&](int64_t R, int& qb, int& qe) {
        if (R >= nbr) { qb = qe = 0; return; }
        qb = brow_ptr[R];
        qe = brow_ptr[R + 1];
        if (qb < 0) { qb = 0; bad = true; }
        if (qe > nblocks) { qe = (int)nblocks; bad = true; }
        if (qe < qb) { qe = qb; bad = true; }
    };

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer of the MMA operands
        int64_t sc = 0;                 // stages issued
        // next stage: wait until the issuer has released it, then set its flags
        auto acquire = [&](int flags) -> int {
            const int s = (int)(sc % kStages), u = (int)(sc / kStages);
            if (u >= 1 && !mbar_wait(sa(&empty[s]), (u - 1) & 1, wait_ns)) return -1;
            stage_flags[s] = flags;
            return s;
        };
        for (int64_t item = blockIdx.x; item < total && !*abort_v; item += gridDim.x) {
            const int64_t R0 = kRowsPerItem * (item / nspans), sp = item % nspans;
            const int nt = tiles_of(sp);
            int pos[kRowsPerItem], end[kRowsPerItem];
            bool any = false;
#pragma unroll
            for (int r = 0; r < kRowsPerItem; r++) {
                blocks_of(R0 + r, pos[r], end[r]);
                any |= pos[r] < end[r];
            }
            bool ok = true, first = true;
            if (!any) {   // no block in any row: an empty stage tells the issuer
                const int s = acquire(kFirst | kLast | kEmptyItem);
                if (s < 0) { *abort_v = 1; break; }
                mbar_arrive(&full[s]);
                sc++;
                continue;
            }
            // merge the rows' block columns: each step takes the smallest head column and
            // every row whose head holds it (each stored block exactly once, sorted or not)
            for (;;) {
                int C = INT32_MAX;
#pragma unroll
                for (int r = 0; r < kRowsPerItem; r++)
                    if (pos[r] < end[r]) { const int c = bcol[pos[r]]; C = c < C ? c : C; }
                int q[kRowsPerItem];
                bool more = false;
#pragma unroll
                for (int r = 0; r < kRowsPerItem; r++) {
                    q[r] = (int)nblocks;                         // the zero block
                    if (pos[r] < end[r] && bcol[pos[r]] == C) q[r] = pos[r]++;
                    more |= pos[r] < end[r];
                }
                if (C < 0 || (int64_t)C >= nbr) { bad = true; C = 0; }   // zero-safe: still a valid tile
                const int s = acquire((first ? kFirst : 0) | (more ? 0 : kLast));
                if (s < 0) { ok = false; break; }
                first = false;
                const uint32_t st = sa(stages + (size_t)s * kStageBytes);
                mbar_expect_tx(&full[s], nt * kATile + kBTile);
                for (int u = 0; u < nt; u++)
                    tma_load_2d(st + u * kATile, &tmY, 0, (int)(C * n + sp * kItemJ + u * kTileJ), sa(&full[s]));
#pragma unroll
                for (int r = 0; r < kRowsPerItem; r++)
                    tma_load_2d(st + kTiles * kATile + r * (kBlk * kBlk * 2), &tmH, 0, q[r] * kBlk, sa(&full[s]));
                sc++;
                if (!more) break;
            }
            if (!ok) { *abort_v = 1; break; }
        }
        // wait (bounded) until every copy this thread issued has landed
        for (int s = 0; s < kStages && s < sc; s++) {
            const int64_t last = s + ((sc - 1 - s) / kStages) * kStages;
            mbar_wait(sa(&full[s]), (int)(last / kStages) & 1, kDrainNs);
        }
    } else if (warp == 2 && lane == 0) {
        // ---------------- TMA producer of the epilogue operand chunks
        // chunk g (= item count x kEpiChunks + chunk) goes to slot g & 1, its use g >> 1
        int64_t g = 0;
        for (int64_t item = blockIdx.x; item < total && !*abort_v; item += gridDim.x) {
            const int64_t R0 = kRowsPerItem * (item / nspans), sp = item % nspans;
            bool ok = true;
            for (int ch = 0; ch < kEpiChunks; ch++, g++) {
                const int slot = (int)(g & 1);
                const int64_t use = g >> 1;
                if (use >= 1 && !mbar_wait(sa(&eempty[slot]), (int)((use - 1) & 1), wait_ns)) { ok = false; break; }
                const uint32_t dst = sa(epi + slot * kEpiSlot);
                int64_t row64 = R0 * kBlk + ch * kEpiRows;
                if (row64 >= N) row64 = R0 * kBlk;   // rows past the last block row: not used
                const int row = (int)row64;
                mbar_expect_tx(&efull[slot], has_prev ? 2 * kEpiTile : kEpiTile);
                tma_load_2d(dst, &tmYc, (int)(sp * kItemJ), row, sa(&efull[slot]));
                if (has_prev) tma_load_2d(dst + kEpiTile, &tmYp, (int)(sp * kItemJ), row, sa(&efull[slot]));
            }
            if (!ok) { *abort_v = 1; break; }
        }
        // wait (bounded) until the last copy into each slot has landed
        for (int64_t last = g - 1; last >= 0 && last >= g - 2; last--)
            mbar_wait(sa(&efull[last & 1]), (int)((last >> 1) & 1), kDrainNs);
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer
        int64_t sc = 0;
        int items = 0;
        for (int64_t item = blockIdx.x; item < total && !*abort_v; item += gridDim.x, items++) {
            const int b = items & 1, v = items >> 1;
            if (v >= 1 && !mbar_wait(sa(&tempty[b]), (v - 1) & 1, wait_ns)) { *abort_v = 1; break; }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t acc_addr = tmem + (uint32_t)(b * kAccCols);   // tile u at + u * kRowsN
            const int nt = tiles_of(item % nspans);
            bool ok = true;
            for (;; sc++) {
                const int s = (int)(sc % kStages), u = (int)(sc / kStages);
                if (!mbar_wait(sa(&full[s]), u & 1, wait_ns) || *abort_v) { *abort_v = 1; ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const int flags = stage_flags[s];
                if (!(flags & kEmptyItem)) {
                    const uint32_t st = sa(stages + (size_t)s * kStageBytes);
                    const uint64_t db = desc_kmajor(st + kTiles * kATile, 128);
#pragma unroll
                    for (int u = 0; u < kTiles; u++) {
                        if (u >= nt) break;
                        const uint64_t da = desc_kmajor(st + u * kATile, 128);
#pragma unroll
                        for (int k = 0; k < kBlk / 16; k++) {
                            const uint32_t accumulate = ((flags & kFirst) && k == 0) ? 0u : 1u;
                            asm volatile(
                                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
                                :: "r"(acc_addr + (uint32_t)(u * kRowsN)), "l"(da + 2 * k), "l"(db + 2 * k),
                                   "r"(kIdesc), "r"(accumulate));
                        }
                    }
                }
                umma_commit(&empty[s]);
                if (flags & kLast) { sc++; break; }
            }
            umma_commit(&tfull[b]);   // accumulator b complete (also for an empty item)
            if (!ok) { items++; break; }
        }
        // every MMA this thread issued has completed before TMEM is released
        if (items > 0) {
            const int lb = (items - 1) & 1, lv = (items - 1) >> 1;
            mbar_wait(sa(&tfull[lb]), lv & 1, kDrainNs);
        }
    } else if (warp >= 3) {
        // ---------------- epilogue
        const int quad = warp & 3;
        int items = 0;
        for (int64_t item = blockIdx.x; item < total; item += gridDim.x, items++) {
            const int64_t R0 = kRowsPerItem * (item / nspans), sp = item % nspans;
            const int b = items & 1, v = items >> 1;
            // the warp decides together (the TMEM loads below are warp-collective)
            const bool ok = __all_sync(0xffffffffu, !*abort_v && mbar_wait(sa(&tfull[b]), v & 1, wait_ns));
            if (!ok) { *abort_v = 1; break; }
            asm volatile("tcgen05.fence::after_thread_sync;");
            bool has_acc = false;                                 // else no MMA wrote the accumulator
            for (int r = 0; r < kRowsPerItem; r++) {
                int qb, qe;
                blocks_of(R0 + r, qb, qe);
                has_acc |= qe > qb;
            }
            const int jl = quad * 32 + lane;                      // state within each tile
            const int64_t row0 = R0 * kBlk;
            bool nonfinite = false;
            bool chunks_ok = true;
#pragma unroll 1
            for (int cchunk = 0; cchunk < kEpiChunks; cchunk++) {
                const int64_t g = (int64_t)items * kEpiChunks + cchunk;
                const int slot = (int)(g & 1);
                if (!__all_sync(0xffffffffu, mbar_wait(sa(&efull[slot]), (int)((g >> 1) & 1), wait_ns))) {
                    chunks_ok = false;
                    break;
                }
                const float* ycs = reinterpret_cast<const float*>(epi + slot * kEpiSlot);   // [kEpiRows][kItemJ]
                const float* yps = ycs + kEpiRows * kItemJ;
                uint32_t r[kTiles][kEpiRows];
                const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * kAccCols + cchunk * kEpiRows);
#pragma unroll
                for (int u = 0; u < kTiles; u++) tmem_ld_chunk(taddr + (uint32_t)(u * kRowsN), r[u]);
                asm volatile("tcgen05.wait::ld.sync.aligned;");
                const int64_t rowc = row0 + cchunk * kEpiRows;    // first row of the chunk
                const int64_t Rr = R0 + cchunk / (kBlk / kEpiRows);   // its block row
#pragma unroll
                for (int u = 0; u < kTiles; u++) {
                    const int64_t j = sp * kItemJ + u * kTileJ + jl;
                    if (j >= n || rowc >= N) continue;
                    const int js = u * kTileJ + jl;               // state within the chunk tile
                    float out[kEpiRows];
#pragma unroll
                    for (int tt = 0; tt < kEpiRows; tt++) {
                        const float acc = has_acc ? __uint_as_float(r[u][tt]) : 0.0f;
                        float val = alpha * fmaf(-c, ycs[tt * kItemJ + js], acc);
                        if (has_prev) val = fmaf(-beta, yps[tt * kItemJ + js], val);
                        nonfinite |= !isfinite(val);
                        Yo[(rowc + tt) * ldo + j] = val;
                        out[tt] = val;
                    }
                    // kEpiRows consecutive rows of state j -> 16-byte stores of the block-major copy
                    uint4 pk[kEpiRows / 8];
                    unsigned* pw = reinterpret_cast<unsigned*>(pk);
#pragma unroll
                    for (int tt = 0; tt < kEpiRows / 2; tt++) {
                        __nv_bfloat162 h2 = __floats2bfloat162_rn(out[2 * tt], out[2 * tt + 1]);
                        pw[tt] = *reinterpret_cast<unsigned*>(&h2);
                    }
                    uint4* dst = reinterpret_cast<uint4*>(Ysh_out + (Rr * n + j) * kBlk +
                                                          (cchunk % (kBlk / kEpiRows)) * kEpiRows);
#pragma unroll
                    for (int w = 0; w < kEpiRows / 8; w++) dst[w] = pk[w];
                }
                // release the chunk slot
                __syncwarp();
                if (lane == 0) mbar_arrive(&eempty[slot]);
            }
            if (!chunks_ok) { *abort_v = 1; break; }
            if (nonfinite) raise_status(status, DEV_NONFINITE);
            // release accumulator b
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[b]);
        }
    }

    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTmemCols));
    }
    if (threadIdx.x == 0 && abort_flag) raise_status(status, DEV_TIMEOUT);
    if (bad) raise_status(status, DEV_PATTERN);
}

// BF16 copy of FP64 block values (rounded through FP32), followed by one zero block
// (the stand-in for a block missing from one row of a block-row pair).
__global__ void blocks_to_bf16_kernel(const double* __restrict__ src, __nv_bfloat16* dst, int64_t count) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) dst[i] = __float2bfloat16_rn((float)src[i]);
    else if (i < count + kBlk * kBlk) dst[i] = __float2bfloat16_rn(0.0f);
}

// Block-major BF16 copy of a row-major FP64 block:
//     dst[((r / 64) * n + j) * 64 + r % 64] = bf16(src[r * lds + j]).
__global__ void transpose_to_bf16_kernel(const double* __restrict__ src, int64_t lds, __nv_bfloat16* dst, int64_t N,
                                         int64_t n) {
    __shared__ float t[32][33];
    const int64_t r0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t r = r0 + k, j = j0 + threadIdx.x;
        t[k][threadIdx.x] = (r < N && j < n) ? (float)src[r * lds + j] : 0.0f;
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t j = j0 + k, r = r0 + threadIdx.x;
        if (j < n && r < N) dst[((r / kBlk) * n + j) * kBlk + (r % kBlk)] = __float2bfloat16_rn(t[threadIdx.x][k]);
    }
}

// 2-D BF16 tensor map over a row-major [rows x cols] array, box [box_rows x 64],
// 128-byte swizzle (MMA operand tiles).
int make_map(CUtensorMap* map, const void* base, int64_t cols, int64_t rows, int box_rows) {
    return make_map_bf16(map, base, cols, rows, 64, box_rows, CU_TENSOR_MAP_SWIZZLE_128B);
}

// 2-D FP32 tensor map over a row-major [rows x ld] array, box [kEpiRows rows x kItemJ
// states], no swizzle (epilogue operand chunks; states beyond ld read as zero).
int make_map_f32(CUtensorMap* map, const float* base, int64_t ld, int64_t rows) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return CHFSI_ERR_CUDA;
    if ((reinterpret_cast<uintptr_t>(base) & 15u) || ((ld * 4) % 16)) return CHFSI_ERR_ARG;
    cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
    cuuint32_t box[2] = {(cuuint32_t)kItemJ, (cuuint32_t)kEpiRows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? CHFSI_OK : CHFSI_ERR_CUDA;
}

}  // namespace

int bsr_values_to_bf16(const double* src, void* dst, int64_t count, cudaStream_t s) {
    if (count <= 0) return CHFSI_OK;
    const int64_t total = count + kBlk * kBlk;
    blocks_to_bf16_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(src, static_cast<__nv_bfloat16*>(dst),
                                                                         count);
    CHFSI_LAUNCH_CHECK();
    return CHFSI_OK;
}

int transpose_to_bf16(const double* src, int64_t lds, void* dst, int64_t N, int64_t n, cudaStream_t s) {
    if (N <= 0 || n <= 0) return CHFSI_OK;
    dim3 grid((unsigned)((N + 31) / 32), (unsigned)((n + 31) / 32));
    transpose_to_bf16_kernel<<<grid, dim3(32, 8), 0, s>>>(src, lds, static_cast<__nv_bfloat16*>(dst), N, n);
    CHFSI_LAUNCH_CHECK();
    return CHFSI_OK;
}

// One BF16-operand BSR step on the tensor cores.  h.val must point at BF16
// blocks; ysh_in / ysh_out are state-major (n x N) BF16 copies of Y_cur / Y_out.
int bsr_step_tc(const BsrDev& h, int64_t n, const void* ysh_in, const float* Yc, int64_t ldc, const float* Yp,
                int64_t ldp, float* Yo, int64_t ldo, void* ysh_out, double alpha, double c, double beta,
                unsigned* status, cudaStream_t s) {
    if (n <= 0 || h.nbr <= 0) return CHFSI_OK;
    if (h.bdim != kBlk || h.val_t != Buf::BF16) return CHFSI_ERR_UNSUPPORTED;
    const int64_t N = h.nbr * kBlk;
    if ((h.nblocks + 1) * kBlk > INT32_MAX || N > INT32_MAX || n > INT32_MAX || h.nbr * n + kItemJ > INT32_MAX)
        return CHFSI_ERR_UNSUPPORTED;
    CUtensorMap tmY, tmH, tmYc, tmYp;
    int rc;
    if ((rc = make_map(&tmY, ysh_in, kBlk, h.nbr * n, kTileJ))) return rc;
    if ((rc = make_map(&tmH, h.val, kBlk, (h.nblocks + 1) * kBlk, kBlk))) return rc;   // + the zero block
    if ((rc = make_map_f32(&tmYc, Yc, ldc, N))) return rc;
    if (Yp) {
        if ((rc = make_map_f32(&tmYp, Yp, ldp, N))) return rc;
    } else {
        tmYp = tmYc;   // not read
    }
    const int dev = current_device();
    if (dev < 0) return CHFSI_ERR_CUDA;
    static bool attr[kMaxDevices] = {};
    if (!attr[dev]) {
        CHFSI_CUDA_TRY(cudaFuncSetAttribute(bsr_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
        attr[dev] = true;
    }
    const int64_t nspans = (n + kItemJ - 1) / kItemJ;
    const int64_t total = (h.nbr + kRowsPerItem - 1) / kRowsPerItem * nspans;
    const int sms = sm_count();
    if (sms <= 0) return CHFSI_ERR_CUDA;
    const unsigned grid = (unsigned)(total < sms ? total : sms);   // persistent: one CTA per SM
    bsr_tc_kernel<<<grid, kThreads, kSmemBytes, s>>>(tmY, tmH, tmYc, tmYp, Yp ? 1 : 0, h.nbr, h.brow_ptr, h.bcol,
                                                     h.nblocks, N, n, nspans, Yo, ldo,
                                                     static_cast<__nv_bfloat16*>(ysh_out), (float)alpha, (float)c,
                                                     (float)beta, pipeline_wait_ns(), status);
    CHFSI_LAUNCH_CHECK();
    return CHFSI_OK;
}

}  // namespace chfsi
