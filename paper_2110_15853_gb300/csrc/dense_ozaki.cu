// FP64-accurate dense products on the BF16 tensor cores (Ozaki-scheme splitting),
// for the large products of the ChFSI closure (Algorithm 1 steps 2, 3 and 5,
// Sec. 3.4): the Gram matrix Y^T Y of the Cholesky-QR, X_F = Y R^-1, the projection
// X_F^T (H X_F) and the rotation X_F Q.  GB300's FP64 pipe runs about 1.2 TFLOP/s;
// its BF16 tensor cores about 1.9 PFLOP/s.
//
// Splitting.  The product is C = A_hat B_hat^T with both operands K-major: for
// C = A^T B (Gram form) A_hat = A^T, B_hat = B^T; for C = A B, A_hat = A, B_hat =
// B^T.  Each row r of an operand gets a power-of-two scale 2^{e_r} with
// |A_hat[r][k]| 2^{-e_r} < 1/2 for all k, and the scaled value a is rounded to a
// 56-bit fixed-point number and written as seven balanced base-256 digits
//     a = sum_{t=1..7} d_t 2^{-8t},   d_t integer, |d_t| <= 128,
// (integer arithmetic on the FP64 bit pattern; no FP64 instructions).  Slice t
// stores d_t 2^{-8t} in BF16, which is exact (8 significant bits).  Then
//     C_ij = 2^{e_i + f_j} sum_{t + u <= 8} sum_k a_t[i][k] b_u[j][k]
// keeps every digit product of weight 2^{-64} and above (28 slice pairs; the
// dropped pairs and the 56-bit rounding are below about 2^{-55} of the row scales
// per term, i.e. about 2^{-48} of a typical term).
//
// Exact accumulation.  A product of two slices is d_t g_u 2^{-8(t+u)}, an integer
// multiple of 2^{-8l} at level l = t + u with |d_t g_u| <= 2^14.  Every level l = 2 .. 8
// has its own FP32 accumulator E_l in TMEM, and each is drained before its sums can
// pass 2^24 units (levels 2-5 every 256 K, levels 6-8 every 128 K; at most 4 and 7
// pairs per level), so the tensor-core accumulation -- which truncates rather than
// rounds -- never rounds at all: the sums are exact integers.  The drains add them to
// two 64-bit integers per output element, levels 2-5 in units of 2^{-40} and levels
// 6-8 in units of 2^{-64}.  A work item spans at most 8192 K (longer sums are split
// over items and the FP64 partial tiles added), which bounds the integers by 2^51 and
// 2^46.  C = 2^{e_i + f_j} (2^{-40} hi + 2^{-64} lo), converted once at the end, so the
// only errors are the 56-bit rounding of the inputs and the dropped pairs (weights
// 2^{-72} and below).
//
// Five-slice steps.  A filter step may also use only the first five digits of each
// operand (a 40-bit fixed-point value, truncation below 2^{-41} of the row scale) and
// the 15 pairs of weight 2^{-48} and above (levels 2 .. 6): about 2^{-40} of the row
// scales per term, some 2^{16} times finer than FP32, for 15 slice products instead
// of 28 and three operand stages instead of two.  The digits are the same as above,
// so the same slices serve both step kinds.
//
// Kernel.  Persistent, warp-specialised, one CTA per SM, 128 x 64 output tiles; NS = 7
// slices per operand (or 5 for the 40-bit filter steps):
//   warp 0, lane 0 : TMA producer -- per K-block of 32, the NS A (128-row) and NS B
//                    (64-row) slice tiles (64-byte swizzle) into a ring of two stages
//                    (84 KB each) or, with five slices, three (60 KB each);
//   warp 1         : owns 512 TMEM columns, NS 64-column FP32 accumulators E2 .. E_{NS+1};
//                    lane 0 issues the slice-pair products of a stage as 11 (or 9) MMAs
//                    of M = 128, N = 64 c (B slices stacked), K = 16, twice per K-block;
//   warps 2-17     : epilogue; warp w reads TMEM lanes 32 (w % 4) .. + 31 (one output
//                    row per thread), columns 16 ((w - 2) / 4) .. + 15, and keeps those
//                    16 x 2 integers in registers.
// Drains alternate between group X (E2 .. E5, after K-blocks 5, 13, 21, ...) and group
// Y (E6 .., after K-blocks 3, 7, 11, ...); the issuer runs the other group's MMAs of
// the next stage before it waits for a drain.  Every mbarrier wait is bounded; on a
// timeout the CTA flags DEV_TIMEOUT, stops, waits (bounded) for its copies and MMAs in
// flight, frees TMEM and exits.
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"
#include "tcgen05.cuh"

namespace chfsi {

namespace {

using namespace tc;

constexpr int kSlices = 7;                            // digit planes stored per operand
constexpr int kTileM = 128;                           // output rows per tile (TMEM lanes)
constexpr int kTileN = 64;                            // output columns per tile
constexpr int kRowPad = 128;                          // operand rows are padded to this
// K per stage (a K-block): 32 BF16 = 64-byte rows under the 64-byte swizzle; a stage of
// 7 + 7 slice tiles is 84 KB and two fit in shared memory.  K-blocks of 16 (32-byte
// swizzle, 42 KB stages, five of them) measured slower: 114.7 against 98.4 ms for the
// 20-step BSR filter at 40^3 with 1024 states, since the MMAs of one group that overlap
// the other group's drain halve with the stage.
constexpr int kKB = 32;
constexpr int kSwizzleBytes = 2 * kKB;
constexpr int kMaxItemKB = 8192 / kKB;                // K-blocks per work item (8192 K)
constexpr int kBlockKB = 64 / kKB;                    // K-blocks per 64-wide BSR block
constexpr int kSliceA = kTileM * kKB * 2;             // 8 KB
constexpr int kSliceB = kTileN * kKB * 2;             // 4 KB
constexpr int kPeriodX = 256 / kKB;                   // K-blocks between drains of group X (256 K)
constexpr int kPeriodY = 128 / kKB;                   // K-blocks between drains of group Y (128 K)
constexpr CUtensorMapSwizzle kTmaSwizzle = kKB == 16 ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_64B;
constexpr int kEpiWarps = 16;
constexpr int kColsPerThread = kTileN / (kEpiWarps / 4);   // 16
constexpr int kThreads = 32 * (2 + kEpiWarps);
constexpr uint32_t kTmemCols = 512;
constexpr int kMaxStages = 3;
constexpr int kXEvent = 1, kYEvent = 2, kFullEvent = 3;
static_assert(kSliceB % (8 * kSwizzleBytes) == 0, "swizzle-atom alignment of the tiles");
static_assert(kKB == 16 || kKB == 32, "K-block of one or two 16-wide MMA steps");
static_assert(kColsPerThread == 16, "16-column TMEM loads");

// Shape of a product with NS digit slices per operand (7: FP64-accurate; 5: the
// 40-bit steps): a stage holds NS A and NS B slice tiles; levels 2 .. NS + 1 each have
// an accumulator (E2 .. E_{NS+1}), group X = E2 .. E5, group Y = the rest.
template <int NS>
struct OzShape {
    static constexpr int kStageBytes = NS * (kSliceA + kSliceB);
    static constexpr int kStages = (224 * 1024) / kStageBytes;
    static constexpr int kSmemBytes = kStages * kStageBytes + 1024;
    static constexpr int kAccs = NS;
    static constexpr int kMmas = NS == 7 ? 11 : 9;
    static_assert(NS == 7 || NS == 5, "seven or five slices");
    static_assert(kStages >= 2 && kStages <= kMaxStages, "two or three operand stages");
    static_assert(kSmemBytes + 1024 <= 227 * 1024, "shared memory per CTA");
    static_assert(kAccs * kTileN <= (int)kTmemCols, "accumulators in TMEM");
    static_assert(kStageBytes % 1024 == 0, "swizzle-atom alignment of the stages");
};

// The 28 slice pairs (t, u), 0-based, with t + u <= 6 go to accumulator t + u (level
// t + u + 2).  For one slice t of A, the slices u of B that fall into one accumulator
// group are consecutive, and so are their accumulators, so they run as one MMA with the
// B slices stacked along N (N = 64 c <= 256): 4 MMAs for group X (accumulators 0-3,
// E2 .. E5) and 7 for group Y (accumulators 4-6, E6 .. E8), 11 per K-step instead of 28
// (fewer, wider MMAs: less shared-memory operand traffic per product).  The first MMA of
// each group has t = 0 and covers all of the group's accumulators.
// With five slices the 15 pairs with t + u <= 4 take the same 4 MMAs for group X and
// one MMA per pair of level 6 (accumulator 4, E6) for group Y: 9 per K-step.
// MMA q takes slice mma_t(q) of A and the mma_c(q) slices of B from mma_u(q) on:
//   seven slices: t = {0,1,2,3, 0,1,2,3,4,5,6}, u = {0,0,0,0, 4,3,2,1,0,0,0},
//                 c = {4,3,2,1, 3,3,3,3,3,2,1};
//   five slices:  t = {0,1,2,3, 0,1,2,3,4},     u = {0,0,0,0, 4,3,2,1,0},
//                 c = {4,3,2,1, 1,1,1,1,1}.
// Compile-time functions of q, so that the unrolled issue sequence folds them into
// immediate descriptor offsets (one thread issues every MMA; table loads and
// descriptor rebuilds per MMA made that thread the pace of the pipeline).
constexpr int kMmaX = 4;
__host__ __device__ constexpr int mma_t(int q) { return q < kMmaX ? q : q - kMmaX; }
__host__ __device__ constexpr int mma_u(int q) { return q < kMmaX ? 0 : (q <= 2 * kMmaX ? 2 * kMmaX - q : 0); }
template <int NS>
__host__ __device__ constexpr int mma_c(int q) {
    return q < kMmaX ? kMmaX - q : (NS == 5 ? 1 : (11 - q < 3 ? 11 - q : 3));
}
// Every pair (t, u) with t + u <= NS - 1 exactly once, accumulator t + u.
template <int NS>
constexpr bool mma_covers_pairs(int nmmas) {
    int seen[7][7] = {};
    for (int q = 0; q < nmmas; q++)
        for (int j = 0; j < mma_c<NS>(q); j++) {
            const int t = mma_t(q), u = mma_u(q) + j;
            if (t >= NS || u >= NS || t + u > NS - 1) return false;
            if ((q < kMmaX) != (t + u < kMmaX)) return false;   // groups X (E2 .. E5) and Y
            seen[t][u]++;
        }
    for (int t = 0; t < NS; t++)
        for (int u = 0; u < NS; u++)
            if (seen[t][u] != (t + u <= NS - 1 ? 1 : 0)) return false;
    return true;
}
static_assert(mma_covers_pairs<7>(11) && mma_covers_pairs<5>(9), "slice-pair tables");
static_assert(mma_t(10) == 6 && mma_u(9) == 0 && mma_c<7>(9) == 2 && mma_c<7>(8) == 3, "seven-slice table");

// The MMAs Q0 .. Q1 - 1 of one stage: A slices from descriptor da0, B slices from db0
// (descriptors of the stage's first A and first B tile; a tile's start address is
// da0 + offset / 16, which stays inside the 14-bit field below 256 KB).  The first MMA
// of a group (q = 0 for X, q = kMmaX for Y) covers all of the group's accumulators and
// overwrites them when the group starts fresh.
template <int NS, int Q0, int Q1>
__device__ __forceinline__ void issue_mmas(uint64_t da0, uint64_t db0, uint32_t tmem, bool freshX, bool freshY) {
#pragma unroll
    for (int q = Q0; q < Q1; q++) {
        const int t = mma_t(q), u0 = mma_u(q), c = mma_c<NS>(q);
        const bool fresh = (q == 0 && freshX) || (q == kMmaX && freshY);
        const uint64_t da = da0 + (uint64_t)((t * kSliceA) >> 4);
        const uint64_t db = db0 + (uint64_t)((u0 * kSliceB) >> 4);
        const uint32_t dt = tmem + (uint32_t)((t + u0) * kTileN);
        constexpr uint32_t kIdesc1 = idesc_bf16(kTileM, kTileN);
        const uint32_t idesc = kIdesc1 + (uint32_t)(((kTileN * (c - 1)) >> 3) << 17);
#pragma unroll
        for (int k = 0; k < kKB / 16; k++) {
            const uint32_t accumulate = (fresh && k == 0) ? 0u : 1u;
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
                :: "r"(dt), "l"(da + 2 * k), "l"(db + 2 * k), "r"(idesc), "r"(accumulate));
        }
    }
}

// The drain after K-block kb of an item of KB blocks: 0 none, kXEvent (E2 .. E5),
// kYEvent (E6 ..) or kFullEvent (every accumulator, then the output).
__device__ __forceinline__ int event_at(int kb, int KB) {
    if (kb == KB - 1) return kFullEvent;
    if (kb % kPeriodY == kPeriodY - 1) return kYEvent;
    if (kb % kPeriodX == kPeriodX - 3) return kXEvent;
    return 0;
}

struct OzArgs {
    int64_t M, Nc;            // output rows / columns
    int64_t ldc;
    double* C;                // output (direct mode), or
    double* part;             // split-K partial tiles [splits][Mp][Np] (split mode)
    int64_t Mp, Np;           // partial-tile extents: tilesM * 128, tilesN * 64
    const int* expA;          // biased exponent field of each row's largest |value| (0: zero row)
    const int* expB;
    int64_t rowsA_pad, rowsB_pad;
    int tilesM, tilesN;
    int kb_total;             // K-blocks of 32
    int kb_split;             // K-blocks per split
    int splits;
    int symmetric;            // only tiles that reach the upper triangle (j >= i)
    int b_upper;              // B_hat[j][k] = 0 for k > j: K limited to the tile's last column
    int64_t pairs;            // tiles per split and batch
    int nbatch;               // independent products (diagonal blocks of the split layout)
    int64_t m_batch;          // output rows per batch (M when nbatch = 1)
    int64_t a_batch_rows, b_batch_rows;   // operand rows per batch in the slice arrays
    uint64_t wait_ns;         // limit of the waits on the other roles (drains keep kDrainNs)
    unsigned* status;
    // BSR filter-step mode (bsr != 0): A_hat = Y_cur^T (states x grid points), B_hat = the
    // 64 x 64 blocks of H stacked by rows; a work item is one block row (the 64 output
    // columns, grid rows R * 64 ..) against one tile of 128 states, its K the block
    // columns of the row, and the epilogue applies the recurrence
    // Y_out = alpha (H Y_cur - c Y_cur) - beta Y_prev in FP64 (output in C, ldc).
    int bsr;
    int slices;               // digit slices per operand in the products: 7, or 5 (BSR mode)
    const int32_t* brow_ptr;
    const int32_t* bcol;
    int64_t nbr, nblocks;
    const int* expH;          // exponent field of each grid row of H (over its block row)
    const double* Ycur;
    int64_t ldcur;
    const double* Yprev;      // nullptr: no beta term
    int64_t ldprev;
    double alpha, cshift, beta;
};

struct Item {
    int batch, tm, tn, kb0, KB;
    int qb;                   // BSR mode: first block of the row
};

// Stored block range of block row R, clamped to [0, nblocks] and to kMaxItemKB / kBlockKB
// blocks (the host rejects longer rows); `bad` is set for a malformed row pointer.
__device__ __forceinline__ void bsr_row_range(const OzArgs& g, int64_t R, int& qb, int& nq, bool& bad) {
    int b0 = g.brow_ptr[R], b1 = g.brow_ptr[R + 1];
    if (b0 < 0) { b0 = 0; bad = true; }
    if (b1 > g.nblocks) { b1 = (int)g.nblocks; bad = true; }
    if (b1 < b0) { b1 = b0; bad = true; }
    if (b1 - b0 > kMaxItemKB / kBlockKB) { b1 = b0 + kMaxItemKB / kBlockKB; bad = true; }
    qb = b0;
    nq = b1 - b0;
}

// First column tile of row tile tm that reaches the upper triangle (j >= i).
__device__ __host__ __forceinline__ int first_upper_tn(int tm) { return (tm * kTileM) / kTileN; }

template <bool kBsr>
__device__ __forceinline__ Item decode(const OzArgs& g, int64_t item) {
    Item it;
    if (kBsr) {
        // the state tiles of a block row are consecutive, so its H slices are shared
        // through L2
        const int64_t R = item / g.tilesM;
        bool bad = false;
        int nq;
        bsr_row_range(g, R, it.qb, nq, bad);
        it.batch = 0;
        it.tm = (int)(item % g.tilesM);
        it.tn = (int)R;
        it.kb0 = 0;
        it.KB = kBlockKB * nq;
        return it;
    }
    it.qb = 0;
    const int64_t per_split = g.pairs * g.nbatch;
    const int z = (int)(item / per_split);
    it.batch = (int)((item % per_split) / g.pairs);
    int64_t p = item % g.pairs;
    if (g.symmetric) {
        int tm = 0;
        while (tm < g.tilesM - 1 && p >= g.tilesN - first_upper_tn(tm)) { p -= g.tilesN - first_upper_tn(tm); tm++; }
        it.tm = tm;
        it.tn = first_upper_tn(tm) + (int)p;
    } else {
        it.tm = (int)(p / g.tilesN);
        it.tn = (int)(p % g.tilesN);
    }
    int kend = g.kb_total;
    if (g.b_upper) {
        const int lim = (int)(((int64_t)(it.tn + 1) * kTileN + kKB - 1) / kKB);
        if (lim < kend) kend = lim;
    }
    it.kb0 = z * g.kb_split;
    const int k1 = it.kb0 + g.kb_split < kend ? it.kb0 + g.kb_split : kend;
    it.KB = k1 > it.kb0 ? k1 - it.kb0 : 0;
    return it;
}

// 16 accumulator columns of this warp's 32 TMEM lanes (one row per lane).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

// FP32 power of two 2^p (|p| < 127).
__device__ __forceinline__ float pow2f(int p) { return __int_as_float((127 + p) << 23); }

// x * 2^e for a nonzero double x built from an integer (exact exponent shift);
// results outside the normal range flush to signed zero or infinity.
__device__ __forceinline__ double scale_pow2(double x, int e) {
    const long long b = __double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7ff) + e;
    const long long sign = b & (1ll << 63);
    if (ex <= 0) return __longlong_as_double(sign);
    if (ex >= 0x7ff) return __longlong_as_double(sign | (0x7ffll << 52));
    return __longlong_as_double(b + ((long long)e << 52));
}

// 2^{e} (hi 2^{-40} + lo 2^{-64}) from the two exact integers of an output element.
__device__ __forceinline__ double combine(long long hi, long long lo, int e) {
    double v = 0.0;
    if (hi != 0) v = scale_pow2((double)hi, e - 40);
    if (lo != 0) v += scale_pow2((double)lo, e - 64);
    return v;
}

// One CTA of 18 warps per SM: the register file is split among the SM's four schedulers
// (16,384 registers each) and five of the warps share one of them, which allows 96
// registers a thread; ptxas keeps to that under these launch bounds.  kBsr: the BSR
// filter-step mode (its own instantiation, so that neither mode carries the other's
// epilogue registers).  NS: digit slices per operand (7, or 5 for the 40-bit steps).
template <bool kBsr, int NS>
__global__ void __launch_bounds__(kThreads, 1)
oz_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, OzArgs g,
               int64_t total) {
    using Sh = OzShape<NS>;
    constexpr int kStages = Sh::kStages, kStageBytes = Sh::kStageBytes, kMmas = Sh::kMmas, kAccs = Sh::kAccs;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages], efull, eempty, done;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    bool nonfinite = false, bad_pattern = false;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&efull, 1);
        mbar_init(&eempty, kEpiWarps);
        mbar_init(&done, 1);
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

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer
        int64_t sc = 0;
        for (int64_t item = blockIdx.x; item < total && !*abort_v; item += gridDim.x) {
            const Item it = decode<kBsr>(g, item);
            if (kBsr) {
                int qb, nq;
                bsr_row_range(g, it.tn, qb, nq, bad_pattern);
            }
            bool ok = true;
            for (int kb = 0; kb < it.KB; kb++, sc++) {
                const int s = (int)(sc % kStages);
                const int64_t u = sc / kStages;
                if (u >= 1 && !mbar_wait(sa(&empty[s]), (uint32_t)((u - 1) & 1), g.wait_ns)) { ok = false; break; }
                const uint32_t st = sa(smem + (size_t)s * kStageBytes);
                // K offset in A_hat and in B_hat, and B_hat's first row
                int xa = (it.kb0 + kb) * kKB, xb = xa;
                int64_t rb = it.batch * g.b_batch_rows + (int64_t)it.tn * kTileN;
                if (kBsr) {
                    const int q = it.qb + kb / kBlockKB, half = kb % kBlockKB;
                    int C = g.bcol[q];
                    if (C < 0 || (int64_t)C >= g.nbr) { C = 0; bad_pattern = true; }   // still a valid tile
                    xa = C * 64 + half * kKB;
                    xb = half * kKB;
                    rb = (int64_t)q * 64;
                }
                mbar_expect_tx(&full[s], kStageBytes);
#pragma unroll
                for (int t = 0; t < NS; t++)
                    tma_load_2d(st + t * kSliceA, &tmA, xa,
                                (int)(t * g.rowsA_pad + it.batch * g.a_batch_rows + (int64_t)it.tm * kTileM),
                                sa(&full[s]));
#pragma unroll
                for (int t = 0; t < NS; t++)
                    tma_load_2d(st + NS * kSliceA + t * kSliceB, &tmB, xb, (int)(t * g.rowsB_pad + rb),
                                sa(&full[s]));
            }
            if (!ok) { *abort_v = 1; break; }
        }
        // every copy issued has landed before the CTA can exit
        for (int s = 0; s < kStages && s < sc; s++) {
            const int64_t last = s + ((sc - 1 - s) / kStages) * kStages;
            mbar_wait(sa(&full[s]), (uint32_t)((last / kStages) & 1), kDrainNs);
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer
        int64_t sc = 0, ev_commit = 0, ev_wait = 0;
        bool issued = false;
        for (int64_t item = blockIdx.x; item < total && !*abort_v; item += gridDim.x) {
            const Item it = decode<kBsr>(g, item);
            bool ok = true;
            for (int kb = 0; kb < it.KB; kb++, sc++) {
                const int s = (int)(sc % kStages);
                if (!mbar_wait(sa(&full[s]), (uint32_t)((sc / kStages) & 1), g.wait_ns) || *abort_v) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t st = sa(smem + (size_t)s * kStageBytes);
                // which group starts fresh in this stage (its drain must have ended first)
                const bool resetX = kb == 0 || kb % kPeriodX == kPeriodX - 2;
                const bool resetY = kb == 0 || kb % kPeriodY == 0;
                auto wait_drain = [&]() -> bool {
                    const bool w = mbar_wait(sa(&eempty), (uint32_t)(ev_wait & 1), g.wait_ns);
                    ev_wait++;
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    return w;
                };
                // descriptors of the stage's first A and first B slice tile
                const uint64_t da0 = desc_kmajor(st, kSwizzleBytes);
                const uint64_t db0 = desc_kmajor(st + NS * kSliceA, kSwizzleBytes);
                // after a drain wait that gave up, nothing more is issued into the
                // accumulators that the epilogue may still be reading
                bool w = true;
                if (kb == 0) {
                    if (ev_commit > 0) w = wait_drain();     // the previous item's output drain
                    if (w) issue_mmas<NS, 0, kMmas>(da0, db0, tmem, resetX, resetY);
                } else if (resetX) {                           // E2 .. E5 drained after the last block
                    issue_mmas<NS, kMmaX, kMmas>(da0, db0, tmem, false, resetY);
                    w = wait_drain();
                    if (w) issue_mmas<NS, 0, kMmaX>(da0, db0, tmem, true, false);
                } else if (resetY) {                           // E6 .. drained after the last block
                    issue_mmas<NS, 0, kMmaX>(da0, db0, tmem, resetX, false);
                    w = wait_drain();
                    if (w) issue_mmas<NS, kMmaX, kMmas>(da0, db0, tmem, false, true);
                } else {
                    issue_mmas<NS, 0, kMmas>(da0, db0, tmem, false, false);
                }
                issued = true;
                umma_commit(&empty[s]);
                if (!w) { ok = false; sc++; break; }
                if (event_at(kb, it.KB)) {
                    umma_commit(&efull);
                    ev_commit++;
                }
            }
            if (!ok) { *abort_v = 1; break; }
        }
        // every MMA issued has completed before TMEM is released
        if (issued) {
            umma_commit(&done);
            mbar_wait(sa(&done), 0, kDrainNs);
        }
    } else if (warp >= 2) {
        // ---------------- epilogue: exact drains into 64-bit integers, then the output
        const int q = warp & 3, h = (warp - 2) >> 2;
        const uint32_t lane_base = (uint32_t)(32 * q) << 16;
        int64_t ev = 0;
        long long hi[kColsPerThread], lo[kColsPerThread];
        // BSR mode: Y_out at grid rows col0 + c of state `row` from the product D of
        // the tile (zero for an empty block row)
        auto bsr_out = [&](const Item& it, bool have) {
            const int64_t j = (int64_t)it.tm * kTileM + 32 * q + lane;      // state
            if (j >= g.M) return;
            const int64_t i0 = (int64_t)it.tn * kTileN + h * kColsPerThread;   // first grid row
            const int ea = have ? g.expA[j] : 0;
#pragma unroll
            for (int c = 0; c < kColsPerThread; c++) {
                const int64_t i = i0 + c;
                const int eb = have ? g.expH[i] : 0;
                const double D = (ea != 0 && eb != 0) ? combine(hi[c], lo[c], (ea - 1021) + (eb - 1021)) : 0.0;
                double y = g.alpha * fma(-g.cshift, g.Ycur[i * g.ldcur + j], D);
                if (g.Yprev) y = fma(-g.beta, g.Yprev[i * g.ldprev + j], y);
                nonfinite |= !isfinite(y);
                g.C[i * g.ldc + j] = y;
            }
        };
        for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
            const Item it = decode<kBsr>(g, item);
#pragma unroll
            for (int c = 0; c < kColsPerThread; c++) hi[c] = lo[c] = 0;
            if (kBsr && it.KB == 0) {   // empty block row: no MMA, no drain
                if (*abort_v) break;
                bsr_out(it, false);
                continue;
            }
            bool ok = true;
            for (int kb = 0; kb < it.KB; kb++) {
                const int kind = event_at(kb, it.KB);
                if (!kind) continue;
                if (!__all_sync(0xffffffffu, !*abort_v && mbar_wait(sa(&efull), (uint32_t)(ev & 1), g.wait_ns))) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
                for (int a = 0; a < kAccs; a++) {
                    const bool take = (a < 4) ? (kind & kXEvent) : (kind & kYEvent);
                    if (!take) continue;
                    // E_l (l = a + 2) holds an exact multiple of 2^-8l below 2^24 units
                    const float up = pow2f(8 * (a + 2));
                    const long long mul = 1ll << (a < 4 ? 40 - 8 * (a + 2) : 64 - 8 * (a + 2));
                    uint32_t v[16];
                    tmem_ld16(tmem + lane_base + (uint32_t)(a * kTileN + h * kColsPerThread), v);
                    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
                    for (int c = 0; c < 16; c++) {
                        const long long iv = (long long)__float2int_rn(__uint_as_float(v[c]) * up) * mul;
                        if (a < 4) hi[c] += iv;
                        else lo[c] += iv;
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;");
                __syncwarp();
                if (lane == 0) mbar_arrive(&eempty);
                ev++;
                if (kind == kFullEvent && kBsr) {
                    bsr_out(it, true);
                } else if (kind == kFullEvent) {
                    const int64_t row = (int64_t)it.tm * kTileM + 32 * q + lane;        // within the batch
                    const int64_t orow = it.batch * g.m_batch + row;                     // output row
                    const int64_t col0 = (int64_t)it.tn * kTileN + h * kColsPerThread;
                    const bool valid = row < g.m_batch && orow < g.M;
                    const int ea = valid ? g.expA[it.batch * g.a_batch_rows + row] : 0;
                    const int* expB = g.expB + it.batch * g.b_batch_rows;
                    if (g.part) {
                        const int z = it.kb0 / g.kb_split;
                        double* dst = g.part + ((int64_t)z * g.Mp + row) * g.Np + col0;
#pragma unroll
                        for (int c = 0; c < kColsPerThread; c++) {
                            const int eb = (col0 + c < g.Nc) ? expB[col0 + c] : 0;
                            dst[c] = (ea != 0 && eb != 0) ? combine(hi[c], lo[c], (ea - 1021) + (eb - 1021)) : 0.0;
                        }
                    } else if (valid) {
                        double* dst = g.C + orow * g.ldc + col0;
#pragma unroll
                        for (int c = 0; c < kColsPerThread; c++) {
                            if (col0 + c >= g.Nc) break;
                            const int eb = expB[col0 + c];
                            dst[c] = (ea != 0 && eb != 0) ? combine(hi[c], lo[c], (ea - 1021) + (eb - 1021)) : 0.0;
                        }
                    }
                }
            }
            if (!ok) { *abort_v = 1; break; }
        }
    }

    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTmemCols));
    }
    if (threadIdx.x == 0 && abort_flag) raise_status(g.status, DEV_TIMEOUT);
    if (nonfinite) raise_status(g.status, DEV_NONFINITE);
    if (bad_pattern) raise_status(g.status, DEV_PATTERN);
}

// Largest biased exponent field of each row of A_hat (A_hat[r][k] = src[k * ld + r]
// when trans, else src[r * ld + k]); 0 for a row of zeros (subnormals count as zero).
// Batch z = blockIdx.z reads src + z * src_bstride over K_z = min(Kb, Ktot - z Kb) and
// writes exps + z * rows_pad.  exps must be zeroed first.
template <bool kTrans>
__global__ void oz_exponents_kernel(const double* __restrict__ src, int64_t ld, int64_t rows, int64_t Kb,
                                    int64_t Ktot, int64_t src_bstride, int64_t rows_pad, int* exps,
                                    unsigned* status) {
    const int64_t z = blockIdx.z;
    src += z * src_bstride;
    exps += z * rows_pad;
    const int64_t K = Ktot - z * Kb < Kb ? Ktot - z * Kb : Kb;
    int m = 0;
    bool bad = false;
    if (kTrans) {
        // thread per column of src (row of A_hat), a range of src rows per block row
        const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        const int64_t k0 = (int64_t)blockIdx.y * 256;
        if (r >= rows) return;
        const int64_t k1 = k0 + 256 < K ? k0 + 256 : K;
        for (int64_t k = k0; k < k1; k++) {
            const int ef = (int)((__double_as_longlong(src[k * ld + r]) >> 52) & 0x7ff);
            bad |= ef == 0x7ff;
            m = ef > m ? ef : m;
        }
        if (m) atomicMax(exps + r, m);
    } else {
        // warp per row
        const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        const int lane = threadIdx.x & 31;
        if (r >= rows) return;
        for (int64_t k = lane; k < K; k += 32) {
            const int ef = (int)((__double_as_longlong(src[r * ld + k]) >> 52) & 0x7ff);
            bad |= ef == 0x7ff;
            m = ef > m ? ef : m;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) exps[r] = m;
    }
    if (bad) raise_status(status, DEV_NONFINITE);
}

// The seven BF16 slices of one value x of a row whose largest exponent field is efm.
__device__ __forceinline__ void digits_of(double x, int efm, __nv_bfloat16 (&out)[kSlices]) {
    const long long b = __double_as_longlong(x);
    const int ef = (int)((b >> 52) & 0x7ff);
    long long F = 0;
    if (ef != 0 && efm != 0 && ef != 0x7ff) {
        // F = |x| 2^{-e} 2^{56} < 2^55 with e = efm - 1021: mant 2^{ef - efm + 2}, the
        // right shifts rounded to nearest
        const long long mant = (b & ((1ll << 52) - 1)) | (1ll << 52);
        const int sh = efm - ef - 2;
        if (sh <= 0) F = mant << (-sh);
        else F = sh < 60 ? (mant + (1ll << (sh - 1))) >> sh : 0;
    }
    // balanced base-256 digits, least significant first; the top digit keeps its carry
    int d[kSlices];
    int carry = 0;
#pragma unroll
    for (int t = kSlices - 1; t >= 1; t--) {
        int byte = (int)((F >> (8 * (kSlices - 1 - t))) & 255) + carry;
        carry = byte >= 128;
        d[t] = carry ? byte - 256 : byte;
    }
    d[0] = (int)(F >> (8 * (kSlices - 1))) + carry;
    const bool neg = b < 0;
#pragma unroll
    for (int t = 0; t < kSlices; t++) {
        const float v = (float)(neg ? -d[t] : d[t]) * pow2f(-8 * (t + 1));
        out[t] = __float2bfloat16_rn(v);
    }
}

// Slices of A_hat into [kSlices][nbatch * rows_pad][K_pad] (K contiguous), zero in
// the padding; batch z = blockIdx.z as in oz_exponents_kernel, at rows z * rows_pad.
// Only the first nplanes planes are written (the five-slice steps read no others).
// 32 x 32 tiles through shared memory so that reads and writes are both coalesced
// when A_hat is the transpose of src.
template <bool kTrans>
__global__ void oz_slice_kernel(const double* __restrict__ src, int64_t ld, int64_t rows, int64_t Kb, int64_t Ktot,
                                int64_t src_bstride, const int* __restrict__ exps, int64_t rows_pad, int64_t K_pad,
                                size_t plane, int nplanes, __nv_bfloat16* __restrict__ slices) {
    __shared__ double tile[32][33];
    const int64_t z = blockIdx.z;
    src += z * src_bstride;
    exps += z * rows_pad;
    slices += (size_t)z * rows_pad * K_pad;
    const int64_t K = Ktot - z * Kb < Kb ? Ktot - z * Kb : Kb;
    const int64_t k0 = (int64_t)blockIdx.x * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    // row tiles in a grid-stride loop: gridDim.y is at most 65535
    for (int64_t rt = blockIdx.y; rt * 32 < rows_pad; rt += gridDim.y) {
        const int64_t r0 = rt * 32;
        __syncthreads();   // the previous tile has been read
        for (int i = ty; i < 32; i += blockDim.y) {
            double v = 0.0;
            if (kTrans) {   // src row k0 + i, column r0 + tx  ->  tile[k][r]
                const int64_t k = k0 + i, r = r0 + tx;
                if (k < K && r < rows) v = src[k * ld + r];
                tile[i][tx] = v;
            } else {        // src row r0 + i, column k0 + tx  ->  tile[k][r]
                const int64_t r = r0 + i, k = k0 + tx;
                if (k < K && r < rows) v = src[r * ld + k];
                tile[tx][i] = v;
            }
        }
        __syncthreads();
        for (int i = ty; i < 32; i += blockDim.y) {
            const int64_t r = r0 + i, k = k0 + tx;
            if (r >= rows_pad || k >= K_pad) continue;
            const int efm = r < rows ? exps[r] : 0;
            __nv_bfloat16 dg[kSlices];
            digits_of(tile[tx][i], efm, dg);
#pragma unroll
            for (int t = 0; t < kSlices; t++)
                if (t < nplanes) slices[t * plane + (size_t)r * K_pad + k] = dg[t];
        }
    }
}

// C = sum over splits of the partial tiles; for a symmetric product an element
// below the diagonal takes its mirror above it (always in a computed tile).
__global__ void oz_reduce_kernel(const double* __restrict__ part, int splits, int64_t Mp, int64_t Np, int64_t M,
                                 int64_t Nc, double* C, int64_t ldc, int symmetric) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= M * Nc) return;
    int64_t i = idx / Nc, j = idx % Nc;
    if (symmetric && i > j) { const int64_t t = i; i = j; j = t; }
    double s = 0.0;
    for (int z = 0; z < splits; z++) s += part[((int64_t)z * Mp + i) * Np + j];
    C[(idx / Nc) * ldc + idx % Nc] = s;
}

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Arena stand-in that only counts bytes.
struct CountAr {
    Sizer s;
    template <typename T>
    T* take(size_t n) {
        s.take<T>(n);
        return nullptr;
    }
};

// Workspace pieces of one operand: exponents (int32 per padded row) and slices
// [kSlices][nbatch * rows_pad][K_pad]; batch b holds rows b * rows_pad ...
struct OzOperand {
    int* exps = nullptr;
    __nv_bfloat16* slices = nullptr;
    int64_t rows = 0, K = 0, rows_pad = 0, K_pad = 0;
    int nbatch = 1;
    int64_t plane_rows() const { return (int64_t)nbatch * rows_pad; }
};

template <typename Ar>
void oz_operand_layout(Ar& ar, int64_t rows, int64_t K, int nbatch, int64_t row_pad, OzOperand* op) {
    OzOperand o;
    o.rows = rows;
    o.K = K;
    o.nbatch = nbatch;
    o.rows_pad = round_up(rows, row_pad);
    o.K_pad = round_up(K, 32);   // the slicing kernel's tiles are 32 wide in K
    o.exps = ar.template take<int>((size_t)o.plane_rows());
    o.slices = ar.template take<__nv_bfloat16>((size_t)kSlices * o.plane_rows() * o.K_pad);
    if (op) *op = o;
}

// Exponents and slices of an operand; batch b reads src + b * src_bstride over
// min(o.K, Ktot - b o.K) of the K dimension.  nplanes: slice planes written.
int oz_prepare(const double* src, int64_t ld, bool trans, const OzOperand& o, int64_t Ktot, int64_t src_bstride,
               unsigned* status, cudaStream_t s, int nplanes = kSlices) {
    CHFSI_CUDA_TRY(cudaMemsetAsync(o.exps, 0, sizeof(int) * (size_t)o.plane_rows(), s));
    if (trans) {
        dim3 grid((unsigned)((o.rows + 255) / 256), (unsigned)((o.K + 255) / 256), (unsigned)o.nbatch);
        oz_exponents_kernel<true><<<grid, 256, 0, s>>>(src, ld, o.rows, o.K, Ktot, src_bstride, o.rows_pad, o.exps,
                                                      status);
    } else {
        dim3 grid((unsigned)((o.rows * 32 + 255) / 256), 1, (unsigned)o.nbatch);
        oz_exponents_kernel<false><<<grid, 256, 0, s>>>(src, ld, o.rows, o.K, Ktot, src_bstride, o.rows_pad, o.exps,
                                                       status);
    }
    CHFSI_LAUNCH_CHECK();
    dim3 grid((unsigned)(o.K_pad / 32), (unsigned)std::min<int64_t>(o.rows_pad / 32, 65535), (unsigned)o.nbatch);
    const size_t plane = (size_t)o.plane_rows() * o.K_pad;
    if (trans)
        oz_slice_kernel<true><<<grid, dim3(32, 8), 0, s>>>(src, ld, o.rows, o.K, Ktot, src_bstride, o.exps, o.rows_pad,
                                                          o.K_pad, plane, nplanes, o.slices);
    else
        oz_slice_kernel<false><<<grid, dim3(32, 8), 0, s>>>(src, ld, o.rows, o.K, Ktot, src_bstride, o.exps,
                                                           o.rows_pad, o.K_pad, plane, nplanes, o.slices);
    CHFSI_LAUNCH_CHECK();
    return CHFSI_OK;
}

// Split-K count for a product whose output has `tiles` tiles: at most kMaxItemKB
// K-blocks per work item (the range of the 64-bit accumulators), and enough items
// for about one per SM while each split keeps at least 2048 K.
int oz_splits(int64_t tiles, int kb_total, int sms) {
    const int64_t need = (kb_total + kMaxItemKB - 1) / kMaxItemKB;
    int64_t want = (sms + tiles - 1) / tiles;
    constexpr int64_t kMinSplitKB = 2048 / kKB;
    const int64_t maxs = (kb_total + kMinSplitKB - 1) / kMinSplitKB;
    if (want > maxs) want = maxs;
    const int64_t sp = want > need ? want : need;
    return (int)(sp < 1 ? 1 : sp);
}

struct OzPlan {
    OzOperand A, B;
    double* part = nullptr;
    int splits = 1;
    bool same = false;        // B_hat is A_hat (a Gram matrix)
};

// M x Nc output, K reduction; tn_form: C = A^T B (split over K), else C = A B.
template <typename Ar>
void oz_layout(Ar& ar, bool tn_form, int64_t M, int64_t Nc, int64_t K, bool same, int sms, OzPlan* plan) {
    OzPlan p;
    p.same = same;
    oz_operand_layout(ar, M, K, 1, kRowPad, &p.A);
    if (same) p.B = p.A;
    else oz_operand_layout(ar, Nc, K, 1, kRowPad, &p.B);
    if (tn_form) {
        const int64_t tm = (M + kTileM - 1) / kTileM, tn = (Nc + kTileN - 1) / kTileN;
        p.splits = oz_splits(tm * tn, (int)(p.A.K_pad / kKB), sms > 0 ? sms : 148);
        p.part = ar.template take<double>((size_t)p.splits * (tm * kTileM) * (tn * kTileN));
    }
    if (plan) *plan = p;
}

// One persistent CTA per SM (or per work item, if fewer).
int launch_oz(const CUtensorMap& tmA, const CUtensorMap& tmB, const OzArgs& g, int64_t total, cudaStream_t s) {
    if (total <= 0) return CHFSI_OK;
    const int dev = current_device();
    if (dev < 0) return CHFSI_ERR_CUDA;
    if (g.slices != 7 && !(g.slices == 5 && g.bsr)) return CHFSI_ERR_ARG;
    static bool attr[kMaxDevices] = {};
    if (!attr[dev]) {
        CHFSI_CUDA_TRY(cudaFuncSetAttribute(oz_gemm_kernel<false, 7>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            OzShape<7>::kSmemBytes));
        CHFSI_CUDA_TRY(cudaFuncSetAttribute(oz_gemm_kernel<true, 7>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            OzShape<7>::kSmemBytes));
        CHFSI_CUDA_TRY(cudaFuncSetAttribute(oz_gemm_kernel<true, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            OzShape<5>::kSmemBytes));
        attr[dev] = true;
    }
    const int sms = sm_count();
    if (sms <= 0) return CHFSI_ERR_CUDA;
    const unsigned grid = (unsigned)(total < sms ? total : sms);
    if (g.bsr && g.slices == 5)
        oz_gemm_kernel<true, 5><<<grid, kThreads, OzShape<5>::kSmemBytes, s>>>(tmA, tmB, g, total);
    else if (g.bsr)
        oz_gemm_kernel<true, 7><<<grid, kThreads, OzShape<7>::kSmemBytes, s>>>(tmA, tmB, g, total);
    else
        oz_gemm_kernel<false, 7><<<grid, kThreads, OzShape<7>::kSmemBytes, s>>>(tmA, tmB, g, total);
    CHFSI_LAUNCH_CHECK();
    return CHFSI_OK;
}

// The product of prepared operands.  nbatch > 1: independent products, batch b of the
// output at rows b * m_batch (m_batch rows each, the last one clipped at M).
int oz_run(const OzPlan& p, bool tn_form, double* C, int64_t ldc, int64_t M, int64_t Nc, bool symmetric,
           bool b_upper, unsigned* status, cudaStream_t s, int nbatch = 1, int64_t m_batch = 0) {
    if (M <= 0 || Nc <= 0) return CHFSI_OK;
    const int64_t K_pad = p.A.K_pad;
    if (K_pad > (int64_t)1 << 21 || p.A.plane_rows() * kSlices > INT32_MAX || p.B.plane_rows() * kSlices > INT32_MAX)
        return CHFSI_ERR_UNSUPPORTED;
    if (!tn_form && K_pad > (int64_t)kMaxItemKB * kKB) return CHFSI_ERR_UNSUPPORTED;   // no split-K in the nn form
    if (nbatch > 1 && (tn_form || symmetric || p.A.nbatch != nbatch || p.B.nbatch != nbatch || m_batch <= 0 ||
                       m_batch > p.A.rows_pad))
        return CHFSI_ERR_ARG;
    CUtensorMap tmA, tmB;
    int rc;
    if ((rc = make_map_bf16(&tmA, p.A.slices, K_pad, kSlices * p.A.plane_rows(), kKB, kTileM,
                            kTmaSwizzle)))
        return rc;
    if ((rc = make_map_bf16(&tmB, p.B.slices, K_pad, kSlices * p.B.plane_rows(), kKB, kTileN,
                            kTmaSwizzle)))
        return rc;
    OzArgs g{};
    const int64_t mb = nbatch > 1 ? m_batch : M;
    g.M = M;
    g.Nc = Nc;
    g.ldc = ldc;
    g.nbatch = nbatch;
    g.m_batch = mb;
    g.a_batch_rows = p.A.rows_pad;
    g.b_batch_rows = p.B.rows_pad;
    g.tilesM = (int)((mb + kTileM - 1) / kTileM);
    g.tilesN = (int)((Nc + kTileN - 1) / kTileN);
    g.Mp = (int64_t)g.tilesM * kTileM;
    g.Np = (int64_t)g.tilesN * kTileN;
    g.expA = p.A.exps;
    g.expB = p.B.exps;
    g.rowsA_pad = p.A.plane_rows();
    g.rowsB_pad = p.B.plane_rows();
    g.kb_total = (int)(K_pad / kKB);
    g.splits = tn_form ? p.splits : 1;
    g.kb_split = (g.kb_total + g.splits - 1) / g.splits;
    g.splits = (g.kb_total + g.kb_split - 1) / g.kb_split;   // no empty split
    g.symmetric = symmetric ? 1 : 0;
    g.b_upper = b_upper ? 1 : 0;
    g.slices = kSlices;
    g.wait_ns = pipeline_wait_ns();
    g.status = status;
    g.C = tn_form ? nullptr : C;
    g.part = tn_form ? p.part : nullptr;
    int64_t pairs = 0;
    if (symmetric) {
        for (int tm = 0; tm < g.tilesM; tm++) {
            const int first = first_upper_tn(tm);
            if (first < g.tilesN) pairs += g.tilesN - first;
        }
    } else {
        pairs = (int64_t)g.tilesM * g.tilesN;
    }
    g.pairs = pairs;
    const int64_t total = pairs * g.splits * nbatch;
    if ((rc = launch_oz(tmA, tmB, g, total, s))) return rc;
    if (tn_form) {
        const int64_t cnt = M * Nc;
        oz_reduce_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(p.part, g.splits, g.Mp, g.Np, M, Nc, C, ldc,
                                                                       g.symmetric);
        CHFSI_LAUNCH_CHECK();
    }
    return CHFSI_OK;
}

// Block-diagonal product of the split layout: D slices (prepared once) and the slices
// of the multiplied block (prepared per product).
struct OzBlockDiag {
    OzOperand D, Y;
};

template <typename Ar>
void oz_blockdiag_layout(Ar& ar, int64_t N, int B, int64_t n, OzBlockDiag* out) {
    OzBlockDiag b;
    const int nblk = (int)((N + B - 1) / B);
    oz_operand_layout(ar, (int64_t)nblk * B, B, 1, kRowPad, &b.D);   // rows of all blocks, K = B
    oz_operand_layout(ar, n, B, nblk, 32, &b.Y);                      // per block: n rows (Y columns), K = B
    if (out) *out = b;
}

// BSR filter step: slices of H's blocks (made once per filter call; rows = the 64
// rows of every stored block, K = the block's 64 columns, each row scaled by the
// largest exponent of its grid row over the whole block row, so that the products of
// all block columns share one scale) and of Y_cur^T (made per step; rows = states,
// K = grid points).
struct OzBsr {
    OzOperand H, Y;
    int* expH = nullptr;      // per grid row
};

template <typename Ar>
void oz_bsr_layout(Ar& ar, int64_t nbr, int64_t nblocks, int64_t n, OzBsr* out) {
    OzBsr b;
    // at least one tile of rows, so that the tensor map is valid without stored blocks
    oz_operand_layout(ar, (nblocks > 2 ? nblocks : 2) * 64, 64, 1, kRowPad, &b.H);
    oz_operand_layout(ar, n, nbr * 64, 1, kRowPad, &b.Y);
    b.expH = ar.template take<int>((size_t)(nbr * 64));
    if (out) *out = b;
}

// Largest exponent field of each grid row of H over its block row: thread r of block R
// scans row r of every block of the row; the result goes to expH[R * 64 + r] and to
// the slice exponent of that row in each of the row's blocks.
__global__ void bsr_row_exponents_kernel(const double* __restrict__ val, const int32_t* __restrict__ brow_ptr,
                                         int64_t nblocks, int* expH, int* exps, unsigned* status) {
    const int64_t R = blockIdx.x;
    const int r = threadIdx.x;
    int b0 = brow_ptr[R], b1 = brow_ptr[R + 1];
    b0 = b0 < 0 ? 0 : (b0 > nblocks ? (int)nblocks : b0);
    b1 = b1 < b0 ? b0 : (b1 > nblocks ? (int)nblocks : b1);
    int m = 0;
    bool bad = false;
    for (int q = b0; q < b1; q++) {
        const double* row = val + ((int64_t)q * 64 + r) * 64;
        for (int k = 0; k < 64; k++) {
            const int ef = (int)((__double_as_longlong(row[k]) >> 52) & 0x7ff);
            bad |= ef == 0x7ff;
            m = ef > m ? ef : m;
        }
    }
    expH[R * 64 + r] = m;
    for (int q = b0; q < b1; q++) exps[(int64_t)q * 64 + r] = m;
    if (bad) raise_status(status, DEV_NONFINITE);
}

}  // namespace

size_t ozaki_bsr_bytes(int64_t nbr, int64_t nblocks, int64_t n) {
    CountAr ar;
    oz_bsr_layout(ar, nbr, nblocks, n, nullptr);
    return ar.s.used;
}

int ozaki_bsr_prepare(const BsrDev& h, int64_t n, void* ws, size_t ws_bytes, unsigned* status, cudaStream_t s) {
    if (h.bdim != 64 || h.nbr <= 0) return CHFSI_ERR_UNSUPPORTED;
    if (ws_bytes < ozaki_bsr_bytes(h.nbr, h.nblocks, n)) return CHFSI_ERR_NOMEM;
    Arena ar(ws, ws_bytes);
    OzBsr b;
    oz_bsr_layout(ar, h.nbr, h.nblocks, n, &b);
    if (b.H.plane_rows() * kSlices > INT32_MAX || b.Y.plane_rows() * kSlices > INT32_MAX) return CHFSI_ERR_UNSUPPORTED;
    const double* val = static_cast<const double*>(h.val);
    CHFSI_CUDA_TRY(cudaMemsetAsync(b.H.exps, 0, sizeof(int) * (size_t)b.H.plane_rows(), s));
    bsr_row_exponents_kernel<<<(unsigned)h.nbr, 64, 0, s>>>(val, h.brow_ptr, h.nblocks, b.expH, b.H.exps, status);
    CHFSI_LAUNCH_CHECK();
    dim3 grid((unsigned)(b.H.K_pad / 32), (unsigned)std::min<int64_t>(b.H.rows_pad / 32, 65535), 1);
    oz_slice_kernel<false><<<grid, dim3(32, 8), 0, s>>>(val, 64, h.nblocks * 64, 64, 64, 0, b.H.exps, b.H.rows_pad,
                                                       b.H.K_pad, (size_t)b.H.plane_rows() * b.H.K_pad, kSlices,
                                                       b.H.slices);
    CHFSI_LAUNCH_CHECK();
    return CHFSI_OK;
}

int ozaki_bsr_step(const BsrDev& h, int64_t n, const double* Yc, int64_t ldc, const double* Yp, int64_t ldp,
                   double* Yo, int64_t ldo, double alpha, double c, double beta, void* ws, size_t ws_bytes,
                   unsigned* status, cudaStream_t s, int slices) {
    if (slices != 7 && slices != 5) return CHFSI_ERR_ARG;
    if (n <= 0 || h.nbr <= 0) return CHFSI_OK;
    if (ws_bytes < ozaki_bsr_bytes(h.nbr, h.nblocks, n)) return CHFSI_ERR_NOMEM;
    Arena ar(ws, ws_bytes);
    OzBsr b;
    oz_bsr_layout(ar, h.nbr, h.nblocks, n, &b);
    const int64_t N = h.nbr * 64;
    int rc;
    if ((rc = oz_prepare(Yc, ldc, true, b.Y, N, 0, status, s, slices))) return rc;
    CUtensorMap tmA, tmB;
    if ((rc = make_map_bf16(&tmA, b.Y.slices, b.Y.K_pad, kSlices * b.Y.plane_rows(), kKB, kTileM,
                            kTmaSwizzle)))
        return rc;
    if ((rc = make_map_bf16(&tmB, b.H.slices, b.H.K_pad, kSlices * b.H.plane_rows(), kKB, kTileN,
                            kTmaSwizzle)))
        return rc;
    OzArgs g{};
    g.M = n;
    g.Nc = N;
    g.ldc = ldo;
    g.C = Yo;
    g.nbatch = 1;
    g.m_batch = n;
    g.a_batch_rows = b.Y.rows_pad;
    g.tilesM = (int)((n + kTileM - 1) / kTileM);
    g.tilesN = (int)h.nbr;
    g.expA = b.Y.exps;
    g.expB = b.H.exps;
    g.rowsA_pad = b.Y.plane_rows();
    g.rowsB_pad = b.H.plane_rows();
    g.kb_total = kMaxItemKB;
    g.kb_split = kMaxItemKB;
    g.splits = 1;
    g.pairs = (int64_t)g.tilesM * h.nbr;
    g.wait_ns = pipeline_wait_ns();
    g.status = status;
    g.bsr = 1;
    g.slices = slices;
    g.brow_ptr = h.brow_ptr;
    g.bcol = h.bcol;
    g.nbr = h.nbr;
    g.nblocks = h.nblocks;
    g.expH = b.expH;
    g.Ycur = Yc;
    g.ldcur = ldc;
    g.Yprev = Yp;
    g.ldprev = ldp;
    g.alpha = alpha;
    g.cshift = c;
    g.beta = beta;
    return launch_oz(tmA, tmB, g, g.pairs, s);
}

size_t ozaki_workspace_bytes(bool tn_form, int64_t M, int64_t Nc, int64_t K, bool same) {
    CountAr ar;
    oz_layout(ar, tn_form, M, Nc, K, same, tc::sm_count(), nullptr);
    return ar.s.used;
}

int ozaki_gemm_tn(const double* A, int64_t lda, const double* B, int64_t ldb, int64_t K, int64_t M, int64_t Nc,
                  double* C, int64_t ldc, bool symmetric, void* ws, size_t ws_bytes, unsigned* status,
                  cudaStream_t s) {
    if (M <= 0 || Nc <= 0) return CHFSI_OK;
    // the same operand twice (a Gram matrix) is sliced once; `symmetric` says that the
    // product is known to be symmetric (a Gram matrix, or X^T (H X) for symmetric H):
    // only the tiles on and above the diagonal are computed and the others mirrored
    const bool same = (A == B) && (lda == ldb) && (M == Nc);
    if (symmetric && M != Nc) return CHFSI_ERR_ARG;
    if (ws_bytes < ozaki_workspace_bytes(true, M, Nc, K, same)) return CHFSI_ERR_NOMEM;
    Arena ar(ws, ws_bytes);
    OzPlan p;
    oz_layout(ar, true, M, Nc, K, same, tc::sm_count(), &p);
    int rc;
    if ((rc = oz_prepare(A, lda, true, p.A, K, 0, status, s))) return rc;
    if (!same && (rc = oz_prepare(B, ldb, true, p.B, K, 0, status, s))) return rc;
    return oz_run(p, true, C, ldc, M, Nc, symmetric, false, status, s);
}

int ozaki_gemm_nn(const double* A, int64_t lda, const double* B, int64_t ldb, int64_t M, int64_t K, int64_t Nc,
                  double* C, int64_t ldc, bool b_upper, void* ws, size_t ws_bytes, unsigned* status,
                  cudaStream_t s) {
    if (M <= 0 || Nc <= 0) return CHFSI_OK;
    if (ws_bytes < ozaki_workspace_bytes(false, M, Nc, K, false)) return CHFSI_ERR_NOMEM;
    Arena ar(ws, ws_bytes);
    OzPlan p;
    oz_layout(ar, false, M, Nc, K, false, tc::sm_count(), &p);
    int rc;
    if ((rc = oz_prepare(A, lda, false, p.A, K, 0, status, s))) return rc;
    if ((rc = oz_prepare(B, ldb, true, p.B, K, 0, status, s))) return rc;   // B_hat = B^T: rows are B's columns
    return oz_run(p, false, C, ldc, M, Nc, false, b_upper, status, s);
}

size_t ozaki_blockdiag_bytes(int64_t N, int B, int64_t n) {
    CountAr ar;
    oz_blockdiag_layout(ar, N, B, n, nullptr);
    return ar.s.used;
}

int ozaki_blockdiag_prepare(const double* diag, int64_t N, int B, int64_t n, void* ws, size_t ws_bytes,
                            unsigned* status, cudaStream_t s) {
    if (B <= 0 || B % kTileM || B > kMaxItemKB * kKB) return CHFSI_ERR_UNSUPPORTED;
    if (ws_bytes < ozaki_blockdiag_bytes(N, B, n)) return CHFSI_ERR_NOMEM;
    Arena ar(ws, ws_bytes);
    OzBlockDiag bd;
    oz_blockdiag_layout(ar, N, B, n, &bd);
    // every block is B x B row-major, the blocks stacked: one direct operand of nblk * B rows
    return oz_prepare(diag, B, false, bd.D, B, 0, status, s);
}

int ozaki_blockdiag_apply(const double* Y, int64_t ldy, int64_t N, int B, int64_t n, double* T, int64_t ldt,
                          void* ws, size_t ws_bytes, unsigned* status, cudaStream_t s) {
    if (n <= 0 || N <= 0) return CHFSI_OK;
    if (B <= 0 || B % kTileM || B > kMaxItemKB * kKB) return CHFSI_ERR_UNSUPPORTED;
    if (ws_bytes < ozaki_blockdiag_bytes(N, B, n)) return CHFSI_ERR_NOMEM;
    Arena ar(ws, ws_bytes);
    OzBlockDiag bd;
    oz_blockdiag_layout(ar, N, B, n, &bd);
    // Y_hat of block k = (rows kB .. kB + B - 1 of Y)^T: n rows, K = B (the last block clipped at N)
    int rc;
    if ((rc = oz_prepare(Y, ldy, true, bd.Y, N, (int64_t)B * ldy, status, s))) return rc;
    OzPlan p;
    p.A = bd.D;
    p.A.nbatch = bd.Y.nbatch;
    p.A.rows_pad = B;      // rows per batch in the stacked D operand
    p.B = bd.Y;
    return oz_run(p, false, T, ldt, N, n, false, false, status, s, bd.Y.nbatch, B);
}

}  // namespace chfsi

// ------------------------------------------------------------------ C ABI

namespace {

int oz_abi_check(int32_t op, int64_t M, int64_t Nc, int64_t K, int32_t flags) {
    if (op != CHFSI_OP_TN && op != CHFSI_OP_NN) return CHFSI_ERR_ARG;
    if (M < 0 || Nc < 0 || K < 0) return CHFSI_ERR_ARG;
    if (flags & ~(CHFSI_GEMM_SYMMETRIC | CHFSI_GEMM_B_UPPER)) return CHFSI_ERR_ARG;
    if ((flags & CHFSI_GEMM_SYMMETRIC) && (op != CHFSI_OP_TN || M != Nc)) return CHFSI_ERR_ARG;
    if ((flags & CHFSI_GEMM_B_UPPER) && op != CHFSI_OP_NN) return CHFSI_ERR_ARG;
    if (K > ((int64_t)1 << 21) || M > INT32_MAX / 8 || Nc > INT32_MAX / 8) return CHFSI_ERR_UNSUPPORTED;
    if (op == CHFSI_OP_NN && K > 8192) return CHFSI_ERR_UNSUPPORTED;
    return CHFSI_OK;
}

}  // namespace

int chfsi_ozaki_gemm_workspace_size(int32_t op, int64_t M, int64_t Nc, int64_t K, int32_t flags, size_t* bytes) {
    if (!bytes) return CHFSI_ERR_ARG;
    const int rc = oz_abi_check(op, M, Nc, K, flags);
    if (rc) return rc;
    // the tn form with one operand twice is smaller; size for two distinct operands
    *bytes = chfsi::align_up(chfsi::kStatusBytes) + chfsi::ozaki_workspace_bytes(op == CHFSI_OP_TN, M, Nc, K, false);
    return CHFSI_OK;
}

int chfsi_ozaki_gemm(int32_t op, const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc,
                     int64_t M, int64_t Nc, int64_t K, int32_t flags, void* ws, size_t ws_bytes, void* stream) {
    int rc = oz_abi_check(op, M, Nc, K, flags);
    if (rc) return rc;
    if (M == 0 || Nc == 0) return CHFSI_OK;
    if (!C || ldc < Nc || (reinterpret_cast<uintptr_t>(C) & 7u)) return CHFSI_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (K == 0) {
        for (int64_t i = 0; i < M; i++)
            CHFSI_CUDA_TRY(cudaMemsetAsync(C + i * ldc, 0, sizeof(double) * (size_t)Nc, s));
        return CHFSI_OK;
    }
    if (!A || !B || (reinterpret_cast<uintptr_t>(A) & 7u) || (reinterpret_cast<uintptr_t>(B) & 7u)) return CHFSI_ERR_ARG;
    const bool tn = op == CHFSI_OP_TN;
    if (tn ? (lda < M || ldb < Nc) : (lda < K || ldb < Nc)) return CHFSI_ERR_ARG;
    size_t need = 0;
    if ((rc = chfsi_ozaki_gemm_workspace_size(op, M, Nc, K, flags, &need))) return rc;
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) || ws_bytes < need) return ws ? CHFSI_ERR_NOMEM : CHFSI_ERR_ARG;
    unsigned* st = chfsi::status_word(ws);
    CHFSI_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(unsigned), s));
    char* rest = static_cast<char*>(ws) + chfsi::align_up(chfsi::kStatusBytes);
    const size_t rest_bytes = ws_bytes - chfsi::align_up(chfsi::kStatusBytes);
    if (tn)
        return chfsi::ozaki_gemm_tn(A, lda, B, ldb, K, M, Nc, C, ldc, (flags & CHFSI_GEMM_SYMMETRIC) != 0, rest,
                                    rest_bytes, st, s);
    return chfsi::ozaki_gemm_nn(A, lda, B, ldb, M, K, Nc, C, ldc, (flags & CHFSI_GEMM_B_UPPER) != 0, rest,
                                rest_bytes, st, s);
}
