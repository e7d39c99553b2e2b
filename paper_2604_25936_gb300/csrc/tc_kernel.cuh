// Tensor-core T-MLP kernel for sm_103a (tcgen05 MMA, TMEM accumulators, TMA).
//
// Evaluates Eq. 2 (and Eq. 3 for multiplicative tails) for 128-row tiles of
// points sorted by descending exit layer.  One persistent CTA per SM, 320 threads
// (384 in variant 3):
//   warp 0       TMA producer: streams weight tiles (64 K-columns x W units, one
//                K-block of one layer) from L2 into a ring of stages, 128-byte
//                swizzled (the K-major layout the MMA reads).
//   warp 1       owns TMEM and issues tcgen05.mma from one thread:
//                D[128 x W] (fp32, TMEM) += A[128 x 16] . B[W x 16]^T, A read from TMEM.
//   warps 2..9   epilogue.  Thread (quadrant q, lane i) owns tile row 32 q + i (the
//                TMEM lane restriction); the two warps of a quadrant take half of the
//                units of every K-block each.  Layer 1 of raw coordinates with linear
//                tails entirely on the CUDA cores (W1' x + b1' from the row's coordinates
//                and weights in shared memory; the tensor cores start at layer 2);
//                otherwise layer 1's A operand (the split coordinates of one K = 16 MMA,
//                or the Fourier features).  Then bias, sine, tails, the running sum
//                y_l = y_{l-1} + t_l and the write at each row's exit layer.  The new
//                activations are packed (fp16 pair, bf16 or e4m3) and written with
//                tcgen05.st into TMEM, where the next layer's MMAs read them as the A
//                operand.
//   warps 10,11  (variant 3, SAND queries on raw coordinates) every row of exit layer 1,
//                entirely on the CUDA cores: layer 1, its sine and tail 1 in float32.
// TMEM columns: [0, W) accumulator, then A_hi (W/2 columns of packed fp16 pairs)
// and, in the float32 mode, A_lo.  One MMA stream at N = W: measured on GB300, one
// M=128 N=256 K=16 MMA per 128 cycles when each weight stage's MMAs leave the issuing
// thread as one asm run, so N = 256 is what reaches the tensor cores' rate.
// Overlap of a layer's epilogue with the next layer's MMAs: each epilogue thread
// first loads all of its accumulator columns into registers (128 at W = 256) and
// signals d_drained (the next layer may now overwrite D), then produces the next A
// operand one K-block (64 units) at a time, signalling a_ready[kb] after each; the
// MMAs of the next layer on K-block kb start as soon as a_ready[kb] completes.
// Thread (quadrant, slice s) owns units 64 kb + 32 s .. + 31 of every K-block kb.
// Two epilogue warps per SM sub-partition (not four) leave the MMA-issuing thread
// issue slots when it is on the critical path, and 168 registers per thread.
// A tile runs to the exit layer of its first (deepest) row; rows whose exit layer
// was reached ride along only in the one tile per exit layer that straddles two
// layers; in variant 3 no row of exit layer 1 reaches the tensor cores.
//
// Precision modes (hidden-layer products only; everything else is float32):
//   SPLIT16  a = a_hi + a_lo and w*s = w_hi + w_lo with fp16 terms (s = 2^-e per
//            layer, so max|w s| is in [0.5, 1)); D = A_hi B_hi + A_lo B_hi + A_hi B_lo.
//   F16/BF16 one product with fp16 (scaled) / bf16 operands.
//   FP8      one product (tcgen05 kind::f8f6f4) with e4m3 operands: weights scaled
//            per layer by a power of two so max|w s| is in [128, 256); the sine
//            activations in [-1, 1] are stored unscaled (below 2^-6 the e4m3
//            subnormal spacing 2^-9 is finer than the normal-range rounding).
//            A weight stage then holds 128 K-units and an MMA consumes 32.
// Sine: the argument is formed in radians with one rounding, u = acc * w0/s + w0 b, and
// passed to the hardware sine, which takes it to revolutions (one more rounding,
// relative 2^-24) and reduces it there; for the |u| < 64 of these networks that adds
// under 4e-6 rad to the phase, against the 1e-5 output tolerance.  An explicit exact
// reduction first costs three more instructions per unit, and the epilogue's
// instruction count sets the layer time.
// Every mbarrier wait is bounded (2 s of %globaltimer); on timeout the CTA sets
// SAND_FLAG_TIMEOUT, stops issuing work, drains its copies and MMAs, frees TMEM
// and returns.
#pragma once

#include <cuda.h>

#include "internal.cuh"

namespace sand {

enum TcMode { TC_SPLIT16 = 0, TC_F16 = 1, TC_BF16 = 2, TC_FP8 = 3 };

constexpr int kSlices = 2;                  // epilogue warps per TMEM lane quadrant
constexpr int kSliceUnits = 64 / kSlices;   // units of every 64-unit K-block per epilogue thread
constexpr int kEpiWarps = 4 * kSlices;
// Kernel variant 3 (SAND queries on raw coordinates) adds two warps for the rows of exit layer
// 1, on the CUDA cores (SM sub-partitions 2 and 3); 384 x 168 registers still fit one SM.  The
// other variants keep 320 threads: carried in a full-depth kernel, the extra warps' code costs
// its epilogue registers.
constexpr int kCcWarps = 2;
constexpr int tc_threads(int var) { return 64 + 32 * (kEpiWarps + ((var & 3) == 3 ? kCcWarps : 0)); }
// Variant bit 2 (float32 split mode at W = 336 only): the lo part of the activations lives in
// shared memory instead of TMEM, where the accumulator (336 columns) and the hi part (168) leave
// no room for it; the MMAs read it through a shared-memory descriptor, and a weight stage holds
// one part (hi or lo) of one K-block.
constexpr int kAloVar = 4;
constexpr int kTileM = 128;
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr uint64_t kTimeoutNs = 2000000000ull;
constexpr int kSmemBudget = 227 * 1024;
constexpr int kMaxStages = 8;
constexpr int kMaxKBlocks = 6;  // K padded to a multiple of 64, W <= 336
constexpr int kNumBars = 2 * kMaxStages + kMaxKBlocks + 5;  // full, empty, a_ready[kb], d_full, d_drained, drain, x_full, x_empty
// An epilogue thread's row of a tile: coordinates, exit layer, original index (-1: padding).
struct TcRow {
    float x0, x1, x2;
    int d;
    int64_t idx;
};
// bytes after the weight stages and constants: barriers, TMEM slot + abort flag, the tail
// exchange ((kSlices - 1) slices x 2 values x 128 rows), 16 bytes of alignment slack and two
// buffers of one 16-byte point row per epilogue thread (the next tile's rows are copied in
// while the current tile runs)
constexpr int kRowBufBytes = 2 * kEpiThreads * 16;
constexpr int kMiscBytes = kNumBars * 8 + 16 + (kSlices - 1) * 2 * 128 * 4 + 16 + kRowBufBytes + 16 * 4;
static_assert(kSlices == 2, "the epilogue loads 32 accumulator columns per K-block and thread");

struct TcParams {
    int L, W, D, tail_kind, act, enc, m;
    int first_mma;            // 1-based index of the first layer computed on the tensor cores (1)
    int l1_fold;              // layer 1 is one K = 16 fp16 MMA over split coordinates (not Fourier features)
    float x_scale;            // coordinates are scaled by this before the split
    int all_tails;            // write y_1 .. y_L of every row (out[idx * L + l - 1]) instead of y at the exit layer
    float dyn_r;              // > 0: octree-free dynamic exit (full depth): a row stops at the first layer whose
                              // tail |t_l| < dyn_r; a tile stops issuing MMAs once all its rows have stopped
    uint8_t *exit_out;        // dynamic exit: the layer each row stopped at (optional)
    float *grad;              // gradient variant: dy/dx per point, [n][3]
    float finer_k;            // FINER: 1 / omega0 (the activation of phase u = omega0 z is sin(u + u |u| / omega0))
    int kpad;                 // padded K of the packed weight matrix (multiple of 64; of 128 in the FP8 mode)
    int n_stages;
    uint32_t stage_bytes;     // parts x W x 128: one K-block of the weights (hi and lo in the float32 mode)
    uint32_t tmem_cols;       // power of two >= W + parts * W / 2
    int box_rows;             // rows per TMA box: W, or W / 2 when W > 256 (box dimensions are at most 256)
    int n_split;              // first MMA column group when W > 256 (a multiple of 16)
    float c1[kMaxLayers];     // per layer: w0 / s (sine) or 1 / s (ReLU)
    const float *cvec;        // [L][3][W]: bias' (w0 b for sine, b for ReLU), tail a, tail b
    const float *B;           // [m][3] Fourier matrix
    const float *tb;          // [L][2] tail biases
    const float4 *w1p;        // [W]: s (W1[j][0], W1[j][1], W1[j][2], b1[j]) of a raw-coordinate layer 1,
                              // s = omega0 for the sine families (the phase in radians), 1 for ReLU
    int cc;                   // exit-layer-1 rows of a SAND query run on the CUDA-core warps (raw coordinates)
    uint64_t wait_ns;         // limit of each bounded pipeline wait (the drains after an abort keep 2 s)
    int alo;                  // float32 mode at W = 336: A_lo in shared memory (kernel variant bit kAloVar)
};

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false after `limit` ns (2 s unless the caller set a limit), or (when
// follow_abort) once another thread of the CTA has aborted.  The epilogue warps do not follow
// the flag: every waiter on a phase then agrees on whether it completed, so none is left alone
// at a named barrier; they make each result warp-uniform (__all_sync) before the next
// warp-collective TMEM access.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort, WsHeader *hdr,
                                          uint32_t site, bool follow_abort, uint64_t limit) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    while (true) {
        if (mbar_try(bar, parity)) return true;
        if (follow_abort && *abort) return false;
        if (globaltimer() - t0 > limit) {
            *abort = 1;
            atomicOr(&hdr->flags, (uint32_t)SAND_FLAG_TIMEOUT);
            atomicExch(&hdr->timeout_where, site);
            return false;
        }
    }
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
        : "memory");
}
// Plain asynchronous global -> shared copies (each thread its own bytes; completion per thread).
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(uint32_t dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ float4 lds_f4(uint32_t addr) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr));
    return v;
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void named_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }
// Named barrier among n threads that also counts the threads whose pred is true.
__device__ __forceinline__ int named_count(int id, int n, bool pred) {
    int c;
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %3, 0;\n\tbar.red.popc.u32 %0, %1, %2, p;\n\t}"
                 : "=r"(c) : "r"(id), "r"(n), "r"((unsigned)pred) : "memory");
    return c;
}

// K-major operand in shared memory with 128-byte swizzle: rows of 128 bytes,
// 8-row groups 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
// D[128 x N] (+)= A[128 x 16] . B[N x 16]^T with A read from TMEM (lane = row, 32-bit
// column = two consecutive fp16/bf16 K-elements).
template <int MODE>
__device__ __forceinline__ void mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc) {
    if (MODE == TC_FP8) {  // 32 e4m3 K-elements per row, four to a TMEM column
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
            "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
            "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    }
}
// Runs of MMAs in one asm statement: K-step k reads A at a + 8k TMEM columns and B at
// descriptor b + 2k (32 bytes further in every 128-byte row).  Measured on GB300, the
// single issuing thread keeps the tensor pipe full (one M=128, N=256 MMA per 128 cycles)
// only when a stage's MMAs leave it as one straight run like this; one asm statement
// per MMA, with the address arithmetic between them, issues at 150-190 cycles per MMA.
// The first MMA accumulates iff acc; the rest always do.
#define SAND_MMA_K4(KIND)                                                                                  \
    asm volatile("{\n\t.reg .pred p, t;\n\t.reg .b64 b1, b2, b3;\n\t.reg .b32 a1, a2, a3;\n\t"              \
                 "setp.ne.b32 p, %4, 0;\n\tsetp.ne.b32 t, %3, 0;\n\t"                                       \
                 "add.s64 b1, %2, 2;\n\tadd.s64 b2, %2, 4;\n\tadd.s64 b3, %2, 6;\n\t"                       \
                 "add.s32 a1, %1, 8;\n\tadd.s32 a2, %1, 16;\n\tadd.s32 a3, %1, 24;\n\t"                     \
                 KIND " [%0], [%1], %2, %3, p;\n\t" KIND " [%0], [a1], b1, %3, t;\n\t"                        \
                 KIND " [%0], [a2], b2, %3, t;\n\t" KIND " [%0], [a3], b3, %3, t;\n\t}"                       \
                 ::"r"(d), "r"(a), "l"(b), "r"(idesc), "r"(acc) : "memory")
#define SAND_MMA_K2(KIND)                                                                                  \
    asm volatile("{\n\t.reg .pred p, t;\n\t.reg .b64 b1;\n\t.reg .b32 a1;\n\t"                             \
                 "setp.ne.b32 p, %4, 0;\n\tsetp.ne.b32 t, %3, 0;\n\t"                                       \
                 "add.s64 b1, %2, 2;\n\tadd.s32 a1, %1, 8;\n\t"                                            \
                 KIND " [%0], [%1], %2, %3, p;\n\t" KIND " [%0], [a1], b1, %3, t;\n\t}"                        \
                 ::"r"(d), "r"(a), "l"(b), "r"(idesc), "r"(acc) : "memory")
#define SAND_KIND_F16 "tcgen05.mma.cta_group::1.kind::f16"
#define SAND_KIND_F8 "tcgen05.mma.cta_group::1.kind::f8f6f4"
template <int MODE>
__device__ __forceinline__ void mma_k4(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if (MODE == TC_FP8) SAND_MMA_K4(SAND_KIND_F8);
    else SAND_MMA_K4(SAND_KIND_F16);
}
template <int MODE>
__device__ __forceinline__ void mma_k2(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if (MODE == TC_FP8) SAND_MMA_K2(SAND_KIND_F8);
    else SAND_MMA_K2(SAND_KIND_F16);
}
// Four K-steps, each with two A operands against the same B (the float32 mode's
// A_hi B_hi and A_lo B_hi products).
__device__ __forceinline__ void mma_k4x2(uint32_t d, uint32_t a, uint32_t a2, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n\t.reg .pred p, t;\n\t.reg .b64 b1, b2, b3;\n\t.reg .b32 a1, q1, a2_, q2, a3, q3;\n\t"
                 "setp.ne.b32 p, %5, 0;\n\tsetp.ne.b32 t, %4, 0;\n\t"
                 "add.s64 b1, %3, 2;\n\tadd.s64 b2, %3, 4;\n\tadd.s64 b3, %3, 6;\n\t"
                 "add.s32 a1, %1, 8;\n\tadd.s32 a2_, %1, 16;\n\tadd.s32 a3, %1, 24;\n\t"
                 "add.s32 q1, %2, 8;\n\tadd.s32 q2, %2, 16;\n\tadd.s32 q3, %2, 24;\n\t"
                 SAND_KIND_F16 " [%0], [%1], %3, %4, p;\n\t" SAND_KIND_F16 " [%0], [%2], %3, %4, t;\n\t"
                 SAND_KIND_F16 " [%0], [a1], b1, %4, t;\n\t" SAND_KIND_F16 " [%0], [q1], b1, %4, t;\n\t"
                 SAND_KIND_F16 " [%0], [a2_], b2, %4, t;\n\t" SAND_KIND_F16 " [%0], [q2], b2, %4, t;\n\t"
                 SAND_KIND_F16 " [%0], [a3], b3, %4, t;\n\t" SAND_KIND_F16 " [%0], [q3], b3, %4, t;\n\t}"
                 ::"r"(d), "r"(a), "r"(a2), "l"(b), "r"(idesc), "r"(acc) : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// TMEM -> registers, 32 or 16 consecutive columns of this thread's lane (asynchronous:
// the values may be used only after tmem_wait_ld()).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t *r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t *r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// registers -> TMEM, 16, 8 or 4 consecutive 32-bit columns of this thread's lane.  No
// "memory" clobber: the store touches no memory the compiler tracks, so shared-memory loads
// of the next chunk may be scheduled above it; volatile asm keeps its order relative to
// the tcgen05.wait::st that publishes it.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t *v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
       );
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t *v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr), "r"(v[0]),
                 "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]));
}
__device__ __forceinline__ void tmem_st4(uint32_t taddr, const uint32_t *v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(v[0]), "r"(v[1]),
                 "r"(v[2]), "r"(v[3]));
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// ------------------------------------------------------------------ helpers
// Exit layer of sorted row r: the smallest d with bin_start[d] <= r (bins in descending order),
// from the CTA's shared copy of bin_start.
__device__ __forceinline__ int tc_row_depth(const uint32_t *bin_start, uint32_t r, int L) {
    int d = L;
    for (int k = L - 1; k >= 1; --k)
        if (bin_start[k] <= r) d = k;
    return d;
}

// FINER's sin(omega0 (|z| + 1) z) in terms of the phase u = omega0 z: sin(u + u |u| k), k = 1 / omega0
__device__ __forceinline__ float finer_phase(float u, float k) { return fmaf(u * fabsf(u), k, u); }

template <int ACT>
__device__ __forceinline__ float activate(float t, float fk) {
    if (ACT == SAND_ACT_RELU) return fmaxf(t, 0.f);
    if (ACT == SAND_ACT_FINER) return __sinf(finer_phase(t, fk));
    return __sinf(t);
}

// Two activations -> one packed 16-bit pair (low half = first element) and, in the
// float32 mode, the pair of residuals h - fp16(h).
template <int MODE>
__device__ __forceinline__ void pack2(float a, float b, uint32_t &hi, uint32_t &lo) {
    if (MODE == TC_BF16) {
        __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
        hi = *reinterpret_cast<uint32_t *>(&v);
        lo = 0;
    } else {
        __half2 v = __floats2half2_rn(a, b);
        hi = *reinterpret_cast<uint32_t *>(&v);
        if (MODE == TC_SPLIT16) {
            // residuals h - fp16(h), exact in float32: one mixed-precision FMA each,
            // fp16(h) * -1 + h, straight from the packed pair
            float ra, rb;
            asm("{\n\t.reg .b16 h0, h1, m1;\n\t"
                "mov.b32 {h0, h1}, %2;\n\t"
                "mov.b16 m1, 0xBC00;\n\t"
                "fma.rn.f32.f16 %0, h0, m1, %3;\n\t"
                "fma.rn.f32.f16 %1, h1, m1, %4;\n\t}"
                : "=f"(ra), "=f"(rb)
                : "r"(hi), "f"(a), "f"(b));
            __half2 l = __floats2half2_rn(ra, rb);
            lo = *reinterpret_cast<uint32_t *>(&l);
        } else {
            lo = 0;
        }
    }
}

// Four activations -> four e4m3 bytes of one 32-bit TMEM column (first element lowest).
__device__ __forceinline__ uint32_t pack4_e4m3(float a, float b, float c, float d) {
    const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
    const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, d), __NV_SATFINITE, __NV_E4M3);
    return lo | (hi << 16);
}

template <int CH>
__device__ __forceinline__ void tmem_ld_ch(uint32_t taddr, uint32_t *r) {
    if (CH == 32) tmem_ld32(taddr, r);
    else tmem_ld16(taddr, r);
}
template <int CH>
__device__ __forceinline__ void tmem_st_half(uint32_t taddr, const uint32_t *v) {  // CH / 2 packed columns
    if (CH == 32) tmem_st16(taddr, v);
    else tmem_st8(taddr, v);
}

// ------------------------------------------------------------------ the kernel
// 16 accumulator values (units c0 .. c0+15) of this thread's row: bias, activation,
// tail partial sums and, when write_a, the packed activations into TMEM (A operand).
// GRAD: the four rows of a point (lanes 4p .. 4p+3 of a warp) carry its value (is_val) and the
// derivatives along x, y, z of every activation (forward-mode tangents): a tangent row's
// pre-activation is the derivative of the value row's, without the bias; its activation is
// cos(u) du (sine, one hardware sine of u + pi/2 for the point's u) or [u > 0] du (ReLU);
// FINER: cos(p) (1 + 2 |u| k) du with p = u + u |u| k its phase.
// ALO: a_lo is the shared-memory address of this row in the first 16 KB K-block tile of the A_lo
// operand (128-byte rows, 128-byte swizzle, tiles 1024-byte aligned), not a TMEM address.
// L1: layer 1 of raw coordinates instead, its phase straight from the row's coordinates (x0, x1,
// x2) and s (W1, b1) of every unit, read from shared memory at w1s (three float32 FMAs per unit,
// as on the CUDA-core warps); v and the bias constants unused.
template <int MODE, int ACT, int TAIL, bool GRAD = false, bool ALO = false, bool L1 = false>
__device__ __forceinline__ void epilogue16(const float *cs, int W, float c1, const uint32_t *v, int c0, bool write_a,
                                           uint32_t a_hi, uint32_t a_lo, float &sa, float &sb, bool is_val, float fk,
                                           uint32_t w1s = 0, float x0 = 0.f, float x1 = 0.f, float x2 = 0.f) {
    constexpr bool MULT = TAIL == SAND_TAIL_MULT && !L1;  // tail 1 is affine for both tail kinds
    uint32_t phi[8], plo[8], p8[4];
#pragma unroll
    for (int g = 0; g < 2; ++g) {
        const int j0 = c0 + 8 * g;
        float bv[8];
        if (!L1) {
            const float4 ba = *reinterpret_cast<const float4 *>(cs + j0);
            const float4 bb = *reinterpret_cast<const float4 *>(cs + j0 + 4);
            bv[0] = ba.x; bv[1] = ba.y; bv[2] = ba.z; bv[3] = ba.w;
            bv[4] = bb.x; bv[5] = bb.y; bv[6] = bb.z; bv[7] = bb.w;
        }
        const float4 aa = *reinterpret_cast<const float4 *>(cs + W + j0);
        const float4 ab4 = *reinterpret_cast<const float4 *>(cs + W + j0 + 4);
        const float av[8] = {aa.x, aa.y, aa.z, aa.w, ab4.x, ab4.y, ab4.z, ab4.w};
        float tbv[8];
        if (MULT) {
            const float4 t0 = *reinterpret_cast<const float4 *>(cs + 2 * W + j0);
            const float4 t1 = *reinterpret_cast<const float4 *>(cs + 2 * W + j0 + 4);
            tbv[0] = t0.x; tbv[1] = t0.y; tbv[2] = t0.z; tbv[3] = t0.w;
            tbv[4] = t1.x; tbv[5] = t1.y; tbv[6] = t1.z; tbv[7] = t1.w;
        }
        float h8[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            float hv;
            if (L1) {
                const float4 w = lds_f4(w1s + 16u * (uint32_t)(j0 + i));
                hv = activate<ACT>(fmaf(w.x, x0, fmaf(w.y, x1, fmaf(w.z, x2, w.w))), fk);
            } else if (!GRAD) {
                hv = activate<ACT>(fmaf(__uint_as_float(v[8 * g + i]), c1, bv[i]), fk);
            } else {
                const float u = fmaf(__uint_as_float(v[8 * g + i]), c1, is_val ? bv[i] : 0.f);
                const float uv = __shfl_sync(0xffffffffu, u, (threadIdx.x & 31) & ~3);  // the point's u
                if (ACT == SAND_ACT_RELU) {
                    hv = is_val ? fmaxf(u, 0.f) : (uv > 0.f ? u : 0.f);
                } else if (ACT == SAND_ACT_FINER) {
                    const float pv = finer_phase(uv, fk);  // the point's phase
                    const float sv = __sinf(is_val ? pv : pv + 1.57079632679489662f);
                    hv = is_val ? sv : sv * (u * fmaf(2.f * fabsf(uv), fk, 1.f));
                } else {
                    const float sv = __sinf(is_val ? u : uv + 1.57079632679489662f);
                    hv = is_val ? sv : sv * u;
                }
            }
            h8[i] = hv;
            sa = fmaf(av[i], hv, sa);
            if (MULT) sb = fmaf(tbv[i], hv, sb);
        }
        if (MODE == TC_FP8) {
            p8[2 * g] = pack4_e4m3(h8[0], h8[1], h8[2], h8[3]);
            p8[2 * g + 1] = pack4_e4m3(h8[4], h8[5], h8[6], h8[7]);
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) pack2<MODE>(h8[2 * i], h8[2 * i + 1], phi[4 * g + i], plo[4 * g + i]);
        }
    }
    if (write_a) {
        if (MODE == TC_FP8) {
            tmem_st4(a_hi + (uint32_t)(c0 >> 2), p8);
        } else {
            tmem_st8(a_hi + (uint32_t)(c0 >> 1), phi);
            if (MODE == TC_SPLIT16 && !ALO) tmem_st8(a_lo + (uint32_t)(c0 >> 1), plo);
            if (MODE == TC_SPLIT16 && ALO) {  // units c0 .. c0+15: two 16-byte chunks of K-block c0 / 64
                const uint32_t row = a_lo + (uint32_t)(c0 >> 6) * 16384u, sw = (a_lo >> 7) & 7u;
                const uint32_t c = (uint32_t)(c0 & 63) >> 3;
                asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(row + (((c ^ sw)) << 4)), "r"(plo[0]),
                             "r"(plo[1]), "r"(plo[2]), "r"(plo[3]) : "memory");
                asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(row + ((((c + 1) ^ sw)) << 4)), "r"(plo[4]),
                             "r"(plo[5]), "r"(plo[6]), "r"(plo[7]) : "memory");
            }
        }
    }
}

template <int MODE, int ACT, int TAIL, int VAR>
__global__ void __launch_bounds__(tc_threads(VAR), 1)
tmlp_tc_kernel(const __grid_constant__ CUtensorMap wmap, const TcParams P, const float *__restrict__ pts,
               const float4 *__restrict__ sorted, WsHeader *hdr, int64_t n, int full_depth, float *__restrict__ out) {
    constexpr int PARTS = MODE == TC_SPLIT16 ? 2 : 1;
    constexpr bool MULT = TAIL == SAND_TAIL_MULT;
    constexpr bool EXT = (VAR & 3) == 1;   // extended outputs: all tails, dynamic exit
    constexpr bool GRAD = (VAR & 3) == 2;  // value and input gradient: 32 points x 4 rows per tile
    constexpr bool CCW = (VAR & 3) == 3;   // SAND query with the exit-layer-1 rows on the CUDA-core warps
    constexpr bool ALO = (VAR & kAloVar) != 0 && MODE == TC_SPLIT16;  // A_lo in shared memory
    constexpr int PPT = GRAD ? kTileM / 4 : kTileM;  // points per tile
    constexpr int UPS = MODE == TC_FP8 ? 128 : 64;  // K-units per weight stage (one 128-byte row per unit)
    constexpr int UPK = MODE == TC_FP8 ? 32 : 16;   // K-units per MMA (32 bytes of every row)
    // A stage holds two W x 128-byte sub-blocks: the hi and lo weights of one K-block (float32
    // mode), or two consecutive K-blocks (one-part modes)
    constexpr int KBS = PARTS == 2 ? 1 : 2;         // K-blocks per stage
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int W = P.W, L = P.L;
    const int KB = (W + 63) >> 6;   // K-blocks of 64 units (the last one partial when W % 64 != 0)
    const bool drain_first = (W & 63) == 0 && KB <= 4;  // else: serial epilogue (see below)
    const int KBP = (W + 63) >> 6;  // K-blocks of the A_lo operand in shared memory (ALO)
    uint8_t *alo_base = smem;
    uint8_t *stage_base = smem + (ALO ? (size_t)KBP * 16384 : 0);
    // per-layer constants [L][NC][W]: bias', tail a (and tail b with multiplicative tails), then, for a
    // raw-coordinate layer 1 with linear tails, s (W1, b1) of every unit ([W] float4)
    constexpr int NC = MULT ? 3 : 2;
    const bool w1_smem = P.l1_fold && !MULT;
    float *c_all = reinterpret_cast<float *>(stage_base + (size_t)P.n_stages * P.stage_bytes);
    float4 *w1s = reinterpret_cast<float4 *>(c_all + (size_t)NC * L * W);
    uint64_t *bars = reinterpret_cast<uint64_t *>(w1s + (w1_smem ? W : 0));
    uint64_t *full_bar = bars;
    uint64_t *empty_bar = bars + kMaxStages;
    uint64_t *a_ready = bars + 2 * kMaxStages;  // [kb]: K-block kb of the next A operand is in TMEM (16 warps)
    uint64_t *d_full = a_ready + kMaxKBlocks;   // the layer's accumulator is complete
    uint64_t *d_drained = d_full + 1;           // every epilogue warp has read the accumulator (16 warps)
    uint64_t *drain = d_drained + 1;
    uint64_t *x_full = drain + 1;   // tail partials of slice 1 written (128 arrivals)
    uint64_t *x_empty = x_full + 1; // ... and read by slice 0 (128 arrivals)
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + kNumBars);
    volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);
    // dynamic exit: tiles whose rows have all stopped, as counts: requested by the epilogue,
    // taken up by the MMA thread
    volatile int *skip_req = reinterpret_cast<volatile int *>(tmem_slot + 2);
    volatile int *skip_done = reinterpret_cast<volatile int *>(tmem_slot + 3);
    float *tailx = reinterpret_cast<float *>(tmem_slot + 4);  // [kSlices - 1][2 values][128 rows]
    float4 *rowbuf = reinterpret_cast<float4 *>((reinterpret_cast<uintptr_t>(tailx + (kSlices - 1) * 256) + 15) &
                                                ~uintptr_t(15));  // [2][kEpiThreads]
    uint32_t *s_bin = reinterpret_cast<uint32_t *>(rowbuf + 2 * kEpiThreads);  // [16]: bin_start, read per tile

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t n_rows = full_depth ? n : (int64_t)hdr->n_active;
    // A SAND query's rows are sorted by descending exit layer.  With raw coordinates, the rows of
    // exit layer 1 (bin_start[1] .. n_rows) need only layer 1 and its tail, and two warps of
    // their own compute them on the CUDA cores (W1 x + b1, the activation, the tail) while the
    // tensor-core pipeline runs the deeper rows.  Every exit-layer-1 row takes that path,
    // wherever it falls, so a row's result does not depend on the other rows of the query.
    const bool cc_on = CCW && !full_depth && P.cc;
    const int64_t n_tc_rows = cc_on ? (int64_t)hdr->bin_start[1] : n_rows;  // tensor-core rows
    const int64_t n_tiles = (n_tc_rows + PPT - 1) / PPT;
    auto tile_depth = [&](int64_t t) -> int { return full_depth ? L : tc_row_depth(s_bin, (uint32_t)(t * PPT), L); };
    // Layer 1 of raw coordinates (linear tails) runs on the epilogue warps' CUDA cores (three FMAs
    // per unit from the coordinates, no MMA and no accumulator drain), except in the gradient
    // variant, which keeps the folded K = 16 MMA; the tensor cores then start at layer 2.
    const bool l1cc = !GRAD && w1_smem;
    const int l_mma0 = l1cc ? 2 : P.first_mma;  // first layer on the tensor cores

    if (threadIdx.x == 0) {
        for (int s = 0; s < P.n_stages; ++s) {
            mbar_init(smem_u32(&full_bar[s]), 1);
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        for (int kb = 0; kb < kMaxKBlocks; ++kb) mbar_init(smem_u32(&a_ready[kb]), kEpiWarps);
        mbar_init(smem_u32(d_full), 1);
        mbar_init(smem_u32(d_drained), kEpiWarps);
        mbar_init(smem_u32(drain), 1);
        mbar_init(smem_u32(x_full), (kSlices - 1) * 128);
        mbar_init(smem_u32(x_empty), 128);
        *abort = 0;
        *skip_req = 0;
        *skip_done = 0;
        for (int k = 0; k < 16; ++k) s_bin[k] = hdr->bin_start[k];
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(P.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (warp >= 2 && warp < 2 + kEpiWarps) {  // constants of every layer, resident for the whole kernel
        for (int i = threadIdx.x - 64; i < NC * L * W; i += kEpiThreads) {
            const int l = i / (NC * W), c = (i / W) % NC, j = i % W;
            c_all[i] = __ldg(P.cvec + ((size_t)l * 3 + c) * W + j);
        }
        if (w1_smem)
            for (int j = threadIdx.x - 64; j < W; j += kEpiThreads) w1s[j] = __ldg(P.w1p + j);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t a_hi = tmem + (uint32_t)W, a_lo = tmem + (uint32_t)(W + W / 2);

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            uint32_t it = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
                const int Dt = tile_depth(t);
                for (int l = l_mma0; l <= Dt && ok; ++l) {
                    const int kb_n = ((l == 1 ? P.D : W) + UPS - 1) / UPS;
                    const bool fold_l = l == 1 && P.l1_fold;
                    const int parts_l = fold_l ? 1 : PARTS;  // the folded layer 1 has one block
                    // ALO: one part of one K-block per stage (hi of kb, then lo of kb)
                    const int sb_n = ALO ? (fold_l ? 1 : 2 * kb_n) : (kb_n + KBS - 1) / KBS;
                    for (int sb = 0; sb < sb_n && ok; ++sb, ++it) {
                        const uint32_t s = it % P.n_stages, ph = (it / P.n_stages) & 1;
                        ok = mbar_wait(smem_u32(&empty_bar[s]), ph ^ 1, abort, hdr, 1, true, P.wait_ns);
                        if (!ok) break;
                        // sub-block j: part j of K-block sb (float32 mode), or K-block KBS sb + j
                        const int subs = ALO ? 1 : PARTS == 2 ? parts_l : min(KBS, kb_n - sb * KBS);
                        mbar_arrive_tx(smem_u32(&full_bar[s]), (uint32_t)subs * (uint32_t)W * 128u);
                        for (int j = 0; j < subs; ++j) {
                            const int p = ALO ? (fold_l ? 0 : (sb & 1)) : PARTS == 2 ? j : 0;
                            const int kb = ALO ? (fold_l ? 0 : (sb >> 1)) : PARTS == 2 ? sb : sb * KBS + j;
                            const int row0 = ((l - P.first_mma) * PARTS + p) * W;
                            for (int bx = 0; bx < W; bx += P.box_rows)  // one box of W rows, or two of W/2
                                tma_load_2d(smem_u32(stage_base + (size_t)s * P.stage_bytes + (size_t)(j * W + bx) * 128),
                                            &wmap, smem_u32(&full_bar[s]), kb * UPS, row0 + bx);
                        }
                    }
                }
            }
            if (!ok) {  // drain copies still in flight before the CTA can exit
                const uint32_t first = it > (uint32_t)P.n_stages ? it - P.n_stages : 0u;
                for (uint32_t k = first; k < it; ++k) {
                    const uint32_t s = k % P.n_stages, ph = (k / P.n_stages) & 1;
                    const uint64_t t0 = globaltimer();
                    while (!mbar_try(smem_u32(&full_bar[s]), ph) && globaltimer() - t0 < kTimeoutNs) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t ab = MODE == TC_BF16 ? 1u : 0u;
            const int n0 = W <= 256 ? W : P.n_split, n1 = W - n0;  // MMA N <= 256: two column groups when W > 256
            const uint32_t id_base = (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(kTileM >> 4) << 24);
            const uint32_t idesc0 = id_base | ((uint32_t)(n0 >> 3) << 17);
            const uint32_t idesc1 = id_base | ((uint32_t)(n1 >> 3) << 17);
            const uint32_t id_l1 = (1u << 4) | ((uint32_t)(kTileM >> 4) << 24);  // fp16 operands, fp32 accumulate
            const uint32_t idesc0_l1 = id_l1 | ((uint32_t)(n0 >> 3) << 17);
            const uint32_t idesc1_l1 = id_l1 | ((uint32_t)(n1 >> 3) << 17);
            // At a layer boundary the tensor pipe is idle until this thread issues again, and the
            // epilogue warps sharing its SM sub-partition are busy then, so every instruction
            // between the accumulator's release and the first MMA counts: the stage ring position
            // is kept as running counters (no division), and the first weight stage of a layer is
            // waited for before the accumulator is (its copy landed long before).
            uint32_t s = 0, ph = 0, pdr = 0;
            const uint64_t bd_base = smem_desc(smem_u32(stage_base));
            const uint64_t bd_step = (uint64_t)(P.stage_bytes >> 4);  // descriptor units per stage
            uint32_t pa[kMaxKBlocks] = {0, 0, 0, 0, 0, 0};
            bool ok = true, any_layer = false;
            bool drained_credit = false;  // dynamic exit: the last drained accumulator was not overwritten
            const bool dyn = EXT && P.dyn_r > 0.f;
            int skips_seen = 0;
            for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
                const int Dt = tile_depth(t);
                bool tile_skip = false;
                for (int l = l_mma0; l <= Dt && ok && !tile_skip; ++l) {
                    const int K = l == 1 ? P.D : W;
                    const int kb_n = (K + UPS - 1) / UPS;
                    const int ks_n = (K + UPK - 1) / UPK;  // the last FP8 K-step may be half zero padding
                    int e_seen = -1;  // last 64-unit block of the A operand waited for in this layer
                    ok = mbar_wait(smem_u32(&full_bar[s]), ph, abort, hdr, 3, true, P.wait_ns);
                    if (!ok) break;
                    if (any_layer && drained_credit) {
                        drained_credit = false;
                    } else if (any_layer) {  // the previous layer's accumulator has been read out
                        ok = mbar_wait(smem_u32(d_drained), pdr, abort, hdr, 8, true, P.wait_ns);
                        pdr ^= 1;
                        if (!ok) break;
                    }
                    any_layer = true;
                    const bool fold = l == 1 && P.l1_fold;
                    const int sb_n = ALO ? (fold ? 1 : 2 * kb_n) : (kb_n + KBS - 1) / KBS;
                    for (int sb = 0; sb < sb_n && ok; ++sb) {
                        if (sb > 0) ok = mbar_wait(smem_u32(&full_bar[s]), ph, abort, hdr, 3, true, P.wait_ns);
                        if (!ok) break;
                        tc_fence_after();
                        const uint64_t bd_stage = bd_base + (uint64_t)s * bd_step;
                        const int part = ALO && !fold ? (sb & 1) : 0;  // ALO: the stage's weights are hi (0) or lo (1)
                        for (int jb = 0; jb < KBS && ok && !tile_skip; ++jb) {
                            const int kb = ALO ? (fold ? 0 : sb >> 1) : sb * KBS + jb;
                            if (kb >= kb_n) break;
                            const uint64_t bd = bd_stage + (uint64_t)(jb * W) * 8u;  // this K-block's sub-block
                            const uint64_t bd_lo = bd_stage + (uint64_t)W * 8u;  // float32 mode: the lo weights
                            const int nks = min(4, ks_n - kb * 4);  // K-steps of this stage holding real units
                            // runs of K-steps that read one 64-unit block of the A operand: the whole
                            // stage (16-bit operands), or halves of it (FP8: 128 units per stage)
                            constexpr int SEG = MODE == TC_FP8 ? 2 : 4;
                            for (int g0 = 0; g0 < nks && ok; g0 += SEG) {
                                const int g = kb * 4 + g0;
                                const int e = (g * UPK) >> 6;  // block of the A operand these K-steps read
                                if (e > e_seen) {
                                    ok = mbar_wait(smem_u32(&a_ready[e]), pa[e], abort, hdr, 2, true, P.wait_ns);
                                    pa[e] ^= 1;
                                    e_seen = e;
                                    if (!ok) break;
                                    tc_fence_after();
                                    if (dyn && e == 0 && *skip_req > skips_seen) {  // every row of the tile has stopped
                                        *skip_done = ++skips_seen;
                                        tile_skip = true;
                                        break;
                                    }
                                }
                                const int cnt = min(SEG, nks - g0);
                                const uint32_t acol = (uint32_t)g * 8u;  // 16 fp16 or 32 e4m3 K-elements = 8 TMEM columns
                                const uint32_t acc = g != 0 ? 1u : 0u;
                                const uint32_t a_op = a_hi + acol;
                                if (fold) {  // layer 1: one fp16 K-step per column group, whatever the mode
                                    mma_ts<TC_F16>(tmem, a_op, bd, idesc0_l1, 0u);
                                    if (n1 > 0) mma_ts<TC_F16>(tmem + (uint32_t)n0, a_op, bd + (uint64_t)n0 * 8u, idesc1_l1, 0u);
                                    continue;
                                }
                                for (int grp = 0; grp < (n1 > 0 ? 2 : 1); ++grp) {
                                    // column group grp: accumulator columns and B rows from n0 on for grp 1
                                    const uint32_t dcol = grp ? tmem + (uint32_t)n0 : tmem;
                                    const uint32_t id = grp ? idesc1 : idesc0;
                                    const uint64_t goff = (uint64_t)(2 * g0) + (grp ? (uint64_t)n0 * 8u : 0u);
                                    const uint64_t bk = bd + goff;
                                    if (ALO) {  // A_hi B_hi + A_lo B_hi (hi stage) or A_hi B_lo (lo stage)
                                        const uint32_t alo_k = smem_u32(alo_base) + (uint32_t)kb * 16384u + 32u * (uint32_t)g0;
                                        for (int k = 0; k < cnt; ++k) {
                                            if (part == 0) {
                                                mma_ts<MODE>(dcol, a_op + 8u * k, bk + 2u * k, id, k == 0 ? acc : 1u);
                                                mma_f16(dcol, smem_desc(alo_k + 32u * k), bk + 2u * k, id, 1u);
                                            } else {
                                                mma_ts<MODE>(dcol, a_op + 8u * k, bk + 2u * k, id, 1u);
                                            }
                                        }
                                    } else if (PARTS == 2 && cnt == 4) {
                                        mma_k4x2(dcol, a_op, a_lo + acol, bk, id, acc);   // A_hi B_hi + A_lo B_hi
                                        mma_k4<MODE>(dcol, a_op, bd_lo + goff, id, 1u);  // A_hi B_lo
                                    } else if (cnt == 4) {
                                        mma_k4<MODE>(dcol, a_op, bk, id, acc);
                                    } else if (cnt == 2 && PARTS == 1) {
                                        mma_k2<MODE>(dcol, a_op, bk, id, acc);
                                    } else {  // a ragged last stage: one K-step at a time
                                        for (int k = 0; k < cnt; ++k) {
                                            const uint32_t ak = k == 0 ? acc : 1u;
                                            mma_ts<MODE>(dcol, a_op + 8u * k, bk + 2u * k, id, ak);
                                            if (PARTS == 2) {
                                                mma_ts<MODE>(dcol, a_lo + acol + 8u * k, bk + 2u * k, id, 1u);
                                                mma_ts<MODE>(dcol, a_op + 8u * k, bd_lo + goff + 2u * k, id, 1u);
                                            }
                                        }
                                    }
                                }
                            }
                        }
                        if (tile_skip) break;
                        if (ok) mma_commit(smem_u32(&empty_bar[s]));
                        if (++s == (uint32_t)P.n_stages) { s = 0; ph ^= 1; }
                    }
                    if (tile_skip) {
                        // hand back every weight stage the producer loads for the rest of this tile:
                        // the current one (waited for, unused) and those of layers l .. Dt still to come
                        mbar_arrive(smem_u32(&empty_bar[s]));
                        if (++s == (uint32_t)P.n_stages) { s = 0; ph ^= 1; }
                        int rest = sb_n - 1;
                        for (int l2 = l + 1; l2 <= Dt; ++l2)
                            rest += ALO ? 2 * ((W + UPS - 1) / UPS) : ((W + UPS - 1) / UPS + KBS - 1) / KBS;
                        for (int k = 0; k < rest && ok; ++k) {
                            ok = mbar_wait(smem_u32(&full_bar[s]), ph, abort, hdr, 9, true, P.wait_ns);
                            if (!ok) break;
                            mbar_arrive(smem_u32(&empty_bar[s]));
                            if (++s == (uint32_t)P.n_stages) { s = 0; ph ^= 1; }
                        }
                        drained_credit = true;  // layer l's accumulator drain was waited for, and nothing wrote it since
                        break;
                    }
                    if (ok) mma_commit(smem_u32(d_full));
                }
            }
            if (!ok) {  // let every issued MMA finish before TMEM is released
                mma_commit(smem_u32(drain));
                const uint64_t t0 = globaltimer();
                while (!mbar_try(smem_u32(drain), 0) && globaltimer() - t0 < kTimeoutNs) {
                }
            }
        }
        __syncwarp();
    } else if (warp < 2 + kEpiWarps) {
        // ------------------------------------------------ epilogue warps 2..9
        const int q = warp & 3;                 // TMEM lane quadrant
        const int slice = (warp - 2) >> 2;      // which half of every K-block
        const int su0 = kSliceUnits * slice;    // first unit of this thread in every K-block
        const int r = q * 32 + lane;            // tile row
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        const uint32_t t_lane = tmem + lane_off;
        const uint32_t a_hi_l = a_hi + lane_off;
        // ALO: this row's address in the first A_lo tile in shared memory; else its TMEM lane
        const uint32_t a_lo_l = ALO ? smem_u32(alo_base) + (uint32_t)r * 128u : a_lo + lane_off;
        uint32_t pd = 0, px = 0;
        bool ok = true;
        auto signal = [&](uint64_t *bar, bool after_st) {  // this warp's share is done
            if (after_st) tmem_wait_st();
            if (ALO && after_st) fence_async_smem();  // the A_lo stores -> visible to the tensor core
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(bar));
        };
        // Tail exchange through two mbarriers (bounded waits): slice 1 publishes its
        // partial dot products, slice 0 adds them to its own.
        auto exchange = [&](float &sa, float &sb) {
            if (slice != 0) {
                ok = mbar_wait(smem_u32(x_empty), px ^ 1, abort, hdr, 6, false, P.wait_ns) && ok;
                ok = __all_sync(0xffffffffu, ok);
                px ^= 1;
                tailx[(slice - 1) * 256 + r] = sa;
                if (MULT) tailx[(slice - 1) * 256 + 128 + r] = sb;
                mbar_arrive(smem_u32(x_full));
            } else {
                ok = mbar_wait(smem_u32(x_full), px, abort, hdr, 7, false, P.wait_ns) && ok;
                ok = __all_sync(0xffffffffu, ok);
                px ^= 1;
#pragma unroll
                for (int k = 0; k < kSlices - 1; ++k) {
                    sa += tailx[k * 256 + r];
                    if (MULT) sb += tailx[k * 256 + 128 + r];
                }
                mbar_arrive(smem_u32(x_empty));
            }
        };
        uint32_t q8[4];  // FP8: units c0-8 .. c0+7 (16-unit groups) go out as one 4-column store
        auto st_a8 = [&](int c0, const float *h8) {  // 8 activations of units c0..c0+7 into TMEM
            if (MODE == TC_FP8) {  // c0 runs over both halves of an aligned 16-unit group, low half first
                const int o = (c0 & 8) >> 2;
                q8[o] = pack4_e4m3(h8[0], h8[1], h8[2], h8[3]);
                q8[o + 1] = pack4_e4m3(h8[4], h8[5], h8[6], h8[7]);
                if (o) tmem_st4(a_hi_l + (uint32_t)((c0 - 8) >> 2), q8);
            } else {
                uint32_t phi[4], plo[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) pack2<MODE>(h8[2 * i], h8[2 * i + 1], phi[i], plo[i]);
                asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a_hi_l + (uint32_t)(c0 >> 1)),
                             "r"(phi[0]), "r"(phi[1]), "r"(phi[2]), "r"(phi[3]));
                if (MODE == TC_SPLIT16 && !ALO)  // (ALO serves raw-coordinate models only: no Fourier layer 1)
                    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a_lo_l + (uint32_t)(c0 >> 1)),
                                 "r"(plo[0]), "r"(plo[1]), "r"(plo[2]), "r"(plo[3]));
            }
        };
        if (MODE == TC_FP8 && (W & 31) == 16 && slice == 0) {
            // units W .. W+15 of the last FP8 K-step meet zero weights; they must hold finite values
            const uint32_t z[4] = {0u, 0u, 0u, 0u};
            tmem_st4(a_hi_l + (uint32_t)(W >> 2), z);
        }
        // This thread's row of tile tt (coordinates, exit layer, original index; -1 for padding),
        // copied asynchronously into buffer `buf` of its own 16-byte slot one tile ahead
        // (prefetch_row) and read from there (take_row).  Each thread copies and reads only its
        // own slot, and the two buffers alternate, so no other thread's copy is waited for and
        // no copy lands on a slot whose last read has not been consumed.
        const int et = threadIdx.x - 64;
        auto row_of = [&](int64_t tt) -> int64_t { return GRAD ? tt * PPT + (r >> 2) : tt * kTileM + r; };
        auto prefetch_row = [&](int64_t tt, int buf) {
            const int64_t row = row_of(tt);
            if (tt < n_tiles && row < n_tc_rows) {
                const uint32_t dst = smem_u32(rowbuf + buf * kEpiThreads + et);
                if (full_depth) {  // [n][3] floats, 4-byte aligned
                    cp_async4(dst, pts + 3 * row);
                    cp_async4(dst + 4, pts + 3 * row + 1);
                    cp_async4(dst + 8, pts + 3 * row + 2);
                } else {
                    cp_async16(dst, sorted + row);
                }
            }
            cp_async_commit();
        };
        auto take_row = [&](int64_t tt, int buf) {
            cp_async_wait_all();
            TcRow a{0.f, 0.f, 0.f, 0, -1};
            const int64_t row = row_of(tt);
            if (tt < n_tiles && row < n_tc_rows) {
                const float4 v = rowbuf[buf * kEpiThreads + et];
                a.x0 = v.x; a.x1 = v.y; a.x2 = v.z;
                if (full_depth) {
                    a.idx = row;
                    a.d = L;
                } else {
                    a.idx = __float_as_int(v.w);
                    a.d = tc_row_depth(s_bin, (uint32_t)row, L);
                }
            }
            return a;
        };
        // The A operand of a folded layer 1: 256 x = x_h + x_m + x_l exactly (three fp16 parts,
        // each the rounded residual of the last); K slots [x_h, x_m, x_l, x_h, x_m] x (x, y, z), 0
        // against the packed weights.  Written by one warp per quadrant, signalled by all.
        auto put_a1 = [&](const TcRow &a) {
            if (slice == 0) {
                const float xs[3] = {a.x0 * P.x_scale, a.x1 * P.x_scale, a.x2 * P.x_scale};
                __half hp[3][3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const __half h = __float2half_rn(xs[c]);
                    const float r1 = xs[c] - __half2float(h);
                    const __half m = __float2half_rn(r1);
                    const __half lo = __float2half_rn(r1 - __half2float(m));
                    hp[c][0] = h; hp[c][1] = m; hp[c][2] = lo;
                }
                __half k16[16];
#pragma unroll
                for (int g = 0; g < 5; ++g)
#pragma unroll
                    for (int c = 0; c < 3; ++c) k16[3 * g + c] = hp[c][g < 3 ? g : g - 3];
                k16[15] = __float2half_rn(0.f);
                uint32_t v8[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    __half2 pr = __halves2half2(k16[2 * i], k16[2 * i + 1]);
                    v8[i] = *reinterpret_cast<uint32_t *>(&pr);
                }
                tmem_st8(a_hi_l, v8);
            }
            signal(&a_ready[0], true);
        };
        const int comp = GRAD ? (r & 3) : 0;  // GRAD: 0 = value row, 1..3 = d/dx, d/dy, d/dz row
        const bool is_val = comp == 0;
        // the layer-1 A operand of a row: its coordinates, or (tangent rows) a unit vector; one
        // call for the whole warp (put_a1 holds warp-collective TMEM stores), the row per lane
        auto put_a1_row = [&](const TcRow &row) {
            TcRow a1 = row;
            if (GRAD && !is_val) {
                a1.x0 = comp == 1 ? 1.f : 0.f;
                a1.x1 = comp == 2 ? 1.f : 0.f;
                a1.x2 = comp == 3 ? 1.f : 0.f;
            }
            put_a1(a1);
        };
        // Layer 1 of raw coordinates on the CUDA cores (l1cc): this thread's units of every K-block,
        // written (write_a) as the A operand of layer 2 one K-block at a time, each K-block
        // released to the MMAs as it is done (sig); returns this thread's partial sum of tail 1.
        auto layer1 = [&](const TcRow &a, bool write_a, bool sig) -> float {
            float s1 = 0.f, s1b = 0.f;
            for (int kb = 0; kb < KB; ++kb) {
                for (int c0 = 64 * kb + su0; c0 < 64 * kb + su0 + kSliceUnits && c0 < W; c0 += 16)
                    epilogue16<MODE, ACT, TAIL, false, ALO, true>(c_all, W, 0.f, nullptr, c0, write_a, a_hi_l, a_lo_l, s1, s1b,
                                                                  true, P.finer_k, smem_u32(w1s), a.x0, a.x1, a.x2);
                if (write_a && sig) signal(&a_ready[kb], true);
            }
            return s1;
        };
        int buf = 0;
        prefetch_row(blockIdx.x, 0);
        // Dynamic exit: a skipped tile hands the MMA thread its a_ready[0] phase with no MMA after it,
        // so before a tile sends anything the MMA thread must have taken up every earlier skip (else
        // a second phase of a_ready[0] could complete before it has seen the first, and its parity
        // wait would miss both).  Bounded like every wait.
        int my_skips = 0;
        auto skips_taken = [&]() -> bool {
            const uint64_t t0 = globaltimer();
            bool good = true;
            while (*skip_done < my_skips) {
                if (globaltimer() - t0 > P.wait_ns) {
                    good = false;
                    break;
                }
            }
            good = __all_sync(0xffffffffu, good);
            if (!good) {
                *abort = 1;
                atomicOr(&hdr->flags, (uint32_t)SAND_FLAG_TIMEOUT);
                atomicExch(&hdr->timeout_where, 10u);
            }
            return good;
        };
        for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x, buf ^= 1) {
            if (EXT && P.dyn_r > 0.f && my_skips > 0) {
                // every epilogue warp takes the same decision (named barriers follow in the tile)
                if (named_count(1, kEpiThreads, !skips_taken()) > 0) {
                    ok = false;
                    break;
                }
            }
            const int Dt = tile_depth(t);
            const TcRow cur = take_row(t, buf);
            prefetch_row(t + gridDim.x, buf ^ 1);  // the next tile's rows, in flight during this tile
            const int d = cur.d;
            const int64_t idx = cur.idx;
            const float x0 = cur.x0, x1 = cur.x1, x2 = cur.x2;
            float y = 0.f;
            bool alive = idx >= 0;  // dynamic exit: this row still runs
            // ---- layer 1 on the CUDA cores; or the A operand of layer 1: split coordinates, or the
            // Fourier features
            int l_end = Dt;  // last layer of this tile on the tensor cores
            if (l1cc) {
                const bool dyn = EXT && P.dyn_r > 0.f;
                const bool more = Dt >= 2;
                float s1 = layer1(cur, more, more && !dyn);
                float s1b = 0.f;
                exchange(s1, s1b);
                if (slice == 0) {
                    y = s1 + __ldg(P.tb);  // tail 1 (affine for both tail kinds)
                    if (dyn) {
                        if (alive && (fabsf(y) < P.dyn_r || !more)) {  // the row stops here
                            out[idx] = y;
                            if (P.exit_out) P.exit_out[idx] = (uint8_t)1;
                            alive = false;
                        }
                    } else if (EXT && P.all_tails) {
                        if (idx >= 0) out[idx * L] = y;
                    } else if (d == 1 && idx >= 0) {
                        out[idx] = y;
                    }
                }
                if (dyn && more) {  // as after every layer below: go on, or skip the rest of the tile
                    const int n_alive = named_count(1, kEpiThreads, slice == 0 && alive);
                    if (n_alive > 0) {
                        for (int kb = 0; kb < KB; ++kb) signal(&a_ready[kb], true);
                    } else {
                        ++my_skips;
                        if (threadIdx.x == 64) *skip_req = my_skips;
                        signal(&a_ready[0], true);
                        l_end = 0;
                    }
                }
            } else if (P.l1_fold) {
                put_a1_row(cur);
            } else {
                // Fourier features gamma(x) = [sin 2 pi s, cos 2 pi s]; in_dim == W, same slices as the layers
                for (int kb = 0; kb < KB; ++kb) {
                    for (int k0 = 64 * kb + su0; k0 < 64 * kb + su0 + kSliceUnits && k0 < W; k0 += 8) {
                        float h8[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int k = k0 + i;
                            const int kk = k < P.m ? k : k - P.m;
                            const float ph = fourier_phase(P.B + 3 * kk, x0, x1, x2);
                            float sv, cv;
                            sincospif(2.0f * ph, &sv, &cv);
                            // tangent rows: d gamma / dx_c = 2 pi B_kc (cos, -sin)
                            const float bk = GRAD ? P.B[3 * kk + (is_val ? 0 : comp - 1)] : 0.f;
                            const float tv = 6.28318530717958647692f * bk * (k < P.m ? cv : -sv);
                            h8[i] = (GRAD && !is_val) ? tv : (k < P.m ? sv : cv);
                        }
                        st_a8(k0, h8);
                    }
                    signal(&a_ready[kb], true);
                }
            }
            // ---- tensor-core layers
            for (int l = l_mma0; l <= l_end && ok; ++l) {
                ok = mbar_wait(smem_u32(d_full), pd, abort, hdr, 4, false, P.wait_ns) && ok;
                ok = __all_sync(0xffffffffu, ok);  // the TMEM loads below are warp-collective
                pd ^= 1;
                if (!ok) break;
                tc_fence_after();
                const bool last = l == Dt;
                const bool dyn = EXT && P.dyn_r > 0.f;
                const float *cs = c_all + (size_t)(l - 1) * NC * W;
                const float c1 = P.c1[l - 1];
                float sa = 0.f, sb = 0.f;
                if (!drain_first) {
                    // serial: each K-block read, computed and stored in turn; the next layer may start
                    // overwriting the accumulator only once every warp has read all of it
                    for (int kb = 0; kb < KB; ++kb) {
                        for (int c0 = 64 * kb + su0; c0 < 64 * kb + su0 + kSliceUnits && c0 < W; c0 += 16) {
                            uint32_t v[16];
                            tmem_ld16(t_lane + (uint32_t)c0, v);
                            tmem_wait_ld();
                            epilogue16<MODE, ACT, TAIL, GRAD, ALO>(cs, W, c1, v, c0, !last, a_hi_l, a_lo_l, sa, sb, is_val, P.finer_k);
                        }
                        if (!last && !dyn) signal(&a_ready[kb], true);
                    }
                    signal(d_drained, false);
                } else {
                    // drain the accumulator into registers: K-block 0 first, the others load while
                    // K-block 0 is computed; the next layer starts once all are in
                    uint32_t v[4][kSliceUnits];
                    tmem_ld32(t_lane + (uint32_t)su0, v[0]);
                    tmem_wait_ld();
#pragma unroll
                    for (int kb = 1; kb < 4; ++kb)
                        if (kb < KB) tmem_ld32(t_lane + (uint32_t)(64 * kb + su0), v[kb]);
                    epilogue16<MODE, ACT, TAIL, GRAD, ALO>(cs, W, c1, v[0], su0, !last, a_hi_l, a_lo_l, sa, sb, is_val, P.finer_k);
                    epilogue16<MODE, ACT, TAIL, GRAD, ALO>(cs, W, c1, v[0] + 16, su0 + 16, !last, a_hi_l, a_lo_l, sa, sb, is_val, P.finer_k);
                    tmem_wait_ld();
                    signal(d_drained, false);  // the next layer may overwrite the accumulator
                    if (!last && !dyn) signal(&a_ready[0], true);
#pragma unroll
                    for (int kb = 1; kb < 4; ++kb) {
                        if (kb < KB) {
                            epilogue16<MODE, ACT, TAIL, GRAD, ALO>(cs, W, c1, v[kb], 64 * kb + su0, !last, a_hi_l, a_lo_l, sa, sb, is_val, P.finer_k);
                            epilogue16<MODE, ACT, TAIL, GRAD, ALO>(cs, W, c1, v[kb] + 16, 64 * kb + su0 + 16, !last, a_hi_l,
                                                              a_lo_l, sa, sb, is_val, P.finer_k);
                            if (!last && !dyn) signal(&a_ready[kb], true);
                        }
                    }
                }
                exchange(sa, sb);
                if (GRAD && slice == 0) {
                    // value row: the tail; tangent row: its derivative (product rule for Eq. 3);
                    // y holds the value, or the gradient component along x_comp
                    const float sa_v = __shfl_sync(0xffffffffu, sa, lane & ~3);
                    const float sb_v = __shfl_sync(0xffffffffu, sb, lane & ~3);
                    const float tb0 = __ldg(P.tb + 2 * (l - 1)), tb1 = __ldg(P.tb + 2 * (l - 1) + 1);
                    float tl;
                    if (is_val) tl = (MULT && l >= 2) ? (sa + tb0) * (sb + tb1) : sa + tb0;
                    else tl = (MULT && l >= 2) ? sa * (sb_v + tb1) + (sa_v + tb0) * sb : sa;
                    y += tl;
                    if (d == l && idx >= 0) {
                        if (!is_val) P.grad[3 * idx + comp - 1] = y;
                        else if (out) out[idx] = y;  // a full-depth gradient query may omit the values
                    }
                } else if (slice == 0) {
                    const float t0v = sa + __ldg(P.tb + 2 * (l - 1));
                    float tl = t0v;
                    if (MULT && l >= 2) tl = t0v * (sb + __ldg(P.tb + 2 * (l - 1) + 1));
                    y += tl;
                    if (dyn) {
                        if (alive && (fabsf(tl) < P.dyn_r || last)) {  // the row stops here
                            out[idx] = y;
                            if (P.exit_out) P.exit_out[idx] = (uint8_t)l;
                            alive = false;
                        }
                    } else if (EXT && P.all_tails) {
                        if (idx >= 0) out[idx * L + (l - 1)] = y;
                    } else if (d == l && idx >= 0) {
                        out[idx] = y;
                    }
                }
                if (dyn && !last) {
                    // the tile goes on while any of its rows does: release the next layer (its A
                    // operand is in TMEM already), or tell the MMA thread to skip the tile's rest
                    const int n_alive = named_count(1, kEpiThreads, slice == 0 && alive);
                    if (n_alive > 0) {
                        for (int kb = 0; kb < KB; ++kb) signal(&a_ready[kb], true);
                    } else {
                        ++my_skips;
                        if (threadIdx.x == 64) *skip_req = my_skips;
                        signal(&a_ready[0], true);
                        break;
                    }
                }
            }
        }
        cp_async_wait_all();  // after an abort a prefetched row copy may still be in flight
    } else if (CCW && cc_on) {
        // ------------------------------------------------ CUDA-core warps: exit-layer-1 rows
        // Each thread takes eight rows at a time (r + 64 k of a 512-row step; steps strided over
        // the CTAs), sharing every weight load between them, so that eight independent chains
        // cover the latency of the load, the sine and the tail FMA: the phase
        // W1' x + b1' of every unit (omega0 folded into W1', b1'), the activation, and tail 1
        // (affine for both tail kinds).  The next step's rows load meanwhile.
        constexpr int kCcRows = 8, kCcStep = 32 * kCcWarps * kCcRows;
        const int ct = threadIdx.x - (64 + kEpiThreads);
        const int64_t n_cc = n_rows - n_tc_rows;
        const int64_t stride = (int64_t)gridDim.x * kCcStep;
        const float *ta = c_all + W;  // layer 1's tail weights
        const float tb0 = __ldg(P.tb);
        auto load4 = [&](int64_t base, float4 *v) {
#pragma unroll
            for (int k = 0; k < kCcRows; ++k) {
                const int64_t i = base + 32 * kCcWarps * k;
                v[k] = i < n_cc ? sorted[n_tc_rows + i] : make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
            }
        };
        int64_t base = (int64_t)blockIdx.x * kCcStep + ct;
        float4 v[kCcRows];
        load4(base, v);
        while (base < n_cc) {
            float4 vn[kCcRows];
            load4(base + stride, vn);
            float s[kCcRows];
#pragma unroll
            for (int k = 0; k < kCcRows; ++k) s[k] = 0.f;
#pragma unroll 4
            for (int j = 0; j < W; ++j) {
                // the same unit in every lane: one broadcast (from shared memory with linear tails)
                const float4 w = MULT ? __ldg(P.w1p + j) : lds_f4(smem_u32(w1s + j));
                const float a = ta[j];
#pragma unroll
                for (int k = 0; k < kCcRows; ++k)
                    s[k] = fmaf(a, activate<ACT>(fmaf(w.x, v[k].x, fmaf(w.y, v[k].y, fmaf(w.z, v[k].z, w.w))), P.finer_k), s[k]);
            }
#pragma unroll
            for (int k = 0; k < kCcRows; ++k) {
                const int idx = __float_as_int(v[k].w);
                if (idx >= 0) out[idx] = s[k] + tb0;
                v[k] = vn[k];
            }
            base += stride;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(P.tmem_cols) : "memory");
    }
}

// Launch one instantiation (defined in the per-mode translation units).  VAR 0: the plain
// query; 1: the extended outputs (all tails, dynamic exit); 2: value and input gradient;
// 3: a SAND query on raw coordinates with its exit-layer-1 rows on the CUDA-core warps.
// The plain query path carries none of the others' code, which its single MMA-issuing
// thread would otherwise pay for at every layer.
template <int MODE, int VAR>
cudaError_t launch_tc_mode(const CUtensorMap &map, const TcParams &P, int act, int tail, const float *pts,
                           const float4 *sorted, WsHeader *hdr, int64_t n, int full_depth, float *out, int grid,
                           size_t smem, cudaStream_t s);

size_t tc_smem_bytes(const TcParams &P, int parts);

}  // namespace sand
