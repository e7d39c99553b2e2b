// Tensor-core T-MLP kernel for sm_103a (tcgen05 MMA, TMEM accumulators, TMA).
//
// Evaluates Eq. 2 (and Eq. 3 for multiplicative tails) for 128-row tiles of
// points sorted by descending exit layer.  One persistent CTA per SM, 320 threads:
//   warp 0      TMA producer: streams weight tiles (64 K-columns x W/2 units, one
//               N-half of one K-block of one layer) from L2 into a ring of stages,
//               128-byte swizzled (the K-major layout the MMA reads).
//   warp 1      owns the TMEM accumulator (W fp32 columns) and issues tcgen05.mma
//               from one thread.  Each layer is two accumulators, D0 = units
//               [0, W/2) and D1 = [W/2, W), computed one after the other.
//   warps 2..5  epilogue of D0, warps 6..9 epilogue of D1.  Thread (quadrant q,
//               lane i) owns tile row 32 q + i (TMEM lane restriction).  Layer 1
//               (on the CUDA cores, float32), bias, sine, tails, the running sum
//               y_l = y_{l-1} + t_l and the write at each row's exit layer; the new
//               activations go back to shared memory as the next A operand.
// Overlap: while D1's MMAs run, warps 2-5 turn D0 into activations.  D1 reads the
// first K-half of A first and commits a barrier (a0_free) once it has, so warps
// 2-5 may overwrite that half with the next layer's input; the next layer's MMAs
// on that K-half start while warps 6-9 are still finishing D1.
// A tile runs to the exit layer of its first (deepest) row; rows whose exit layer
// was reached ride along only in the one tile per exit layer that straddles two
// layers; tiles of exit layer 1 never touch the tensor cores.
//
// Precision modes (hidden-layer products only; everything else is float32):
//   SPLIT16  a = a_hi + a_lo and w*s = w_hi + w_lo with fp16 terms (s = 2^-e per
//            layer, so max|w s| is in [0.5, 1)); D = A_hi B_hi + A_lo B_hi + A_hi B_lo.
//   F16/BF16 one product with fp16 (scaled) / bf16 operands.
// Sine: the argument is formed in revolutions, t = acc * w0/(2 pi s) + w0 b/(2 pi)
// (one rounding, like forming it in radians), reduced exactly, f = t - rint(t), and
// the hardware sine is applied to 2 pi f in [-pi, pi].
// Every mbarrier wait is bounded (2 s of %globaltimer); on timeout the CTA sets
// SAND_FLAG_TIMEOUT, stops issuing work, drains its copies and MMAs, frees TMEM
// and returns.
#pragma once

#include <cuda.h>

#include "internal.cuh"

namespace sand {

enum TcMode { TC_SPLIT16 = 0, TC_F16 = 1, TC_BF16 = 2 };

constexpr int kTcThreads = 320;
constexpr int kTileM = 128;
constexpr int kEpiThreads = 256;
constexpr uint64_t kTimeoutNs = 2000000000ull;
constexpr int kSmemBudget = 227 * 1024;
constexpr int kMaxStages = 8;
constexpr int kNumBars = 2 * kMaxStages + 8;  // full, empty, a_ready[2], d_full[2], a0_free, drain, x_full, x_empty
// bytes after the operand tiles and constants: barriers, TMEM slot + abort flag, tail exchange
constexpr int kMiscBytes = kNumBars * 8 + 16 + 1024;

struct TcParams {
    int L, W, D, tail_kind, act, enc, m;
    int first_mma;            // 1-based index of the first layer computed on the tensor cores
    int kpad;                 // padded K of the packed weight matrix (multiple of 64)
    int n_stages;
    uint32_t stage_bytes;     // (W / 2) * 128
    uint32_t a_part_bytes;    // 128 * kpad * 2
    uint32_t tmem_cols;
    float c1[kMaxLayers];     // per layer: w0 / (2 pi s) (sine) or 1 / s (ReLU)
    const float *cvec;        // [L][3][W]: bias' (w0 b / 2 pi for sine, b for ReLU), tail a, tail b
    const float *w1p;         // [3][W] first-layer weights (times w0 / 2 pi for sine), transposed
    const float *B;           // [m][3] Fourier matrix
    const float *tb;          // [L][2] tail biases
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
// Bounded wait: false after 2 s, or (when follow_abort) once another thread of the
// CTA has aborted.  The epilogue warps do not follow the flag: every waiter on a
// phase then agrees on whether it completed, so none is left alone at a named barrier.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort, WsHeader *hdr,
                                          uint32_t site, bool follow_abort) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    while (true) {
        if (mbar_try(bar, parity)) return true;
        if (follow_abort && *abort) return false;
        if (globaltimer() - t0 > kTimeoutNs) {
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
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void named_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }

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
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ int tc_row_depth(const WsHeader *hdr, uint32_t r, int L) {
    int d = L;
    for (int k = L - 1; k >= 1; --k)
        if (hdr->bin_start[k] <= r) d = k;
    return d;
}

// sin(2 pi t) for a phase t in revolutions: exact reduction to [-1/2, 1/2], then the hardware sine.
__device__ __forceinline__ float sin_rev(float t) {
    const float f = t - rintf(t);
    return __sinf(f * 6.28318530717958647692f);
}

template <int ACT>
__device__ __forceinline__ float activate(float t) {
    if (ACT == SAND_ACT_RELU) return fmaxf(t, 0.f);
    return sin_rev(t);
}

template <int MODE>
__device__ __forceinline__ void pack8(const float *h, uint4 &hi, uint4 &lo) {
    uint32_t H[4], Lo[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (MODE == TC_BF16) {
            __nv_bfloat162 b = __floats2bfloat162_rn(h[2 * i], h[2 * i + 1]);
            H[i] = *reinterpret_cast<uint32_t *>(&b);
            Lo[i] = 0;
        } else {
            __half2 a = __floats2half2_rn(h[2 * i], h[2 * i + 1]);
            H[i] = *reinterpret_cast<uint32_t *>(&a);
            if (MODE == TC_SPLIT16) {
                const float2 back = __half22float2(a);
                __half2 l = __floats2half2_rn(h[2 * i] - back.x, h[2 * i + 1] - back.y);
                Lo[i] = *reinterpret_cast<uint32_t *>(&l);
            } else {
                Lo[i] = 0;
            }
        }
    }
    hi = make_uint4(H[0], H[1], H[2], H[3]);
    lo = make_uint4(Lo[0], Lo[1], Lo[2], Lo[3]);
}

// Store 8 consecutive activations (columns j .. j+7, j % 8 == 0) of row r into the swizzled A operand.
template <int MODE>
__device__ __forceinline__ void store_a8(uint8_t *a_base, uint32_t a_part_bytes, int r, int j, const float *h) {
    uint4 hi, lo;
    pack8<MODE>(h, hi, lo);
    const int kb = j >> 6, c = (j & 63) >> 3;
    const uint32_t off = (uint32_t)kb * 16384u + (uint32_t)r * 128u + (uint32_t)((c ^ (r & 7)) << 4);
    *reinterpret_cast<uint4 *>(a_base + off) = hi;
    if (MODE == TC_SPLIT16) *reinterpret_cast<uint4 *>(a_base + a_part_bytes + off) = lo;
}

// ------------------------------------------------------------------ the kernel
template <int MODE, int ACT, int TAIL>
__global__ void __launch_bounds__(kTcThreads, 1)
tmlp_tc_kernel(const __grid_constant__ CUtensorMap wmap, const TcParams P, const float *__restrict__ pts,
               const float4 *__restrict__ sorted, WsHeader *hdr, int64_t n, int full_depth, float *__restrict__ out) {
    constexpr int PARTS = MODE == TC_SPLIT16 ? 2 : 1;
    constexpr bool MULT = TAIL == SAND_TAIL_MULT;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int W = P.W, L = P.L;
    const int hw = W >> 1;
    uint8_t *a_base = smem;
    uint8_t *stage_base = smem + PARTS * P.a_part_bytes;
    float *c_l1 = reinterpret_cast<float *>(stage_base + (size_t)P.n_stages * P.stage_bytes);  // [5][W]: w1p x3, bias', a
    float *c_ring = c_l1 + 5 * W;                                                              // [2][3][W]
    uint64_t *bars = reinterpret_cast<uint64_t *>(c_ring + 6 * W);
    uint64_t *full_bar = bars;
    uint64_t *empty_bar = bars + kMaxStages;
    uint64_t *a_ready = bars + 2 * kMaxStages;  // [2]
    uint64_t *d_full = a_ready + 2;             // [2]
    uint64_t *a0_free = d_full + 2;
    uint64_t *drain = a0_free + 1;
    uint64_t *x_full = drain + 1;   // tail partials of the D1 warps written (128 arrivals)
    uint64_t *x_empty = x_full + 1; // ... and read by the D0 warps (128 arrivals)
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + kNumBars);
    volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);
    float *tailx = reinterpret_cast<float *>(tmem_slot + 4);  // [2 values][128 rows] from the D1 warps

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t n_rows = full_depth ? n : (int64_t)hdr->n_active;
    const int64_t n_tiles = (n_rows + kTileM - 1) / kTileM;
    auto tile_depth = [&](int64_t t) -> int { return full_depth ? L : tc_row_depth(hdr, (uint32_t)(t * kTileM), L); };

    if (threadIdx.x == 0) {
        for (int s = 0; s < P.n_stages; ++s) {
            mbar_init(smem_u32(&full_bar[s]), 1);
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        mbar_init(smem_u32(&a_ready[0]), 4);
        mbar_init(smem_u32(&a_ready[1]), 4);
        mbar_init(smem_u32(&d_full[0]), 1);
        mbar_init(smem_u32(&d_full[1]), 1);
        mbar_init(smem_u32(a0_free), 1);
        mbar_init(smem_u32(drain), 1);
        mbar_init(smem_u32(x_full), 128);
        mbar_init(smem_u32(x_empty), 128);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(P.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (warp >= 2 && P.first_mma == 2) {  // first-layer constants: w1p (3 rows), bias', tail a
        for (int i = threadIdx.x - 64; i < 5 * W; i += kEpiThreads) {
            const int row = i / W, j = i % W;
            c_l1[i] = row < 3 ? P.w1p[row * W + j] : P.cvec[(row - 3) * W + j];
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            uint32_t it = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
                const int Dt = tile_depth(t);
                for (int l = P.first_mma; l <= Dt && ok; ++l) {
                    const int kb_n = (l == 1 ? P.D : W) >> 6;
                    for (int h = 0; h < 2 && ok; ++h)
                        for (int kb = 0; kb < kb_n && ok; ++kb)
                            for (int p = 0; p < PARTS && ok; ++p, ++it) {
                                const uint32_t s = it % P.n_stages, ph = (it / P.n_stages) & 1;
                                ok = mbar_wait(smem_u32(&empty_bar[s]), ph ^ 1, abort, hdr, 1, true);
                                if (!ok) break;
                                mbar_arrive_tx(smem_u32(&full_bar[s]), P.stage_bytes);
                                tma_load_2d(smem_u32(stage_base + (size_t)s * P.stage_bytes), &wmap, smem_u32(&full_bar[s]),
                                            kb * 64, ((l - P.first_mma) * PARTS + p) * W + h * hw);
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
            const uint32_t idesc = (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(hw >> 3) << 17) |
                                   ((uint32_t)(kTileM >> 4) << 24);
            const uint32_t a_addr = smem_u32(a_base);
            uint32_t it = 0, pa0 = 0, pa1 = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
                const int Dt = tile_depth(t);
                for (int l = P.first_mma; l <= Dt && ok; ++l) {
                    const int K = l == 1 ? P.D : W;
                    const int kb_n = K >> 6;
                    const int g_half = K >> 5;  // first K-step (of 16) in the second half of A
                    const int kb_last_first_half = (g_half - 1) >> 2;
                    for (int h = 0; h < 2 && ok; ++h) {
                        const uint32_t d_addr = tmem + (uint32_t)(h * hw);
                        for (int kb = 0; kb < kb_n && ok; ++kb) {
                            for (int p = 0; p < PARTS && ok; ++p, ++it) {
                                const uint32_t s = it % P.n_stages, ph = (it / P.n_stages) & 1;
                                ok = mbar_wait(smem_u32(&full_bar[s]), ph, abort, hdr, 3, true);
                                if (!ok) break;
                                tc_fence_after();
                                const uint32_t b_addr = smem_u32(stage_base + (size_t)s * P.stage_bytes);
#pragma unroll
                                for (int ks = 0; ks < 4; ++ks) {
                                    const int g = kb * 4 + ks;
                                    if (h == 0 && p == 0 && (g == 0 || g == g_half)) {
                                        uint32_t &pr = g == 0 ? pa0 : pa1;
                                        ok = mbar_wait(smem_u32(&a_ready[g == 0 ? 0 : 1]), pr, abort, hdr, 2, true);
                                        pr ^= 1;
                                        if (!ok) break;
                                        tc_fence_after();
                                    }
                                    const uint64_t bd = smem_desc(b_addr + ks * 32);
                                    const uint32_t a_off = (uint32_t)kb * 16384u + ks * 32;
                                    const uint64_t ahi = smem_desc(a_addr + a_off);
                                    if (p == 0) {
                                        mma_f16(d_addr, ahi, bd, idesc, g != 0);
                                        if (PARTS == 2) mma_f16(d_addr, smem_desc(a_addr + P.a_part_bytes + a_off), bd, idesc, 1);
                                    } else {
                                        mma_f16(d_addr, ahi, bd, idesc, 1);
                                    }
                                }
                                mma_commit(smem_u32(&empty_bar[s]));
                                if (h == 1 && p == PARTS - 1 && kb == kb_last_first_half) mma_commit(smem_u32(a0_free));
                            }
                        }
                        if (ok) mma_commit(smem_u32(&d_full[h]));
                    }
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
    } else {
        // ------------------------------------------------ epilogue warps 2..9
        const int q = warp & 3;                 // TMEM lane quadrant
        const int grp = (warp - 2) >> 2;        // 0: units [0, W/2) (D0), 1: units [W/2, W) (D1)
        const int r = q * 32 + lane;            // tile row
        const int et = threadIdx.x - 64;        // 0..255
        const int j_begin = grp * hw;
        const uint32_t t_lane = tmem + ((uint32_t)(q * 32) << 16);
        const int gt = et & 127;                // thread index within the group
        uint32_t pd = 0, pf = 0;                // phases of d_full[grp] and (group 0) a0_free
        uint32_t px = 0;                        // phase of x_full (group 0) / x_empty (group 1)
        bool pending_free = false;              // group 0: an a0_free phase not yet waited for
        bool ok = true;
        // Tail exchange through two mbarriers (bounded waits, no cross-group named barrier):
        // the D1 warps publish their partial dot products, the D0 warps add them to their own.
        auto publish = [&](float sa, float sb) {
            ok = mbar_wait(smem_u32(x_empty), px ^ 1, abort, hdr, 6, false) && ok;
            px ^= 1;
            tailx[r] = sa;
            if (MULT) tailx[128 + r] = sb;
            mbar_arrive(smem_u32(x_full));
        };
        auto collect = [&](float &sa, float &sb) {
            ok = mbar_wait(smem_u32(x_full), px, abort, hdr, 7, false) && ok;
            px ^= 1;
            sa += tailx[r];
            if (MULT) sb += tailx[128 + r];
            mbar_arrive(smem_u32(x_empty));
        };
        auto group_sync = [&]() { named_sync(2 + grp, 128); };
        auto wait_a_free = [&]() {
            if (grp == 0 && pending_free) {
                ok = mbar_wait(smem_u32(a0_free), pf, abort, hdr, 5, false) && ok;
                pf ^= 1;
                pending_free = false;
            }
        };
        auto load_consts = [&](int l) {  // this group's columns of layer l's bias', tail a, tail b -> ring slot l & 1
            float *dst = c_ring + (l & 1) * 3 * W;
            const float *src = P.cvec + (size_t)(l - 1) * 3 * W;
            if (gt < hw) {
                const int j = j_begin + gt;
                dst[j] = __ldg(src + j);
                dst[W + j] = __ldg(src + W + j);
                dst[2 * W + j] = __ldg(src + 2 * W + j);
            }
        };
        for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
            const int Dt = tile_depth(t);
            const int64_t row = t * kTileM + r;
            int d = 0;
            int64_t idx = -1;
            float x0 = 0.f, x1 = 0.f, x2 = 0.f;
            if (row < n_rows) {
                if (full_depth) {
                    idx = row;
                    d = L;
                    x0 = pts[3 * row]; x1 = pts[3 * row + 1]; x2 = pts[3 * row + 2];
                } else {
                    const float4 v = sorted[row];
                    x0 = v.x; x1 = v.y; x2 = v.z;
                    idx = __float_as_int(v.w);
                    d = tc_row_depth(hdr, (uint32_t)row, L);
                }
            }
            float y = 0.f;
            if (Dt >= P.first_mma) load_consts(P.first_mma);
            // ---- layer 1 on the CUDA cores (or the Fourier features feeding an MMA layer 1)
            if (P.first_mma == 2) {
                float ta = 0.f;
                const bool write_a = Dt > 1;
                if (write_a) wait_a_free();
                for (int j0 = j_begin; j0 < j_begin + hw; j0 += 8) {
                    float h8[8];
                    const float4 w0a = *reinterpret_cast<const float4 *>(c_l1 + j0);
                    const float4 w0b = *reinterpret_cast<const float4 *>(c_l1 + j0 + 4);
                    const float4 w1a = *reinterpret_cast<const float4 *>(c_l1 + W + j0);
                    const float4 w1b = *reinterpret_cast<const float4 *>(c_l1 + W + j0 + 4);
                    const float4 w2a = *reinterpret_cast<const float4 *>(c_l1 + 2 * W + j0);
                    const float4 w2b = *reinterpret_cast<const float4 *>(c_l1 + 2 * W + j0 + 4);
                    const float4 ba = *reinterpret_cast<const float4 *>(c_l1 + 3 * W + j0);
                    const float4 bb = *reinterpret_cast<const float4 *>(c_l1 + 3 * W + j0 + 4);
                    const float4 aa = *reinterpret_cast<const float4 *>(c_l1 + 4 * W + j0);
                    const float4 ab4 = *reinterpret_cast<const float4 *>(c_l1 + 4 * W + j0 + 4);
                    const float w0v[8] = {w0a.x, w0a.y, w0a.z, w0a.w, w0b.x, w0b.y, w0b.z, w0b.w};
                    const float w1v[8] = {w1a.x, w1a.y, w1a.z, w1a.w, w1b.x, w1b.y, w1b.z, w1b.w};
                    const float w2v[8] = {w2a.x, w2a.y, w2a.z, w2a.w, w2b.x, w2b.y, w2b.z, w2b.w};
                    const float bv[8] = {ba.x, ba.y, ba.z, ba.w, bb.x, bb.y, bb.z, bb.w};
                    const float av[8] = {aa.x, aa.y, aa.z, aa.w, ab4.x, ab4.y, ab4.z, ab4.w};
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        float u = fmaf(w0v[i], x0, bv[i]);
                        u = fmaf(w1v[i], x1, u);
                        u = fmaf(w2v[i], x2, u);
                        const float hv = activate<ACT>(u);
                        h8[i] = hv;
                        ta = fmaf(av[i], hv, ta);
                    }
                    if (write_a) store_a8<MODE>(a_base, P.a_part_bytes, r, j0, h8);
                }
                if (write_a) {
                    fence_async_smem();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&a_ready[grp]));
                }
                if (grp == 1) {
                    publish(ta, 0.f);
                } else {
                    float sb = 0.f;
                    collect(ta, sb);
                    y = ta + __ldg(P.tb);
                    if (d == 1 && idx >= 0) out[idx] = y;
                }
                group_sync();  // this group's constants for the first tensor-core layer are visible
            } else {
                // Fourier features gamma(x) = [sin 2 pi s, cos 2 pi s] over this group's half of in_dim
                const int hd = P.D >> 1;
                wait_a_free();
                for (int k0 = grp * hd; k0 < grp * hd + hd; k0 += 8) {
                    float h8[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int k = k0 + i;
                        const int kk = k < P.m ? k : k - P.m;
                        const float ph = fourier_phase(P.B + 3 * kk, x0, x1, x2);
                        float sv, cv;
                        sincospif(2.0f * ph, &sv, &cv);
                        h8[i] = k < P.m ? sv : cv;
                    }
                    store_a8<MODE>(a_base, P.a_part_bytes, r, k0, h8);
                }
                fence_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&a_ready[grp]));
                group_sync();  // this group's constants for the first tensor-core layer are visible
            }
            // ---- tensor-core layers
            for (int l = P.first_mma; l <= Dt; ++l) {
                ok = mbar_wait(smem_u32(&d_full[grp]), pd, abort, hdr, 4, false);
                pd ^= 1;
                if (!ok) break;
                tc_fence_after();
                if (grp == 0) pending_free = true;  // this layer's MMAs will release the first K-half of A
                const bool last = l == Dt;
                if (!last) load_consts(l + 1);
                const float *cs = c_ring + (l & 1) * 3 * W;
                const float c1 = P.c1[l - 1];
                float sa = 0.f, sb = 0.f;
                for (int c0 = j_begin; c0 < j_begin + hw; c0 += 32) {
                    float v[32];
                    tmem_ld32(t_lane + (uint32_t)c0, v);
                    if (!last && c0 == j_begin) wait_a_free();
#pragma unroll
                    for (int g = 0; g < 4; ++g) {
                        const int j0 = c0 + 8 * g;
                        const float4 ba = *reinterpret_cast<const float4 *>(cs + j0);
                        const float4 bb = *reinterpret_cast<const float4 *>(cs + j0 + 4);
                        const float4 aa = *reinterpret_cast<const float4 *>(cs + W + j0);
                        const float4 ab4 = *reinterpret_cast<const float4 *>(cs + W + j0 + 4);
                        const float bv[8] = {ba.x, ba.y, ba.z, ba.w, bb.x, bb.y, bb.z, bb.w};
                        const float av[8] = {aa.x, aa.y, aa.z, aa.w, ab4.x, ab4.y, ab4.z, ab4.w};
                        float tbv[8];
                        if (MULT) {
                            const float4 ta4 = *reinterpret_cast<const float4 *>(cs + 2 * W + j0);
                            const float4 tb4 = *reinterpret_cast<const float4 *>(cs + 2 * W + j0 + 4);
                            tbv[0] = ta4.x; tbv[1] = ta4.y; tbv[2] = ta4.z; tbv[3] = ta4.w;
                            tbv[4] = tb4.x; tbv[5] = tb4.y; tbv[6] = tb4.z; tbv[7] = tb4.w;
                        }
                        float h8[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const float hv = activate<ACT>(fmaf(v[8 * g + i], c1, bv[i]));
                            h8[i] = hv;
                            sa = fmaf(av[i], hv, sa);
                            if (MULT) sb = fmaf(tbv[i], hv, sb);
                        }
                        if (!last) store_a8<MODE>(a_base, P.a_part_bytes, r, j0, h8);
                    }
                }
                tc_fence_before();
                if (!last) {
                    fence_async_smem();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&a_ready[grp]));
                }
                if (grp == 1) {
                    publish(sa, sb);
                } else {
                    collect(sa, sb);
                    const float t0v = sa + __ldg(P.tb + 2 * (l - 1));
                    float tl = t0v;
                    if (MULT && l >= 2) tl = t0v * (sb + __ldg(P.tb + 2 * (l - 1) + 1));
                    y += tl;
                    if (d == l && idx >= 0) out[idx] = y;
                }
                group_sync();  // next layer's constants of this group are visible; this layer's slot is free
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(P.tmem_cols) : "memory");
    }
}

// Launch one instantiation (defined in the per-mode translation units).
template <int MODE>
cudaError_t launch_tc_mode(const CUtensorMap &map, const TcParams &P, int act, int tail, const float *pts,
                           const float4 *sorted, WsHeader *hdr, int64_t n, int full_depth, float *out, int grid,
                           size_t smem, cudaStream_t s);

size_t tc_smem_bytes(const TcParams &P, int parts);

}  // namespace sand
