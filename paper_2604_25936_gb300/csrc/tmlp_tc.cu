// Tensor-core T-MLP kernel for sm_103a (tcgen05 MMA, TMEM accumulators, TMA).
//
// Evaluates Eq. 2 (and Eq. 3 for multiplicative tails) for 128-row tiles of
// points sorted by descending exit layer.  Per CTA (persistent, one per SM):
//   warp 0      TMA producer: streams the packed weight tiles of every hidden
//               layer (K-blocks of 64, one per stage) from L2 into a ring of
//               shared-memory stages (128-byte swizzle, the UMMA K-major layout).
//   warp 1      allocates the TMEM accumulator and issues tcgen05.mma from one
//               thread: D[128 x W] (fp32, TMEM) = A[128 x K] . B[W x K]^T.
//   warps 2..9  epilogue: layer 1 (x -> h_1 on the CUDA cores, float32), then for
//               each hidden layer the TMEM -> register load, bias, omega0, sine
//               with exact Cody-Waite reduction, the tails and the running sum
//               y_l = y_{l-1} + t_l, writing y at each row's exit layer; the new
//               activations go back to shared memory as the next A operand.
//               Thread (quadrant q, lane i) owns tile row 32q + i (TMEM lane
//               restriction); warps 2-5 take the first half of the units, 6-9 the second.
// A tile runs to the exit layer of its first (deepest) row; rows whose exit
// layer was reached keep riding in the tile until it ends (this only happens in
// the one tile per exit layer that straddles two layers), and tiles of exit
// layer 1 never touch the tensor cores.
//
// Precision modes (hidden-layer products only; everything else is float32):
//   SPLIT16  a = a_hi + a_lo and w*s = w_hi + w_lo with fp16 terms (s = 2^-e
//            per layer, so max|w s| is in [0.5, 1)), D = A_hi B_hi + A_lo B_hi
//            + A_hi B_lo accumulated in fp32: float32-class products.
//   F16/BF16 one product with fp16 (scaled) / bf16 operands.
// Every mbarrier wait is bounded (2 s of globaltimer); on timeout the CTA sets
// SAND_FLAG_TIMEOUT in the workspace header, stops issuing work, drains its
// outstanding copies, frees TMEM and exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <string.h>

#include <cmath>
#include <vector>

#include "tc.cuh"

namespace sand {

enum TcMode { TC_SPLIT16 = 0, TC_F16 = 1, TC_BF16 = 2 };

constexpr int kTcThreads = 320;
constexpr int kTileM = 128;
constexpr int kEpiThreads = 256;
constexpr uint64_t kTimeoutNs = 2000000000ull;
constexpr int kSmemBudget = 227 * 1024;
constexpr int kMaxStages = 8;
// bytes after the operand tiles: barriers (2 * kMaxStages + 4) * 8, TMEM slot and abort flag 16, tail exchange 1024
constexpr int kMiscBytes = (2 * kMaxStages + 4) * 8 + 16 + 1024;

struct TcParams {
    int L, W, D, tail_kind, act, enc, m;
    float omega0;
    int first_mma;           // 1-based index of the first layer computed on the tensor cores
    int kpad;                // padded K of the packed weight matrix (multiple of 64)
    int n_stages;
    uint32_t stage_bytes;    // W * 128
    uint32_t a_part_bytes;   // 128 * kpad * 2
    uint32_t tmem_cols;
    float inv_s[kMaxLayers];       // 1 / s_l for layer l (index l - 1)
    const float *bias[kMaxLayers]; // b_l (index l - 1)
    const float *W1T;              // [3][W] first-layer weights, transposed
    const float *B;                // [m][3] Fourier matrix
    const float *tw;               // [L][2][W]
    const float *tb;               // [L][2]
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
                                          uint32_t site, bool follow_abort = true) {
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
template <int MODE>
__global__ void __launch_bounds__(kTcThreads, 1)
tmlp_tc_kernel(const __grid_constant__ CUtensorMap wmap, const TcParams P, const float *__restrict__ pts,
               const float4 *__restrict__ sorted, WsHeader *hdr, int64_t n, int full_depth, float *__restrict__ out) {
    constexpr int PARTS = MODE == TC_SPLIT16 ? 2 : 1;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *a_base = smem;
    uint8_t *stage_base = smem + PARTS * P.a_part_bytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(stage_base + (size_t)P.n_stages * P.stage_bytes);
    uint64_t *full_bar = bars;
    uint64_t *empty_bar = bars + P.n_stages;
    uint64_t *a_full = bars + 2 * P.n_stages;
    uint64_t *d_full = a_full + 1;
    uint64_t *drain = a_full + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * kMaxStages + 4);
    volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);
    float *tailx = reinterpret_cast<float *>(tmem_slot + 4);  // [2 values][128 rows] from the second-half threads

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int L = P.L, W = P.W;
    const int64_t n_rows = full_depth ? n : (int64_t)hdr->n_active;
    const int64_t n_tiles = (n_rows + kTileM - 1) / kTileM;
    auto tile_depth = [&](int64_t t) -> int { return full_depth ? L : tc_row_depth(hdr, (uint32_t)(t * kTileM), L); };

    if (threadIdx.x == 0) {
        for (int s = 0; s < P.n_stages; ++s) {
            mbar_init(smem_u32(&full_bar[s]), 1);
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        mbar_init(smem_u32(a_full), kEpiThreads / 32);
        mbar_init(smem_u32(d_full), 1);
        mbar_init(smem_u32(drain), 1);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(P.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
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
                    for (int kb = 0; kb < kb_n && ok; ++kb)
                        for (int p = 0; p < PARTS && ok; ++p, ++it) {
                            const uint32_t s = it % P.n_stages, ph = (it / P.n_stages) & 1;
                            ok = mbar_wait(smem_u32(&empty_bar[s]), ph ^ 1, abort, hdr, 1);
                            if (!ok) break;
                            mbar_arrive_tx(smem_u32(&full_bar[s]), P.stage_bytes);
                            tma_load_2d(smem_u32(stage_base + (size_t)s * P.stage_bytes), &wmap, smem_u32(&full_bar[s]),
                                        kb * 64, ((l - P.first_mma) * PARTS + p) * W);
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
            const uint32_t idesc = (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(W >> 3) << 17) | ((uint32_t)(kTileM >> 4) << 24);
            const uint32_t a_addr = smem_u32(a_base);
            uint32_t it = 0, pa = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
                const int Dt = tile_depth(t);
                for (int l = P.first_mma; l <= Dt && ok; ++l) {
                    ok = mbar_wait(smem_u32(a_full), pa, abort, hdr, 2);
                    pa ^= 1;
                    if (!ok) break;
                    tc_fence_after();
                    const int kb_n = (l == 1 ? P.D : W) >> 6;
                    for (int kb = 0; kb < kb_n && ok; ++kb)
                        for (int p = 0; p < PARTS && ok; ++p, ++it) {
                            const uint32_t s = it % P.n_stages, ph = (it / P.n_stages) & 1;
                            ok = mbar_wait(smem_u32(&full_bar[s]), ph, abort, hdr, 3);
                            if (!ok) break;
                            tc_fence_after();
                            const uint32_t b_addr = smem_u32(stage_base + (size_t)s * P.stage_bytes);
#pragma unroll
                            for (int ks = 0; ks < 4; ++ks) {
                                const uint64_t bd = smem_desc(b_addr + ks * 32);
                                const uint32_t a_off = (uint32_t)kb * 16384u + ks * 32;
                                const uint64_t ahi = smem_desc(a_addr + a_off);
                                if (p == 0) {
                                    mma_f16(tmem, ahi, bd, idesc, (kb | ks) != 0);
                                    if (PARTS == 2) mma_f16(tmem, smem_desc(a_addr + P.a_part_bytes + a_off), bd, idesc, 1);
                                } else {
                                    mma_f16(tmem, ahi, bd, idesc, 1);
                                }
                            }
                            mma_commit(smem_u32(&empty_bar[s]));
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
    } else {
        // ------------------------------------------------ epilogue warps 2..9
        const int q = warp & 3;                 // TMEM lane quadrant
        const int half = (warp - 2) >> 2;       // which half of the units
        const int r = q * 32 + lane;            // tile row
        const int hw = W >> 1;
        const int j_begin = half * hw;
        const uint32_t t_lane = tmem + ((uint32_t)(q * 32) << 16);
        const bool mult = P.tail_kind == SAND_TAIL_MULT;
        const float w0 = P.omega0;
        uint32_t pd = 0;
        bool ok = true;
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
            // ---- layer 1 on the CUDA cores (or the Fourier features feeding an MMA layer 1)
            if (P.first_mma == 2) {
                const float *a1 = P.tw;
                const float *bb1 = P.bias[0];
                float ta = 0.f;
                for (int j0 = j_begin; j0 < j_begin + hw; j0 += 8) {
                    float h8[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int j = j0 + i;
                        float acc = __ldg(P.W1T + j) * x0;
                        acc = fmaf(__ldg(P.W1T + W + j), x1, acc);
                        acc = fmaf(__ldg(P.W1T + 2 * W + j), x2, acc);
                        const float u = acc + __ldg(bb1 + j);
                        const float hv = P.act == SAND_ACT_RELU ? fmaxf(u, 0.f) : sin_reduced(w0 * u);
                        h8[i] = hv;
                        ta = fmaf(__ldg(a1 + j), hv, ta);
                    }
                    if (Dt > 1) store_a8<MODE>(a_base, P.a_part_bytes, r, j0, h8);
                }
                if (Dt > 1) {
                    fence_async_smem();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(a_full));
                }
                if (half == 1) tailx[r] = ta;
                named_sync(1, kEpiThreads);
                if (half == 0) {
                    y = ta + tailx[r] + __ldg(P.tb);
                    if (d == 1 && idx >= 0) out[idx] = y;
                }
                named_sync(1, kEpiThreads);
            } else {
                // Fourier features gamma(x) = [sin 2 pi s, cos 2 pi s] over this thread's half of in_dim
                const int hd = P.D >> 1;
                for (int k0 = half * hd; k0 < half * hd + hd; k0 += 8) {
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
                if (lane == 0) mbar_arrive(smem_u32(a_full));
            }
            // ---- tensor-core layers
            for (int l = P.first_mma; l <= Dt; ++l) {
                ok = mbar_wait(smem_u32(d_full), pd, abort, hdr, 4, false);
                pd ^= 1;
                if (!ok) break;
                tc_fence_after();
                const float *bl = P.bias[l - 1];
                const float *ta_w = P.tw + (size_t)(l - 1) * 2 * W;
                const float *tb_w = ta_w + W;
                const float inv_s = P.inv_s[l - 1];
                const bool last = l == Dt;
                const bool lm = mult && l >= 2;
                float sa = 0.f, sb = 0.f;
                for (int c0 = j_begin; c0 < j_begin + hw; c0 += 32) {
                    float v[32];
                    tmem_ld32(t_lane + (uint32_t)c0, v);
#pragma unroll
                    for (int g = 0; g < 4; ++g) {
                        float h8[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int j = c0 + 8 * g + i;
                            const float u = fmaf(v[8 * g + i], inv_s, __ldg(bl + j));
                            const float hv = P.act == SAND_ACT_RELU ? fmaxf(u, 0.f) : sin_reduced(w0 * u);
                            h8[i] = hv;
                            sa = fmaf(__ldg(ta_w + j), hv, sa);
                            if (lm) sb = fmaf(__ldg(tb_w + j), hv, sb);
                        }
                        if (!last) store_a8<MODE>(a_base, P.a_part_bytes, r, c0 + 8 * g, h8);
                    }
                }
                tc_fence_before();
                if (!last) {
                    fence_async_smem();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(a_full));
                }
                if (half == 1) {
                    tailx[r] = sa;
                    tailx[128 + r] = sb;
                }
                named_sync(1, kEpiThreads);
                if (half == 0) {
                    const float c_a = __ldg(P.tb + 2 * (l - 1)), c_b = __ldg(P.tb + 2 * (l - 1) + 1);
                    const float t0v = sa + tailx[r] + c_a;
                    const float tl = lm ? t0v * (sb + tailx[128 + r] + c_b) : t0v;
                    y += tl;
                    if (d == l && idx >= 0) out[idx] = y;
                }
                named_sync(1, kEpiThreads);
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

// ------------------------------------------------------------------ host side
static int mode_of(int precision) {
    switch (precision) {
        case SAND_FP32: return TC_SPLIT16;
        case SAND_FP16: return TC_F16;
        case SAND_BF16: return TC_BF16;
        default: return -1;
    }
}

bool tc_supported(const sand_tmlp_desc &d, int precision) {
    if (mode_of(precision) < 0) return false;
    if (d.width != 64 && d.width != 128 && d.width != 256) return false;
    if (d.encoder == SAND_ENC_FOURIER && (d.in_dim % 64 != 0 || d.in_dim > 256)) return false;
    return d.n_layers >= 1;
}

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

struct TcPack {
    CUtensorMap map;
    TcParams P;
    int mode;
};

sand_status tc_prepare(TcModel *tc, const sand_tmlp_desc &d, const float *params, int precision) {
    const int mode = mode_of(precision);
    if (mode < 0 || !tc_supported(d, precision)) {
        set_error("precision %d not supported on the tensor-core path for this model", precision);
        return SAND_EUNSUPPORTED;
    }
    if (tc->packed_precision == precision && tc->d_pack) return SAND_OK;
    tc_release(tc);
    const int L = d.n_layers, W = d.width, D = d.in_dim, mf = d.n_freq;
    const int first = d.encoder == SAND_ENC_FOURIER ? 1 : 2;
    const int parts = mode == TC_SPLIT16 ? 2 : 1;
    const int kpad = (first == 1 && D > W) ? D : W;
    const int n_mma = L - first + 1;  // may be 0 for a one-layer SIREN
    const float *p = params;
    if (d.encoder == SAND_ENC_FOURIER) p += (size_t)mf * 3;
    const float *W1 = p; p += (size_t)W * D;
    p += W;
    const float *Wh = p;
    const size_t rows = (size_t)(n_mma > 0 ? n_mma : 1) * parts * W;
    std::vector<uint16_t> packed(rows * kpad, 0);
    std::vector<float> inv_s(kMaxLayers, 1.f);
    for (int li = 0; li < n_mma; ++li) {
        const int l = first + li;  // 1-based layer
        const int K = l == 1 ? D : W;
        const float *Wl = l == 1 ? W1 : Wh + (size_t)(l - 2) * W * W;
        float amax = 0.f;
        for (size_t i = 0; i < (size_t)W * K; ++i) amax = fmaxf(amax, fabsf(Wl[i]));
        float s = 1.f;
        if (mode != TC_BF16 && amax > 0.f) {
            int e;
            frexpf(amax, &e);          // amax = f * 2^e, f in [0.5, 1)
            s = ldexpf(1.f, -e);       // amax * s in [0.5, 1)
        }
        inv_s[l - 1] = 1.f / s;
        for (int nrow = 0; nrow < W; ++nrow)
            for (int k = 0; k < K; ++k) {
                const float w = Wl[(size_t)nrow * K + k] * s;
                uint16_t hi, lo = 0;
                if (mode == TC_BF16) {
                    __nv_bfloat16 b = __float2bfloat16_rn(w);
                    memcpy(&hi, &b, 2);
                } else {
                    __half h = __float2half_rn(w);
                    memcpy(&hi, &h, 2);
                    if (mode == TC_SPLIT16) {
                        __half l2 = __float2half_rn(w - __half2float(h));
                        memcpy(&lo, &l2, 2);
                    }
                }
                packed[((size_t)(li * parts + 0) * W + nrow) * kpad + k] = hi;
                if (parts == 2) packed[((size_t)(li * parts + 1) * W + nrow) * kpad + k] = lo;
            }
    }
    auto *pk = new TcPack();
    memset(pk, 0, sizeof(TcPack));
    void *dbuf = nullptr;
    if (cudaMalloc(&dbuf, packed.size() * 2) != cudaSuccess) {
        cudaGetLastError();
        delete pk;
        set_error("cannot allocate packed weights");
        return SAND_ENOMEM;
    }
    if (cudaMemcpy(dbuf, packed.data(), packed.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(dbuf);
        delete pk;
        set_error("cannot upload packed weights");
        return SAND_ECUDA;
    }
    auto enc = encode_fn();
    if (!enc) {
        cudaFree(dbuf);
        delete pk;
        set_error("cuTensorMapEncodeTiled unavailable");
        return SAND_EUNSUPPORTED;
    }
    cuuint64_t gdim[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
    cuuint64_t gstride[1] = {(cuuint64_t)kpad * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)W};
    cuuint32_t estride[2] = {1, 1};
    CUresult cr = enc(&pk->map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, dbuf, gdim, gstride, box, estride,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) {
        cudaFree(dbuf);
        delete pk;
        set_error("cuTensorMapEncodeTiled failed (%d)", (int)cr);
        return SAND_ECUDA;
    }
    TcParams &P = pk->P;
    P.L = L; P.W = W; P.D = D; P.tail_kind = d.tail_kind; P.act = d.activation; P.enc = d.encoder; P.m = mf;
    P.omega0 = d.omega0;
    P.first_mma = first;
    P.kpad = kpad;
    P.stage_bytes = (uint32_t)W * 128u;
    P.a_part_bytes = (uint32_t)kTileM * kpad * 2u;
    P.tmem_cols = W <= 32 ? 32 : (W <= 64 ? 64 : (W <= 128 ? 128 : 256));
    const int fixed = 1024 /*alignment slack*/ + parts * (int)P.a_part_bytes + kMiscBytes;
    int stages = (kSmemBudget - fixed) / (int)P.stage_bytes;
    if (stages > kMaxStages) stages = kMaxStages;
    if (stages < 2) {
        cudaFree(dbuf);
        delete pk;
        set_error("shared memory too small for this width");
        return SAND_EUNSUPPORTED;
    }
    P.n_stages = stages;
    for (int l = 0; l < kMaxLayers; ++l) P.inv_s[l] = inv_s[l];
    pk->mode = mode;
    tc->d_pack = dbuf;
    tc->pack_bytes = packed.size() * 2;
    tc->host = pk;
    tc->packed_precision = precision;
    return SAND_OK;
}

static size_t tc_smem_bytes(const TcParams &P, int parts) {
    return 1024 + (size_t)parts * P.a_part_bytes + (size_t)P.n_stages * P.stage_bytes + kMiscBytes;
}

cudaError_t launch_tmlp_tc(const TcModel &tc, const TmlpDev &M, const float *pts, int64_t n, int full_depth, void *ws,
                           float *out, int num_sms, cudaStream_t s) {
    TcPack *pk = static_cast<TcPack *>(tc.host);
    if (!pk) return cudaErrorInvalidValue;
    TcParams P = pk->P;
    for (int l = 0; l < kMaxLayers; ++l) P.bias[l] = M.bias[l];
    P.W1T = M.WT[0];
    P.B = M.B;
    P.tw = M.tw;
    P.tb = M.tb;
    WsLayout Lw = ws_layout(full_depth ? 0 : n);
    char *base = static_cast<char *>(ws);
    WsHeader *hdr = reinterpret_cast<WsHeader *>(base);
    const float4 *sorted = full_depth ? nullptr : reinterpret_cast<const float4 *>(base + Lw.sorted);
    const int parts = pk->mode == TC_SPLIT16 ? 2 : 1;
    const size_t smem = tc_smem_bytes(P, parts);
    int64_t tiles = (n + kTileM - 1) / kTileM;
    int grid = num_sms;
    if (tiles < grid) grid = (int)(tiles > 0 ? tiles : 1);
    cudaError_t e;
    switch (pk->mode) {
        case TC_SPLIT16:
            e = cudaFuncSetAttribute(tmlp_tc_kernel<TC_SPLIT16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            tmlp_tc_kernel<TC_SPLIT16><<<grid, kTcThreads, smem, s>>>(pk->map, P, pts, sorted, hdr, n, full_depth, out);
            break;
        case TC_F16:
            e = cudaFuncSetAttribute(tmlp_tc_kernel<TC_F16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            tmlp_tc_kernel<TC_F16><<<grid, kTcThreads, smem, s>>>(pk->map, P, pts, sorted, hdr, n, full_depth, out);
            break;
        default:
            e = cudaFuncSetAttribute(tmlp_tc_kernel<TC_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            tmlp_tc_kernel<TC_BF16><<<grid, kTcThreads, smem, s>>>(pk->map, P, pts, sorted, hdr, n, full_depth, out);
            break;
    }
    return cudaGetLastError();
}

void tc_release(TcModel *tc) {
    if (!tc) return;
    if (tc->d_pack) cudaFree(tc->d_pack);
    delete static_cast<TcPack *>(tc->host);
    tc->d_pack = nullptr;
    tc->host = nullptr;
    tc->packed_precision = -1;
}

}  // namespace sand
