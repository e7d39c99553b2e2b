// T-MLP training steps (Sec. 3.3): the loss over every tail (Eq. 4) with the L1 SDF loss
// (Eq. 8), its gradient for every parameter, and Adam (Sec. 4.1).
//
// Layout of a step for a batch of n points (rows padded to B = a multiple of 128 with zero
// points whose gradient contributions are zero), width W, L layers; z_l = W_l h_{l-1} + b_l is
// the pre-activation of layer l, h_l = act(z_l), y_l = y_{l-1} + t_l:
//   tr_amax, tr_pack   per layer l >= 2: a power-of-two scale s_l (max|W_l s_l| in [0.5, 1)) and
//                      W_l s_l split into fp16 hi + lo, as rows [out][in] (forward) and [in][out]
//                      (backward), the K-major layout the MMA reads;
//   tr_fwd1            layer 1 (fan-in 3) on the CUDA cores: z_1, tail 1, y_1;
//   tr_gemm<FWD>       l = 2..L: Z = act(Z_{l-1}) (W_l s_l)^T / s_l + b_l on the tensor cores; the
//                      epilogue stores z_l and the row's tail factors and y_l;
//   tr_loss            per row: G'_k = sum_{i>=k} sign(y_i - y_gt) (an integer; dL/dt_k = G'_k / n)
//                      and |y_i - y_gt| summed per block;
//   tr_top             delta'_L = G'_L dt_L/dh_L * act'(z_L)   (delta' = n dL/dz);
//   tr_tsplit          act(z_l)^T (l = 1..L-1) and each delta'_l^T, transposed and split into
//                      fp16 hi + lo: the weight gradient's operands, K (the batch) contiguous;
//   tr_gemm<BWD>       l = L..2: delta'_{l-1} = (delta'_l W_l + G'_{l-1} dt_{l-1}/dh_{l-1}) * act'(z_{l-1});
//   tr_gemm<DW>        l = 2..L: partial sums over row ranges of delta'_l^T act(Z_{l-1}), split over
//                      the CTAs along the rows (the reduction dimension);
//   tr_colsum          per layer and row range: the column sums for b_l, the tail weights and
//                      biases, and W_1 (sum of delta'_1 x^T);
//   tr_finalize        adds the partials in a fixed order and divides by n: the gradient in the
//                      parameter-block order;
//   tr_adam            one Adam update of the float32 master parameters.
// Every value stays float32 in memory; activations are recomputed from the stored z where an
// operand needs them.  Each product is D = A_hi B_hi + A_lo B_hi + A_hi B_lo (a = hi + lo, fp16
// each) by tcgen05.mma (kind::f16, M = 128, N = W, fp32 accumulator in TMEM) from shared memory
// in the 128-byte swizzled K-major layout.  The forward and backward A operands are split on the
// fly by the GEMM's producer warps; the packed weights and the weight gradient's operands are
// split beforehand and arrive by TMA.  The epilogue sends each 32 x 32 block of its output out
// by a TMA store from a shared-memory staging tile.  delta' = n dL/dz keeps the backward operands away
// from the fp16 subnormals; 1/n is applied once, at the end.
#include <math.h>
#include <string.h>

#include <utility>
#include <vector>

#include "internal.cuh"
#include "tc.cuh"
#include "tc_kernel.cuh"

namespace sand {

enum TrEpi { TR_FWD = 0, TR_BWD = 1, TR_DW = 2 };

constexpr int kTrProdWarps = 4;           // warps 0..3 produce operands
constexpr int kTrProducers = 32 * kTrProdWarps;
constexpr int kTrMmaWarp = 4;             // TMEM owner and MMA issuer
constexpr int kTrThreads = 32 * 9;        // warps 5..8: epilogue
constexpr int kTrBM = 128;                 // rows of a tile (MMA M)
constexpr int kTrMaxStages = 4;
constexpr int kTrSmem = 227 * 1024;
constexpr int kTrStoreTile = 32 * 32 * 4;  // an epilogue warp's staging tile: 32 rows x 32 float32 (SW128)

struct TrGemm {
    int M, N, K;          // output rows (bounds), columns (= MMA N), reduction length
    int m_tiles, splits;  // tiles: m_tiles row tiles x splits of the K range
    int kb_per_split;     // 64-element K-blocks per split
    int act;
    float omega0;
    // A operand: FWD act(a[row][k]); BWD a[row][k]   (ld = a_ld); DW: rows a_row0 + m (hi) and
    // a_row0 + W + m (lo) of the kernel's A tensor map (delta'^T split into fp16, k contiguous)
    const float *a;
    int a_ld;
    int a_row0;
    // B operand by TMA through the kernel's B tensor map, rows b_row0 + n (hi) and b_row0 + N + n
    // (lo): FWD / BWD the packed weights; DW act(z)^T split into fp16 (k contiguous)
    int b_row0;
    int box_rows;  // DW: rows per TMA box of either map (min(128, W))
    int n_stages;
    uint32_t stage_bytes;
    // epilogue
    float *out;               // FWD: z_l [B][W]; BWD: delta'_{l-1} [B][W]; DW: partials [split][M][N]
    int out_row0;             // row of the kernel's output tensor map holding row 0 of out
    const float *inv_s;       // device: 1 / s_l
    const float *bias;        // FWD: b_l
    const float *tw;          // FWD: tail weights of l (a at tw, b at tw + N); BWD: of l - 1
    const float *tbias;       // FWD: tail biases of l (c, e)
    int mult;                 // FWD: tail l multiplicative; BWD: tail l - 1 multiplicative
    const float *y_prev;      // FWD: y_{l-1} per row
    float *y_out, *ta_out, *tb_out;  // FWD: y_l and the tail factors per row
    const float *z_prev;      // BWD: z_{l-1} [B][W]
    const float *g_prev;      // BWD: G'_{l-1} per row
    const float *ta_prev, *tb_prev;  // BWD: tail factors of layer l - 1 per row
    unsigned *status;         // bit 0: a bounded wait gave up
};

__device__ __forceinline__ float tr_act(int act, float z, float w0) {
    if (act == SAND_ACT_RELU) return fmaxf(z, 0.f);
    if (act == SAND_ACT_FINER) return __sinf(w0 * (fabsf(z) + 1.f) * z);
    return __sinf(w0 * z);
}
__device__ __forceinline__ float tr_slope(int act, float z, float w0) {
    if (act == SAND_ACT_RELU) return z > 0.f ? 1.f : 0.f;
    if (act == SAND_ACT_FINER) return w0 * fmaf(2.f, fabsf(z), 1.f) * __cosf(w0 * (fabsf(z) + 1.f) * z);
    return w0 * __cosf(w0 * z);
}

// Split 8 floats into fp16 hi and lo parts (lo = fp16(v - hi), v - hi exact in float32), packed pairs.
__device__ __forceinline__ void tr_split8(const float *v, uint4 &hi, uint4 &lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const __half2 hp = __floats2half2_rn(v[2 * i], v[2 * i + 1]);
        const float2 hf = __half22float2(hp);
        const __half2 lp = __floats2half2_rn(v[2 * i] - hf.x, v[2 * i + 1] - hf.y);
        h[i] = *reinterpret_cast<const uint32_t *>(&hp);
        l[i] = *reinterpret_cast<const uint32_t *>(&lp);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// Byte offset of 16-byte chunk c (K elements 8c .. 8c+7) of row r in a K-major tile of 128-byte
// rows with the 128-byte swizzle (the layout of tcgen05 shared-memory descriptors, layout type
// SWIZZLE_128B; the tile starts 1024-byte aligned).
__device__ __forceinline__ uint32_t tr_swz(int r, int c) { return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)); }

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint4 v) {
    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                 : "memory");
}

// Tensor-map store of a shared-memory tile (bulk-group completion), and the waits on it.
__device__ __forceinline__ void tr_tma_store_2d(const CUtensorMap *map, uint32_t src, int x, int y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(src), "r"(x), "r"(y)
                 : "memory");
}
__device__ __forceinline__ void tr_bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the source of every committed store has been read (the staging tile may be rewritten)
__device__ __forceinline__ void tr_bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// every committed store has completed
__device__ __forceinline__ void tr_bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Warp-uniform bounded wait: lane 0 waits, the result is broadcast (the callers go on to
// warp-collective instructions, which every lane must reach together).
__device__ __forceinline__ bool tr_wait_warp(uint32_t bar, uint32_t parity, volatile int *abort, unsigned *status) {
    int ok = 1;
    if ((threadIdx.x & 31) == 0) {
        if (!mbar_try(bar, parity)) {
            const uint64_t t0 = globaltimer();
            while (true) {
                if (mbar_try(bar, parity)) break;
                if (*abort) { ok = 0; break; }
                if (globaltimer() - t0 > kTimeoutNs) {
                    *abort = 1;
                    atomicOr(status, 1u);
                    ok = 0;
                    break;
                }
            }
        }
    }
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// The A tile of one FWD / BWD stage (64 K-elements of 128 rows) from global memory into shared
// memory, split into fp16 hi and lo parts, by the kTrProducers producer threads (the packed
// weights come by TMA).
// Every global load of a group is issued before any of its values is used, so a stage costs a
// few memory latencies rather than one per chunk.
template <int EPI>
__device__ __forceinline__ void tr_produce_stage(const TrGemm &P, int pt, int m0, int k0, uint32_t ahi, uint32_t alo,
                                                 uint32_t bhi, uint32_t blo) {
    (void)bhi;
    (void)blo;
    {
        // A[r][kk] = (act of) a[m0 + r][k0 + kk]: chunk it = (row it / 8, 8 K-elements it % 8), 32
        // contiguous bytes; eight consecutive threads read one row's 256 bytes
        constexpr int NA = kTrBM * 8 / kTrProducers;
        float4 va[NA][2];
#pragma unroll
        for (int j = 0; j < NA; ++j) {
            const int it = pt + j * kTrProducers;
            const int row = m0 + (it >> 3), kk = k0 + 8 * (it & 7);
            const bool in = row < P.M && kk + 8 <= P.K;
            const float4 *src = reinterpret_cast<const float4 *>(P.a + (size_t)row * P.a_ld + kk);
            va[j][0] = in ? __ldg(src) : make_float4(0.f, 0.f, 0.f, 0.f);
            va[j][1] = in ? __ldg(src + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int j = 0; j < NA; ++j) {
            const int it = pt + j * kTrProducers;
            float v[8] = {va[j][0].x, va[j][0].y, va[j][0].z, va[j][0].w, va[j][1].x, va[j][1].y, va[j][1].z, va[j][1].w};
            if (EPI == TR_FWD) {  // act(0) = 0 for every activation: padding stays 0
#pragma unroll
                for (int e = 0; e < 8; ++e) v[e] = tr_act(P.act, v[e], P.omega0);
            }
            uint4 hi, lo;
            tr_split8(v, hi, lo);
            st_shared_v4(ahi + tr_swz(it >> 3, it & 7), hi);
            st_shared_v4(alo + tr_swz(it >> 3, it & 7), lo);
        }
    }
}

// Persistent GEMM: CTA b takes tiles b, b + grid, ...; tile t is rows 128 (t % m_tiles) .. + 127
// and K-blocks of split t / m_tiles.  Two accumulators in TMEM let the epilogue of one tile run
// while the MMAs of the next one do.  The B operand of a stage (hi and lo) comes by TMA (bmap,
// 128-byte swizzle: the layout tr_swz writes) on its own barrier; DW's A operand too (amap), so
// its producer is one thread of warp 0 and its stages hold no generic-proxy writes.
//   warps 0..3  producers (operands into the shared-memory stage ring)
//   warp 4      TMEM owner, MMA issuer (one thread)
//   warps 5..8  epilogue: thread (quadrant warp & 3, lane i) owns tile row 32 (warp & 3) + i
template <int EPI>
__global__ void __launch_bounds__(kTrThreads, 1) tr_gemm_kernel(const __grid_constant__ CUtensorMap amap,
                                                                const __grid_constant__ CUtensorMap bmap,
                                                                const __grid_constant__ CUtensorMap omap, const TrGemm P) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    // after the stage ring (1024-byte aligned): the epilogue warps' output staging tiles
    uint8_t *stage_out = smem + (size_t)P.n_stages * P.stage_bytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(stage_out + 4 * kTrStoreTile);
    uint64_t *full = bars;                       // [stage]: operands written (kTrProducers arrivals)
    uint64_t *empty = bars + kTrMaxStages;       // [stage]: the stage's MMAs completed (commit)
    uint64_t *acc_full = bars + 2 * kTrMaxStages;   // [2]: an accumulator is complete (commit)
    uint64_t *acc_empty = acc_full + 2;             // [2]: ... and read out (4 epilogue warps)
    uint64_t *drain = acc_empty + 2;
    uint64_t *bfull = drain + 1;                    // [stage]: FWD / BWD: the stage's weights landed (TMA)
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bfull + kTrMaxStages);
    volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);
    // FWD / BWD epilogue constants of the layer in shared memory: [0, N) bias (FWD), [N, 3N) tail
    // weights a and b.  Every row reads each of them once per column; through L1 they would miss,
    // the producers' operand stream evicting them.
    float *s_c = reinterpret_cast<float *>(tmem_slot + 4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int N = P.N;
    const uint32_t a_bytes = kTrBM * 128, b_bytes = (uint32_t)N * 128;
    const int kb_all = (P.K + 63) / 64;
    const int n_tiles = P.m_tiles * P.splits;
    uint32_t tcols = 32;
    while (tcols < 2u * (uint32_t)N) tcols <<= 1;
    auto tile_kb = [&](int t, int &m0, int &kb0, int &kb1) {
        m0 = (t % P.m_tiles) * kTrBM;
        const int sp = t / P.m_tiles;
        kb0 = sp * P.kb_per_split;
        kb1 = min(kb_all, kb0 + P.kb_per_split);
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < P.n_stages; ++s) {
            mbar_init(smem_u32(&full[s]), kTrProducers);
            mbar_init(smem_u32(&bfull[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&acc_full[b]), 1);
            mbar_init(smem_u32(&acc_empty[b]), 4);
        }
        mbar_init(smem_u32(drain), 1);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kTrMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(tcols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (EPI != TR_DW)
        for (int i = threadIdx.x; i < 3 * N; i += kTrThreads)
            s_c[i] = i < N ? (EPI == TR_FWD ? __ldg(P.bias + i) : 0.f) : __ldg(P.tw + (i - N));
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp < kTrProdWarps) {
        // ------------------------------------------------ producers
        const int pt = threadIdx.x;
        uint32_t it = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < n_tiles && ok && (EPI != TR_DW || warp == 0); t += gridDim.x) {
            int m0, kb0, kb1;
            tile_kb(t, m0, kb0, kb1);
            for (int kb = kb0; kb < kb1 && ok; ++kb, ++it) {
                const uint32_t s = it % (uint32_t)P.n_stages, round = it / (uint32_t)P.n_stages;
                if (round > 0) {
                    ok = tr_wait_warp(smem_u32(&empty[s]), (round - 1) & 1u, abort, P.status);
                    if (!ok) break;
                }
                const uint32_t st = smem_u32(smem + (size_t)s * P.stage_bytes);
                if (EPI == TR_DW) {  // both operands: boxes of 64 K-elements x box_rows rows
                    if (pt == 0) {
                        const int ar = min(kTrBM, P.M), br = P.box_rows;
                        mbar_arrive_tx(smem_u32(&bfull[s]), (uint32_t)(2 * ar + 2 * N) * 128u);
                        for (int part = 0; part < 2; ++part) {
                            for (int r = 0; r < ar; r += br)
                                tma_load_2d(st + part * a_bytes + r * 128, &amap, smem_u32(&bfull[s]), kb * 64,
                                            P.a_row0 + part * P.M + m0 + r);
                            for (int r = 0; r < N; r += br)
                                tma_load_2d(st + 2 * a_bytes + part * b_bytes + r * 128, &bmap, smem_u32(&bfull[s]),
                                            kb * 64, P.b_row0 + part * N + r);
                        }
                    }
                    continue;
                }
                if (pt == 0) {  // the weights: two TMA boxes of 64 K-elements x N rows
                    mbar_arrive_tx(smem_u32(&bfull[s]), 2 * b_bytes);
                    tma_load_2d(st + 2 * a_bytes, &bmap, smem_u32(&bfull[s]), kb * 64, P.b_row0);
                    tma_load_2d(st + 2 * a_bytes + b_bytes, &bmap, smem_u32(&bfull[s]), kb * 64, P.b_row0 + N);
                }
                tr_produce_stage<EPI>(P, pt, m0, kb * 64, st, st + a_bytes, st + 2 * a_bytes, st + 2 * a_bytes + b_bytes);
                fence_async_smem();  // generic-proxy writes -> visible to the tensor core's async proxy
                mbar_arrive(smem_u32(&full[s]));
            }
        }
        if (pt == 0 && !ok) {
            // after an abort, let the weight copies still in flight land before the CTA exits
            const uint32_t first = it > (uint32_t)P.n_stages ? it - (uint32_t)P.n_stages : 0u;
            for (uint32_t k = first; k < it; ++k) {
                const uint32_t s2 = k % (uint32_t)P.n_stages, ph2 = (k / (uint32_t)P.n_stages) & 1u;
                const uint64_t t0 = globaltimer();
                while (!mbar_try(smem_u32(&bfull[s2]), ph2) && globaltimer() - t0 < kTimeoutNs) {
                }
            }
        }
    } else if (warp == kTrMmaWarp) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kTrBM >> 4) << 24);
            bool ok = true;
            uint32_t it = 0, ti = 0;
            auto wait = [&](uint32_t bar, uint32_t parity) {
                if (mbar_try(bar, parity)) return true;
                const uint64_t t0 = globaltimer();
                while (!mbar_try(bar, parity)) {
                    if (*abort) return false;
                    if (globaltimer() - t0 > kTimeoutNs) {
                        *abort = 1;
                        atomicOr(P.status, 1u);
                        return false;
                    }
                }
                return true;
            };
            for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x, ++ti) {
                int m0, kb0, kb1;
                tile_kb(t, m0, kb0, kb1);
                const uint32_t b = ti & 1u, use = ti >> 1;
                if (use > 0) {
                    ok = wait(smem_u32(&acc_empty[b]), (use - 1) & 1u);
                    if (!ok) break;
                    tc_fence_after();
                }
                const uint32_t d = tmem + b * (uint32_t)N;
                uint32_t acc = 0;
                for (int kb = kb0; kb < kb1 && ok; ++kb, ++it) {
                    const uint32_t s = it % (uint32_t)P.n_stages, round = it / (uint32_t)P.n_stages;
                    if (EPI != TR_DW) ok = wait(smem_u32(&full[s]), round & 1u);
                    if (ok) ok = wait(smem_u32(&bfull[s]), round & 1u);
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t st = smem_u32(smem + (size_t)s * P.stage_bytes);
                    const uint32_t ahi = st, alo = st + a_bytes, bhi = st + 2 * a_bytes, blo = bhi + b_bytes;
                    const int ksteps = min(4, (P.K - kb * 64 + 15) / 16);
                    for (int k = 0; k < ksteps; ++k) {
                        const uint64_t dah = smem_desc(ahi + 32 * k), dal = smem_desc(alo + 32 * k);
                        const uint64_t dbh = smem_desc(bhi + 32 * k), dbl = smem_desc(blo + 32 * k);
                        mma_f16(d, dah, dbh, idesc, acc);
                        mma_f16(d, dal, dbh, idesc, 1u);
                        mma_f16(d, dah, dbl, idesc, 1u);
                        acc = 1u;
                    }
                    mma_commit(smem_u32(&empty[s]));
                }
                if (ok) mma_commit(smem_u32(&acc_full[b]));
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
        // ------------------------------------------------ epilogue
        const int q = warp & 3;
        const int r = q * 32 + lane;
        bool ok = true;
        uint32_t ti = 0;
        const float inv_s = EPI == TR_DW ? 1.f : __ldg(P.inv_s);
        // each 32 x 32 output chunk leaves through the warp's staging tile by one TMA store: a
        // thread writes its row's 128 bytes (swizzled, so the eight rows of a store phase hit
        // distinct banks), instead of 32 rows' scattered float4 stores through L1
        const uint32_t stg = smem_u32(stage_out) + (uint32_t)(q * kTrStoreTile);
        auto put = [&](int c0, int row0, const float *o) {
            if (lane == 0) tr_bulk_wait_read();
            __syncwarp();
#pragma unroll
            for (int j = 0; j < 8; ++j)
                st_shared_v4(stg + tr_swz(lane, j), make_uint4(__float_as_uint(o[4 * j]), __float_as_uint(o[4 * j + 1]),
                                                                __float_as_uint(o[4 * j + 2]), __float_as_uint(o[4 * j + 3])));
            fence_async_smem();
            __syncwarp();
            if (lane == 0) {
                tr_tma_store_2d(&omap, stg, c0, row0);
                tr_bulk_commit();
            }
        };
        for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x, ++ti) {
            int m0, kb0, kb1;
            tile_kb(t, m0, kb0, kb1);
            const uint32_t b = ti & 1u, use = ti >> 1;
            ok = tr_wait_warp(smem_u32(&acc_full[b]), use & 1u, abort, P.status);
            if (!ok) break;
            tc_fence_after();
            const uint32_t t_lane = tmem + b * (uint32_t)N + ((uint32_t)(q * 32) << 16);
            const int row = m0 + r;
            const bool live = row < P.M;
            const int split = t / P.m_tiles;
            float sa = 0.f, sb = 0.f;
            float gl = 0.f, tav = 0.f, tbv = 0.f;
            if (EPI == TR_BWD && live) {
                gl = __ldg(P.g_prev + row);
                tav = __ldg(P.ta_prev + row);
                tbv = __ldg(P.tb_prev + row);
            }
            // BWD: z_{l-1} of the row, one 32-column chunk ahead of its use
            float4 zc[8], zn[8];
            if (EPI == TR_BWD) {
                const float4 *zp = reinterpret_cast<const float4 *>(P.z_prev + (size_t)(live ? row : 0) * N);
#pragma unroll
                for (int j = 0; j < 8; ++j) zn[j] = __ldg(zp + j);
            }
            for (int c0 = 0; c0 < N; c0 += 32) {
                uint32_t v[32];
                tmem_ld32(t_lane + (uint32_t)c0, v);
                if (EPI == TR_BWD) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) zc[j] = zn[j];
                    if (c0 + 32 < N) {
                        const float4 *zp = reinterpret_cast<const float4 *>(P.z_prev + (size_t)(live ? row : 0) * N + c0 + 32);
#pragma unroll
                        for (int j = 0; j < 8; ++j) zn[j] = __ldg(zp + j);
                    }
                }
                tmem_wait_ld();
                // rows >= M: whole warps (M is a multiple of 32: the tile of a 64-wide weight gradient)
                if (!live) continue;
                const int orow = P.out_row0 + (EPI == TR_DW ? split * P.M : 0) + m0 + q * 32;
                if (EPI == TR_DW) {
                    put(c0, orow, reinterpret_cast<const float *>(v));
                } else if (EPI == TR_FWD) {
                    float z[32];
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const int col = c0 + i;
                        z[i] = fmaf(__uint_as_float(v[i]), inv_s, s_c[col]);
                        const float h = tr_act(P.act, z[i], P.omega0);
                        sa = fmaf(s_c[N + col], h, sa);
                        if (P.mult) sb = fmaf(s_c[2 * N + col], h, sb);
                    }
                    put(c0, orow, z);
                } else {  // TR_BWD
                    float dd[32];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float zv[4] = {zc[j].x, zc[j].y, zc[j].z, zc[j].w};
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int col = c0 + 4 * j + e;
                            // dt_{l-1}/dh_{l-1}: a (affine tail) or tb a + ta b (Eq. 3)
                            const float tvec = P.mult ? fmaf(tbv, s_c[N + col], tav * s_c[2 * N + col]) : s_c[N + col];
                            const float g = fmaf(__uint_as_float(v[4 * j + e]), inv_s, gl * tvec);
                            dd[4 * j + e] = g * tr_slope(P.act, zv[e], P.omega0);
                        }
                    }
                    put(c0, orow, dd);
                }
            }
            // the accumulator has been read: the MMAs of the tile after next may overwrite it
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&acc_empty[b]));
            if (EPI == TR_FWD && live) {
                const float ta = sa + __ldg(P.tbias);
                const float tb = P.mult ? sb + __ldg(P.tbias + 1) : 1.f;
                P.y_out[row] = __ldg(P.y_prev + row) + ta * tb;
                P.ta_out[row] = ta;
                P.tb_out[row] = tb;
            }
        }
        if (lane == 0) tr_bulk_wait_all();  // the staging tiles stay valid until every store is done
        __syncwarp();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kTrMmaWarp) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
    }
}

// ---------------------------------------------------------------------------------------- small kernels
// Per-layer weight scales: s_l = 2^-e with max|W_l| = f 2^e, f in [0.5, 1) (1 for an all-zero layer).
__global__ void tr_amax_kernel(const float *Wh, int W, float *scale, float *inv_scale) {
    const int li = blockIdx.x;
    const float4 *w = reinterpret_cast<const float4 *>(Wh + (size_t)li * W * W);  // W * W is a multiple of 4
    float m = 0.f;
    for (int i = threadIdx.x; i < W * W / 4; i += blockDim.x) {
        const float4 v = w[i];
        m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    }
    __shared__ float red[32];
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float a = 0.f;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) a = fmaxf(a, red[i]);
        int e = 0;
        if (a > 0.f) frexpf(a, &e);
        scale[li] = ldexpf(1.f, -e);
        inv_scale[li] = ldexpf(1.f, e);
    }
}

// W_l s_l as fp16 hi + lo: forward rows [li][part][out][in], backward rows [li][part][in][out].
__global__ void tr_pack_kernel(const float *Wh, int W, int n_layers_h, const float *scale, uint16_t *wf, uint16_t *wb) {
    const int64_t total = (int64_t)n_layers_h * W * W;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int li = (int)(i / ((int64_t)W * W));
        const int rem = (int)(i % ((int64_t)W * W));
        const int j = rem / W, k = rem % W;
        const float w = Wh[i] * scale[li];
        const __half h = __float2half_rn(w);
        const __half l = __float2half_rn(w - __half2float(h));
        const uint16_t hb = *reinterpret_cast<const uint16_t *>(&h), lb = *reinterpret_cast<const uint16_t *>(&l);
        const size_t base = (size_t)li * 2 * W * W;
        wf[base + (size_t)j * W + k] = hb;
        wf[base + (size_t)W * W + (size_t)j * W + k] = lb;
        wb[base + (size_t)k * W + j] = hb;
        wb[base + (size_t)W * W + (size_t)k * W + j] = lb;
    }
}

// Layer 1 (fan-in 3) on the CUDA cores, one warp per row: z_1 = W_1 x + b_1, tail 1 (affine), y_1.
__global__ void tr_fwd1_kernel(const float *pts, int64_t n, int64_t B, int W, int act, float w0, const float *W1,
                               const float *b1, const float *tw1, const float *tb1, float *Z1, float *Y1, float *TA1,
                               float *TB1) {
    const int lane = threadIdx.x & 31;
    for (int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; row < B;
         row += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        float x0 = 0.f, x1 = 0.f, x2 = 0.f;
        if (row < n) {
            x0 = pts[3 * row];
            x1 = pts[3 * row + 1];
            x2 = pts[3 * row + 2];
        }
        float s = 0.f;
        for (int j = lane; j < W; j += 32) {
            const float z = fmaf(W1[3 * j], x0, fmaf(W1[3 * j + 1], x1, fmaf(W1[3 * j + 2], x2, b1[j])));
            Z1[row * W + j] = z;
            s = fmaf(tw1[j], tr_act(act, z, w0), s);
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            const float ta = s + tb1[0];
            Y1[row] = ta;
            TA1[row] = ta;
            TB1[row] = 1.f;
        }
    }
}

// The weight-gradient operands, transposed and split: out[z][0][n][k] + out[z][1][n][k] = f(X[z][k][n])
// (hi = fp16 of the value, lo = fp16 of the rest, as the GEMM producers split) for n < W, k < B, with
// f the activation (act >= 0) or the identity (act < 0): rows of `cap` fp16, k contiguous, the
// K-major layout the weight-gradient GEMM loads by TMA.  One block per 64 x 64 tile, through shared
// memory so that both the reads (along n) and the writes (along k) are coalesced.
__global__ void __launch_bounds__(256) tr_tsplit_kernel(const float *X, int W, int act, float w0, uint16_t *out,
                                                       int64_t cap) {
    __shared__ float tile[64][65];
    const int64_t k0 = (int64_t)blockIdx.x * 64;
    const int n0 = blockIdx.y * 64;
    const float *Xz = X + (size_t)blockIdx.z * cap * W;
    uint16_t *hi = out + (size_t)blockIdx.z * 2 * W * cap, *lo = hi + (size_t)W * cap;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int idx = threadIdx.x + 256 * i, r = idx >> 6, c = idx & 63;
        const float v = Xz[(k0 + r) * W + n0 + c];
        tile[r][c] = act >= 0 ? tr_act(act, v, w0) : v;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int idx = threadIdx.x + 256 * i, nl = idx >> 5, kp = idx & 31;
        const float a = tile[2 * kp][nl], b = tile[2 * kp + 1][nl];
        const __half2 hp = __floats2half2_rn(a, b);
        const float2 hf = __half22float2(hp);
        const __half2 lp = __floats2half2_rn(a - hf.x, b - hf.y);
        const size_t at = (size_t)(n0 + nl) * cap + k0 + 2 * kp;
        *reinterpret_cast<__half2 *>(hi + at) = hp;
        *reinterpret_cast<__half2 *>(lo + at) = lp;
    }
}

// Per row: G'_k = sum_{i >= k} sign(y_i - y_gt) (0 for padding rows); per block: sum of |y_i - y_gt|.
__global__ void tr_loss_kernel(const float *Y, const float *gt, int64_t n, int64_t B, int64_t ld, int L, float *G,
                               float *loss_part) {
    float s = 0.f;
    for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < B; row += (int64_t)gridDim.x * blockDim.x) {
        float g = 0.f;
        const float t = row < n ? gt[row] : 0.f;
        for (int l = L - 1; l >= 0; --l) {
            if (row < n) {
                const float r = Y[(size_t)l * ld + row] - t;
                s += fabsf(r);
                g += r > 0.f ? 1.f : (r < 0.f ? -1.f : 0.f);
            }
            G[(size_t)l * ld + row] = g;
        }
    }
    __shared__ float red[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float a = 0.f;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) a += red[i];
        loss_part[blockIdx.x] = a;
    }
}

// delta'_L = G'_L dt_L/dh_L * act'(z_L).
__global__ void tr_top_kernel(const float *ZL, const float *GL, const float *TAL, const float *TBL, const float *twL,
                              int mult, int64_t B, int W, int act, float w0, float *DL) {
    const int64_t total = B * W;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = i / W;
        const int k = (int)(i % W);
        const float tv = mult ? fmaf(TBL[row], twL[k], TAL[row] * twL[W + k]) : twL[k];
        DL[i] = GL[row] * tv * tr_slope(act, ZL[i], w0);
    }
}

// Column sums over the rows [s R, (s+1) R) of one layer (blockIdx.y = layer l - 1, blockIdx.x = s),
// one thread per unit j: sum delta'_l, sum G'_l tb h_l, sum G'_l ta h_l, and for l = 1
// sum delta'_1 x_c; thread 0 also writes sum G'_l tb and sum G'_l ta.  Partials [L][S][slots].
// Four rows per iteration with their own accumulators keep four rows of loads in flight.
constexpr int kTrSlots = 6;  // per unit: db, da, dbt, dW1 x, y, z
__global__ void tr_colsum_kernel(const float *Z, const float *D, const float *G, const float *TA, const float *TB,
                                 const float *pts, int64_t n, int64_t B, int64_t ld, int W, int act, float w0,
                                 const int *mult_of, int64_t rows_per, float *part, float *part_bias) {
    const int l = blockIdx.y;  // 0-based layer
    const int s = blockIdx.x;
    const int j = threadIdx.x < W ? threadIdx.x : W - 1;  // threads beyond W repeat the last unit, write nothing
    const int64_t r0 = (int64_t)s * rows_per, r1 = min(B, r0 + rows_per);
    const bool mult = mult_of[l] != 0;
    const float *Zl = Z + (size_t)l * ld * W, *Dl = D + (size_t)l * ld * W;
    const float *Gl = G + (size_t)l * ld, *TAl = TA + (size_t)l * ld, *TBl = TB + (size_t)l * ld;
    float a[4][8];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int k = 0; k < 8; ++k) a[u][k] = 0.f;
    // delta' is 0 on padding rows (row >= n), so their coordinates may be any finite value: the
    // point index is clamped and no load is conditional, which keeps four rows of loads in flight
    auto add_row = [&](float *acc, int64_t rr) {
        const float d = Dl[rr * W + j];
        const float g = Gl[rr];
        const float tb = TBl[rr], ta = TAl[rr];
        const float h = tr_act(act, Zl[rr * W + j], w0);
        acc[0] += d;
        acc[1] = fmaf(g * tb, h, acc[1]);
        if (mult) acc[2] = fmaf(g * ta, h, acc[2]);
        if (l == 0) {
            const int64_t pr = rr < n ? rr : n - 1;
            acc[3] = fmaf(d, pts[3 * pr], acc[3]);
            acc[4] = fmaf(d, pts[3 * pr + 1], acc[4]);
            acc[5] = fmaf(d, pts[3 * pr + 2], acc[5]);
        }
        acc[6] = fmaf(g, tb, acc[6]);
        acc[7] = fmaf(g, ta, acc[7]);
    };
    int64_t row = r0;
    for (; row + 4 <= r1; row += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) add_row(a[u], row + u);
    }
    for (; row < r1; ++row) add_row(a[0], row);
    float t[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) t[k] = (a[0][k] + a[1][k]) + (a[2][k] + a[3][k]);
    if (threadIdx.x < W) {
        float *p = part + (((size_t)l * gridDim.x + s) * kTrSlots) * W;
#pragma unroll
        for (int k = 0; k < kTrSlots; ++k) p[k * W + j] = t[k];
    }
    if (threadIdx.x == 0) {
        part_bias[((size_t)l * gridDim.x + s) * 2] = t[6];
        part_bias[((size_t)l * gridDim.x + s) * 2 + 1] = mult ? t[7] : 0.f;
    }
}

// The gradient in the parameter-block order (W1, b1, Wh, bh, tail_w, tail_b): partials added in a
// fixed order, divided by n.
__global__ void tr_finalize_kernel(const float *part, const float *part_bias, const float *dw_part, int S, int S_dw,
                                   int W, int L, float inv_n, float *grad) {
    const size_t oW1 = 0, ob1 = (size_t)3 * W, oWh = ob1 + W, obh = oWh + (size_t)(L - 1) * W * W;
    const size_t otw = obh + (size_t)(L - 1) * W, otb = otw + (size_t)L * 2 * W;
    const size_t total = otb + (size_t)L * 2;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        // the partials of element i: count values `stride` apart from `base` (eight running sums,
        // added in a fixed order)
        const float *base;
        size_t stride;
        int count;
        if (i >= oWh && i < obh) {  // dW_l, l >= 2: rows out, columns in
            const size_t li = (i - oWh) / ((size_t)W * W), rem = (i - oWh) % ((size_t)W * W);
            base = dw_part + li * S_dw * (size_t)W * W + rem;
            stride = (size_t)W * W;
            count = S_dw;
        } else if (i >= otb) {  // tail biases
            const size_t l = (i - otb) / 2, which = (i - otb) % 2;
            base = part_bias + l * S * 2 + which;
            stride = 2;
            count = S;
        } else {
            int l, slot, j;
            if (i < ob1) { l = 0; slot = 3 + (int)((i - oW1) % 3); j = (int)((i - oW1) / 3); }
            else if (i < oWh) { l = 0; slot = 0; j = (int)(i - ob1); }
            else if (i < otw) { l = 1 + (int)((i - obh) / W); slot = 0; j = (int)((i - obh) % W); }
            else { l = (int)((i - otw) / (2 * W)); slot = 1 + (int)(((i - otw) % (2 * W)) / W); j = (int)((i - otw) % W); }
            base = part + ((size_t)l * S * kTrSlots + slot) * W + j;
            stride = (size_t)kTrSlots * W;
            count = S;
        }
        float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        int s = 0;
        for (; s + 16 <= count; s += 16) {  // sixteen loads in flight, added in the order of the loop below
            float v[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) v[u] = base[(size_t)(s + u) * stride];
#pragma unroll
            for (int u = 0; u < 8; ++u) acc[u] += v[u];
#pragma unroll
            for (int u = 0; u < 8; ++u) acc[u] += v[8 + u];
        }
        for (; s + 8 <= count; s += 8) {
#pragma unroll
            for (int u = 0; u < 8; ++u) acc[u] += base[(size_t)(s + u) * stride];
        }
        for (; s < count; ++s) acc[0] += base[(size_t)s * stride];
        const float v = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
        grad[i] = v * inv_n;
    }
}

// One Adam update: m <- b1 m + (1 - b1) g; v <- b2 v + (1 - b2) g^2; p <- p - lr m_hat / (sqrt(v_hat) + eps).
__global__ void tr_adam_kernel(float *p, const float *g, float *m, float *v, int64_t np, float lr, float b1, float b2,
                               float eps, float c1, float c2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = fmaf(b1, m[i], (1.f - b1) * gi);
        const float vi = fmaf(b2, v[i], (1.f - b2) * gi * gi);
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

__global__ void tr_loss_final_kernel(const float *loss_part, int nb, float inv_n, float *loss) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        float s = 0.f;
        for (int i = 0; i < nb; ++i) s += loss_part[i];
        *loss = s * inv_n;
    }
}

}  // namespace sand

using namespace sand;

struct sand_trainer_s {
    sand_model m = nullptr;
    int device = 0, num_sms = 0;
    int L = 0, W = 0, act = 0, tail = 0;
    float w0 = 30.f;
    int64_t cap = 0;  // padded rows
    float lr = 1e-4f, b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    int64_t step = 0;
    size_t np = 0;
    void *mem = nullptr;
    float *params = nullptr, *grad = nullptr, *am = nullptr, *av = nullptr;
    float *scale = nullptr, *inv_scale = nullptr;
    uint16_t *wf = nullptr, *wb = nullptr;
    CUtensorMap map_f{}, map_b{};  // TMA maps over wf and wb: rows of W fp16, boxes of 64 x W
    // weight-gradient operands [L-1][hi, lo][W][cap] fp16: delta'_l^T (l = 2..L) and act(z_l)^T
    // (l = 1..L-1), with their TMA maps (boxes of 64 x min(128, W))
    uint16_t *dt = nullptr, *ht = nullptr;
    CUtensorMap map_dt{}, map_ht{};
    // TMA maps over the GEMM outputs, rows of W float32 in boxes of 32 x 32: Z and D ([L][cap]
    // rows) and the weight-gradient partials ([L-1][S_dw][W] rows)
    CUtensorMap map_z{}, map_d{}, map_dw{};
    float *Z = nullptr, *D = nullptr, *Y = nullptr, *TA = nullptr, *TB = nullptr, *G = nullptr;
    float *dw_part = nullptr, *part = nullptr, *part_bias = nullptr, *loss_part = nullptr, *loss = nullptr;
    int *mult_of = nullptr;
    unsigned *status = nullptr;
    int S = 0, S_dw = 0, loss_blocks = 0;
};

namespace {

constexpr int kTrColsumSplits = 256;
constexpr int kTrLossBlocks = 304;

size_t tr_stage_bytes(int N) { return (size_t)2 * kTrBM * 128 + (size_t)2 * N * 128; }

int tr_stages(int N) {
    const size_t misc = 1024 + 4 * kTrStoreTile + 8 * (3 * kTrMaxStages + 5) + 16 + (size_t)3 * N * 4;
    int s = (int)((kTrSmem - misc) / tr_stage_bytes(N));
    return s > kTrMaxStages ? kTrMaxStages : s;
}

size_t tr_smem(int N, int stages) {
    return 1024 + (size_t)stages * tr_stage_bytes(N) + 4 * kTrStoreTile + 8 * (3 * kTrMaxStages + 5) + 16 +
           (size_t)3 * N * 4;
}

template <int EPI>
cudaError_t tr_launch(const CUtensorMap &amap, const CUtensorMap &bmap, const CUtensorMap &omap, TrGemm P, int num_sms,
                      cudaStream_t s) {
    P.n_stages = tr_stages(P.N);
    P.stage_bytes = (uint32_t)tr_stage_bytes(P.N);
    const int n_tiles = P.m_tiles * P.splits;
    const dim3 grid((unsigned)(n_tiles < num_sms ? n_tiles : num_sms));
    const size_t smem = tr_smem(P.N, P.n_stages);
    cudaError_t e = cudaFuncSetAttribute(tr_gemm_kernel<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    tr_gemm_kernel<EPI><<<grid, kTrThreads, smem, s>>>(amap, bmap, omap, P);
    return cudaGetLastError();
}

}  // namespace

extern "C" {

sand_status sand_trainer_create(sand_model m, const sand_train_opts *opts, sand_trainer *out) {
    if (!m || !out) {
        set_error("NULL model or output");
        return SAND_EINVAL;
    }
    *out = nullptr;
    const sand_tmlp_desc &d = model_desc_ref(m);
    if (d.encoder != SAND_ENC_NONE || (d.width != 64 && d.width != 128 && d.width != 256) || d.n_layers < 2) {
        set_error("training takes raw-coordinate models of width 64, 128 or 256 with at least 2 layers");
        return SAND_EUNSUPPORTED;
    }
    sand_train_opts o{};
    if (opts) o = *opts;
    if (o.max_points == 0) o.max_points = (int64_t)1 << 17;
    if (o.lr == 0.f) o.lr = 1e-4f;
    if (o.beta1 == 0.f) o.beta1 = 0.9f;
    if (o.beta2 == 0.f) o.beta2 = 0.999f;
    if (o.eps == 0.f) o.eps = 1e-8f;
    if (o.max_points < 1 || o.max_points > ((int64_t)1 << 26) || !(o.lr > 0.f) || !(o.beta1 >= 0.f && o.beta1 < 1.f) ||
        !(o.beta2 >= 0.f && o.beta2 < 1.f) || !(o.eps > 0.f)) {
        set_error("training options out of range");
        return SAND_EINVAL;
    }
    auto *T = new sand_trainer_s();
    T->m = m;
    T->device = model_device(m);
    T->L = d.n_layers;
    T->W = d.width;
    T->act = d.activation;
    T->tail = d.tail_kind;
    T->w0 = d.omega0;
    T->cap = (o.max_points + kTrBM - 1) / kTrBM * kTrBM;
    T->lr = o.lr;
    T->b1 = o.beta1;
    T->b2 = o.beta2;
    T->eps = o.eps;
    T->np = model_param_count(m);
    const int L = T->L, W = T->W;
    const int64_t B = T->cap;
    T->S = kTrColsumSplits;
    T->S_dw = 0;
    T->loss_blocks = kTrLossBlocks;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(T->device);
    cudaDeviceGetAttribute(&T->num_sms, cudaDevAttrMultiProcessorCount, T->device);
    const int m_tiles = (W + kTrBM - 1) / kTrBM;
    T->S_dw = T->num_sms / m_tiles;
    if (T->S_dw < 1) T->S_dw = 1;
    // one allocation, 256-byte aligned pieces
    std::vector<std::pair<void **, size_t>> parts = {
        {(void **)&T->params, T->np * 4}, {(void **)&T->grad, T->np * 4}, {(void **)&T->am, T->np * 4},
        {(void **)&T->av, T->np * 4}, {(void **)&T->scale, 4 * kMaxLayers}, {(void **)&T->inv_scale, 4 * kMaxLayers},
        {(void **)&T->wf, (size_t)(L - 1) * 2 * W * W * 2}, {(void **)&T->wb, (size_t)(L - 1) * 2 * W * W * 2},
        {(void **)&T->dt, (size_t)(L - 1) * 2 * W * B * 2}, {(void **)&T->ht, (size_t)(L - 1) * 2 * W * B * 2},
        {(void **)&T->Z, (size_t)L * B * W * 4}, {(void **)&T->D, (size_t)L * B * W * 4},
        {(void **)&T->Y, (size_t)L * B * 4}, {(void **)&T->TA, (size_t)L * B * 4}, {(void **)&T->TB, (size_t)L * B * 4},
        {(void **)&T->G, (size_t)L * B * 4}, {(void **)&T->dw_part, (size_t)(L - 1) * T->S_dw * W * W * 4},
        {(void **)&T->part, (size_t)L * T->S * kTrSlots * W * 4}, {(void **)&T->part_bias, (size_t)L * T->S * 2 * 4},
        {(void **)&T->loss_part, (size_t)T->loss_blocks * 4}, {(void **)&T->loss, 4},
        {(void **)&T->mult_of, 4 * kMaxLayers}, {(void **)&T->status, 4}};
    size_t total = 0;
    for (auto &p : parts) total += (p.second + 255) / 256 * 256;
    if (cudaMalloc(&T->mem, total) != cudaSuccess) {
        cudaGetLastError();
        if (prev >= 0) cudaSetDevice(prev);
        delete T;
        set_error("cannot allocate %zu bytes of training buffers", total);
        return SAND_ENOMEM;
    }
    size_t off = 0;
    for (auto &p : parts) {
        *p.first = static_cast<char *>(T->mem) + off;
        off += (p.second + 255) / 256 * 256;
    }
    const uint32_t box_r = W < kTrBM ? (uint32_t)W : (uint32_t)kTrBM;
    if (!encode_u16_rows(&T->map_f, T->wf, (uint64_t)W, (uint64_t)(L - 1) * 2 * W, 64u, (uint32_t)W) ||
        !encode_u16_rows(&T->map_b, T->wb, (uint64_t)W, (uint64_t)(L - 1) * 2 * W, 64u, (uint32_t)W) ||
        !encode_u16_rows(&T->map_dt, T->dt, (uint64_t)B, (uint64_t)(L - 1) * 2 * W, 64u, box_r) ||
        !encode_u16_rows(&T->map_ht, T->ht, (uint64_t)B, (uint64_t)(L - 1) * 2 * W, 64u, box_r) ||
        !encode_f32_rows(&T->map_z, T->Z, (uint64_t)W, (uint64_t)L * B, 32u, 32u) ||
        !encode_f32_rows(&T->map_d, T->D, (uint64_t)W, (uint64_t)L * B, 32u, 32u) ||
        !encode_f32_rows(&T->map_dw, T->dw_part, (uint64_t)W, (uint64_t)(L - 1) * T->S_dw * W, 32u, 32u)) {
        if (prev >= 0) cudaSetDevice(prev);
        cudaFree(T->mem);
        delete T;
        set_error("cannot encode the TMA tensor maps of the training buffers");
        return SAND_ECUDA;
    }
    std::vector<int> mult(kMaxLayers, 0);
    for (int l = 1; l < L; ++l) mult[l] = T->tail == SAND_TAIL_MULT ? 1 : 0;
    cudaError_t e = cudaMemset(T->mem, 0, total);
    if (e == cudaSuccess) e = cudaMemcpy(T->params, model_params(m), T->np * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(T->mult_of, mult.data(), 4 * kMaxLayers, cudaMemcpyHostToDevice);
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        cudaFree(T->mem);
        delete T;
        return cuda_fail(e, "training buffer set-up");
    }
    *out = T;
    return SAND_OK;
}

sand_status sand_train_step(sand_trainer T, const float *d_points, const float *d_targets, int64_t n, float *d_loss,
                            float *d_grad, int update, void *stream) {
    if (!T) {
        set_error("NULL trainer");
        return SAND_EINVAL;
    }
    if (n < 1 || n > T->cap || !d_points || !d_targets) {
        set_error("need 1 <= n <= %lld points and targets", (long long)T->cap);
        return SAND_EINVAL;
    }
    if ((reinterpret_cast<uintptr_t>(d_points) & 3) || (reinterpret_cast<uintptr_t>(d_targets) & 3) ||
        (reinterpret_cast<uintptr_t>(d_loss) & 3) || (reinterpret_cast<uintptr_t>(d_grad) & 3)) {
        set_error("device buffers must be 4-byte aligned");
        return SAND_EINVAL;
    }
    const int L = T->L, W = T->W;
    const int64_t B = (n + kTrBM - 1) / kTrBM * kTrBM;  // rows of this batch
    const int64_t cap = T->cap;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(T->device) != cudaSuccess) {
        set_error("cannot select device %d", T->device);
        return SAND_ECUDA;
    }
    struct Restore {
        int p;
        ~Restore() { if (p >= 0) cudaSetDevice(p); }
    } restore{prev};
    // parameter-block offsets (no Fourier matrix)
    const size_t oW1 = 0, ob1 = (size_t)3 * W, oWh = ob1 + W, obh = oWh + (size_t)(L - 1) * W * W;
    const size_t otw = obh + (size_t)(L - 1) * W, otb = otw + (size_t)L * 2 * W;
    float *P = T->params;
    auto Zl = [&](int l) { return T->Z + (size_t)(l - 1) * cap * W; };  // layers 1-based; rows 0..B used
    auto Dl = [&](int l) { return T->D + (size_t)(l - 1) * cap * W; };
    auto row = [&](float *base, int l) { return base + (size_t)(l - 1) * cap; };
    // weights of this step: scales and split packing
    tr_amax_kernel<<<L - 1, 1024, 0, s>>>(P + oWh, W, T->scale, T->inv_scale);
    tr_pack_kernel<<<2 * T->num_sms, 256, 0, s>>>(P + oWh, W, L - 1, T->scale, T->wf, T->wb);
    // forward
    {
        int64_t blocks = (B * 32 + 255) / 256;
        if (blocks > 8 * T->num_sms) blocks = 8 * T->num_sms;
        tr_fwd1_kernel<<<(unsigned)blocks, 256, 0, s>>>(d_points, n, B, W, T->act, T->w0, P + oW1, P + ob1, P + otw,
                                                         P + otb, Zl(1), row(T->Y, 1), row(T->TA, 1), row(T->TB, 1));
        SAND_CUDA(cudaGetLastError(), "layer-1 kernel");
    }
    const int row_tiles = (int)(B / kTrBM);
    const bool mult = T->tail == SAND_TAIL_MULT;
    for (int l = 2; l <= L; ++l) {
        TrGemm g{};
        g.M = (int)B;
        g.N = W;
        g.K = W;
        g.act = T->act;
        g.omega0 = T->w0;
        g.a = Zl(l - 1);
        g.a_ld = W;
        g.b_row0 = (l - 2) * 2 * W;
        g.out = Zl(l);
        g.out_row0 = (int)((l - 1) * cap);
        g.inv_s = T->inv_scale + (l - 2);
        g.bias = P + obh + (size_t)(l - 2) * W;
        g.tw = P + otw + (size_t)(l - 1) * 2 * W;
        g.tbias = P + otb + (size_t)(l - 1) * 2;
        g.mult = mult;
        g.y_prev = row(T->Y, l - 1);
        g.y_out = row(T->Y, l);
        g.ta_out = row(T->TA, l);
        g.tb_out = row(T->TB, l);
        g.status = T->status;
        g.m_tiles = row_tiles;
        g.splits = 1;
        g.kb_per_split = W / 64;
        SAND_CUDA(tr_launch<TR_FWD>(T->map_f, T->map_f, T->map_z, g, T->num_sms, s), "forward GEMM");
    }
    // loss, dL/dt (as the integers G'), delta'_L
    tr_loss_kernel<<<T->loss_blocks, 256, 0, s>>>(T->Y, d_targets, n, B, cap, L, T->G, T->loss_part);
    SAND_CUDA(cudaGetLastError(), "loss kernel");
    {
        int64_t blocks = (B * W + 255) / 256;
        if (blocks > 8 * T->num_sms) blocks = 8 * T->num_sms;
        tr_top_kernel<<<(unsigned)blocks, 256, 0, s>>>(Zl(L), row(T->G, L), row(T->TA, L), row(T->TB, L),
                                                        P + otw + (size_t)(L - 1) * 2 * W, mult && L >= 2 ? 1 : 0, B,
                                                        W, T->act, T->w0, Dl(L));
        SAND_CUDA(cudaGetLastError(), "top-layer delta kernel");
    }
    // the weight-gradient operands known so far: act(z_l)^T for l = 1..L-1 and delta'_L^T
    tr_tsplit_kernel<<<dim3((unsigned)(B / 64), (unsigned)(W / 64), (unsigned)(L - 1)), 256, 0, s>>>(
        Zl(1), W, T->act, T->w0, T->ht, cap);
    SAND_CUDA(cudaGetLastError(), "activation transpose kernel");
    tr_tsplit_kernel<<<dim3((unsigned)(B / 64), (unsigned)(W / 64), 1), 256, 0, s>>>(
        Dl(L), W, -1, 0.f, T->dt + (size_t)(L - 2) * 2 * W * cap, cap);
    SAND_CUDA(cudaGetLastError(), "delta transpose kernel");
    // backward: delta'_{l-1} from delta'_l, and the weight-gradient partials of layer l
    const int m_tiles = (W + kTrBM - 1) / kTrBM;
    const int kb_all = (int)(B / 64);
    const int kb_per = (kb_all + T->S_dw - 1) / T->S_dw;
    const int splits = (kb_all + kb_per - 1) / kb_per;
    for (int l = L; l >= 2; --l) {
        TrGemm g{};
        g.M = (int)B;
        g.N = W;
        g.K = W;
        g.act = T->act;
        g.omega0 = T->w0;
        g.a = Dl(l);
        g.a_ld = W;
        g.b_row0 = (l - 2) * 2 * W;
        g.out = Dl(l - 1);
        g.out_row0 = (int)((l - 2) * cap);
        g.inv_s = T->inv_scale + (l - 2);
        g.tw = P + otw + (size_t)(l - 2) * 2 * W;
        g.mult = mult && l - 1 >= 2;
        g.z_prev = Zl(l - 1);
        g.g_prev = row(T->G, l - 1);
        g.ta_prev = row(T->TA, l - 1);
        g.tb_prev = row(T->TB, l - 1);
        g.status = T->status;
        g.m_tiles = row_tiles;
        g.splits = 1;
        g.kb_per_split = W / 64;
        SAND_CUDA(tr_launch<TR_BWD>(T->map_b, T->map_b, T->map_d, g, T->num_sms, s), "backward GEMM");
        // delta'_{l-1}, transposed and split for the weight gradient of layer l - 1
        if (l - 1 >= 2) {
            tr_tsplit_kernel<<<dim3((unsigned)(B / 64), (unsigned)(W / 64), 1), 256, 0, s>>>(
                Dl(l - 1), W, -1, 0.f, T->dt + (size_t)(l - 3) * 2 * W * cap, cap);
            SAND_CUDA(cudaGetLastError(), "delta transpose kernel");
        }
        TrGemm w{};
        w.M = W;
        w.N = W;
        w.K = (int)B;
        w.kb_per_split = kb_per;
        w.act = T->act;
        w.omega0 = T->w0;
        w.a_row0 = (l - 2) * 2 * W;
        w.b_row0 = (l - 2) * 2 * W;
        w.box_rows = (int)(W < kTrBM ? W : kTrBM);
        w.out = T->dw_part + (size_t)(l - 2) * T->S_dw * W * W;
        w.out_row0 = (l - 2) * T->S_dw * W;
        w.status = T->status;
        w.m_tiles = m_tiles;
        w.splits = splits;
        SAND_CUDA(tr_launch<TR_DW>(T->map_dt, T->map_ht, T->map_dw, w, T->num_sms, s), "weight-gradient GEMM");
        if (splits < T->S_dw)  // unused split slots must read as zero
            SAND_CUDA(cudaMemsetAsync(w.out + (size_t)splits * W * W, 0, (size_t)(T->S_dw - splits) * W * W * 4, s),
                      "partials reset");
    }
    // column sums, the gradient, the loss
    {
        const int64_t rows_per = (B + T->S - 1) / T->S;
        tr_colsum_kernel<<<dim3((unsigned)T->S, (unsigned)L), W, 0, s>>>(T->Z, T->D, T->G, T->TA, T->TB, d_points, n, B,
                                                                         cap, W, T->act, T->w0, T->mult_of, rows_per,
                                                                         T->part, T->part_bias);
        SAND_CUDA(cudaGetLastError(), "column-sum kernel");
        // one element per thread: each sums its S (or S_dw) partials with sixteen loads in flight
        const unsigned fin_blocks = (unsigned)((T->np + 255) / 256);
        tr_finalize_kernel<<<fin_blocks, 256, 0, s>>>(T->part, T->part_bias, T->dw_part, T->S, T->S_dw, W, L,
                                                      (float)(1.0 / (double)n), T->grad);
        SAND_CUDA(cudaGetLastError(), "gradient kernel");
        tr_loss_final_kernel<<<1, 32, 0, s>>>(T->loss_part, T->loss_blocks, (float)(1.0 / (double)n),
                                              d_loss ? d_loss : T->loss);
        SAND_CUDA(cudaGetLastError(), "loss reduction");
    }
    if (d_grad) SAND_CUDA(cudaMemcpyAsync(d_grad, T->grad, T->np * 4, cudaMemcpyDeviceToDevice, s), "gradient copy");
    if (update) {
        T->step += 1;
        const double c1 = 1.0 / (1.0 - pow((double)T->b1, (double)T->step));
        const double c2 = 1.0 / (1.0 - pow((double)T->b2, (double)T->step));
        tr_adam_kernel<<<2 * T->num_sms, 256, 0, s>>>(T->params, T->grad, T->am, T->av, (int64_t)T->np, T->lr, T->b1,
                                                      T->b2, T->eps, (float)c1, (float)c2);
        SAND_CUDA(cudaGetLastError(), "Adam kernel");
    }
    return SAND_OK;
}

sand_status sand_trainer_params(sand_trainer T, float *h_params, size_t n_params) {
    if (!T || !h_params) {
        set_error("NULL trainer or output");
        return SAND_EINVAL;
    }
    if (n_params != T->np) {
        set_error("the model has %zu parameters, not %zu", T->np, n_params);
        return SAND_EINVAL;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(T->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(h_params, T->params, T->np * 4, cudaMemcpyDeviceToHost);
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) return cuda_fail(e, "parameter read-back");
    return SAND_OK;
}

sand_status sand_trainer_commit(sand_trainer T) {
    if (!T) {
        set_error("NULL trainer");
        return SAND_EINVAL;
    }
    std::vector<float> h(T->np);
    sand_status st = sand_trainer_params(T, h.data(), h.size());
    if (st) return st;
    return model_replace_params(T->m, h.data());
}

sand_status sand_trainer_status(sand_trainer T, void *stream) {
    if (!T) {
        set_error("NULL trainer");
        return SAND_EINVAL;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(T->device);
    unsigned v = 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(&v, T->status, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) return cuda_fail(e, "status read-back");
    if (v & 1u) {
        set_error("a bounded device-side wait of a training kernel gave up");
        return SAND_ETIMEOUT;
    }
    return SAND_OK;
}

sand_status sand_trainer_destroy(sand_trainer T) {
    if (!T) return SAND_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(T->device);
    cudaDeviceSynchronize();
    cudaFree(T->mem);
    if (prev >= 0) cudaSetDevice(prev);
    delete T;
    return SAND_OK;
}

}  // extern "C"
