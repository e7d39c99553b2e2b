// Host side of the tensor-core T-MLP path: weight packing, TMA tensor map,
// launch configuration.  The kernel is in tc_kernel.cuh; one translation unit
// per precision mode instantiates it (tc_inst_*.cu) so they build in parallel.
#include <cudaTypedefs.h>
#include <cuda_fp8.h>
#include <string.h>

#include <cmath>
#include <vector>

#include "tc.cuh"
#include "tc_kernel.cuh"

namespace sand {

static int mode_of(int precision) {
    switch (precision) {
        case SAND_FP32: return TC_SPLIT16;
        case SAND_FP16: return TC_F16;
        case SAND_BF16: return TC_BF16;
        case SAND_FP8: return TC_FP8;
        default: return -1;
    }
}

bool tc_supported(const sand_tmlp_desc &d, int precision) {
    if (mode_of(precision) < 0) return false;
    if (d.width != 64 && d.width != 128 && d.width != 256 && d.width != 336) return false;
    // width 336 in the float32 split: the accumulator (336 columns) plus the hi operand (168) fill TMEM, so the lo
    // operand goes to shared memory (kernel variant kAloVar), which serves raw-coordinate models only
    if (d.width == 336 && mode_of(precision) == TC_SPLIT16 && d.encoder != SAND_ENC_NONE) return false;
    if (d.encoder == SAND_ENC_FOURIER && d.in_dim != d.width) return false;
    // FP8 stores the activations unscaled, which holds for the sine's [-1, 1] only
    if (mode_of(precision) == TC_FP8 && d.activation == SAND_ACT_RELU) return false;  // |h| <= 1 only for sines
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

bool encode_f32_rows(CUtensorMap *map, const void *base, uint64_t inner, uint64_t rows, uint32_t box_inner,
                     uint32_t box_rows) {
    auto enc = encode_fn();
    if (!enc) return false;
    cuuint64_t gdim[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    cuuint64_t gstride[1] = {(cuuint64_t)inner * 4};
    cuuint32_t box[2] = {box_inner, box_rows};
    cuuint32_t estride[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(base), gdim, gstride, box, estride,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool encode_u16_rows(CUtensorMap *map, const void *base, uint64_t inner, uint64_t rows, uint32_t box_inner,
                     uint32_t box_rows) {
    auto enc = encode_fn();
    if (!enc) return false;
    cuuint64_t gdim[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    cuuint64_t gstride[1] = {(cuuint64_t)inner * 2};
    cuuint32_t box[2] = {box_inner, box_rows};
    cuuint32_t estride[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, const_cast<void *>(base), gdim, gstride, box, estride,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct TcPack {
    CUtensorMap map;
    TcParams P;
    int mode;
};

size_t tc_smem_bytes(const TcParams &P, int parts) {
    (void)parts;  // the A operand lives in TMEM (its lo part in shared memory when P.alo)
    const size_t alo = P.alo ? (size_t)((P.W + 63) / 64) * 16384 : 0;
    const bool mult = P.tail_kind == SAND_TAIL_MULT;
    const size_t consts = (size_t)4 * (mult ? 3 : 2) * P.L * P.W;          // per-layer constants
    const size_t w1 = P.l1_fold && !mult ? (size_t)16 * P.W : 0;           // raw-coordinate layer 1
    return 1024 /*alignment slack*/ + alo + (size_t)P.n_stages * P.stage_bytes + consts + w1 + kMiscBytes;
}

sand_status tc_prepare(TcModel *tc, const sand_tmlp_desc &d, const float *params, int precision) {
    const int mode = mode_of(precision);
    if (mode < 0 || !tc_supported(d, precision)) {
        set_error("precision %d not supported on the tensor-core path for this model", precision);
        return SAND_EUNSUPPORTED;
    }
    if (tc->packed_precision == precision && tc->d_pack) return SAND_OK;
    tc_release(tc);
    const int L = d.n_layers, W = d.width, D = d.in_dim, mf = d.n_freq;
    const bool sine = d.activation != SAND_ACT_RELU;  // SIREN or FINER: phase in radians
    // Layer 1 always runs on the tensor cores.  Fourier features feed it as a W-wide A
    // operand; raw coordinates feed one K = 16 MMA whose K slots hold the cross terms of a
    // three-part fp16 split of 256 x (exact for float32 x) and a two-part split of the
    // weights, which gives float32-class products (fold1).
    const int first = 1;
    const bool fold1 = d.encoder != SAND_ENC_FOURIER;
    const float x_scale = 256.f;  // keeps the smallest coordinate part out of the fp16 subnormals
    const int parts = mode == TC_SPLIT16 ? 2 : 1;
    const bool fp8 = mode == TC_FP8;
    const int eb = fp8 ? 1 : 2;                   // bytes per packed weight
    const int ups = fp8 ? 128 : 64;               // K-units per 128-byte weight row of a stage
    const int kpad = (W + ups - 1) / ups * ups;   // K padded with zero weights to whole stages
    const int n_mma = L - first + 1;
    const float *p = params;
    const float *B = nullptr;
    if (d.encoder == SAND_ENC_FOURIER) { B = p; p += (size_t)mf * 3; }
    const float *W1 = p; p += (size_t)W * D;
    const float *b1 = p; p += W;
    const float *Wh = p; p += (size_t)(L - 1) * W * W;
    const float *bh = p; p += (size_t)(L - 1) * W;
    const float *tw = p; p += (size_t)L * 2 * W;
    const float *tbias = p;
    const double turn = sine ? (double)d.omega0 : 1.0;  // omega0 folded into the constants: phase in radians

    // packed hidden-layer weights, rows [(li * parts + part) * W + unit][k]
    const size_t rows = (size_t)(n_mma > 0 ? n_mma : 1) * parts * W;
    std::vector<uint8_t> packed(rows * kpad * eb, 0);
    std::vector<float> c1(kMaxLayers, 1.f);
    for (int li = 0; li < n_mma; ++li) {
        const int l = first + li;
        const int K = l == 1 ? D : W;
        if (l == 1 && fold1) {
            // B row of unit j (fp16 bits, K = 16): [w_h x3 coords] x 3, [w_l x3] x 2, 0, against
            // A = [x_h, x_m, x_l, x_h, x_m] (three coordinates each), so the product sums
            // x_h w_h + x_m w_h + x_l w_h + x_h w_l + x_m w_l
            float amax = 0.f;
            for (size_t i = 0; i < (size_t)W * D; ++i) amax = fmaxf(amax, fabsf(W1[i]));
            float s = 1.f;
            if (amax > 0.f) {
                int e;
                frexpf(amax, &e);
                s = ldexpf(1.f, -e);
            }
            c1[0] = (float)(turn / ((double)s * x_scale));
            for (int j = 0; j < W; ++j) {
                uint16_t wh[3], wl[3];
                for (int k = 0; k < 3; ++k) {
                    const float w = W1[(size_t)j * 3 + k] * s;
                    const __half h = __float2half_rn(w);
                    const __half lo = __float2half_rn(w - __half2float(h));
                    memcpy(&wh[k], &h, 2);
                    memcpy(&wl[k], &lo, 2);
                }
                uint16_t row[16] = {wh[0], wh[1], wh[2], wh[0], wh[1], wh[2], wh[0], wh[1], wh[2],
                                    wl[0], wl[1], wl[2], wl[0], wl[1], wl[2], 0};
                memcpy(&packed[(size_t)j * kpad * eb], row, sizeof row);  // the first 32 bytes of the row
            }
            continue;
        }
        const float *Wl = l == 1 ? W1 : Wh + (size_t)(l - 2) * W * W;
        float amax = 0.f;
        for (size_t i = 0; i < (size_t)W * K; ++i) amax = fmaxf(amax, fabsf(Wl[i]));
        float s = 1.f;
        if (mode != TC_BF16 && amax > 0.f) {
            int e;
            frexpf(amax, &e);      // amax = f 2^e, f in [0.5, 1)
            // amax s in [0.5, 1) (fp16) or [128, 256) (e4m3, largest finite 448); a power of two, so exact
            s = ldexpf(1.f, fp8 ? 8 - e : -e);
        }
        c1[l - 1] = (float)(turn / (double)s);
        for (int nr = 0; nr < W; ++nr)
            for (int k = 0; k < K; ++k) {
                const float w = Wl[(size_t)nr * K + k] * s;
                const size_t at = ((size_t)(li * parts) * W + nr) * kpad + k;
                if (fp8) {
                    packed[at] = (uint8_t)__nv_cvt_float_to_fp8(w, __NV_SATFINITE, __NV_E4M3);
                    continue;
                }
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
                memcpy(&packed[at * 2], &hi, 2);
                if (parts == 2) memcpy(&packed[(at + (size_t)W * kpad) * 2], &lo, 2);
            }
    }
    // per-layer constants [L][3][W]: bias' (omega0 b for sine), tail a, tail b
    std::vector<float> cvec((size_t)L * 3 * W, 0.f), tbv((size_t)L * 2);
    for (int l = 1; l <= L; ++l) {
        const float *bl = l == 1 ? b1 : bh + (size_t)(l - 2) * W;
        for (int j = 0; j < W; ++j) {
            cvec[((size_t)(l - 1) * 3 + 0) * W + j] = (float)(turn * (double)bl[j]);
            cvec[((size_t)(l - 1) * 3 + 1) * W + j] = tw[((size_t)(l - 1) * 2 + 0) * W + j];
            cvec[((size_t)(l - 1) * 3 + 2) * W + j] = l >= 2 ? tw[((size_t)(l - 1) * 2 + 1) * W + j] : 0.f;
        }
        tbv[2 * (l - 1)] = tbias[2 * (l - 1)];
        tbv[2 * (l - 1) + 1] = tbias[2 * (l - 1) + 1];
    }
    const size_t off_c = (packed.size() + 255) / 256 * 256;
    const size_t off_tb = off_c + cvec.size() * 4;
    const size_t off_B = off_tb + tbv.size() * 4;
    // layer 1 of raw coordinates for the CUDA-core path of exit-layer-1 rows: omega0 (sine
    // families; 1 for ReLU) times (W1[j][0..2], b1[j]), each product rounded once to float32
    const size_t off_w1 = (off_B + (size_t)mf * 3 * 4 + 15) / 16 * 16;
    const size_t total = off_w1 + (size_t)W * 16 + 16;
    std::vector<uint8_t> blob(total, 0);
    if (fold1) {
        std::vector<float> w1p((size_t)W * 4);
        for (int j = 0; j < W; ++j) {
            for (int c = 0; c < 3; ++c) w1p[(size_t)j * 4 + c] = (float)(turn * (double)W1[(size_t)j * D + c]);
            w1p[(size_t)j * 4 + 3] = (float)(turn * (double)b1[j]);
        }
        memcpy(blob.data() + off_w1, w1p.data(), w1p.size() * 4);
    }
    memcpy(blob.data(), packed.data(), packed.size());
    memcpy(blob.data() + off_c, cvec.data(), cvec.size() * 4);
    memcpy(blob.data() + off_tb, tbv.data(), tbv.size() * 4);
    if (B) memcpy(blob.data() + off_B, B, (size_t)mf * 3 * 4);

    auto *pk = new TcPack();
    memset(pk, 0, sizeof(TcPack));
    uint8_t *dbuf = nullptr;
    if (cudaMalloc(&dbuf, total) != cudaSuccess) {
        cudaGetLastError();
        delete pk;
        set_error("cannot allocate packed weights");
        return SAND_ENOMEM;
    }
    if (cudaMemcpy(dbuf, blob.data(), total, cudaMemcpyHostToDevice) != cudaSuccess) {
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
    cuuint64_t gstride[1] = {(cuuint64_t)kpad * eb};
    const int box_rows = W <= 256 ? W : W / 2;
    cuuint32_t box[2] = {(cuuint32_t)ups, (cuuint32_t)box_rows};  // 128 bytes per row: the swizzle span
    cuuint32_t estride[2] = {1, 1};
    CUresult cr = enc(&pk->map, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, dbuf, gdim,
                      gstride, box, estride,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) {
        cudaFree(dbuf);
        delete pk;
        set_error("cuTensorMapEncodeTiled failed (%d)", (int)cr);
        return SAND_ECUDA;
    }
    TcParams &P = pk->P;
    P.L = L; P.W = W; P.D = fold1 ? 16 : D; P.l1_fold = fold1 ? 1 : 0; P.x_scale = x_scale; P.tail_kind = d.tail_kind; P.act = d.activation; P.enc = d.encoder; P.m = mf;
    P.first_mma = first;
    P.finer_k = d.activation == SAND_ACT_FINER ? (float)(1.0 / (double)d.omega0) : 0.f;
    P.kpad = kpad;
    P.alo = (mode == TC_SPLIT16 && W > 256) ? 1 : 0;
    // hi and lo of one K-block, or two K-blocks of the one-part modes; with A_lo in shared memory one part
    P.stage_bytes = (P.alo ? 1u : 2u) * (uint32_t)W * 128u;
    P.box_rows = box_rows;
    P.n_split = W <= 256 ? W : 176;
    {   // accumulator (W columns) + A_hi (W/2; FP8: ceil32(W)/4) [+ A_lo (W/2)], rounded up to a power of two
        const uint32_t a_cols = fp8 ? (uint32_t)((W + 31) / 32 * 8) : (uint32_t)(W / 2);
        uint32_t need = (uint32_t)W + (uint32_t)(P.alo ? 1 : parts) * a_cols, cols = 32;
        while (cols < need) cols <<= 1;
        P.tmem_cols = cols;
    }
    for (int l = 0; l < kMaxLayers; ++l) P.c1[l] = c1[l];
    P.cvec = reinterpret_cast<const float *>(dbuf + off_c);
    P.tb = reinterpret_cast<const float *>(dbuf + off_tb);
    P.B = B ? reinterpret_cast<const float *>(dbuf + off_B) : nullptr;
    P.w1p = reinterpret_cast<const float4 *>(dbuf + off_w1);
    P.cc = fold1 ? 1 : 0;
    P.n_stages = 1;
    const size_t fixed = tc_smem_bytes(P, parts) - P.stage_bytes;
    int stages = (int)((kSmemBudget - (long)fixed) / (long)P.stage_bytes);
    if (stages > kMaxStages) stages = kMaxStages;
    if (stages < 2) {
        cudaFree(dbuf);
        delete pk;
        set_error("shared memory too small for width %d", W);
        return SAND_EUNSUPPORTED;
    }
    P.n_stages = stages;
    pk->mode = mode;
    tc->d_pack = dbuf;
    tc->pack_bytes = total;
    tc->host = pk;
    tc->packed_precision = precision;
    return SAND_OK;
}

cudaError_t launch_tmlp_tc(const TcModel &tc, const TmlpDev &M, const float *pts, int64_t n, int full_depth, void *ws,
                           float *out, int num_sms, cudaStream_t s, int all_tails, float dyn_r, uint8_t *exit_out,
                           float *grad, uint64_t wait_ns) {
    (void)M;
    TcPack *pk = static_cast<TcPack *>(tc.host);
    if (!pk) return cudaErrorInvalidValue;
    TcParams P = pk->P;
    P.all_tails = all_tails && full_depth ? 1 : 0;
    P.dyn_r = full_depth && !P.all_tails ? dyn_r : 0.f;
    P.exit_out = P.dyn_r > 0.f ? exit_out : nullptr;
    P.grad = P.all_tails || P.dyn_r > 0.f ? nullptr : grad;
    P.wait_ns = wait_ns ? wait_ns : kTimeoutNs;
    WsLayout Lw = ws_layout(full_depth ? 0 : n);
    char *base = static_cast<char *>(ws);
    WsHeader *hdr = reinterpret_cast<WsHeader *>(base);
    const float4 *sorted = full_depth ? nullptr : reinterpret_cast<const float4 *>(base + Lw.sorted);
    const int parts = pk->mode == TC_SPLIT16 ? 2 : 1;
    const size_t smem = tc_smem_bytes(P, parts);
    const int64_t ppt = P.grad ? kTileM / 4 : kTileM;  // points per tile (gradient: 4 rows per point)
    const int64_t tiles = (n + ppt - 1) / ppt;
    int grid = num_sms;
    if (tiles < grid) grid = (int)(tiles > 0 ? tiles : 1);
    const int var = (P.grad ? 2 : (P.all_tails || P.dyn_r > 0.f) ? 1 : (!full_depth && P.cc) ? 3 : 0) |
                    (P.alo ? kAloVar : 0);
#define SAND_ARGS pk->map, P, P.act, P.tail_kind, pts, sorted, hdr, n, full_depth, out, grid, smem, s
    if (pk->mode == TC_SPLIT16 && (var & kAloVar)) {
        switch (var & 3) {
            case 3: return launch_tc_mode<TC_SPLIT16, 7>(SAND_ARGS);
            case 2: return launch_tc_mode<TC_SPLIT16, 6>(SAND_ARGS);
            case 1: return launch_tc_mode<TC_SPLIT16, 5>(SAND_ARGS);
            default: return launch_tc_mode<TC_SPLIT16, 4>(SAND_ARGS);
        }
    }
#undef SAND_ARGS
#define SAND_LAUNCH(M)                                                                                                  \
    (var == 3   ? launch_tc_mode<M, 3>(pk->map, P, P.act, P.tail_kind, pts, sorted, hdr, n, full_depth, out, grid, smem, s) \
     : var == 2 ? launch_tc_mode<M, 2>(pk->map, P, P.act, P.tail_kind, pts, sorted, hdr, n, full_depth, out, grid, smem, s) \
     : var == 1 ? launch_tc_mode<M, 1>(pk->map, P, P.act, P.tail_kind, pts, sorted, hdr, n, full_depth, out, grid, smem, s) \
                : launch_tc_mode<M, 0>(pk->map, P, P.act, P.tail_kind, pts, sorted, hdr, n, full_depth, out, grid, smem, s))
    switch (pk->mode) {
        case TC_SPLIT16: return SAND_LAUNCH(TC_SPLIT16);
        case TC_F16: return SAND_LAUNCH(TC_F16);
        case TC_FP8: return SAND_LAUNCH(TC_FP8);
        default: return SAND_LAUNCH(TC_BF16);
    }
#undef SAND_LAUNCH
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
