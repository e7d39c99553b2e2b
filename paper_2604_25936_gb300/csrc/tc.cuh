// Tensor-core (tcgen05) T-MLP path: packed weights and launcher.
#pragma once

#include <cuda.h>

#include "internal.cuh"

namespace sand {

struct TcModel {
    int packed_precision = -1;   // precision the packed buffers hold, -1 = none
    void *d_pack = nullptr;      // packed hidden-layer weights (fp16 / bf16, K-major rows)
    size_t pack_bytes = 0;
    void *host = nullptr;        // tensor map and kernel parameters
};

bool tc_supported(const sand_tmlp_desc &d, int precision);
sand_status tc_prepare(TcModel *tc, const sand_tmlp_desc &d, const float *params, int precision);
// all_tails (with full_depth): out[i * L + l - 1] = y_l for every layer l of every point.
// dyn_r > 0 (with full_depth): octree-free dynamic exit at |t_l| < dyn_r, exit layers to exit_out.
// grad: also dy/dx per point ([n][3], forward-mode tangents as three more rows per point).
// A 2-D TMA tensor map over rows of `inner` 16-bit elements (row pitch 2 inner bytes), boxes of
// box_inner x box_rows with the 128-byte swizzle (box_inner x 2 = 128 bytes: one swizzle span).
// False when the driver entry point or the encoding fails.
bool encode_u16_rows(CUtensorMap *map, const void *base, uint64_t inner, uint64_t rows, uint32_t box_inner,
                     uint32_t box_rows);
// The same over rows of `inner` float32 elements (box_inner x 4 = 128 bytes).
bool encode_f32_rows(CUtensorMap *map, const void *base, uint64_t inner, uint64_t rows, uint32_t box_inner,
                     uint32_t box_rows);

cudaError_t launch_tmlp_tc(const TcModel &tc, const TmlpDev &M, const float *pts, int64_t n, int full_depth, void *ws,
                           float *out, int num_sms, cudaStream_t s, int all_tails = 0, float dyn_r = 0.f,
                           uint8_t *exit_out = nullptr, float *grad = nullptr, uint64_t wait_ns = 0);
void tc_release(TcModel *tc);

}  // namespace sand
