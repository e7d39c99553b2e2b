// Internal declarations of libsand (not part of the C-ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include "sand.h"

namespace sand {

constexpr int kMaxLayers = 14;       // exit layers 1..14; count[15] of the stats counts NaN points
constexpr int kMaxWidth = 512;
constexpr int kLookupThreads = 256;
constexpr int kLookupChunk = 2048;   // points staged through shared memory per step
constexpr int kMaxLookupBlocks = 1216;
constexpr uint8_t kExitNaN = 0xFF;

// ---------------------------------------------------------------- device views
struct TmlpDev {
    int L, W, D, tail_kind, act, enc, m;
    float omega0;
    const float *B;                 // [m][3] Fourier matrix
    const float *WT[kMaxLayers];    // layer l (0-based): transposed weights [fan_in][W]
    const float *bias[kMaxLayers];  // [W]
    const float *tw;                // [L][2][W]
    const float *tb;                // [L][2]
};

// Device encodings of the depth map (lossless re-encodings of the octree at its finest level).
//   dense (levels <= kDenseMaxLevel): grid[R^3] exit layer per finest cell (x fastest), far[R^3]
//     the stored SDF per finest cell, or nullptr when the map has no far leaves;
//   bricks (deeper maps): one entry per cell of level - 3 (R/8 per axis, x fastest).  An entry
//     {0x80000000 | d, far bits} is a cell inside one leaf of exit layer d; an entry {b, f} points
//     to brick b: 8^3 exit layers (x fastest) at bricks[512 b ..], and, when any of them is 0,
//     their stored SDF values at far_blocks[512 f ..] (f = 0xFFFFFFFF: no far leaf in the brick).
constexpr int kDenseMaxLevel = 7;
constexpr int kMaxMapLevel = 10;
struct MapDev {
    const uint8_t *grid;
    const float *far;
    int level;            // R = 1 << level
    int n_layers;
    const uint2 *coarse;  // brick encoding (nullptr: dense)
    const uint8_t *bricks;
    const float *far_blocks;
};

// Workspace header, at offset 0 of every query workspace.
struct WsHeader {
    uint32_t tile_counter;
    uint32_t flags;
    uint32_t n_active;          // points with exit layer >= 1
    uint32_t n_blocks;          // lookup grid size used by the query
    uint32_t count[16];         // points per exit layer 0..14, [15] = NaN points
    uint32_t bin_start[16];     // first sorted row of exit layer d (rows sorted by descending d)
    uint32_t timeout_where;
    uint32_t pad[27];
};
static_assert(sizeof(WsHeader) <= 1024, "workspace header");

struct WsLayout {
    size_t header = 0, hist = 0, exit = 0, sorted = 0, total = 0;
};

constexpr size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

constexpr WsLayout ws_layout(int64_t n) {
    WsLayout w;
    w.header = 0;
    w.hist = 1024;
    w.exit = align_up(w.hist + sizeof(uint32_t) * 16 * kMaxLookupBlocks, 256);
    w.sorted = align_up(w.exit + (size_t)n, 256);
    w.total = align_up(w.sorted + (size_t)n * 16, 256);
    return w;
}

// ---------------------------------------------------------------- device math
// 2*pi split into three float32 parts (Cody & Waite 1980): C1 and C2 carry 16
// significant bits each, so k*C1 and k*C2 are exact for |k| <= 128.  Derived
// from 2*pi with 200-bit arithmetic; C1 + C2 + C3 differs from 2*pi by 4.9e-18.
#define SAND_TWO_PI_C1 6.2830810546875f
#define SAND_TWO_PI_C2 1.0425224900245667e-04f
#define SAND_TWO_PI_C3 2.430840251310684e-10f
#define SAND_INV_TWO_PI 0.15915493667125702f

// sin(a) for |a| <= ~800: reduce a to r in [-pi, pi] with the split above,
// then the hardware sine approximation on the reduced argument.
__device__ __forceinline__ float sin_reduced(float a) {
    float k = rintf(a * SAND_INV_TWO_PI);
    float r = fmaf(-k, SAND_TWO_PI_C1, a);
    r = fmaf(-k, SAND_TWO_PI_C2, r);
    r = fmaf(-k, SAND_TWO_PI_C3, r);
    return __sinf(r);
}
__device__ __forceinline__ void sincos_reduced(float a, float *s, float *c) {
    float k = rintf(a * SAND_INV_TWO_PI);
    float r = fmaf(-k, SAND_TWO_PI_C1, a);
    r = fmaf(-k, SAND_TWO_PI_C2, r);
    r = fmaf(-k, SAND_TWO_PI_C3, r);
    __sincosf(r, s, c);
}

// Fourier features gamma_k = sin(2 pi s_k), gamma_{m+k} = cos(2 pi s_k), s_k = B_k . x.
// s_k is accumulated as an unevaluated float32 pair (error-free products with
// FMA and Knuth's two-sum), reduced modulo 1 exactly, so the phase error does
// not grow with |s_k|.  Returns the reduced s in [-0.5, 0.5].
__device__ __forceinline__ float fourier_phase(const float *Bk, float x, float y, float z) {
    float p0 = Bk[0] * x, e0 = fmaf(Bk[0], x, -p0);
    float p1 = Bk[1] * y, e1 = fmaf(Bk[1], y, -p1);
    float p2 = Bk[2] * z, e2 = fmaf(Bk[2], z, -p2);
    float s = p0 + p1;
    float bv = s - p0;
    float err = (p0 - (s - bv)) + (p1 - bv);
    float s2 = s + p2;
    bv = s2 - s;
    err += (s - (s2 - bv)) + (p2 - bv);
    err += e0 + e1 + e2;
    float k = rintf(s2);
    return (s2 - k) + err;   // s2 - k is exact (Sterbenz) for |s2| < 2^23
}

// ---------------------------------------------------------------- host helpers
void set_error(const char *fmt, ...);
sand_status cuda_fail(cudaError_t e, const char *what);
// Return the status of a failed CUDA runtime call from the enclosing function.
#define SAND_CUDA(call, what)                              \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// Kernel launchers (stream-ordered, no host synchronisation).  With d_count set, the
// lookup and scatter grids are sized for n points but process min(n, *d_count).
cudaError_t launch_lookup(const MapDev &map, const float *pts, int64_t n, int max_depth, float *out, float *grad,
                          uint8_t *exit_layers, void *ws, cudaStream_t s, const uint32_t *d_count = nullptr);
cudaError_t launch_scatter(const float *pts, int64_t n, int n_layers, void *ws, cudaStream_t s,
                           const uint32_t *d_count = nullptr);
cudaError_t launch_tmlp_simt(const TmlpDev &M, const float *pts, int64_t n, int full_depth, void *ws,
                             float *out, float *grad, int num_sms, cudaStream_t s);
cudaError_t launch_init_header(void *ws, cudaStream_t s);

// Model facts for entry points outside api.cu.
int model_device(sand_model m);
bool model_has_map(sand_model m);
bool model_precision_supported(sand_model m, int precision);  // some kernel of the library takes it
bool model_precision_ready(sand_model m, int precision);  // device weights for `precision` exist already
sand_status model_prepare(sand_model m, int precision);   // pack device weights for `precision` (may allocate)
// A SAND query of min(n, *d_count) points whose count is produced on the device (buffers
// sized for n); opts->d_workspace must hold ws_layout(n).  Full-depth mode is not offered.
sand_status query_device_count(sand_model m, const float *d_points, int64_t n, const uint32_t *d_count, float *d_out,
                               float *d_grad, const sand_query_opts *opts, cudaStream_t s);
// y_1 .. y_L of n points (d_out [n][L]) on the tensor cores in `precision` (the model's workspace).
sand_status model_eval_all_tails(sand_model m, const float *d_pts, int64_t n, float *d_out, int precision,
                                 cudaStream_t s);
int model_layers(sand_model m);
// Grow-only device buffer owned by the model for the sphere tracer (stream-ordered reuse).
sand_status model_trace_buffer(sand_model m, size_t bytes, void **out);
// The model's shape, host copy of its float32 parameter block and device.
const sand_tmlp_desc &model_desc_ref(sand_model m);
const float *model_params(sand_model m);
size_t model_param_count(sand_model m);
// Replace the parameter block (same shape): the CUDA-core weights are re-uploaded and the packed
// tensor-core weights dropped (rebuilt by the next tensor-core query).  Synchronises the device.
sand_status model_replace_params(sand_model m, const float *h_params);

}  // namespace sand
