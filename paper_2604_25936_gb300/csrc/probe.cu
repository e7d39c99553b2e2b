// Issue-rate probes for the roofline denominators of the epilogue pipes: float32 FMA
// (the tail dot products, bias and scale of every accumulator value) and the hardware
// sine of a radian argument (one per unit per row-layer of a sine network, Eq. 2).
// Each thread runs kProbeChains independent dependency chains so that issue, not
// latency, bounds the rate once a few warps share a scheduler.
#include "internal.cuh"

namespace sand {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;

__global__ void __launch_bounds__(kProbeThreads) probe_ffma_kernel(int iters, float *__restrict__ sink) {
    float a[kProbeChains];
    const float m = 1.0f - 1.0e-7f * (float)(threadIdx.x & 31);  // |m| < 1: the chains stay bounded
    const float c = 1.0e-7f;
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = 1.0f + 1.0e-3f * k + 1.0e-6f * threadIdx.x;
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) a[k] = fmaf(a[k], m, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) s += a[k];
    sink[(size_t)blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kProbeThreads) probe_sin_kernel(int iters, float *__restrict__ sink) {
    float a[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = 0.5f + 0.25f * k + 1.0e-4f * threadIdx.x;
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) a[k] = __sinf(a[k]) * 3.0f;  // stays within [-3, 3]
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) s += a[k];
    sink[(size_t)blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

}  // namespace sand

using namespace sand;

extern "C" {

sand_status sand_probe_rate(int kind, int device, int n_blocks, int iters, float *d_sink, void *stream) {
    if (kind != SAND_PROBE_FFMA && kind != SAND_PROBE_SIN) { set_error("unknown probe kind %d", kind); return SAND_EINVAL; }
    if (n_blocks <= 0 || n_blocks > (1 << 20) || iters <= 0) {
        set_error("n_blocks must be in 1..2^20 and iters > 0");
        return SAND_EINVAL;
    }
    if (!d_sink || (reinterpret_cast<uintptr_t>(d_sink) & 3)) { set_error("d_sink must be a 4-byte aligned device buffer"); return SAND_EINVAL; }
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
        set_error("cannot select device %d", device);
        return SAND_ECUDA;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (kind == SAND_PROBE_FFMA) probe_ffma_kernel<<<n_blocks, kProbeThreads, 0, s>>>(iters, d_sink);
    else probe_sin_kernel<<<n_blocks, kProbeThreads, 0, s>>>(iters, d_sink);
    const cudaError_t e = cudaGetLastError();
    cudaSetDevice(prev);
    if (e != cudaSuccess) { set_error("probe launch: %s", cudaGetErrorString(e)); return SAND_ECUDA; }
    return SAND_OK;
}

}  // extern "C"
