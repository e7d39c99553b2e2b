// sand_query_sdf_noalloc: a SAND query that allocates no device memory.
//
// Some callers cannot allocate device memory while they query: a host
// framework whose own pool owns the GPU's memory budget (a raw cudaMalloc
// beside it can push the process over that budget or fragment the pool), or a
// latency-critical serving loop where cudaMalloc's implicit device-wide
// synchronisation would stall work already queued on other streams.  This
// entry point takes the query's scratch from a fixed array in device memory
// instead of a caller workspace or the model's grown-on-demand workspace.
//
// The array, g_noalloc_scratch, is a file-scope __device__ variable sized for
// kNoAllocMaxPoints points.  Each GPU on which the library's module is loaded
// (with CUDA's lazy loading: on its first use on that GPU) holds it until the
// process exits.  In host code its name is only a host-side stand-in, so its
// device address is looked up once per device with cudaGetSymbolAddress (with
// that device current) on the first call on that device, and passed on.  That
// first call should therefore come before any stream capture.  All calls share
// the one array and leave their scratch in it; everything the query needs
// zeroed (the counters in the workspace header) is cleared by the query itself
// on its stream, but two calls that overlap on the GPU (different streams, no
// ordering) race on the array and corrupt each other's results.
#include <mutex>

#include "internal.cuh"

namespace sand {

constexpr int64_t kNoAllocMaxPoints = SAND_NOALLOC_MAX_POINTS;
constexpr size_t kNoAllocBytes = ws_layout(kNoAllocMaxPoints).total;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

static void *g_noalloc_addr[kNoAllocMaxDevices];
static std::mutex g_noalloc_mu;

}  // namespace sand

using namespace sand;

extern "C" sand_status sand_query_sdf_noalloc(sand_model m, const float *d_points, int64_t n, float *d_out,
                                              const sand_query_opts *opts, void *stream) {
    if (!m) {
        set_error("NULL model");
        return SAND_EINVAL;
    }
    if (n < 0 || n > kNoAllocMaxPoints) {
        set_error("n = %lld is outside 0..%lld, the most points the no-allocation scratch holds", (long long)n,
                  (long long)kNoAllocMaxPoints);
        return SAND_EINVAL;
    }
    if (n == 0) return SAND_OK;
    sand_query_opts o{};
    if (opts) o = *opts;
    if (o.d_workspace) {
        set_error("sand_query_sdf_noalloc uses its own static scratch; pass d_workspace = NULL");
        return SAND_EINVAL;
    }
    if (!model_precision_supported(m, o.precision)) {
        set_error("precision %d is not supported for this model", o.precision);
        return SAND_EUNSUPPORTED;
    }
    if (!model_precision_ready(m, o.precision)) {
        set_error("precision %d has no packed device weights now (a model keeps those of its most recent "
                  "tensor-core precision only); run one sand_query_sdf with it first (that call may allocate) "
                  "or use SAND_FP32_SIMT", o.precision);
        return SAND_EUNSUPPORTED;
    }
    const int dev = model_device(m);
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        set_error("device %d outside the 0..%d range this entry point tracks", dev, kNoAllocMaxDevices - 1);
        return SAND_EUNSUPPORTED;
    }
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            int prev = -1;
            cudaGetDevice(&prev);
            cudaError_t e = cudaSetDevice(dev);
            void *p = nullptr;
            if (e == cudaSuccess) e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (prev >= 0) cudaSetDevice(prev);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
            g_noalloc_addr[dev] = p;
        }
        scratch = g_noalloc_addr[dev];
    }
    o.d_workspace = scratch;
    o.workspace_bytes = kNoAllocBytes;
    return sand_query_sdf(m, d_points, n, d_out, &o, stream);
}
