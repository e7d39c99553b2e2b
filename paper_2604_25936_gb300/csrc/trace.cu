// Sphere tracing of the SAND SDF: rays march by the queried distance until they
// hit the surface, leave the domain or run out of steps; the input gradient
// (the surface normal direction) is evaluated at the hits.
//
// The march runs on the device without host round trips.  Each step:
//   query   SAND query (lookup, binning, T-MLP) of the active rays' points; the
//           point count lives in device memory (the grids are sized for n_rays)
//   march   t += y per active ray, or a final state (hit / left / out of steps / NaN);
//           writes a keep flag per active-list entry and a count per block
//   compact stable compaction of the kept entries (prefix of the block counts, then a
//           block scan), writing the next active list, its points and its count.
// The active list stays in ray order, so the result does not depend on timing.
#include "internal.cuh"

namespace sand {

constexpr int kTrThreads = 256;
constexpr int kTrItems = 8;
constexpr int kTrChunk = kTrThreads * kTrItems;  // active-list entries per block

// Parameter interval [t0, t1] of the ray inside [-1, 1]^3 (slab method), t0 >= 0.
__device__ __forceinline__ bool ray_box(float ox, float oy, float oz, float dx, float dy, float dz, float &t0,
                                        float &t1) {
    t0 = 0.f;
    t1 = INFINITY;
    const float o[3] = {ox, oy, oz}, d[3] = {dx, dy, dz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.f) {
            if (o[a] < -1.f || o[a] > 1.f) return false;
            continue;
        }
        const float inv = 1.f / d[a];
        float ta = (-1.f - o[a]) * inv, tb = (1.f - o[a]) * inv;
        if (ta > tb) { const float tmp = ta; ta = tb; tb = tmp; }
        t0 = fmaxf(t0, ta);
        t1 = fminf(t1, tb);
    }
    return t0 <= t1;
}

struct TraceRays {
    const float *orig;   // [3] shared origin, or [n][3] when per_ray
    const float *dir;    // [n][3]
    int per_ray;
    int64_t n;
    float *T;            // [n] ray parameter
    uint8_t *state;      // [n] sand_ray_state
    uint8_t *steps;      // [n] SDF queries made
};

__device__ __forceinline__ void ray_of(const TraceRays &R, int64_t r, float *o, float *d) {
    const float *po = R.per_ray ? R.orig + 3 * r : R.orig;
    o[0] = po[0]; o[1] = po[1]; o[2] = po[2];
    d[0] = R.dir[3 * r]; d[1] = R.dir[3 * r + 1]; d[2] = R.dir[3 * r + 2];
}

// Block-wide sum of one value per thread (every thread gets the total).
__device__ __forceinline__ uint32_t block_sum(uint32_t v, uint32_t *red) {
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    uint32_t t = 0;
    for (int w = 0; w < kTrThreads / 32; ++w) t += red[w];
    return t;
}

// Start of every ray: enter the domain (or miss it); the identity active list is flagged.
__global__ void __launch_bounds__(kTrThreads) trace_init_kernel(TraceRays R, uint8_t *flags, uint32_t *bcnt) {
    __shared__ uint32_t red[kTrThreads / 32];
    const int64_t c0 = (int64_t)blockIdx.x * kTrChunk;
    uint32_t kept = 0;
    for (int i = 0; i < kTrItems; ++i) {
        const int64_t r = c0 + i * kTrThreads + threadIdx.x;
        if (r >= R.n) break;
        float o[3], d[3], t0, t1;
        ray_of(R, r, o, d);
        const bool in = ray_box(o[0], o[1], o[2], d[0], d[1], d[2], t0, t1);
        R.T[r] = in ? t0 : 0.f;
        R.state[r] = in ? SAND_RAY_STEPS : SAND_RAY_MISS;
        R.steps[r] = 0;
        flags[r] = in ? 1 : 0;
        kept += in;
    }
    const uint32_t tot = block_sum(kept, red);
    if (threadIdx.x == 0) bcnt[blockIdx.x] = tot;
}

// One step for the active entries j < *cnt_in: ray r = act[j] moves by y = sdf[j].
__global__ void __launch_bounds__(kTrThreads)
trace_march_kernel(TraceRays R, const uint32_t *__restrict__ act, const float *__restrict__ sdf,
                   const uint32_t *__restrict__ cnt_in, int max_steps, float eps, uint8_t *flags, uint32_t *bcnt) {
    __shared__ uint32_t red[kTrThreads / 32];
    const int64_t n_act = *cnt_in;
    const int64_t c0 = (int64_t)blockIdx.x * kTrChunk;
    uint32_t kept = 0;
    for (int i = 0; i < kTrItems; ++i) {
        const int64_t j = c0 + i * kTrThreads + threadIdx.x;
        if (j >= n_act) break;
        const int64_t r = act[j];
        const float y = sdf[j];
        const int k = R.steps[r] + 1;
        R.steps[r] = (uint8_t)k;
        uint8_t st = SAND_RAY_STEPS;
        bool keep = false;
        if (isnan(y)) {
            st = SAND_RAY_NAN;
        } else if (fabsf(y) < eps) {
            st = SAND_RAY_HIT;
        } else {
            const float t = R.T[r] + y;
            R.T[r] = t;
            float o[3], d[3], t0, t1;
            ray_of(R, r, o, d);
            ray_box(o[0], o[1], o[2], d[0], d[1], d[2], t0, t1);
            if (t > t1 || t < t0) st = SAND_RAY_MISS;
            else if (k >= max_steps) st = SAND_RAY_STEPS;
            else keep = true;
        }
        R.state[r] = st;
        flags[j] = keep ? 1 : 0;
        kept += keep;
    }
    const uint32_t tot = block_sum(kept, red);
    if (threadIdx.x == 0) bcnt[blockIdx.x] = tot;
}

// Stable compaction of the flagged entries j < n_act (n_act = *cnt_in, or n_host when
// cnt_in is null; the list is the identity when act is null) into act_out / pts, and
// the count into *cnt_out.  Every block of the grid wrote bcnt[b] before this launch.
__global__ void __launch_bounds__(kTrThreads)
trace_compact_kernel(TraceRays R, const uint32_t *__restrict__ act, const uint32_t *__restrict__ cnt_in, int64_t n_host,
                     const uint8_t *__restrict__ flags, const uint32_t *__restrict__ bcnt, uint32_t *__restrict__ act_out,
                     float *__restrict__ pts, uint32_t *__restrict__ cnt_out) {
    __shared__ uint32_t red[kTrThreads / 32];
    __shared__ uint32_t wsum[kTrThreads / 32];
    const int64_t n_act = cnt_in ? (int64_t)*cnt_in : n_host;
    uint32_t before = 0;  // kept entries in the blocks before this one
    for (int b = threadIdx.x; b < (int)blockIdx.x; b += kTrThreads) before += bcnt[b];
    before = block_sum(before, red);
    const int64_t c0 = (int64_t)blockIdx.x * kTrChunk + (int64_t)threadIdx.x * kTrItems;  // 8 consecutive entries
    uint32_t mine = 0;
    uint8_t f[kTrItems];
#pragma unroll
    for (int i = 0; i < kTrItems; ++i) {
        f[i] = (c0 + i < n_act) ? flags[c0 + i] : 0;
        mine += f[i];
    }
    // exclusive scan of `mine` over the block (warp shuffles, then the warp totals)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = mine;
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += v;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    uint32_t wbefore = 0, total = 0;
    for (int w = 0; w < kTrThreads / 32; ++w) {
        if (w < warp) wbefore += wsum[w];
        total += wsum[w];
    }
    uint32_t pos = before + wbefore + inc - mine;
#pragma unroll
    for (int i = 0; i < kTrItems; ++i) {
        if (!f[i]) continue;
        const int64_t j = c0 + i;
        const int64_t r = act ? (int64_t)act[j] : j;
        float o[3], d[3];
        ray_of(R, r, o, d);
        const float t = R.T[r];
        act_out[pos] = (uint32_t)r;
        pts[3 * (int64_t)pos] = fmaf(t, d[0], o[0]);
        pts[3 * (int64_t)pos + 1] = fmaf(t, d[1], o[1]);
        pts[3 * (int64_t)pos + 2] = fmaf(t, d[2], o[2]);
        ++pos;
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *cnt_out = before + total;
}

// Flag the rays that hit (for the gradient pass).
__global__ void __launch_bounds__(kTrThreads) trace_hits_kernel(TraceRays R, uint8_t *flags, uint32_t *bcnt) {
    __shared__ uint32_t red[kTrThreads / 32];
    const int64_t c0 = (int64_t)blockIdx.x * kTrChunk;
    uint32_t kept = 0;
    for (int i = 0; i < kTrItems; ++i) {
        const int64_t r = c0 + i * kTrThreads + threadIdx.x;
        if (r >= R.n) break;
        const bool h = R.state[r] == SAND_RAY_HIT;
        flags[r] = h ? 1 : 0;
        kept += h;
    }
    const uint32_t tot = block_sum(kept, red);
    if (threadIdx.x == 0) bcnt[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kTrThreads)
trace_scatter_grad_kernel(const uint32_t *__restrict__ hits, const uint32_t *__restrict__ cnt,
                          const float *__restrict__ g, float *__restrict__ grad) {
    const int64_t n_hit = *cnt;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_hit; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = hits[j];
        grad[3 * r] = g[3 * j];
        grad[3 * r + 1] = g[3 * j + 1];
        grad[3 * r + 2] = g[3 * j + 2];
    }
}

struct TraceLayout {
    size_t T, state, steps, flags, act0, act1, bcnt, cnt, pts, sdf, g, ws, total;
};

static TraceLayout trace_layout(int64_t n, bool want_t, bool want_state, bool want_steps) {
    TraceLayout L{};
    const size_t np = (size_t)((n + kTrChunk - 1) / kTrChunk) * kTrChunk;  // whole blocks
    const int64_t blocks = (n + kTrChunk - 1) / kTrChunk;
    size_t o = 0;
    auto take = [&](size_t bytes) { const size_t at = o; o = align_up(o + bytes, 256); return at; };
    L.T = want_t ? (size_t)-1 : take(np * 4);
    L.state = want_state ? (size_t)-1 : take(np);
    L.steps = want_steps ? (size_t)-1 : take(np);
    L.flags = take(np);
    L.act0 = take(np * 4);
    L.act1 = take(np * 4);
    L.bcnt = take((size_t)blocks * 4 + 4);
    L.cnt = take(16);
    L.pts = take(np * 12);
    L.sdf = take(np * 4);
    L.g = take(np * 12);
    L.ws = take(ws_layout(n).total);
    L.total = o;
    return L;
}

}  // namespace sand

using namespace sand;

extern "C" {

size_t sand_trace_state_bytes(int64_t n_rays) {
    return n_rays < 0 ? 0 : trace_layout(n_rays, false, false, false).total;
}

sand_status sand_sphere_trace(sand_model m, const float *d_origin, int per_ray_origin, const float *d_dirs,
                              int64_t n_rays, const sand_trace_opts *topts, const sand_query_opts *qopts, float *d_t,
                              uint8_t *d_state, uint8_t *d_steps, float *d_grad, void *stream) {
    set_error("");
    if (!m) { set_error("NULL model"); return SAND_EINVAL; }
    if (n_rays < 0 || n_rays > 0x7fffffffLL) { set_error("n_rays outside 0..2^31-1"); return SAND_EINVAL; }
    if (n_rays == 0) return SAND_OK;
    if (!topts || !d_origin || !d_dirs) { set_error("NULL trace options, origin or directions"); return SAND_EINVAL; }
    if (topts->max_steps < 1 || topts->max_steps > 255) { set_error("max_steps outside 1..255"); return SAND_EINVAL; }
    if (!(topts->hit_eps > 0.f)) { set_error("hit_eps must be positive"); return SAND_EINVAL; }
    if (topts->poll_every < 0) { set_error("poll_every < 0"); return SAND_EINVAL; }
    if (!model_has_map(m)) { set_error("no depth map loaded"); return SAND_ENOMAP; }
    const uintptr_t mis = reinterpret_cast<uintptr_t>(d_origin) | reinterpret_cast<uintptr_t>(d_dirs) |
                          reinterpret_cast<uintptr_t>(d_t) | reinterpret_cast<uintptr_t>(d_grad);
    if (mis & 3) { set_error("device buffers must be 4-byte aligned"); return SAND_EINVAL; }
    sand_query_opts q{};
    if (qopts) q = *qopts;
    if (q.full_depth || q.d_exit_layers || q.d_workspace || q.stage_events || q.wait_limit_us) {
        set_error("trace queries take only precision and max_depth from the query options");
        return SAND_EINVAL;
    }
    int cur = 0;
    cudaGetDevice(&cur);
    const int dev = model_device(m);
    if (cur != dev && cudaSetDevice(dev) != cudaSuccess) { set_error("cannot select device %d", dev); return SAND_ECUDA; }
    struct Restore { int d; bool on; ~Restore() { if (on) cudaSetDevice(d); } } restore{cur, cur != dev};
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    const TraceLayout L = trace_layout(n_rays, d_t != nullptr, d_state != nullptr, d_steps != nullptr);
    void *buf = nullptr;
    sand_status st = model_trace_buffer(m, L.total, &buf);
    if (st) return st;
    char *b = static_cast<char *>(buf);
    TraceRays R{d_origin, d_dirs, per_ray_origin ? 1 : 0, n_rays,
                d_t ? d_t : reinterpret_cast<float *>(b + L.T),
                d_state ? d_state : reinterpret_cast<uint8_t *>(b + L.state),
                d_steps ? d_steps : reinterpret_cast<uint8_t *>(b + L.steps)};
    uint8_t *flags = reinterpret_cast<uint8_t *>(b + L.flags);
    uint32_t *act[2] = {reinterpret_cast<uint32_t *>(b + L.act0), reinterpret_cast<uint32_t *>(b + L.act1)};
    uint32_t *bcnt = reinterpret_cast<uint32_t *>(b + L.bcnt);
    uint32_t *cnt = reinterpret_cast<uint32_t *>(b + L.cnt);  // [0], [1] active lists, [2] hits
    float *pts = reinterpret_cast<float *>(b + L.pts);
    float *sdf = reinterpret_cast<float *>(b + L.sdf);
    float *g = reinterpret_cast<float *>(b + L.g);
    q.d_workspace = b + L.ws;
    q.workspace_bytes = ws_layout(n_rays).total;

    const int blocks = (int)((n_rays + kTrChunk - 1) / kTrChunk);
    if (d_grad) SAND_CUDA(cudaMemsetAsync(d_grad, 0, (size_t)n_rays * 12, s), "clear gradients");
    trace_init_kernel<<<blocks, kTrThreads, 0, s>>>(R, flags, bcnt);
    trace_compact_kernel<<<blocks, kTrThreads, 0, s>>>(R, nullptr, nullptr, n_rays, flags, bcnt, act[0], pts, cnt + 0);
    SAND_CUDA(cudaGetLastError(), "trace start");
    const int poll = topts->poll_every;
    for (int k = 0; k < topts->max_steps; ++k) {
        uint32_t *cin = cnt + (k & 1), *cout = cnt + ((k + 1) & 1);
        if (poll > 0 && k > 0 && k % poll == 0) {  // stop once no ray is active
            uint32_t h = 0;
            SAND_CUDA(cudaMemcpyAsync(&h, cin, 4, cudaMemcpyDeviceToHost, s), "read active count");
            SAND_CUDA(cudaStreamSynchronize(s), "stream synchronize");
            if (h == 0) break;
        }
        st = query_device_count(m, pts, n_rays, cin, sdf, nullptr, &q, s);
        if (st) return st;
        trace_march_kernel<<<blocks, kTrThreads, 0, s>>>(R, act[k & 1], sdf, cin, topts->max_steps, topts->hit_eps,
                                                         flags, bcnt);
        trace_compact_kernel<<<blocks, kTrThreads, 0, s>>>(R, act[k & 1], cin, 0, flags, bcnt, act[(k + 1) & 1], pts,
                                                           cout);
        SAND_CUDA(cudaGetLastError(), "trace step");
    }
    if (d_grad) {
        trace_hits_kernel<<<blocks, kTrThreads, 0, s>>>(R, flags, bcnt);
        trace_compact_kernel<<<blocks, kTrThreads, 0, s>>>(R, nullptr, nullptr, n_rays, flags, bcnt, act[0], pts, cnt + 2);
        SAND_CUDA(cudaGetLastError(), "gather hits");
        st = query_device_count(m, pts, n_rays, cnt + 2, sdf, g, &q, s);
        if (st) return st;
        int sg = blocks * 8;
        if (sg > 4096) sg = 4096;
        trace_scatter_grad_kernel<<<sg, kTrThreads, 0, s>>>(act[0], cnt + 2, g, d_grad);
        SAND_CUDA(cudaGetLastError(), "scatter gradients");
    }
    return SAND_OK;
}

}  // extern "C"
