// C-ABI of libsand: model and depth-map loading, workspace handling and the
// query entry points (declared and documented in include/sand.h).
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <new>
#include <vector>

#include "internal.cuh"
#include "tc.cuh"

struct sand_model_s {
    int device = 0;
    int num_sms = 0;
    sand_tmlp_desc desc{};
    std::vector<float> params;        // host copy of the float32 master parameters
    float *d_simt = nullptr;          // transposed float32 weights for the CUDA-core kernel
    sand::TmlpDev simt{};
    sand::TcModel tc{};               // packed tensor-core weights (per precision, built lazily)
    uint8_t *d_grid = nullptr;        // dense exit-layer grid
    float *d_far = nullptr;           // dense far-value grid (only when the map has far leaves)
    uint2 *d_coarse = nullptr;        // brick encoding of deeper maps: coarse table, bricks, far blocks
    uint8_t *d_bricks = nullptr;
    float *d_farblk = nullptr;
    size_t map_bytes = 0;             // device bytes of the map's encoding
    int map_level = -1;
    void *d_ws = nullptr;             // default workspace
    size_t ws_bytes = 0;
    float *d_stage = nullptr;         // staging for host-memory queries: points then outputs
    size_t stage_bytes = 0;
    cudaStream_t copy_in = nullptr;   // host-memory queries: the copy streams of the chunk pipeline
    cudaStream_t copy_out = nullptr;
    void *d_trace = nullptr;          // sphere-tracer state (rays, active lists, points, workspace)
    size_t trace_bytes = 0;
};

namespace sand {

static thread_local std::string g_err;

void set_error(const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}

sand_status cuda_fail(cudaError_t e, const char *what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return SAND_ECUDA;
}

struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};


static size_t param_count(const sand_tmlp_desc &d) {
    size_t L = d.n_layers, W = d.width, D = d.in_dim, m = d.n_freq;
    size_t n = W * D + W + (L - 1) * W * W + (L - 1) * W + L * 2 * W + L * 2;
    if (d.encoder == SAND_ENC_FOURIER) n += m * 3;
    return n;
}

static sand_status validate_desc(const sand_tmlp_desc &d) {
    if (d.n_layers < 1 || d.n_layers > kMaxLayers) { set_error("n_layers %d outside 1..%d", d.n_layers, kMaxLayers); return SAND_EFORMAT; }
    if (d.width < 1 || d.width > kMaxWidth) { set_error("width %d outside 1..%d", d.width, kMaxWidth); return SAND_EFORMAT; }
    if (d.tail_kind != SAND_TAIL_LINEAR && d.tail_kind != SAND_TAIL_MULT) { set_error("bad tail_kind %d", d.tail_kind); return SAND_EFORMAT; }
    if (d.activation != SAND_ACT_SINE && d.activation != SAND_ACT_RELU && d.activation != SAND_ACT_FINER) { set_error("bad activation %d", d.activation); return SAND_EFORMAT; }
    if (d.encoder == SAND_ENC_FOURIER) {
        if (d.n_freq < 1 || d.in_dim != 2 * d.n_freq || d.in_dim > kMaxWidth) { set_error("Fourier encoder needs in_dim = 2 n_freq <= %d", kMaxWidth); return SAND_EFORMAT; }
    } else if (d.encoder == SAND_ENC_NONE) {
        if (d.in_dim != 3) { set_error("in_dim must be 3 without an encoder"); return SAND_EFORMAT; }
    } else {
        set_error("bad encoder %d", d.encoder);
        return SAND_EFORMAT;
    }
    if (!(d.omega0 > 0.f) || !(d.omega0 < 1e4f)) { set_error("omega0 out of range"); return SAND_EFORMAT; }
    return SAND_OK;
}

// Pack the CUDA-core layout: per layer the transposed weights [fan_in][W] and biases.
static sand_status pack_simt(sand_model_s *m) {
    const sand_tmlp_desc &d = m->desc;
    const int L = d.n_layers, W = d.width, D = d.in_dim, mf = d.n_freq;
    const float *p = m->params.data();
    const float *B = nullptr;
    if (d.encoder == SAND_ENC_FOURIER) { B = p; p += (size_t)mf * 3; }
    const float *W1 = p; p += (size_t)W * D;
    const float *b1 = p; p += W;
    const float *Wh = p; p += (size_t)(L - 1) * W * W;
    const float *bh = p; p += (size_t)(L - 1) * W;
    const float *tw = p; p += (size_t)L * 2 * W;
    const float *tb = p;
    std::vector<float> buf;
    std::vector<size_t> off_WT(L), off_b(L);
    size_t off_B = 0, off_tw, off_tb;
    auto push = [&](size_t n) { size_t o = buf.size(); buf.resize(o + ((n + 63) / 64) * 64, 0.f); return o; };
    if (B) { off_B = push((size_t)mf * 3); memcpy(&buf[off_B], B, sizeof(float) * mf * 3); }
    for (int l = 0; l < L; ++l) {
        const int K = l == 0 ? D : W;
        const float *Wl = l == 0 ? W1 : Wh + (size_t)(l - 1) * W * W;
        off_WT[l] = push((size_t)K * W);
        for (int j = 0; j < W; ++j)
            for (int k = 0; k < K; ++k) buf[off_WT[l] + (size_t)k * W + j] = Wl[(size_t)j * K + k];
        off_b[l] = push(W);
        memcpy(&buf[off_b[l]], l == 0 ? b1 : bh + (size_t)(l - 1) * W, sizeof(float) * W);
    }
    off_tw = push((size_t)L * 2 * W);
    memcpy(&buf[off_tw], tw, sizeof(float) * L * 2 * W);
    off_tb = push((size_t)L * 2);
    memcpy(&buf[off_tb], tb, sizeof(float) * L * 2);
    SAND_CUDA(cudaMalloc(&m->d_simt, sizeof(float) * buf.size()), "cudaMalloc(weights)");
    SAND_CUDA(cudaMemcpy(m->d_simt, buf.data(), sizeof(float) * buf.size(), cudaMemcpyHostToDevice), "cudaMemcpy(weights)");
    TmlpDev &M = m->simt;
    M.L = L; M.W = W; M.D = D; M.tail_kind = d.tail_kind; M.act = d.activation; M.enc = d.encoder; M.m = mf;
    M.omega0 = d.omega0;
    M.B = B ? m->d_simt + off_B : nullptr;
    for (int l = 0; l < kMaxLayers; ++l) {
        M.WT[l] = l < L ? m->d_simt + off_WT[l] : nullptr;
        M.bias[l] = l < L ? m->d_simt + off_b[l] : nullptr;
    }
    M.tw = m->d_simt + off_tw;
    M.tb = m->d_simt + off_tb;
    return SAND_OK;
}

static void release(sand_model_s *m) {
    if (!m) return;
    cudaFree(m->d_simt);
    tc_release(&m->tc);
    cudaFree(m->d_grid);
    cudaFree(m->d_far);
    cudaFree(m->d_coarse);
    cudaFree(m->d_bricks);
    cudaFree(m->d_farblk);
    cudaFree(m->d_ws);
    cudaFree(m->d_stage);
    cudaFree(m->d_trace);
    if (m->copy_in) cudaStreamDestroy(m->copy_in);
    if (m->copy_out) cudaStreamDestroy(m->copy_out);
    m->copy_in = m->copy_out = nullptr;
}

static sand_status ensure_workspace(sand_model_s *m, int64_t n, bool grad, void **ws, size_t *bytes) {
    (void)grad;
    size_t need = ws_layout(n).total;
    if (m->ws_bytes < need) {
        cudaFree(m->d_ws);
        m->d_ws = nullptr;
        m->ws_bytes = 0;
        if (cudaMalloc(&m->d_ws, need) != cudaSuccess) {
            cudaGetLastError();
            set_error("cannot allocate a %zu-byte workspace", need);
            return SAND_ENOMEM;
        }
        m->ws_bytes = need;
    }
    *ws = m->d_ws;
    *bytes = m->ws_bytes;
    return SAND_OK;
}

// Fill the dense grid from the octree (iterative descent; validates the tree).
static sand_status densify(const sand_depth_map_desc &d, const int32_t *child, const uint8_t *depth, const float *far,
                           int model_layers, std::vector<uint8_t> &grid, std::vector<float> &fgrid, bool &has_far) {
    const int ML = d.max_level;
    const int64_t R = (int64_t)1 << ML;
    grid.assign((size_t)(R * R * R), 0);
    has_far = false;
    for (int i = 0; i < d.n_nodes; ++i)
        if (child[i] < 0 && depth[i] == 0) { has_far = true; break; }
    if (has_far) fgrid.assign((size_t)(R * R * R), 0.f);
    struct Item { int32_t node; int level; int64_t cx, cy, cz; };
    std::vector<Item> stack;
    stack.push_back({0, 0, 0, 0, 0});
    int64_t visited = 0;
    while (!stack.empty()) {
        Item it = stack.back();
        stack.pop_back();
        if (++visited > d.n_nodes) { set_error("octree has a cycle or shared children"); return SAND_EFORMAT; }
        const int32_t c = child[it.node];
        if (c >= 0) {
            if (it.level >= ML) { set_error("node %d below max_level %d", it.node, ML); return SAND_EFORMAT; }
            if ((int64_t)c + 8 > d.n_nodes || c <= it.node) { set_error("bad child index %d at node %d", c, it.node); return SAND_EFORMAT; }
            for (int o = 0; o < 8; ++o)
                stack.push_back({c + o, it.level + 1, 2 * it.cx + (o & 1), 2 * it.cy + ((o >> 1) & 1), 2 * it.cz + ((o >> 2) & 1)});
            continue;
        }
        const int dv = depth[it.node];
        if (dv > d.n_layers || dv > model_layers) { set_error("leaf %d exit layer %d exceeds %d layers", it.node, dv, model_layers); return SAND_EFORMAT; }
        const int64_t s = (int64_t)1 << (ML - it.level);
        for (int64_t z = it.cz * s; z < (it.cz + 1) * s; ++z)
            for (int64_t y = it.cy * s; y < (it.cy + 1) * s; ++y) {
                const size_t row = (size_t)((z * R + y) * R);
                memset(&grid[row + it.cx * s], dv, (size_t)s);
                if (has_far)
                    for (int64_t x = it.cx * s; x < (it.cx + 1) * s; ++x) fgrid[row + x] = far[it.node];
            }
    }
    return SAND_OK;
}

// Brick encoding of a map deeper than kDenseMaxLevel (iterative descent; validates the tree like
// densify): leaves at or above the coarse level (max_level - 3) fill coarse entries directly;
// a node at the coarse level with children becomes a brick of 8^3 finest cells.
static sand_status brickify(const sand_depth_map_desc &d, const int32_t *child, const uint8_t *depth, const float *far,
                            int model_layers, std::vector<uint2> &coarse, std::vector<uint8_t> &bricks,
                            std::vector<float> &farblk) {
    const int ML = d.max_level, CL = ML - 3;
    const int64_t Rc = (int64_t)1 << CL;
    coarse.assign((size_t)(Rc * Rc * Rc), make_uint2(0x80000000u, 0u));
    bricks.clear();
    farblk.clear();
    struct Item { int32_t node; int level; int64_t cx, cy, cz; };
    std::vector<Item> stack, sub;
    stack.push_back({0, 0, 0, 0, 0});
    int64_t visited = 0;
    auto check_node = [&](const Item &it, int32_t c) -> sand_status {
        if (++visited > d.n_nodes) { set_error("octree has a cycle or shared children"); return SAND_EFORMAT; }
        if (c >= 0) {
            if (it.level >= ML) { set_error("node %d below max_level %d", it.node, ML); return SAND_EFORMAT; }
            if ((int64_t)c + 8 > d.n_nodes || c <= it.node) { set_error("bad child index %d at node %d", c, it.node); return SAND_EFORMAT; }
        } else {
            const int dv = depth[it.node];
            if (dv > d.n_layers || dv > model_layers) { set_error("leaf %d exit layer %d exceeds %d layers", it.node, dv, model_layers); return SAND_EFORMAT; }
        }
        return SAND_OK;
    };
    while (!stack.empty()) {
        const Item it = stack.back();
        stack.pop_back();
        const int32_t c = child[it.node];
        sand_status st = check_node(it, c);
        if (st) return st;
        if (c < 0) {  // a leaf covering (2^(CL - level))^3 coarse cells
            uint32_t fbits;
            memcpy(&fbits, &far[it.node], 4);
            const int64_t s = (int64_t)1 << (CL - it.level);
            for (int64_t z = it.cz * s; z < (it.cz + 1) * s; ++z)
                for (int64_t y = it.cy * s; y < (it.cy + 1) * s; ++y)
                    for (int64_t x = it.cx * s; x < (it.cx + 1) * s; ++x)
                        coarse[(size_t)((z * Rc + y) * Rc + x)] = make_uint2(0x80000000u | depth[it.node], fbits);
            continue;
        }
        if (it.level < CL) {
            for (int o = 0; o < 8; ++o)
                stack.push_back({c + o, it.level + 1, 2 * it.cx + (o & 1), 2 * it.cy + ((o >> 1) & 1), 2 * it.cz + ((o >> 2) & 1)});
            continue;
        }
        // a brick: the subtree below this coarse cell, at the finest level (8 cells per axis)
        const uint32_t b = (uint32_t)(bricks.size() / 512);
        bricks.resize(bricks.size() + 512, 0);
        uint32_t fb = 0xFFFFFFFFu;
        sub.clear();
        for (int o = 0; o < 8; ++o) sub.push_back({c + o, it.level + 1, o & 1, (o >> 1) & 1, (o >> 2) & 1});
        while (!sub.empty()) {
            const Item s2 = sub.back();
            sub.pop_back();
            const int32_t c2 = child[s2.node];
            st = check_node(s2, c2);
            if (st) return st;
            if (c2 >= 0) {
                for (int o = 0; o < 8; ++o)
                    sub.push_back({c2 + o, s2.level + 1, 2 * s2.cx + (o & 1), 2 * s2.cy + ((o >> 1) & 1), 2 * s2.cz + ((o >> 2) & 1)});
                continue;
            }
            const int dv = depth[s2.node];
            if (dv == 0 && fb == 0xFFFFFFFFu) {
                fb = (uint32_t)(farblk.size() / 512);
                farblk.resize(farblk.size() + 512, 0.f);
            }
            const int64_t s = (int64_t)1 << (ML - s2.level);
            for (int64_t z = s2.cz * s; z < (s2.cz + 1) * s; ++z)
                for (int64_t y = s2.cy * s; y < (s2.cy + 1) * s; ++y)
                    for (int64_t x = s2.cx * s; x < (s2.cx + 1) * s; ++x) {
                        const size_t local = (size_t)((z * 8 + y) * 8 + x);
                        bricks[(size_t)b * 512 + local] = (uint8_t)dv;
                        if (dv == 0) farblk[(size_t)fb * 512 + local] = far[s2.node];
                    }
        }
        coarse[(size_t)((it.cz * Rc + it.cy) * Rc + it.cx)] = make_uint2(b, fb);
    }
    return SAND_OK;
}

static sand_status model_precheck(sand_model m) {
    if (!m) { set_error("NULL model"); return SAND_EINVAL; }
    return SAND_OK;
}

int model_device(sand_model m) { return m->device; }
int model_layers(sand_model m) { return m->desc.n_layers; }
bool model_has_map(sand_model m) { return m->map_level >= 0; }
bool model_precision_supported(sand_model m, int precision) {
    return precision == SAND_FP32_SIMT || tc_supported(m->desc, precision);
}
bool model_precision_ready(sand_model m, int precision) {
    if (precision == SAND_FP32_SIMT) return true;
    return m->tc.packed_precision == precision && m->tc.d_pack != nullptr;
}

sand_status model_prepare(sand_model m, int precision) {
    if (precision == SAND_FP32_SIMT) return SAND_OK;
    if (!tc_supported(m->desc, precision)) {
        set_error("precision %d is not supported for this model on the tensor-core path", precision);
        return SAND_EUNSUPPORTED;
    }
    DeviceGuard g(m->device);
    return tc_prepare(&m->tc, m->desc, m->params.data(), precision);
}

}  // namespace sand

using namespace sand;

extern "C" {

const char *sand_last_error(void) { return g_err.c_str(); }

sand_status sand_load_tmlp_mem(const sand_tmlp_desc *desc, const float *h_params, size_t n_params, int device,
                               sand_model *out) {
    g_err.clear();
    if (!desc || !h_params || !out) { set_error("NULL argument"); return SAND_EINVAL; }
    *out = nullptr;
    sand_status st = validate_desc(*desc);
    if (st) return st;
    if (n_params != param_count(*desc)) {
        set_error("parameter block has %zu floats, the descriptor implies %zu", n_params, param_count(*desc));
        return SAND_EFORMAT;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        set_error("CUDA device %d not available (%d devices)", device, ndev);
        return SAND_EUNSUPPORTED;
    }
    DeviceGuard g(device);
    auto *m = new sand_model_s();
    m->device = device;
    m->desc = *desc;
    m->params.assign(h_params, h_params + n_params);
    cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, device);
    st = pack_simt(m);
    if (st) { release(m); delete m; return st; }
    *out = m;
    return SAND_OK;
}

// Bytes from the current position of f to its end (-1 if unknown): a size field read from a
// file is checked against this before anything is allocated for it.
static long long bytes_left(FILE *f) {
    const long at = ftell(f);
    if (at < 0 || fseek(f, 0, SEEK_END) != 0) return -1;
    const long end = ftell(f);
    if (end < 0 || fseek(f, at, SEEK_SET) != 0) return -1;
    return (long long)end - (long long)at;
}

sand_status sand_load_tmlp(const char *path, int device, sand_model *out) {
    g_err.clear();
    if (!path || !out) { set_error("NULL argument"); return SAND_EINVAL; }
    FILE *f = fopen(path, "rb");
    if (!f) { set_error("cannot open %s", path); return SAND_EINVAL; }
    char magic[4];
    uint32_t ver;
    int32_t h[7];
    float w0;
    uint64_t np;
    bool ok = fread(magic, 1, 4, f) == 4 && memcmp(magic, "TMLP", 4) == 0 && fread(&ver, 4, 1, f) == 1 && ver == 1 &&
              fread(h, 4, 7, f) == 7 && fread(&w0, 4, 1, f) == 1 && fread(&np, 8, 1, f) == 1 && np < (1ull << 31);
    ok = ok && bytes_left(f) >= (long long)np * 4;  // the parameter block is there in full
    std::vector<float> p;
    if (ok) {
        try {
            p.resize(np);
        } catch (const std::bad_alloc &) {
            fclose(f);
            set_error("%s: cannot hold %llu parameters in host memory", path, (unsigned long long)np);
            return SAND_ENOMEM;
        }
        ok = fread(p.data(), 4, np, f) == np;
    }
    fclose(f);
    if (!ok) { set_error("%s: not a version-1 TMLP model file (or truncated)", path); return SAND_EFORMAT; }
    sand_tmlp_desc d{h[0], h[1], h[2], h[3], h[4], h[5], h[6], w0};
    return sand_load_tmlp_mem(&d, p.data(), p.size(), device, out);
}

sand_status sand_load_depth_map_mem(sand_model m, const sand_depth_map_desc *desc, const int32_t *h_child,
                                    const uint8_t *h_depth, const float *h_far) {
    g_err.clear();
    sand_status st = model_precheck(m);
    if (st) return st;
    if (!desc || !h_child || !h_depth || !h_far) { set_error("NULL argument"); return SAND_EINVAL; }
    if (desc->max_level < 0 || desc->max_level > kMaxMapLevel) {
        set_error("max_level %d outside 0..%d", desc->max_level, kMaxMapLevel);
        return SAND_EUNSUPPORTED;
    }
    if (desc->n_nodes < 1) { set_error("empty octree"); return SAND_EFORMAT; }
    const bool dense = desc->max_level <= kDenseMaxLevel;
    std::vector<uint8_t> grid;
    std::vector<float> fgrid;
    std::vector<uint2> coarse;
    bool has_far = false;
    if (dense) st = densify(*desc, h_child, h_depth, h_far, m->desc.n_layers, grid, fgrid, has_far);
    else st = brickify(*desc, h_child, h_depth, h_far, m->desc.n_layers, coarse, grid, fgrid);
    if (st) return st;
    DeviceGuard g(m->device);
    for (void *p : {(void *)m->d_grid, (void *)m->d_far, (void *)m->d_coarse, (void *)m->d_bricks, (void *)m->d_farblk})
        cudaFree(p);
    m->d_grid = nullptr;
    m->d_far = nullptr;
    m->d_coarse = nullptr;
    m->d_bricks = nullptr;
    m->d_farblk = nullptr;
    m->map_level = -1;
    m->map_bytes = 0;
    auto upload = [&](void **dst, const void *src, size_t bytes, const char *what) -> sand_status {
        if (!bytes) return SAND_OK;
        SAND_CUDA(cudaMalloc(dst, bytes), what);
        SAND_CUDA(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice), what);
        m->map_bytes += bytes;
        return SAND_OK;
    };
    if (dense) {
        st = upload((void **)&m->d_grid, grid.data(), grid.size(), "depth grid upload");
        if (!st && has_far) st = upload((void **)&m->d_far, fgrid.data(), fgrid.size() * sizeof(float), "far grid upload");
    } else {
        st = upload((void **)&m->d_coarse, coarse.data(), coarse.size() * sizeof(uint2), "coarse table upload");
        if (!st) st = upload((void **)&m->d_bricks, grid.data(), grid.size(), "brick upload");
        if (!st) st = upload((void **)&m->d_farblk, fgrid.data(), fgrid.size() * sizeof(float), "far block upload");
    }
    if (st) return st;
    m->map_level = desc->max_level;
    return SAND_OK;
}

sand_status sand_load_depth_map(sand_model m, const char *path) {
    g_err.clear();
    sand_status st = model_precheck(m);
    if (st) return st;
    if (!path) { set_error("NULL path"); return SAND_EINVAL; }
    FILE *f = fopen(path, "rb");
    if (!f) { set_error("cannot open %s", path); return SAND_EINVAL; }
    char magic[4];
    uint32_t ver;
    int32_t h[3];
    float bbox[6];
    bool ok = fread(magic, 1, 4, f) == 4 && memcmp(magic, "SDMO", 4) == 0 && fread(&ver, 4, 1, f) == 1 && ver == 1 &&
              fread(h, 4, 3, f) == 3 && fread(bbox, 4, 6, f) == 6 && h[2] > 0 && h[2] < (1 << 30);
    ok = ok && bbox[0] == -1.f && bbox[1] == -1.f && bbox[2] == -1.f && bbox[3] == 1.f && bbox[4] == 1.f && bbox[5] == 1.f;
    // child [n] int32, depth [n] u8 padded to 4 bytes, far [n] float32: all there in full
    ok = ok && bytes_left(f) >= 8 * (long long)h[2] + ((long long)h[2] + 3) / 4 * 4;
    std::vector<int32_t> child;
    std::vector<uint8_t> depth;
    std::vector<float> far;
    if (ok) {
        const size_t n = (size_t)h[2];
        try {
            child.resize(n);
            depth.resize((n + 3) / 4 * 4);
            far.resize(n);
        } catch (const std::bad_alloc &) {
            fclose(f);
            set_error("%s: cannot hold %zu octree nodes in host memory", path, n);
            return SAND_ENOMEM;
        }
        ok = fread(child.data(), 4, n, f) == n && fread(depth.data(), 1, depth.size(), f) == depth.size() &&
             fread(far.data(), 4, n, f) == n;
    }
    fclose(f);
    if (!ok) { set_error("%s: not a version-1 SDMO depth map over [-1,1]^3 (or truncated)", path); return SAND_EFORMAT; }
    sand_depth_map_desc d{h[0], h[1], h[2]};
    return sand_load_depth_map_mem(m, &d, child.data(), depth.data(), far.data());
}

size_t sand_workspace_bytes(sand_model m, int64_t n, int with_grad) {
    (void)m;
    (void)with_grad;
    return ws_layout(n < 0 ? 0 : n).total;
}

static sand_status run_query(sand_model m, const float *d_points, int64_t n, float *d_out, float *d_grad,
                             const sand_query_opts *opts, void *stream, const uint32_t *d_count = nullptr) {
    sand_status st = model_precheck(m);
    if (st) return st;
    sand_query_opts o{};
    if (opts) o = *opts;
    if (n < 0 || n > 0x7fffffffLL) { set_error("n = %lld outside 0..2^31-1", (long long)n); return SAND_EINVAL; }
    if (n == 0) return SAND_OK;
    if (!d_points || (!d_out && !d_grad)) { set_error("NULL points or output"); return SAND_EINVAL; }
    if ((reinterpret_cast<uintptr_t>(d_points) & 3) || (reinterpret_cast<uintptr_t>(d_out) & 3) ||
        (reinterpret_cast<uintptr_t>(d_grad) & 3)) { set_error("device buffers must be 4-byte aligned"); return SAND_EINVAL; }
    if (o.max_depth < 0) { set_error("max_depth < 0"); return SAND_EINVAL; }
    if (o.all_tails && (!o.full_depth || d_grad)) {
        set_error("all_tails needs full_depth and no gradient");
        return SAND_EINVAL;
    }
    if (!o.full_depth && m->map_level < 0) { set_error("no depth map loaded"); return SAND_ENOMAP; }
    if (o.full_depth && o.d_exit_layers) { set_error("exit layers are not produced in full-depth mode"); return SAND_EINVAL; }
    if (o.full_depth && d_count) { set_error("full-depth mode needs a host point count"); return SAND_EINVAL; }
    // the CUDA-core kernel serves SAND_FP32_SIMT only; every other precision runs on the tensor
    // cores or is refused (no silent switch of kernels)
    const bool simt = o.precision == SAND_FP32_SIMT;
    if (o.all_tails && simt) { set_error("all_tails runs on the tensor-core precisions only"); return SAND_EUNSUPPORTED; }
    if (!simt && !tc_supported(m->desc, o.precision)) {
        set_error("precision %d is not supported for this model on the tensor-core path", o.precision);
        return SAND_EUNSUPPORTED;
    }
    DeviceGuard g(m->device);
    if (!g.ok) { set_error("cannot select device %d", m->device); return SAND_ECUDA; }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void *ws = o.d_workspace;
    size_t wsb = o.workspace_bytes;
    const size_t need = ws_layout(o.full_depth ? 0 : n).total;
    if (ws) {
        if ((reinterpret_cast<uintptr_t>(ws) & 255) || wsb < need) {
            set_error("workspace must be 256-byte aligned and >= %zu bytes", need);
            return SAND_EINVAL;
        }
    } else {
        st = ensure_workspace(m, o.full_depth ? 0 : n, d_grad != nullptr, &ws, &wsb);
        if (st) return st;
    }
    cudaEvent_t *ev = o.stage_events ? reinterpret_cast<cudaEvent_t *>(const_cast<void **>(o.stage_events)) : nullptr;
    if (ev) SAND_CUDA(cudaEventRecord(ev[0], s), "event record");
    SAND_CUDA(launch_init_header(ws, s), "workspace reset");
    if (!o.full_depth) {
        MapDev map{m->d_grid, m->d_far, m->map_level, m->desc.n_layers, m->d_coarse, m->d_bricks, m->d_farblk};
        SAND_CUDA(launch_lookup(map, d_points, n, o.max_depth, d_out, d_grad, o.d_exit_layers, ws, s, d_count),
                  "lookup kernel");
        SAND_CUDA(launch_scatter(d_points, n, m->desc.n_layers, ws, s, d_count), "scatter kernel");
    }
    if (ev) SAND_CUDA(cudaEventRecord(ev[1], s), "event record");
    if (simt) {
        SAND_CUDA(launch_tmlp_simt(m->simt, d_points, n, o.full_depth, ws, d_out, d_grad, m->num_sms, s), "T-MLP kernel");
    } else {
        st = tc_prepare(&m->tc, m->desc, m->params.data(), o.precision);
        if (st) return st;
        SAND_CUDA(launch_tmlp_tc(m->tc, m->simt, d_points, n, o.full_depth, ws, d_out, m->num_sms, s, o.all_tails, 0.f,
                                 nullptr, d_grad, (uint64_t)o.wait_limit_us * 1000ull),
                  "tensor-core T-MLP kernel");
    }
    if (ev) SAND_CUDA(cudaEventRecord(ev[2], s), "event record");
    return SAND_OK;
}

}  // extern "C"

namespace sand {
sand_status query_device_count(sand_model m, const float *d_points, int64_t n, const uint32_t *d_count, float *d_out,
                               float *d_grad, const sand_query_opts *opts, cudaStream_t s) {
    if (!d_count || !opts || !opts->d_workspace || opts->full_depth) {
        set_error("device-count query needs a count, a workspace and SAND mode");
        return SAND_EINVAL;
    }
    return run_query(m, d_points, n, d_out, d_grad, opts, s, d_count);
}

sand_status model_eval_all_tails(sand_model m, const float *d_pts, int64_t n, float *d_out, int precision,
                                 cudaStream_t s) {
    sand_status st = model_precheck(m);
    if (st) return st;
    if (n <= 0) return SAND_OK;
    if (!tc_supported(m->desc, precision)) {
        set_error("precision %d is not supported for this model on the tensor-core path", precision);
        return SAND_EUNSUPPORTED;
    }
    void *ws = nullptr;
    size_t wsb = 0;
    st = ensure_workspace(m, 0, false, &ws, &wsb);
    if (st) return st;
    st = tc_prepare(&m->tc, m->desc, m->params.data(), precision);
    if (st) return st;
    SAND_CUDA(launch_init_header(ws, s), "workspace reset");
    SAND_CUDA(launch_tmlp_tc(m->tc, m->simt, d_pts, n, 1, ws, d_out, m->num_sms, s, 1), "all-tails T-MLP kernel");
    return SAND_OK;
}

const sand_tmlp_desc &model_desc_ref(sand_model m) { return m->desc; }
const float *model_params(sand_model m) { return m->params.data(); }
size_t model_param_count(sand_model m) { return m->params.size(); }

sand_status model_replace_params(sand_model m, const float *h_params) {
    DeviceGuard g(m->device);
    SAND_CUDA(cudaDeviceSynchronize(), "device synchronize");
    memcpy(m->params.data(), h_params, m->params.size() * sizeof(float));
    cudaFree(m->d_simt);
    m->d_simt = nullptr;
    tc_release(&m->tc);
    return pack_simt(m);
}

sand_status model_trace_buffer(sand_model m, size_t bytes, void **out) {
    if (m->trace_bytes < bytes) {
        cudaFree(m->d_trace);
        m->d_trace = nullptr;
        m->trace_bytes = 0;
        if (cudaMalloc(&m->d_trace, bytes) != cudaSuccess) {
            cudaGetLastError();
            set_error("cannot allocate %zu bytes of sphere-tracer state", bytes);
            return SAND_ENOMEM;
        }
        m->trace_bytes = bytes;
    }
    *out = m->d_trace;
    return SAND_OK;
}
}  // namespace sand

extern "C" {

sand_status sand_query_sdf(sand_model m, const float *d_points, int64_t n, float *d_out, const sand_query_opts *opts,
                           void *stream) {
    g_err.clear();
    if (n > 0 && !d_out) { set_error("NULL d_out"); return SAND_EINVAL; }
    return run_query(m, d_points, n, d_out, nullptr, opts, stream);
}

sand_status sand_query_sdf_dynamic(sand_model m, const float *d_points, int64_t n, float r, float *d_out,
                                   uint8_t *d_exit_layers, const sand_query_opts *opts, void *stream) {
    g_err.clear();
    sand_status st = model_precheck(m);
    if (st) return st;
    if (n < 0 || n > 0x7fffffffLL) { set_error("n = %lld outside 0..2^31-1", (long long)n); return SAND_EINVAL; }
    if (n == 0) return SAND_OK;
    if (!d_points || !d_out) { set_error("NULL points or output"); return SAND_EINVAL; }
    if (!(r > 0.f)) { set_error("r must be positive"); return SAND_EINVAL; }
    if ((reinterpret_cast<uintptr_t>(d_points) & 3) || (reinterpret_cast<uintptr_t>(d_out) & 3)) {
        set_error("device buffers must be 4-byte aligned");
        return SAND_EINVAL;
    }
    sand_query_opts o{};
    if (opts) o = *opts;
    if (o.full_depth || o.all_tails || o.d_exit_layers || o.max_depth || o.d_workspace || o.stage_events ||
        o.wait_limit_us) {
        set_error("dynamic queries take only the precision from the query options");
        return SAND_EINVAL;
    }
    if (!tc_supported(m->desc, o.precision)) {
        set_error("precision %d is not supported for this model on the tensor-core path", o.precision);
        return SAND_EUNSUPPORTED;
    }
    DeviceGuard g(m->device);
    if (!g.ok) { set_error("cannot select device %d", m->device); return SAND_ECUDA; }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void *ws = nullptr;
    size_t wsb = 0;
    st = ensure_workspace(m, 0, false, &ws, &wsb);
    if (st) return st;
    st = tc_prepare(&m->tc, m->desc, m->params.data(), o.precision);
    if (st) return st;
    SAND_CUDA(launch_init_header(ws, s), "workspace reset");
    SAND_CUDA(launch_tmlp_tc(m->tc, m->simt, d_points, n, 1, ws, d_out, m->num_sms, s, 0, r, d_exit_layers),
              "dynamic-exit T-MLP kernel");
    return SAND_OK;
}

sand_status sand_query_sdf_grad(sand_model m, const float *d_points, int64_t n, float *d_out, float *d_grad,
                                const sand_query_opts *opts, void *stream) {
    g_err.clear();
    if (n > 0 && !d_grad) { set_error("NULL d_grad"); return SAND_EINVAL; }
    sand_query_opts o{};
    if (opts) o = *opts;
    if (!o.full_depth && n > 0 && !d_out) {
        set_error("d_out is required for SAND gradient queries (far leaves write their stored value there)");
        return SAND_EINVAL;
    }
    return run_query(m, d_points, n, d_out, d_grad, &o, stream);
}

sand_status sand_query_sdf_host(sand_model m, const float *h_points, int64_t n, float *h_out, const sand_query_opts *opts,
                                void *stream) {
    g_err.clear();
    sand_status st = model_precheck(m);
    if (st) return st;
    if (n == 0) return SAND_OK;
    if (!h_points || !h_out || n < 0) { set_error("bad host buffers"); return SAND_EINVAL; }
    sand_query_opts o{};
    if (opts) o = *opts;
    if (o.d_exit_layers || o.all_tails) {
        set_error("d_exit_layers and all_tails are not available for host queries");
        return SAND_EINVAL;
    }
    DeviceGuard g(m->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t need = (size_t)n * 16;
    if (m->stage_bytes < need) {
        cudaFree(m->d_stage);
        m->d_stage = nullptr;
        m->stage_bytes = 0;
        if (cudaMalloc(&m->d_stage, need) != cudaSuccess) {
            cudaGetLastError();
            set_error("cannot allocate %zu bytes of staging", need);
            return SAND_ENOMEM;
        }
        m->stage_bytes = need;
    }
    float *d_pts = m->d_stage;
    float *d_out = m->d_stage + (size_t)n * 3;
    // A pipeline of chunks: chunk k's points go up on copy_in, its query runs on the caller's
    // stream once they are there, and its values come down on copy_out once it is done, so
    // the copies of one chunk overlap the queries of the others.  The input is cut into blocks
    // of kHostBlock consecutive points; of every ten blocks, chunk 0 takes the first, chunk 1
    // the next four, chunk 2 four more and chunk 3 the last, packed together on the device.
    // The first chunk is small because nothing overlaps its upload, the last because nothing
    // overlaps its download; spread over the whole input, every chunk gets about the same mix
    // of exit layers (a contiguous slab of a spatially ordered input may be all far field or
    // all surface, which leaves one kind of warp of the T-MLP kernel idle).  Each chunk is a
    // query of its own points (a point's result does not depend on the other points).
    constexpr int kHostChunks = 4;
    constexpr int64_t kHostBlock = (int64_t)1 << 18;
    const int64_t n_blocks = (n + kHostBlock - 1) / kHostBlock;
    auto chunk_of = [](int64_t b) {
        const int r = (int)(b % 10);
        return r == 0 ? 0 : r <= 4 ? 1 : r <= 8 ? 2 : 3;
    };
    const int n_chunks = n < ((int64_t)1 << 20) ? 1 : kHostChunks;
    if (n_chunks <= 1) {
        SAND_CUDA(cudaMemcpyAsync(d_pts, h_points, (size_t)n * 12, cudaMemcpyHostToDevice, s), "H2D points");
        st = run_query(m, d_pts, n, d_out, nullptr, &o, stream);
        if (st) {
            cudaStreamSynchronize(s);
            return st;
        }
        SAND_CUDA(cudaMemcpyAsync(h_out, d_out, (size_t)n * 4, cudaMemcpyDeviceToHost, s), "D2H values");
        SAND_CUDA(cudaStreamSynchronize(s), "stream synchronize");
        return SAND_OK;
    }
    if (!m->copy_in && cudaStreamCreateWithFlags(&m->copy_in, cudaStreamNonBlocking) != cudaSuccess) {
        m->copy_in = nullptr;
        return cuda_fail(cudaGetLastError(), "copy stream");
    }
    if (!m->copy_out && cudaStreamCreateWithFlags(&m->copy_out, cudaStreamNonBlocking) != cudaSuccess) {
        m->copy_out = nullptr;
        return cuda_fail(cudaGetLastError(), "copy stream");
    }
    cudaEvent_t ev[2 * kHostChunks + 1];
    int n_ev = 0;
    for (; n_ev < 2 * n_chunks + 1; ++n_ev)
        if (cudaEventCreateWithFlags(&ev[n_ev], cudaEventDisableTiming) != cudaSuccess) break;
    cudaError_t ce = n_ev == 2 * n_chunks + 1 ? cudaSuccess : cudaGetLastError();
    // the copies follow whatever the caller queued on its stream before this call
    if (ce == cudaSuccess) ce = cudaEventRecord(ev[2 * n_chunks], s);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(m->copy_in, ev[2 * n_chunks], 0);
    int64_t base = 0;  // first device row of chunk k
    for (int k = 0; k < n_chunks && ce == cudaSuccess && st == SAND_OK; ++k) {
        int64_t cnt = 0;
        for (int64_t b = 0; b < n_blocks && ce == cudaSuccess; ++b) {
            if (chunk_of(b) != k) continue;
            const int64_t off = b * kHostBlock, len = n - off < kHostBlock ? n - off : kHostBlock;
            ce = cudaMemcpyAsync(d_pts + 3 * (base + cnt), h_points + 3 * off, (size_t)len * 12, cudaMemcpyHostToDevice,
                                 m->copy_in);
            cnt += len;
        }
        if (cnt == 0) continue;  // (fewer than ten blocks: the later chunks may be empty)
        if (ce == cudaSuccess) ce = cudaEventRecord(ev[2 * k], m->copy_in);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(s, ev[2 * k], 0);
        if (ce != cudaSuccess) break;
        st = run_query(m, d_pts + 3 * base, cnt, d_out + base, nullptr, &o, stream);
        if (st) break;
        ce = cudaEventRecord(ev[2 * k + 1], s);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(m->copy_out, ev[2 * k + 1], 0);
        int64_t at = base;
        for (int64_t b = 0; b < n_blocks && ce == cudaSuccess; ++b) {
            if (chunk_of(b) != k) continue;
            const int64_t off = b * kHostBlock, len = n - off < kHostBlock ? n - off : kHostBlock;
            ce = cudaMemcpyAsync(h_out + off, d_out + at, (size_t)len * 4, cudaMemcpyDeviceToHost, m->copy_out);
            at += len;
        }
        base += cnt;
    }
    // every path waits for all three streams: no copy may still touch the caller's buffers
    const cudaError_t e1 = cudaStreamSynchronize(m->copy_in);
    const cudaError_t e2 = cudaStreamSynchronize(s);
    const cudaError_t e3 = cudaStreamSynchronize(m->copy_out);
    for (int i = 0; i < n_ev; ++i) cudaEventDestroy(ev[i]);
    if (st) return st;
    if (ce != cudaSuccess) return cuda_fail(ce, "host query pipeline");
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess)
        return cuda_fail(e1 != cudaSuccess ? e1 : e2 != cudaSuccess ? e2 : e3, "stream synchronize");
    return SAND_OK;
}

sand_status sand_read_stats(sand_model m, const void *d_workspace, sand_query_stats *out, void *stream) {
    g_err.clear();
    sand_status st = model_precheck(m);
    if (st) return st;
    if (!out) { set_error("NULL output"); return SAND_EINVAL; }
    const void *ws = d_workspace ? d_workspace : m->d_ws;
    if (!ws) { set_error("no workspace"); return SAND_EINVAL; }
    DeviceGuard g(m->device);
    WsHeader h;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    SAND_CUDA(cudaMemcpyAsync(&h, ws, sizeof h, cudaMemcpyDeviceToHost, s), "read stats");
    SAND_CUDA(cudaStreamSynchronize(s), "stream synchronize");
    out->flags = h.flags;
    out->n_network = h.n_active;
    memcpy(out->count, h.count, sizeof out->count);
    if (h.flags & SAND_FLAG_TIMEOUT) {
        set_error("a device-side wait timed out (site %u)", h.timeout_where);
        return SAND_ETIMEOUT;
    }
    return SAND_OK;
}

sand_status sand_model_desc(sand_model m, sand_tmlp_desc *out) {
    g_err.clear();
    sand_status st = model_precheck(m);
    if (st) return st;
    if (!out) { set_error("NULL output"); return SAND_EINVAL; }
    *out = m->desc;
    return SAND_OK;
}

sand_status sand_free(sand_model m) {
    g_err.clear();
    if (!m) return SAND_OK;
    {
        DeviceGuard g(m->device);
        cudaDeviceSynchronize();
        release(m);
    }
    delete m;
    return SAND_OK;
}

}  // extern "C"
