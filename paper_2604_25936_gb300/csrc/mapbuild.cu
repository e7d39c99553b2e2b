// Network-depth map from the network itself (Sec. 3.2, Eq. 5-7).
//
// For every selected leaf of a pointer octree over [-1, 1]^3, k^3 cell-centred sample
// points are generated on the device, the T-MLP gives all cumulative outputs y_1 .. y_L
// of each (the tensor-core kernel's all-tails mode), Eq. 5 gives each sample its depth
//   near leaf: min{ i : |y_L - y_i| < r  and  sign y_i = sign y_L }
//   far leaf (only on request): min{ i : sign y_i = sign y_L }
// (sign(0) taken as +1; i = L always qualifies), and Eq. 6 max-pools them per leaf.
// Far leaves otherwise keep depth 0: they answer with their stored value (Eq. 7).
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace sand {

constexpr int kMapThreads = 256;

// Sample j of the chunk: leaf j >> 3 lk, offsets (s + 1/2) side / k per axis, x fastest.
// Every value is a dyadic rational with at most 14 significant bits: exact in float32.
__global__ void __launch_bounds__(kMapThreads)
map_samples_kernel(const int4 *__restrict__ cells, int64_t n_pts, int lk, float *__restrict__ pts) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_pts) return;
    const int k = 1 << lk;
    const int4 c = cells[j >> (3 * lk)];  // (level, ix, iy, iz)
    const int s = (int)(j & ((1 << (3 * lk)) - 1));
    const int sx = s & (k - 1), sy = (s >> lk) & (k - 1), sz = s >> (2 * lk);
    const float side = ldexpf(2.f, -c.x);
    const float h = ldexpf(side, -lk);
    pts[3 * j] = (-1.f + (float)c.y * side) + ((float)sx + 0.5f) * h;
    pts[3 * j + 1] = (-1.f + (float)c.z * side) + ((float)sy + 0.5f) * h;
    pts[3 * j + 2] = (-1.f + (float)c.w * side) + ((float)sz + 0.5f) * h;
}

// Eq. 5 for every sample, Eq. 6 by atomicMax into its leaf.
__global__ void __launch_bounds__(kMapThreads)
map_depth_kernel(const float *__restrict__ ys, int L, int64_t n_pts, int lk3, const uint8_t *__restrict__ leaf_near,
                 float r, unsigned *__restrict__ leaf_depth) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_pts) return;
    const int64_t leaf = j >> lk3;
    const bool near = leaf_near[leaf] != 0;
    const float *y = ys + j * L;
    const float yl = y[L - 1];
    const bool pos_l = yl >= 0.f;
    int d = L;
    for (int i = 0; i < L - 1; ++i) {
        const bool same_sign = (y[i] >= 0.f) == pos_l;
        if (same_sign && (!near || fabsf(yl - y[i]) < r)) {
            d = i + 1;
            break;
        }
    }
    atomicMax(leaf_depth + leaf, (unsigned)d);
}

}  // namespace sand

using namespace sand;

extern "C" {

sand_status sand_build_depth_map(sand_model m, const sand_depth_map_desc *desc, const int32_t *h_child,
                                 const uint8_t *h_near, const sand_map_build_opts *opts, uint8_t *h_depth_out,
                                 void *stream) {
    set_error("");
    if (!m || !desc || !h_child || !h_near || !opts || !h_depth_out) { set_error("NULL argument"); return SAND_EINVAL; }
    const int n_nodes = desc->n_nodes;
    if (n_nodes < 1 || desc->max_level < 0 || desc->max_level > 9) {
        set_error("octree: need n_nodes >= 1 and max_level in 0..9");
        return SAND_EINVAL;
    }
    const int k = opts->samples_per_axis;
    int lk = 0;
    while ((1 << lk) < k) ++lk;
    if (k < 1 || k > 16 || (1 << lk) != k) { set_error("samples_per_axis must be a power of two in 1..16"); return SAND_EINVAL; }
    if (!(opts->r > 0.f)) { set_error("r must be positive"); return SAND_EINVAL; }
    const int L = model_layers(m);
    if (desc->n_layers != L) { set_error("octree n_layers %d differs from the model's %d", desc->n_layers, L); return SAND_EINVAL; }

    // leaves (iterative descent; validates the child links: children after their parent, in range)
    struct Cell { int node, level, ix, iy, iz; };
    std::vector<Cell> leaves;
    std::vector<Cell> stack{{0, 0, 0, 0, 0}};
    while (!stack.empty()) {
        const Cell c = stack.back();
        stack.pop_back();
        const int ch = h_child[c.node];
        if (ch < 0) {
            if (h_near[c.node] || opts->far_sign) leaves.push_back(c);
            continue;
        }
        if (ch <= c.node || ch > n_nodes - 8 || c.level >= desc->max_level) {
            set_error("octree node %d has invalid children %d", c.node, ch);
            return SAND_EFORMAT;
        }
        for (int o = 0; o < 8; ++o)
            stack.push_back({ch + o, c.level + 1, 2 * c.ix + (o & 1), 2 * c.iy + ((o >> 1) & 1), 2 * c.iz + ((o >> 2) & 1)});
    }
    memset(h_depth_out, 0, (size_t)n_nodes);
    if (leaves.empty()) return SAND_OK;

    const int dev = model_device(m);
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != dev && cudaSetDevice(dev) != cudaSuccess) { set_error("cannot select device %d", dev); return SAND_ECUDA; }
    struct Restore { int d; bool on; ~Restore() { if (on) cudaSetDevice(d); } } restore{cur, cur != dev};
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    const int64_t nl = (int64_t)leaves.size();
    const int lk3 = 3 * lk;
    const int64_t per_leaf = (int64_t)1 << lk3;
    const int64_t chunk_leaves = std::max<int64_t>(1, ((int64_t)1 << 22) / per_leaf);  // <= 4 M samples per pass
    std::vector<int4> cells(nl);
    std::vector<uint8_t> near(nl);
    for (int64_t i = 0; i < nl; ++i) {
        cells[i] = make_int4(leaves[i].level, leaves[i].ix, leaves[i].iy, leaves[i].iz);
        near[i] = h_near[leaves[i].node] ? 1 : 0;
    }
    const int64_t max_pts = std::min(nl, chunk_leaves) * per_leaf;
    int4 *d_cells = nullptr;
    uint8_t *d_near = nullptr;
    unsigned *d_depth = nullptr;
    float *d_pts = nullptr, *d_ys = nullptr;
    sand_status st = SAND_OK;
    auto fail = [&](cudaError_t e, const char *what) { st = cuda_fail(e, what); };
    cudaError_t e;
    if ((e = cudaMalloc(&d_cells, nl * sizeof(int4))) != cudaSuccess) fail(e, "cudaMalloc(cells)");
    else if ((e = cudaMalloc(&d_near, nl)) != cudaSuccess) fail(e, "cudaMalloc(near)");
    else if ((e = cudaMalloc(&d_depth, nl * sizeof(unsigned))) != cudaSuccess) fail(e, "cudaMalloc(depths)");
    else if ((e = cudaMalloc(&d_pts, max_pts * 12)) != cudaSuccess) fail(e, "cudaMalloc(samples)");
    else if ((e = cudaMalloc(&d_ys, max_pts * 4 * (int64_t)L)) != cudaSuccess) fail(e, "cudaMalloc(outputs)");
    if (st == SAND_OK) {
        if ((e = cudaMemcpyAsync(d_cells, cells.data(), nl * sizeof(int4), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
            (e = cudaMemcpyAsync(d_near, near.data(), nl, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
            (e = cudaMemsetAsync(d_depth, 0, nl * sizeof(unsigned), s)) != cudaSuccess)
            fail(e, "upload leaves");
    }
    for (int64_t l0 = 0; st == SAND_OK && l0 < nl; l0 += chunk_leaves) {
        const int64_t cl = std::min(chunk_leaves, nl - l0);
        const int64_t np = cl * per_leaf;
        const int blocks = (int)((np + kMapThreads - 1) / kMapThreads);
        map_samples_kernel<<<blocks, kMapThreads, 0, s>>>(d_cells + l0, np, lk, d_pts);
        if ((e = cudaGetLastError()) != cudaSuccess) { fail(e, "sample kernel"); break; }
        st = model_eval_all_tails(m, d_pts, np, d_ys, opts->precision, s);
        if (st) break;
        map_depth_kernel<<<blocks, kMapThreads, 0, s>>>(d_ys, L, np, lk3, d_near + l0, opts->r, d_depth + l0);
        if ((e = cudaGetLastError()) != cudaSuccess) { fail(e, "depth kernel"); break; }
    }
    std::vector<unsigned> depth(nl);
    if (st == SAND_OK) {
        if ((e = cudaMemcpyAsync(depth.data(), d_depth, nl * sizeof(unsigned), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            fail(e, "read depths");
    }
    cudaFree(d_cells);
    cudaFree(d_near);
    cudaFree(d_depth);
    cudaFree(d_pts);
    cudaFree(d_ys);
    if (st) return st;
    for (int64_t i = 0; i < nl; ++i) h_depth_out[leaves[i].node] = (uint8_t)depth[i];
    return SAND_OK;
}

}  // extern "C"
