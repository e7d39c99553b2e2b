// Depth-map lookup and exit-layer binning.
//
// lookup  : point -> finest cell of the depth map -> exit layer d (Sec. 3.4);
//           d = 0 writes the stored far value (Eq. 7); LOD clamp d <- min(d, max_depth).
// scan    : exclusive scan of the per-block exit-layer histograms in the order
//           (d = L .. 1, block 0 .. G-1), giving every block its output offset per layer.
// scatter : stable counting sort of the network points by descending exit layer into
//           a packed float4 (x, y, z, original index) array read by the T-MLP kernels.
//
// Cell index (bit-exact with the octree descent of the oracle): for R = 2^level
// cells per axis over [-1, 1], i = clamp(floor(x * R/2), -R/2, R/2 - 1) + R/2.
// x * R/2 is exact in float32 (power-of-two scale), so the index equals the one
// exact arithmetic gives, including ties at cell boundaries (upper cell) and -0.
#include "internal.cuh"

namespace sand {

__device__ __forceinline__ int cell_index(float v, float hr, int half) {
    float f = floorf(v * hr);
    f = fminf(fmaxf(f, -hr), hr - 1.0f);
    return (int)f + half;
}

// Stage kLookupChunk points [c0, c0 + cn) of the AoS array into shared memory.
__device__ __forceinline__ void stage_points(float *sp, const float *pts, int64_t c0, int cn, bool vec) {
    const int nf = cn * 3;
    const float *src = pts + c0 * 3;
    if (vec) {  // src is 16-byte aligned: c0 is a multiple of kLookupChunk and pts is 16-byte aligned
        const float4 *s4 = reinterpret_cast<const float4 *>(src);
        float4 *d4 = reinterpret_cast<float4 *>(sp);
        const int n4 = nf >> 2;
        for (int i = threadIdx.x; i < n4; i += blockDim.x) d4[i] = __ldg(s4 + i);
        for (int i = (n4 << 2) + threadIdx.x; i < nf; i += blockDim.x) sp[i] = __ldg(src + i);
    } else {
        for (int i = threadIdx.x; i < nf; i += blockDim.x) sp[i] = __ldg(src + i);
    }
}

// COARSE: the map is a coarse table with bricks (map.coarse), else a dense finest-level grid.
template <bool COARSE>
__global__ void __launch_bounds__(kLookupThreads)
lookup_kernel(MapDev map, const float *__restrict__ pts, int64_t n, int64_t per_block, int max_depth,
              float *__restrict__ out, float *__restrict__ grad, uint8_t *__restrict__ exit_ws,
              uint8_t *__restrict__ exit_user, WsHeader *hdr, uint32_t *__restrict__ hist, int n_blocks, int vec,
              const uint32_t *__restrict__ d_count) {
    __shared__ __align__(16) float sp[kLookupChunk * 3];
    __shared__ uint32_t cnt[16];
    if (d_count) n = min(n, (int64_t)*d_count);  // point count produced on the device (grid sized for the maximum)
    if (threadIdx.x < 16) cnt[threadIdx.x] = 0;
    const int R = 1 << map.level;
    const int half = R >> 1;
    const float hr = (float)R * 0.5f;
    const int64_t start = (int64_t)blockIdx.x * per_block;
    const int64_t end = min(n, start + per_block);
    const int lane = threadIdx.x & 31;
    for (int64_t c0 = start; c0 < end; c0 += kLookupChunk) {
        const int cn = (int)min((int64_t)kLookupChunk, end - c0);
        __syncthreads();
        stage_points(sp, pts, c0, cn, vec != 0);
        __syncthreads();
        // A thread's kPerThread points in three passes, so that the loads of one pass are all in
        // flight together: (1) cell indices and the first map load (the dense grid's depth, or the
        // coarse entry); (2) the brick's depth where the coarse cell is not uniform; (3) far values
        // where the depth is 0, then the writes and the bin counts.
        constexpr int kPerThread = kLookupChunk / kLookupThreads;
        int dk[kPerThread];       // depth; -1 = no point, -2 = NaN coordinate
        uint32_t ek[kPerThread];  // dense: unused; coarse: the entry's second word (uniform far value or far block)
        uint32_t ck[kPerThread];  // dense: cell index (64-bit below); coarse: brick element index
#pragma unroll
        for (int k = 0; k < kPerThread; ++k) {
            const int p = k * kLookupThreads + threadIdx.x;
            dk[k] = -1;
            ek[k] = 0u;
            ck[k] = 0u;
            if (p < cn) {
                const float x = sp[3 * p], y = sp[3 * p + 1], z = sp[3 * p + 2];
                if (isnan(x) || isnan(y) || isnan(z)) {
                    dk[k] = -2;
                } else {
                    const int ix = cell_index(x, hr, half), iy = cell_index(y, hr, half), iz = cell_index(z, hr, half);
                    if (!COARSE) {  // dense grid
                        dk[k] = __ldg(map.grid + ((int64_t)iz * R + iy) * R + ix);
                    } else {  // coarse table of cells 8 finest cells wide, then a brick
                        const int Rc = R >> 3;
                        const uint2 e = __ldg(map.coarse + ((int64_t)(iz >> 3) * Rc + (iy >> 3)) * Rc + (ix >> 3));
                        const uint32_t local = (uint32_t)((((iz & 7) << 3) + (iy & 7)) * 8 + (ix & 7));
                        ek[k] = e.y;
                        if (e.x & 0x80000000u) {
                            dk[k] = (int)(e.x & 0xFFu) | 0x100;  // uniform cell: bit 8 marks "far value in ek"
                        } else {
                            ck[k] = e.x * 512u + local;
                            dk[k] = 0x200;  // brick load pending
                        }
                        if (!(e.x & 0x80000000u) && e.y != 0xFFFFFFFFu) ek[k] = e.y * 512u + local;
                    }
                }
            }
        }
        if (COARSE) {
#pragma unroll
            for (int k = 0; k < kPerThread; ++k)
                if (dk[k] == 0x200) dk[k] = 0x200 | __ldg(map.bricks + ck[k]);
        }
#pragma unroll
        for (int k = 0; k < kPerThread; ++k) {
            const int p = k * kLookupThreads + threadIdx.x;
            int bin = 16;  // 16 = no point
            if (dk[k] != -1) {
                const int64_t i = c0 + p;
                uint8_t e;
                if (dk[k] == -2) {
                    e = kExitNaN;
                    bin = 15;
                    const float qnan = __int_as_float(0x7fc00000);
                    if (out) out[i] = qnan;
                    if (grad) grad[3 * i] = grad[3 * i + 1] = grad[3 * i + 2] = qnan;
                } else {
                    int d = dk[k] & 0xFF;
                    if (d == 0 && out) {
                        float fv = 0.0f;
                        if (!COARSE) {
                            if (map.far) {
                                const float x = sp[3 * p], y = sp[3 * p + 1], z = sp[3 * p + 2];
                                const int ix = cell_index(x, hr, half), iy = cell_index(y, hr, half),
                                          iz = cell_index(z, hr, half);
                                fv = __ldg(map.far + ((int64_t)iz * R + iy) * R + ix);
                            }
                        } else if (dk[k] & 0x100) {
                            fv = __uint_as_float(ek[k]);
                        } else if (ek[k] != 0xFFFFFFFFu) {
                            fv = __ldg(map.far_blocks + ek[k]);
                        }
                        out[i] = fv;
                    }
                    if (d > 0 && max_depth > 0 && d > max_depth) d = max_depth;
                    if (d == 0 && grad) grad[3 * i] = grad[3 * i + 1] = grad[3 * i + 2] = 0.0f;
                    e = (uint8_t)d;
                    bin = d;
                }
                exit_ws[i] = e;
                if (exit_user) exit_user[i] = e;
            }
            const unsigned peers = __match_any_sync(0xffffffffu, bin);
            if (bin < 16 && lane == __ffs(peers) - 1) atomicAdd(&cnt[bin], (uint32_t)__popc(peers));
        }
    }
    __syncthreads();
    if (threadIdx.x < 16) {
        const uint32_t c = cnt[threadIdx.x];
        hist[threadIdx.x * n_blocks + blockIdx.x] = c;
        if (c) atomicAdd(&hdr->count[threadIdx.x], c);
        if (threadIdx.x == 15 && c) atomicOr(&hdr->flags, (uint32_t)SAND_FLAG_NAN_INPUT);
    }
}

// Single-block exclusive scan over hist[d][g] for d = L .. 1 (descending exit layer), g = 0 .. G-1.
__global__ void __launch_bounds__(1024) scan_kernel(WsHeader *hdr, uint32_t *hist, int n_blocks, int L) {
    __shared__ uint32_t part[1024];
    const int total = L * n_blocks;
    const int per = (total + blockDim.x - 1) / blockDim.x;
    const int b0 = threadIdx.x * per, b1 = min(total, b0 + per);
    auto at = [&](int f) -> uint32_t & { return hist[(L - f / n_blocks) * n_blocks + (f % n_blocks)]; };
    uint32_t s = 0;
    for (int f = b0; f < b1; ++f) s += at(f);
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {  // Hillis-Steele inclusive scan
        uint32_t v = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t run = threadIdx.x ? part[threadIdx.x - 1] : 0u;
    for (int f = b0; f < b1; ++f) {
        uint32_t v = at(f);
        if (f % n_blocks == 0) hdr->bin_start[L - f / n_blocks] = run;
        at(f) = run;
        run += v;
    }
    if (threadIdx.x == blockDim.x - 1) hdr->n_active = part[blockDim.x - 1];
}

__global__ void __launch_bounds__(kLookupThreads)
scatter_kernel(const float *__restrict__ pts, int64_t n, int64_t per_block, const uint8_t *__restrict__ exit_ws,
               const uint32_t *__restrict__ hist, int n_blocks, int L, float4 *__restrict__ sorted, int vec,
               const uint32_t *__restrict__ d_count) {
    if (d_count) n = min(n, (int64_t)*d_count);
    constexpr int kPerThread = kLookupChunk / kLookupThreads;  // sub-chunks of a chunk
    constexpr int kWarps = kLookupThreads / 32;
    constexpr int kSeg = kPerThread * kWarps / 16;  // (sub-chunk, warp) entries per prefix thread
    static_assert(kLookupThreads == 256 && kPerThread % 4 == 0 && kSeg * 16 == kPerThread * kWarps, "scatter layout");
    __shared__ __align__(16) float sp[kLookupChunk * 3];
    // per (sub-chunk k, warp w) in point order f = k * kWarps + w, per exit layer: the count, then
    // its offset from the layer's base in this chunk (padded rows: the prefix pass reads down a
    // column); base[c & 1][d] is layer d's next output position at the start of chunk c
    __shared__ uint16_t pos_of[kPerThread * kWarps][17];
    __shared__ uint32_t base[2][16];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x < 16)
        base[0][threadIdx.x] = (threadIdx.x >= 1 && threadIdx.x <= L) ? hist[threadIdx.x * n_blocks + blockIdx.x] : 0u;
    int par = 0;
    const int64_t start = (int64_t)blockIdx.x * per_block;
    const int64_t end = min(n, start + per_block);
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int64_t c0 = start; c0 < end; c0 += kLookupChunk) {
        const int cn = (int)min((int64_t)kLookupChunk, end - c0);
        __syncthreads();  // the previous chunk is written out
        stage_points(sp, pts, c0, cn, vec != 0);
        // the exit layers of this thread's points of the chunk, loaded together with the staging
        // (four bytes a word), not one latency per sub-chunk
        uint32_t dpk[kPerThread / 4] = {};
#pragma unroll
        for (int k = 0; k < kPerThread; ++k) {
            const int p = k * kLookupThreads + threadIdx.x;
            if (p < cn) dpk[k >> 2] |= (uint32_t)exit_ws[c0 + p] << (8 * (k & 3));
        }
        for (int i = threadIdx.x; i < kPerThread * kWarps * 17; i += kLookupThreads) (&pos_of[0][0])[i] = 0;
        __syncthreads();
        // (1) every warp counts each exit layer in each sub-chunk
#pragma unroll
        for (int k = 0; k < kPerThread; ++k) {
            const int d = (int)((dpk[k >> 2] >> (8 * (k & 3))) & 0xFFu);
            const bool net = d >= 1 && d <= L;
            const unsigned peers = __match_any_sync(0xffffffffu, net ? d : 0);
            if (net && (peers & lt_mask) == 0u) pos_of[k * kWarps + warp][d] = (uint16_t)__popc(peers);
        }
        __syncthreads();
        // (2) per exit layer b, sixteen threads turn the counts into offsets: each sums kSeg
        // consecutive entries, a 16-lane shuffle scan gives the exclusive prefix, the base moves on
        {
            const int b = threadIdx.x >> 4, j = threadIdx.x & 15;
            uint32_t v[kSeg], sum = 0;
#pragma unroll
            for (int i = 0; i < kSeg; ++i) {
                v[i] = pos_of[kSeg * j + i][b];
                sum += v[i];
            }
            uint32_t incl = sum;
#pragma unroll
            for (int o = 1; o < 16; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o, 16);
                if (j >= o) incl += t;
            }
            uint32_t run = incl - sum;
#pragma unroll
            for (int i = 0; i < kSeg; ++i) {
                pos_of[kSeg * j + i][b] = (uint16_t)run;
                run += v[i];
            }
            if (j == 15) base[par ^ 1][b] = base[par][b] + run;
        }
        __syncthreads();
        // (3) every network point to its position: the sub-chunk's and warp's start plus its rank
#pragma unroll
        for (int k = 0; k < kPerThread; ++k) {
            const int p = k * kLookupThreads + threadIdx.x;
            const int d = (int)((dpk[k >> 2] >> (8 * (k & 3))) & 0xFFu);
            const bool net = d >= 1 && d <= L;
            const unsigned peers = __match_any_sync(0xffffffffu, net ? d : 0);
            if (net) {
                const uint32_t pos = base[par][d] + pos_of[k * kWarps + warp][d] + (uint32_t)__popc(peers & lt_mask);
                sorted[pos] = make_float4(sp[3 * p], sp[3 * p + 1], sp[3 * p + 2], __int_as_float((int)(c0 + p)));
            }
        }
        par ^= 1;
    }
}

static void lookup_grid(int64_t n, int *g, int64_t *per_block) {
    int64_t chunks = (n + kLookupChunk - 1) / kLookupChunk;
    int64_t blocks = chunks < kMaxLookupBlocks ? chunks : kMaxLookupBlocks;
    if (blocks < 1) blocks = 1;
    int64_t chunks_per_block = (chunks + blocks - 1) / blocks;
    *per_block = chunks_per_block * kLookupChunk;
    *g = (int)((n + *per_block - 1) / *per_block);
    if (*g < 1) *g = 1;
}

cudaError_t launch_init_header(void *ws, cudaStream_t s) { return cudaMemsetAsync(ws, 0, sizeof(WsHeader), s); }

cudaError_t launch_lookup(const MapDev &map, const float *pts, int64_t n, int max_depth, float *out, float *grad,
                          uint8_t *exit_layers, void *ws, cudaStream_t s, const uint32_t *d_count) {
    WsLayout L = ws_layout(n);
    char *base = static_cast<char *>(ws);
    int g;
    int64_t per;
    lookup_grid(n, &g, &per);
    const int vec = (reinterpret_cast<uintptr_t>(pts) & 15) == 0;
    auto kernel = map.coarse ? lookup_kernel<true> : lookup_kernel<false>;
    kernel<<<g, kLookupThreads, 0, s>>>(map, pts, n, per, max_depth, out, grad, reinterpret_cast<uint8_t *>(base + L.exit),
                                        exit_layers, reinterpret_cast<WsHeader *>(base),
                                        reinterpret_cast<uint32_t *>(base + L.hist), g, vec, d_count);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const float *pts, int64_t n, int n_layers, void *ws, cudaStream_t s, const uint32_t *d_count) {
    WsLayout L = ws_layout(n);
    char *base = static_cast<char *>(ws);
    int g;
    int64_t per;
    lookup_grid(n, &g, &per);
    const int vec = (reinterpret_cast<uintptr_t>(pts) & 15) == 0;
    scan_kernel<<<1, 1024, 0, s>>>(reinterpret_cast<WsHeader *>(base), reinterpret_cast<uint32_t *>(base + L.hist), g,
                                   n_layers);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    scatter_kernel<<<g, kLookupThreads, 0, s>>>(pts, n, per, reinterpret_cast<const uint8_t *>(base + L.exit),
                                                reinterpret_cast<const uint32_t *>(base + L.hist), g, n_layers,
                                                reinterpret_cast<float4 *>(base + L.sorted), vec, d_count);
    return cudaGetLastError();
}

}  // namespace sand
