// Reference T-MLP kernel on the CUDA cores (plain float32 FMA).
//
// Evaluates Eq. 2 (and Eq. 3 for multiplicative tails) for tiles of rows:
//   h_0 = x (or Fourier features), h_l = act(W_l h_{l-1} + b_l),
//   t_l = a_l.h_l + c_l  (or (a_l.h_l + c_l)(b_l.h_l + e_l) for l >= 2),
//   y_l = y_{l-1} + t_l, and writes y_d at each row's exit layer d.
// With GRAD, each point carries three tangent rows (forward-mode derivative
// along x, y, z) through the same weights: dh_l = act'(u_l) * (W_l dh_{l-1}),
// dt_l = a_l.dh_l (linear) or (a.dh)(b.h + e) + (a.h + c)(b.dh) (mult).
//
// Rows come either from the exit-layer-sorted float4 array written by the
// scatter kernel (SAND query) or straight from the caller's points (full depth).
// One block of 256 threads owns a tile of ROWS rows; thread j computes output
// unit j (and j + 256 ...) for all rows, so each weight read feeds ROWS FMAs.
#include "internal.cuh"

namespace sand {

__device__ __forceinline__ int row_depth(const WsHeader *hdr, uint32_t r, int L) {
    // rows are sorted by descending exit layer: d(r) = min{d : bin_start[d] <= r}
    int d = L;
    for (int k = L - 1; k >= 1; --k)
        if (hdr->bin_start[k] <= r) d = k;
    return d;
}

template <bool GRAD, int ROWS>
__global__ void __launch_bounds__(256)
tmlp_simt_kernel(TmlpDev M, const float *__restrict__ pts, const float4 *__restrict__ sorted,
                 const WsHeader *__restrict__ hdr, int64_t n, int full_depth, float *__restrict__ out,
                 float *__restrict__ grad) {
    constexpr int P = GRAD ? ROWS / 4 : ROWS;   // points per tile
    constexpr int Q = 256 / ROWS;               // threads sharing one row in the tail reduction
    extern __shared__ __align__(16) float smem[];
    const int W = M.W, D = M.D, L = M.L;
    const int Kmax = D > W ? D : W;
    float *hA = smem;                  // [Kmax][ROWS]
    float *hB = hA + Kmax * ROWS;      // [Kmax][ROWS]
    float *part = hB + Kmax * ROWS;    // [2][Q][ROWS]
    __shared__ int s_idx[P], s_dep[P];
    __shared__ float s_y[P], s_g[P][3], s_x[P][3];
    __shared__ int s_tdepth;
    const int tid = threadIdx.x;

    const int64_t n_rows = full_depth ? n : (int64_t)hdr->n_active;
    const int64_t n_tiles = (n_rows + P - 1) / P;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        __syncthreads();
        if (tid < P) {
            const int64_t r = tile * P + tid;
            int idx = -1, d = 0;
            float x = 0.f, y = 0.f, z = 0.f;
            if (r < n_rows) {
                if (full_depth) {
                    idx = (int)r;
                    d = L;
                    x = pts[3 * r]; y = pts[3 * r + 1]; z = pts[3 * r + 2];
                } else {
                    const float4 v = sorted[r];
                    x = v.x; y = v.y; z = v.z;
                    idx = __float_as_int(v.w);
                    d = row_depth(hdr, (uint32_t)r, L);
                }
            }
            s_idx[tid] = idx; s_dep[tid] = d; s_y[tid] = 0.f;
            s_g[tid][0] = s_g[tid][1] = s_g[tid][2] = 0.f;
            s_x[tid][0] = x; s_x[tid][1] = y; s_x[tid][2] = z;
        }
        __syncthreads();
        if (tid == 0) {
            int m = 0;
            for (int p = 0; p < P; ++p) m = max(m, s_dep[p]);
            s_tdepth = m;
        }
        // ---- features h_0 (and their derivatives) into hA[k][row]
        if (M.enc == SAND_ENC_FOURIER) {
            for (int e = tid; e < M.m * P; e += 256) {
                const int k = e / P, p = e % P;
                const float r = fourier_phase(M.B + 3 * k, s_x[p][0], s_x[p][1], s_x[p][2]);
                float sv, cv;
                sincospif(2.0f * r, &sv, &cv);
                hA[k * ROWS + p] = sv;
                hA[(M.m + k) * ROWS + p] = cv;
                if (GRAD) {
                    const float tau = 6.283185307179586f;
                    for (int c = 0; c < 3; ++c) {
                        const float bk = M.B[3 * k + c] * tau;
                        hA[k * ROWS + (c + 1) * P + p] = bk * cv;
                        hA[(M.m + k) * ROWS + (c + 1) * P + p] = -bk * sv;
                    }
                }
            }
        } else {
            for (int e = tid; e < 3 * ROWS; e += 256) {
                const int k = e / ROWS, r = e % ROWS;
                float v;
                if (r < P) v = s_x[r][k];
                else v = ((r / P) - 1 == k) ? 1.0f : 0.0f;
                hA[k * ROWS + r] = v;
            }
        }
        __syncthreads();
        const int tdepth = s_tdepth;
        float *hin = hA, *hout = hB;
        for (int l = 0; l < tdepth; ++l) {
            const int K = l == 0 ? D : W;
            const float *__restrict__ WT = M.WT[l];
            const float *__restrict__ bias = M.bias[l];
            for (int j0 = 0; j0 < W; j0 += 256) {
                const int j = j0 + tid;
                const bool on = j < W;
                float acc[ROWS];
#pragma unroll
                for (int r = 0; r < ROWS; ++r) acc[r] = 0.f;
                if (on) {
                    for (int k = 0; k < K; ++k) {
                        const float w = __ldg(WT + (size_t)k * W + j);
                        const float4 *h4 = reinterpret_cast<const float4 *>(hin + k * ROWS);
#pragma unroll
                        for (int r4 = 0; r4 < ROWS / 4; ++r4) {
                            const float4 hv = h4[r4];
                            acc[4 * r4 + 0] = fmaf(w, hv.x, acc[4 * r4 + 0]);
                            acc[4 * r4 + 1] = fmaf(w, hv.y, acc[4 * r4 + 1]);
                            acc[4 * r4 + 2] = fmaf(w, hv.z, acc[4 * r4 + 2]);
                            acc[4 * r4 + 3] = fmaf(w, hv.w, acc[4 * r4 + 3]);
                        }
                    }
                    const float b = __ldg(bias + j);
#pragma unroll
                    for (int p = 0; p < P; ++p) {
                        const float u = acc[p] + b;
                        float hv, dact;
                        if (M.act == SAND_ACT_RELU) {
                            hv = u > 0.f ? u : 0.f;
                            dact = u > 0.f ? 1.f : 0.f;
                        } else if (M.act == SAND_ACT_FINER) {  // sin(w0 (|u| + 1) u), slope w0 (2 |u| + 1) cos
                            const float au = fabsf(u);
                            float sv, cv;
                            sincosf(M.omega0 * fmaf(au, u, u), &sv, &cv);
                            hv = sv;
                            dact = M.omega0 * fmaf(2.f, au, 1.f) * cv;
                        } else {
                            float sv, cv;
                            sincosf(M.omega0 * u, &sv, &cv);
                            hv = sv;
                            dact = M.omega0 * cv;
                        }
                        hout[j * ROWS + p] = hv;
                        if (GRAD) {
#pragma unroll
                            for (int c = 1; c < 4; ++c) hout[j * ROWS + c * P + p] = dact * acc[c * P + p];
                        }
                    }
                }
            }
            __syncthreads();
            // ---- tails: partial dot products over units j = q, q + Q, ...
            {
                const int r = tid % ROWS, q = tid / ROWS;
                const float *a = M.tw + (size_t)l * 2 * W;
                const float *bb = a + W;
                const bool mult = (M.tail_kind == SAND_TAIL_MULT) && l >= 1;
                float sa = 0.f, sb = 0.f;
                for (int j = q; j < W; j += Q) {
                    const float hv = hout[j * ROWS + r];
                    sa = fmaf(__ldg(a + j), hv, sa);
                    if (mult) sb = fmaf(__ldg(bb + j), hv, sb);
                }
                part[q * ROWS + r] = sa;
                part[(Q + q) * ROWS + r] = sb;
            }
            __syncthreads();
            if (tid < P) {
                const int p = tid;
                float da[4], db[4];
#pragma unroll
                for (int c = 0; c < (GRAD ? 4 : 1); ++c) {
                    float s0 = 0.f, s1 = 0.f;
                    for (int q = 0; q < Q; ++q) {
                        s0 += part[q * ROWS + c * P + p];
                        s1 += part[(Q + q) * ROWS + c * P + p];
                    }
                    da[c] = s0;
                    db[c] = s1;
                }
                const float c0 = M.tb[2 * l], c1 = M.tb[2 * l + 1];
                const bool mult = (M.tail_kind == SAND_TAIL_MULT) && l >= 1;
                const float t0 = da[0] + c0;
                const float t1 = db[0] + c1;
                s_y[p] += mult ? t0 * t1 : t0;
                if (GRAD) {
#pragma unroll
                    for (int c = 1; c < 4; ++c) s_g[p][c - 1] += mult ? (da[c] * t1 + t0 * db[c]) : da[c];
                }
                if (l + 1 == s_dep[p] && s_idx[p] >= 0) {
                    const int64_t o = s_idx[p];
                    if (out) out[o] = s_y[p];
                    if (GRAD) {
                        grad[3 * o] = s_g[p][0];
                        grad[3 * o + 1] = s_g[p][1];
                        grad[3 * o + 2] = s_g[p][2];
                    }
                }
            }
            float *t = hin; hin = hout; hout = t;
            __syncthreads();
        }
    }
}

template <bool GRAD, int ROWS>
static cudaError_t launch_one(const TmlpDev &M, const float *pts, const float4 *sorted, const WsHeader *hdr, int64_t n,
                              int full_depth, float *out, float *grad, int num_sms, cudaStream_t s) {
    const int Kmax = M.D > M.W ? M.D : M.W;
    const size_t smem = sizeof(float) * ((size_t)2 * Kmax * ROWS + 2 * (256 / ROWS) * ROWS);
    auto kern = tmlp_simt_kernel<GRAD, ROWS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    constexpr int P = GRAD ? ROWS / 4 : ROWS;
    int64_t tiles = (n + P - 1) / P;
    int64_t grid = (int64_t)num_sms * per_sm;
    if (grid > tiles) grid = tiles;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, 256, smem, s>>>(M, pts, sorted, hdr, n, full_depth, out, grad);
    return cudaGetLastError();
}

cudaError_t launch_tmlp_simt(const TmlpDev &M, const float *pts, int64_t n, int full_depth, void *ws, float *out,
                             float *grad, int num_sms, cudaStream_t s) {
    WsLayout Lw = ws_layout(full_depth ? 0 : n);
    char *base = static_cast<char *>(ws);
    const WsHeader *hdr = reinterpret_cast<const WsHeader *>(base);
    const float4 *sorted = full_depth ? nullptr : reinterpret_cast<const float4 *>(base + Lw.sorted);
    const bool wide = M.W > 320 || M.D > 320;
    if (grad) {
        return wide ? launch_one<true, 32>(M, pts, sorted, hdr, n, full_depth, out, grad, num_sms, s)
                    : launch_one<true, 64>(M, pts, sorted, hdr, n, full_depth, out, grad, num_sms, s);
    }
    return wide ? launch_one<false, 32>(M, pts, sorted, hdr, n, full_depth, out, grad, num_sms, s)
                : launch_one<false, 64>(M, pts, sorted, hdr, n, full_depth, out, grad, num_sms, s);
}

}  // namespace sand
