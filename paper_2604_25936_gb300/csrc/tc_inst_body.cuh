// One instantiation of the tensor-core T-MLP kernel per activation (SIREN, ReLU, FINER) and tail kind, for the
// precision mode SAND_INST_MODE and the kernel variant SAND_INST_VAR (0 plain, 1 extended
// outputs, 2 gradient, 3 SAND query with CUDA-core warps), set by the including translation unit.
#include "tc_kernel.cuh"

namespace sand {

template <int ACT, int TAIL>
static cudaError_t launch_one(const CUtensorMap &map, const TcParams &P, const float *pts, const float4 *sorted,
                              WsHeader *hdr, int64_t n, int full_depth, float *out, int grid, size_t smem,
                              cudaStream_t s) {
    auto kern = tmlp_tc_kernel<SAND_INST_MODE, ACT, TAIL, SAND_INST_VAR>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, tc_threads(SAND_INST_VAR), smem, s>>>(map, P, pts, sorted, hdr, n, full_depth, out);
    return cudaGetLastError();
}

template <>
cudaError_t launch_tc_mode<SAND_INST_MODE, SAND_INST_VAR>(const CUtensorMap &map, const TcParams &P, int act, int tail,
                                                          const float *pts, const float4 *sorted, WsHeader *hdr,
                                                          int64_t n, int full_depth, float *out, int grid,
                                                          size_t smem, cudaStream_t s) {
    if (act == SAND_ACT_RELU)
        return tail == SAND_TAIL_MULT
                   ? launch_one<SAND_ACT_RELU, SAND_TAIL_MULT>(map, P, pts, sorted, hdr, n, full_depth, out, grid, smem, s)
                   : launch_one<SAND_ACT_RELU, SAND_TAIL_LINEAR>(map, P, pts, sorted, hdr, n, full_depth, out, grid, smem, s);
    if (act == SAND_ACT_FINER)
        return tail == SAND_TAIL_MULT
                   ? launch_one<SAND_ACT_FINER, SAND_TAIL_MULT>(map, P, pts, sorted, hdr, n, full_depth, out, grid, smem, s)
                   : launch_one<SAND_ACT_FINER, SAND_TAIL_LINEAR>(map, P, pts, sorted, hdr, n, full_depth, out, grid, smem, s);
    return tail == SAND_TAIL_MULT
               ? launch_one<SAND_ACT_SINE, SAND_TAIL_MULT>(map, P, pts, sorted, hdr, n, full_depth, out, grid, smem, s)
               : launch_one<SAND_ACT_SINE, SAND_TAIL_LINEAR>(map, P, pts, sorted, hdr, n, full_depth, out, grid, smem, s);
}

}  // namespace sand
