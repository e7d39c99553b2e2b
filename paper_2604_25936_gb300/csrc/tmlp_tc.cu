// Tensor-core T-MLP path (tcgen05).  Not yet available: every precision
// reports unsupported so callers fall back to nothing silently.
#include "tc.cuh"

namespace sand {

bool tc_supported(const sand_tmlp_desc &, int) { return false; }
sand_status tc_prepare(TcModel *, const sand_tmlp_desc &, const float *, int) {
    set_error("tensor-core path not built");
    return SAND_EUNSUPPORTED;
}
cudaError_t launch_tmlp_tc(const TcModel &, const sand_tmlp_desc &, int, const float *, int64_t, int, void *, float *,
                           int, cudaStream_t) {
    return cudaErrorNotSupported;
}
void tc_release(TcModel *tc) {
    if (tc && tc->d_pack) cudaFree(tc->d_pack);
}

}  // namespace sand
