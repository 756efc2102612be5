// kernels_fused2d.cu -- fused path for 2D finite differences (not enabled yet).
#include "fused2d.h"

namespace pdhg {

bool fused2d_supported(int, int, int, int, int64_t, int64_t, int64_t, double) { return false; }
size_t fused2d_workspace_bytes(int64_t, int64_t, int64_t) { return 0; }
cudaError_t fused2d_init(Fused2D *f, const Params<float> &, void *ws, const float *twx, const float *twy,
                         const float *theta) {
    f->ws = ws; f->twx = twx; f->twy = twy; f->theta = theta; f->pending = false;
    return cudaSuccess;
}
cudaError_t fused2d_cols(Fused2D *, const Params<float> &, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t fused2d_rows(Fused2D *, const Params<float> &, float *, float *, float *, float *, const float *,
                         cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace pdhg
