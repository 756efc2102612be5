// fused2d.h -- the fused two-kernel iteration for 2D finite differences (FP32).
#pragma once

#include "common.cuh"

namespace pdhg {

struct Fused2D {
    void *ws;            // fused-path scratch inside the caller's workspace
    const float *twx, *twy, *theta;
    bool pending;        // a dual update (spectrum in ws) is waiting to be applied
};

bool fused2d_supported(int dims, int space, int time, int prec, int64_t nx, int64_t ny, int64_t nt, double nu);
size_t fused2d_workspace_bytes(int64_t nx, int64_t ny, int64_t nt);
cudaError_t fused2d_init(Fused2D *f, const Params<float> &P, void *ws, const float *twx, const float *twy,
                         const float *theta);
cudaError_t fused2d_cols(Fused2D *f, const Params<float> &P, cudaStream_t s);
cudaError_t fused2d_rows(Fused2D *f, const Params<float> &P, float *u, float *phi, float *lam, float *lamt,
                         const float *u0, cudaStream_t s);

}  // namespace pdhg
