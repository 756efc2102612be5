// fused2d.h -- the fused four-kernel iteration for 2D finite differences (float32).
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace pdhg {

struct Fused2D {
    CUtensorMap tmC;         // the spectrum as rows-C's TMA source (nx = 1024), 64-byte aligned
    int *err;                // device flag: a pipelined rows-C stage wait gave up
    float2 *spec;            // spectrum [l][kx][y]: X, then spill, then K_d^{-1} R, in place
    float2 *twM;             // staged Stockham twiddles of length M = nx/2 (stockham.cuh)
    float2 *twY;             // staged twiddles of length ny (radix 4; ny = 1024: the 4x8x8x4 plan)
    float2 *twM8;            // radix-8 staged twiddles of length M (stockham.cuh)
    float *thetaT;           // theta per mode, [kx][ky]
    const float2 *twN;       // W_nx^k, k <= nx/2 (the plain path's table)
    int tc;                  // time slices per rows-R block
    int nsm;                 // multiprocessors of the device (persistent rows-C grid)
    int rows_slots;          // resident rows-R blocks on the device
    uint64_t wait_ns;        // budget of each bounded device wait
};

constexpr uint64_t FUSED2D_WAIT_NS_DEFAULT = 1000000000ull;   // 1 s

bool fused2d_supported(int dims, int space, int time, int prec, int64_t nx, int64_t ny, int64_t nt, double nu);
size_t fused2d_workspace_bytes(int64_t nx, int64_t ny, int64_t nt);
void fused2d_layout(Fused2D *f, void *ws, int64_t nx, int64_t ny, int64_t nt);
cudaError_t fused2d_init(Fused2D *f, const Params<float> &P, void *ws, const float *twx, const float *twy,
                         const float *theta);
cudaError_t fused2d_primal(const Params<float> &P, float *u, const float *phit, float *lam, float *lamt,
                           const float *u0, cudaStream_t s);
cudaError_t fused2d_rowsR(Fused2D *f, const Params<float> &P, const float *u, cudaStream_t s);
// residual norms of a 2D finite-difference state (fused path and plain 2D handles): gx
// blocks per slice row, records at partials[(l gx + bx) * 6] (the generic check's layout)
template <typename T> bool check2d_applies(const Params<T> &P);
template <typename T>
cudaError_t launch_check2d(const Params<T> &P, const T *u, const T *phi, const T *lam, const T *u0,
                           double *partials, int gx, cudaStream_t s);
cudaError_t fused2d_cols(Fused2D *f, const Params<float> &P, cudaStream_t s);
// time slices per rows-R block for nt slices, `rows` row blocks and `slots` resident blocks
int rowsR_chunk(int nt, int rows, int slots, bool bdf2);
cudaError_t fused2d_rowsC(Fused2D *f, const Params<float> &P, float *phi, float *phit, cudaStream_t s);

}  // namespace pdhg
