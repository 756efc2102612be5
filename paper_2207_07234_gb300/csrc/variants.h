// variants.h -- device helpers of the drivers of Algorithms 2 and 3 (Sec. 3.4, 3.5)
// and of the mixed-precision solve.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pdhg {

// Algorithm 2's transfer from ntc to 2 ntc slices (same horizon), S values per slice:
//   u_f^{2l} = u_c^l, u_f^{2l+1} = (u_c^l + u_c^{l+1}) / 2          (u^l at time l h)
//   phi_f^{2l+1} = phi_c^l, phi_f^{2l} = (phi_c^{l-1} + phi_c^l) / 2 (phi^l at time (l+1) h),
//   phi_f^0 = phi_c^0, and phit_f = phi_f.
template <typename T>
cudaError_t launch_interp_t(const T *uc, const T *phic, T *uf, T *phif, T *phitf, int64_t S, int64_t ntc,
                            cudaStream_t s);

// u[l S + i] = u0[i] for l < nslices, i < S (one launch for the initial state)
template <typename T>
cudaError_t launch_fill_slices(T *u, const T *u0, int64_t S, int64_t nslices, cudaStream_t s);

// dst[i] = (double)src[i], i < n (the float32 -> float64 hand-over of a mixed solve)
cudaError_t launch_widen(const float *src, double *dst, int64_t n, cudaStream_t s);

}  // namespace pdhg
