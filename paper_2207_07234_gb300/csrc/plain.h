// plain.h -- launchers of the per-stage kernels (kernels_plain.cu).
#pragma once

#include <string>

#include "common.cuh"

namespace pdhg {

// sets the message returned by pdhg_last_error() on the calling thread
void set_last_error(const std::string &msg);

template <typename T> cudaError_t init_plain_attributes();
template <typename T>
cudaError_t launch_primal(const Params<T> &P, T *u, const T *phit, T *lam, T *lamt, const T *u0, cudaStream_t s);
template <typename T>
cudaError_t launch_residual_rfft(const Params<T> &P, const T *u, void *spec, const void *twx, cudaStream_t s);
template <typename T>
cudaError_t launch_fft_y(const Params<T> &P, void *spec, const void *twy, int inverse, cudaStream_t s);
template <typename T>
cudaError_t launch_tsolve(const Params<T> &P, void *spec, const T *theta, const void *V, cudaStream_t s);
template <typename T>
cudaError_t launch_dual_irfft(const Params<T> &P, const void *spec, T *phi, T *phit, const void *twx, cudaStream_t s);
template <typename T> int64_t check_blocks(const Params<T> &P);
// sum_l <phi^l, Lap_h u^{l+1}> (FD) into out[0] (float64), partials as for launch_check
template <typename T>
cudaError_t launch_phi_lap(const Params<T> &P, const T *u, const T *phi, double *partials, double *out, cudaStream_t s);
template <typename T>
cudaError_t launch_check(const Params<T> &P, const T *u, const T *phi, const T *lam, const T *u0, double *partials,
                         double *out, cudaStream_t s);

}  // namespace pdhg
