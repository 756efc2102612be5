// kernels_variants.cu -- the transfer between time meshes of Algorithm 2 (Sec. 3.4).
#include <algorithm>

#include "variants.h"

namespace pdhg {

template <typename T>
__global__ void k_interp_t(const T *__restrict__ uc, const T *__restrict__ phic, T *__restrict__ uf,
                           T *__restrict__ phif, T *__restrict__ phitf, int64_t S, int64_t ntc) {
    const int64_t ntf = 2 * ntc;
    const int64_t nu = (ntf + 1) * S, total = nu + ntf * S;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        if (i < nu) {
            const int64_t m = i / S, j = i - m * S, l = m >> 1;     // fine slice m, coarse l
            uf[i] = (m & 1) ? (T)0.5 * (uc[l * S + j] + uc[(l + 1) * S + j]) : uc[l * S + j];
        } else {
            const int64_t k = i - nu, m = k / S, j = k - m * S, l = m >> 1;
            T v;
            if (m & 1) v = phic[l * S + j];
            else if (m == 0) v = phic[j];
            else v = (T)0.5 * (phic[(l - 1) * S + j] + phic[l * S + j]);
            phif[k] = v;
            phitf[k] = v;
        }
    }
}

template <typename T>
cudaError_t launch_interp_t(const T *uc, const T *phic, T *uf, T *phif, T *phitf, int64_t S, int64_t ntc,
                            cudaStream_t s) {
    const int64_t total = (4 * ntc + 1) * S;
    const int64_t blocks = std::min<int64_t>((total + 255) / 256, 152 * 8);
    k_interp_t<T><<<(unsigned)blocks, 256, 0, s>>>(uc, phic, uf, phif, phitf, S, ntc);
    return cudaGetLastError();
}

__global__ void k_widen(const float *__restrict__ src, double *__restrict__ dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (double)src[i];
}

cudaError_t launch_widen(const float *src, double *dst, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 8);
    k_widen<<<(unsigned)blocks, 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

// u[l S + i] = u0[i] for l < nslices (the initial state: u0 extended in t)
template <typename T>
__global__ void k_fill_slices(T *__restrict__ u, const T *__restrict__ u0, int64_t S, int64_t total) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
        u[i] = u0[i % S];
}

template <typename T>
cudaError_t launch_fill_slices(T *u, const T *u0, int64_t S, int64_t nslices, cudaStream_t s) {
    const int64_t total = S * nslices;
    if (total <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((total + 255) / 256, 152 * 8);
    k_fill_slices<T><<<(unsigned)blocks, 256, 0, s>>>(u, u0, S, total);
    return cudaGetLastError();
}

template cudaError_t launch_fill_slices<float>(float *, const float *, int64_t, int64_t, cudaStream_t);
template cudaError_t launch_fill_slices<double>(double *, const double *, int64_t, int64_t, cudaStream_t);
template cudaError_t launch_interp_t<float>(const float *, const float *, float *, float *, float *, int64_t, int64_t,
                                            cudaStream_t);
template cudaError_t launch_interp_t<double>(const double *, const double *, double *, double *, double *, int64_t,
                                             int64_t, cudaStream_t);

}  // namespace pdhg
