// plain.h -- launchers of the per-stage kernels (kernels_plain.cu).
#pragma once

#include <algorithm>
#include <string>

#include "../../include/pdhg.h"
#include "common.cuh"

namespace pdhg {

// sets the message returned by pdhg_last_error() on the calling thread
void set_last_error(const std::string &msg);
// pdhg_create's checks of the grid, the scheme and the coefficients (not u0, not the
// step sizes, not the path); reports through pdhg_last_error()
pdhg_status check_shape(const pdhg_problem *p, const pdhg_grid *g, const pdhg_scheme *s);

template <typename T> cudaError_t init_plain_attributes();
template <typename T>
cudaError_t launch_primal(const Params<T> &P, T *u, const T *phit, T *lam, T *lamt, const T *u0, cudaStream_t s);
template <typename T>
cudaError_t launch_residual_rfft(const Params<T> &P, const T *u, void *spec, const void *twx, cudaStream_t s);
template <typename T>
cudaError_t launch_fft_y(const Params<T> &P, void *spec, const void *twy, int inverse, cudaStream_t s);
template <typename T>
cudaError_t launch_tsolve(const Params<T> &P, void *spec, const T *theta, const void *V, cudaStream_t s);
// tab[l * modes + m] = rho_l of mode m (the t-solve's pivots), l < nt
template <typename T>
cudaError_t launch_rho_table(const T *theta, int64_t modes, int nt, T *tab, cudaStream_t s);
template <typename T>
cudaError_t launch_dual_irfft(const Params<T> &P, const void *spec, T *phi, T *phit, const void *twx, cudaStream_t s);
template <typename T> int64_t check_blocks(const Params<T> &P);
// float64 state, preconditioner in float32 (FD, nx a power of two): R^l in float64 -> float32
// x-spectrum; float32 x-spectrum of z -> phi, phit in float64.  twx32: W_nx^k, k <= nx/2, float32.
cudaError_t launch_residual_rfft_p32(const Params<double> &P, const double *u, void *spec, const void *twx32,
                                     cudaStream_t s);
cudaError_t launch_dual_irfft_p32(const Params<double> &P, const void *spec, double *phi, double *phit,
                                  const void *twx32, cudaStream_t s);
// sum of nblocks records of 6 partial sums (partials[6 b + k]) into out[0..5], fixed order
cudaError_t launch_reduce6(const double *partials, int64_t nblocks, double *out, cudaStream_t s);
// sum_l <phi^l, Lap_h u^{l+1}> (FD) into out[0] (float64), partials as for launch_check
template <typename T>
cudaError_t launch_phi_lap(const Params<T> &P, const T *u, const T *phi, double *partials, double *out, cudaStream_t s);
template <typename T>
// Residual sums (Eq. 2.12) into out[0..5]: slice rows 0..nt (slices = 0), or only
// the first `slices` rows.
cudaError_t launch_check(const Params<T> &P, const T *u, const T *phi, const T *lam, const T *u0, double *partials,
                         double *out, cudaStream_t s, int slices = 0);

// ---- batched launches (many 1D instances per launch) ----
// One instance: its parameters and device arrays (those of an ordinary handle).
template <typename T>
struct BatchInst {
    Params<T> P;
    T *u, *phi, *phit, *lam, *lamt;
    const T *u0;
    void *spec;               // Cplx<T> spectrum of the plain path
    const void *twx, *V;      // twiddles, DG eigenvectors
    const T *theta;
    int64_t part_off;         // first 6-double partial record of this instance
    int32_t gx;               // residual-check blocks per slice row
};
// one block of a batched launch: instance and the block's coordinates in that
// instance's own grid (bx = blockIdx.x, l = blockIdx.y of the single launch)
struct BatchEntry { int32_t inst, bx, l, pad; };
// slices per primal entry of the per-stage batch launch (k_b_primal loops over them)
constexpr int BATCH_PRIMAL_SPAN = 16;
// Units (dofs, or DG cells) per block of a slice row in the residual check: 256
// threads x 16 units, one float32 partial per thread folded into float64 once.  Fewer,
// wider blocks keep the float64 block reductions (GB300's float64 rate is a small
// fraction of float32's) from bounding the check.  At most 32 blocks per slice row
// (grid-stride beyond), or 1216 / (nt + 1) when there are few rows (1216 = 8 blocks
// on each of 152 multiprocessors), so that a check of a one- or two-slice problem
// still fills the GPU.
constexpr int64_t CHECK_UNITS_PER_BLOCK = 4096;
inline int64_t check_blocks_per_row(int64_t units, int64_t nt) {
    const int64_t cap = std::max<int64_t>(32, 1216 / (nt + 1));
    return std::min<int64_t>((units + CHECK_UNITS_PER_BLOCK - 1) / CHECK_UNITS_PER_BLOCK, cap);
}
enum { BATCH_PRIMAL, BATCH_RESIDUAL, BATCH_TSOLVE, BATCH_DUAL, BATCH_CHECK, BATCH_REDUCE };
// kind: one of BATCH_*; nblocks table entries (BATCH_REDUCE: entries of `list`,
// instance ids, each summing its partial records into out[inst * 6 ..]).
template <typename T>
cudaError_t launch_batch(int kind, const BatchInst<T> *I, const BatchEntry *tab, int64_t nblocks, size_t smem,
                         const int32_t *list, double *partials, double *out, cudaStream_t s);
// One iteration of every queued instance in one cooperative launch of `grid` blocks of
// 256 threads: queue q (nq entries, pad = stage | items << 2), need[4 inst + stage] items
// per instance and stage, counters cnt[1 + 4 count] (zeroed before the launch), *err set
// when a bounded wait (wait_ns) gives up.
template <typename T>
cudaError_t launch_batch_persistent(const BatchInst<T> *I, const BatchEntry *q, int64_t nq, const int32_t *need,
                                    unsigned int *cnt, int *err, uint64_t wait_ns, int grid, size_t smem,
                                    cudaStream_t s);
// resident blocks per multiprocessor of the persistent batch kernel with `smem` bytes
template <typename T> cudaError_t batch_persistent_occupancy(size_t smem, int *blocks_per_sm);

}  // namespace pdhg
