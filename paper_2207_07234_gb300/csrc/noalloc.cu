// noalloc.cu -- pdhg_residual_noalloc: the residual norms for a caller-held
// state without a handle, a workspace or any allocation.
//
// Who needs this: code that must not allocate device memory at all -- for
// example a host that hands the library pre-registered buffers only, or code
// running while the allocator is not available (inside another framework's
// allocator callbacks or under a memory budget that forbids new segments).
// Such callers cannot supply the workspace of pdhg_create, so this entry point
// keeps its scratch (the per-block partial sums of the reduction) in a
// fixed-size array in device global memory that is part of the library image.
//
// The array is loaded with the library on every GPU that uses it and stays
// there until the process exits.  Every call uses the same array: two calls
// whose kernels overlap on the GPU (different streams, no ordering) race on it
// and give wrong results; calls issued in order on one stream are safe.  The
// reduction writes every partial it reads, so nothing has to be cleared
// between calls.
//
// Host code cannot pass the array's name to a kernel (in host code it is only
// a stand-in for the device symbol), so the device address is looked up with
// cudaGetSymbolAddress once per device, with that device current, by the
// first call made on it.  Make that first call before any stream capture.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <mutex>
#include <string>

#include "../../include/pdhg.h"
#include "plain.h"

using namespace pdhg;

namespace {

constexpr size_t kScratchBytes = size_t(2) << 20;               // 2 MiB
constexpr int64_t kOutDoubles = 8;                              // reduction result slot
constexpr int64_t kMaxPartialBlocks =
    (int64_t)((kScratchBytes - 256) / (6 * sizeof(double)));   // 43,685 blocks of 6 doubles

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {nullptr};

pdhg_status err(pdhg_status st, const std::string &m) {
    pdhg::set_last_error(m);
    return st;
}

// Device address of the scratch array for the current device (set up once per device).
pdhg_status scratch_address(void **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return err(PDHG_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return err(PDHG_ERR_UNSUPPORTED, "device index out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return err(PDHG_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return PDHG_OK;
}

template <typename T>
pdhg_status run(const pdhg_problem *p, const pdhg_grid *g, const pdhg_scheme *s, const void *u, const void *phi,
                const void *lam, const void *u0, const void *gamma, double out[4], cudaStream_t stream) {
    Params<T> P;
    memset(&P, 0, sizeof(P));
    const bool dg = s->space >= PDHG_SPACE_DG_P2_LF;
    P.dims = g->dims; P.space = s->space; P.time = s->time; P.init = s->init;
    P.nx = (int32_t)g->nx; P.ny = (int32_t)(g->dims == 2 ? g->ny : 1); P.nt = (int32_t)g->nt;
    const int nm = s->space == PDHG_SPACE_DG_P2_LF ? 3 : 2;
    P.S = dg ? nm * g->nx : (int64_t)g->nx * P.ny;
    P.nkx = (int32_t)(g->nx / 2 + 1);
    P.lines = dg ? nm : P.ny;
    double ht = g->T / (double)g->nt, hx = g->lx / (double)g->nx;
    double hy = g->dims == 2 ? g->ly / (double)g->ny : 1.0;
    P.alpha = (T)p->alpha; P.beta = (T)p->beta; P.nu = (T)p->nu; P.lf_a = (T)p->lf_a;
    P.ht = (T)ht; P.inv_ht = (T)(1.0 / ht); P.inv_hx = (T)(1.0 / hx); P.inv_hy = (T)(1.0 / hy);
    P.gamma_half = (const T *)gamma;

    int64_t nblocks = check_blocks<T>(P);
    if (nblocks > kMaxPartialBlocks)
        return err(PDHG_ERR_UNSUPPORTED,
                   "problem too large for the fixed scratch: min(ceil(units/256), 32)*(nt+1) = " +
                       std::to_string(nblocks) + " > " + std::to_string(kMaxPartialBlocks) +
                       " partial blocks (units = dofs, or cells for DG)");
    void *base = nullptr;
    pdhg_status st = scratch_address(&base);
    if (st != PDHG_OK) return st;
    double *partials = (double *)base;
    double *red = (double *)((char *)base + kScratchBytes - 256);
    cudaError_t e = launch_check<T>(P, (const T *)u, (const T *)phi, (const T *)lam, (const T *)u0, partials, red,
                                    stream);
    if (e != cudaSuccess) return err(PDHG_ERR_CUDA, std::string("residual kernels: ") + cudaGetErrorString(e));
    double acc[6];
    e = cudaMemcpyAsync(acc, red, sizeof(acc), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return err(PDHG_ERR_CUDA, std::string("read-back: ") + cudaGetErrorString(e));
    double wx = g->dims == 2 ? hx * hy : hx;
    double a2 = ht * wx * acc[0], b2 = ht * wx * acc[1], gap = ht * wx * acc[2], c2 = wx * acc[3];
    if (s->init == PDHG_INIT_LAMBDA) {
        a2 += c2;
        b2 += wx * acc[4];
        gap += wx * acc[5];
    }
    out[0] = sqrt(a2); out[1] = sqrt(b2); out[2] = sqrt(c2); out[3] = gap;
    return PDHG_OK;
}

}  // namespace

static_assert(kOutDoubles * sizeof(double) <= 256, "reduction slot fits the reserved tail");

extern "C" pdhg_status pdhg_residual_noalloc(const pdhg_problem *prob, const pdhg_grid *grid,
                                             const pdhg_scheme *scheme, const void *u, const void *phi,
                                             const void *lambda, const void *u0, const void *gamma_half,
                                             double out[4], void *stream) {
    if (!prob || !grid || !scheme || !u || !phi || !u0 || !out)
        return err(PDHG_ERR_INVALID_ARG, "null argument");
    if (scheme->init == PDHG_INIT_LAMBDA && !lambda) return err(PDHG_ERR_INVALID_ARG, "lambda is NULL");
    if (grid->dims != 1 && grid->dims != 2) return err(PDHG_ERR_INVALID_ARG, "dims must be 1 or 2");
    if (grid->nt < 1 || grid->nt > 65534 || grid->nx < 2 || (grid->dims == 2 && grid->ny < 2))
        return err(PDHG_ERR_INVALID_ARG, "bad grid size");
    if (!(grid->T > 0) || !(grid->lx > 0) || (grid->dims == 2 && !(grid->ly > 0)))
        return err(PDHG_ERR_INVALID_ARG, "T, lx, ly must be positive");
    if (scheme->space < PDHG_SPACE_FD_UPWIND || scheme->space > PDHG_SPACE_DG_P1_LF ||
        (scheme->time != PDHG_TIME_BE && scheme->time != PDHG_TIME_BDF2) ||
        (scheme->init != PDHG_INIT_LAMBDA && scheme->init != PDHG_INIT_PINNED))
        return err(PDHG_ERR_INVALID_ARG, "bad scheme");
    if (scheme->space >= PDHG_SPACE_DG_P2_LF && (grid->dims != 1 || gamma_half || prob->nu != 0))
        return err(PDHG_ERR_UNSUPPORTED, "DG is 1D without viscous terms");
    if ((scheme->space == PDHG_SPACE_FD_LF || scheme->space == PDHG_SPACE_DG_P2_LF ||
         scheme->space == PDHG_SPACE_DG_P1_LF) && !(prob->lf_a > 0))
        return err(PDHG_ERR_INVALID_ARG, "lf_a must be given (> 0) for Lax-Friedrichs schemes");
    if (gamma_half && grid->dims != 1) return err(PDHG_ERR_UNSUPPORTED, "gamma_half is 1D only");
    cudaStream_t s = (cudaStream_t)stream;
    if (scheme->precision == PDHG_FP64)
        return run<double>(prob, grid, scheme, u, phi, lambda, u0, gamma_half, out, s);
    if (scheme->precision == PDHG_FP32)
        return run<float>(prob, grid, scheme, u, phi, lambda, u0, gamma_half, out, s);
    return err(PDHG_ERR_INVALID_ARG, "bad precision");
}
