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
// cudaGetSymbolAddress, with the device current, by the first call made in its
// CUDA context.  The address is cached per device together with that
// context's unique id (cuCtxGetId): after a cudaDeviceReset the device's new
// primary context has a new id, and the next call looks the address up again.
// Make the first call in a context before any stream capture.
#include <cuda.h>
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
unsigned long long g_ctx[kMaxDevices] = {0};    // id of the context g_addr[dev] belongs to

typedef CUresult (*ctx_current_fn)(CUcontext *);
typedef CUresult (*ctx_id_fn)(CUcontext, unsigned long long *);

// Unique id of the calling thread's current CUDA context (0: none current, or the
// driver does not report one, in which case the address is looked up on every call).
unsigned long long current_context_id() {
    static ctx_current_fn get_current = nullptr;
    static ctx_id_fn get_id = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (ctx_current_fn)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (ctx_id_fn)f;
    }
    if (!get_current || !get_id) return 0;
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

pdhg_status err(pdhg_status st, const std::string &m) {
    pdhg::set_last_error(m);
    return st;
}

// Device address of the scratch array for the current device, set up once per
// device and context (looked up again when the device's context has changed).
pdhg_status scratch_address(void **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return err(PDHG_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return err(PDHG_ERR_UNSUPPORTED, "device index out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    const unsigned long long ctx = current_context_id();
    if (!g_addr[dev] || ctx == 0 || ctx != g_ctx[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return err(PDHG_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_addr[dev] = p;
        g_ctx[dev] = current_context_id();        // the lookup has made the context current
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
                   "problem too large for the fixed scratch: min(ceil(units/4096), max(32, 1216/(nt+1)))*(nt+1) = " +
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
    // pdhg_create's checks of the grid, scheme and coefficients (sizes within the
    // library's limits, so that every index stays in range), with this call's
    // gamma_half in place of prob->gamma_half
    pdhg_problem shape = *prob;
    shape.gamma_half = (const double *)gamma_half;
    const pdhg_status vs = check_shape(&shape, grid, scheme);
    if (vs != PDHG_OK) return vs;
    if ((scheme->space == PDHG_SPACE_FD_LF || scheme->space == PDHG_SPACE_DG_P2_LF ||
         scheme->space == PDHG_SPACE_DG_P1_LF) && !(prob->lf_a > 0))
        return err(PDHG_ERR_INVALID_ARG, "lf_a must be given (> 0) for Lax-Friedrichs schemes");
    cudaStream_t s = (cudaStream_t)stream;
    if (scheme->precision == PDHG_FP64)
        return run<double>(prob, grid, scheme, u, phi, lambda, u0, gamma_half, out, s);
    if (scheme->precision == PDHG_FP32)
        return run<float>(prob, grid, scheme, u, phi, lambda, u0, gamma_half, out, s);
    return err(PDHG_ERR_INVALID_ARG, "bad precision");
}
