// Zero-lag solve that allocates no device memory.
//
// Some callers of this library cannot call cudaMalloc at the point where
// they want to solve: code running while a CUDA graph is being captured by
// someone else, processes under a memory pool or allocator they must not
// bypass, or hosts that forbid allocation after start-up for deterministic
// memory use.  For them tdbem_zero_lag_solve_static solves A x = b with the
// context's zero-lag matrix (built by tdbem_prepare) using scratch memory
// that lives in a fixed file-scope device array instead of memory
// allocated per call.
//
// It always runs plain Jacobi sweeps (the count tdbem_prepare derived from
// the matrix and solver_tol), also when a learned SAI preconditioner is
// installed with tdbem_set_precond: tdbem_step then runs the SAI sweeps, and
// the two solutions agree to the solver tolerance rather than bit for bit.
//
// The array holds three vectors of at most kStaticMaxNs doubles (b and the
// two Jacobi iterates; 6 MiB): every GPU that loads this library keeps it
// until the process exits.  All calls on a device share it and it keeps the
// last call's contents, so calls that overlap on the GPU (different
// streams, or different contexts on the same device without ordering)
// race; the iterates are written before they are read, so no clearing is
// needed.  In host code the array's name is only a host-side stand-in, not
// a device address: its address is taken once per device with
// cudaGetSymbolAddress (with that device current) in the first call on the
// device, which should therefore come before any stream capture.
#include <mutex>

#include "tdbem_internal.cuh"

namespace {

constexpr int kStaticMaxNs = 262144;
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_solve_scratch[3 * kStaticMaxNs];

double *g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// One Jacobi sweep x' = D^-1 (b - R x) (xin == nullptr: x' = D^-1 b).
__global__ void k_static_sweep(int ns, int width, const double *__restrict__ aoff, const int32_t *__restrict__ acol,
                               const double *__restrict__ ainv, const double *__restrict__ b,
                               const double *__restrict__ xin, double *xout)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns) return;
    double s = b[i];
    if (xin) {
        for (int k = 0; k < width; ++k) {
            int cidx = acol[(int64_t)k * ns + i];
            if (cidx >= 0) s -= aoff[(int64_t)k * ns + i] * xin[cidx];
        }
    }
    xout[i] = s * ainv[i];
}

// Device address of the scratch array on the current device (set up once).
cudaError_t scratch_address(int dev, double **out)
{
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_solve_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = (double *)p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int tdbem_zero_lag_solve_static(const tdbem_ctx *cc, const double *b, double *x, int32_t on_device)
{
    tdbem_ctx *c = const_cast<tdbem_ctx *>(cc);
    if (!c || !b || !x) return TDBEM_ERR_ARG;
    const int ns = c->ns;
    if (ns > kStaticMaxNs) {
        c->err = "tdbem_zero_lag_solve_static: ns = " + std::to_string(ns) + " exceeds the static scratch limit of " +
                 std::to_string(kStaticMaxNs) + " elements";
        return TDBEM_ERR_ARG;
    }
    if (!c->prepared) {
        c->err = "zero-lag solve before prepare";
        return TDBEM_ERR_STATE;
    }
    cudaError_t e = cudaSetDevice(c->dev);
    double *scr = nullptr;
    if (e == cudaSuccess) e = scratch_address(c->dev, &scr);
    if (e != cudaSuccess) {
        c->err = std::string("tdbem_zero_lag_solve_static: ") + cudaGetErrorString(e);
        return TDBEM_ERR_CUDA;
    }
    cudaStream_t st = c->user;
    double *db = scr, *xa = scr + kStaticMaxNs, *xb = scr + 2 * kStaticMaxNs;
    const double *bin = b;
    if (!on_device) {
        e = cudaMemcpyAsync(db, b, ns * sizeof(double), cudaMemcpyHostToDevice, st);
        bin = db;
    }
    const int K = c->solve_iters;
    double *last = nullptr;
    for (int it = 0; it < K && e == cudaSuccess; ++it) {
        const double *xin = (it == 0) ? nullptr : ((it & 1) ? xa : xb);
        double *xout = (it & 1) ? xb : xa;
        if (it == K - 1 && on_device) xout = x;
        k_static_sweep<<<(ns + 127) / 128, 128, 0, st>>>(ns, c->ell_w, c->d_aoff, c->d_acol, c->d_ainv, bin, xin,
                                                          xout);
        e = cudaGetLastError();
        last = xout;
    }
    if (e == cudaSuccess && !on_device) {
        e = cudaMemcpyAsync(x, last, ns * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) {
        c->err = std::string("tdbem_zero_lag_solve_static: ") + cudaGetErrorString(e);
        return TDBEM_ERR_CUDA;
    }
    return TDBEM_OK;
}
