// The field off the boundary: the representation formula of the exterior
// problem (Section 2.1; Eq. bie is its limit on S), discretised like the
// boundary equation in compact form (Section 2.4):
//
//   u(x, t_a) = u_in(x, t_a) + sum_j sum_{g=1}^{a} ( C_U^(g)(x, E_j) q_j^{a-g}
//                                                   - C_W^(g)(x, E_j) u_j^{a-g} )
//
// with the coefficients of the marching (coef_math.cuh) evaluated at the
// field point, which lies off S (no self term, no free term).  One CTA per
// field point: its threads take the elements in turn, compute the lag window
// of (x, E_j) and the window's coefficients once, and add their terms to
// kFieldChunk steps at a time; the per-step sums over the threads are
// reduced in a fixed tree order (deterministic).
#include "tdbem_internal.cuh"

namespace tdbem {

namespace {

constexpr int kFieldThreads = 256;
constexpr int kFieldChunk = 8;

__device__ double incident_value(const Incident &in, const double x[3], int alpha)
{
    if (!in.on) return 0.0;
    const double s = alpha * in.dt - in.t0 - (in.k[0] * x[0] + in.k[1] * x[1] + in.k[2] * x[2]) / in.c;
    if (in.shape == 0) {
        const double a = s / in.width;
        return exp(-a * a);
    }
    const double cs = in.c * s;
    return (cs >= 0.0 && cs <= in.width) ? 0.5 * (1.0 - cos(2.0 * 3.14159265358979323846 * cs / in.width)) : 0.0;
}

__global__ void k_field(BsTable T, int ns, int d, double cdt, int kinds, const double *__restrict__ pts,
                        const double *__restrict__ V, const double *__restrict__ u, const double *__restrict__ q,
                        Incident inc, int a0, int na, double *out, int *flag)
{
    __shared__ double red[kFieldChunk][kFieldThreads];
    const int p = blockIdx.x, tid = threadIdx.x;
    const double x[3] = {pts[3 * p], pts[3 * p + 1], pts[3 * p + 2]};
    const double X[3] = {x[0] / cdt, x[1] / cdt, x[2] / cdt};
    const double nx[3] = {0.0, 0.0, 0.0};
    const int amax = a0 + na - 1;
    for (int c0 = 0; c0 < na; c0 += kFieldChunk) {
        double acc[kFieldChunk];
        for (int k = 0; k < kFieldChunk; ++k) acc[k] = 0.0;
        for (int j = tid; j < ns; j += blockDim.x) {
            const double *Vj = V + 9 * (int64_t)j;
            double rmin, rmax;
            tri_dist(X, Vj, rmin, rmax);
            if (rmin < 1e-9) {
                atomicOr(flag, 2);  // point on the boundary
                continue;
            }
            int g0, cnt;
            lag_window(rmin, rmax, d, amax, g0, cnt);
            for (int g = g0; g < g0 + cnt; ++g) {
                double cf[4];
                coef_set(T, X, nx, Vj, (double)g, false, kinds, cdt, cf);
                for (int k = 0; k < kFieldChunk && c0 + k < na; ++k) {
                    const int a = a0 + c0 + k, b = a - g;
                    if (b < 0) continue;
                    double v = 0.0;
                    if (kinds & 1) v += cf[0] * q[(int64_t)b * ns + j];
                    if (kinds & 2) v -= cf[1] * u[(int64_t)b * ns + j];
                    acc[k] += v;
                }
            }
        }
        for (int k = 0; k < kFieldChunk; ++k) red[k][tid] = acc[k];
        __syncthreads();
        for (int w = blockDim.x / 2; w; w >>= 1) {
            if (tid < w)
                for (int k = 0; k < kFieldChunk; ++k) red[k][tid] += red[k][tid + w];
            __syncthreads();
        }
        if (tid < kFieldChunk && c0 + tid < na)
            out[(int64_t)(c0 + tid) * gridDim.x + p] = red[tid][0] + incident_value(inc, x, a0 + c0 + tid);
        __syncthreads();
    }
}

}  // namespace

}  // namespace tdbem

extern "C" int tdbem_eval_field(const tdbem_ctx *cc, const double *points, int32_t npts, int32_t a0, int32_t na,
                                double *out)
{
    using namespace tdbem;
    tdbem_ctx *c = const_cast<tdbem_ctx *>(cc);
    if (!c) return TDBEM_ERR_ARG;
    if (!points || !out || npts < 1 || na < 1) {
        c->err = "tdbem_eval_field: empty point set or step range";
        return TDBEM_ERR_ARG;
    }
    if (!c->prepared) {
        c->err = "tdbem_eval_field before prepare";
        return TDBEM_ERR_STATE;
    }
    if (a0 < 1 || (int64_t)a0 + na - 1 > c->alpha) {
        c->err = "tdbem_eval_field: steps must lie in 1 .. steps taken";
        return TDBEM_ERR_ARG;
    }
    const int kinds = (c->ku_kind >= 0 ? 1 : 0) | (c->kw_kind >= 0 ? 2 : 0);
    double *dp = nullptr, *dout = nullptr;
    int *dflag = nullptr;
    cudaError_t e = cudaSetDevice(c->dev);
    if (e == cudaSuccess) e = cudaMalloc(&dp, (size_t)npts * 3 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&dout, (size_t)npts * na * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&dflag, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyAsync(dp, points, (size_t)npts * 3 * sizeof(double), cudaMemcpyHostToDevice, c->s);
    if (e == cudaSuccess) e = cudaMemsetAsync(dflag, 0, sizeof(int), c->s);
    if (e == cudaSuccess) {
        k_field<<<npts, kFieldThreads, 0, c->s>>>(c->bs, c->ns, c->P.d, c->cdt, kinds, dp, c->d_V, c->d_u, c->d_q, c->inc,
                                                  a0, na, dout, dflag);
        e = cudaGetLastError();
    }
    int flag = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, (size_t)npts * na * sizeof(double), cudaMemcpyDeviceToHost, c->s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, dflag, sizeof(int), cudaMemcpyDeviceToHost, c->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->s);
    cudaFree(dp);
    cudaFree(dout);
    cudaFree(dflag);
    if (e != cudaSuccess) {
        c->err = std::string("tdbem_eval_field: ") + cudaGetErrorString(e);
        return TDBEM_ERR_CUDA;
    }
    if (flag & 2) {
        c->err = "tdbem_eval_field: a point lies on the boundary";
        return TDBEM_ERR_ARG;
    }
    return TDBEM_OK;
}
