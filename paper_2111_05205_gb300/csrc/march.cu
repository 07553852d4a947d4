// Per-step kernels of the time marching (Section 2.5, Eq. linear): the
// history sum that forms b^{a-1}, and the zero-lag solve A x^{a-1} = b^{a-1}.
#include "tdbem_internal.cuh"

namespace tdbem {

constexpr int kNearThreads = 128;

// Incident-wave term e_i(t_a) of the total-field equation: u_in (OBIE) or
// (d/dn_x - c^-1 d/dt) u_in (BMBIE) for the plane pulse
// u_in = f(t - t0 - k.x/c), f(s) = exp(-(s/width)^2).
__device__ __forceinline__ double incident_term(const Incident &in, const double *xc, const double *n, int alpha)
{
    double kx = in.k[0] * xc[0] + in.k[1] * xc[1] + in.k[2] * xc[2];
    double s = alpha * in.dt - in.t0 - kx / in.c;
    double a = s / in.width;
    double f = exp(-a * a);
    if (!in.bie) return f;
    double df = -2.0 * a / in.width * f;
    double kn = in.k[0] * n[0] + in.k[1] * n[1] + in.k[2] * n[2];
    // d/dn_x f(t - k.x/c) = -(k.n/c) f';  c^-1 d/dt f = f'/c
    return -(1.0 + kn) / in.c * df;
}

// b_i = -e_i - sum_j sum_{g in window(i,j), g <= a} (KU^(g)_ij q_j^{a-g} - KW^(g)_ij u_j^{a-g})
// One CTA per row i; each warp walks 32-pair blocks of the row.  Window
// slot s of a block is stored packed (lanes with cnt > s, in lane order),
// so every load of the coefficient stream is a contiguous warp access; the
// history entries x_j^{a-g} of one slot differ only by the lanes' g0.
// The row sum is reduced in a fixed order (deterministic).
__global__ void __launch_bounds__(kNearThreads) k_near_sum(int ns, int nblk, int alpha,
                                                           const uint16_t *__restrict__ meta,
                                                           const int64_t *__restrict__ boff,
                                                           const double *__restrict__ ku,
                                                           const double *__restrict__ kw,
                                                           const double *__restrict__ u,
                                                           const double *__restrict__ q,
                                                           const double *__restrict__ exc, Incident inc,
                                                           const double *__restrict__ xc,
                                                           const double *__restrict__ nrm, double *b)
{
    __shared__ double red[kNearThreads / 32];
    const int i = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const uint16_t *mrow = meta + (int64_t)i * ns;
    const int64_t *orow = boff + (int64_t)i * nblk;
    double acc = 0.0;
    for (int bk = warp; bk < nblk; bk += kNearThreads / 32) {
        int j = bk * 32 + lane;
        unsigned m = (j < ns) ? mrow[j] : 0u;
        int g0 = m & kMaxG0, cnt = m >> kG0Bits;
        int64_t pos = orow[bk];
        int sm = (int)__reduce_max_sync(0xffffffffu, (unsigned)cnt);
        // lag g = g0 + s reaches back to beta = alpha - g
        int beta = alpha - g0;
        for (int s = 0; s < sm; ++s, --beta) {
            unsigned mask = __ballot_sync(0xffffffffu, cnt > s);
            if (cnt > s && beta >= 0) {
                int64_t idx = pos + __popc(mask & lt);
                int64_t h = (int64_t)beta * ns + j;
                if (ku) acc -= ku[idx] * q[h];
                if (kw) acc += kw[idx] * u[h];
            }
            pos += __popc(mask);
        }
    }
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kNearThreads / 32; ++w) t += red[w];
        double e = 0.0;
        if (exc)
            e = exc[i];
        else if (inc.on)
            e = incident_term(inc, xc + 3 * i, nrm + 3 * i, alpha);
        b[i] = t - e;
    }
}

cudaError_t launch_near_sum(tdbem_ctx *c, int alpha, const double *d_exc)
{
    k_near_sum<<<c->ns, kNearThreads, 0, c->s>>>(c->ns, c->nblk, alpha, c->d_meta, c->d_boff, c->d_ku, c->d_kw,
                                                c->d_u, c->d_q, d_exc, c->inc, c->d_xc, c->d_n, c->d_b);
    return cudaGetLastError();
}

// One Jacobi sweep x' = D^-1 (b - R x) of the zero-lag system (A = D + R,
// R in the ELL store).  it = 0 starts from x = D^-1 b.  The last sweep adds
// the solution to the unknown component of step a-1 (u where phi = 1, q
// where phi = 0) and flags a non-finite value (flag bit 1).
__global__ void k_jacobi(int ns, const double *__restrict__ aoff, const int32_t *__restrict__ acol,
                         const double *__restrict__ ainv, const double *__restrict__ b,
                         const double *__restrict__ xin, double *xout, int last, int64_t row,
                         const int8_t *__restrict__ phi, double *u, double *q, int *flag)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns) return;
    double s = b[i];
    if (xin) {
#pragma unroll
        for (int k = 0; k < kEllWidth; ++k) {
            int cidx = acol[(int64_t)k * ns + i];
            if (cidx >= 0) s -= aoff[(int64_t)k * ns + i] * xin[cidx];
        }
    }
    double x = s * ainv[i];
    if (last) {
        if (phi[i])
            u[row + i] += x;
        else
            q[row + i] += x;
        if (!isfinite(x)) atomicOr(flag, 1);
    } else {
        xout[i] = x;
    }
}

cudaError_t launch_jacobi(tdbem_ctx *c, int alpha, int it, int last)
{
    const double *xin = (it == 0) ? nullptr : ((it & 1) ? c->d_xa : c->d_xb);
    double *xout = (it & 1) ? c->d_xb : c->d_xa;
    int64_t row = (int64_t)(alpha - 1) * c->ns;
    k_jacobi<<<(c->ns + 127) / 128, 128, 0, c->s>>>(c->ns, c->d_aoff, c->d_acol, c->d_ainv, c->d_b, xin, xout, last,
                                                   row, c->d_phi, c->d_u, c->d_q, c->d_flag);
    return cudaGetLastError();
}

// x[n][i] = x_i^{a0+n}: u where phi_i = 1, q where phi_i = 0.
__global__ void k_gather_x(int ns, int nsteps, int a0, const int8_t *__restrict__ phi,
                           const double *__restrict__ u, const double *__restrict__ q, double *x)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= (int64_t)nsteps * ns) return;
    int i = (int)(k % ns);
    int64_t h = (int64_t)a0 * ns + k;
    x[k] = phi[i] ? u[h] : q[h];
}

cudaError_t launch_gather_x(tdbem_ctx *c, int a0, int nsteps, double *x)
{
    int64_t n = (int64_t)nsteps * c->ns;
    k_gather_x<<<(int)((n + 255) / 256), 256, 0, c->s>>>(c->ns, nsteps, a0, c->d_phi, c->d_u, c->d_q, x);
    return cudaGetLastError();
}

}  // namespace tdbem
