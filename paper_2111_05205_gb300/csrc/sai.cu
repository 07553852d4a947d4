// Learned sparse approximate inverse (SAI) for the zero-lag system of
// Eq. linear.  The paper only says the system is sparse and solved every
// step; this component is an addition of this library.
//
// For row i of A (pattern: the diagonal and the off-diagonal entries of the
// ELL store, at most W slots) a small network maps per-slot features to the
// row of a left SAI M on the same pattern; the zero-lag solve then runs
// preconditioned Richardson sweeps x <- x + M (b - A x) instead of Jacobi
// sweeps (Jacobi is M = D^-1).  Features of slot k (k = 0: the diagonal;
// then the off-diagonal entries by decreasing |A_ij|): A_ij/A_ii, A_jj/A_ii,
// A_ji/A_ii (what the first Neumann term -A_ij/(A_ii A_jj) of A^-1 and the
// symmetry of the pattern depend on), the distance |x_i - x_j| / (c dt) and
// a validity flag.  Network: in = 5W ->
// hidden H (ReLU) -> W outputs o_k, M_ij = o_k / A_ii.  FP16 weights, FP32
// arithmetic.  Training minimises sum_i || e_i^T - m_i^T A ||^2 over rows
// of zero-lag matrices the method assembles, with hand-written forward,
// backward and Adam kernels.
#include <cuda_fp16.h>

#include <algorithm>

#include "tdbem_internal.cuh"

namespace tdbem {

constexpr int kSaiMaxW = 16;
constexpr int kSaiMaxH = 64;

constexpr int kSaiF = 5;  // features per slot

struct SaiRow {
    int n;                 // valid slots (diagonal first)
    int col[kSaiMaxW];
    float feat[kSaiF * kSaiMaxW];
    double inv_diag;
};

// Entry A_jl (l any column) from the ELL store.
__device__ __forceinline__ double a_entry(int j, int l, int ns, int ell_w, const double *aoff, const int32_t *acol,
                                          const double *ainv)
{
    if (j == l) return 1.0 / ainv[j];
    for (int k = 0; k < ell_w; ++k)
        if (acol[(int64_t)k * ns + j] == l) return aoff[(int64_t)k * ns + j];
    return 0.0;
}

// Slots of row i in the canonical order: the diagonal, then off-diagonal
// entries with |A_ij| >= 1e-12 |A_ii| by decreasing magnitude quantised to
// 2^-20 of |A_ii| (ties by column), so that entries equal up to rounding --
// common on symmetric meshes -- keep one order on every implementation.  Features of slot k (column j): A_ij/A_ii, A_jj/A_ii, A_ji/A_ii,
// |x_i - x_j|/(c dt), 1.
__device__ __forceinline__ long long sai_key(double v, double ainv_i)
{
    return (long long)floor(fabs(v * ainv_i) * 1048576.0);
}

__device__ void sai_row(int i, int ns, int ell_w, int W, const double *aoff, const int32_t *acol,
                        const double *ainv, const double *xc, double cdt, SaiRow &R)
{
    double ad = 1.0 / ainv[i];
    int cols[kSaiMaxW];
    double vals[kSaiMaxW];
    long long keys[kSaiMaxW];
    keys[0] = 0;
    int n = 0;
    cols[n] = i;
    vals[n++] = ad;
    for (int k = 0; k < ell_w && n < W; ++k) {
        int j = acol[(int64_t)k * ns + i];
        if (j < 0) continue;
        double v = aoff[(int64_t)k * ns + i];
        if (!(fabs(v) >= 1e-12 * fabs(ad))) continue;
        long long kv = sai_key(v, ainv[i]);
        int p = n++;
        while (p > 1 && (keys[p - 1] < kv || (keys[p - 1] == kv && cols[p - 1] > j))) {
            vals[p] = vals[p - 1];
            cols[p] = cols[p - 1];
            keys[p] = keys[p - 1];
            --p;
        }
        vals[p] = v;
        cols[p] = j;
        keys[p] = kv;
    }
    R.n = n;
    R.inv_diag = ainv[i];
    for (int k = 0; k < W; ++k) {
        bool ok = k < n;
        R.col[k] = ok ? cols[k] : -1;
        double dx = 0, dy = 0, dz = 0;
        if (ok) {
            dx = xc[3 * i] - xc[3 * cols[k]];
            dy = xc[3 * i + 1] - xc[3 * cols[k] + 1];
            dz = xc[3 * i + 2] - xc[3 * cols[k] + 2];
        }
        float *f = R.feat + kSaiF * k;
        f[0] = ok ? (float)(vals[k] * ainv[i]) : 0.f;
        f[1] = ok ? (float)(ainv[i] / ainv[cols[k]]) : 0.f;
        f[2] = ok ? (float)(a_entry(cols[k], i, ns, ell_w, aoff, acol, ainv) * ainv[i]) : 0.f;
        f[3] = ok ? (float)(sqrt(dx * dx + dy * dy + dz * dz) / cdt) : 0.f;
        f[4] = ok ? 1.f : 0.f;
    }
}

// Analytic part of the SAI row: Jacobi on the diagonal and the first
// Neumann term -A_ij/(A_ii A_jj) off it, in units of 1/A_ii (the network
// learns a correction to it).
__device__ __forceinline__ float sai_base(int k, const float *f)
{
    if (f[kSaiF * k + 4] == 0.f) return 0.f;
    return k == 0 ? 1.f : -f[kSaiF * k] / f[kSaiF * k + 1];
}

// Forward pass of one row: hidden activations h and outputs o (including
// the analytic part).
__device__ void sai_forward(int W, int H, const __half *w1, const __half *b1, const __half *w2, const __half *b2,
                            const float *in, float *h, float *o)
{
    const int F = kSaiF * W;
    for (int a = 0; a < H; ++a) {
        float s = __half2float(b1[a]);
        for (int f = 0; f < F; ++f) s += __half2float(w1[a * F + f]) * in[f];
        h[a] = s > 0.f ? s : 0.f;
    }
    for (int k = 0; k < W; ++k) {
        float s = __half2float(b2[k]);
        for (int a = 0; a < H; ++a) s += __half2float(w2[k * H + a]) * h[a];
        o[k] = s + sai_base(k, in);
    }
}

// Loss and gradient contributions of row i, added to grad[] and *loss.
__device__ void sai_row_grad(int i, int ns, int ell_w, int W, int H, const double *__restrict__ aoff,
                             const int32_t *__restrict__ acol, const double *__restrict__ ainv,
                             const double *__restrict__ xc, double cdt, const __half *__restrict__ w16, float *grad,
                             float *loss)
{
    const int F = kSaiF * W;
    const __half *w1 = w16, *b1 = w1 + H * F, *w2 = b1 + H, *b2 = w2 + W * H;
    float *g1 = grad, *gb1 = g1 + H * F, *g2 = gb1 + H, *gb2 = g2 + W * H;
    SaiRow R;
    sai_row(i, ns, ell_w, W, aoff, acol, ainv, xc, cdt, R);
    float h[kSaiMaxH], o[kSaiMaxW];
    sai_forward(W, H, w1, b1, w2, b2, R.feat, h, o);
    // residual over the union of the columns of rows j_k
    int lc[kSaiMaxW * (kSaiMaxW + 1)];
    double lv[kSaiMaxW * (kSaiMaxW + 1)];
    int nl = 0;
    auto add = [&](int l, double v) {
        for (int t = 0; t < nl; ++t)
            if (lc[t] == l) {
                lv[t] += v;
                return;
            }
        lc[nl] = l;
        lv[nl++] = v;
    };
    add(i, -1.0);
    for (int k = 0; k < R.n; ++k) {
        int j = R.col[k];
        double m = o[k] * R.inv_diag;
        add(j, m / ainv[j]);
        for (int e = 0; e < ell_w; ++e) {
            int l = acol[(int64_t)e * ns + j];
            if (l >= 0) add(l, m * aoff[(int64_t)e * ns + j]);
        }
    }
    double L = 0.0;
    for (int t = 0; t < nl; ++t) L += lv[t] * lv[t];
    atomicAdd(loss, (float)L);
    // dL/do_k = 2 sum_l r_l A_{j_k, l} / A_ii
    float go[kSaiMaxW];
    for (int k = 0; k < W; ++k) {
        go[k] = 0.f;
        if (k >= R.n) continue;
        double s = 0.0;
        for (int t = 0; t < nl; ++t) s += lv[t] * a_entry(R.col[k], lc[t], ns, ell_w, aoff, acol, ainv);
        go[k] = (float)(2.0 * s * R.inv_diag);
    }
    for (int k = 0; k < W; ++k) {
        if (go[k] == 0.f) continue;
        atomicAdd(&gb2[k], go[k]);
        for (int a = 0; a < H; ++a)
            if (h[a] != 0.f) atomicAdd(&g2[k * H + a], go[k] * h[a]);
    }
    for (int a = 0; a < H; ++a) {
        if (h[a] <= 0.f) continue;
        float gh = 0.f;
        for (int k = 0; k < W; ++k) gh += __half2float(w2[k * H + a]) * go[k];
        if (gh == 0.f) continue;
        atomicAdd(&gb1[a], gh);
        for (int f = 0; f < F; ++f)
            if (R.feat[f] != 0.f) atomicAdd(&g1[a * F + f], gh * R.feat[f]);
    }
}

// One training pass over the rows of one matrix: loss of every row and the
// gradients of the weights (FP32).  Residual of row i: r_l = sum_k
// M_{i,j_k} A_{j_k, l} - delta_il over the columns l of the rows j_k.  The
// CTA's rows add their gradients in shared memory (nw floats), then the CTA
// adds its sums to the global gradient, one atomic per non-zero weight.
__global__ void k_sai_train_rows(int ns, int ell_w, int W, int H, int nw, const double *__restrict__ aoff,
                                 const int32_t *__restrict__ acol, const double *__restrict__ ainv,
                                 const double *__restrict__ xc, double cdt, const __half *__restrict__ w16,
                                 float *grad, float *loss)
{
    extern __shared__ float gsh[];  // [nw] gradient, [1] loss
    for (int e = threadIdx.x; e <= nw; e += blockDim.x) gsh[e] = 0.f;
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ns) sai_row_grad(i, ns, ell_w, W, H, aoff, acol, ainv, xc, cdt, w16, gsh, gsh + nw);
    __syncthreads();
    for (int e = threadIdx.x; e <= nw; e += blockDim.x) {
        const float v = gsh[e];
        if (v != 0.f) atomicAdd(e < nw ? grad + e : loss, v);
    }
}

// Adam on the FP32 master weights; FP16 copies for the forward pass.
__global__ void k_sai_adam(int n, float *w, float *m, float *v, const float *grad, float scale, float lr, float b1,
                           float b2, float eps, int t, __half *w16)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    float g = grad[e] * scale;
    m[e] = b1 * m[e] + (1.f - b1) * g;
    v[e] = b2 * v[e] + (1.f - b2) * g * g;
    float mh = m[e] / (1.f - powf(b1, (float)t)), vh = v[e] / (1.f - powf(b2, (float)t));
    w[e] -= lr * mh / (sqrtf(vh) + eps);
    w16[e] = __float2half(w[e]);
}

// M of a context on the pattern of A (ELL store: [W][ns] values, columns).
__global__ void k_sai_apply_net(int ns, int ell_w, int W, int H, const double *__restrict__ aoff,
                                const int32_t *__restrict__ acol, const double *__restrict__ ainv,
                                const double *__restrict__ xc, double cdt, const __half *__restrict__ w16, double *mval,
                                int32_t *mcol)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns) return;
    const int F = kSaiF * W;
    const __half *w1 = w16, *b1 = w1 + H * F, *w2 = b1 + H, *b2 = w2 + W * H;
    SaiRow R;
    sai_row(i, ns, ell_w, W, aoff, acol, ainv, xc, cdt, R);
    float h[kSaiMaxH], o[kSaiMaxW];
    sai_forward(W, H, w1, b1, w2, b2, R.feat, h, o);
    for (int k = 0; k < W; ++k) {
        mval[(int64_t)k * ns + i] = (k < R.n) ? (double)o[k] * R.inv_diag : 0.0;
        mcol[(int64_t)k * ns + i] = R.col[k];
    }
}

// The preconditioned sweeps x_{k+1} = x_k + M (b - A x_k), x_0 = M b, are
// run as x_0 = c = M b, x_{k+1} = c + G x_k with G = I - M A formed once
// when the SAI is installed (ELL store [gw][ns]): one gather per entry of G
// instead of recomputing rows of A x for every entry of M.
__device__ __forceinline__ double sai_mb(int i, int ns, int W, const double *__restrict__ mval,
                                         const int32_t *__restrict__ mcol, const double *__restrict__ b)
{
    double s = 0.0;
    for (int k = 0; k < W; ++k) {
        const int j = mcol[(int64_t)k * ns + i];
        if (j >= 0) s += mval[(int64_t)k * ns + i] * b[j];
    }
    return s;
}

template <typename LDX>
__device__ __forceinline__ double sai_g_row(int i, int ns, int gw, const double *__restrict__ gval,
                                            const int32_t *__restrict__ gcol, const double *__restrict__ cb,
                                            const double *x, LDX ldx)
{
    double s = cb[i];
    // four entries at a time (columns and values, then the gathers of x)
    int k = 0;
    for (; k + 4 <= gw; k += 4) {
        int l[4];
        double g[4], xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            l[u] = gcol[(int64_t)(k + u) * ns + i];
            g[u] = gval[(int64_t)(k + u) * ns + i];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) xv[u] = l[u] >= 0 ? ldx(x + l[u]) : 0.0;
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (l[u] >= 0) s += g[u] * xv[u];
    }
    for (; k < gw; ++k) {
        const int l = gcol[(int64_t)k * ns + i];
        if (l >= 0) s += gval[(int64_t)k * ns + i] * ldx(x + l);
    }
    return s;
}

// The last sweep adds x_K to the unknown component of step a-1 and flags a
// non-finite value (flag bit 1).
__device__ __forceinline__ void sai_store(int i, double s, int64_t row, const int8_t *__restrict__ phi, double *u,
                                          double *q, float2 *us, float2 *qs, const int32_t *__restrict__ hpos,
                                          int *flag)
{
    double *hh = phi[i] ? u : q;
    double v = hh[row + i] + s;
    hh[row + i] = v;
    if (us) {
        float hi = __double2float_rn(v);
        (phi[i] ? us : qs)[row + (hpos ? hpos[i] : i)] = make_float2(hi, __double2float_rn(v - (double)hi));
    }
    if (!isfinite(s)) atomicOr(flag, 1);
}

// One sweep per launch: it = 0 forms c = M b (x_0 = c); it > 0 one step of
// x = c + G x; the last sweep stores.
__global__ void k_sai_sweep(int ns, int W, int gw, const double *__restrict__ mval, const int32_t *__restrict__ mcol,
                            const double *__restrict__ gval, const int32_t *__restrict__ gcol,
                            const double *__restrict__ b, double *cb, const double *__restrict__ x, double *xout,
                            int first, int last, int64_t row, const int8_t *__restrict__ phi, double *u, double *q,
                            float2 *us, float2 *qs, const int32_t *__restrict__ hpos, int *flag)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns) return;
    double s;
    if (first) {
        s = sai_mb(i, ns, W, mval, mcol, b);
        cb[i] = s;
    } else {
        s = sai_g_row(i, ns, gw, gval, gcol, cb, x, [](const double *p) { return *p; });
    }
    if (last)
        sai_store(i, s, row, phi, u, q, us, qs, hpos, flag);
    else
        xout[i] = s;
}

// All K sweeps of one step in one cooperative launch (rows grid-strided),
// a bounded grid barrier between sweeps (x read with ld.global.cg, as in
// the fused Jacobi solve); the same arithmetic as K launches of k_sai_sweep.
__global__ void __launch_bounds__(256) k_sai_fused(int ns, int W, int gw, const double *__restrict__ mval,
                                                   const int32_t *__restrict__ mcol, const double *__restrict__ gval,
                                                   const int32_t *__restrict__ gcol, const double *__restrict__ b,
                                                   double *cb, double *xa, double *xb, int K, int64_t row,
                                                   const int8_t *__restrict__ phi, double *u, double *q, float2 *us,
                                                   float2 *qs, const int32_t *__restrict__ hpos, int *flag,
                                                   unsigned *bar)
{
    for (int it = 0; it < K; ++it) {
        const double *xin = (it & 1) ? xa : xb;
        double *xout = (it & 1) ? xb : xa;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += gridDim.x * blockDim.x) {
            double s;
            if (it == 0) {
                s = sai_mb(i, ns, W, mval, mcol, b);
                cb[i] = s;
            } else {
                s = sai_g_row(i, ns, gw, gval, gcol, cb, xin, [](const double *p) { return __ldcg(p); });
            }
            if (it == K - 1)
                sai_store(i, s, row, phi, u, q, us, qs, hpos, flag);
            else
                xout[i] = s;
        }
        if (it < K - 1) grid_barrier(bar, flag);
    }
}

}  // namespace tdbem

struct tdbem_sai {
    int W = 0, H = 0, nw = 0, t = 0;
    float *w = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr, *loss = nullptr;
    __half *w16 = nullptr;
    std::string err;
};

using namespace tdbem;

namespace {

int sai_fail(tdbem_sai *S, int code, const std::string &m)
{
    if (S) S->err = m;
    return code;
}

// Deterministic weight initialisation (splitmix64 -> uniform +-sqrt(6/(fan_in+fan_out))).
uint64_t splitmix(uint64_t &x)
{
    uint64_t z = (x += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

}  // namespace

extern "C" {

int tdbem_sai_create(int32_t width, int32_t hidden, uint64_t seed, tdbem_sai **out)
{
    if (!out || width < 2 || width > kSaiMaxW || hidden < 1 || hidden > kSaiMaxH) return TDBEM_ERR_ARG;
    tdbem_sai *S = new tdbem_sai();
    S->W = width;
    S->H = hidden;
    const int F = kSaiF * width;
    S->nw = hidden * F + hidden + width * hidden + width;
    std::vector<float> w(S->nw, 0.f);
    uint64_t st = seed;
    float a1 = sqrtf(6.f / (F + hidden)), a2 = sqrtf(6.f / (hidden + width));
    for (int e = 0; e < hidden * F; ++e) w[e] = a1 * (2.f * (float)((splitmix(st) >> 11) * 0x1.0p-53) - 1.f);
    for (int e = 0; e < width * hidden; ++e)
        w[hidden * F + hidden + e] = a2 * (2.f * (float)((splitmix(st) >> 11) * 0x1.0p-53) - 1.f);
    // the output layer starts small: M starts at the analytic first-order
    // Neumann SAI
    for (int e = 0; e < width * hidden; ++e) w[hidden * F + hidden + e] *= 0.01f;
    std::vector<__half> w16(S->nw);
    for (int e = 0; e < S->nw; ++e) w16[e] = __float2half(w[e]);
    bool ok = cudaMalloc(&S->w, S->nw * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&S->m, S->nw * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&S->v, S->nw * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&S->grad, S->nw * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&S->loss, sizeof(float)) == cudaSuccess &&
              cudaMalloc(&S->w16, S->nw * sizeof(__half)) == cudaSuccess;
    if (ok) {
        cudaMemcpy(S->w, w.data(), S->nw * sizeof(float), cudaMemcpyHostToDevice);
        cudaMemcpy(S->w16, w16.data(), S->nw * sizeof(__half), cudaMemcpyHostToDevice);
        cudaMemset(S->m, 0, S->nw * sizeof(float));
        cudaMemset(S->v, 0, S->nw * sizeof(float));
    }
    if (!ok) {
        tdbem_sai_destroy(S);
        return TDBEM_ERR_OOM;
    }
    *out = S;
    return TDBEM_OK;
}

void tdbem_sai_destroy(tdbem_sai *S)
{
    if (!S) return;
    cudaFree(S->w);
    cudaFree(S->m);
    cudaFree(S->v);
    cudaFree(S->grad);
    cudaFree(S->loss);
    cudaFree(S->w16);
    delete S;
}

const char *tdbem_sai_last_error(const tdbem_sai *S) { return S ? S->err.c_str() : "null trainer"; }

int tdbem_sai_weights(tdbem_sai *S, float *inout, int64_t *count, int32_t set)
{
    if (!S || !count) return TDBEM_ERR_ARG;
    *count = S->nw;
    if (!inout) return TDBEM_OK;
    if (set) {
        std::vector<__half> w16(S->nw);
        for (int e = 0; e < S->nw; ++e) w16[e] = __float2half(inout[e]);
        if (cudaMemcpy(S->w, inout, S->nw * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(S->w16, w16.data(), S->nw * sizeof(__half), cudaMemcpyHostToDevice) != cudaSuccess)
            return sai_fail(S, TDBEM_ERR_CUDA, "weight upload");
        cudaMemset(S->m, 0, S->nw * sizeof(float));
        cudaMemset(S->v, 0, S->nw * sizeof(float));
        S->t = 0;
    } else {
        // the FP16 weights the network computes with, as floats
        std::vector<__half> w16(S->nw);
        if (cudaMemcpy(w16.data(), S->w16, S->nw * sizeof(__half), cudaMemcpyDeviceToHost) != cudaSuccess)
            return sai_fail(S, TDBEM_ERR_CUDA, "weight download");
        for (int e = 0; e < S->nw; ++e) inout[e] = __half2float(w16[e]);
    }
    return TDBEM_OK;
}

static int sai_pass(tdbem_sai *S, tdbem_ctx *c, float *loss_host)
{
    if (!c || !c->prepared || !c->d_aoff) return sai_fail(S, TDBEM_ERR_STATE, "context not prepared");
    cudaMemsetAsync(S->grad, 0, S->nw * sizeof(float), c->s);
    cudaMemsetAsync(S->loss, 0, sizeof(float), c->s);
    k_sai_train_rows<<<(c->ns + 127) / 128, 128, (S->nw + 1) * sizeof(float), c->s>>>(
        c->ns, c->ell_w, S->W, S->H, S->nw, c->d_aoff, c->d_acol, c->d_ainv, c->d_xc, c->cdt, S->w16, S->grad,
        S->loss);
    if (cudaGetLastError() != cudaSuccess) return sai_fail(S, TDBEM_ERR_CUDA, "training kernel");
    if (loss_host) cudaMemcpyAsync(loss_host, S->loss, sizeof(float), cudaMemcpyDeviceToHost, c->s);
    return TDBEM_OK;
}

// Loss and gradient of one context's rows at the current weights (no update).
int tdbem_sai_gradient(tdbem_sai *S, tdbem_ctx *c, float *grad, float *loss)
{
    if (!S || !grad || !loss) return TDBEM_ERR_ARG;
    int r = sai_pass(S, c, loss);
    if (r != TDBEM_OK) return r;
    if (cudaMemcpyAsync(grad, S->grad, S->nw * sizeof(float), cudaMemcpyDeviceToHost, c->s) != cudaSuccess ||
        cudaStreamSynchronize(c->s) != cudaSuccess)
        return sai_fail(S, TDBEM_ERR_CUDA, "gradient download");
    return TDBEM_OK;
}

// Adam over the contexts' rows for `epochs` passes (one update per context
// and pass, gradient scaled by 1/ns); loss_out: mean row loss of the last pass.
int tdbem_sai_train(tdbem_sai *S, tdbem_ctx *const *ctxs, int32_t n, int32_t epochs, float lr, float *loss_out)
{
    if (!S || !ctxs || n < 1 || epochs < 1) return TDBEM_ERR_ARG;
    double tot = 0.0;
    int64_t rows = 0;
    for (int ep = 0; ep < epochs; ++ep) {
        tot = 0.0;
        rows = 0;
        for (int k = 0; k < n; ++k) {
            tdbem_ctx *c = ctxs[k];
            float L = 0.f;
            int r = sai_pass(S, c, &L);
            if (r != TDBEM_OK) return r;
            S->t += 1;
            k_sai_adam<<<(S->nw + 255) / 256, 256, 0, c->s>>>(S->nw, S->w, S->m, S->v, S->grad, 1.f / c->ns, lr,
                                                              0.9f, 0.999f, 1e-8f, S->t, S->w16);
            if (cudaStreamSynchronize(c->s) != cudaSuccess) return sai_fail(S, TDBEM_ERR_CUDA, "training step");
            tot += L;
            rows += c->ns;
        }
    }
    if (loss_out) *loss_out = (float)(tot / rows);
    return TDBEM_OK;
}

// Installs the learned M as the zero-lag solver of a context when its
// a-priori sweep count (||I - M A||_inf = q': error <= q'^K) is below
// Jacobi's; otherwise Jacobi stays (the fallback).
// *sweeps receives the sweeps of the solver in use, *contraction its q.
int tdbem_set_precond(tdbem_ctx *c, const tdbem_sai *S, int32_t *use_sai, int32_t *sweeps, double *contraction)
{
    if (!c || !S) return TDBEM_ERR_ARG;
    if (!c->prepared) return TDBEM_ERR_STATE;
    if (c->P.precond == 0) {
        c->err = "the context was created with precond = 0 (Jacobi only)";
        return TDBEM_ERR_STATE;
    }
    const int ns = c->ns, W = S->W, E = c->ell_w;
    double *mval = nullptr;
    int32_t *mcol = nullptr;
    if (cudaMalloc(&mval, (size_t)W * ns * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&mcol, (size_t)W * ns * sizeof(int32_t)) != cudaSuccess)
        return TDBEM_ERR_OOM;
    c->allocs.push_back(mval);
    c->allocs.push_back(mcol);
    k_sai_apply_net<<<(ns + 127) / 128, 128, 0, c->s>>>(ns, E, W, S->H, c->d_aoff, c->d_acol, c->d_ainv, c->d_xc,
                                                         c->cdt, S->w16, mval, mcol);
    std::vector<double> mv((size_t)W * ns), av((size_t)E * ns), ai(ns);
    std::vector<int32_t> mc((size_t)W * ns), ac((size_t)E * ns);
    cudaMemcpyAsync(mv.data(), mval, mv.size() * sizeof(double), cudaMemcpyDeviceToHost, c->s);
    cudaMemcpyAsync(mc.data(), mcol, mc.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, c->s);
    cudaMemcpyAsync(av.data(), c->d_aoff, av.size() * sizeof(double), cudaMemcpyDeviceToHost, c->s);
    cudaMemcpyAsync(ac.data(), c->d_acol, ac.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, c->s);
    cudaMemcpyAsync(ai.data(), c->d_ainv, ai.size() * sizeof(double), cudaMemcpyDeviceToHost, c->s);
    if (cudaStreamSynchronize(c->s) != cudaSuccess) return TDBEM_ERR_CUDA;
    // q' = max_i sum_l |delta_il - (M A)_il|, and the rows of G = I - M A
    double qmax = 0.0;
    std::vector<std::pair<int, double>> acc;
    std::vector<std::vector<std::pair<int, double>>> grows(ns);
    for (int i = 0; i < ns; ++i) {
        acc.clear();
        auto add = [&](int l, double v) {
            for (auto &p : acc)
                if (p.first == l) {
                    p.second += v;
                    return;
                }
            acc.push_back({l, v});
        };
        add(i, -1.0);
        for (int k = 0; k < W; ++k) {
            int j = mc[(size_t)k * ns + i];
            if (j < 0) continue;
            double m = mv[(size_t)k * ns + i];
            add(j, m / ai[j]);
            for (int e = 0; e < E; ++e) {
                int l = ac[(size_t)e * ns + j];
                if (l >= 0) add(l, m * av[(size_t)e * ns + j]);
            }
        }
        double s = 0.0;
        for (auto &p : acc) s += fabs(p.second);
        qmax = std::max(qmax, s);
        for (auto &p : acc)
            if (p.second != 0.0) grows[i].push_back({p.first, -p.second});
    }
    double tol = c->P.solver_tol > 0 ? c->P.solver_tol : 1e-16;
    int K = (qmax > 0.0 && qmax < 1.0) ? std::max(1, (int)ceil(log(tol) / log(qmax))) : 1 << 30;
    // one launch per sweep for either solver
    bool better = qmax < 1.0 && K < c->solve_iters;
    if (better) {
        // G in an ELL store [gw][ns] (unused slots: column -1)
        size_t gw = 1;
        for (auto &r : grows) gw = std::max(gw, r.size());
        std::vector<double> gv(gw * ns, 0.0);
        std::vector<int32_t> gc(gw * ns, -1);
        for (int i = 0; i < ns; ++i)
            for (size_t k = 0; k < grows[i].size(); ++k) {
                gc[k * ns + i] = grows[i][k].first;
                gv[k * ns + i] = grows[i][k].second;
            }
        double *gval = nullptr, *cb = nullptr;
        int32_t *gcol = nullptr;
        if (cudaMalloc(&gval, gv.size() * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&gcol, gc.size() * sizeof(int32_t)) != cudaSuccess ||
            cudaMalloc(&cb, (size_t)ns * sizeof(double)) != cudaSuccess)
            return TDBEM_ERR_OOM;
        c->allocs.push_back(gval);
        c->allocs.push_back(gcol);
        c->allocs.push_back(cb);
        if (cudaMemcpy(gval, gv.data(), gv.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(gcol, gc.data(), gc.size() * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess)
            return TDBEM_ERR_CUDA;
        c->sai_gval = gval;
        c->sai_gcol = gcol;
        c->sai_gw = (int)gw;
        c->sai_cb = cb;
        c->sai_val = mval;
        c->sai_col = mcol;
        c->sai_w = W;
        c->sai_iters = K;
        c->sai_contraction = qmax;
        // the K sweeps in one cooperative launch where the device allows it
        c->sai_grid = 0;
        int coop = 0, nsm = 0, per = 0;
        if (c->d_bar && cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->dev) == cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sai_fused, 256, 0) == cudaSuccess && coop &&
            per >= 1)
            c->sai_grid = (int)std::min<int64_t>(((int64_t)ns + 255) / 256, (int64_t)per * nsm);
    }
    if (use_sai) *use_sai = better ? 1 : 0;
    if (sweeps) *sweeps = better ? K : c->solve_iters;
    if (contraction) *contraction = qmax;
    return TDBEM_OK;
}

}  // extern "C"

namespace tdbem {

// The SAI-preconditioned zero-lag solve of one step: all K sweeps in one
// cooperative launch.
cudaError_t launch_sai_fused(tdbem_ctx *c, int alpha)
{
    int ns = c->ns, W = c->sai_w, gw = c->sai_gw, K = c->sai_iters;
    int64_t row = (int64_t)(alpha - 1) * ns;
    void *args[] = {&ns, &W, &gw, &c->sai_val, &c->sai_col, &c->sai_gval, &c->sai_gcol, &c->d_b, &c->sai_cb,
                    &c->d_xa, &c->d_xb, &K, &row, &c->d_phi, &c->d_u, &c->d_q, &c->d_us, &c->d_qs, &c->d_hpos,
                    &c->d_flag, &c->d_bar};
    return cudaLaunchCooperativeKernel((const void *)k_sai_fused, dim3(c->sai_grid), dim3(256), args, 0, c->s);
}

// The SAI-preconditioned zero-lag solve of one step (sweep it of K).
cudaError_t launch_sai_sweep(tdbem_ctx *c, int alpha, int it)
{
    const int ns = c->ns;
    const bool last = (it == c->sai_iters - 1);
    const double *xin = (it & 1) ? c->d_xa : c->d_xb;
    double *xout = (it & 1) ? c->d_xb : c->d_xa;
    int64_t row = (int64_t)(alpha - 1) * ns;
    k_sai_sweep<<<(ns + 127) / 128, 128, 0, c->s>>>(ns, c->sai_w, c->sai_gw, c->sai_val, c->sai_col, c->sai_gval,
                                                    c->sai_gcol, c->d_b, c->sai_cb, xin, xout, it == 0, last, row,
                                                    c->d_phi, c->d_u, c->d_q, c->d_us, c->d_qs, c->d_hpos,
                                                    c->d_flag);
    return cudaGetLastError();
}

}  // namespace tdbem
