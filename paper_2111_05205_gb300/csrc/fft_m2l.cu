// FFT form of the near-future M2L (Section 4: the complexity estimate after
// Algorithm 1 applies the M2L through the FFT).
//
// With equispaced interpolation nodes and the observation box equal to the
// source box (half-width h), the node differences of an interaction pair are
// x_a - y_b = -(S - O) s + h (w_a - w_b) and t_m - s_n = l T dt + dt +
// h_t (w_m - w_n), functions of a - b and m - n only: every near-future
// block U_l (l = 1..mu) of a cell offset is a four-level Toeplitz matrix.
// Embedded in a circulant of Ns = 2 ps points per spatial axis and Nt = 2 pt
// in time, it acts as a circular convolution, so
//   L_{k+l}(O) += IFFT( sum_{S in IL(O)} FFT(u_{S-O,l}) . FFT(M_k(S)) )
// restricted to the first ps^3 x pt grid points.  The sum over the
// interaction list is taken between the transforms, so each cell's moment
// is transformed once per interval and each (cell, block) local once.
//
// Grid index g = f1 + Ns (f2 + Ns (f3 + Ns ft)) (the vector index of moments
// and locals, b1 + ps (b2 + ps (b3 + ps n)), zero-padded).  Transforms and
// products run in FP32 on the CUDA cores; the locals stay FP64.
//   k_fft_fwd:  one CTA per cell: time axis first (pt nonzero inputs of Nt),
//               then per time frequency the three spatial axes in shared
//               memory; writes Mhat [nc][N].
//   k_fft_mul:  one CTA per C frequencies: the moments' and the current
//               block's kernel spectra of those frequencies in shared memory,
//               a warp per observation cell summing its pairs; writes Yhat
//               [nc][mu][N].
//   k_fft_inv:  one CTA per (cell, block): per time frequency the three
//               spatial axes (only the ps outputs each), then the time axis
//               (only the pt outputs), added into the FP64 ring of locals.
// The spectra of the kernel samples are formed at set-up with axis passes
// through global memory (k_fft_samples, k_dft_axis).
#include <math.h>

#include <algorithm>

#include "tdbem_internal.cuh"

namespace tdbem {

namespace {

constexpr int kFftThreads = 256;
constexpr int kFftMaxN = 16;                    // 2 x the largest order
constexpr size_t kFftMulSmem = 200 * 1024;      // shared memory of one products CTA

__device__ __forceinline__ float2 cfma(float2 acc, float2 a, float2 b)
{
    acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
    return acc;
}

// e^{sign 2 pi i j / n}, j = 0..n-1, into tw (the CTA's threads share it)
__device__ __forceinline__ void twiddles(float2 *tw, int n, int sign)
{
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double sn, cs;
        sincospi(2.0 * j / n, &sn, &cs);
        tw[j] = make_float2((float)cs, (float)(sign * sn));
    }
}

// Index difference at circular position f of an N-point axis (N = 2p):
// 0..p-1 at f = 0..p-1, -(p-1)..-1 at f = p+1..2p-1; position p is unused.
__device__ __forceinline__ bool circ_diff(int f, int p, int N, int *D)
{
    if (f < p) {
        *D = f;
        return true;
    }
    if (f > N - p) {
        *D = f - N;
        return true;
    }
    return false;
}

// Circulant samples of the near-future kernel blocks of each offset:
// out[o][blk][g] = U(-(S - O) s + hsp D_s, (blk + 1) T dt + dt + htp D_t),
// U(r, tau) = (c tau - r)_+^d / r, hsp and htp the node spacings.
__global__ void k_fft_samples(int nfo, int nbl, int ps, int pt, int Ns, int Nt, double s, double h, double Tdt,
                              double dt, double c, int d, const int32_t *__restrict__ codes, float2 *out)
{
    const int64_t N = (int64_t)Ns * Ns * Ns * Nt;
    const int64_t total = (int64_t)nfo * nbl * N;
    const double hsp = ps > 1 ? 2.0 * h / (ps - 1) : 0.0, htp = pt > 1 ? Tdt / (pt - 1) : 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = e % N;
        const int64_t r1 = e / N;
        const int blk = (int)(r1 % nbl);
        const int o = codes[r1 / nbl];
        const int dx = o % 7 - 3, dy = (o / 7) % 7 - 3, dz = o / 49 - 3;
        const int f1 = (int)(g % Ns), f2 = (int)((g / Ns) % Ns), f3 = (int)((g / ((int64_t)Ns * Ns)) % Ns),
                  ft = (int)(g / ((int64_t)Ns * Ns * Ns));
        int D1, D2, D3, Dt;
        float v = 0.f;
        if (circ_diff(f1, ps, Ns, &D1) && circ_diff(f2, ps, Ns, &D2) && circ_diff(f3, ps, Ns, &D3) &&
            circ_diff(ft, pt, Nt, &Dt)) {
            const double rx = -dx * s + hsp * D1, ry = -dy * s + hsp * D2, rz = -dz * s + hsp * D3;
            const double r = sqrt(rx * rx + ry * ry + rz * rz);
            const double z = c * ((blk + 1) * Tdt + dt + htp * Dt) - r;
            if (z > 0.0) {
                double pz = 1.0;
                for (int k = 0; k < d; ++k) pz *= z;
                v = (float)(pz / r);
            }
        }
        out[e] = make_float2(v, 0.f);
    }
}

// One forward DFT axis of nvec grids (set-up): out = sum_j in[.., j, ..]
// e^{-2 pi i f j / n} along axis 0..2 (space, n = Ns) or 3 (time, n = Nt).
__global__ void k_dft_axis(int64_t nvec, int Ns, int Nt, int axis, const float2 *__restrict__ in, float2 *out)
{
    __shared__ float2 tw[kFftMaxN];
    const int n = axis < 3 ? Ns : Nt;
    twiddles(tw, n, -1);
    __syncthreads();
    const int64_t N = (int64_t)Ns * Ns * Ns * Nt;
    const int64_t stride = axis == 0 ? 1 : axis == 1 ? Ns : axis == 2 ? (int64_t)Ns * Ns : (int64_t)Ns * Ns * Ns;
    const int64_t total = nvec * N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int f = (int)(((e % N) / stride) % n);
        const int64_t base = e - (int64_t)f * stride;
        float2 acc = make_float2(0.f, 0.f);
        for (int j = 0; j < n; ++j) acc = cfma(acc, in[base + j * stride], tw[(f * j) % n]);
        out[e] = acc;
    }
}

size_t fwd_smem(int ps, int pt, int Ns, int Nt)
{
    const int P3 = ps * ps * ps;
    return (size_t)(Ns + Nt + P3 * Nt + ps * ps * Ns + ps * Ns * Ns) * sizeof(float2);
}

size_t inv_smem(int ps, int pt, int Ns, int Nt)
{
    const int P3 = ps * ps * ps;
    return (size_t)(Ns + Nt + Ns * Ns * Ns + Ns * Ns * ps + Ns * ps * ps + P3) * sizeof(float2) +
           (size_t)P3 * pt * sizeof(float);
}

}  // namespace

// Spectra of the moments of the current source interval, one CTA per cell.
__global__ void __launch_bounds__(kFftThreads) k_fft_fwd(int nc, int ps, int pt, int Ns, int Nt,
                                                         const double *__restrict__ M, float2 *Mhat, StepWhen w)
{
    if (w.alpha && when_interval(w) < 0) return;
    extern __shared__ float2 fsh[];
    const int P3 = ps * ps * ps;
    float2 *tws = fsh, *twt = tws + Ns, *Z = twt + Nt, *A1 = Z + P3 * Nt, *A2 = A1 + ps * ps * Ns;
    const int S = blockIdx.x;
    twiddles(tws, Ns, -1);
    twiddles(twt, Nt, -1);
    __syncthreads();
    const double *m = M + (int64_t)S * P3 * pt;
    // time axis: Z[b][ft] = sum_{n < pt} M[b + P3 n] e^{-2 pi i ft n / Nt}
    for (int e = threadIdx.x; e < P3 * Nt; e += blockDim.x) {
        const int b = e / Nt, ft = e % Nt;
        float2 acc = make_float2(0.f, 0.f);
        for (int n = 0; n < pt; ++n) acc = cfma(acc, make_float2((float)m[b + P3 * n], 0.f), twt[(ft * n) % Nt]);
        Z[e] = acc;
    }
    const int64_t N3 = (int64_t)Ns * Ns * Ns;
    float2 *out = Mhat + (int64_t)S * N3 * Nt;
    for (int ft = 0; ft < Nt; ++ft) {
        __syncthreads();
        // x: A1[b3][b2][f1] = sum_b1 Z[b1 + ps (b2 + ps b3)][ft] e^{-2 pi i f1 b1 / Ns}
        for (int e = threadIdx.x; e < ps * ps * Ns; e += blockDim.x) {
            const int f1 = e % Ns, r = e / Ns;  // r = b2 + ps b3
            float2 acc = make_float2(0.f, 0.f);
            for (int b1 = 0; b1 < ps; ++b1) acc = cfma(acc, Z[(b1 + ps * r) * Nt + ft], tws[(f1 * b1) % Ns]);
            A1[e] = acc;
        }
        __syncthreads();
        // y: A2[b3][f2][f1] = sum_b2 A1[b3][b2][f1] e^{-2 pi i f2 b2 / Ns}
        for (int e = threadIdx.x; e < ps * Ns * Ns; e += blockDim.x) {
            const int f1 = e % Ns, f2 = (e / Ns) % Ns, b3 = e / (Ns * Ns);
            float2 acc = make_float2(0.f, 0.f);
            for (int b2 = 0; b2 < ps; ++b2) acc = cfma(acc, A1[(b3 * ps + b2) * Ns + f1], tws[(f2 * b2) % Ns]);
            A2[e] = acc;
        }
        __syncthreads();
        // z: Mhat[S][ft][f3][f2][f1] = sum_b3 A2[b3][f2][f1] e^{-2 pi i f3 b3 / Ns}
        for (int e = threadIdx.x; e < (int)N3; e += blockDim.x) {
            const int f12 = e % (Ns * Ns), f3 = e / (Ns * Ns);
            float2 acc = make_float2(0.f, 0.f);
            for (int b3 = 0; b3 < ps; ++b3) acc = cfma(acc, A2[b3 * Ns * Ns + f12], tws[(f3 * b3) % Ns]);
            out[(int64_t)ft * N3 + e] = acc;
        }
    }
}

// Yhat[O][blk][g] = sum over the pairs (O, S) of Khat[offset][blk][g] Mhat[S][g]
// for the C frequencies g0 .. g0 + C - 1 of this CTA and blocks lb .. le-1.
// Lane l of a warp takes frequency l % C of every (32 / C)-th pair; the
// partial sums are combined by shuffles.
__global__ void __launch_bounds__(kFftThreads) k_fft_mul(int nc, int64_t N, int nbl, int lb, int le, int nfo, int C,
                                                         const int64_t *__restrict__ ooff,
                                                         const int32_t *__restrict__ fS,
                                                         const int16_t *__restrict__ fo,
                                                         const float2 *__restrict__ Khat,
                                                         const float2 *__restrict__ Mhat, float2 *Yhat, StepWhen w)
{
    if (w.alpha && when_interval(w) < 0) return;
    extern __shared__ float2 fsh[];
    float2 *Ms = fsh, *Ks = fsh + (size_t)nc * C;
    const int64_t g0 = (int64_t)blockIdx.x * C;
    for (int e = threadIdx.x; e < nc * C; e += blockDim.x) {
        const int S = e / C, f = e % C;
        Ms[e] = (g0 + f < N) ? Mhat[(int64_t)S * N + g0 + f] : make_float2(0.f, 0.f);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int f = lane % C, sub = lane / C, G = 32 / C;
    for (int blk = lb; blk < le; ++blk) {
        __syncthreads();
        for (int e = threadIdx.x; e < nfo * C; e += blockDim.x) {
            const int o = e / C, ff = e % C;
            Ks[e] = (g0 + ff < N) ? Khat[((int64_t)o * nbl + blk) * N + g0 + ff] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        for (int O = warp; O < nc; O += nw) {
            float2 acc = make_float2(0.f, 0.f);
            const int64_t q1 = ooff[O + 1];
            for (int64_t q = ooff[O] + sub; q < q1; q += G) acc = cfma(acc, Ks[fo[q] * C + f], Ms[fS[q] * C + f]);
            for (int o = C; o < 32; o <<= 1) {
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
            }
            if (sub == 0 && g0 + f < N) Yhat[((int64_t)O * nbl + blk) * N + g0 + f] = acc;
        }
    }
}

// Inverse transforms of Yhat[O][lb + blockIdx.y], restricted to the ps^3 x pt
// node grid, added into ring slot (k + blk + 1) mod nslot of cell O.
__global__ void __launch_bounds__(kFftThreads) k_fft_inv(int nc, int ps, int pt, int Ns, int Nt, int nbl, int lb,
                                                         int nslot, int k, const float2 *__restrict__ Yhat,
                                                         double *ring, StepWhen w)
{
    if (w.alpha && (k = when_interval(w)) < 0) return;
    extern __shared__ float2 fsh[];
    const int P3 = ps * ps * ps, P = P3 * pt;
    const int N3 = Ns * Ns * Ns;
    float2 *tws = fsh, *twt = tws + Ns, *Sl = twt + Nt, *B1 = Sl + N3, *B2 = B1 + Ns * Ns * ps, *Wf = B2 + Ns * ps * ps;
    float *acc = reinterpret_cast<float *>(Wf + P3);
    const int O = blockIdx.x, blk = lb + blockIdx.y;
    twiddles(tws, Ns, 1);
    twiddles(twt, Nt, 1);
    for (int e = threadIdx.x; e < P; e += blockDim.x) acc[e] = 0.f;
    const float2 *y = Yhat + ((int64_t)O * nbl + blk) * N3 * Nt;
    for (int ft = 0; ft < Nt; ++ft) {
        __syncthreads();
        for (int e = threadIdx.x; e < N3; e += blockDim.x) Sl[e] = y[(int64_t)ft * N3 + e];
        __syncthreads();
        // x: B1[f3][f2][a1] = sum_f1 Sl[f3][f2][f1] e^{2 pi i f1 a1 / Ns}
        for (int e = threadIdx.x; e < Ns * Ns * ps; e += blockDim.x) {
            const int a1 = e % ps, r = e / ps;  // r = f2 + Ns f3
            float2 c = make_float2(0.f, 0.f);
            for (int f1 = 0; f1 < Ns; ++f1) c = cfma(c, Sl[r * Ns + f1], tws[(f1 * a1) % Ns]);
            B1[e] = c;
        }
        __syncthreads();
        // y: B2[f3][a2][a1] = sum_f2 B1[f3][f2][a1] e^{2 pi i f2 a2 / Ns}
        for (int e = threadIdx.x; e < Ns * ps * ps; e += blockDim.x) {
            const int a1 = e % ps, a2 = (e / ps) % ps, f3 = e / (ps * ps);
            float2 c = make_float2(0.f, 0.f);
            for (int f2 = 0; f2 < Ns; ++f2) c = cfma(c, B1[(f3 * Ns + f2) * ps + a1], tws[(f2 * a2) % Ns]);
            B2[e] = c;
        }
        __syncthreads();
        // z: Wf[a1 + ps (a2 + ps a3)] = sum_f3 B2[f3][a2][a1] e^{2 pi i f3 a3 / Ns}
        for (int e = threadIdx.x; e < P3; e += blockDim.x) {
            const int a12 = e % (ps * ps), a3 = e / (ps * ps);
            float2 c = make_float2(0.f, 0.f);
            for (int f3 = 0; f3 < Ns; ++f3) c = cfma(c, B2[f3 * ps * ps + a12], tws[(f3 * a3) % Ns]);
            Wf[e] = c;
        }
        __syncthreads();
        // time: acc[a + P3 m] += Re(Wf[a] e^{2 pi i ft m / Nt}), m < pt
        for (int e = threadIdx.x; e < P; e += blockDim.x) {
            const int a = e % P3, m = e / P3;
            const float2 t = twt[(ft * m) % Nt], v = Wf[a];
            acc[e] = fmaf(v.x, t.x, fmaf(-v.y, t.y, acc[e]));
        }
    }
    const double inv = 1.0 / ((double)N3 * Nt);
    double *r = ring + ((int64_t)((k + blk + 1) % nslot) * nc + O) * P;
    for (int e = threadIdx.x; e < P; e += blockDim.x) r[e] += (double)acc[e] * inv;
}

namespace {

template <typename T>
cudaError_t fft_alloc(tdbem_ctx *c, T **p, size_t n)
{
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(n * sizeof(T), 16));
    if (e == cudaSuccess) {
        c->allocs.push_back(q);
        *p = (T *)q;
        e = cudaMemsetAsync(q, 0, std::max<size_t>(n * sizeof(T), 16), c->s);
    }
    return e;
}

void fft_free(tdbem_ctx *c, void *p)
{
    auto it = std::find(c->allocs.begin(), c->allocs.end(), p);
    if (it != c->allocs.end()) c->allocs.erase(it);
    cudaFree(p);
}

}  // namespace

#define FT_TRY(x)                         \
    do {                                  \
        cudaError_t e_ = (x);             \
        if (e_ != cudaSuccess) return e_; \
    } while (0)

// Set-up of one level's FFT form: the pairs (per observation cell in list
// order: source cell, offset index), the products' frequency chunk, the
// transforms' buffers, and the spectra of the kernel samples of every
// offset and near-future block (FP64 samples, FP32 axis passes).
cudaError_t fft_m2l_level_setup(tdbem_ctx *c, FmmLevel &V, const std::vector<int32_t> &pS,
                                const std::vector<int16_t> &po, const std::vector<int32_t> &codes, double Tdt,
                                std::string &why)
{
    Fmm &F = c->fmm;
    const int ps = F.ps, pt = F.pt, Ns = F.fNs, Nt = F.fNt, nbl = F.ngb;
    const int64_t N = F.fN;
    V.nfo = (int)codes.size();
    int C = 32;
    while (C > 1 && (size_t)(V.nc + V.nfo) * C * sizeof(float2) > kFftMulSmem) C >>= 1;
    if ((size_t)(V.nc + V.nfo) * C * sizeof(float2) > kFftMulSmem) {
        why = "FFT M2L: too many cells at one level for the products' shared memory";
        return cudaSuccess;
    }
    V.fC = C;
    FT_TRY(fft_alloc(c, &V.fS, pS.size()));
    FT_TRY(fft_alloc(c, &V.fo, po.size()));
    FT_TRY(cudaMemcpyAsync(V.fS, pS.data(), pS.size() * sizeof(int32_t), cudaMemcpyHostToDevice, c->s));
    FT_TRY(cudaMemcpyAsync(V.fo, po.data(), po.size() * sizeof(int16_t), cudaMemcpyHostToDevice, c->s));
    FT_TRY(fft_alloc(c, &V.Mhat, (size_t)V.nc * N));
    FT_TRY(fft_alloc(c, &V.Yhat, (size_t)V.nc * nbl * N));
    FT_TRY(fft_alloc(c, &V.Khat, (size_t)V.nfo * nbl * N));
    float2 *tmp = nullptr;
    int32_t *d_codes = nullptr;
    FT_TRY(fft_alloc(c, &tmp, (size_t)V.nfo * nbl * N));
    FT_TRY(fft_alloc(c, &d_codes, codes.size()));
    FT_TRY(cudaMemcpyAsync(d_codes, codes.data(), codes.size() * sizeof(int32_t), cudaMemcpyHostToDevice, c->s));
    k_fft_samples<<<152 * 32, 256, 0, c->s>>>(V.nfo, nbl, ps, pt, Ns, Nt, V.s, V.hs, Tdt, c->P.dt, c->P.c, c->P.d,
                                              d_codes, V.Khat);
    FT_TRY(cudaGetLastError());
    // four axis passes: Khat -> tmp -> Khat -> tmp -> Khat
    for (int axis = 0; axis < 4; ++axis) {
        const float2 *in = (axis & 1) ? tmp : V.Khat;
        float2 *out = (axis & 1) ? V.Khat : tmp;
        k_dft_axis<<<152 * 32, 256, 0, c->s>>>((int64_t)V.nfo * nbl, Ns, Nt, axis, in, out);
        FT_TRY(cudaGetLastError());
    }
    FT_TRY(cudaStreamSynchronize(c->s));
    fft_free(c, tmp);
    fft_free(c, d_codes);
    FT_TRY(cudaFuncSetAttribute(k_fft_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem(ps, pt, Ns, Nt)));
    FT_TRY(cudaFuncSetAttribute(k_fft_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)inv_smem(ps, pt, Ns, Nt)));
    FT_TRY(cudaFuncSetAttribute(k_fft_mul, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFftMulSmem));
    // algorithmic flops of one application: a complex multiply-add (8 flops)
    // per pair, block and grid point
    V.flops_app = 8.0 * (double)V.np * nbl * (double)N;
    return cudaSuccess;
}

cudaError_t fft_m2l_forward(tdbem_ctx *c, FmmLevel &V, cudaStream_t s, const StepWhen &w)
{
    Fmm &F = c->fmm;
    k_fft_fwd<<<V.nc, kFftThreads, fwd_smem(F.ps, F.pt, F.fNs, F.fNt), s>>>(V.nc, F.ps, F.pt, F.fNs, F.fNt, V.M,
                                                                            V.Mhat, w);
    return cudaGetLastError();
}

cudaError_t fft_m2l_apply(tdbem_ctx *c, FmmLevel &V, int kl, int lb, int le, cudaStream_t s, const StepWhen &w)
{
    Fmm &F = c->fmm;
    if (le <= lb) return cudaSuccess;
    const int C = V.fC;
    const int64_t grid = (F.fN + C - 1) / C;
    k_fft_mul<<<(unsigned)grid, kFftThreads, (size_t)(V.nc + V.nfo) * C * sizeof(float2), s>>>(
        V.nc, F.fN, F.ngb, lb, le, V.nfo, C, V.ooff, V.fS, V.fo, V.Khat, V.Mhat, V.Yhat, w);
    FT_TRY(cudaGetLastError());
    k_fft_inv<<<dim3(V.nc, le - lb), kFftThreads, inv_smem(F.ps, F.pt, F.fNs, F.fNt), s>>>(
        V.nc, F.ps, F.pt, F.fNs, F.fNt, F.ngb, lb, F.nslot, kl, V.Yhat, V.ring, w);
    return cudaGetLastError();
}

}  // namespace tdbem
