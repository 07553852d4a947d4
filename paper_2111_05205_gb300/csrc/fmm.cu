// Interpolation-based space-time FMM for the far part of the history sum
// (Section 3: P2M, M2M, M2L, L2L, L2P; Section 4: near- and distant-future
// M2L with the O(Nt) recurrence of Formula 1 / Algorithm 1).
//
// Readings (the paper defers the hierarchy to its earlier study):
//   - Lagrange interpolation on the p Chebyshev points of the first kind,
//     cos((2a+1) pi / (2p)), in each of x1..x3, y1..y3, t, s;
//   - source box of a level-l cell: its cube enlarged by rho, the largest
//     centroid-to-vertex distance of the mesh (half-width s_l/2 + rho), as a
//     source element reaches up to rho beyond the cell of its centroid;
//     observation box: the cube itself (half-width s_l/2), as the
//     observation points are the centroids, which lie in their cells;
//   - a leaf interval holds Lt = floor((s_L - rho)/(c dt)) steps (no source
//     of an interval reaches an interaction-list target in the same
//     interval); level l holds T_l = Lt 2^(L-l) steps; source interval J_k
//     covers sigma in [k T, (k+1) T), observation interval I_k covers steps
//     alpha in [k T + 1, (k+1) T + 1);
//   - mu: the smallest integer with c (mu T_l + 1) dt > sqrt(3)(3 s_l + h_l + o_l)
//     on every level (h_l, o_l the source and observation half-widths), so
//     that the kernel is a polynomial of degree d over the node domain of
//     every distant-future interval (Section 4.2).
// Vector index of moments and locals: b1 + ps (b2 + ps (b3 + ps n)), as in
// the matrix form of Eq. m2l.
#include <math.h>

#include <algorithm>
#include <type_traits>

#include <cublas_v2.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "tdbem_internal.cuh"

namespace tdbem {

constexpr int kMaxP = 8;

// Interpolation node a of p on [-1, 1]: Chebyshev points of the first kind,
// or (eq, the FFT form) p equispaced points with both ends.
__device__ __forceinline__ double fmm_node(int p, int a, bool eq)
{
    if (eq) return p > 1 ? -1.0 + 2.0 * a / (p - 1) : 0.0;
    return cos((2.0 * a + 1.0) * 3.14159265358979323846 / (2.0 * p));
}

// Lagrange basis of the p nodes at xi (values and derivatives).
__device__ void lag_basis(int p, double xi, double *val, double *der, bool eq)
{
    double w[kMaxP];
    for (int a = 0; a < p; ++a) w[a] = fmm_node(p, a, eq);
    for (int a = 0; a < p; ++a) {
        double v = 1.0, dv = 0.0;
        for (int b = 0; b < p; ++b) {
            if (b == a) continue;
            double den = w[a] - w[b];
            double f = (xi - w[b]) / den;
            dv = dv * f + v / den;
            v *= f;
        }
        val[a] = v;
        if (der) der[a] = dv;
    }
}

__device__ __forceinline__ void cell_centre(uint64_t key, int lev, const double *box, double s, double c[3])
{
    int co[3] = {0, 0, 0};
    for (int b = 0; b < lev; ++b)
        for (int a = 0; a < 3; ++a) co[a] |= (int)((key >> (3 * b + a)) & 1u) << b;
    for (int a = 0; a < 3; ++a) c[a] = box[a] + (co[a] + 0.5) * s;
}

// rho = max over elements of the centroid-to-vertex distance (each
// operation rounded separately, as the reference definition).
__global__ void k_rho(int ns, const double *__restrict__ xyz, const int32_t *__restrict__ tri,
                      const double *__restrict__ xc, unsigned long long *out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns) return;
    double m = 0.0;
    for (int a = 0; a < 3; ++a) {
        double d0 = __dsub_rn(xyz[3 * tri[3 * i + a]], xc[3 * i]);
        double d1 = __dsub_rn(xyz[3 * tri[3 * i + a] + 1], xc[3 * i + 1]);
        double d2 = __dsub_rn(xyz[3 * tri[3 * i + a] + 2], xc[3 * i + 2]);
        double r = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2)));
        m = fmax(m, r);
    }
    atomicMax(out, (unsigned long long)__double_as_longlong(m));  // non-negative doubles order as integers
}

// P2M weights of each element for its leaf box: At[j][b] = int_E ell_b dS,
// As[j][b] = int_E n_y . grad ell_b dS (collapsed Gauss-Legendre rule, exact
// for the degree 3(ps-1) of ell_b on a flat triangle), and the L2P values
// Dv[i][a] = ell_a(x_i), Dn[i][a] = n_x . grad ell_a(x_i).
__global__ void k_element_weights(int ns, int ps, int L, const double *__restrict__ box, double s, double hs, double ho,
                                  const double *__restrict__ xyz, const int32_t *__restrict__ tri,
                                  const double *__restrict__ xc, const double *__restrict__ nrm,
                                  const uint64_t *__restrict__ key, int nq, const double *__restrict__ qx,
                                  const double *__restrict__ qw, double *At, double *As, double *Dv, double *Dn, bool eq)
{
    int j = blockIdx.x;
    if (j >= ns) return;
    const int P3 = ps * ps * ps;
    double cen[3];
    cell_centre(key[j], L, box, s, cen);
    double v[9];
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 3; ++k) v[3 * a + k] = xyz[3 * tri[3 * j + a] + k];
    double e1[3] = {v[3] - v[0], v[4] - v[1], v[5] - v[2]}, e2[3] = {v[6] - v[0], v[7] - v[1], v[8] - v[2]};
    double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    double area2 = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    const double *n = nrm + 3 * j;
    for (int b = threadIdx.x; b < P3; b += blockDim.x) {
        int b1 = b % ps, b2 = (b / ps) % ps, b3 = b / (ps * ps);
        double at = 0.0, as = 0.0;
        for (int q = 0; q < nq * nq; ++q) {
            double u = qx[q / nq], t = qx[q % nq] * (1.0 - u);
            double w = qw[q / nq] * qw[q % nq] * (1.0 - u) * area2;
            double y[3];
            for (int k = 0; k < 3; ++k) y[k] = v[k] + u * e1[k] + t * e2[k];
            double l[3][kMaxP], dl[3][kMaxP];
            for (int k = 0; k < 3; ++k) lag_basis(ps, (y[k] - cen[k]) / hs, l[k], dl[k], eq);
            double val = l[0][b1] * l[1][b2] * l[2][b3];
            double g0 = dl[0][b1] * l[1][b2] * l[2][b3] / hs, g1 = l[0][b1] * dl[1][b2] * l[2][b3] / hs,
                   g2 = l[0][b1] * l[1][b2] * dl[2][b3] / hs;
            at += w * val;
            as += w * (g0 * n[0] + g1 * n[1] + g2 * n[2]);
        }
        At[(int64_t)j * P3 + b] = at;
        As[(int64_t)j * P3 + b] = as;
        // L2P values at the collocation point of element j (observation box)
        double l[3][kMaxP], dl[3][kMaxP];
        for (int k = 0; k < 3; ++k) lag_basis(ps, (xc[3 * j + k] - cen[k]) / ho, l[k], dl[k], eq);
        Dv[(int64_t)j * P3 + b] = l[0][b1] * l[1][b2] * l[2][b3];
        Dn[(int64_t)j * P3 + b] = (dl[0][b1] * l[1][b2] * l[2][b3] * n[0] + l[0][b1] * dl[1][b2] * l[2][b3] * n[1] +
                                  l[0][b1] * l[1][b2] * dl[2][b3] * n[2]) / ho;
    }
}

// M2L operator bank of one level: op[t][blk][row][col] for the offsets
// o = offs[t] = (dx+3) + 7((dy+3) + 7(dz+3)) (the cell offset S - O) in the
// order the batched GEMMs use, blk = l-1 for the near future l = 1..nblk
// (nblk = mu: the GEMM blocks; blocks past mu would hold l = mu + 1 and the
// p-th derivative U^(p) at I_{k+mu+1} of Eq. U_expand, which the library
// forms from their exact low-rank expansion instead), row = a + P3 m,
// col = b + P3 n:
//   U(x_a, y_b, t_m, s_n) = (c (t_m - s_n) - r)_+^d / r,
//   U^(p) = C(d, p) (c (t_m - s_n) - r)_+^(d-p) / r,
// x_a - y_b = -offset s + ho w_a - hs w_b, t_m - s_n = l T dt + dt + ht (w_m - w_n).
__global__ void k_m2l_operators(int ps, int pt, int d, int mu, int nblk, double s, double hs, double ho, double T_dt, double dt,
                                double ht, double c, int noff, const int32_t *__restrict__ offs, double *op, bool eq)
{
    const int P3 = ps * ps * ps, P = P3 * pt;
    int64_t total = (int64_t)noff * nblk * P * P;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int col = (int)(e % P);
        int64_t r1 = e / P;
        int row = (int)(r1 % P);
        int64_t r2 = r1 / P;
        int blk = (int)(r2 % nblk);
        int o = offs[r2 / nblk];
        int dx = o % 7 - 3, dy = (o / 7) % 7 - 3, dz = o / 49 - 3;
        if (max(abs(dx), max(abs(dy), abs(dz))) <= 1) {
            op[e] = 0.0;
            continue;
        }
        int a = row % P3, m = row / P3, b = col % P3, n = col / P3;
        int a1 = a % ps, a2 = (a / ps) % ps, a3 = a / (ps * ps);
        int b1 = b % ps, b2 = (b / ps) % ps, b3 = b / (ps * ps);
        double rx = -dx * s + ho * fmm_node(ps, a1, eq) - hs * fmm_node(ps, b1, eq);
        double ry = -dy * s + ho * fmm_node(ps, a2, eq) - hs * fmm_node(ps, b2, eq);
        double rz = -dz * s + ho * fmm_node(ps, a3, eq) - hs * fmm_node(ps, b3, eq);
        double r = sqrt(rx * rx + ry * ry + rz * rz);
        int l = (blk <= mu) ? blk + 1 : mu + 1;
        int pw = (blk <= mu) ? 0 : blk - mu;
        double tdiff = l * T_dt + dt + ht * (fmm_node(pt, m, eq) - fmm_node(pt, n, eq));
        double z = c * tdiff - r;
        double v = 0.0;
        if (z > 0.0) {
            double binom = 1.0;
            for (int k = 0; k < pw; ++k) binom = binom * (d - k) / (k + 1);
            double pz = 1.0;
            for (int k = 0; k < d - pw; ++k) pz *= z;
            v = binom * pz / r;
        }
        op[e] = v;
    }
}

}  // namespace tdbem

namespace tdbem {

// P2M at the leaf level for source interval k (Section 3, moment M_{b,n}):
// M[c][b + P3 n] += pref sum_{sigma in J_k} sum_{j in c}
//                   (At[j][b] tau_j^sigma - As[j][b] sigma_j^sigma) ell_n(t_sigma),
// with tau, sigma the folded histories of Eq. tau / Eq. sigma.  The sum over
// sigma does not involve the spatial node b, so it is taken first, once per
// (element, temporal node) by k_p2m_time: Tq[p][n] = sum_sigma tau_j^sigma
// ell_n(t_sigma) (Tu likewise with sigma_j), j = perm[p] the element at
// sorted position p; then k_p2m_moments forms every entry of every leaf
// cell's moment, one thread per entry:
// M[c][b + P3 n] += pref sum_{p in c} (At[j][b] Tq[p][n] - As[j][b] Tu[p][n]).
__global__ void k_p2m_time(int ns, int pt, int Lt, int k, int d, int smax_hist, const int32_t *__restrict__ perm,
                           const double *__restrict__ q, const double *__restrict__ u, const double *__restrict__ wk,
                           const double *__restrict__ tl, double *Tq, double *Tu, StepWhen w)
{
    if (w.alpha && (k = when_interval(w)) < 0) return;
    const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (x >= (int64_t)ns * pt) return;
    const int p = (int)(x / pt), n = (int)(x % pt);
    const int j = perm[p];
    double tq = 0.0, tu = 0.0;
    for (int t = 0; t < Lt; ++t) {
        const int sg = k * Lt + t;
        if (sg > smax_hist) break;
        double tau = 0.0, sig = 0.0;
        for (int kk = 0; kk <= d + 1 && kk <= sg; ++kk) {
            tau += wk[kk] * q[(int64_t)(sg - kk) * ns + j];
            sig += wk[kk] * u[(int64_t)(sg - kk) * ns + j];
        }
        tq += tau * tl[t * 8 + n];
        tu += sig * tl[t * 8 + n];
    }
    Tq[x] = tq;
    Tu[x] = tu;
}

// One thread per moment entry e = b + P3 n of leaf cell c (grid: cells x
// ceil(P / 256)).
__global__ void k_p2m_moments(int P3, int P, const int32_t *__restrict__ cstart, const int32_t *__restrict__ perm,
                              const double *__restrict__ At, const double *__restrict__ As,
                              const double *__restrict__ Tq, const double *__restrict__ Tu, double pref, double *M,
                              StepWhen w)
{
    if (w.alpha && when_interval(w) < 0) return;
    const int c = blockIdx.x;
    const int e = blockIdx.y * blockDim.x + threadIdx.x;
    if (e >= P) return;
    const int pt = P / P3, b = e % P3, n = e / P3;
    const int p0 = cstart[c], p1 = cstart[c + 1];
    double acc = 0.0;
    for (int p = p0; p < p1; ++p) {
        const int64_t r = (int64_t)perm[p] * P3 + b;
        acc += At[r] * Tq[(int64_t)p * pt + n] - As[r] * Tu[(int64_t)p * pt + n];
    }
    M[(int64_t)c * P + e] += pref * acc;
}

// One mode product of a separable transfer on a [ps, ps, ps, pt] tensor:
// out[.., e_axis, ..] = sum_q A[e_axis][q] in[.., q, ..] (A [p][p], row-major;
// `transpose` uses A[q][e_axis]).
__device__ void mode_product(int ps, int pt, int axis, const double *A, bool transpose, const double *in,
                             double *out)
{
    const int P3 = ps * ps * ps, P = P3 * pt;
    int stride = (axis == 0) ? 1 : (axis == 1) ? ps : (axis == 2) ? ps * ps : P3;
    int p = (axis == 3) ? pt : ps;
    for (int e = threadIdx.x; e < P; e += blockDim.x) {
        int idx = (e / stride) % p;
        int base = e - idx * stride;
        double acc = 0.0;
        for (int qq = 0; qq < p; ++qq) acc += (transpose ? A[qq * p + idx] : A[idx * p + qq]) * in[base + qq * stride];
        out[e] = acc;
    }
}

__device__ __forceinline__ int find_key_f(const uint64_t *__restrict__ keys, int n, uint64_t k)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        int m = (lo + hi) >> 1;
        if (keys[m] < k)
            lo = m + 1;
        else
            hi = m;
    }
    return lo;
}

// M2M (Section 3; the paper's cost p_s^6 p_t^2, done here separably): the
// parent's moment accumulates every child's moment transferred by the 1-D
// matrices S[pos][b'][b] = ell_b'((child node b - parent centre)/h_parent)
// per axis and T[half][n'][n] = ell_n'((w_n + 2 half - 1)/2) in time.
__global__ void k_m2m(int ps, int pt, int ncp, const uint64_t *__restrict__ pkey, int ncc,
                      const uint64_t *__restrict__ ckey, const double *__restrict__ Mc, double *Mp,
                      const double *__restrict__ Sm, const double *__restrict__ Tm, int half, StepWhen w)
{
    if (w.alpha) {
        const int kl = when_interval(w);
        if (kl < 0) return;
        half = kl & 1;
    }
    extern __shared__ double sh[];
    const int P = ps * ps * ps * pt;
    double *b0 = sh, *b1 = sh + P;
    int p = blockIdx.x;
    uint64_t K = pkey[p];
    int c = find_key_f(ckey, ncc, K << 3);
    for (; c < ncc && (ckey[c] >> 3) == K; ++c) {
        int pos = (int)(ckey[c] & 7u);
        for (int e = threadIdx.x; e < P; e += blockDim.x) b0[e] = Mc[(int64_t)c * P + e];
        __syncthreads();
        mode_product(ps, pt, 0, Sm + ((pos & 1) * ps * ps), false, b0, b1);
        __syncthreads();
        mode_product(ps, pt, 1, Sm + (((pos >> 1) & 1) * ps * ps), false, b1, b0);
        __syncthreads();
        mode_product(ps, pt, 2, Sm + (((pos >> 2) & 1) * ps * ps), false, b0, b1);
        __syncthreads();
        mode_product(ps, pt, 3, Tm + half * pt * pt, false, b1, b0);
        __syncthreads();
        for (int e = threadIdx.x; e < P; e += blockDim.x) Mp[(int64_t)p * P + e] += b0[e];
        __syncthreads();
    }
}

// L2L (Section 3): child local += transposed transfer of the parent local,
// for the child interval kc (slot kc of the child ring) inside the parent
// interval kc / 2.
__global__ void k_l2l(int ps, int pt, int ncp, const uint64_t *__restrict__ pkey, int ncc,
                      const uint64_t *__restrict__ ckey, const double *__restrict__ Lpr, double *Lcr, int nslot,
                      const double *__restrict__ Sm, const double *__restrict__ Tm, int kc, StepWhen w)
{
    extern __shared__ double sh[];
    const int P = ps * ps * ps * pt;
    if (w.alpha) {
        const int i = when_interval(w);
        if (i < 0) return;
        kc = i + 1;
    }
    const int half = kc & 1;
    const double *Lp = Lpr + (int64_t)((kc / 2) % nslot) * ncp * P;
    double *Lc = Lcr + (int64_t)(kc % nslot) * ncc * P;
    double *b0 = sh, *b1 = sh + P;
    int c = blockIdx.x;
    int p = find_key_f(pkey, ncp, ckey[c] >> 3);
    int pos = (int)(ckey[c] & 7u);
    for (int e = threadIdx.x; e < P; e += blockDim.x) b0[e] = Lp[(int64_t)p * P + e];
    __syncthreads();
    mode_product(ps, pt, 0, Sm + ((pos & 1) * ps * ps), true, b0, b1);
    __syncthreads();
    mode_product(ps, pt, 1, Sm + (((pos >> 1) & 1) * ps * ps), true, b1, b0);
    __syncthreads();
    mode_product(ps, pt, 2, Sm + (((pos >> 2) & 1) * ps * ps), true, b0, b1);
    __syncthreads();
    mode_product(ps, pt, 3, Tm + half * pt * pt, true, b1, b0);
    __syncthreads();
    for (int e = threadIdx.x; e < P; e += blockDim.x) Lc[(int64_t)c * P + e] += b0[e];
}

// Distant-future recurrences of Formula 1 (Eq. m2l_expand_rec1, Eq. m2l_rec,
// Eq. m2l_expand_rec2) for every entry of every cell of one level:
//   D_p <- D_p + G_p + sum_{m<=p-2} c_m^p(k) A_{p,m}
//   L_{k+mu+2} <- L_{k+mu+1} + sum_p D_p T^p
//   A_{p,m} <- A_{p,m} + G_p k^m
__global__ void k_m2l_recurrence(int64_t n, int d, int mu, int nslot, int k, const double *__restrict__ G, double *D,
                                 double *Aux, double *ring, double Tlen, StepWhen w)
{
    if (w.alpha && (k = when_interval(w)) < 0) return;
    // c_m^p(k) of Eq. cmp, p = 2..d, m = 0..p-2 (index (p-2)(p-1)/2 + m):
    // C(p, m) ((k-1)^(p-m) - 2 k^(p-m) + (k+1)^(p-m)) (-1)^m, integers
    // exact in FP64
    double cmp[kMaxD * (kMaxD - 1) / 2 + 1];
    for (int p = 2; p <= d; ++p)
        for (int m = 0; m <= p - 2; ++m) {
            double binom = 1.0;
            for (int i = 0; i < m; ++i) binom = binom * (p - i) / (i + 1);
            const int e = p - m;
            double a = 1.0, b = 1.0, c = 1.0;
            for (int i = 0; i < e; ++i) {
                a *= (double)k - 1.0;
                b *= (double)k;
                c *= (double)k + 1.0;
            }
            cmp[(p - 2) * (p - 1) / 2 + m] = binom * (a - 2.0 * b + c) * ((m & 1) ? -1.0 : 1.0);
        }
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        double g[kMaxD + 1];
        for (int p = 1; p <= d; ++p) g[p] = G[(int64_t)(p - 1) * n + e];
        // auxiliaries before their update
        int ai = 0;
        for (int p = 1; p <= d; ++p) {
            double s = D[(int64_t)(p - 1) * n + e] + g[p];
            for (int m = 0; m <= p - 2; ++m) s += cmp[(p - 2) * (p - 1) / 2 + m] * Aux[(int64_t)((p - 2) * (p - 1) / 2 + m) * n + e];
            D[(int64_t)(p - 1) * n + e] = s;
        }
        double lnew = ring[(int64_t)((k + mu + 1) % nslot) * n + e];
        double tp = 1.0;
        for (int p = 1; p <= d; ++p) {
            tp *= Tlen;
            lnew += D[(int64_t)(p - 1) * n + e] * tp;
        }
        ring[(int64_t)((k + mu + 2) % nslot) * n + e] = lnew;
        for (int p = 2; p <= d; ++p) {
            double km = 1.0;
            for (int m = 0; m <= p - 2; ++m) {
                ai = (p - 2) * (p - 1) / 2 + m;
                Aux[(int64_t)ai * n + e] += g[p] * km;
                km *= (double)k;
            }
        }
    }
}

// L2P (Eq. target_m2l) at the leaf level for the Lt steps of observation
// interval I_k: far[t][i] = sum_{a,m} D_a(x_i) ell_m(t_alpha) L_{a,m}, with
// the Burton-Miller operator (d/dn_x - c^-1 d/dt) applied to ell_a ell_m.
// The spatial sum is taken first, once per temporal node:
// Yn[m] = sum_a (n.grad ell_a)(x_i) L_{a,m}, Yv[m] = sum_a ell_a(x_i) L_{a,m};
// then far[t] = sum_m (ell_m(t) Yn[m] - ell_m'(t) Yv[m] / c) (BMBIE) or
// sum_m ell_m(t) Yv[m] (OBIE).  One warp per element: the lanes read the
// element's basis rows and the cell's locals contiguously and the sums are
// reduced by shuffles.
__global__ void k_l2p(int ns, int P3, int pt, int Lt, int bie, double c, const int32_t *__restrict__ e2c,
                      const double *__restrict__ ring, int nslot, int nc, int k1, const double *__restrict__ Dv,
                      const double *__restrict__ Dn, const double *__restrict__ tl, const double *__restrict__ dtl,
                      double *far, StepWhen w)
{
    if (w.alpha) {
        const int i = when_interval(w);
        if (i < 0) return;
        k1 = i + 1;
    }
    const double *Lloc = ring + (int64_t)(k1 % nslot) * nc * P3 * pt;
    const int lane = threadIdx.x & 31;
    const int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (i >= ns) return;  // whole warps leave together
    const double *L = Lloc + (int64_t)e2c[i] * P3 * pt;
    const double *dv = Dv + (int64_t)i * P3, *dn = Dn + (int64_t)i * P3;
    double yv[8], yn[8];
    for (int m = 0; m < 8; ++m) yv[m] = yn[m] = 0.0;
    for (int a = lane; a < P3; a += 32) {
        const double v = dv[a], w = bie ? dn[a] : 0.0;
#pragma unroll
        for (int m = 0; m < 8; ++m)
            if (m < pt) {
                const double Lam = L[a + P3 * m];
                yv[m] += v * Lam;
                yn[m] += w * Lam;
            }
    }
#pragma unroll
    for (int m = 0; m < 8; ++m)
        if (m < pt)
            for (int o = 16; o; o >>= 1) {
                yv[m] += __shfl_xor_sync(0xffffffffu, yv[m], o);
                yn[m] += __shfl_xor_sync(0xffffffffu, yn[m], o);
            }
    for (int t = lane; t < Lt; t += 32) {
        double s = 0.0;
#pragma unroll
        for (int m = 0; m < 8; ++m)
            if (m < pt) s += bie ? (tl[t * 8 + m] * yn[m] - dtl[t * 8 + m] * yv[m] / c) : tl[t * 8 + m] * yv[m];
        far[(int64_t)t * ns + i] = s;
    }
}

}  // namespace tdbem

namespace tdbem {

// M2L as dense GEMMs grouped by symmetry class of the cell offset.  Column
// j of a class's GEMM is one interaction pair (O, S) whose offset is g(c):
// it holds the source moment with its spatial node index permuted by g,
// B_j[b + P3 n] = M_S[g(b) + P3 n], so that the class's canonical operator
// stack applies; row a + P3 m + P blk of the product then belongs to node
// g(a) of O's local (a reduction reads it back through g^-1).
__global__ void k_m2l_gather(int64_t np, int P3, int P, const int32_t *__restrict__ pS, const uint8_t *__restrict__ pg,
                             const int16_t *__restrict__ perm, const double *__restrict__ M, double *B, StepWhen w)
{
    if (w.alpha && when_interval(w) < 0) return;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < np * P; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t col = e / P;
        const int r = (int)(e % P), b = r % P3;
        B[e] = M[(int64_t)pS[col] * P + perm[pg[col] * P3 + b] + (r - b)];
    }
}

// Terms of the split of x into nterm BF16 numbers, x ~ t_0 + t_1 + ..,
// t_k = bf16(x - t_0 - .. - t_{k-1}) (round to nearest), as bit patterns.
__device__ __forceinline__ void split_bf16(double x, int nterm, uint16_t *t)
{
    for (int k = 0; k < nterm; ++k) {
        const __nv_bfloat16 h = __double2bfloat16(x);
        t[k] = __bfloat16_as_ushort(h);
        x -= (double)__bfloat162float(h);
    }
}

// Gather with the split: Bt[k][col][r] for r < P (the columns' padding to Kp
// stays zero).
__global__ void k_m2l_gather_split(int64_t np, int P3, int P, int Kp, int nterm, const int32_t *__restrict__ pS,
                                   const uint8_t *__restrict__ pg, const int16_t *__restrict__ perm,
                                   const double *__restrict__ M, uint16_t *Bt, StepWhen w)
{
    if (w.alpha && when_interval(w) < 0) return;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < np * P; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t col = e / P;
        const int r = (int)(e % P), b = r % P3;
        uint16_t t[kTcMaxTerms];
        split_bf16(M[(int64_t)pS[col] * P + perm[pg[col] * P3 + b] + (r - b)], nterm, t);
        for (int k = 0; k < nterm; ++k) Bt[((int64_t)k * np + col) * Kp + r] = t[k];
    }
}

// Operator terms: opt[k][c][row][col] (row < R, col < P) from the FP64
// stacks op[c][row][col]; padding rows and columns stay zero.
__global__ void k_split_operators(int ncls, int R, int P, int Rp, int Kp, int nterm, const double *__restrict__ op,
                                  uint16_t *opt)
{
    const int64_t n = (int64_t)ncls * R * P;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int col = (int)(e % P);
        const int64_t cr = e / P;
        const int row = (int)(cr % R), c = (int)(cr / R);
        uint16_t t[kTcMaxTerms];
        split_bf16(op[e], nterm, t);
        for (int k = 0; k < nterm; ++k) opt[(((int64_t)k * ncls + c) * Rp + row) * Kp + col] = t[k];
    }
}

// Scaled FP16 form (precision 4): x = 2^e (h_0 + h_1) with h_0 = fp16(x 2^-e),
// h_1 = fp16(x 2^-e - h_0); the power of two puts the largest |entry| of a
// row (operators) or of a cell's moment (moments) in [2^13, 2^14), within
// FP16's range, so the two terms carry about 22 significant bits of every
// entry near that maximum.  The scales leave the GEMM's FP32 accumulation
// exact in exponent and are applied in its epilogue.
__device__ __forceinline__ int f16_exp(double m)
{
    return m > 0.0 ? ilogb(m) - 13 : 0;
}

__device__ __forceinline__ void split_f16(double x, uint16_t *t)
{
    const __half h0 = __double2half(x);
    t[0] = __half_as_ushort(h0);
    t[1] = __half_as_ushort(__double2half(x - (double)__half2float(h0)));
}

// Operator terms of the scaled FP16 form: one warp per operator row
// (class c, row < R): its largest |entry|, its scale ascale[c Rp + row] and
// the two FP16 terms of every entry.
__global__ void k_split_operators_f16(int ncls, int R, int P, int Rp, int Kp, const double *__restrict__ op,
                                      uint16_t *opt, float *ascale)
{
    const int lane = threadIdx.x & 31;
    const int64_t nrow = (int64_t)ncls * R;
    for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; w < nrow;
         w += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int c = (int)(w / R), row = (int)(w % R);
        const double *o = op + w * P;
        double m = 0.0;
        for (int k = lane; k < P; k += 32) m = fmax(m, fabs(o[k]));
        for (int sft = 16; sft; sft >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, sft));
        const int e = f16_exp(m);
        const double inv = ldexp(1.0, -e);
        for (int k = lane; k < P; k += 32) {
            uint16_t t[2];
            split_f16(o[k] * inv, t);
            opt[((int64_t)c * Rp + row) * Kp + k] = t[0];
            opt[(((int64_t)ncls + c) * Rp + row) * Kp + k] = t[1];
        }
        if (lane == 0) ascale[(int64_t)c * Rp + row] = ldexpf(1.f, e);
    }
}

// Scale exponent of every cell's moment (scaled FP16 form): one CTA per cell.
__global__ void k_cell_scale(int P, const double *__restrict__ M, int *cexp, StepWhen w)
{
    if (w.alpha && when_interval(w) < 0) return;
    __shared__ double red[8];
    const double *m = M + (int64_t)blockIdx.x * P;
    double v = 0.0;
    for (int k = threadIdx.x; k < P; k += blockDim.x) v = fmax(v, fabs(m[k]));
    for (int sft = 16; sft; sft >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, sft));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) v = fmax(v, red[k]);
        v = fmax(v, red[0]);
        cexp[blockIdx.x] = f16_exp(v);
    }
}

// Gather of the scaled FP16 form: Bt[k][col][r] = term k of M_S[g(b) +
// P3 n] 2^-e_S, and bscale[col] = 2^e_S.
__global__ void k_m2l_gather_f16(int64_t np, int P3, int P, int Kp, const int32_t *__restrict__ pS,
                                 const uint8_t *__restrict__ pg, const int16_t *__restrict__ perm,
                                 const double *__restrict__ M, const int *__restrict__ cexp, uint16_t *Bt,
                                 float *bscale, StepWhen w)
{
    if (w.alpha && when_interval(w) < 0) return;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < np * P; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t col = e / P;
        const int r = (int)(e % P), b = r % P3;
        const int S = pS[col], ex = cexp[S];
        uint16_t t[2];
        split_f16(ldexp(M[(int64_t)S * P + perm[pg[col] * P3 + b] + (r - b)], -ex), t);
        Bt[col * Kp + r] = t[0];
        Bt[(np + col) * Kp + r] = t[1];
        if (r == 0) bscale[col] = ldexpf(1.f, ex);
    }
}

// Largest |entry| of each (class, block) of the FP64 operator stacks, for
// skipping GEMM tiles whose rows are all zero (blocks before the wavefront
// reaches the node domain).  One CTA per (class, block).
__global__ void k_block_maxabs(int P, int nblk, const double *__restrict__ op, double *out)
{
    __shared__ double red[256];
    const double *q = op + (int64_t)blockIdx.x * P * P;
    double m = 0.0;
    for (int64_t e = threadIdx.x; e < (int64_t)P * P; e += blockDim.x) m = fmax(m, fabs(q[e]));
    red[threadIdx.x] = m;
    __syncthreads();
    for (int w = blockDim.x / 2; w; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

// Exact sum of two floats (two-sum of Knuth): a + b = s + e.
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float b)
{
    const float s = hi + b;
    const float bb = s - hi;
    lo += (hi - (s - bb)) + (b - bb);
    hi = s;
}

// Per observation cell O (one CTA): every row e = a' + P3 m + P blk of O's
// locals summed over O's pairs in interaction-list order, pair t's product
// read at row g_t^-1(a') + P3 m + P blk.  FP32 products are summed in
// double-float (a float pair updated by two-sums, about 48 bits): the far
// field cancels terms 1e4-1e5 larger than itself, so a plain FP32 sum is not
// enough, and FP64 adds are 57 times slower than FP32 ones on this GPU.
// Near-future rows go to the ring of locals, derivative rows to G.
template <typename TC>
__global__ void k_m2l_reduce(int nc, int P3, int P, int nblk, int mu, int nslot, int k, const int64_t *__restrict__ ooff,
                             const int64_t *__restrict__ oidx, const uint8_t *__restrict__ og,
                             const int16_t *__restrict__ iperm, const TC *__restrict__ C, double *ring, double *G,
                             StepWhen w)
{
    if (w.alpha && (k = when_interval(w)) < 0) return;
    __shared__ int64_t cols[kMaxIL];
    __shared__ int32_t gofs[kMaxIL];
    const int R = nblk * P;
    const int O = blockIdx.x;
    const int64_t t0 = ooff[O];
    const int nt = (int)(ooff[O + 1] - t0);
    for (int t = threadIdx.x; t < nt; t += blockDim.x) {
        cols[t] = oidx[t0 + t] * R;
        gofs[t] = og[t0 + t] * P3;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < R; e += blockDim.x) {
        const int a = e % P3, rest = e - a;
        double s = 0.0;
        if (sizeof(TC) == 4) {
            float hi = 0.f, lo = 0.f;
            int t = 0;
            for (; t + 8 <= nt; t += 8) {
                float f[8];
#pragma unroll
                for (int v = 0; v < 8; ++v) f[v] = (float)C[cols[t + v] + iperm[gofs[t + v] + a] + rest];
#pragma unroll
                for (int v = 0; v < 8; ++v) two_sum_acc(hi, lo, f[v]);
            }
            for (; t < nt; ++t) two_sum_acc(hi, lo, (float)C[cols[t] + iperm[gofs[t] + a] + rest]);
            s = (double)hi + (double)lo;
        } else {
            for (int t = 0; t < nt; ++t) s += (double)C[cols[t] + iperm[gofs[t] + a] + rest];
        }
        const int blk = e / P, r = e % P;
        if (blk <= mu)
            ring[((int64_t)((k + blk + 1) % nslot) * nc + O) * P + r] += s;
        else
            G[((int64_t)(blk - mu - 1) * nc + O) * P + r] = s;
    }
}

// The same reduction with coalesced reads (tensor-core forms): one CTA per
// (observation cell, chunk of rows [r0, r0 + nrow) of the range [rb, re),
// r0 and nrow multiples of P3); for
// each pair in list order the CTA reads the chunk of the pair's product
// contiguously and adds row a_c + rest to the double-float accumulator of
// row perm_g(a_c) + rest in shared memory (the same additions in the same
// order as k_m2l_reduce, so the same bits); a barrier between pairs.
__global__ void k_m2l_reduce_smem(int nc, int P3, int P, int nblk, int mu, int nslot, int k, int nrow, int rb,
                                  int re, const int64_t *__restrict__ ooff, const int64_t *__restrict__ oidx,
                                  const uint8_t *__restrict__ og, const int16_t *__restrict__ perm,
                                  const float *__restrict__ C, double *ring, StepWhen w)
{
    if (w.alpha && (k = when_interval(w)) < 0) return;
    extern __shared__ float acc[];  // [nrow] hi, [nrow] lo
    float *hi = acc, *lo = acc + nrow;
    const int R = nblk * P;
    const int O = blockIdx.x;
    const int r0 = rb + blockIdx.y * nrow;  // rows [rb, re), rb a multiple of P3
    const int n = min(nrow, re - r0);
    const int64_t t0 = ooff[O];
    const int nt = (int)(ooff[O + 1] - t0);
    for (int e = threadIdx.x; e < n; e += blockDim.x) hi[e] = lo[e] = 0.f;
    for (int t = 0; t < nt; ++t) {
        __syncthreads();
        const float *col = C + oidx[t0 + t] * R + r0;
        const int16_t *pg = perm + og[t0 + t] * P3;
        for (int e = threadIdx.x; e < n; e += blockDim.x) {
            const int a = (r0 + e) % P3;
            const int d = e - a + pg[a];
            float h = hi[d], l = lo[d];
            two_sum_acc(h, l, col[e]);
            hi[d] = h;
            lo[d] = l;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int row = r0 + e;
        const int blk = row / P, r = row % P;
        ring[((int64_t)((k + blk + 1) % nslot) * nc + O) * P + r] += (double)hi[e] + (double)lo[e];
    }
}

// Rows per CTA of k_m2l_reduce_smem: the largest multiple of P3 whose two
// float accumulators fit in shared memory.
static int reduce_rows(int P3, int R)
{
    const int per = (kTcSmemBudget / (2 * (int)sizeof(float))) / P3 * P3;
    return std::min(per, R);
}

// Distance powers between the nodes of a canonical offset's observation and
// source boxes: kr[c][e][a][b] = r_ab^(e-1) (e = 0: 1/r), e = 0..d (the
// slot e = 1, r^0 = 1, is not read), r_ab = |-c s + ho w_a - hs w_b|.
template <typename T>
__global__ void k_dist_powers(int ncls, int ps, int d, double s, double hs, double ho, const int32_t *__restrict__ codes,
                              T *out, bool eq)
{
    const int P3 = ps * ps * ps;
    const int64_t n = (int64_t)ncls * (d + 1) * P3 * P3;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(e % P3), a = (int)((e / P3) % P3);
        const int ex = (int)((e / ((int64_t)P3 * P3)) % (d + 1)), c = (int)(e / ((int64_t)P3 * P3 * (d + 1)));
        const int o = codes[c];
        const int dx = o % 7 - 3, dy = (o / 7) % 7 - 3, dz = o / 49 - 3;
        const int a1 = a % ps, a2 = (a / ps) % ps, a3 = a / (ps * ps);
        const int b1 = b % ps, b2 = (b / ps) % ps, b3 = b / (ps * ps);
        const double rx = -dx * s + ho * fmm_node(ps, a1, eq) - hs * fmm_node(ps, b1, eq);
        const double ry = -dy * s + ho * fmm_node(ps, a2, eq) - hs * fmm_node(ps, b2, eq);
        const double rz = -dz * s + ho * fmm_node(ps, a3, eq) - hs * fmm_node(ps, b3, eq);
        const double r = sqrt(rx * rx + ry * ry + rz * rz);
        double v = 1.0 / r;
        for (int k = 0; k < ex; ++k) v *= r;
        if constexpr (std::is_same<T, double>::value) {
            out[e] = v;
        } else {
            const float hi = (float)v;
            out[e] = make_float2(hi, (float)(v - (double)hi));
        }
    }
}

// Double-float (a float pair, ~48 bits) arithmetic: acc += x y by the exact
// FMA two-product of the leading parts and the two-sum of Knuth; df_add
// adds two double-float numbers.
__device__ __forceinline__ void df_fma(float2 &acc, float2 x, float2 y)
{
    const float p = x.x * y.x;
    const float pe = fmaf(x.x, y.x, -p) + (x.x * y.y + x.y * y.x);
    const float s = acc.x + p;
    const float bb = s - acc.x;
    const float e = (acc.x - (s - bb)) + (p - bb);
    const float lo = acc.y + pe + e;
    acc.x = s + lo;
    acc.y = lo - (acc.x - s);
}

__device__ __forceinline__ float2 df_add(float2 a, float2 b)
{
    const float s = a.x + b.x;
    const float bb = s - a.x;
    const float e = (a.x - (s - bb)) + (b.x - bb) + a.y + b.y;
    const float hi = s + e;
    return make_float2(hi, e - (hi - s));
}

template <typename T>
__device__ __forceinline__ void gen_fma(T &acc, T x, T y)
{
    if constexpr (std::is_same<T, double>::value) acc = fma(x, y, acc);
    else df_fma(acc, x, y);
}

template <typename T>
__device__ __forceinline__ T gen_add(T a, T b)
{
    if constexpr (std::is_same<T, double>::value) return a + b;
    else return df_add(a, b);
}

template <typename T>
__device__ __forceinline__ T gen_shfl(T v, int o)
{
    if constexpr (std::is_same<T, double>::value) return __shfl_xor_sync(0xffffffffu, v, o);
    else return make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}

template <typename T>
__device__ __forceinline__ double gen_val(T v)
{
    if constexpr (std::is_same<T, double>::value) return v;
    else return (double)v.x + (double)v.y;
}

template <typename T>
__device__ __forceinline__ T gen_from(double v)
{
    if constexpr (std::is_same<T, double>::value) {
        return v;
    } else {
        const float hi = (float)v;
        return make_float2(hi, (float)(v - (double)hi));
    }
}

// The last near-future block (p = 0: the local L_{k+mu+1,k} itself) and the
// derivative contributions G_p (p = 1..d) of one level's M2L (the U^(p) of
// Eq. U_expand at I_{k+mu+1}, applied to the moments of every interaction
// pair of a cell), from the binomial expansion of
// U^(p) = C(d,p) z^q / r, q = d - p, z = A + c ht w_m - c ht w_n - r,
// A = c ((mu+1) T + 1) dt (mu is chosen so that z > 0 on the whole node
// domain of I_{k+mu+1} x J_k, so the kernel there is this polynomial):
//   G_p[a, m] = C(d,p) sum_{i+j+k=q} q!/(i! j! k!) (c ht w_m)^i (-c ht)^j
//               sum_{e<=k} C(k,e) A^(k-e) (-1)^e F_{e,j}[a],
//   F_{e,j}[a] = sum_pairs sum_b r_ab^(e-1) mu_j[b],  mu_j[b] = sum_n w_n^j M[b, n]
// (the pair's moment, node indices permuted by its symmetry element).  So
// these rows need spatial products only (e + j <= d; e = 1 is a plain sum)
// instead of d + 1 P x P operator blocks per pair; they are summed in FP64
// (FP64 form) or double-float (tensor-core forms): the distant-future
// recurrence starts from L_{k+mu+1} and adds the G_p of every later
// interval, so it carries their rounding into every later interval (an
// FP32-grade L_{k+mu+1} made the march drift linearly in time), and
// amplifies the G_p's with the square of the number of intervals.  One CTA per observation cell; per pair, one warp
// per observation node at a time, its lanes striding the source nodes.
// Kernel 1: time moments j = 0..d of every GEMM column (pair), node indices
// permuted by the column's symmetry element (template D = d + 1 moments):
//   mu[col][j][b] = sum_n w_n^j M_S[g(b) + P3 n],  ssum[col][j] = sum_b mu[col][j][b].
template <typename T, int D>
__global__ void k_deriv_moments(int64_t np, int P3, int pt, const int32_t *__restrict__ pS,
                                const uint8_t *__restrict__ pg, const int16_t *__restrict__ perm,
                                const double *__restrict__ wt, const double *__restrict__ M, T *mu, double *ssum,
                                StepWhen w)
{
    if (w.alpha && when_interval(w) < 0) return;
    const int64_t col = blockIdx.x;
    const int P = P3 * pt;
    const int Sc = pS[col], g = pg[col];
    double wn[kMaxP];
#pragma unroll
    for (int n = 0; n < kMaxP; ++n) wn[n] = n < pt ? wt[n] : 0.0;
    double part[D];
#pragma unroll
    for (int j = 0; j < D; ++j) part[j] = 0.0;
    for (int b = threadIdx.x; b < P3; b += blockDim.x) {
        const double *m = M + (int64_t)Sc * P + perm[g * P3 + b];
        double w[D];
#pragma unroll
        for (int j = 0; j < D; ++j) w[j] = 0.0;
        for (int n = 0; n < pt; ++n) {
            const double x = m[(int64_t)P3 * n];
            double pw = 1.0;
#pragma unroll
            for (int j = 0; j < D; ++j) {
                w[j] += pw * x;
                pw *= wn[n];
            }
        }
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const T v = gen_from<T>(w[j]);
            mu[(col * D + j) * P3 + b] = v;
            part[j] += gen_val(v);
        }
    }
    __shared__ double red[D][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < D; ++j) {
        double v = part[j];
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[j][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < D) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[threadIdx.x][w];
        ssum[col * D + threadIdx.x] = v;
    }
}

// Kernel 2: per symmetry class, the distance-power matrices times the
// columns' time moments, in FP64 or double-float on the CUDA cores:
//   Fp[col][e][j][a] = sum_b r_ab^(e-1) mu[col][j][b]  (e != 1, e + j <= D - 1),
// a in the canonical node order (D = d + 1).  One CTA per (class, 8
// columns), one thread per row a; the matrices go through shared memory cw
// columns at a time (rows padded to cw + 1 entries), so each chunk serves 8
// columns, in two buffers: the next chunk is copied (cp.async, 8 bytes per
// entry) while the current one is used.
constexpr int kDerivCols = 8;

__device__ __forceinline__ void cp_async8(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <typename T>
__device__ __forceinline__ void deriv_chunk_load(const T *__restrict__ K, int P3, int cw, int b0, T *buf)
{
    for (int x = threadIdx.x; x < P3 * cw; x += blockDim.x) {
        const int row = x / cw, cc = x % cw;
        T *dst = buf + row * (cw + 1) + cc;
        if (b0 + cc < P3)
            cp_async8(dst, K + (int64_t)row * P3 + b0 + cc);
        else
            *dst = gen_from<T>(0.0);
    }
}

template <typename T, int D>
__global__ void __launch_bounds__(512) k_deriv_products(int P3, int cw, const int4 *__restrict__ jobs, const T *__restrict__ kr,
                                 const T *__restrict__ mu, T *Fp, StepWhen w)
{
    if (w.alpha && when_interval(w) < 0) return;
    extern __shared__ double shm_d[];
    T *mus = reinterpret_cast<T *>(shm_d);    // [kDerivCols][D][P3]
    T *kc[2] = {mus + kDerivCols * D * P3, mus + kDerivCols * D * P3 + P3 * (cw + 1)};  // [P3][cw + 1] each
    const int4 job = jobs[blockIdx.x];        // class, first column, columns
    const int cls = job.x, ncol = job.z;
    const int64_t col0 = job.y;
    const int r = threadIdx.x;
    for (int x = threadIdx.x; x < kDerivCols * D * P3; x += blockDim.x) {
        const int t = x / (D * P3);
        mus[x] = t < ncol ? mu[col0 * D * P3 + x] : gen_from<T>(0.0);
    }
    const int nch = (P3 + cw - 1) / cw;
#pragma unroll
    for (int e = 0; e < D; ++e) {
        if (e == 1) continue;
        T acc[kDerivCols][D];
#pragma unroll
        for (int t = 0; t < kDerivCols; ++t)
#pragma unroll
            for (int j = 0; j < D; ++j) acc[t][j] = gen_from<T>(0.0);
        const T *K = kr + ((int64_t)cls * D + e) * P3 * P3;
        __syncthreads();  // both buffers free (previous e done)
        deriv_chunk_load(K, P3, cw, 0, kc[0]);
        cp_async_commit();
        for (int ci = 0; ci < nch; ++ci) {
            const int b0 = ci * cw;
            if (ci + 1 < nch) {
                deriv_chunk_load(K, P3, cw, b0 + cw, kc[(ci + 1) & 1]);
                cp_async_commit();
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();
            if (r < P3) {
                const T *kb = kc[ci & 1];
                const int nb = min(cw, P3 - b0);
                for (int cc = 0; cc < nb; ++cc) {
                    const T x = kb[r * (cw + 1) + cc];
#pragma unroll
                    for (int t = 0; t < kDerivCols; ++t)
#pragma unroll
                        for (int j = 0; j + e < D; ++j) gen_fma(acc[t][j], x, mus[(t * D + j) * P3 + b0 + cc]);
                }
            }
            __syncthreads();  // kc[ci & 1] is refilled by the next iteration's copy
        }
        if (r < P3)
#pragma unroll
            for (int t = 0; t < kDerivCols; ++t)
                if (t < ncol)
#pragma unroll
                    for (int j = 0; j + e < D; ++j)
                        Fp[(((col0 + t) * D + e) * D + j) * P3 + r] = acc[t][j];
    }
}

// Kernel 3: per observation cell, F_{e,j}[a'] = sum over its pairs (list
// order) of Fp[col][e][j][g^-1(a')], and S_j = sum of ssum; then
// V_p[a', m] = sum_{e,j} coef[p][m][e][j] F_{e,j}[a'] (F_{1,j} = S_j), with
// the binomial-expansion coefficients of Eq. U_expand tabulated per level
// at setup (deriv_coef_table): V_0 is added to the local L_{k+mu+1} (ring
// slot k + mu + 1), V_p (p >= 1) is G_p.  D = d + 1.
template <typename T, int D>
__global__ void k_deriv_assemble(int nc, int P3, int pt, int nslot, int k, int mu, const int64_t *__restrict__ ooff,
                                 const int64_t *__restrict__ oidx, const uint8_t *__restrict__ og,
                                 const int16_t *__restrict__ iperm, const T *__restrict__ Fp,
                                 const double *__restrict__ ssum, const double *__restrict__ coef, double *ring,
                                 double *G, StepWhen w)
{
    if (w.alpha && (k = when_interval(w)) < 0) return;
    const int O = blockIdx.x;
    const int P = P3 * pt;
    const int64_t t0 = ooff[O], t1 = ooff[O + 1];
    __shared__ double S[D];
    if (threadIdx.x < D) {
        double v = 0.0;
        for (int64_t t = t0; t < t1; ++t) v += ssum[oidx[t] * D + threadIdx.x];
        S[threadIdx.x] = v;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < P3; r += blockDim.x) {
        T F[D][D];
#pragma unroll
        for (int e = 0; e < D; ++e)
#pragma unroll
            for (int j = 0; j < D; ++j) F[e][j] = gen_from<T>(0.0);
        for (int64_t t = t0; t < t1; ++t) {
            const int64_t col = oidx[t];
            const int a = iperm[og[t] * P3 + r];
#pragma unroll
            for (int e = 0; e < D; ++e) {
                if (e == 1) continue;
#pragma unroll
                for (int j = 0; j + e < D; ++j) F[e][j] = gen_add(F[e][j], Fp[((col * D + e) * D + j) * P3 + a]);
            }
        }
        double Fv[D][D];
#pragma unroll
        for (int e = 0; e < D; ++e)
#pragma unroll
            for (int j = 0; j < D; ++j) Fv[e][j] = (e == 1) ? S[j] : gen_val(F[e][j]);
        for (int p = 0; p < D; ++p)
            for (int m = 0; m < pt; ++m) {
                const double *cf = coef + ((int64_t)p * pt + m) * D * D;
                double v = 0.0;
#pragma unroll
                for (int e = 0; e < D; ++e)
#pragma unroll
                    for (int j = 0; j + e < D; ++j) v += cf[e * D + j] * Fv[e][j];
                if (p == 0)
                    ring[((int64_t)((k + mu + 1) % nslot) * nc + O) * P + r + (int64_t)P3 * m] += v;
                else
                    G[((int64_t)(p - 1) * nc + O) * P + r + (int64_t)P3 * m] = v;
            }
    }
}

// Shared memory of the products kernel (the columns' moments and two
// chunk buffers) and its chunk width: 32 columns of the distance-power
// matrices, else 16 or 8, whichever fits first.
static size_t deriv_shm(int D, int P3, size_t el, int *cw)
{
    size_t b = 0;
    for (int w : {32, 16, 8}) {
        *cw = w;
        b = ((size_t)kDerivCols * D * P3 + 2 * (size_t)P3 * (w + 1)) * el;
        if (b <= (size_t)kTcSmemBudget) break;
    }
    return b;
}

// D = d + 1 (moments j = 0..d, distance powers e = 0..d, rows p = 0..d).
// parts: bit 0 the time moments (they read the level's moments M), bit 1
// the products and the assembly (they read only the moments' products).
template <typename T, int D>
static cudaError_t launch_deriv_d(int nc, int P3, int pt, int nslot, int k, int mu, const FmmLevel &V,
                                  const double *wt, const int16_t *perm, const int16_t *iperm, cudaStream_t s,
                                  StepWhen w, int parts)
{
    T *dm = reinterpret_cast<T *>(V.dmu), *Fp = reinterpret_cast<T *>(V.dF);
    const int bdim = std::max(128, (P3 + 31) / 32 * 32);
    if (parts & 1)
        k_deriv_moments<T, D><<<(unsigned)V.np, 128, 0, s>>>(V.np, P3, pt, V.pS, V.pg, perm, wt, V.M, dm, V.dss, w);
    if (!(parts & 2)) return cudaGetLastError();
    int cw = 32;
    const size_t shm = deriv_shm(D, P3, sizeof(T), &cw);
    if (shm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_deriv_products<T, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)shm);
        if (e != cudaSuccess) return e;
    }
    k_deriv_products<T, D><<<V.njobs, bdim, shm, s>>>(P3, cw, V.djobs, reinterpret_cast<const T *>(V.kr), dm, Fp, w);
    k_deriv_assemble<T, D><<<nc, 256, 0, s>>>(nc, P3, pt, nslot, k, mu, V.ooff, V.oidx, V.og, iperm, Fp, V.dss,
                                              V.dcoef, V.ring, V.G, w);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_deriv(int d, int nc, int P3, int pt, int nslot, int k, int mu, const FmmLevel &V,
                                const double *wt, const int16_t *perm, const int16_t *iperm, cudaStream_t s,
                                StepWhen w, int parts)
{
    switch (d) {
    case 1: return launch_deriv_d<T, 2>(nc, P3, pt, nslot, k, mu, V, wt, perm, iperm, s, w, parts);
    case 2: return launch_deriv_d<T, 3>(nc, P3, pt, nslot, k, mu, V, wt, perm, iperm, s, w, parts);
    case 3: return launch_deriv_d<T, 4>(nc, P3, pt, nslot, k, mu, V, wt, perm, iperm, s, w, parts);
    default: return launch_deriv_d<T, 5>(nc, P3, pt, nslot, k, mu, V, wt, perm, iperm, s, w, parts);
    }
}

// Zeroes a level's moment accumulator after its M2M (graph-replayed steps;
// plain stepping uses a memset).
__global__ void k_zero_when(int64_t n, double *x, StepWhen w)
{
    if (when_interval(w) < 0) return;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        x[e] = 0.0;
}


namespace {

double h_node(int p, int a, bool eq)
{
    if (eq) return p > 1 ? -1.0 + 2.0 * a / (p - 1) : 0.0;
    return cos((2.0 * a + 1.0) * M_PI / (2.0 * p));
}

void h_lagrange(int p, double xi, double *val, double *der, bool eq)
{
    for (int a = 0; a < p; ++a) {
        double v = 1.0, dv = 0.0;
        for (int b = 0; b < p; ++b) {
            if (b == a) continue;
            double den = h_node(p, a, eq) - h_node(p, b, eq);
            double f = (xi - h_node(p, b, eq)) / den;
            dv = dv * f + v / den;
            v *= f;
        }
        val[a] = v;
        if (der) der[a] = dv;
    }
}

// Gauss-Legendre nodes and weights on [0, 1] (Newton on P_n).
void gauss_legendre01(int n, std::vector<double> &x, std::vector<double> &w)
{
    x.resize(n);
    w.resize(n);
    for (int i = 0; i < n; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            double pn = (n == 1) ? z : p1, pm = (n == 1) ? 1.0 : p0;
            dp = n * (z * pn - pm) / (z * z - 1.0);
            double dz = pn / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = 0.5 * (1.0 - z);
        w[i] = 1.0 / ((1.0 - z * z) * dp * dp);
    }
}

template <typename T>
cudaError_t falloc(tdbem_ctx *c, T **p, size_t n)
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

}  // namespace

#define F_TRY(x)                        \
    do {                                \
        cudaError_t e_ = (x);           \
        if (e_ != cudaSuccess) return e_; \
    } while (0)

// Symmetries of the cube: g = 8 pi + sigma acts on vectors as
// (g v)_k = s_k v_{pi(k)}, pi the permutation kPerm[pi] of the axes and s_k =
// -1 where bit k of sigma is set.  On a node multi-index of p Chebyshev
// points per axis (w_{p-1-i} = -w_i) it acts as (g b)_k = b_{pi(k)}, or
// p - 1 - b_{pi(k)} where s_k = -1.
static const int kPerm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

static int sym_node(int p, int g, int b)
{
    const int *pi = kPerm[g >> 3];
    const int bb[3] = {b % p, (b / p) % p, b / (p * p)};
    int out[3];
    for (int k = 0; k < 3; ++k) out[k] = ((g >> k) & 1) ? p - 1 - bb[pi[k]] : bb[pi[k]];
    return out[0] + p * (out[1] + p * out[2]);
}

// o = g(c) with c the canonical offset (|c_0| >= |c_1| >= |c_2| >= 0, ties in
// axis order); returns g.
static int sym_decompose(const int o[3], int c[3])
{
    int idx[3] = {0, 1, 2};
    std::stable_sort(idx, idx + 3, [&](int x, int y) { return abs(o[x]) > abs(o[y]); });
    int pi[3];
    for (int r = 0; r < 3; ++r) {
        c[r] = abs(o[idx[r]]);
        pi[idx[r]] = r;
    }
    int pidx = 0;
    while (!(kPerm[pidx][0] == pi[0] && kPerm[pidx][1] == pi[1] && kPerm[pidx][2] == pi[2])) ++pidx;
    int sigma = 0;
    for (int k = 0; k < 3; ++k)
        if (o[k] < 0) sigma |= 1 << k;
    return 8 * pidx + sigma;
}

// GEMM tiles of one level for tile width bn: per class, the 128-row blocks
// of its operator stack that are not all zero (bm: largest |entry| of every
// (class, stack block)), times its columns in chunks of bn; *flops = the
// algorithmic flops of the tiles kept.
// The tiles whose rows start in the first near-future block (r0 < P) come
// first (*nu of them, *flops_u their flops), then the others.
static std::vector<TcTile> m2l_tiles(const Fmm &F, const FmmLevel &V, int bn, const std::vector<double> &bm,
                                     double *flops, int *nu = nullptr, double *flops_u = nullptr)
{
    std::vector<TcTile> t;
    double fl = 0.0;
    if (flops_u) *flops_u = 0.0;
    for (int part = 0; part < 2; ++part) {
        for (int ci = 0; ci < V.ncls; ++ci) {
            const int64_t n = V.cbase[ci + 1] - V.cbase[ci];
            if (n == 0) continue;
            for (int r0 = 0; r0 < F.R; r0 += kTcBM) {
                if ((r0 < F.P) != (part == 0)) continue;
                const int r1 = std::min(F.R, r0 + kTcBM);
                bool zero = true;
                for (int blk = r0 / F.P; blk <= (r1 - 1) / F.P; ++blk)
                    if (bm[(size_t)ci * F.ngb + blk] != 0.0) zero = false;
                if (zero) continue;  // these rows of the products stay zero
                fl += 2.0 * (r1 - r0) * F.P * (double)n;
                if (part == 0 && flops_u) *flops_u += 2.0 * (r1 - r0) * F.P * (double)n;
                for (int64_t j0 = 0; j0 < n; j0 += bn)
                    t.push_back({ci * F.Rp + r0, (int32_t)(V.cbase[ci] + j0), r1 - r0,
                                 (int32_t)std::min<int64_t>(bn, n - j0), (V.cbase[ci] + j0) * (int64_t)F.R + r0});
            }
        }
        if (part == 0 && nu) *nu = (int)t.size();
    }
    *flops = fl;
    return t;
}

static TcGemmArgs m2l_args(tdbem_ctx *c, const FmmLevel &V, StepWhen w = StepWhen{}, int gsel = 0)
{
    const Fmm &F = c->fmm;
    TcGemmArgs g{};
    g.nta = F.nta;
    g.ntb = F.ntb;
    g.a_term_rows = V.ncls * F.Rp;
    g.b_term_rows = (int32_t)V.np;
    g.nprod = F.nprod;
    for (int p = 0; p < F.nprod; ++p) g.prod[p] = F.prod[p];
    g.kchunks = F.Kp / kTcBK;
    g.nstage = tc_stages(F.nta, F.ntb, V.tile_n);
    g.fmt = F.f16 ? 0 : 1;
    g.a_scale = F.f16 ? V.ascale : nullptr;
    g.b_scale = F.f16 ? V.bscale : nullptr;
    g.ldc = F.R;
    g.C = V.C32;
    g.tiles = gsel == 2 ? V.tiles + V.ntiles_u : V.tiles;
    g.err = c->d_flag;
    g.when = w;
    return g;
}

// The products of one M2L application: every class's canonical operator
// stack times its gathered columns.
// gsel: 0 every tile; 1 the tiles of the first near-future block (rows
// below P); 2 the others (the tile list keeps the first ones in front).
static cudaError_t m2l_products(tdbem_ctx *c, FmmLevel &V, StepWhen w = StepWhen{}, int gsel = 0)
{
    Fmm &F = c->fmm;
    if (c->split) {
        const int nt = gsel == 0 ? V.ntiles : gsel == 1 ? V.ntiles_u : V.ntiles - V.ntiles_u;
        // the deferred tiles run beside the history sums: half the SMs
        return tc_gemm_launch(V.mapA, V.mapB, m2l_args(c, V, w, gsel), nt, V.tile_n, c->s, gsel == 2 ? 2 : 1);
    }
    if (gsel == 2) return cudaSuccess;  // the FP64 form's GEMMs run whole (no deferred part)
    if (w.alpha) return cudaErrorNotSupported;  // the FP64 form's library GEMMs cannot be predicated
    const double one = 1.0, zero = 0.0;
    for (int ci = 0; ci < V.ncls; ++ci) {
        const int64_t c0 = V.cbase[ci], n = V.cbase[ci + 1] - c0;
        if (n == 0) continue;
        cublasStatus_t st = cublasDgemm(F.blas, CUBLAS_OP_T, CUBLAS_OP_N, F.R, (int)n, F.P, &one,
                                        V.op + (size_t)ci * F.R * F.P, F.P, V.Bbuf + (size_t)c0 * F.P, F.P, &zero,
                                        V.Cbuf + (size_t)c0 * F.R, F.R);
        if (st != CUBLAS_STATUS_SUCCESS) {
            c->err = "cuBLAS status " + std::to_string((int)st) + " in the FP64 M2L GEMM";
            return cudaErrorUnknown;
        }
    }
    return cudaSuccess;
}

// Coefficients of the rows of the last near-future block (p = 0) and the
// derivative rows (p = 1..d) (Eq. U_expand expanded binomially in the time
// nodes): U^(p) = C(d,p) z^q / r, q = d - p, z = A + cht w_m - cht w_n - r,
// A = c ((mu+1) T + 1) dt, cht = c T dt / 2, gives
// V_p[a,m] = sum_{e,j} coef[p][m][e][j] F_{e,j}[a] with F_{e,j}[a] =
// sum_b r_ab^(e-1) sum_n w_n^j M[b,n] and
// coef = C(d,p) sum_{i+j+k=q, k>=e} C(q,i) C(q-i,j) (cht w_m)^i (-cht)^j C(k,e) A^(k-e) (-1)^e
// (layout [d+1][pt][d+1][d+1]).
static std::vector<double> deriv_coef_table(int d, int pt, double A, double cht, bool eq)
{
    auto binom = [](int n, int k) {
        double v = 1.0;
        for (int i = 0; i < k; ++i) v = v * (n - i) / (i + 1);
        return v;
    };
    const int E = d + 1;
    std::vector<double> t((size_t)E * pt * E * E, 0.0);
    for (int p = 0; p <= d; ++p) {
        const int q = d - p;
        for (int m = 0; m < pt; ++m) {
            const double wm = h_node(pt, m, eq);
            for (int i = 0; i <= q; ++i)
                for (int j = 0; i + j <= q; ++j) {
                    const int k = q - i - j;
                    for (int e = 0; e <= k; ++e)
                        t[(((size_t)p * pt + m) * E + e) * E + j] +=
                            binom(d, p) * binom(q, i) * binom(q - i, j) * std::pow(cht * wm, i) * std::pow(-cht, j) *
                            binom(k, e) * std::pow(A, k - e) * ((e & 1) ? -1.0 : 1.0);
                }
        }
    }
    return t;
}

// Tile-width tuner of the tensor-core M2L (the level's classes, column
// counts and zero blocks are fixed): times the level's GEMM with 128- and
// 256-column tiles on its real operators, keeps the faster and uploads its
// tile list and the moments' tensor map.
static cudaError_t m2l_tune(tdbem_ctx *c, FmmLevel &V, const std::vector<double> &bm)
{
    Fmm &F = c->fmm;
    cudaStream_t s = c->s;
    double fl = 0.0;
    std::vector<TcTile> t128 = m2l_tiles(F, V, 128, bm, &fl);
    F_TRY(falloc(c, &V.tiles, std::max<size_t>(t128.size(), 1)));
    cudaEvent_t e0, e1;
    F_TRY(cudaEventCreate(&e0));
    F_TRY(cudaEventCreate(&e1));
    int best = 128;
    float best_ms = 1e30f;
    V.tune.clear();
    cudaError_t err = cudaSuccess;
    for (int bn : {128, 256}) {
        std::vector<TcTile> t = bn == 128 ? t128 : m2l_tiles(F, V, bn, bm, &fl);
        if ((err = cudaMemcpyAsync(V.tiles, t.data(), t.size() * sizeof(TcTile), cudaMemcpyHostToDevice, s)) !=
            cudaSuccess)
            break;
        if ((err = tc_make_map(&V.mapB, V.Bt, (int64_t)F.ntb * V.np, F.Kp, bn)) != cudaSuccess) break;
        V.tile_n = bn;
        V.ntiles = (int)t.size();
        if ((err = m2l_products(c, V)) != cudaSuccess) break;  // warm-up
        cudaEventRecord(e0, s);
        err = m2l_products(c, V);
        cudaEventRecord(e1, s);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        if (err != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        V.tune.push_back({bn, ms});
        if (ms < best_ms) {
            best_ms = ms;
            best = bn;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return err;
    std::vector<TcTile> t = m2l_tiles(F, V, best, bm, &fl, &V.ntiles_u, &V.flops_u);
    F_TRY(cudaMemcpyAsync(V.tiles, t.data(), t.size() * sizeof(TcTile), cudaMemcpyHostToDevice, s));
    F_TRY(tc_make_map(&V.mapB, V.Bt, (int64_t)F.ntb * V.np, F.Kp, best));
    V.tile_n = best;
    V.ntiles = (int)t.size();
    V.flops_app = fl;
    int flag = 0;
    F_TRY(cudaMemcpyAsync(&flag, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    F_TRY(cudaStreamSynchronize(s));
    return (flag & 8) ? cudaErrorLaunchTimeout : cudaSuccess;
}

// Hierarchy parameters, per-element P2M/L2P tables, transfer matrices and
// the M2L operator banks (setup; after the tree is built).
cudaError_t fmm_setup(tdbem_ctx *c, std::string &why)
{
    Fmm &F = c->fmm;
    const int ns = c->ns, L = c->P.depth, d = c->P.d;
    F.on = true;
    F.L = L;
    F.ps = c->P.ps;
    F.pt = c->P.pt;
    if (F.ps < 2 || F.ps > kMaxP || F.pt < 2 || F.pt > kMaxP || L < 2) {
        why = "FMM needs 2 <= ps, pt <= 8 and depth >= 2";
        return cudaSuccess;
    }
    F.P3 = F.ps * F.ps * F.ps;
    F.P = F.P3 * F.pt;
    // precision 5: near-future M2L blocks by the FFT, on equispaced nodes
    // with the observation box equal to the source box (Toeplitz blocks)
    F.fft = c->P.precision == 5;
    F.fNs = 2 * F.ps;
    F.fNt = 2 * F.pt;
    F.fN = (int64_t)F.fNs * F.fNs * F.fNs * F.fNt;
    if (F.P > 4096) {
        why = "FMM needs ps^3 pt <= 4096";
        return cudaSuccess;
    }
    {
        int cw = 0;
        if (deriv_shm(d + 1, F.P3, c->split ? sizeof(float2) : sizeof(double), &cw) > (size_t)kTcSmemBudget) {
            why = "FMM: ps^3 too large for the exact rows at this B-spline order";
            return cudaSuccess;
        }
    }
    double box[4];
    F_TRY(cudaMemcpy(box, c->tree.box, sizeof(box), cudaMemcpyDeviceToHost));
    unsigned long long *d_rho = nullptr;
    F_TRY(cudaMalloc(&d_rho, sizeof(unsigned long long)));
    F_TRY(cudaMemset(d_rho, 0, sizeof(unsigned long long)));
    k_rho<<<(ns + 127) / 128, 128, 0, c->s>>>(ns, c->d_xyz, c->d_tri, c->d_xc, d_rho);
    unsigned long long rb = 0;
    F_TRY(cudaMemcpyAsync(&rb, d_rho, sizeof(rb), cudaMemcpyDeviceToHost, c->s));
    F_TRY(cudaStreamSynchronize(c->s));
    cudaFree(d_rho);
    memcpy(&F.rho, &rb, sizeof(double));
    const double cdt = c->cdt;
    F.lev.assign(L + 1, FmmLevel{});
    for (int l = 0; l <= L; ++l) {
        F.lev[l].s = box[3] / (double)(1 << l);
        F.lev[l].hs = F.lev[l].s / 2.0 + F.rho;
        F.lev[l].ho = F.fft ? F.lev[l].hs : F.lev[l].s / 2.0;
    }
    F.Lt = (int)floor((F.lev[L].s - F.rho) / cdt);
    if (F.Lt < 1 || !(2.0 * F.rho < F.lev[L].s)) {
        why = "infeasible hierarchy: leaf cells too small for c dt and the element size";
        return cudaSuccess;
    }
    int mu = 0;
    for (int l = 2; l <= L; ++l) {
        F.lev[l].T = F.Lt << (L - l);
        double rmax = sqrt(3.0) * (3.0 * F.lev[l].s + F.lev[l].hs + F.lev[l].ho);
        mu = std::max(mu, (int)floor((rmax / cdt - 1.0) / F.lev[l].T) + 1);
    }
    F.lev[L].T = F.Lt;
    F.mu = std::max(mu, c->P.mu);
    F.nblk = F.mu + 1 + d;
    F.nd = d * (d - 1) / 2;
    F.nslot = F.mu + 2;
    const int P = F.P, P3 = F.P3, ps = F.ps, pt = F.pt;
    if (2 * P * sizeof(double) > 48 * 1024) {
        // M2M and L2L stage two [P] tensors in shared memory (64 KB at P = 4096)
        F_TRY(cudaFuncSetAttribute(k_m2m, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(2 * P * sizeof(double))));
        F_TRY(cudaFuncSetAttribute(k_l2l, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(2 * P * sizeof(double))));
    }
    // operator blocks applied as GEMMs: the near future l = 1..mu; the block
    // l = mu + 1 lies wholly in the polynomial regime and is formed exactly
    // with the derivative rows (k_deriv_*), since the recurrence of Formula 1
    // starts from it
    F.ngb = F.mu;
    F.R = F.ngb * P;
    F.Rp = (F.R + kTcBM - 1) / kTcBM * kTcBM;
    F.Kp = (P + kTcBK - 1) / kTcBK * kTcBK;
    if (!c->split) {
        // FP64 form: the products are FP64 GEMMs of the library
        if (cublasCreate(&F.blas) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
        cublasSetStream(F.blas, c->s);
        cublasSetMathMode(F.blas, CUBLAS_DEFAULT_MATH);
    } else {
        // the second stream of the deferred boundary work (fmm_boundary), at
        // the lowest priority
        int lo_prio = 0, hi_prio = 0;
        F_TRY(cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio));
        F_TRY(cudaStreamCreateWithPriority(&F.side, cudaStreamNonBlocking, lo_prio));
        F_TRY(cudaEventCreateWithFlags(&F.ev_urgent, cudaEventDisableTiming));
        F_TRY(cudaEventCreateWithFlags(&F.ev_deferred, cudaEventDisableTiming));
        // tensor-core forms: BF16 terms of operators and moments, and the
        // products (A term, B term) kept: all with s + t < nterm
        // (precision 4: two FP16 terms with power-of-two scales, products
        // (0,0), (0,1), (1,0))
        const int nterm = F.fft ? 0 : c->P.precision == 1 ? 3 : (c->P.precision == 2 || c->P.precision == 4) ? 2 : 1;
        F.nta = F.ntb = nterm;
        F.f16 = c->P.precision == 4;
        F.nprod = 0;
        for (int sum = 0; sum < nterm; ++sum)
            for (int a = 0; a <= sum; ++a) F.prod[F.nprod++] = (a << 4) | (sum - a);
    }
    // node permutations of the 48 symmetries of the cube
    {
        std::vector<int16_t> pm(48 * P3), ip(48 * P3);
        for (int g = 0; g < 48; ++g)
            for (int b = 0; b < P3; ++b) {
                const int gb = sym_node(ps, g, b);
                pm[g * P3 + b] = (int16_t)gb;
                ip[g * P3 + gb] = (int16_t)b;
            }
        F_TRY(falloc(c, &F.perm, pm.size()));
        F_TRY(falloc(c, &F.iperm, ip.size()));
        F_TRY(cudaMemcpyAsync(F.perm, pm.data(), pm.size() * sizeof(int16_t), cudaMemcpyHostToDevice, c->s));
        F_TRY(cudaMemcpyAsync(F.iperm, ip.data(), ip.size() * sizeof(int16_t), cudaMemcpyHostToDevice, c->s));
        F_TRY(cudaStreamSynchronize(c->s));
    }

    // per-element tables (leaf boxes)
    F_TRY(falloc(c, &F.At, (size_t)ns * P3));
    F_TRY(falloc(c, &F.As, (size_t)ns * P3));
    F_TRY(falloc(c, &F.Dv, (size_t)ns * P3));
    F_TRY(falloc(c, &F.Dn, (size_t)ns * P3));
    std::vector<double> qx, qw;
    int nq = 2 * ps + 2;
    gauss_legendre01(nq, qx, qw);
    double *d_qx, *d_qw;
    F_TRY(falloc(c, &d_qx, nq));
    F_TRY(falloc(c, &d_qw, nq));
    F_TRY(cudaMemcpyAsync(d_qx, qx.data(), nq * sizeof(double), cudaMemcpyHostToDevice, c->s));
    F_TRY(cudaMemcpyAsync(d_qw, qw.data(), nq * sizeof(double), cudaMemcpyHostToDevice, c->s));
    k_element_weights<<<ns, 128, 0, c->s>>>(ns, ps, L, c->tree.box, F.lev[L].s, F.lev[L].hs, F.lev[L].ho, c->d_xyz, c->d_tri,
                                           c->d_xc, c->d_n, c->tree.key, nq, d_qx, d_qw, F.At, F.As, F.Dv, F.Dn, F.fft);
    F_TRY(cudaGetLastError());

    // time tables of a leaf interval: source position t (sigma = k Lt + t)
    // and observation position t (alpha = k Lt + 1 + t) share the local
    // coordinate (2t - (Lt - 1)) / Lt
    std::vector<double> tl((size_t)F.Lt * 8, 0.0), dtl((size_t)F.Lt * 8, 0.0);
    for (int t = 0; t < F.Lt; ++t) {
        double v[kMaxP], dv[kMaxP];
        h_lagrange(pt, (2.0 * t - (F.Lt - 1)) / F.Lt, v, dv, F.fft);
        for (int m = 0; m < pt; ++m) {
            tl[t * 8 + m] = v[m];
            dtl[t * 8 + m] = dv[m] / (F.Lt * c->P.dt / 2.0);
        }
    }
    F_TRY(falloc(c, &F.tl, tl.size()));
    F_TRY(falloc(c, &F.dtl, dtl.size()));
    F_TRY(cudaMemcpyAsync(F.tl, tl.data(), tl.size() * sizeof(double), cudaMemcpyHostToDevice, c->s));
    F_TRY(cudaMemcpyAsync(F.dtl, dtl.data(), dtl.size() * sizeof(double), cudaMemcpyHostToDevice, c->s));
    // B-spline fold weights w^{kappa,d} (Eq. w)
    double wk[kMaxD + 2];
    for (int kk = 0; kk <= d + 1; ++kk) {
        double pr = 1.0;
        for (int m = 0; m <= d + 1; ++m)
            if (m != kk) pr *= (double)(m - kk);
        wk[kk] = (d + 1) / pr;
    }
    F_TRY(falloc(c, &F.wk, d + 2));
    F_TRY(cudaMemcpyAsync(F.wk, wk, (d + 2) * sizeof(double), cudaMemcpyHostToDevice, c->s));
    // time transfer (level independent): T[half][n'][n] = ell_n'((w_n + 2 half - 1)/2)
    std::vector<double> tm(2 * pt * pt);
    for (int h = 0; h < 2; ++h)
        for (int n = 0; n < pt; ++n) {
            double v[kMaxP];
            h_lagrange(pt, (h_node(pt, n, F.fft) + 2.0 * h - 1.0) / 2.0, v, nullptr, F.fft);
            for (int np_ = 0; np_ < pt; ++np_) tm[h * pt * pt + np_ * pt + n] = v[np_];
        }
    F_TRY(falloc(c, &F.Tm, tm.size()));
    {
        std::vector<double> wt(pt);
        for (int n = 0; n < pt; ++n) wt[n] = h_node(pt, n, F.fft);
        F_TRY(falloc(c, &F.wt, wt.size()));
        F_TRY(cudaMemcpyAsync(F.wt, wt.data(), wt.size() * sizeof(double), cudaMemcpyHostToDevice, c->s));
    }
    F_TRY(cudaMemcpyAsync(F.Tm, tm.data(), tm.size() * sizeof(double), cudaMemcpyHostToDevice, c->s));
    F_TRY(falloc(c, &F.far, (size_t)F.Lt * ns));
    F_TRY(falloc(c, &F.Tq, (size_t)ns * pt));
    F_TRY(falloc(c, &F.Tu, (size_t)ns * pt));

    for (int l = 2; l <= L; ++l) {
        FmmLevel &V = F.lev[l];
        V.nc = c->tree.levels[l].nc;
        F_TRY(falloc(c, &V.M, (size_t)V.nc * P));
        F_TRY(falloc(c, &V.ring, (size_t)F.nslot * V.nc * P));
        F_TRY(falloc(c, &V.D, (size_t)std::max(d, 1) * V.nc * P));
        F_TRY(falloc(c, &V.A, (size_t)std::max(F.nd, 1) * V.nc * P));
        F_TRY(falloc(c, &V.G, (size_t)std::max(d, 1) * V.nc * P));
        // spatial transfers between this level (child) and level l-1
        // (parent): S[pos][b'][b] = ell_b'(((pos - 1/2) s_l + h_l w_b) / h_{l-1})
        // on the source boxes (M2M) and on the observation boxes (L2L)
        if (l > 2) {
            for (int kind = 0; kind < 2; ++kind) {
                const double hc = kind ? V.ho : V.hs, hp = kind ? F.lev[l - 1].ho : F.lev[l - 1].hs;
                std::vector<double> sm(2 * ps * ps);
                for (int pos = 0; pos < 2; ++pos)
                    for (int b = 0; b < ps; ++b) {
                        double v[kMaxP];
                        h_lagrange(ps, ((pos - 0.5) * V.s + hc * h_node(ps, b, F.fft)) / hp, v, nullptr, F.fft);
                        for (int bp = 0; bp < ps; ++bp) sm[pos * ps * ps + bp * ps + b] = v[bp];
                    }
                double **dst = kind ? &V.So : &V.Sm;
                F_TRY(falloc(c, dst, sm.size()));
                F_TRY(cudaMemcpyAsync(*dst, sm.data(), sm.size() * sizeof(double), cudaMemcpyHostToDevice, c->s));
            }
        }
        // interaction pairs as GEMM columns, grouped by the symmetry class of
        // their offset (classes by canonical offset code, pairs by observation
        // cell and list position), and per observation cell in list order
        std::vector<int32_t> codes;  // canonical offset of each class
        // FFT form: per pair in observation-cell order, source cell and the
        // index of its offset S - O among the level's distinct offsets
        std::vector<int32_t> fpS, fcodes;
        std::vector<int16_t> fpo;
        {
            const TreeLevel &T = c->tree.levels[l];
            std::vector<int32_t> cnt(V.nc), il((size_t)V.nc * 189);
            std::vector<uint64_t> keys(V.nc);
            F_TRY(cudaMemcpy(cnt.data(), T.ilcount, V.nc * sizeof(int32_t), cudaMemcpyDeviceToHost));
            F_TRY(cudaMemcpy(il.data(), T.il, il.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
            F_TRY(cudaMemcpy(keys.data(), T.ckey, V.nc * sizeof(uint64_t), cudaMemcpyDeviceToHost));
            auto coord = [&](uint64_t key, int a) {
                int v = 0;
                for (int b = 0; b < l; ++b) v |= (int)((key >> (3 * b + a)) & 1u) << b;
                return v;
            };
            std::vector<int> pcls, pgrp;  // per (O, t): class code and symmetry element
            std::vector<char> used(343, 0);
            for (int O = 0; O < V.nc; ++O)
                for (int t = 0; t < cnt[O]; ++t) {
                    const int S = il[(size_t)O * 189 + t];
                    int o[3], cc[3];
                    for (int a = 0; a < 3; ++a) o[a] = coord(keys[S], a) - coord(keys[O], a);
                    const int g = sym_decompose(o, cc);
                    const int code = (cc[0] + 3) + 7 * ((cc[1] + 3) + 7 * (cc[2] + 3));
                    pcls.push_back(code);
                    pgrp.push_back(g);
                    used[code] = 1;
                    if (F.fft) {
                        const int oc = (o[0] + 3) + 7 * ((o[1] + 3) + 7 * (o[2] + 3));
                        auto it = std::find(fcodes.begin(), fcodes.end(), oc);
                        if (it == fcodes.end()) {
                            fcodes.push_back(oc);
                            it = fcodes.end() - 1;
                        }
                        fpS.push_back(S);
                        fpo.push_back((int16_t)(it - fcodes.begin()));
                    }
                }
            std::vector<int> cls_of(343, -1);
            for (int code = 0; code < 343; ++code)
                if (used[code]) {
                    cls_of[code] = (int)codes.size();
                    codes.push_back(code);
                }
            V.ncls = (int)codes.size();
            V.np = (int64_t)pcls.size();
            V.cbase.assign(V.ncls + 1, 0);
            for (int code : pcls) V.cbase[cls_of[code] + 1]++;
            for (int ci = 0; ci < V.ncls; ++ci) V.cbase[ci + 1] += V.cbase[ci];
            std::vector<int64_t> fill(V.cbase.begin(), V.cbase.end() - 1), ooff(V.nc + 1, 0), oidx(V.np);
            std::vector<int32_t> hS(V.np);
            std::vector<uint8_t> hg(V.np), og(V.np), hc(V.np);
            int64_t q = 0;
            for (int O = 0; O < V.nc; ++O) {
                ooff[O + 1] = ooff[O] + cnt[O];
                for (int t = 0; t < cnt[O]; ++t, ++q) {
                    const int64_t col = fill[cls_of[pcls[q]]]++;
                    hS[col] = il[(size_t)O * 189 + t];
                    hg[col] = (uint8_t)pgrp[q];
                    hc[col] = (uint8_t)cls_of[pcls[q]];
                    oidx[q] = col;
                    og[q] = (uint8_t)pgrp[q];
                }
            }
            F_TRY(falloc(c, &V.pS, (size_t)V.np));
            F_TRY(falloc(c, &V.pg, (size_t)V.np));
            F_TRY(falloc(c, &V.ooff, (size_t)V.nc + 1));
            F_TRY(falloc(c, &V.oidx, (size_t)V.np));
            F_TRY(falloc(c, &V.og, (size_t)V.np));
            F_TRY(falloc(c, &V.pc, (size_t)V.np));
            F_TRY(cudaMemcpyAsync(V.pc, hc.data(), V.np, cudaMemcpyHostToDevice, c->s));
            F_TRY(cudaMemcpyAsync(V.pS, hS.data(), V.np * sizeof(int32_t), cudaMemcpyHostToDevice, c->s));
            F_TRY(cudaMemcpyAsync(V.pg, hg.data(), V.np, cudaMemcpyHostToDevice, c->s));
            F_TRY(cudaMemcpyAsync(V.ooff, ooff.data(), (V.nc + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, c->s));
            F_TRY(cudaMemcpyAsync(V.oidx, oidx.data(), V.np * sizeof(int64_t), cudaMemcpyHostToDevice, c->s));
            F_TRY(cudaMemcpyAsync(V.og, og.data(), V.np, cudaMemcpyHostToDevice, c->s));
            F_TRY(cudaStreamSynchronize(c->s));
        }
        const double Tdt = V.T * c->P.dt;
        V.Tlen = c->P.c * Tdt;
        if (V.np > 0) {
            // canonical operator stacks of the level's classes (FP64)
            // (not in the FFT form, whose blocks are applied as spectra)
            const size_t nop = (size_t)V.ncls * F.R * P;
            double *op = nullptr;
            int32_t *d_codes = nullptr;
            F_TRY(falloc(c, &d_codes, (size_t)V.ncls));
            F_TRY(cudaMemcpyAsync(d_codes, codes.data(), V.ncls * sizeof(int32_t), cudaMemcpyHostToDevice, c->s));
            if (!F.fft) {
                F_TRY(falloc(c, &op, nop));
                k_m2l_operators<<<152 * 32, 256, 0, c->s>>>(ps, pt, d, F.mu, F.ngb, V.s, V.hs, V.ho, Tdt, c->P.dt,
                                                            Tdt / 2.0, c->P.c, V.ncls, d_codes, op, F.fft);
                F_TRY(cudaGetLastError());
            }
            // distance powers of the derivative rows (Eq. U_expand)
            const size_t nkr = (size_t)V.ncls * (d + 1) * P3 * P3;
            if (c->split) {
                float2 *kr = nullptr;
                F_TRY(falloc(c, &kr, nkr));
                k_dist_powers<float2><<<152 * 8, 256, 0, c->s>>>(V.ncls, ps, d, V.s, V.hs, V.ho, d_codes, kr, F.fft);
                V.kr = kr;
            } else {
                double *kr = nullptr;
                F_TRY(falloc(c, &kr, nkr));
                k_dist_powers<double><<<152 * 8, 256, 0, c->s>>>(V.ncls, ps, d, V.s, V.hs, V.ho, d_codes, kr, F.fft);
                V.kr = kr;
            }
            F_TRY(cudaGetLastError());
            // spatial products per pair: (e, j) with e + j <= d, e != 1
            V.flops_deriv = 2.0 * P3 * P3 * (double)V.np * ((d + 1) + (d - 1) * d / 2);
            {
                // work of the derivative rows: buffers and (class, 8-column) jobs
                const size_t el = c->split ? sizeof(float2) : sizeof(double);
                F_TRY(falloc(c, (char **)&V.dmu, (size_t)V.np * (d + 1) * P3 * el));
                F_TRY(falloc(c, (char **)&V.dF, (size_t)V.np * (d + 1) * (d + 1) * P3 * el));
                F_TRY(falloc(c, &V.dss, (size_t)V.np * (d + 1)));
                std::vector<int4> jobs;
                for (int ci = 0; ci < V.ncls; ++ci)
                    for (int64_t c0 = V.cbase[ci]; c0 < V.cbase[ci + 1]; c0 += kDerivCols)
                        jobs.push_back(make_int4(ci, (int)c0, (int)std::min<int64_t>(kDerivCols, V.cbase[ci + 1] - c0), 0));
                V.njobs = (int)jobs.size();
                const double A = c->P.c * ((F.mu + 1) * Tdt + c->P.dt), cht = c->P.c * Tdt / 2.0;
                std::vector<double> tab = deriv_coef_table(d, pt, A, cht, F.fft);
                F_TRY(falloc(c, &V.dcoef, tab.size()));
                F_TRY(cudaMemcpyAsync(V.dcoef, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, c->s));
                F_TRY(falloc(c, &V.djobs, std::max<size_t>(jobs.size(), 1)));
                F_TRY(cudaMemcpyAsync(V.djobs, jobs.data(), jobs.size() * sizeof(int4), cudaMemcpyHostToDevice, c->s));
            }
            if (F.fft) {
                F_TRY(fft_m2l_level_setup(c, V, fpS, fpo, fcodes, Tdt, why));
                if (!why.empty()) return cudaSuccess;
            } else if (!c->split) {
                V.op = op;
                F_TRY(falloc(c, &V.Bbuf, (size_t)V.np * P));
                F_TRY(falloc(c, &V.Cbuf, (size_t)V.np * F.R));
                V.flops_app = 2.0 * F.R * P * (double)V.np;
            } else {
                // BF16 terms of the operators; zero blocks; the FP64 stacks go
                F_TRY(falloc(c, &V.opt, (size_t)F.nta * V.ncls * F.Rp * F.Kp));
                if (F.f16) {
                    F_TRY(falloc(c, &V.ascale, (size_t)V.ncls * F.Rp));
                    F_TRY(falloc(c, &V.bscale, (size_t)V.np));
                    F_TRY(falloc(c, &V.cexp, (size_t)V.nc));
                    k_split_operators_f16<<<152 * 32, 256, 0, c->s>>>(V.ncls, F.R, P, F.Rp, F.Kp, op, V.opt,
                                                                      V.ascale);
                } else {
                    k_split_operators<<<152 * 32, 256, 0, c->s>>>(V.ncls, F.R, P, F.Rp, F.Kp, F.nta, op, V.opt);
                }
                F_TRY(cudaGetLastError());
                double *d_bm = nullptr;
                F_TRY(falloc(c, &d_bm, (size_t)V.ncls * F.ngb));
                k_block_maxabs<<<V.ncls * F.ngb, 256, 0, c->s>>>(P, F.ngb, op, d_bm);
                F_TRY(cudaGetLastError());
                std::vector<double> bm((size_t)V.ncls * F.ngb);
                F_TRY(cudaMemcpyAsync(bm.data(), d_bm, bm.size() * sizeof(double), cudaMemcpyDeviceToHost, c->s));
                F_TRY(cudaStreamSynchronize(c->s));
                for (void *p : {(void *)op, (void *)d_bm}) {
                    auto it = std::find(c->allocs.begin(), c->allocs.end(), p);
                    if (it != c->allocs.end()) c->allocs.erase(it);
                    cudaFree(p);
                }
                F_TRY(falloc(c, &V.Bt, (size_t)F.ntb * V.np * F.Kp));
                F_TRY(falloc(c, &V.C32, (size_t)V.np * F.R));
                F_TRY(tc_make_map(&V.mapA, V.opt, (int64_t)F.nta * V.ncls * F.Rp, F.Kp, kTcBM));
                F_TRY(m2l_tune(c, V, bm));
            }
        }
    }
    return cudaStreamSynchronize(c->s);
}

// Parts of a boundary's far-field work (fmm_boundary_part).
enum { FB_URGENT = 1, FB_DEFERRED = 2, FB_ALL = 3 };

// The far-field work at the boundary after leaf interval k, or a part of it:
//   urgent (what the next L_t steps' far field needs): P2M, and per level
//     whose interval ended the gather, the GEMM tiles of the first
//     near-future block, its reduction into the local L_{k+1}, the time
//     moments of the exact rows, M2M into the parent and the clearing of
//     the level's moments; the L2L of the levels whose interval starts; L2P;
//   deferred (needed from the next boundary on): the GEMM tiles and the
//     reduction of the near-future blocks 2..mu, the exact rows (products,
//     assembly into L_{k+mu+1} and G) and the recurrence of Formula 1.
// graph = true: every pass of every level is launched, each kernel deciding
// on the device whether it runs (StepWhen); k is not used; part = FB_ALL.
static cudaError_t fmm_boundary_part(tdbem_ctx *c, int k, bool graph, int part)
{
    Fmm &F = c->fmm;
    const int L = F.L, d = c->P.d, P = F.P;
    cudaStream_t s = c->s;
    const bool urgent = part & FB_URGENT, deferred = part & FB_DEFERRED;
    const double pref = 1.0 / (4.0 * M_PI * pow(c->cdt, d));
    const TreeLevel &TL = c->tree.levels[L];
    auto when = [&](int span) {
        StepWhen w;
        if (graph) {
            w.alpha = c->d_alpha;
            w.alim = c->P.nt - 1;
            w.lt = F.Lt;
            w.span = span;
        }
        return w;
    };
    if (urgent) {
        if (!graph) c->far_kernels += 2;
        const int64_t nx = (int64_t)c->ns * F.pt;
        k_p2m_time<<<(int)((nx + 255) / 256), 256, 0, s>>>(c->ns, F.pt, F.Lt, k, d, c->P.nt - 2, c->tree.perm, c->d_q,
                                                           c->d_u, F.wk, F.tl, F.Tq, F.Tu, when(1));
        k_p2m_moments<<<dim3(TL.nc, (P + 255) / 256), 256, 0, s>>>(F.P3, P, TL.cstart, c->tree.perm, F.At, F.As, F.Tq,
                                                                   F.Tu, pref, F.lev[L].M, when(1));
        F_TRY(cudaGetLastError());
    }
    size_t shm = 2 * P * sizeof(double);
    for (int l = L; l >= 2; --l) {
        int span = 1 << (L - l);
        if (!graph && (k + 1) % span) break;
        int kl = graph ? 0 : (k + 1) / span - 1;
        const StepWhen w = when(span);
        FmmLevel &V = F.lev[l];
        const TreeLevel &T = c->tree.levels[l];
        // M2L for source interval kl of this level: gather (permuted by each
        // column's symmetry), one GEMM per symmetry class, per-cell
        // reduction into the locals (near future), exact rows
        if (V.np > 0) {
            cudaEvent_t ev = nullptr;
            if (!graph) phase_begin(c, &ev);
            if (F.fft) {
                // FFT form: spectra of the moments (urgent), then the products
                // and inverse transforms of the first block (urgent) or of
                // blocks 2..mu (deferred), added into the ring of locals
                cudaEvent_t eg = nullptr;
                if (!graph) phase_begin(c, &eg);
                if (urgent) F_TRY(fft_m2l_forward(c, V, s, w));
                F_TRY(fft_m2l_apply(c, V, kl, urgent ? 0 : 1, deferred ? F.ngb : 1, s, w));
                if (!graph) {
                    phase_end(c, PH_GEMM, eg);
                    c->launches[PH_GEMM] += 1;
                    c->far_kernels += (urgent ? 1 : 0) + 2;
                }
            } else {
                if (urgent) {
                    const int64_t n = V.np * P;
                    const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
                    if (!graph) c->far_kernels += 1;
                    if (F.f16) {
                        k_cell_scale<<<V.nc, 256, 0, s>>>(P, V.M, V.cexp, w);
                        k_m2l_gather_f16<<<grid, 256, 0, s>>>(V.np, F.P3, P, F.Kp, V.pS, V.pg, F.perm, V.M, V.cexp,
                                                             V.Bt, V.bscale, w);
                    } else if (c->split)
                        k_m2l_gather_split<<<grid, 256, 0, s>>>(V.np, F.P3, P, F.Kp, F.ntb, V.pS, V.pg, F.perm, V.M,
                                                                V.Bt, w);
                    else
                        k_m2l_gather<<<grid, 256, 0, s>>>(V.np, F.P3, P, V.pS, V.pg, F.perm, V.M, V.Bbuf, w);
                    F_TRY(cudaGetLastError());
                }
                // GEMM tiles: all (FB_ALL), or those of the first block / the rest
                const int gsel = (part == FB_ALL) ? 0 : (urgent ? 1 : 2);
                if (graph) {
                    F_TRY(m2l_products(c, V, w, gsel));
                } else {
                    cudaEvent_t eg;
                    phase_begin(c, &eg);
                    F_TRY(m2l_products(c, V, w, gsel));
                    phase_end(c, PH_GEMM, eg);
                    c->launches[PH_GEMM] += c->split ? 1 : (gsel == 2 ? 0 : V.ncls);
                    c->gemm_tc_flops += (gsel == 0 ? V.flops_app : gsel == 1 ? V.flops_u : V.flops_app - V.flops_u) *
                                        (c->split ? F.nprod : 1);
                }
                if (!graph) c->far_kernels += 1;
                if (c->split) {
                    // rows [0, P): the first block (urgent); [P, R): blocks 2..mu
                    const int rb = urgent ? 0 : P, re = deferred ? F.R : P;
                    if (re > rb) {
                        const int nrow = reduce_rows(F.P3, re - rb);
                        const size_t rshm = 2 * sizeof(float) * (size_t)nrow;
                        if (rshm > 48 * 1024)
                            F_TRY(cudaFuncSetAttribute(k_m2l_reduce_smem, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       (int)rshm));
                        k_m2l_reduce_smem<<<dim3(V.nc, (re - rb + nrow - 1) / nrow), 512, rshm, s>>>(
                            V.nc, F.P3, P, F.ngb, F.mu, F.nslot, kl, nrow, rb, re, V.ooff, V.oidx, V.og, F.perm, V.C32,
                            V.ring, w);
                    }
                } else {
                    k_m2l_reduce<double><<<V.nc, 256, 0, s>>>(V.nc, F.P3, P, F.ngb, F.mu, F.nslot, kl, V.ooff, V.oidx,
                                                              V.og, F.iperm, V.Cbuf, V.ring, V.G, w);
                }
                F_TRY(cudaGetLastError());
            }
            // the block L_{k+mu+1,k} and the derivative contributions G (exact
            // low-rank form of Eq. U_expand): moments now, the rest deferred
            const int dparts = (urgent ? 1 : 0) | (deferred ? 2 : 0);
            if (c->split)
                F_TRY(launch_deriv<float2>(d, V.nc, F.P3, F.pt, F.nslot, kl, F.mu, V, F.wt, F.perm, F.iperm, s, w,
                                           dparts));
            else
                F_TRY(launch_deriv<double>(d, V.nc, F.P3, F.pt, F.nslot, kl, F.mu, V, F.wt, F.perm, F.iperm, s, w,
                                           dparts));
            if (!graph) {
                c->far_kernels += (urgent ? 1 : 0) + (deferred ? 2 : 0);
                phase_end(c, PH_M2L, ev);
                if (urgent) {
                    c->launches[PH_M2L] += 1;
                    c->m2l_flops += V.flops_app + V.flops_deriv;
                }
            }
        } else if (!graph && deferred) {
            // (G of a level without pairs stays zero from its allocation on)
            F_TRY(cudaMemsetAsync(V.G, 0, (size_t)d * V.nc * P * sizeof(double), s));
        }
        int64_t n = (int64_t)V.nc * P;
        if (deferred) {
            if (!graph) ++c->far_kernels;
            k_m2l_recurrence<<<(int)std::min<int64_t>((n + 255) / 256, 152 * 16), 256, 0, s>>>(
                n, d, F.mu, F.nslot, kl, V.G, V.D, V.A, V.ring, V.Tlen, w);
            F_TRY(cudaGetLastError());
        }
        if (urgent) {
            // M2M into the parent, then clear this level's accumulator
            if (l > 2) {
                FmmLevel &Pv = F.lev[l - 1];
                const TreeLevel &PT = c->tree.levels[l - 1];
                if (!graph) ++c->far_kernels;
                k_m2m<<<Pv.nc, 128, shm, s>>>(F.ps, F.pt, Pv.nc, PT.ckey, V.nc, T.ckey, V.M, Pv.M, V.Sm, F.Tm, kl & 1,
                                              w);
                F_TRY(cudaGetLastError());
            }
            if (graph) {
                k_zero_when<<<(int)std::min<int64_t>((n + 255) / 256, 152 * 8), 256, 0, s>>>(n, V.M, w);
                F_TRY(cudaGetLastError());
            } else {
                F_TRY(cudaMemsetAsync(V.M, 0, (size_t)V.nc * P * sizeof(double), s));
            }
        }
    }
    if (!urgent) return cudaSuccess;
    // L2L into the levels whose interval starts at leaf interval k + 1
    for (int l = 2; l < L; ++l) {
        int span = 1 << (L - l - 1);  // leaf intervals per level-(l+1) interval
        if (!graph && (k + 1) % span) continue;
        int kc = graph ? 0 : (k + 1) / span;
        FmmLevel &Pv = F.lev[l], &Cv = F.lev[l + 1];
        if (!graph) ++c->far_kernels;
        k_l2l<<<Cv.nc, 128, shm, s>>>(F.ps, F.pt, Pv.nc, c->tree.levels[l].ckey, Cv.nc, c->tree.levels[l + 1].ckey,
                                      Pv.ring, Cv.ring, F.nslot, Cv.So, F.Tm, kc, when(span));
        F_TRY(cudaGetLastError());
    }
    // L2P for observation interval k + 1
    FmmLevel &V = F.lev[L];
    if (!graph) ++c->far_kernels;
    k_l2p<<<(int)(((int64_t)c->ns * 32 + 127) / 128), 128, 0, s>>>(c->ns, F.P3, F.pt, F.Lt, c->P.bie, c->P.c,
                                                                    c->tree.e2c, V.ring, F.nslot, V.nc, k + 1, F.Dv,
                                                                    F.Dn, F.tl, F.dtl, F.far, when(1));
    return cudaGetLastError();
}

// Far field at the boundary after leaf interval k (every source of J_k is
// known): P2M, M2M + M2L up the levels whose interval ended, L2L down the
// levels whose interval starts, and L2P of the leaf local of I_{k+1}.
//
// Plain stepping in a tensor-core form overlaps: the urgent part runs on
// the context's stream (after the previous boundary's deferred part), the
// deferred part on the second stream F.side, under the history sums of the
// following steps.  The two parts write disjoint rows of the locals (block
// 1 vs blocks 2..mu+1), and the next urgent part waits for the deferred one
// before it touches any state the deferred part uses, so the results equal
// the sequential order's bit for bit.
//
// graph = true (capture of a graph-replayed step): sequential, every pass of
// every level launched, each kernel reading the step from c->d_alpha and
// deciding on the device whether it runs (StepWhen); the phase timers and
// counters of plain stepping are left alone.
cudaError_t fmm_boundary(tdbem_ctx *c, int k, bool graph)
{
    Fmm &F = c->fmm;
    if (graph || !F.side || !F.overlap) return fmm_boundary_part(c, k, graph, FB_ALL);
    F_TRY(cudaStreamWaitEvent(c->s, F.ev_deferred, 0));
    F_TRY(fmm_boundary_part(c, k, false, FB_URGENT));
    F_TRY(cudaEventRecord(F.ev_urgent, c->s));
    F_TRY(cudaStreamWaitEvent(F.side, F.ev_urgent, 0));
    cudaStream_t keep = c->s;
    c->s = F.side;
    cudaError_t e = fmm_boundary_part(c, k, false, FB_DEFERRED);
    c->s = keep;
    F_TRY(e);
    F_TRY(cudaEventRecord(F.ev_deferred, F.side));
    return cudaSuccess;
}

// Orders the context's stream after the last deferred far-field work (before
// the FMM state is read, saved or the call returns).
cudaError_t fmm_join(tdbem_ctx *c)
{
    Fmm &F = c->fmm;
    if (!F.side) return cudaSuccess;
    return cudaStreamWaitEvent(c->s, F.ev_deferred, 0);
}

#undef F_TRY

void fmm_free(tdbem_ctx *c)
{
    if (c->fmm.blas) cublasDestroy(c->fmm.blas);
    c->fmm.blas = nullptr;
    if (c->fmm.side) {
        cudaStreamSynchronize(c->fmm.side);
        cudaStreamDestroy(c->fmm.side);
        cudaEventDestroy(c->fmm.ev_urgent);
        cudaEventDestroy(c->fmm.ev_deferred);
        c->fmm.side = nullptr;
    }
}

}  // namespace tdbem
