// Interpolation-based space-time FMM for the far part of the history sum
// (Section 3: P2M, M2M, M2L, L2L, L2P; Section 4: near- and distant-future
// M2L with the O(Nt) recurrence of Formula 1 / Algorithm 1).
//
// Readings (the paper defers the hierarchy to its earlier study):
//   - Lagrange interpolation on the p Chebyshev points of the first kind,
//     cos((2a+1) pi / (2p)), in each of x1..x3, y1..y3, t, s;
//   - the box of a level-l cell is its cube enlarged by rho, the largest
//     centroid-to-vertex distance of the mesh (half-width s_l/2 + rho);
//   - a leaf interval holds Lt = floor((s_L - rho)/(c dt)) steps (no source
//     of an interval reaches an interaction-list target in the same
//     interval); level l holds T_l = Lt 2^(L-l) steps; source interval J_k
//     covers sigma in [k T, (k+1) T), observation interval I_k covers steps
//     alpha in [k T + 1, (k+1) T + 1);
//   - mu: the smallest integer with c (mu T_l + 1) dt > sqrt(3)(3 s_l + 2 h_l)
//     on every level, so that the kernel is a polynomial of degree d over the
//     node domain of every distant-future interval (Section 4.2).
// Vector index of moments and locals: b1 + ps (b2 + ps (b3 + ps n)), as in
// the matrix form of Eq. m2l.
#include <math.h>

#include <algorithm>

#include <cublas_v2.h>

#include "tdbem_internal.cuh"

namespace tdbem {

constexpr int kMaxP = 8;

__device__ __forceinline__ double cheb_node(int p, int a) { return cos((2.0 * a + 1.0) * 3.14159265358979323846 / (2.0 * p)); }

// Lagrange basis of the p Chebyshev nodes at xi (values and derivatives).
__device__ void lag_basis(int p, double xi, double *val, double *der)
{
    double w[kMaxP];
    for (int a = 0; a < p; ++a) w[a] = cheb_node(p, a);
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
__global__ void k_element_weights(int ns, int ps, int L, const double *__restrict__ box, double s, double hs,
                                  const double *__restrict__ xyz, const int32_t *__restrict__ tri,
                                  const double *__restrict__ xc, const double *__restrict__ nrm,
                                  const uint64_t *__restrict__ key, int nq, const double *__restrict__ qx,
                                  const double *__restrict__ qw, double *At, double *As, double *Dv, double *Dn)
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
            for (int k = 0; k < 3; ++k) lag_basis(ps, (y[k] - cen[k]) / hs, l[k], dl[k]);
            double val = l[0][b1] * l[1][b2] * l[2][b3];
            double g0 = dl[0][b1] * l[1][b2] * l[2][b3] / hs, g1 = l[0][b1] * dl[1][b2] * l[2][b3] / hs,
                   g2 = l[0][b1] * l[1][b2] * dl[2][b3] / hs;
            at += w * val;
            as += w * (g0 * n[0] + g1 * n[1] + g2 * n[2]);
        }
        At[(int64_t)j * P3 + b] = at;
        As[(int64_t)j * P3 + b] = as;
        // L2P values at the collocation point of element j
        double l[3][kMaxP], dl[3][kMaxP];
        for (int k = 0; k < 3; ++k) lag_basis(ps, (xc[3 * j + k] - cen[k]) / hs, l[k], dl[k]);
        Dv[(int64_t)j * P3 + b] = l[0][b1] * l[1][b2] * l[2][b3];
        Dn[(int64_t)j * P3 + b] = (dl[0][b1] * l[1][b2] * l[2][b3] * n[0] + l[0][b1] * dl[1][b2] * l[2][b3] * n[1] +
                                  l[0][b1] * l[1][b2] * dl[2][b3] * n[2]) / hs;
    }
}

// M2L operator bank of one level: op[t][blk][row][col] for the offsets
// o = offs[t] = (dx+3) + 7((dy+3) + 7(dz+3)) (the cell offset S - O) in the
// order the batched GEMMs use, blk = l-1 (near future l =
// 1..mu+1) or mu+p (the p-th derivative U^(p) at I_{k+mu+1}, Eq. U_expand),
// row = a + P3 m, col = b + P3 n:
//   U(x_a, y_b, t_m, s_n) = (c (t_m - s_n) - r)_+^d / r,
//   U^(p) = C(d, p) (c (t_m - s_n) - r)_+^(d-p) / r,
// x_a - y_b = -offset s + h (w_a - w_b), t_m - s_n = l T dt + dt + ht (w_m - w_n).
__global__ void k_m2l_operators(int ps, int pt, int d, int mu, double s, double hs, double T_dt, double dt,
                                double ht, double c, int noff, const int32_t *__restrict__ offs, double *op)
{
    const int P3 = ps * ps * ps, P = P3 * pt, nblk = mu + 1 + d;
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
        double rx = -dx * s + hs * (cheb_node(ps, a1) - cheb_node(ps, b1));
        double ry = -dy * s + hs * (cheb_node(ps, a2) - cheb_node(ps, b2));
        double rz = -dz * s + hs * (cheb_node(ps, a3) - cheb_node(ps, b3));
        double r = sqrt(rx * rx + ry * ry + rz * rz);
        int l = (blk <= mu) ? blk + 1 : mu + 1;
        int pw = (blk <= mu) ? 0 : blk - mu;
        double tdiff = l * T_dt + dt + ht * (cheb_node(pt, m) - cheb_node(pt, n));
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
// (element, temporal node): Tq[j][n] = sum_sigma tau_j^sigma ell_n(t_sigma)
// (Tu likewise with sigma_j), staged in shared memory for kP2MChunk
// elements at a time; then M[b + P3 n] += pref sum_j (At Tq - As Tu).
constexpr int kP2MChunk = 32;

__global__ void k_p2m(int P3, int P, int Lt, int k, int d, int ns, int smax_hist, const int32_t *__restrict__ cstart,
                      const int32_t *__restrict__ perm, const double *__restrict__ At, const double *__restrict__ As,
                      const double *__restrict__ q, const double *__restrict__ u, const double *__restrict__ wk,
                      const double *__restrict__ tl, double pref, double *M)
{
    __shared__ double Tq[kP2MChunk][8], Tu[kP2MChunk][8];
    __shared__ int jj[kP2MChunk];
    const int c = blockIdx.x, pt = P / P3;
    const int e0 = cstart[c], e1 = cstart[c + 1];
    for (int base = e0; base < e1; base += kP2MChunk) {
        const int nj = min(kP2MChunk, e1 - base);
        for (int x = threadIdx.x; x < nj * pt; x += blockDim.x) {
            const int jl = x / pt, n = x % pt;
            const int j = perm[base + jl];
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
            Tq[jl][n] = tq;
            Tu[jl][n] = tu;
            if (n == 0) jj[jl] = j;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < P; e += blockDim.x) {
            const int b = e % P3, n = e / P3;
            double acc = 0.0;
            for (int jl = 0; jl < nj; ++jl) {
                const int64_t r = (int64_t)jj[jl] * P3 + b;
                acc += At[r] * Tq[jl][n] - As[r] * Tu[jl][n];
            }
            M[(int64_t)c * P + e] += pref * acc;
        }
        __syncthreads();
    }
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
                      const double *__restrict__ Sm, const double *__restrict__ Tm, int half)
{
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

// L2L (Section 3): child local += transposed transfer of the parent local.
__global__ void k_l2l(int ps, int pt, int ncp, const uint64_t *__restrict__ pkey, int ncc,
                      const uint64_t *__restrict__ ckey, const double *__restrict__ Lp, double *Lc,
                      const double *__restrict__ Sm, const double *__restrict__ Tm, int half)
{
    extern __shared__ double sh[];
    const int P = ps * ps * ps * pt;
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
                                 double *Aux, double *ring, const double *__restrict__ cmp, double Tlen)
{
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
                      const double *__restrict__ Lloc, const double *__restrict__ Dv, const double *__restrict__ Dn,
                      const double *__restrict__ tl, const double *__restrict__ dtl, double *far)
{
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

// M2L as dense GEMMs grouped by cell offset: the moments of the source
// cells of every interaction pair, ordered by (offset, observation cell),
// are gathered into the columns of B; for each offset one GEMM multiplies
// the offset's operator stack [(mu+1+d) P x P] with its slice of B; the
// per-cell sums over the cell's pairs (fixed order) feed the locals.
template <typename TB>
__global__ void k_m2l_gather(int64_t np, int P, const int32_t *__restrict__ pS, const int64_t *__restrict__ pcol,
                             const double *__restrict__ M, TB *B)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < np * P; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t pr = e / P;
        int r = (int)(e % P);
        B[pcol[pr] * P + r] = (TB)M[(int64_t)pS[pr] * P + r];
    }
}

__global__ void k_to_float(int64_t n, const double *__restrict__ a, float *b)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        b[e] = (float)a[e];
}

// Exact sum of two floats (two-sum of Knuth): a + b = s + e.
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float b)
{
    const float s = hi + b;
    const float bb = s - hi;
    lo += (hi - (s - bb)) + (b - bb);
    hi = s;
}

template <typename TC>
__global__ void k_m2l_reduce(int nc, int P, int nblk, int mu, int nslot, int k, const int64_t *__restrict__ ooff,
                             const int64_t *__restrict__ oidx, const TC *__restrict__ C, double *ring, double *G)
{
    // The cell's column indices are staged in shared memory (an interaction
    // list holds at most 189 cells), so the operand loads do not wait on
    // index loads.  Each thread sums 4 consecutive entries (one 16-byte load
    // per column when R = nblk P is a multiple of 4) over the cell's columns
    // in list order, 8 columns' loads at a time.  FP32 columns are summed in
    // double-float (a float pair with two-sum updates, about 48 bits): the
    // far field cancels terms 1e4-1e5 larger than itself, so a plain FP32
    // sum is not enough, and FP64 adds are 57 times slower on this GPU.
    __shared__ int64_t cols[kMaxIL];
    const int R = nblk * P;
    const int O = blockIdx.x;
    const int64_t t0 = ooff[O];
    const int nt = (int)(ooff[O + 1] - t0);
    for (int t = threadIdx.x; t < nt; t += blockDim.x) cols[t] = oidx[t0 + t] * R;
    __syncthreads();
    for (int e0 = 4 * threadIdx.x; e0 < R; e0 += 4 * blockDim.x) {
        double s[4] = {0.0, 0.0, 0.0, 0.0};
        if ((R & 3) == 0 && sizeof(TC) == 4) {
            float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
            int t = 0;
            for (; t + 8 <= nt; t += 8) {
                float4 f[8];
#pragma unroll
                for (int v = 0; v < 8; ++v) f[v] = *reinterpret_cast<const float4 *>(C + cols[t + v] + e0);
#pragma unroll
                for (int v = 0; v < 8; ++v) {
                    two_sum_acc(hi[0], lo[0], f[v].x);
                    two_sum_acc(hi[1], lo[1], f[v].y);
                    two_sum_acc(hi[2], lo[2], f[v].z);
                    two_sum_acc(hi[3], lo[3], f[v].w);
                }
            }
            for (; t < nt; ++t) {
                const float4 f = *reinterpret_cast<const float4 *>(C + cols[t] + e0);
                two_sum_acc(hi[0], lo[0], f.x);
                two_sum_acc(hi[1], lo[1], f.y);
                two_sum_acc(hi[2], lo[2], f.z);
                two_sum_acc(hi[3], lo[3], f.w);
            }
            for (int q = 0; q < 4; ++q) s[q] = (double)hi[q] + (double)lo[q];
        } else {
            for (int q = 0; q < 4 && e0 + q < R; ++q)
                for (int t = 0; t < nt; ++t) s[q] += (double)C[cols[t] + e0 + q];
        }
        for (int q = 0; q < 4 && e0 + q < R; ++q) {
            const int e = e0 + q, blk = e / P, r = e % P;
            if (blk <= mu)
                ring[((int64_t)((k + blk + 1) % nslot) * nc + O) * P + r] += s[q];
            else
                G[((int64_t)(blk - mu - 1) * nc + O) * P + r] = s[q];
        }
    }
}

namespace {

double h_cheb(int p, int a) { return cos((2.0 * a + 1.0) * M_PI / (2.0 * p)); }

void h_lagrange(int p, double xi, double *val, double *der)
{
    for (int a = 0; a < p; ++a) {
        double v = 1.0, dv = 0.0;
        for (int b = 0; b < p; ++b) {
            if (b == a) continue;
            double den = h_cheb(p, a) - h_cheb(p, b);
            double f = (xi - h_cheb(p, b)) / den;
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

// c_m^p(k) of Eq. cmp for p = 2..d, m = 0..p-2 (index (p-2)(p-1)/2 + m).
void cmp_table(int d, int k, double *out)
{
    for (int p = 2; p <= d; ++p)
        for (int m = 0; m <= p - 2; ++m) {
            double binom = 1.0;
            for (int i = 0; i < m; ++i) binom = binom * (p - i) / (i + 1);
            int e = p - m;
            double v = pow((double)k - 1.0, e) - 2.0 * pow((double)k, e) + pow((double)k + 1.0, e);
            out[(p - 2) * (p - 1) / 2 + m] = binom * v * ((m & 1) ? -1.0 : 1.0);
        }
}

}  // namespace

#define F_TRY(x)                        \
    do {                                \
        cudaError_t e_ = (x);           \
        if (e_ != cudaSuccess) return e_; \
    } while (0)

// Groups the level's offsets (in pair-count order) into nbk buckets of equal
// offset count; each offset owns a slab of its bucket's largest pair count.
static void m2l_layout(FmmLevel &V, int nbk)
{
    nbk = std::max(1, std::min<int>(nbk, (int)V.ord.size()));
    V.colbase.assign(343, 0);
    V.buckets.clear();
    int64_t col = 0;
    for (int bk = 0; bk < nbk; ++bk) {
        size_t lo = V.ord.size() * bk / nbk, hi = V.ord.size() * (bk + 1) / nbk;
        if (hi <= lo) continue;
        FmmBucket B;
        B.first = (int)lo;
        B.count = (int)(hi - lo);
        B.n = V.ostart[V.ord[lo] + 1] - V.ostart[V.ord[lo]];
        for (size_t t = lo; t < hi; ++t) {
            V.colbase[V.ord[t]] = col;
            col += B.n;
        }
        V.buckets.push_back(B);
    }
    V.ncol = std::max<int64_t>(col, 1);
    V.nbk = nbk;
}

// The batched GEMMs of one M2L application (operator stacks x gathered moments).
static cublasStatus_t m2l_gemms(tdbem_ctx *c, FmmLevel &V)
{
    Fmm &F = c->fmm;
    const int P = F.P, R = F.nblk * P;
    const long long sA = (long long)R * P;
    cublasStatus_t st = CUBLAS_STATUS_SUCCESS;
    for (const FmmBucket &B : V.buckets) {
        if (st != CUBLAS_STATUS_SUCCESS) break;
        int64_t cb = V.colbase[V.ord[B.first]];
        if (c->split) {
            const float one = 1.0f, zero = 0.0f;
            st = cublasGemmStridedBatchedEx(F.blas, CUBLAS_OP_T, CUBLAS_OP_N, R, (int)B.n, P, &one,
                                            V.op32 + (size_t)B.first * sA, CUDA_R_32F, P, sA,
                                            V.Bbuf32 + (size_t)cb * P, CUDA_R_32F, P, (long long)B.n * P, &zero,
                                            V.Cbuf32 + (size_t)cb * R, CUDA_R_32F, R, (long long)B.n * R, B.count,
                                            CUBLAS_COMPUTE_32F_EMULATED_16BFX9, CUBLAS_GEMM_DEFAULT);
        } else {
            const double one = 1.0, zero = 0.0;
            st = cublasDgemmStridedBatched(F.blas, CUBLAS_OP_T, CUBLAS_OP_N, R, (int)B.n, P, &one,
                                           V.op + (size_t)B.first * sA, P, sA, V.Bbuf + (size_t)cb * P, P,
                                           (long long)B.n * P, &zero, V.Cbuf + (size_t)cb * R, R, (long long)B.n * R,
                                           B.count);
        }
    }
    return st;
}

// Autotuner: times the level's M2L GEMMs for 1, 2, 4, .. 32 buckets on the
// real operators and shapes, keeps the fastest, and uploads the pair
// columns of that layout.
static cudaError_t m2l_tune_and_finalize(tdbem_ctx *c, FmmLevel &V)
{
    cudaStream_t s = c->s;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best = 1;
    float best_ms = 1e30f;
    V.tune.clear();
    for (int nbk = 1; nbk <= 32; nbk *= 2) {
        if (nbk > 1 && nbk > (int)V.ord.size()) break;
        m2l_layout(V, nbk);
        if (m2l_gemms(c, V) != CUBLAS_STATUS_SUCCESS) continue;  // warm-up; skip layouts the library rejects
        cudaEventRecord(e0, s);
        cublasStatus_t st = m2l_gemms(c, V);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (st != CUBLAS_STATUS_SUCCESS) continue;
        V.tune.push_back({nbk, ms});
        if (ms < best_ms) {
            best_ms = ms;
            best = nbk;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_ms >= 1e30f) return cudaErrorUnknown;
    m2l_layout(V, best);
    std::vector<int64_t> pcol(V.np);
    for (int o = 0; o < 343; ++o)
        for (int64_t t = V.ostart[o]; t < V.ostart[o + 1]; ++t) pcol[t] = V.colbase[o] + (t - V.ostart[o]);
    std::vector<int64_t> ooff(V.nc + 1, 0);
    for (int32_t O : V.hpO) ooff[O + 1]++;
    for (int O = 0; O < V.nc; ++O) {
        if (ooff[O + 1] > kMaxIL) return cudaErrorInvalidValue;  // the reduction stages one list in shared memory
        ooff[O + 1] += ooff[O];
    }
    std::vector<int64_t> oidx(V.np), fill(ooff.begin(), ooff.end() - 1);
    for (int64_t t = 0; t < V.np; ++t) oidx[fill[V.hpO[t]]++] = pcol[t];
    cudaError_t e;
    if ((e = cudaMemcpyAsync(V.pS, V.hpS.data(), V.np * sizeof(int32_t), cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return e;
    if ((e = cudaMemcpyAsync(V.pcol, pcol.data(), V.np * sizeof(int64_t), cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return e;
    if ((e = cudaMemcpyAsync(V.ooff, ooff.data(), (V.nc + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
        return e;
    if ((e = cudaMemcpyAsync(V.oidx, oidx.data(), V.np * sizeof(int64_t), cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return e;
    V.hpO.clear();
    V.hpS.clear();
    return cudaStreamSynchronize(s);
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
    if (F.P > 4096) {
        why = "FMM needs ps^3 pt <= 4096";
        return cudaSuccess;
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
    }
    F.Lt = (int)floor((F.lev[L].s - F.rho) / cdt);
    if (F.Lt < 1 || !(2.0 * F.rho < F.lev[L].s)) {
        why = "infeasible hierarchy: leaf cells too small for c dt and the element size";
        return cudaSuccess;
    }
    int mu = 0;
    for (int l = 2; l <= L; ++l) {
        F.lev[l].T = F.Lt << (L - l);
        double rmax = sqrt(3.0) * (3.0 * F.lev[l].s + 2.0 * F.lev[l].hs);
        mu = std::max(mu, (int)floor((rmax / cdt - 1.0) / F.lev[l].T) + 1);
    }
    F.lev[L].T = F.Lt;
    F.mu = std::max(mu, c->P.mu);
    F.nblk = F.mu + 1 + d;
    F.nd = d * (d - 1) / 2;
    F.nslot = F.mu + 2;
    const int P = F.P, P3 = F.P3, ps = F.ps, pt = F.pt;
    if (cublasCreate(&F.blas) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
    cublasSetStream(F.blas, c->s);
    cublasSetMathMode(F.blas, CUBLAS_DEFAULT_MATH);
    if (c->split) {
        cublasSetEmulationStrategy(F.blas, CUBLAS_EMULATION_STRATEGY_EAGER);
        // moments and operators are finite: the unknowns are checked every
        // step (a non-finite value stops the march), so the emulation need
        // not scan its operands for infinities and NaNs
        cublasSetEmulationSpecialValuesSupport(F.blas, CUDA_EMULATION_SPECIAL_VALUES_SUPPORT_NONE);
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
    k_element_weights<<<ns, 128, 0, c->s>>>(ns, ps, L, c->tree.box, F.lev[L].s, F.lev[L].hs, c->d_xyz, c->d_tri,
                                           c->d_xc, c->d_n, c->tree.key, nq, d_qx, d_qw, F.At, F.As, F.Dv, F.Dn);
    F_TRY(cudaGetLastError());

    // time tables of a leaf interval: source position t (sigma = k Lt + t)
    // and observation position t (alpha = k Lt + 1 + t) share the local
    // coordinate (2t - (Lt - 1)) / Lt
    std::vector<double> tl((size_t)F.Lt * 8, 0.0), dtl((size_t)F.Lt * 8, 0.0);
    for (int t = 0; t < F.Lt; ++t) {
        double v[kMaxP], dv[kMaxP];
        h_lagrange(pt, (2.0 * t - (F.Lt - 1)) / F.Lt, v, dv);
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
            h_lagrange(pt, (h_cheb(pt, n) + 2.0 * h - 1.0) / 2.0, v, nullptr);
            for (int np_ = 0; np_ < pt; ++np_) tm[h * pt * pt + np_ * pt + n] = v[np_];
        }
    F_TRY(falloc(c, &F.Tm, tm.size()));
    F_TRY(cudaMemcpyAsync(F.Tm, tm.data(), tm.size() * sizeof(double), cudaMemcpyHostToDevice, c->s));
    F_TRY(falloc(c, &F.cmp, 16));
    F_TRY(falloc(c, &F.far, (size_t)F.Lt * ns));

    for (int l = 2; l <= L; ++l) {
        FmmLevel &V = F.lev[l];
        V.nc = c->tree.levels[l].nc;
        F_TRY(falloc(c, &V.M, (size_t)V.nc * P));
        F_TRY(falloc(c, &V.ring, (size_t)F.nslot * V.nc * P));
        F_TRY(falloc(c, &V.D, (size_t)std::max(d, 1) * V.nc * P));
        F_TRY(falloc(c, &V.A, (size_t)std::max(F.nd, 1) * V.nc * P));
        F_TRY(falloc(c, &V.G, (size_t)std::max(d, 1) * V.nc * P));
        // spatial transfer from this level (child) to level l-1 (parent):
        // S[pos][b'][b] = ell_b'(((pos - 1/2) s_l + h_l w_b) / h_{l-1})
        if (l > 2) {
            std::vector<double> sm(2 * ps * ps);
            for (int pos = 0; pos < 2; ++pos)
                for (int b = 0; b < ps; ++b) {
                    double v[kMaxP];
                    h_lagrange(ps, ((pos - 0.5) * V.s + V.hs * h_cheb(ps, b)) / F.lev[l - 1].hs, v, nullptr);
                    for (int bp = 0; bp < ps; ++bp) sm[pos * ps * ps + bp * ps + b] = v[bp];
                }
            F_TRY(falloc(c, &V.Sm, sm.size()));
            F_TRY(cudaMemcpyAsync(V.Sm, sm.data(), sm.size() * sizeof(double), cudaMemcpyHostToDevice, c->s));
        }
        // interaction pairs grouped by offset, and per observation cell
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
            std::vector<std::vector<std::pair<int, int>>> byoff(343);
            for (int O = 0; O < V.nc; ++O)
                for (int t = 0; t < cnt[O]; ++t) {
                    int S = il[(size_t)O * 189 + t];
                    int o = (coord(keys[S], 0) - coord(keys[O], 0) + 3) +
                            7 * ((coord(keys[S], 1) - coord(keys[O], 1) + 3) + 7 * (coord(keys[S], 2) - coord(keys[O], 2) + 3));
                    byoff[o].push_back({O, S});
                }
            std::vector<int32_t> pS, pO;
            V.ostart.assign(344, 0);
            for (int o = 0; o < 343; ++o) {
                V.ostart[o] = (int64_t)pS.size();
                for (auto &pr : byoff[o]) {
                    pO.push_back(pr.first);
                    pS.push_back(pr.second);
                }
            }
            V.ostart[343] = (int64_t)pS.size();
            V.np = (int64_t)pS.size();
            // offsets that occur, by decreasing pair count; the grouping into
            // batched GEMMs (buckets) is chosen after the operators exist
            std::vector<int> ord;
            for (int o = 0; o < 343; ++o)
                if (V.ostart[o + 1] > V.ostart[o]) ord.push_back(o);
            std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
                return V.ostart[a + 1] - V.ostart[a] > V.ostart[b + 1] - V.ostart[b];
            });
            V.ord = ord;
            V.hpO = pO;
            V.hpS = pS;
            m2l_layout(V, 1);  // the widest layout sizes the buffers
            size_t ncol = (size_t)V.ncol;
            F_TRY(falloc(c, &V.pS, (size_t)V.np));
            F_TRY(falloc(c, &V.pcol, (size_t)V.np));
            F_TRY(falloc(c, &V.ooff, (size_t)V.nc + 1));
            F_TRY(falloc(c, &V.oidx, (size_t)V.np));
            if (c->split) {
                F_TRY(falloc(c, &V.Bbuf32, ncol * P));
                F_TRY(falloc(c, &V.Cbuf32, ncol * F.nblk * P));
            } else {
                F_TRY(falloc(c, &V.Bbuf, ncol * P));
                F_TRY(falloc(c, &V.Cbuf, ncol * F.nblk * P));
            }
            F_TRY(cudaStreamSynchronize(c->s));
        }
        double Tdt = V.T * c->P.dt;
        {
            // operators of the offsets that occur, in bucket order
            size_t noff = std::max<size_t>(V.ord.size(), 1);
            size_t nop = noff * F.nblk * P * P;
            F_TRY(falloc(c, &V.op, nop));
            int32_t *d_offs = nullptr;
            F_TRY(falloc(c, &d_offs, noff));
            if (!V.ord.empty())
                F_TRY(cudaMemcpyAsync(d_offs, V.ord.data(), V.ord.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                                      c->s));
            k_m2l_operators<<<152 * 32, 256, 0, c->s>>>(ps, pt, d, F.mu, V.s, V.hs, Tdt, c->P.dt, Tdt / 2.0, c->P.c,
                                                        (int)V.ord.size(), d_offs, V.op);
            F_TRY(cudaGetLastError());
            if (c->split) {
                // mixed form: FP32 operators for the emulated-FP32 tensor-core GEMM
                F_TRY(falloc(c, &V.op32, nop));
                k_to_float<<<152 * 32, 256, 0, c->s>>>((int64_t)nop, V.op, V.op32);
                F_TRY(cudaGetLastError());
                F_TRY(cudaStreamSynchronize(c->s));
                auto it = std::find(c->allocs.begin(), c->allocs.end(), (void *)V.op);
                if (it != c->allocs.end()) c->allocs.erase(it);
                cudaFree(V.op);
                V.op = nullptr;
            }
        }
        V.Tlen = c->P.c * Tdt;
        if (V.np > 0) F_TRY(m2l_tune_and_finalize(c, V));
    }
    return cudaStreamSynchronize(c->s);
}

// Far field at the boundary after leaf interval k (every source of J_k is
// known): P2M, M2M + M2L up the levels whose interval ended, L2L down the
// levels whose interval starts, and L2P of the leaf local of I_{k+1}.
cudaError_t fmm_boundary(tdbem_ctx *c, int k)
{
    Fmm &F = c->fmm;
    const int L = F.L, d = c->P.d, P = F.P;
    cudaStream_t s = c->s;
    const double pref = 1.0 / (4.0 * M_PI * pow(c->cdt, d));
    const TreeLevel &TL = c->tree.levels[L];
    k_p2m<<<TL.nc, 128, 0, s>>>(F.P3, P, F.Lt, k, d, c->ns, c->P.nt - 2, TL.cstart, c->tree.perm, F.At, F.As, c->d_q,
                                c->d_u, F.wk, F.tl, pref, F.lev[L].M);
    F_TRY(cudaGetLastError());
    size_t shm = 2 * P * sizeof(double);
    for (int l = L; l >= 2; --l) {
        int span = 1 << (L - l);
        if ((k + 1) % span) break;
        int kl = (k + 1) / span - 1;
        FmmLevel &V = F.lev[l];
        const TreeLevel &T = c->tree.levels[l];
        // M2L for source interval kl of this level: gather, one GEMM per
        // offset, per-cell reduction into the locals (near future) and G
        if (V.np > 0) {
            const int R = F.nblk * P;
            cudaEvent_t ev;
            phase_begin(c, &ev);
            cublasStatus_t st;
            if (c->split) {
                // FP32 operands, FP32-accurate products on the BF16 tensor
                // cores (three BF16 terms per operand), FP64 locals
                k_m2l_gather<float><<<152 * 8, 256, 0, s>>>(V.np, P, V.pS, V.pcol, V.M, V.Bbuf32);
                st = m2l_gemms(c, V);
                k_m2l_reduce<float><<<V.nc, 256, 0, s>>>(V.nc, P, F.nblk, F.mu, F.nslot, kl, V.ooff, V.oidx, V.Cbuf32,
                                                         V.ring, V.G);
            } else {
                k_m2l_gather<double><<<152 * 8, 256, 0, s>>>(V.np, P, V.pS, V.pcol, V.M, V.Bbuf);
                st = m2l_gemms(c, V);
                k_m2l_reduce<double><<<V.nc, 256, 0, s>>>(V.nc, P, F.nblk, F.mu, F.nslot, kl, V.ooff, V.oidx, V.Cbuf,
                                                          V.ring, V.G);
            }
            if (st != CUBLAS_STATUS_SUCCESS) {
                c->err = "cuBLAS status " + std::to_string((int)st) + " in the M2L GEMM";
                return cudaErrorUnknown;
            }
            phase_end(c, PH_M2L, ev);
            c->launches[PH_M2L] += 1;
            c->m2l_flops += 2.0 * (double)R * P * (double)V.np;  // algorithmic (unpadded) flops
            F_TRY(cudaGetLastError());
        } else {
            F_TRY(cudaMemsetAsync(V.G, 0, (size_t)d * V.nc * P * sizeof(double), s));
        }
        double cm[16] = {0};
        cmp_table(d, kl, cm);
        F_TRY(cudaMemcpyAsync(F.cmp, cm, sizeof(cm), cudaMemcpyHostToDevice, s));
        int64_t n = (int64_t)V.nc * P;
        k_m2l_recurrence<<<(int)std::min<int64_t>((n + 255) / 256, 152 * 16), 256, 0, s>>>(
            n, d, F.mu, F.nslot, kl, V.G, V.D, V.A, V.ring, F.cmp, V.Tlen);
        F_TRY(cudaGetLastError());
        // M2M into the parent, then clear this level's accumulator
        if (l > 2) {
            FmmLevel &Pv = F.lev[l - 1];
            const TreeLevel &PT = c->tree.levels[l - 1];
            k_m2m<<<Pv.nc, 128, shm, s>>>(F.ps, F.pt, Pv.nc, PT.ckey, V.nc, T.ckey, V.M, Pv.M, V.Sm, F.Tm, kl & 1);
            F_TRY(cudaGetLastError());
        }
        F_TRY(cudaMemsetAsync(V.M, 0, (size_t)V.nc * P * sizeof(double), s));
    }
    // L2L into the levels whose interval starts at leaf interval k + 1
    for (int l = 2; l < L; ++l) {
        int span = 1 << (L - l - 1);  // leaf intervals per level-(l+1) interval
        if ((k + 1) % span) continue;
        int kc = (k + 1) / span, kp = kc / 2;
        FmmLevel &Pv = F.lev[l], &Cv = F.lev[l + 1];
        k_l2l<<<Cv.nc, 128, shm, s>>>(F.ps, F.pt, Pv.nc, c->tree.levels[l].ckey, Cv.nc, c->tree.levels[l + 1].ckey,
                                      Pv.ring + (size_t)(kp % F.nslot) * Pv.nc * P,
                                      Cv.ring + (size_t)(kc % F.nslot) * Cv.nc * P, Cv.Sm, F.Tm, kc & 1);
        F_TRY(cudaGetLastError());
    }
    // L2P for observation interval k + 1
    FmmLevel &V = F.lev[L];
    k_l2p<<<(int)(((int64_t)c->ns * 32 + 127) / 128), 128, 0, s>>>(c->ns, F.P3, F.pt, F.Lt, c->P.bie, c->P.c, c->tree.e2c,
                                              V.ring + (size_t)((k + 1) % F.nslot) * V.nc * P, F.Dv, F.Dn, F.tl,
                                              F.dtl, F.far);
    return cudaGetLastError();
}

#undef F_TRY

void fmm_free(tdbem_ctx *c)
{
    if (c->fmm.blas) cublasDestroy(c->fmm.blas);
    c->fmm.blas = nullptr;
}

}  // namespace tdbem
