// Influence-coefficient arithmetic of the time-domain BEM (device side).
//
// For a collocation point x and a flat triangle E at lag g (lengths in units
// of c*dt, time in units of dt) the compact coefficients fold the kappa-sum
// of Eq. discretised_single_layer_potential into the B-spline of the retarded
// time (Section 2.4, the identity that precedes Remark gamma_bound):
//
//   Chat_U = 1/(4 pi) int_E N(g - r)/r dS
//   Chat_W = 1/(4 pi) int_E n_y.(x - y) [N(g - r)/r^3 + N'(g - r)/r^2] dS
//
// with N = N^{0,d} (Eq. decompose) and n_y the paper's normal (into V).  The
// Burton-Miller coefficients (Eq. U_W_BM) add the normal derivative at x and
// -c^-1 d/dt = -d/dg.  The spatial integrals follow Appendix B: the foot O of
// x on the plane of E splits E into three signed sub-triangles O-a-b; in
// polar coordinates about O the radial integral is exact through
// rho drho = r dr, which leaves one-dimensional angular integrals of
// functions of r_e(theta), the distance from x to the edge point.
//
// How the angular integrals are done here (not the paper's closed forms,
// which lose digits for d >= 2 as its Section 5.1.3 observes):
//   - only the wavefront shell g-d-1 < r < g needs quadrature: inside it
//     every integrand vanishes, outside it is a constant whose angular
//     integral is an exact angle;
//   - the shell is split at the integer radii (the B-spline knots) and at
//     the foot of O on the edge line, so each piece is analytic;
//   - on each piece the edge parameter s (distance from that foot) is
//     replaced by s = h sinh(u) (h = in-plane distance of O to the edge
//     line), which turns dtheta = h ds/(h^2+s^2) into du/cosh(u) and keeps
//     every singularity of the integrand at distance pi/2 from the real u
//     axis, so fixed panels of Gauss-Legendre converge geometrically;
//   - differences such as N(g - |z|) - N(g - r) are formed from the factor
//     r - |z| = rho^2/(r + |z|) when both arguments lie on one polynomial
//     piece, so no digits cancel when the element is far and seen face-on.
// The in-plane gradient needed by the Burton-Miller operator uses the
// divergence theorem (edge integrals), with the substitution s = R sinh(v).
//
// Everything is __host__ __device__ plain C++ arithmetic so that the same
// code runs in the kernels; the B-spline pieces come from a table built by
// the de Boor-Cox recursion (bspline_table()).
#pragma once

#include <math.h>

#ifdef __CUDACC__
#define TD_HD __host__ __device__ __forceinline__
#else
#define TD_HD inline
#endif

namespace tdbem {

constexpr int kMaxD = 4;

// Piecewise-polynomial form of N^{0,d}: on [k, k+1] (k = 0..d)
// N(k + t) = sum_m c[k][m] t^m, t in [0, 1]; gcum[k] = int_0^k N.
struct BsTable {
    int d;
    double c[kMaxD + 1][kMaxD + 1];
    double gcum[kMaxD + 2];
};

// de Boor-Cox recursion N^e(tau) = tau/e N^{e-1}(tau) + (e+1-tau)/e N^{e-1}(tau-1)
// applied to the local polynomials (host side, at context creation).
inline void bspline_table(int d, BsTable *T)
{
    double P[kMaxD + 1][kMaxD + 2][kMaxD + 2] = {};
    P[0][0][0] = 1.0;
    for (int e = 1; e <= d; ++e)
        for (int k = 0; k <= e; ++k)
            for (int m = 0; m < e; ++m) {
                if (k <= e - 1) {
                    double a = P[e - 1][k][m];
                    P[e][k][m] += (double)k / e * a;
                    P[e][k][m + 1] += a / e;
                }
                if (k >= 1) {
                    double a = P[e - 1][k - 1][m];
                    P[e][k][m] += (double)(e + 1 - k) / e * a;
                    P[e][k][m + 1] -= a / e;
                }
            }
    T->d = d;
    for (int k = 0; k <= kMaxD; ++k)
        for (int m = 0; m <= kMaxD; ++m) T->c[k][m] = (k <= d && m <= d) ? P[d][k][m] : 0.0;
    T->gcum[0] = 0.0;
    for (int k = 0; k <= d; ++k) {
        double s = 0.0;
        for (int m = 0; m <= d; ++m) s += T->c[k][m] / (m + 1);
        T->gcum[k + 1] = T->gcum[k] + s;
    }
}

// Piece index and local coordinate of tau; `left` selects the left limit
// at a knot (tau exactly integer -> piece tau-1 at t = 1).
TD_HD void bs_locate(double tau, bool left, int &k, double &t)
{
    double f = floor(tau);
    k = (int)f;
    t = tau - f;
    if (left && t == 0.0) {
        k -= 1;
        t = 1.0;
    }
}

TD_HD double bs_N(const BsTable &T, int k, double t)
{
    if (k < 0 || k > T.d) return 0.0;
    double s = 0.0;
    for (int m = T.d; m >= 0; --m) s = s * t + T.c[k][m];
    return s;
}

TD_HD double bs_dN(const BsTable &T, int k, double t)
{
    if (k < 0 || k > T.d) return 0.0;
    double s = 0.0;
    for (int m = T.d; m >= 1; --m) s = s * t + m * T.c[k][m];
    return s;
}

TD_HD double bs_G(const BsTable &T, int k, double t)
{
    if (k < 0) return 0.0;
    if (k > T.d) return 1.0;
    double s = 0.0;
    for (int m = T.d; m >= 0; --m) s = s * t + T.c[k][m] / (m + 1);
    return T.gcum[k] + s * t;
}

// Differences P(tb) - P(ta) on one piece k, from dl = tb - ta given to full
// relative accuracy: P(tb) - P(ta) = dl * sum_m c_m S_m with
// S_m = sum_{l<m} tb^l ta^{m-1-l}.  Out: dG, dN, ddN.
TD_HD void bs_piece_diff(const BsTable &T, int k, double tb, double ta, double dl,
                         double &dG, double &dN, double &ddN)
{
    double S[kMaxD + 3];
    S[1] = 1.0;
    double tap = 1.0;
    for (int m = 1; m <= T.d + 1; ++m) {
        tap *= ta;
        S[m + 1] = tb * S[m] + tap;
    }
    double sG = 0.0, sN = 0.0, sdN = 0.0;
    for (int m = 0; m <= T.d; ++m) {
        double c = T.c[k][m];
        sG += c / (m + 1) * S[m + 1];
        if (m >= 1) sN += c * S[m];
        if (m >= 2) sdN += m * c * S[m - 1];
    }
    dG = dl * sG;
    dN = dl * sN;
    ddN = dl * sdN;
}

// 10-point Gauss-Legendre on [-1, 1] (nodes x_k > 0 and their weights; the
// rule is symmetric).
TD_HD double gl10_x(int k)
{
    const double x[5] = {0.1488743389816312108848260, 0.4333953941292471907992659,
                         0.6794095682990244062343274, 0.8650633666889845107320967,
                         0.9739065285171717200779640};
    return x[k];
}
TD_HD double gl10_w(int k)
{
    const double w[5] = {0.2955242247147528701738930, 0.2692667193099963550912269,
                         0.2190863625159820439955349, 0.1494513491505805931457763,
                         0.0666713443086881375935688};
    return w[k];
}

// Values of the integrands at the foot's retarded time tau0 = g - |z|.
struct Foot {
    double g, z, az, sz;
    int k0;
    double t0, N0, dN0, G0;
};

TD_HD void foot_init(const BsTable &T, double g, double z, Foot &F)
{
    F.g = g;
    F.z = z;
    F.az = fabs(z);
    F.sz = (z < 0.0) ? -1.0 : 1.0;  // z == 0: the limit from the side n points to
    bs_locate(g - F.az, true, F.k0, F.t0);
    F.N0 = bs_N(T, F.k0, F.t0);
    F.dN0 = bs_dN(T, F.k0, F.t0);
    F.G0 = bs_G(T, F.k0, F.t0);
}

// Angular integrands at an edge point at distance r from x and rho^2 = r^2 - z^2
// from O (5 components):
//   0: G(tau0) - G(g - r)                              (4 pi Chat_U)
//   1: sz N(tau0) - z N(g - r)/r                       (4 pi Chat_W)
//   2: N(tau0) - N(g - r)                              (4 pi d/dg Chat_U)
//   3: sz N'(tau0) - z N'(g - r)/r                     (4 pi d/dg Chat_W)
//   4: N(g-r)/r - z^2 N'(g-r)/r^2 - z^2 N(g-r)/r^3 + N'(tau0)   (-4 pi d/dz Chat_W)
TD_HD void shell_integrands(const BsTable &T, const Foot &F, double r, double rho2, double f[5])
{
    int k;
    double t;
    bs_locate(F.g - r, false, k, t);
    double Nt = bs_N(T, k, t), dNt = bs_dN(T, k, t);
    double del = rho2 / (r + F.az);  // r - |z| without cancellation
    double DG, DN, DdN;
    if (k == F.k0) {
        bs_piece_diff(T, k, F.t0, t, del, DG, DN, DdN);
    } else {
        DG = F.G0 - bs_G(T, k, t);
        DN = F.N0 - Nt;
        DdN = F.dN0 - dNt;
    }
    double ir = 1.0 / r;
    f[0] = DG;
    f[1] = F.sz * (DN + Nt * del * ir);
    f[2] = DN;
    f[3] = F.sz * (DdN + dNt * del * ir);
    f[4] = DdN + dNt * rho2 * ir * ir + Nt * rho2 * ir * ir * ir;
}

// Sub-triangle O-a-b (pa = a - O, pb = b - O, in the plane; ng the unit
// geometric normal of E).  Adds the signed angular integrals to acc[0..4]
// (ncomp = 2: only components 0, 1) and, if `edge`, the edge integrals
// int_a^b N/r ds and int_a^b (N'/r^2 + N/r^3) ds to eint[0..1].
TD_HD void subtriangle(const BsTable &T, const Foot &F, const double pa[3], const double pb[3],
                       const double ng[3], int ncomp, bool edge, double acc[5], double eint[2])
{
    const int d = T.d;
    double e[3] = {pb[0] - pa[0], pb[1] - pa[1], pb[2] - pa[2]};
    double L = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
    double th[3] = {e[0] / L, e[1] / L, e[2] / L};
    double sa = pa[0] * th[0] + pa[1] * th[1] + pa[2] * th[2];
    double sb = sa + L;
    double cr[3] = {pa[1] * pb[2] - pa[2] * pb[1], pa[2] * pb[0] - pa[0] * pb[2],
                    pa[0] * pb[1] - pa[1] * pb[0]};
    double A2 = cr[0] * ng[0] + cr[1] * ng[1] + cr[2] * ng[2];
    double la = sqrt(pa[0] * pa[0] + pa[1] * pa[1] + pa[2] * pa[2]);
    double lb = sqrt(pb[0] * pb[0] + pb[1] * pb[1] + pb[2] * pb[2]);
    bool ang = fabs(A2) > 1e-14 * la * lb;
    double h = fabs(A2) / L;
    double sgn = (A2 > 0.0) ? 1.0 : -1.0;
    double R2 = h * h + F.z * F.z;
    double R = sqrt(R2);
    if (!ang && !(edge && R > 1e-12)) return;

    // breakpoints: ends, the foot s = 0, the knot radii g-d-1 .. g
    double bp[2 * (kMaxD + 2) + 3];
    int nb = 0;
    bp[nb++] = sa;
    bp[nb++] = sb;
    if (sa < 0.0 && sb > 0.0) bp[nb++] = 0.0;
    int gi = (int)F.g;
    for (int kk = gi - d - 1; kk <= gi; ++kk) {
        if (kk <= 0) continue;
        double q = ((double)kk - R) * ((double)kk + R);
        if (q <= 0.0) continue;
        double s = sqrt(q);
        if (s > sa && s < sb) bp[nb++] = s;
        if (-s > sa && -s < sb) bp[nb++] = -s;
    }
    for (int i = 1; i < nb; ++i)
        for (int j = i; j > 0 && bp[j] < bp[j - 1]; --j) {
            double tmp = bp[j];
            bp[j] = bp[j - 1];
            bp[j - 1] = tmp;
        }
    const double rin = F.g - d - 1, rout = F.g;
    for (int iv = 0; iv + 1 < nb; ++iv) {
        double s1 = bp[iv], s2 = bp[iv + 1];
        if (!(s2 > s1)) continue;
        double sm = 0.5 * (s1 + s2);
        double rm = sqrt(R2 + sm * sm);
        if (rm <= rin) continue;
        if (rm >= rout) {
            if (ang) {
                double dth = sgn * atan2(h * (s2 - s1), h * h + s1 * s2);
                acc[0] += dth * F.G0;
                acc[1] += dth * F.sz * F.N0;
                if (ncomp > 2) {
                    acc[2] += dth * F.N0;
                    acc[3] += dth * F.sz * F.dN0;
                    acc[4] += dth * F.dN0;
                }
            }
            continue;
        }
        double a = fmin(fabs(s1), fabs(s2)), b = fmax(fabs(s1), fabs(s2));
        if (ang) {
            double u1 = asinh(a / h), u2 = asinh(b / h);
            int np = (int)ceil((u2 - u1) / 0.8);
            if (np < 1) np = 1;
            double hw = 0.5 * (u2 - u1) / np;
            double loc[5] = {0, 0, 0, 0, 0};
            for (int p = 0; p < np; ++p) {
                double c = u1 + (2 * p + 1) * hw;
                for (int q = 0; q < 10; ++q) {
                    double xq = (q < 5) ? -gl10_x(q) : gl10_x(q - 5);
                    double wq = gl10_w(q < 5 ? q : q - 5);
                    double u = c + hw * xq;
                    double ch = cosh(u);
                    double rho = h * ch;
                    double rho2 = rho * rho;
                    double r = sqrt(rho2 + F.z * F.z);
                    double f[5];
                    shell_integrands(T, F, r, rho2, f);
                    double wt = wq * hw / ch;
                    for (int m = 0; m < ncomp; ++m) loc[m] += wt * f[m];
                }
            }
            for (int m = 0; m < ncomp; ++m) acc[m] += sgn * loc[m];
        }
        if (edge && R > 1e-12) {
            double v1 = asinh(a / R), v2 = asinh(b / R);
            int np = (int)ceil((v2 - v1) / 0.8);
            if (np < 1) np = 1;
            double hw = 0.5 * (v2 - v1) / np;
            double e0 = 0.0, e1 = 0.0;
            for (int p = 0; p < np; ++p) {
                double c = v1 + (2 * p + 1) * hw;
                for (int q = 0; q < 10; ++q) {
                    double xq = (q < 5) ? -gl10_x(q) : gl10_x(q - 5);
                    double wq = gl10_w(q < 5 ? q : q - 5);
                    double v = c + hw * xq;
                    double ch = cosh(v);
                    double r = R * ch;
                    int k;
                    double t;
                    bs_locate(F.g - r, false, k, t);
                    double Nt = bs_N(T, k, t), dNt = bs_dN(T, k, t);
                    double ir = 1.0 / r;
                    // ds = R cosh(v) dv = r dv
                    double wt = wq * hw * r;
                    e0 += wt * Nt * ir;
                    e1 += wt * (dNt * ir * ir + Nt * ir * ir * ir);
                }
            }
            eint[0] += e0;
            eint[1] += e1;
        }
    }
}

// Coefficient set of collocation point X (normal nx, the paper's) against
// triangle V[9] at lag g; X and V in units of c*dt.  kinds: bit 0 C_U,
// bit 1 C_W, bit 2 Ubar, bit 3 Wbar.  out[4] = {C_U, C_W, Ubar, Wbar} in
// physical units (C_U = cdt Chat_U, C_W = Chat_W, Ubar = n_x.grad Chat_U -
// d/dg Chat_U, Wbar = (n_x.grad Chat_W - d/dg Chat_W)/cdt).
TD_HD void coef_set(const BsTable &T, const double X[3], const double nx[3], const double V[9],
                    double g, bool self, int kinds, double cdt, double out[4])
{
    double e1[3] = {V[3] - V[0], V[4] - V[1], V[5] - V[2]};
    double e2[3] = {V[6] - V[0], V[7] - V[1], V[8] - V[2]};
    double ng[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                    e1[0] * e2[1] - e1[1] * e2[0]};
    double ln = sqrt(ng[0] * ng[0] + ng[1] * ng[1] + ng[2] * ng[2]);
    ng[0] /= ln;
    ng[1] /= ln;
    ng[2] /= ln;
    // paper's normal of E: ez = -ng
    double xv[3] = {X[0] - V[0], X[1] - V[1], X[2] - V[2]};
    double z = self ? 0.0 : -(ng[0] * xv[0] + ng[1] * xv[1] + ng[2] * xv[2]);
    Foot F;
    foot_init(T, g, z, F);
    double O[3] = {X[0] + z * ng[0], X[1] + z * ng[1], X[2] + z * ng[2]};
    bool bm = (kinds & 12) != 0;
    bool edges = bm && !self;
    int ncomp = bm ? 5 : 2;
    double acc[5] = {0, 0, 0, 0, 0};
    double gu[3] = {0, 0, 0}, gw[3] = {0, 0, 0};
    for (int a = 0; a < 3; ++a) {
        int b = (a + 1) % 3;
        double pa[3] = {V[3 * a] - O[0], V[3 * a + 1] - O[1], V[3 * a + 2] - O[2]};
        double pb[3] = {V[3 * b] - O[0], V[3 * b + 1] - O[1], V[3 * b + 2] - O[2]};
        double ei[2] = {0, 0};
        subtriangle(T, F, pa, pb, ng, ncomp, edges, acc, ei);
        if (edges) {
            // outward in-plane normal of the edge: (b - a) x ng
            double ee[3] = {pb[0] - pa[0], pb[1] - pa[1], pb[2] - pa[2]};
            double nu[3] = {ee[1] * ng[2] - ee[2] * ng[1], ee[2] * ng[0] - ee[0] * ng[2],
                            ee[0] * ng[1] - ee[1] * ng[0]};
            double l = sqrt(nu[0] * nu[0] + nu[1] * nu[1] + nu[2] * nu[2]);
            for (int k = 0; k < 3; ++k) {
                gu[k] -= nu[k] / l * ei[0];
                gw[k] -= z * nu[k] / l * ei[1];
            }
        }
    }
    const double inv4pi = 0.07957747154594766788444188168625718;  // 1/(4 pi)
    double cu = inv4pi * acc[0], cw = inv4pi * acc[1];
    out[0] = cdt * cu;
    out[1] = cw;
    out[2] = out[3] = 0.0;
    if (!bm) return;
    double dgu = inv4pi * acc[2], dgw = inv4pi * acc[3];
    double dzu = -cw, dzw = -inv4pi * acc[4];
    // grad = d/dz along ez = -ng, plus the in-plane part (-1/(4 pi) sum nu int)
    double ndz = -(nx[0] * ng[0] + nx[1] * ng[1] + nx[2] * ng[2]);
    double ngu = ndz * dzu + inv4pi * (nx[0] * gu[0] + nx[1] * gu[1] + nx[2] * gu[2]);
    double ngw = ndz * dzw + inv4pi * (nx[0] * gw[0] + nx[1] * gw[1] + nx[2] * gw[2]);
    out[2] = ngu - dgu;
    out[3] = (ngw - dgw) / cdt;
}

// Distance from X to the closed triangle V (closest point by the Voronoi
// regions of vertices, edges and face) and to its farthest vertex.
TD_HD void tri_dist(const double X[3], const double V[9], double &rmin, double &rmax)
{
    const double *A = V, *B = V + 3, *C = V + 6;
    double ab[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
    double ac[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
    double ap[3] = {X[0] - A[0], X[1] - A[1], X[2] - A[2]};
    auto dot = [](const double *u, const double *v) { return u[0] * v[0] + u[1] * v[1] + u[2] * v[2]; };
    double Q[3];
    double d1 = dot(ab, ap), d2 = dot(ac, ap);
    double bp[3] = {X[0] - B[0], X[1] - B[1], X[2] - B[2]};
    double d3 = dot(ab, bp), d4 = dot(ac, bp);
    double cp[3] = {X[0] - C[0], X[1] - C[1], X[2] - C[2]};
    double d5 = dot(ab, cp), d6 = dot(ac, cp);
    double va = d3 * d6 - d5 * d4, vb = d5 * d2 - d1 * d6, vc = d1 * d4 - d3 * d2;
    if (d1 <= 0 && d2 <= 0) {
        for (int k = 0; k < 3; ++k) Q[k] = A[k];
    } else if (d3 >= 0 && d4 <= d3) {
        for (int k = 0; k < 3; ++k) Q[k] = B[k];
    } else if (vc <= 0 && d1 >= 0 && d3 <= 0) {
        double v = d1 / (d1 - d3);
        for (int k = 0; k < 3; ++k) Q[k] = A[k] + v * ab[k];
    } else if (d6 >= 0 && d5 <= d6) {
        for (int k = 0; k < 3; ++k) Q[k] = C[k];
    } else if (vb <= 0 && d2 >= 0 && d6 <= 0) {
        double w = d2 / (d2 - d6);
        for (int k = 0; k < 3; ++k) Q[k] = A[k] + w * ac[k];
    } else if (va <= 0 && (d4 - d3) >= 0 && (d5 - d6) >= 0) {
        double w = (d4 - d3) / ((d4 - d3) + (d5 - d6));
        for (int k = 0; k < 3; ++k) Q[k] = B[k] + w * (C[k] - B[k]);
    } else {
        double den = 1.0 / (va + vb + vc);
        double v = vb * den, w = vc * den;
        for (int k = 0; k < 3; ++k) Q[k] = A[k] + ab[k] * v + ac[k] * w;
    }
    double dq[3] = {X[0] - Q[0], X[1] - Q[1], X[2] - Q[2]};
    rmin = sqrt(dot(dq, dq));
    double m = 0.0;
    for (int a = 0; a < 3; ++a) {
        double dv[3] = {X[0] - V[3 * a], X[1] - V[3 * a + 1], X[2] - V[3 * a + 2]};
        double t = dot(dv, dv);
        m = t > m ? t : m;
    }
    rmax = sqrt(m);
}

// Lag window [g0, g0+cnt) of a pair: the shell g-d-1 < r < g meets
// [rmin, rmax] iff rmin < g < rmax + d + 1; lags are 1 .. gcap.
TD_HD void lag_window(double rmin, double rmax, int d, int gcap, int &g0, int &cnt)
{
    int lo = (int)floor(rmin) + 1;
    int hi = (int)ceil(rmax + d + 1) - 1;
    if (lo < 1) lo = 1;
    if (hi > gcap) hi = gcap;
    g0 = lo;
    cnt = hi >= lo ? hi - lo + 1 : 0;
}

}  // namespace tdbem
