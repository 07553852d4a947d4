/*
 * Oracle: plain, slow, FP64 CPU evaluation of the discretised layer-potential
 * coefficients of the time-domain BEM of Takahashi, Tanigawa & Miyazawa
 * (arXiv 2111.05205).  TEST INFRASTRUCTURE ONLY: the tests, the smoke check
 * and the benchmark's CPU-baseline leg call this code; the product path never
 * does.  It shares no code with the CUDA library.
 *
 * What it computes (normalised units: lengths divided by c*dt, time in dt):
 *
 *   B-spline basis N^{0,d}(tau) by the truncated-power decomposition
 *   (Section 2.3, Eq. decompose, Eq. w), its derivative and its integral.
 *
 *   Compact coefficients (Section 2.4, the identity below Eq. bie_disc that
 *   folds the kappa-sum into a B-spline of the retarded time):
 *     C_U^(g) = c dt/(4 pi) * int_E N(g - r)/r dS
 *     C_W^(g) =  1/(4 pi) * int_E n_y.(x-y) [N(g-r)/r^3 + N'(g-r)/r^2] dS
 *   and the Burton-Miller coefficients (Eq. U_W_BM)
 *     Ubar = (d/dn_x - d/dg) C_U / (c dt),  Wbar = (d/dn_x - d/dg) C_W / (c dt),
 *   with d/dn_x the derivative along the normal at the collocation point and
 *   d/dg = dt d/dt.
 *
 *   Tau-form single/double-layer coefficients U^(g), W^(g) of Eq.
 *   discretised_single_layer_potential / discretised_double_layer_potential,
 *   used by the tests to check the identity C^(g) = sum_k w^k U^(g-k).
 *
 * How (Appendix B): the foot O of the perpendicular from x to the plane of E
 * splits E into three signed sub-triangles O-V1-V2.  In polar coordinates
 * about O the radial integral is done in closed form through rho drho = r dr,
 * leaving angular integrals of functions of r_e(theta), the distance from x to
 * the edge point at angle theta.  Those are done by adaptive Gauss-Kronrod
 * (7/15) split at the angles where r_e crosses a knot radius of the B-spline.
 * In-plane gradients use the divergence theorem (edge integrals, also
 * adaptive Gauss-Kronrod split at the knot crossings).
 *
 * Conventions (readings of the paper, see the design notes):
 *   - normals n are the paper's: they point INTO the scatterer V (the outward
 *     normal of the exterior domain); the mesh gives n_geo = -n;
 *   - the free term is absorbed by evaluating every coefficient as the limit
 *     of the collocation point approaching S from the side n points to
 *     (z -> 0+ with z = n_y.(x - y)); for the self element this gives the
 *     double-layer jump C_W^(g)_ii = N(g)/2 and left limits N'(g^-) of the
 *     B-spline derivative at knots.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846264338327950288

/* ------------------------------------------------------------------ */
/* B-spline temporal basis, Section 2.3                                */
/* ------------------------------------------------------------------ */

/* Eq. (w): w^{kappa,d} = (d+1) / prod_{k=0, k!=kappa}^{d+1} (k - kappa). */
double orc_w(int kappa, int d)
{
    double p = 1.0;
    for (int k = 0; k <= d + 1; ++k)
        if (k != kappa) p *= (double)(k - kappa);
    return (double)(d + 1) / p;
}

/* (x)_+^e with the convention (x)_+^0 = 1 for x > 0 and 0 for x <= 0. */
static double tpow(double x, int e)
{
    if (x <= 0.0) return 0.0;
    double r = 1.0;
    for (int i = 0; i < e; ++i) r *= x;
    return r;
}

/* (x)_>=^e: like tpow but with (0)^0 = 1 (right-sided truncated powers). */
static double tpow_ge(double x, int e)
{
    if (x < 0.0) return 0.0;
    double r = 1.0;
    for (int i = 0; i < e; ++i) r *= x;
    return r;
}

/* Eq. (decompose) with dt = 1 and beta = 0: N^{0,d}(tau).
 * For tau past the middle of the support the same decomposition is used in
 * its right-sided form: because the (d+1)-th difference with weights w of a
 * degree-d polynomial vanishes, sum_k w^k (tau-k)_+^d equals
 * -(-1)^d sum_k w^k (k-tau)_+^d; this avoids summing large truncated
 * powers that cancel near the end of the support. */
double orc_N(int d, double tau)
{
    if (tau <= 0.0 || tau >= (double)(d + 1)) return 0.0; /* Remark (support) */
    double s = 0.0;
    if (2.0 * tau <= (double)(d + 1)) {
        for (int k = 0; k <= d + 1; ++k) s += orc_w(k, d) * tpow(tau - k, d);
    } else {
        for (int k = 0; k <= d + 1; ++k) s += orc_w(k, d) * tpow(k - tau, d);
        s = (d & 1) ? s : -s;
    }
    return s;
}

/* dN/dtau; at a knot the left limit. */
double orc_dN(int d, double tau)
{
    if (tau <= 0.0 || tau > (double)(d + 1)) return 0.0;
    double s = 0.0;
    if (2.0 * tau <= (double)(d + 1)) {
        /* (0)_+^0 = 0: the term of a knot at tau switches on after it */
        for (int k = 0; k <= d + 1; ++k) s += orc_w(k, d) * (double)d * tpow(tau - k, d - 1);
    } else {
        /* derivative of -(-1)^d (k - tau)_+^d is (-1)^d d (k - tau)_+^{d-1};
         * (0)^0 = 1 keeps the left limit at a knot */
        for (int k = 0; k <= d + 1; ++k) s += orc_w(k, d) * (double)d * tpow_ge(k - tau, d - 1);
        s = (d & 1) ? -s : s;
    }
    return s;
}

/* G(tau) = int_0^tau N^{0,d}; G = 1 past the support since int N = 1. */
double orc_G(int d, double tau)
{
    if (tau <= 0.0) return 0.0;
    if (tau >= (double)(d + 1)) return 1.0;
    double s = 0.0;
    if (2.0 * tau <= (double)(d + 1)) {
        for (int k = 0; k <= d + 1; ++k) s += orc_w(k, d) * tpow(tau - k, d + 1);
        return s / (double)(d + 1);
    }
    /* 1 - int_tau^{d+1} N with the right-sided form */
    for (int k = 0; k <= d + 1; ++k) s += orc_w(k, d) * tpow(k - tau, d + 1);
    s /= (double)(d + 1);
    return (d & 1) ? 1.0 - s : 1.0 + s;
}

/* Gc(tau) = int_tau^{d+1} N^{0,d} = 1 - G(tau), evaluated without the
 * cancellation of 1 - G near the end of the support. */
double orc_Gc(int d, double tau)
{
    if (tau >= (double)(d + 1)) return 0.0;
    if (tau <= 0.0) return 1.0;
    if (2.0 * tau <= (double)(d + 1)) return 1.0 - orc_G(d, tau);
    double s = 0.0;
    for (int k = 0; k <= d + 1; ++k) s += orc_w(k, d) * tpow(k - tau, d + 1);
    s /= (double)(d + 1);
    return (d & 1) ? s : -s;
}

/* G(b) - G(a) = int_a^b N, from whichever end avoids cancellation. */
static double G_diff(int d, double b, double a)
{
    double mid = 0.5 * (double)(d + 1);
    if (a <= mid && b <= mid) return orc_G(d, b) - orc_G(d, a);
    return orc_Gc(d, a) - orc_Gc(d, b);
}

/* ------------------------------------------------------------------ */
/* small vector helpers                                                */
/* ------------------------------------------------------------------ */

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static void sub3(const double *a, const double *b, double *c) { c[0] = a[0] - b[0]; c[1] = a[1] - b[1]; c[2] = a[2] - b[2]; }
static double norm3(const double *a) { return sqrt(dot3(a, a)); }

/* ------------------------------------------------------------------ */
/* radial profiles                                                     */
/* ------------------------------------------------------------------ */

#define ORC_NC 6 /* number of integrand components carried together */

typedef struct {
    int d;
    double g;      /* lag gamma (normalised retarded time) */
    int tauform;   /* 0: compact B-spline form; 1: truncated power form */
    double z;      /* signed height of x over the element plane */
    double sz;     /* sign taken for z (z == 0: +1, the limit from the n side) */
} profile_t;

/* Angular integrands at edge distance r.  With rho drho = r dr the radial
 * integral from the foot (r = |z|) to the edge (r = r_e) is done in closed
 * form; the components are those radial integrals (and their derivatives)
 * as functions of r = r_e:
 * compact form,
 *   0: G(g-|z|) - G(g-r)                            -> 4 pi Chat_U
 *   1: N(g-|z|) sz - z N(g-r)/r                     -> 4 pi Chat_W
 *   2: N(g-|z|) - N(g-r)                            -> 4 pi d/dg Chat_U
 *   3: N'(g-|z|) sz - z N'(g-r)/r                   -> 4 pi d/dg Chat_W
 *   4: N(g-r)/r - z^2 N'(g-r)/r^2 - z^2 N(g-r)/r^3 + N'(g-|z|)
 *                                                   -> -4 pi d/dz Chat_W
 * tau form (kernel (g-r)_+^d / r),
 *   0: ((g-|z|)_+^{d+1} - (g-r)_+^{d+1}) / (d+1)   -> 4 pi U / (c dt)
 *   1: (g-|z|)_+^d sz - z (g-r)_+^d / r             -> 4 pi W
 */
static void profile_eval(const profile_t *p, double r, double *f)
{
    double t = p->g - r, t0 = p->g - fabs(p->z), z = p->z;
    if (!p->tauform) {
        double n = orc_N(p->d, t), dn = orc_dN(p->d, t);
        double n0 = orc_N(p->d, t0), dn0 = orc_dN(p->d, t0);
        f[0] = G_diff(p->d, t0, t);
        f[1] = n0 * p->sz - z * n / r;
        f[2] = n0 - n;
        f[3] = dn0 * p->sz - z * dn / r;
        f[4] = n / r - z * z * dn / (r * r) - z * z * n / (r * r * r) + dn0;
        f[5] = 0.0;
        /* magnitudes of the terms: the rounding noise of f is ~eps times these */
        f[ORC_NC + 0] = fmin(orc_G(p->d, t0) + orc_G(p->d, t), orc_Gc(p->d, t) + orc_Gc(p->d, t0));
        f[ORC_NC + 1] = fabs(n0) + fabs(z * n / r);
        f[ORC_NC + 2] = fabs(n0) + fabs(n);
        f[ORC_NC + 3] = fabs(dn0) + fabs(z * dn / r);
        f[ORC_NC + 4] = fabs(n / r) + fabs(z * z * dn / (r * r)) + fabs(z * z * n / (r * r * r)) + fabs(dn0);
        f[ORC_NC + 5] = 0.0;
    } else {
        double a0 = tpow(t0, p->d + 1), a1 = tpow(t, p->d + 1);
        f[0] = (a0 - a1) / (double)(p->d + 1);
        f[1] = tpow(t0, p->d) * p->sz - z * tpow(t, p->d) / r;
        f[2] = f[3] = f[4] = f[5] = 0.0;
        f[ORC_NC + 0] = (a0 + a1) / (double)(p->d + 1);
        f[ORC_NC + 1] = tpow(t0, p->d) + fabs(z * tpow(t, p->d) / r);
        f[ORC_NC + 2] = f[ORC_NC + 3] = f[ORC_NC + 4] = f[ORC_NC + 5] = 0.0;
    }
}

/* knot radii where the profile changes polynomial piece */
static int profile_knots(const profile_t *p, double *R)
{
    if (!p->tauform) {
        int n = 0;
        for (int k = 0; k <= p->d + 1; ++k) R[n++] = p->g - (double)k;
        return n;
    }
    R[0] = p->g;
    return 1;
}

/* ------------------------------------------------------------------ */
/* adaptive Gauss-Kronrod 7/15                                         */
/* ------------------------------------------------------------------ */

static const double XGK[8] = {
    0.991455371120812639206854697526329, 0.949107912342758524526189684047851,
    0.864864423359769072789712788640926, 0.741531185599394439863864773280788,
    0.586087235467691130294144845693013, 0.405845151377397166906606412076961,
    0.207784955007898467600689403773245, 0.000000000000000000000000000000000};
static const double WGK[8] = {
    0.022935322010529224963732008058970, 0.063092092629978553290700663189204,
    0.104790010322250183839876322541518, 0.140653259715525918745189590510238,
    0.169004726639267902826583426598550, 0.190350578064785409913256402421014,
    0.204432940075298892414161999234649, 0.209482141084727828012999174891714};
static const double WG[4] = {
    0.129484966168869693270611432679082, 0.279705391489276667901467771423780,
    0.381830050505118944950369775488975, 0.417959183673469387755102040816327};

/* An integrand writes ORC_NC values f[0..NC-1] and, in f[NC..2NC-1], the
 * magnitudes of the terms they were summed from (their rounding noise is
 * about eps times those). */
typedef void (*integrand_fn)(void *ctx, double t, double *f);

/* Panel budget of one integrate() call: refinement stops (and the event is
 * counted) if the error test is still failing after this many panels, so
 * that rounding noise in an integrand can never make the recursion blow
 * up.  The tests check that the count stays zero. */
#define ORC_PANEL_BUDGET 20000
static long orc_budget_events = 0;
long orc_budget_hits(void) { return orc_budget_events; }
static _Thread_local long orc_panels = 0;

/* One Gauss-Kronrod 7/15 panel on [a, b] for every component: K (the
 * Kronrod result), E (error estimate of K in the usual way of QUADPACK's
 * 15-point rule: resasc * min(1, (200 |K - G| / resasc)^1.5), at least
 * 50 eps int |f|) and A (int |f|). */
static void gk15(integrand_fn fn, void *ctx, double a, double b, double *K, double *E, double *A)
{
    double c = 0.5 * (a + b), h = 0.5 * (b - a);
    double fv[15][2 * ORC_NC];
    fn(ctx, c, fv[14]);
    for (int j = 0; j < 7; ++j) {
        fn(ctx, c - h * XGK[j], fv[2 * j]);
        fn(ctx, c + h * XGK[j], fv[2 * j + 1]);
    }
    for (int m = 0; m < ORC_NC; ++m) {
        double k = WGK[7] * fv[14][m], g = WG[3] * fv[14][m];
        double ab = WGK[7] * fmax(fabs(fv[14][m]), fv[14][ORC_NC + m]);
        for (int j = 0; j < 7; ++j) {
            double s = fv[2 * j][m] + fv[2 * j + 1][m];
            k += WGK[j] * s;
            ab += WGK[j] * (fmax(fabs(fv[2 * j][m]), fv[2 * j][ORC_NC + m]) +
                            fmax(fabs(fv[2 * j + 1][m]), fv[2 * j + 1][ORC_NC + m]));
            if (j & 1) g += WG[j >> 1] * s;
        }
        double mean = 0.5 * k, asc = WGK[7] * fabs(fv[14][m] - mean);
        for (int j = 0; j < 7; ++j)
            asc += WGK[j] * (fabs(fv[2 * j][m] - mean) + fabs(fv[2 * j + 1][m] - mean));
        double ah = fabs(h);
        K[m] = k * h;
        A[m] = ab * ah;
        asc *= ah;
        double err = fabs((k - g) * h);
        if (asc != 0.0 && err != 0.0) {
            double r = pow(200.0 * err / asc, 1.5);
            err = asc * (r < 1.0 ? r : 1.0);
        }
        E[m] = err;
    }
}

/* tol: local tolerance (halved per level); floor: fixed absolute tolerance
 * below which the rounding noise of the integrand (e.g. of the B-spline
 * sums) cannot be resolved. */
static void adapt(integrand_fn fn, void *ctx, double a, double b, const double *tol,
                  const double *floor_, int depth, double *out)
{
    double K[ORC_NC], E[ORC_NC], A[ORC_NC];
    gk15(fn, ctx, a, b, K, E, A);
    int ok = 1;
    for (int m = 0; m < ORC_NC; ++m)
        if (E[m] > tol[m] && E[m] > floor_[m] && E[m] > 8.0 * 2.220446049250313e-16 * A[m]) ok = 0;
    ++orc_panels;
    if (!ok && (depth >= 40 || orc_panels > ORC_PANEL_BUDGET)) {
        if (orc_panels == ORC_PANEL_BUDGET + 1 || depth >= 40) {
#pragma omp atomic
            ++orc_budget_events;
        }
        ok = 1;
    }
    if (ok) {
        for (int m = 0; m < ORC_NC; ++m) out[m] += K[m];
        return;
    }
    double c = 0.5 * (a + b), t2[ORC_NC];
    for (int m = 0; m < ORC_NC; ++m) t2[m] = 0.5 * tol[m];
    adapt(fn, ctx, a, c, t2, floor_, depth + 1, out);
    adapt(fn, ctx, c, b, t2, floor_, depth + 1, out);
}

/* integrate fn over [a, b] to ~1e-15 relative of int |f| */
static void integrate(integrand_fn fn, void *ctx, double a, double b, double *out)
{
    if (!(b > a)) return;
    double K[ORC_NC], E[ORC_NC], A[ORC_NC], tol[ORC_NC], fl[ORC_NC];
    gk15(fn, ctx, a, b, K, E, A);
    for (int m = 0; m < ORC_NC; ++m) {
        tol[m] = 1e-15 * A[m] + 1e-300;
        fl[m] = 1e-17 * A[m] + 1e-300;
    }
    orc_panels = 0;
    adapt(fn, ctx, a, b, tol, fl, 0, out);
}

/* ------------------------------------------------------------------ */
/* angular integrals over one sub-triangle O-a-b                      */
/* ------------------------------------------------------------------ */

typedef struct {
    const profile_t *prof;
    double pa[3], e[3]; /* in-plane, relative to O */
    double A2;          /* (pa x pb).n: twice the signed area of O-a-b */
    double z2;          /* z^2 */
} ang_ctx;

/* The angle integral over the sub-triangle O-a-b is taken along its edge:
 * with P(lam) = pa + lam (pb - pa), dtheta = A2 / |P|^2 dlam, so
 * int_0^phi f(r_e(theta)) dtheta = int_0^1 f(r(lam)) A2 / |P(lam)|^2 dlam,
 * r(lam) = sqrt(|P|^2 + z^2).  The parametrisation stays well conditioned
 * for thin sub-triangles (O close to the edge's line). */
static void ang_fn(void *vctx, double lam, double *f)
{
    ang_ctx *c = (ang_ctx *)vctx;
    double P[3];
    for (int k = 0; k < 3; ++k) P[k] = c->pa[k] + lam * c->e[k];
    double p2 = dot3(P, P);
    double r = sqrt(p2 + c->z2);
    profile_eval(c->prof, r, f);
    double wgt = c->A2 / p2;
    for (int m = 0; m < ORC_NC; ++m) {
        f[m] *= wgt;
        f[ORC_NC + m] *= fabs(wgt);
    }
}

/* signed angle from p to q about n */
static double signed_angle(const double *p, const double *q, const double *n)
{
    double c[3];
    cross3(p, q, c);
    return atan2(dot3(c, n), dot3(p, q));
}

/* Adds to out[] the integrals over the angle of the sub-triangle O-a-b
 * (signed, positive when a -> b turns counter-clockwise about n); returns
 * that angle (0 for a degenerate sub-triangle, O on the edge's line). */
static double subtri_angular(const profile_t *prof, const double *pa, const double *pb,
                             const double *n, double z, double *out)
{
    ang_ctx c;
    c.prof = prof;
    c.z2 = z * z;
    memcpy(c.pa, pa, sizeof c.pa);
    sub3(pb, pa, c.e);
    double xp[3];
    cross3(pa, pb, xp);
    c.A2 = dot3(xp, n);
    double la = norm3(pa), lb = norm3(pb), le = norm3(c.e);
    if (la == 0.0 || lb == 0.0 || fabs(c.A2) <= 1e-14 * la * lb) return 0.0;
    double phi = signed_angle(pa, pb, n);
    /* breakpoints: edge points at in-plane distance sqrt(R^2 - z^2) */
    double R[8], br[32];
    int nk = profile_knots(prof, R), nb = 0;
    double pe = dot3(pa, c.e);
    for (int k = 0; k < nk; ++k) {
        double rr = R[k] * R[k] - z * z;
        if (R[k] <= 0.0 || rr <= 0.0) continue;
        /* |pa + lam e|^2 = rr */
        double A = le * le, B = 2.0 * pe, C = la * la - rr;
        double disc = B * B - 4.0 * A * C;
        if (disc < 0.0) continue;
        double sq = sqrt(disc);
        double ls[2] = {(-B - sq) / (2.0 * A), (-B + sq) / (2.0 * A)};
        for (int q = 0; q < 2; ++q)
            if (ls[q] > 0.0 && ls[q] < 1.0) br[nb++] = ls[q];
    }
    br[nb++] = 0.0;
    br[nb++] = 1.0;
    for (int i = 1; i < nb; ++i)
        for (int j = i; j > 0 && br[j] < br[j - 1]; --j) { double t = br[j]; br[j] = br[j - 1]; br[j - 1] = t; }
    double acc[ORC_NC] = {0};
    for (int i = 0; i + 1 < nb; ++i) integrate(ang_fn, &c, br[i], br[i + 1], acc);
    for (int m = 0; m < ORC_NC; ++m) out[m] += acc[m];
    return phi;
}

/* ------------------------------------------------------------------ */
/* edge line integrals (in-plane gradients)                           */
/* ------------------------------------------------------------------ */

typedef struct {
    const profile_t *prof;
    double pa[3], e[3];
    double z2, len;
} edge_ctx;

/* components at lambda: 0: N/r, 1: N'/r^2, 2: N/r^3  (compact profile) */
static void edge_fn(void *vctx, double lam, double *f)
{
    edge_ctx *c = (edge_ctx *)vctx;
    double P[3];
    for (int m = 0; m < 3; ++m) P[m] = c->pa[m] + lam * c->e[m];
    double r = sqrt(dot3(P, P) + c->z2);
    double t = c->prof->g - r;
    double n = orc_N(c->prof->d, t), dn = orc_dN(c->prof->d, t);
    f[0] = c->len * n / r;
    f[1] = c->len * dn / (r * r);
    f[2] = c->len * n / (r * r * r);
    f[3] = f[4] = f[5] = 0.0;
    for (int m = 0; m < ORC_NC; ++m) f[ORC_NC + m] = fabs(f[m]);
}

static void edge_line(const profile_t *prof, const double *pa, const double *pb, double z, double *out3)
{
    edge_ctx c;
    c.prof = prof;
    c.z2 = z * z;
    memcpy(c.pa, pa, sizeof c.pa);
    sub3(pb, pa, c.e);
    c.len = norm3(c.e);
    double R[8], br[32];
    int nk = profile_knots(prof, R), nb = 0;
    double la = norm3(pa), pe = dot3(pa, c.e);
    for (int k = 0; k < nk; ++k) {
        double rr = R[k] * R[k] - z * z;
        if (R[k] <= 0.0 || rr <= 0.0) continue;
        double A = c.len * c.len, B = 2.0 * pe, C = la * la - rr;
        double disc = B * B - 4.0 * A * C;
        if (disc < 0.0) continue;
        double sq = sqrt(disc);
        double ls[2] = {(-B - sq) / (2.0 * A), (-B + sq) / (2.0 * A)};
        for (int q = 0; q < 2; ++q)
            if (ls[q] > 0.0 && ls[q] < 1.0) br[nb++] = ls[q];
    }
    br[nb++] = 0.0;
    br[nb++] = 1.0;
    for (int i = 1; i < nb; ++i)
        for (int j = i; j > 0 && br[j] < br[j - 1]; --j) { double t = br[j]; br[j] = br[j - 1]; br[j - 1] = t; }
    double acc[ORC_NC] = {0};
    for (int i = 0; i + 1 < nb; ++i) integrate(edge_fn, &c, br[i], br[i + 1], acc);
    out3[0] += acc[0];
    out3[1] += acc[1];
    out3[2] += acc[2];
}

/* ------------------------------------------------------------------ */
/* one coefficient set                                                 */
/* ------------------------------------------------------------------ */

/*
 * Parts of the coefficient set in normalised units (lengths / c dt) for the
 * collocation point x against triangle v (9 coordinates, counter-clockwise
 * about n_geo = -n_y) at lag g:
 *   parts[0] = Chat_U = 1/(4 pi) int N(g - r)/r dS
 *   parts[1] = Chat_W = 1/(4 pi) int n_y.(x-y) [N/r^3 + N'/r^2] dS
 *   parts[2] = d/dg Chat_U,  parts[3] = d/dg Chat_W
 *   parts[4..6]  = grad_x Chat_U,  parts[7..9] = grad_x Chat_W  (global axes)
 * self = 1: x is this triangle's own collocation point (z = 0, limit from the
 * n_y side, and the in-plane gradients, which are not needed there, are 0).
 */
void orc_coef_parts(const double *x, const double *v, double g, int d, double cdt, int self,
                    int want_grad, double *parts)
{
    double X[3], V[3][3];
    for (int k = 0; k < 3; ++k) X[k] = x[k] / cdt;
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 3; ++k) V[a][k] = v[3 * a + k] / cdt;
    double e1[3], e2[3], ng[3], ez[3];
    sub3(V[1], V[0], e1);
    sub3(V[2], V[0], e2);
    cross3(e1, e2, ng);
    double ln = norm3(ng);
    for (int k = 0; k < 3; ++k) { ng[k] /= ln; ez[k] = -ng[k]; }
    double xv[3];
    sub3(X, V[0], xv);
    double z = self ? 0.0 : dot3(ez, xv);
    double sz = (z < 0.0) ? -1.0 : 1.0; /* z == 0: limit from the n side */
    double az = fabs(z);
    double O[3], p[3][3];
    for (int k = 0; k < 3; ++k) O[k] = X[k] - z * ez[k];
    for (int a = 0; a < 3; ++a) sub3(V[a], O, p[a]);

    profile_t prof = {d, g, 0, z, sz};
    double I[ORC_NC] = {0};
    for (int a = 0; a < 3; ++a) subtri_angular(&prof, p[a], p[(a + 1) % 3], ng, z, I);
    (void)az;

    const double inv4pi = 1.0 / (4.0 * ORC_PI);
    double cu = inv4pi * I[0];
    double cw = inv4pi * I[1];
    parts[0] = cu;
    parts[1] = cw;
    parts[2] = inv4pi * I[2];
    parts[3] = inv4pi * I[3];
    for (int k = 4; k < 10; ++k) parts[k] = 0.0;
    if (!want_grad) return;
    /* normal (z) derivatives: d/dz Chat_U = -Chat_W and the second
     * z-derivative of int N(g-r)/r dS for Chat_W */
    double dz_cu = -cw;
    double dz_cw = -inv4pi * I[4];
    double gu[3] = {0, 0, 0}, gw[3] = {0, 0, 0};
    if (!self) {
        /* in-plane gradients by the divergence theorem:
         * grad_par int F dS = -sum_edges nu_e int_e F dl */
        for (int a = 0; a < 3; ++a) {
            double L[3] = {0, 0, 0}, ee[3], nu[3];
            edge_line(&prof, p[a], p[(a + 1) % 3], z, L);
            sub3(p[(a + 1) % 3], p[a], ee);
            cross3(ee, ng, nu); /* outward in-plane normal of the edge */
            double l = norm3(nu);
            for (int k = 0; k < 3; ++k) {
                gu[k] += -inv4pi * (nu[k] / l) * L[0];
                gw[k] += -inv4pi * z * (nu[k] / l) * (L[1] + L[2]);
            }
        }
    }
    for (int k = 0; k < 3; ++k) {
        parts[4 + k] = dz_cu * ez[k] + gu[k];
        parts[7 + k] = dz_cw * ez[k] + gw[k];
    }
}

/*
 * x[3]: collocation point; nx[3]: the paper's normal at x (into V);
 * v[9]: triangle vertices, counter-clockwise about n_geo (= -ny);
 * g: lag; d: B-spline order; cdt: c*dt; self: 1 if x is the collocation
 * point of this very triangle (then z = 0 and the limit z -> 0+ is taken).
 * out[4] = { C_U, C_W, Ubar, Wbar } in physical units:
 *   C_U = c dt Chat_U, C_W = Chat_W,
 *   Ubar = n_x.grad Chat_U - d/dg Chat_U,
 *   Wbar = (n_x.grad Chat_W - d/dg Chat_W) / (c dt).
 */
void orc_coef(const double *x, const double *nx, const double *v, double g, int d, double cdt,
              int self, int want_bm, double *out)
{
    double P[10];
    orc_coef_parts(x, v, g, d, cdt, self, want_bm, P);
    out[0] = cdt * P[0];
    out[1] = P[1];
    out[2] = out[3] = 0.0;
    if (!want_bm) return;
    double ngu = nx[0] * P[4] + nx[1] * P[5] + nx[2] * P[6];
    double ngw = nx[0] * P[7] + nx[1] * P[8] + nx[2] * P[9];
    out[2] = ngu - P[2];
    out[3] = (ngw - P[3]) / cdt;
}

/* Tau-form coefficients with kernel (c t_g - r)_+^d / (4 pi (c dt)^d r):
 * out[0] = U^(g), out[1] = W^(g) (double layer, same normal and limit
 * conventions as above). */
void orc_coef_tau(const double *x, const double *v, double g, int d, double cdt, int self, double *out)
{
    double X[3], V[3][3];
    for (int k = 0; k < 3; ++k) X[k] = x[k] / cdt;
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 3; ++k) V[a][k] = v[3 * a + k] / cdt;
    double e1[3], e2[3], ng[3], ez[3];
    sub3(V[1], V[0], e1);
    sub3(V[2], V[0], e2);
    cross3(e1, e2, ng);
    double ln = norm3(ng);
    for (int k = 0; k < 3; ++k) { ng[k] /= ln; ez[k] = -ng[k]; }
    double xv[3];
    sub3(X, V[0], xv);
    double z = self ? 0.0 : dot3(ez, xv);
    double sz = (z < 0.0) ? -1.0 : 1.0, az = fabs(z);
    double O[3], p[3][3];
    for (int k = 0; k < 3; ++k) O[k] = X[k] - z * ez[k];
    for (int a = 0; a < 3; ++a) sub3(V[a], O, p[a]);
    profile_t prof = {d, g, 1, z, sz};
    double I[ORC_NC] = {0};
    for (int a = 0; a < 3; ++a) subtri_angular(&prof, p[a], p[(a + 1) % 3], ng, z, I);
    (void)az;
    double inv4pi = 1.0 / (4.0 * ORC_PI);
    out[0] = cdt * inv4pi * I[0];
    out[1] = inv4pi * I[1];
}

/* ------------------------------------------------------------------ */
/* windows and dense all-pairs driver                                  */
/* ------------------------------------------------------------------ */

static double seg_dist2(const double *x, const double *a, const double *b)
{
    double ab[3], ax[3];
    sub3(b, a, ab);
    sub3(x, a, ax);
    double t = dot3(ax, ab) / dot3(ab, ab);
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    double d[3];
    for (int k = 0; k < 3; ++k) d[k] = ax[k] - t * ab[k];
    return dot3(d, d);
}

/* distance from x to the closed triangle v, and to its farthest vertex */
void orc_tri_dist(const double *x, const double *v, double *rmin, double *rmax)
{
    const double *A = v, *B = v + 3, *C = v + 6;
    double e1[3], e2[3], n[3], xa[3];
    sub3(B, A, e1);
    sub3(C, A, e2);
    cross3(e1, e2, n);
    double nn = dot3(n, n);
    sub3(x, A, xa);
    double h = dot3(xa, n) / nn;
    double P[3];
    for (int k = 0; k < 3; ++k) P[k] = x[k] - h * n[k];
    /* barycentric of P */
    double c0[3], c1[3], c2[3], pa[3], pb[3], pc[3];
    sub3(A, P, pa);
    sub3(B, P, pb);
    sub3(C, P, pc);
    cross3(pb, pc, c0);
    cross3(pc, pa, c1);
    cross3(pa, pb, c2);
    double l0 = dot3(c0, n), l1 = dot3(c1, n), l2 = dot3(c2, n);
    double r2;
    if (l0 >= 0 && l1 >= 0 && l2 >= 0) {
        r2 = h * h * nn;
    } else {
        r2 = seg_dist2(x, A, B);
        double t = seg_dist2(x, B, C);
        if (t < r2) r2 = t;
        t = seg_dist2(x, C, A);
        if (t < r2) r2 = t;
    }
    *rmin = sqrt(r2);
    double m = 0.0, d[3];
    for (int a = 0; a < 3; ++a) {
        sub3(x, v + 3 * a, d);
        double t = dot3(d, d);
        if (t > m) m = t;
    }
    *rmax = sqrt(m);
}

/*
 * Dense coefficients for every (lag g in [1, gmax], row i, column j):
 * out_k[(g * ns + i) * ns + j] for k in {cu, cw, ub, wb}; NULL pointers skip
 * that kind (want_bm = ub or wb non-NULL).  tri[ns*9] vertex coordinates,
 * xc[ns*3] collocation points, nx[ns*3] the paper's normals.  Lags outside a
 * pair's support window are left untouched (the caller zero-fills).
 * OpenMP over rows.  Returns the largest lag touched.
 */
int orc_dense(int ns, const double *tri, const double *xc, const double *nx, int d, double cdt,
              int gmax, double *cu, double *cw, double *ub, double *wb)
{
    int want_bm = (ub != NULL) || (wb != NULL);
    int gtop = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(max : gtop)
    for (int i = 0; i < ns; ++i) {
        for (int j = 0; j < ns; ++j) {
            double rmin, rmax;
            orc_tri_dist(xc + 3 * i, tri + 9 * j, &rmin, &rmax);
            int g0 = (int)floor(rmin / cdt) + 1;
            int g1 = (int)ceil(rmax / cdt + d + 1) - 1;
            if (g0 < 1) g0 = 1;
            if (g1 > gmax) g1 = gmax;
            for (int g = g0; g <= g1; ++g) {
                double o[4];
                orc_coef(xc + 3 * i, nx + 3 * i, tri + 9 * j, (double)g, d, cdt, i == j, want_bm, o);
                size_t idx = ((size_t)g * ns + i) * ns + j;
                if (cu) cu[idx] = o[0];
                if (cw) cw[idx] = o[1];
                if (ub) ub[idx] = o[2];
                if (wb) wb[idx] = o[3];
                if (g > gtop) gtop = g;
            }
        }
    }
    return gtop;
}

/* Coefficients of selected rows for every column and lag (sampled checks):
 * out_k[(r * (gmax+1) + g) * ns + j] for r < nrows. */
void orc_rows(int ns, const double *tri, const double *xc, const double *nx, int d, double cdt,
              int gmax, int nrows, const int *rows, double *cu, double *cw, double *ub, double *wb)
{
    int want_bm = (ub != NULL) || (wb != NULL);
#pragma omp parallel for schedule(dynamic, 1) collapse(2)
    for (int r = 0; r < nrows; ++r) {
        for (int j = 0; j < ns; ++j) {
            int i = rows[r];
            double rmin, rmax;
            orc_tri_dist(xc + 3 * i, tri + 9 * j, &rmin, &rmax);
            int g0 = (int)floor(rmin / cdt) + 1;
            int g1 = (int)ceil(rmax / cdt + d + 1) - 1;
            if (g0 < 1) g0 = 1;
            if (g1 > gmax) g1 = gmax;
            for (int g = g0; g <= g1; ++g) {
                double o[4];
                orc_coef(xc + 3 * i, nx + 3 * i, tri + 9 * j, (double)g, d, cdt, i == j, want_bm, o);
                size_t idx = ((size_t)r * (gmax + 1) + g) * ns + j;
                if (cu) cu[idx] = o[0];
                if (cw) cw[idx] = o[1];
                if (ub) ub[idx] = o[2];
                if (wb) wb[idx] = o[3];
            }
        }
    }
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
