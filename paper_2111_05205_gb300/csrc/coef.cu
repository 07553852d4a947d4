// Setup kernels: element geometry, lag windows, influence coefficients and
// the zero-lag matrix (Section 2.3-2.5, Appendix B).
#include "tdbem_internal.cuh"

namespace tdbem {

__constant__ BsTable c_bs;

void set_bspline_table(const BsTable &T, cudaStream_t s)
{
    cudaMemcpyToSymbolAsync(c_bs, &T, sizeof(BsTable), 0, cudaMemcpyHostToDevice, s);
}

// Collocation points (centroids, Section 2.3), the paper's normals and the
// vertices, normalised by c*dt.
__global__ void k_geometry(int ns, const double *__restrict__ xyz, const int32_t *__restrict__ tri,
                           double inv_cdt, double *V, double *X, double *xc, double *n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns) return;
    double v[9];
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 3; ++k) v[3 * a + k] = xyz[3 * tri[3 * i + a] + k];
    for (int k = 0; k < 3; ++k) {
        double c = (v[k] + v[3 + k] + v[6 + k]) / 3.0;
        xc[3 * i + k] = c;
        X[3 * i + k] = c * inv_cdt;
    }
    for (int k = 0; k < 9; ++k) V[9 * i + k] = v[k] * inv_cdt;
    double e1[3] = {v[3] - v[0], v[4] - v[1], v[5] - v[2]};
    double e2[3] = {v[6] - v[0], v[7] - v[1], v[8] - v[2]};
    double g[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    double l = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    for (int k = 0; k < 3; ++k) n[3 * i + k] = -g[k] / l;
}

cudaError_t launch_geometry(tdbem_ctx *c)
{
    int ns = c->ns;
    k_geometry<<<(ns + 127) / 128, 128, 0, c->s>>>(ns, c->d_xyz, c->d_tri, 1.0 / c->cdt, c->d_V, c->d_X,
                                                   c->d_xc, c->d_n);
    return cudaGetLastError();
}

// Pair lists: row i owns pairs p in [prow[i], prow[i+1]) with column
// col[p] (col == nullptr: the dense list j = p - prow[i]); the pairs of a
// row are cut into blocks of 32 (global block indices [rowblk[i],
// rowblk[i+1])).  Row of a global block index.
__device__ __forceinline__ int row_of_block(const int64_t *__restrict__ rowblk, int ns, int64_t gb)
{
    int lo = 0, hi = ns - 1;
    while (lo < hi) {
        int m = (lo + hi + 1) >> 1;
        if (rowblk[m] <= gb)
            lo = m;
        else
            hi = m - 1;
    }
    return lo;
}

// Lag window of every pair (Remark gamma_bound, per pair): meta = g0 |
// cnt << 12, and the number of coefficients of each 32-pair block.  flags:
// max cnt, max g0, max lag.
__global__ void k_windows(int ns, int d, int gcap, const int64_t *__restrict__ prow, const int32_t *__restrict__ col,
                          const int64_t *__restrict__ rowblk, int64_t nbt, const double *__restrict__ X,
                          const double *__restrict__ V, uint16_t *meta, int32_t *btot, int *maxcnt, int *maxg0,
                          int *gtop)
{
    int lane = threadIdx.x & 31;
    int lc = 0, lg = 0, lt = 0;
    for (int64_t gb = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; gb < nbt;
         gb += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        int i = row_of_block(rowblk, ns, gb);
        int64_t p = prow[i] + (gb - rowblk[i]) * 32 + lane;
        int cnt = 0, g0 = 0;
        if (p < prow[i + 1]) {
            int j = col ? col[p] : (int)(p - prow[i]);
            double x[3] = {X[3 * i], X[3 * i + 1], X[3 * i + 2]};
            double v[9];
            for (int k = 0; k < 9; ++k) v[k] = V[9 * j + k];
            double rmin, rmax;
            tri_dist(x, v, rmin, rmax);
            if (i == j) rmin = 0.0;
            lag_window(rmin, rmax, d, gcap, g0, cnt);
            if (cnt == 0) g0 = 0;
            lc = max(lc, cnt);
            lg = max(lg, g0);
            if (cnt) lt = max(lt, g0 + cnt - 1);
            int cs = min(cnt, kMaxCnt), gs = min(g0, kMaxG0);
            meta[p] = (uint16_t)(gs | (cs << kG0Bits));
            cnt = cs;
        }
        int tot = __reduce_add_sync(0xffffffffu, cnt);
        if (lane == 0) btot[gb] = tot;
    }
    for (int o = 16; o; o >>= 1) {
        lc = max(lc, __shfl_xor_sync(0xffffffffu, lc, o));
        lg = max(lg, __shfl_xor_sync(0xffffffffu, lg, o));
        lt = max(lt, __shfl_xor_sync(0xffffffffu, lt, o));
    }
    if (lane == 0) {
        atomicMax(maxcnt, lc);
        atomicMax(maxg0, lg);
        atomicMax(gtop, lt);
    }
}

cudaError_t launch_windows(tdbem_ctx *c, int *d_maxcnt, int *d_maxg0, int *d_gtop)
{
    int64_t blocks = (c->nbt * 32 + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    if (blocks < 1) blocks = 1;
    k_windows<<<(int)blocks, 256, 0, c->s>>>(c->ns, c->P.d, c->P.nt - 1, c->d_prow, c->d_col, c->d_rowblk, c->nbt,
                                             c->d_X, c->d_V, c->d_meta, c->d_btot, d_maxcnt, d_maxg0, d_gtop);
    return cudaGetLastError();
}

// One warp per (32-pair block, window slot s): lane l computes the
// coefficient of its pair at lag g0 + s if s < cnt and stores it at the
// block's slot-major packed position.
__global__ void __launch_bounds__(128) k_coefficients(int ns, int smax, int kinds, int ku_kind, int kw_kind,
                                                      double cdt, const int64_t *__restrict__ prow,
                                                      const int32_t *__restrict__ col,
                                                      const int64_t *__restrict__ rowblk, int64_t nbt,
                                                      const double *__restrict__ X,
                                                      const double *__restrict__ nrm, const double *__restrict__ V,
                                                      const uint16_t *__restrict__ meta,
                                                      const int64_t *__restrict__ boff, double *ku, double *kw)
{
    int64_t nw = nbt * smax;
    int lane = threadIdx.x & 31;
    unsigned lt = (1u << lane) - 1u;
    for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; w < nw;
         w += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        int s = (int)(w % smax);
        int64_t gb = w / smax;
        int i = row_of_block(rowblk, ns, gb);
        int64_t p = prow[i] + (gb - rowblk[i]) * 32 + lane;
        bool valid = p < prow[i + 1];
        unsigned m = valid ? meta[p] : 0u;
        int g0 = m & kMaxG0, cnt = m >> kG0Bits;
        if (__reduce_max_sync(0xffffffffu, (unsigned)cnt) <= (unsigned)s) continue;
        int64_t pos = boff[gb];
        for (int q = 0; q < s; ++q) pos += __popc(__ballot_sync(0xffffffffu, cnt > q));
        unsigned mask = __ballot_sync(0xffffffffu, cnt > s);
        if (cnt <= s) continue;
        pos += __popc(mask & lt);
        int j = col ? col[p] : (int)(p - prow[i]);
        double x[3] = {X[3 * i], X[3 * i + 1], X[3 * i + 2]};
        double nx[3] = {nrm[3 * i], nrm[3 * i + 1], nrm[3 * i + 2]};
        double v[9];
        for (int k = 0; k < 9; ++k) v[k] = V[9 * j + k];
        double out[4];
        coef_set(c_bs, x, nx, v, (double)(g0 + s), i == j, kinds, cdt, out);
        if (ku) ku[pos] = out[ku_kind];
        if (kw) kw[pos] = out[kw_kind];
    }
}

cudaError_t launch_coefficients(tdbem_ctx *c)
{
    int kinds = 0;
    if (c->ku_kind >= 0) kinds |= 1 << c->ku_kind;
    if (c->kw_kind >= 0) kinds |= 1 << c->kw_kind;
    int64_t nw = c->nbt * c->smax;
    int64_t blocks = (nw * 32 + 127) / 128;
    if (blocks > 152 * 128) blocks = 152 * 128;
    if (blocks < 1) blocks = 1;
    k_coefficients<<<(int)blocks, 128, 0, c->s>>>(c->ns, c->smax, kinds, c->ku_kind, c->kw_kind, c->cdt, c->d_prow,
                                                  c->d_col, c->d_rowblk, c->nbt, c->d_X, c->d_n, c->d_V, c->d_meta,
                                                  c->d_boff, c->d_ku, c->d_kw);
    return cudaGetLastError();
}

// Zero-lag matrix of Eq. linear: A_ij = KU^(1)_ij (1 - phi_j) - KW^(1)_ij phi_j
// over the pairs whose window starts at lag 1.  One warp per row; the
// off-diagonal entries go to an ELL store [width][ns] (column -1 = empty),
// the diagonal to ainv = 1/A_ii.  With aoff == nullptr the kernel only
// counts: flag[1] = the widest row.  flag bit 1: row wider than the ELL
// store; bit 2: zero diagonal.
__global__ void k_zero_lag(int ns, int width, const int64_t *__restrict__ prow, const int32_t *__restrict__ col,
                           const int64_t *__restrict__ rowblk, const uint16_t *__restrict__ meta,
                           const int64_t *__restrict__ boff, const double *__restrict__ ku,
                           const double *__restrict__ kw, const int8_t *__restrict__ phi, double *aoff,
                           int32_t *acol, double *ainv, int *flag)
{
    int lane = threadIdx.x & 31;
    unsigned lt = (1u << lane) - 1u;
    int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= ns) return;
    int used = 0;
    double diag = 0.0;
    for (int64_t gb = rowblk[i]; gb < rowblk[i + 1]; ++gb) {
        int64_t p = prow[i] + (gb - rowblk[i]) * 32 + lane;
        bool valid = p < prow[i + 1];
        unsigned m = valid ? meta[p] : 0u;
        int j = valid ? (col ? col[p] : (int)(p - prow[i])) : -1;
        int g0 = m & kMaxG0, cnt = m >> kG0Bits;
        unsigned m0 = __ballot_sync(0xffffffffu, cnt > 0);
        bool hit = cnt > 0 && g0 == 1;
        unsigned mh = __ballot_sync(0xffffffffu, hit && j != i);
        double a = 0.0;
        if (hit && aoff) {
            int64_t pos = boff[gb] + __popc(m0 & lt);
            a = phi[j] ? (kw ? -kw[pos] : 0.0) : (ku ? ku[pos] : 0.0);
            if (j == i) {
                diag = a;
            } else {
                int slot = used + __popc(mh & lt);
                if (slot < width) {
                    aoff[(int64_t)slot * ns + i] = a;
                    acol[(int64_t)slot * ns + i] = j;
                } else {
                    atomicOr(flag, 2);
                }
            }
        }
        used += __popc(mh);
    }
    for (int o = 16; o; o >>= 1) diag += __shfl_xor_sync(0xffffffffu, diag, o);
    if (!aoff) {
        if (lane == 0) atomicMax(flag + 1, used);
        return;
    }
    if (lane == 0) {
        for (int s = used; s < width; ++s) {
            aoff[(int64_t)s * ns + i] = 0.0;
            acol[(int64_t)s * ns + i] = -1;
        }
        if (diag == 0.0) atomicOr(flag, 4);
        ainv[i] = 1.0 / diag;
    }
}

cudaError_t launch_zero_lag(tdbem_ctx *c, bool count_only)
{
    int blocks = (c->ns * 32 + 127) / 128;
    k_zero_lag<<<blocks, 128, 0, c->s>>>(c->ns, c->ell_w, c->d_prow, c->d_col, c->d_rowblk, c->d_meta, c->d_boff,
                                         c->d_ku, c->d_kw, c->d_phi, count_only ? nullptr : c->d_aoff, c->d_acol,
                                         c->d_ainv, c->d_flag);
    return cudaGetLastError();
}

// Known data to B-spline coefficients by collocation at t_a (one thread per
// element, marching in a): fbar^{a-1} = (f(t_a) - sum_{g=2..d} N(g) fbar^{a-g}) / N(1),
// written to the known component of the histories (u where phi = 0, q
// where phi = 1); the unknown components stay zero.
__global__ void k_known_collocation(int ns, int nt, const double *__restrict__ f, const int8_t *__restrict__ phi,
                                    double *u, double *q)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns) return;
    const int d = c_bs.d;
    double Ng[kMaxD + 2];
    for (int g = 0; g <= d + 1; ++g) Ng[g] = bs_N(c_bs, g, 0.0);  // N at the knot g (continuous)
    double *h = phi[i] ? q : u;
    for (int a = 1; a <= nt - 1; ++a) {
        double s = f[(int64_t)(a - 1) * ns + i];
        for (int g = 2; g <= d; ++g)
            if (a - g >= 0) s -= Ng[g] * h[(int64_t)(a - g) * ns + i];
        h[(int64_t)(a - 1) * ns + i] = s / Ng[1];
    }
}

cudaError_t launch_known_collocation(tdbem_ctx *c, const double *d_f)
{
    k_known_collocation<<<(c->ns + 127) / 128, 128, 0, c->s>>>(c->ns, c->P.nt, d_f, c->d_phi, c->d_u, c->d_q);
    return cudaGetLastError();
}

}  // namespace tdbem
