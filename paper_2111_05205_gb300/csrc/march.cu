// Per-step kernels of the time marching (Section 2.5, Eq. linear): the
// history sum that forms b^{a-1}, and the zero-lag solve A x^{a-1} = b^{a-1}.
#include "tdbem_internal.cuh"

namespace tdbem {

constexpr int kNearThreads = 128;
constexpr int kNearWarps = kNearThreads / 32;
constexpr int kNearMinBlocks = 10;  // split form: 48 registers, 40 resident warps per SM (measured best)
constexpr int kMaxFull = 4;         // full window slots handled by the unrolled bodies
constexpr int kNearPrefetch = 2;  // blocks of a warp whose coefficients are asked of L2 ahead

// Incident-wave term e_i(t_a) of the total-field equation: u_in (OBIE) or
// (d/dn_x - c^-1 d/dt) u_in (BMBIE) for the plane pulse
// u_in = f(t - t0 - k.x/c), f(s) = exp(-(s/width)^2).
__device__ __forceinline__ double incident_term(const Incident &in, const double *xc, const double *n, int alpha)
{
    double kx = in.k[0] * xc[0] + in.k[1] * xc[1] + in.k[2] * xc[2];
    double s = alpha * in.dt - in.t0 - kx / in.c;
    double f, df;
    if (in.shape == 0) {
        double a = s / in.width;
        f = exp(-a * a);
        df = -2.0 * a / in.width * f;
    } else {
        // raised cosine 0.5 (1 - cos(2 pi c s / width)) for 0 <= c s <= width
        // (Eq. uin with ct - x_1 = c s), zero elsewhere
        const double w = 2.0 * 3.14159265358979323846 * in.c / in.width, cs = in.c * s;
        const bool on = cs >= 0.0 && cs <= in.width;
        f = on ? 0.5 * (1.0 - cos(w * s)) : 0.0;
        df = on ? 0.5 * w * sin(w * s) : 0.0;
    }
    if (!in.bie) return f;
    double kn = in.k[0] * n[0] + in.k[1] * n[1] + in.k[2] * n[2];
    // d/dn_x f(t - k.x/c) = -(k.n/c) f';  c^-1 d/dt f = f'/c
    return -(1.0 + kn) / in.c * df;
}

// Double-float helpers of the split-precision history sum: a value v is
// held as (hi, lo) = (fl32(v), fl32(v - hi)), 48 significant bits; the
// product of two such values is formed exactly in its leading part
// (hi*hi and its FMA residual) plus the two cross terms, and added to a
// (hi, lo) accumulator by the two-sum of Knuth.  Relative error of one
// product ~2^-47, so the FP32 pipes (57x the FP64 rate on this GPU) carry
// an FP64-grade sum.
struct DF {
    float h, l;
};

__device__ __forceinline__ void df_fma(DF &acc, float ch, float cl, float xh, float xl)
{
    float ph = ch * xh;
    float pe = fmaf(ch, xh, -ph);
    pe = fmaf(ch, xl, pe);
    pe = fmaf(cl, xh, pe);
    float s = acc.h + ph;
    float bb = s - acc.h;
    float err = (acc.h - (s - bb)) + (ph - bb);
    acc.l += err + pe;
    acc.h = s;
}

__device__ __forceinline__ void df_renorm(DF &a)
{
    float s = a.h + a.l;
    a.l = a.l - (s - a.h);
    a.h = s;
}

// Element types of the history sum: FP64, or a float pair (hi, lo) in the
// same 8 bytes for the split form.
template <bool SPLIT>
struct NearV {
    using T = double;
};
template <>
struct NearV<true> {
    using T = float2;
};

template <bool SPLIT, bool NEG>
__device__ __forceinline__ void near_fma(DF &dacc, double &acc, const typename NearV<SPLIT>::T &c,
                                         const typename NearV<SPLIT>::T &x)
{
    if constexpr (SPLIT) {
        if (NEG)
            df_fma(dacc, -c.x, -c.y, x.x, x.y);
        else
            df_fma(dacc, c.x, c.y, x.x, x.y);
    } else {
        if (NEG)
            acc = fma(-c, x, acc);
        else
            acc = fma(c, x, acc);
    }
}

// One 32-pair block of a row: lane l holds pair (i, j_l) whose window is
// lags g0_l .. g0_l + cnt_l - 1.  Slot s of the block is stored packed (the
// lanes with cnt > s, in lane order) from offset o.  The N slots below the
// block's smallest count hold all 32 lanes, so lane l of slot s sits at
// o + 32 s + l; the first tail slot (s = N, lanes with cnt > N) is located
// by a ballot.  N is a template constant, so neither the full slots nor the
// loads carry a per-slot test, and the loads of all N + 1 slots are issued
// before any is used.  (In typical windows the counts of a block differ by
// at most one, so this covers every slot of nearly every block.)  In the
// early steps a lag can reach before the first step (beta < 0): the
// histories are allocated with as many zero rows before step 0 as the
// largest stored lag, so those terms read zeros and add nothing.
template <bool HU, bool HW, bool SPLIT, int N>
__device__ __forceinline__ void near_slots(const typename NearV<SPLIT>::T *__restrict__ kub,
                                           const typename NearV<SPLIT>::T *__restrict__ kwb,
                                           const typename NearV<SPLIT>::T *__restrict__ hqb,
                                           const typename NearV<SPLIT>::T *__restrict__ hub, int ns, int lane,
                                           unsigned lt, int cnt, bool tail, DF &dacc, double &acc)
{
    using V = typename NearV<SPLIT>::T;
    V cu[N + 1], xu[N + 1], cw[N + 1], xw[N + 1];
#pragma unroll
    for (int s = 0; s < N; ++s) {
        if (HU) {
            cu[s] = __ldcs(kub + 32 * s + lane);
            xu[s] = *(hqb - (int64_t)s * ns);
        }
        if (HW) {
            cw[s] = __ldcs(kwb + 32 * s + lane);
            xw[s] = *(hub - (int64_t)s * ns);
        }
    }
    bool on = false;
    if (tail) {  // warp-uniform
        const unsigned mask = __ballot_sync(0xffffffffu, cnt > N);
        on = cnt > N;
        if (on) {
            const int idx = 32 * N + __popc(mask & lt);
            if (HU) {
                cu[N] = __ldcs(kub + idx);
                xu[N] = *(hqb - (int64_t)N * ns);
            }
            if (HW) {
                cw[N] = __ldcs(kwb + idx);
                xw[N] = *(hub - (int64_t)N * ns);
            }
        }
    }
#pragma unroll
    for (int s = 0; s < N; ++s) {
        if (HU) near_fma<SPLIT, true>(dacc, acc, cu[s], xu[s]);
        if (HW) near_fma<SPLIT, false>(dacc, acc, cw[s], xw[s]);
    }
    if (on) {
        if (HU) near_fma<SPLIT, true>(dacc, acc, cu[N], xu[N]);
        if (HW) near_fma<SPLIT, false>(dacc, acc, cw[N], xw[N]);
    }
}

// Slots s0 <= s < cmax of a block, one at a time, each located by a ballot
// (blocks whose counts differ by more than one, or exceed the unrolled
// range).
template <bool HU, bool HW, bool SPLIT>
__device__ __forceinline__ void near_slots_rest(const typename NearV<SPLIT>::T *__restrict__ kub,
                                             const typename NearV<SPLIT>::T *__restrict__ kwb,
                                             const typename NearV<SPLIT>::T *__restrict__ hqb,
                                             const typename NearV<SPLIT>::T *__restrict__ hub, int ns, int lane,
                                             unsigned lt, int cnt, int s0, int cmin, int cmax, DF &dacc,
                                             double &acc)
{
    using V = typename NearV<SPLIT>::T;
    // offset of slot s0: full slots hold 32 entries, tail slots their lanes
    int pos = 32 * min(s0, cmin);
    for (int s = cmin; s < s0; ++s) pos += __popc(__ballot_sync(0xffffffffu, cnt > s));
    for (int s = s0; s < cmax; ++s) {
        const unsigned mask = __ballot_sync(0xffffffffu, cnt > s);
        if (cnt > s) {
            const int idx = pos + __popc(mask & lt);
            const int64_t h = (int64_t)s * ns;
            if (HU) near_fma<SPLIT, true>(dacc, acc, __ldcs(kub + idx), *(hqb - h));
            if (HW) near_fma<SPLIT, false>(dacc, acc, __ldcs(kwb + idx), *(hub - h));
        }
        pos += __popc(mask);
    }
}

template <bool HU, bool HW, bool SPLIT>
__device__ __forceinline__ void near_block(const typename NearV<SPLIT>::T *__restrict__ kub,
                                           const typename NearV<SPLIT>::T *__restrict__ kwb,
                                           const typename NearV<SPLIT>::T *__restrict__ hqb,
                                           const typename NearV<SPLIT>::T *__restrict__ hub, int cnt, int ns,
                                           int lane, unsigned lt, DF &dacc, double &acc)
{
    const int cmin = (int)__reduce_min_sync(0xffffffffu, (unsigned)cnt);
    const int cmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)cnt);
    const bool tail = cmax > cmin;
    // both kinds at once keep twice the values per slot in registers
    constexpr int MF = (HU && HW) ? kMaxFull / 2 : kMaxFull;
    const int nf = cmin < MF ? cmin : MF;
#define TDBEM_NEAR_CASE(n)                                                                                     \
    case n:                                                                                                    \
        if constexpr (n <= MF) near_slots<HU, HW, SPLIT, n>(kub, kwb, hqb, hub, ns, lane, lt, cnt, tail, dacc, acc); \
        break;
    switch (nf) {  // warp-uniform
        TDBEM_NEAR_CASE(0)
        TDBEM_NEAR_CASE(1)
        TDBEM_NEAR_CASE(2)
        TDBEM_NEAR_CASE(3)
        TDBEM_NEAR_CASE(4)
        TDBEM_NEAR_CASE(5)
        TDBEM_NEAR_CASE(6)
    }
#undef TDBEM_NEAR_CASE
    // slots the unrolled bodies did not reach
    const int done = nf + (tail ? 1 : 0);
    if (done < cmax)
        near_slots_rest<HU, HW, SPLIT>(kub, kwb, hqb, hub, ns, lane, lt, cnt, done, cmin, cmax, dacc, acc);
}

// Asks L2 to fetch the coefficient bytes [a, e) of a block ahead of its
// use, so the warp's own loads wait for an L2 hit rather than HBM: lane l
// names the l-th 128-byte line of the range (a block spans at most 31).
// (One bulk prefetch per block through the copy engine measured slower.)
__device__ __forceinline__ void near_prefetch(const double *k, int64_t a, int64_t e, int lane)
{
    const size_t end = __cvta_generic_to_global(k + e);
    const size_t p = (__cvta_generic_to_global(k + a) & ~(size_t)127) + 128 * (size_t)lane;
    if (p < end) asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

template <bool HU, bool HW, bool SPLIT, int WPR, bool COL>
__device__ __forceinline__ void near_row(int i, int wr, int ns, int alpha, const int64_t *__restrict__ prow,
                                         const int32_t *__restrict__ crow, const int64_t *__restrict__ rowblk,
                                         const uint16_t *__restrict__ meta, const int64_t *__restrict__ boff,
                                         const double *__restrict__ ku, const double *__restrict__ kw,
                                         const double *__restrict__ u_, const double *__restrict__ q,
                                         const float2 *__restrict__ us, const float2 *__restrict__ qs, DF &dacc,
                                         double &acc)
{
    using V = typename NearV<SPLIT>::T;
    constexpr int W = WPR;  // the row's warps take its blocks in turn
    const V *hq, *hu;
    if constexpr (SPLIT) {
        hq = qs;
        hu = us;
    } else {
        hq = q;
        hu = u_;
    }
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t p0 = prow[i];
    const int npr = (int)(prow[i + 1] - p0);
    const uint16_t *mrow = meta + p0;
    const int64_t *orow = boff + rowblk[i];
    const int nblk = (int)(rowblk[i + 1] - rowblk[i]);
    const V *kuv = reinterpret_cast<const V *>(ku);
    const V *kwv = reinterpret_cast<const V *>(kw);
    // the warp asks L2 for the coefficients of its block kNearPrefetch blocks
    // ahead (here: of its first kNearPrefetch blocks)
    for (int t = 0; t < kNearPrefetch; ++t) {
        const int pb = wr + W * t;
        if (pb < nblk) {
            if (HU) near_prefetch(ku, orow[pb], orow[pb + 1], lane);
            if (HW) near_prefetch(kw, orow[pb], orow[pb + 1], lane);
        }
    }
    // metadata and columns of the first block; the next block's are fetched
    // while the current one is summed
    int bk = wr;
    unsigned mnext = 0u;
    int64_t onext = 0;
    int jnext = 0;
    if (bk < nblk) {
        const int pr = bk * 32 + lane;
        mnext = (pr < npr) ? mrow[pr] : 0u;
        if constexpr (COL) jnext = (pr < npr) ? crow[pr] : 0;
        onext = orow[bk];
    }
    for (; bk < nblk; bk += W) {
        {
            const int pb = bk + W * kNearPrefetch;
            if (pb < nblk) {
                if (HU) near_prefetch(ku, orow[pb], orow[pb + 1], lane);
                if (HW) near_prefetch(kw, orow[pb], orow[pb + 1], lane);
            }
        }
        const int j = COL ? jnext : ((bk * 32 + lane < npr) ? bk * 32 + lane : 0);
        const unsigned m = mnext;
        const int64_t o = onext;
        const int nb = bk + W;
        if (nb < nblk) {
            const int pn = nb * 32 + lane;
            mnext = (pn < npr) ? mrow[pn] : 0u;
            if constexpr (COL) jnext = (pn < npr) ? crow[pn] : 0;
            onext = orow[nb];
        }
        // cnt = 0 past the row's end; lag g = g0 + s reaches back to
        // beta = alpha - g0 - s
        const int g0 = (int)(m & kMaxG0), cnt = (int)(m >> kG0Bits);
        const int64_t hb = (int64_t)(alpha - g0) * ns + j;
        near_block<HU, HW, SPLIT>(kuv + o, kwv + o, hq + hb, hu + hb, cnt, ns, lane, lt, dacc, acc);
        if (SPLIT) df_renorm(dacc);
    }
}

// b_i = -e_i - sum_j sum_{g in window(i,j), g <= a} (KU^(g)_ij q_j^{a-g} - KW^(g)_ij u_j^{a-g})
// WPR warps per row i (4: the CTA's warps share the row's 32-pair blocks in
// turn; 1: four rows per CTA); COL: the rows carry explicit columns (near
// lists: the list of the row's leaf cell, col + coff[e2c[i]], shared by all
// rows of the cell; rows taken in the octree's sorted order rowperm, so
// that the rows of a cell run together and find the cell's columns and the
// neighbours' histories in cache), else the column is the pair index (all
// pairs).  Every load of the
// coefficient stream is a contiguous warp access, and the history entries
// x_j^{a-g} of one slot differ only by the lanes' g0.  The row sum is
// reduced in a fixed order (deterministic).
// SPLIT = false: FP64 coefficients and FP64 FMA.  SPLIT = true: each
// coefficient is a float pair (hi, lo) in the same 8 bytes, the histories
// are read from their float-pair copies and the sum runs in double-float.
template <bool HU, bool HW, bool SPLIT, int WPR, bool COL>
__global__ void __launch_bounds__(kNearThreads, SPLIT ? kNearMinBlocks : 8) k_near_sum(int ns, int alpha, const int *__restrict__ alpha_dev,
                                                              const int64_t *__restrict__ prow,
                                                              const int32_t *__restrict__ col,
                                                              const int64_t *__restrict__ coff,
                                                              const int32_t *__restrict__ e2c,
                                                              const int32_t *__restrict__ rowperm,
                                                              const int64_t *__restrict__ rowblk,
                                                              const uint16_t *__restrict__ meta,
                                                              const int64_t *__restrict__ boff,
                                                              const double *__restrict__ ku,
                                                              const double *__restrict__ kw,
                                                              const double *__restrict__ u_,
                                                              const double *__restrict__ q,
                                                              const float2 *__restrict__ us,
                                                              const float2 *__restrict__ qs,
                                                              const double *__restrict__ exc, Incident inc,
                                                              const double *__restrict__ xc,
                                                              const double *__restrict__ nrm,
                                                              const double *__restrict__ far, int far_lt, int alim,
                                                              double *b)
{
    __shared__ double red[kNearWarps];
    if (alpha_dev) {
        // graph-replayed steps: an instance past its last step (alim = Nt-1)
        // does nothing while the others of its batch go on (whole CTA)
        alpha = *alpha_dev;
        if (alpha > alim) return;
    }
    // WPR warps per row, kNearWarps / WPR rows per CTA
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.x * (kNearWarps / WPR) + warp / WPR, wr = warp % WPR;
    const int i = (COL && r < ns) ? rowperm[r] : r;
    double acc = 0.0;
    DF dacc = {0.f, 0.f};
    if (i < ns) {
        const int32_t *crow = COL ? col + coff[e2c[i]] : nullptr;
        near_row<HU, HW, SPLIT, WPR, COL>(i, wr, ns, alpha, prow, crow, rowblk, meta, boff, ku, kw, u_, q, us, qs,
                                          dacc, acc);
    }
    if (SPLIT) acc = (double)dacc.h + (double)dacc.l;
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (lane == 0 && wr == 0 && i < ns) {
        double t = 0.0;
        for (int w = 0; w < WPR; ++w) t += red[warp + w];
        double e = 0.0;
        if (exc)
            e = exc[i];
        else if (inc.on)
            e = incident_term(inc, xc + 3 * i, nrm + 3 * i, alpha);
        // far field of the step: far[(alpha - 1) % Lt] when the kernel reads
        // the step from the device (far_lt = Lt), else already offset
        if (far) e += far[(far_lt ? (int64_t)((alpha - 1) % far_lt) * ns : 0) + i];
        b[i] = t - e;
    }
}

template <bool SPLIT, int WPR, bool COL>
static cudaError_t near_dispatch(tdbem_ctx *c, int alpha, const double *d_exc, const double *d_far)
{
    bool hu = c->d_ku != nullptr, hw = c->d_kw != nullptr;
    auto k = hu ? (hw ? k_near_sum<true, true, SPLIT, WPR, COL> : k_near_sum<true, false, SPLIT, WPR, COL>)
                : (hw ? k_near_sum<false, true, SPLIT, WPR, COL> : k_near_sum<false, false, SPLIT, WPR, COL>);
    constexpr int rows = kNearWarps / WPR;
    // the kernel uses a pair's column only to address the history: in the
    // split form with near lists that is the column's sorted position
    const int32_t *hcol = COL ? ((SPLIT && c->d_chcol) ? c->d_chcol : c->d_ccol) : nullptr;
    k<<<(c->ns + rows - 1) / rows, kNearThreads, 0, c->s>>>(c->ns, alpha, c->alpha_dev_on ? c->d_alpha : nullptr, c->d_prow, hcol,
                                       COL ? c->d_coff : nullptr, COL ? c->tree.e2c : nullptr,
                                       COL ? c->tree.perm : nullptr, c->d_rowblk, c->d_meta, c->d_boff,
                                       c->d_ku, c->d_kw, c->d_u, c->d_q, c->d_us, c->d_qs, d_exc, c->inc, c->d_xc,
                                       c->d_n, d_far, c->alpha_dev_on && d_far ? c->fmm.Lt : 0, c->P.nt - 1, c->d_b);
    return cudaGetLastError();
}

cudaError_t launch_near_sum(tdbem_ctx *c, int alpha, const double *d_exc, const double *d_far)
{
    // all pairs (no column list): long rows, four warps each
    if (!c->d_col)
        return c->split ? near_dispatch<true, kNearWarps, false>(c, alpha, d_exc, d_far)
                        : near_dispatch<false, kNearWarps, false>(c, alpha, d_exc, d_far);
    if (c->near_wpr == 1)
        return c->split ? near_dispatch<true, 1, true>(c, alpha, d_exc, d_far)
                        : near_dispatch<false, 1, true>(c, alpha, d_exc, d_far);
    return c->split ? near_dispatch<true, kNearWarps, true>(c, alpha, d_exc, d_far)
                    : near_dispatch<false, kNearWarps, true>(c, alpha, d_exc, d_far);
}

__device__ __forceinline__ float2 split2(double v)
{
    float h = __double2float_rn(v);
    return make_float2(h, __double2float_rn(v - (double)h));
}

// In-place conversion of FP64 values to (hi, lo) float pairs.
__global__ void k_split_inplace(int64_t n, double *v)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        double x = v[k];
        reinterpret_cast<float2 *>(v)[k] = split2(x);
    }
}

// Float-pair copies of FP64 values.
// out = the float-pair copy of v ([nt][ns]); with hpos, element i of a
// step goes to position hpos[i] of that step's row.
__global__ void k_split_copy(int64_t n, int ns, const double *__restrict__ v, const int32_t *__restrict__ hpos,
                             float2 *out)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = k % ns;
        out[hpos ? k - i + hpos[i] : k] = split2(v[k]);
    }
}

cudaError_t launch_split_coefficients(tdbem_ctx *c)
{
    if (c->d_ku) k_split_inplace<<<152 * 16, 256, 0, c->s>>>(c->ncoef, c->d_ku);
    if (c->d_kw) k_split_inplace<<<152 * 16, 256, 0, c->s>>>(c->ncoef, c->d_kw);
    return cudaGetLastError();
}

cudaError_t launch_split_histories(tdbem_ctx *c)
{
    int64_t n = (int64_t)c->P.nt * c->ns;
    k_split_copy<<<152 * 16, 256, 0, c->s>>>(n, c->ns, c->d_u, c->d_hpos, c->d_us);
    k_split_copy<<<152 * 16, 256, 0, c->s>>>(n, c->ns, c->d_q, c->d_hpos, c->d_qs);
    return cudaGetLastError();
}

// One row of a Jacobi sweep x' = D^-1 (b - R x) of the zero-lag system
// (A = D + R, R in the ELL store); xin = nullptr starts from x = D^-1 b.
// LDX loads an entry of x (the fused kernel reads past L2 coherence points).
// Shared by the one-sweep and the fused kernels, so both give the same bits.
template <typename LDX>
__device__ __forceinline__ double jacobi_row(int i, int ns, int width, const double *__restrict__ aoff,
                                             const int32_t *__restrict__ acol, const double *__restrict__ ainv,
                                             const double *__restrict__ b, const double *xin, LDX ldx)
{
    double s = b[i];
    if (xin) {
        // four entries at a time: their columns and values first, then the
        // four gathers of x, so that the loads of a group are in flight together
        int k = 0;
        for (; k + 4 <= width; k += 4) {
            int cidx[4];
            double a[4], xv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                cidx[u] = acol[(int64_t)(k + u) * ns + i];
                a[u] = aoff[(int64_t)(k + u) * ns + i];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) xv[u] = cidx[u] >= 0 ? ldx(xin + cidx[u]) : 0.0;
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (cidx[u] >= 0) s -= a[u] * xv[u];
        }
        for (; k < width; ++k) {
            int cidx = acol[(int64_t)k * ns + i];
            if (cidx >= 0) s -= aoff[(int64_t)k * ns + i] * ldx(xin + cidx);
        }
    }
    return s * ainv[i];
}

// The last sweep adds the solution to the unknown component of step a-1 (u
// where phi = 1, q where phi = 0) and flags a non-finite value (flag bit 1).
// The float-pair copy holds element i at position hpos[i] (identity when
// hpos is null).
__device__ __forceinline__ void jacobi_store(int i, double x, int64_t row, const int8_t *__restrict__ phi, double *u,
                                             double *q, float2 *us, float2 *qs, const int32_t *__restrict__ hpos,
                                             int *flag)
{
    double *h = phi[i] ? u : q;
    double v = h[row + i] + x;
    h[row + i] = v;
    if (us) (phi[i] ? us : qs)[row + (hpos ? hpos[i] : i)] = split2(v);
    if (!isfinite(x)) atomicOr(flag, 1);
}

// One Jacobi sweep; it = 0 starts from x = D^-1 b, the last one stores.
__global__ void k_jacobi(int ns, int width, const double *__restrict__ aoff, const int32_t *__restrict__ acol,
                         const double *__restrict__ ainv, const double *__restrict__ b,
                         const double *__restrict__ xin, double *xout, int last, int64_t row,
                         const int *__restrict__ alpha_dev, const int8_t *__restrict__ phi, double *u, double *q,
                         float2 *us, float2 *qs, const int32_t *__restrict__ hpos, int alim, int *flag)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns) return;
    if (alpha_dev) {
        const int a = *alpha_dev;
        if (a > alim) return;  // instance past its last step
        row = (int64_t)(a - 1) * ns;
    }
    const double x = jacobi_row(i, ns, width, aoff, acol, ainv, b, xin, [](const double *p) { return *p; });
    if (last)
        jacobi_store(i, x, row, phi, u, q, us, qs, hpos, flag);
    else
        xout[i] = x;
}

// All K sweeps of one step in one cooperative launch (rows grid-strided),
// with a grid barrier between sweeps; the same ping-pong buffers and row
// arithmetic as K launches of k_jacobi.  x is read with ld.global.cg: a CTA
// must not see an earlier sweep's value from its own L1.
__global__ void __launch_bounds__(256) k_jacobi_fused(int ns, int width, const double *__restrict__ aoff,
                                                      const int32_t *__restrict__ acol,
                                                      const double *__restrict__ ainv, const double *__restrict__ b,
                                                      double *xa, double *xb, int K, int64_t row,
                                                      const int8_t *__restrict__ phi, double *u, double *q,
                                                      float2 *us, float2 *qs, const int32_t *__restrict__ hpos,
                                                      int *flag, unsigned *bar)
{
    for (int it = 0; it < K; ++it) {
        const double *xin = (it == 0) ? nullptr : ((it & 1) ? xa : xb);
        double *xout = (it & 1) ? xb : xa;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += gridDim.x * blockDim.x) {
            const double x = jacobi_row(i, ns, width, aoff, acol, ainv, b, xin, [](const double *p) { return __ldcg(p); });
            if (it == K - 1)
                jacobi_store(i, x, row, phi, u, q, us, qs, hpos, flag);
            else
                xout[i] = x;
        }
        if (it < K - 1) grid_barrier(bar, flag);
    }
}

// Three grid barriers in a row (the probe of the bounded wait below).
__global__ void k_barrier_probe(unsigned *bar, int *flag, int rounds)
{
    for (int r = 0; r < rounds; ++r) grid_barrier(bar, flag);
}

cudaError_t setup_jacobi_fused(tdbem_ctx *c)
{
    c->jac_grid = 0;
    int coop = 0, nsm = 0, per = 0;
    cudaError_t e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_jacobi_fused, 256, 0);
    if (e != cudaSuccess) return e;
    if (!coop || per < 1 || !c->d_bar) return cudaSuccess;  // K one-sweep launches instead
    e = cudaMemsetAsync(c->d_bar, 0, 2 * sizeof(unsigned), c->s);
    if (e != cudaSuccess) return e;
    c->jac_grid = (int)std::min<int64_t>(((int64_t)c->ns + 255) / 256, (int64_t)per * nsm);
    return cudaSuccess;
}

cudaError_t launch_jacobi_fused(tdbem_ctx *c, int alpha)
{
    int ns = c->ns, width = c->ell_w, K = c->solve_iters;
    int64_t row = (int64_t)(alpha - 1) * c->ns;
    void *args[] = {&ns, &width, &c->d_aoff, &c->d_acol, &c->d_ainv, &c->d_b, &c->d_xa, &c->d_xb, &K, &row,
                    &c->d_phi, &c->d_u, &c->d_q, &c->d_us, &c->d_qs, &c->d_hpos, &c->d_flag, &c->d_bar};
    return cudaLaunchCooperativeKernel((const void *)k_jacobi_fused, dim3(c->jac_grid), dim3(256), args, 0, c->s);
}

cudaError_t launch_jacobi(tdbem_ctx *c, int alpha, int it, int last)
{
    const double *xin = (it == 0) ? nullptr : ((it & 1) ? c->d_xa : c->d_xb);
    double *xout = (it & 1) ? c->d_xb : c->d_xa;
    int64_t row = (int64_t)(alpha - 1) * c->ns;
    k_jacobi<<<(c->ns + 127) / 128, 128, 0, c->s>>>(c->ns, c->ell_w, c->d_aoff, c->d_acol, c->d_ainv, c->d_b, xin, xout, last,
                                                   row, c->alpha_dev_on ? c->d_alpha : nullptr, c->d_phi, c->d_u,
                                                   c->d_q, c->d_us, c->d_qs, c->d_hpos, c->P.nt - 1, c->d_flag);
    return cudaGetLastError();
}

// Advances the device-side step counter (graph-replayed steps), stopping
// one past the last step alim = Nt-1.
__global__ void k_alpha_next(int *alpha_dev, int alim)
{
    if (*alpha_dev <= alim) *alpha_dev += 1;
}

cudaError_t launch_alpha_next(tdbem_ctx *c)
{
    k_alpha_next<<<1, 1, 0, c->s>>>(c->d_alpha, c->P.nt - 1);
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

extern "C" int tdbem_grid_barrier_probe(int32_t nblocks, int32_t starve, int32_t *timed_out)
{
    using namespace tdbem;
    if (nblocks < 1 || !timed_out) return TDBEM_ERR_ARG;
    *timed_out = 0;
    unsigned *bar = nullptr;
    int *flag = nullptr;
    cudaError_t e = cudaMalloc(&bar, 2 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&flag, sizeof(int));
    // starve: an arrival count no CTA can complete, so every wait runs out
    const unsigned init[2] = {starve ? 0x80000000u : 0u, 0u};
    if (e == cudaSuccess) e = cudaMemcpy(bar, init, sizeof(init), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(flag, 0, sizeof(int));
    int rounds = 3;
    void *args[] = {&bar, &flag, &rounds};
    if (e == cudaSuccess) e = cudaLaunchCooperativeKernel((const void *)k_barrier_probe, dim3(nblocks), dim3(32), args, 0, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int f = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&f, flag, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(bar);
    cudaFree(flag);
    if (e != cudaSuccess) return TDBEM_ERR_CUDA;
    *timed_out = (f & 4) ? 1 : 0;
    return TDBEM_OK;
}
