// C ABI of libtdbem: context life cycle, setup (tdbem_prepare) and the
// time-marching driver (Section 2.5, Eq. linear).
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>

#include "tdbem_internal.cuh"

using namespace tdbem;

namespace {

int fail(tdbem_ctx *c, int code, const std::string &msg)
{
    if (c) c->err = msg;
    return code;
}

#define TD_CUDA(call)                                                                                    \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess)                                                                           \
            return fail(c, e_ == cudaErrorMemoryAllocation ? TDBEM_ERR_OOM : TDBEM_ERR_CUDA,             \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                           \
    } while (0)

template <typename T>
cudaError_t dalloc(tdbem_ctx *c, T **p, size_t n)
{
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, n * sizeof(T) > 0 ? n * sizeof(T) : 16);
    if (e == cudaSuccess) {
        c->allocs.push_back(q);
        *p = (T *)q;
    }
    return e;
}

void dfree(tdbem_ctx *c, void *p)
{
    if (!p) return;
    auto it = std::find(c->allocs.begin(), c->allocs.end(), p);
    if (it != c->allocs.end()) c->allocs.erase(it);
    cudaFree(p);
}

// Orders the context's stream after the user's stream (call entry) and the
// user's stream after the context's stream (call exit).
cudaError_t join(cudaStream_t from, cudaStream_t to)
{
    cudaEvent_t e;
    cudaError_t r = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    if (r != cudaSuccess) return r;
    r = cudaEventRecord(e, from);
    if (r == cudaSuccess) r = cudaStreamWaitEvent(to, e, 0);
    cudaEventDestroy(e);
    return r;
}

cudaEvent_t take_event(tdbem_ctx *c)
{
    if (!c->pool.empty()) {
        cudaEvent_t e = c->pool.back();
        c->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Accumulates the elapsed times of all recorded phase intervals (waits for
// them).
void harvest(tdbem_ctx *c)
{
    for (auto &p : c->pending) {
        cudaEventSynchronize(p.b);
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) c->ms[p.phase] += ms;
        c->pool.push_back(p.a);
        c->pool.push_back(p.b);
    }
    c->pending.clear();
}

struct PhaseTimer {
    tdbem_ctx *c;
    int phase;
    cudaEvent_t a;
    PhaseTimer(tdbem_ctx *c_, int ph) : c(c_), phase(ph)
    {
        if (c->pending.size() > 8192) harvest(c);
        a = take_event(c);
        cudaEventRecord(a, c->s);
    }
    ~PhaseTimer()
    {
        cudaEvent_t b = take_event(c);
        cudaEventRecord(b, c->s);
        c->pending.push_back({phase, a, b});
    }
};

}  // namespace

void tdbem::phase_begin(tdbem_ctx *c, cudaEvent_t *e)
{
    if (c->pending.size() > 8192) harvest(c);
    *e = take_event(c);
    cudaEventRecord(*e, c->s);
}

void tdbem::phase_end(tdbem_ctx *c, int phase, cudaEvent_t a)
{
    cudaEvent_t b = take_event(c);
    cudaEventRecord(b, c->s);
    c->pending.push_back({phase, a, b});
}

namespace {

int check_flags(tdbem_ctx *c)
{
    int f = 0;
    TD_CUDA(cudaMemcpy(&f, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (f & 1) return fail(c, TDBEM_ERR_DIVERGED, "non-finite solution value (divergence guard)");
    if (f & 8) return fail(c, TDBEM_ERR_TIMEOUT, "M2L tensor-core GEMM: a pipeline wait timed out");
    if (f & 4) {
        // a grid barrier of the fused solve gave up waiting: reset it and
        // solve with one launch per sweep from now on
        cudaMemset(c->d_bar, 0, 2 * sizeof(unsigned));
        c->jac_grid = 0;
        c->sai_grid = 0;
        return fail(c, TDBEM_ERR_TIMEOUT, "zero-lag solve: grid barrier timed out");
    }
    return TDBEM_OK;
}

}  // namespace

extern "C" {

int tdbem_create(const tdbem_params *p, void *stream, tdbem_ctx **out)
{
    tdbem_ctx *c = nullptr;
    if (!p || !out) return TDBEM_ERR_ARG;
    *out = nullptr;
    if (!(p->c > 0) || !(p->dt > 0) || p->nt < 2 || p->d < 1 || p->d > kMaxD || (p->bie != 0 && p->bie != 1) ||
        (p->algo != 0 && p->algo != 1) || p->precision < 0 || p->precision > 5 || (p->precond != 0 && p->precond != 1))
        return TDBEM_ERR_ARG;
    c = new tdbem_ctx();
    c->P = *p;
    c->cdt = p->c * p->dt;
    c->split = (p->precision >= 1);
    c->user = (cudaStream_t)stream;
    cudaGetDevice(&c->dev);
    // the context's stream at the highest priority: the deferred far-field
    // work of the FMM runs on a lower-priority second stream, and the block
    // scheduler then serves the per-step kernels first
    int lo_prio = 0, hi_prio = 0;
    cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
    if (cudaStreamCreateWithPriority(&c->s, cudaStreamNonBlocking, hi_prio) != cudaSuccess) {
        delete c;
        return TDBEM_ERR_CUDA;
    }
    bspline_table(p->d, &c->bs);
    c->inc.on = 0;
    c->inc.bie = p->bie;
    c->inc.c = p->c;
    c->inc.dt = p->dt;
    if (dalloc(c, &c->d_flag, 4) != cudaSuccess) {
        tdbem_destroy(c);
        return TDBEM_ERR_OOM;
    }
    cudaMemset(c->d_flag, 0, 4 * sizeof(int));
    *out = c;
    return TDBEM_OK;
}

void tdbem_destroy(tdbem_ctx *c)
{
    if (!c) return;
    if (c->s) cudaStreamSynchronize(c->s);
    harvest(c);
    for (auto e : c->pool) cudaEventDestroy(e);
    if (c->graph) cudaGraphExecDestroy(c->graph);
    for (void *p : c->allocs) cudaFree(p);
    free_tree(c);
    fmm_free(c);
    if (c->s) cudaStreamDestroy(c->s);
    delete c;
}

const char *tdbem_last_error(const tdbem_ctx *c)
{
    if (!c) return "null context";
    return c->err.c_str();
}

int tdbem_set_mesh(tdbem_ctx *c, const double *xyz, int32_t nv, const int32_t *tri, int32_t ns)
{
    if (!c) return TDBEM_ERR_ARG;
    if (c->prepared) return fail(c, TDBEM_ERR_STATE, "mesh set after prepare");
    if (!xyz || !tri || nv < 3 || ns < 1) return fail(c, TDBEM_ERR_ARG, "empty mesh");
    for (int64_t k = 0; k < 3 * (int64_t)ns; ++k)
        if (tri[k] < 0 || tri[k] >= nv) return fail(c, TDBEM_ERR_ARG, "triangle vertex index out of range");
    for (int i = 0; i < ns; ++i) {
        const double *a = xyz + 3 * tri[3 * i], *b = xyz + 3 * tri[3 * i + 1], *d = xyz + 3 * tri[3 * i + 2];
        double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, e2[3] = {d[0] - a[0], d[1] - a[1], d[2] - a[2]};
        double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        double l1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
        double l2 = sqrt(e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2]);
        if (!(sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]) > 1e-12 * l1 * l2))
            return fail(c, TDBEM_ERR_ARG, "degenerate triangle " + std::to_string(i));
    }
    c->nv = nv;
    c->ns = ns;
    c->xyz.assign(xyz, xyz + 3 * (int64_t)nv);
    c->tri.assign(tri, tri + 3 * (int64_t)ns);
    c->phi.assign(ns, 0);
    c->kbar.clear();
    return TDBEM_OK;
}

int tdbem_set_bc(tdbem_ctx *c, const int8_t *phi)
{
    if (!c || !phi) return TDBEM_ERR_ARG;
    if (c->prepared) return fail(c, TDBEM_ERR_STATE, "bc set after prepare");
    if (c->ns == 0) return fail(c, TDBEM_ERR_STATE, "bc before mesh");
    for (int i = 0; i < c->ns; ++i)
        if (phi[i] != 0 && phi[i] != 1) return fail(c, TDBEM_ERR_ARG, "phi must be 0 or 1");
    c->phi.assign(phi, phi + c->ns);
    return TDBEM_OK;
}

int tdbem_set_known(tdbem_ctx *c, const double *f)
{
    if (!c) return TDBEM_ERR_ARG;
    if (c->prepared) return fail(c, TDBEM_ERR_STATE, "known data set after prepare");
    if (c->ns == 0) return fail(c, TDBEM_ERR_STATE, "known data before mesh");
    if (!f) {
        c->kbar.clear();
        return TDBEM_OK;
    }
    int64_t n = (int64_t)(c->P.nt - 1) * c->ns;
    for (int64_t k = 0; k < n; ++k)
        if (!isfinite(f[k])) return fail(c, TDBEM_ERR_ARG, "non-finite known data");
    c->kbar.assign(f, f + n);
    return TDBEM_OK;
}

int tdbem_set_incident_plane(tdbem_ctx *c, const double dir[3], double t0, double width, int32_t shape)
{
    if (!c || !dir) return TDBEM_ERR_ARG;
    if (shape != 0 && shape != 1) return fail(c, TDBEM_ERR_ARG, "shape must be 0 (Gaussian) or 1 (raised cosine)");
    double l = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
    if (!(l > 0) || !(width > 0)) return fail(c, TDBEM_ERR_ARG, "bad direction or width");
    c->inc.on = 1;
    for (int k = 0; k < 3; ++k) c->inc.k[k] = dir[k] / l;
    c->inc.t0 = t0;
    c->inc.width = width;
    c->inc.shape = shape;
    return TDBEM_OK;
}

// Steps 0..Nt-1 of the histories back to their state before the first step:
// the known data (collocated, Eq. linear) and zero unknown components, and
// the float-pair copies of the split form.
static int reset_histories(tdbem_ctx *c)
{
    const int nt = c->P.nt, ns = c->ns;
    const size_t nh = (size_t)nt * ns;
    TD_CUDA(cudaMemsetAsync(c->d_u, 0, nh * sizeof(double), c->s));
    TD_CUDA(cudaMemsetAsync(c->d_q, 0, nh * sizeof(double), c->s));
    if (!c->kbar.empty()) {
        double *d_f = nullptr;
        TD_CUDA(dalloc(c, &d_f, (size_t)(nt - 1) * ns));
        TD_CUDA(cudaMemcpyAsync(d_f, c->kbar.data(), (size_t)(nt - 1) * ns * sizeof(double),
                                cudaMemcpyHostToDevice, c->s));
        TD_CUDA(launch_known_collocation(c, d_f));
        TD_CUDA(cudaStreamSynchronize(c->s));
        dfree(c, d_f);
    }
    if (c->split) TD_CUDA(launch_split_histories(c));
    return TDBEM_OK;
}

int tdbem_prepare(tdbem_ctx *c)
{
    if (!c) return TDBEM_ERR_ARG;
    if (c->prepared) return fail(c, TDBEM_ERR_STATE, "already prepared");
    if (c->ns == 0) return fail(c, TDBEM_ERR_STATE, "no mesh");
    auto t_start = std::chrono::steady_clock::now();
    const int ns = c->ns, nt = c->P.nt;
    TD_CUDA(cudaSetDevice(c->dev));
    TD_CUDA(join(c->user, c->s));
    set_bspline_table(c->bs, c->s);

    // which histories can be non-zero, hence which coefficient kinds
    bool any_d = false, any_n = false;
    for (int i = 0; i < ns; ++i) (c->phi[i] ? any_n : any_d) = true;
    bool has_k = !c->kbar.empty();
    bool q_nz = any_d || (has_k && any_n);
    bool u_nz = any_n || (has_k && any_d);
    c->ku_kind = q_nz ? (c->P.bie ? KIND_UB : KIND_CU) : -1;
    c->kw_kind = u_nz ? (c->P.bie ? KIND_WB : KIND_CW) : -1;

    // geometry
    TD_CUDA(dalloc(c, &c->d_xyz, 3 * (size_t)c->nv));
    TD_CUDA(dalloc(c, &c->d_tri, 3 * (size_t)ns));
    TD_CUDA(dalloc(c, &c->d_V, 9 * (size_t)ns));
    TD_CUDA(dalloc(c, &c->d_X, 3 * (size_t)ns));
    TD_CUDA(dalloc(c, &c->d_xc, 3 * (size_t)ns));
    TD_CUDA(dalloc(c, &c->d_n, 3 * (size_t)ns));
    TD_CUDA(dalloc(c, &c->d_phi, (size_t)ns));
    TD_CUDA(cudaMemcpyAsync(c->d_xyz, c->xyz.data(), 3 * sizeof(double) * c->nv, cudaMemcpyHostToDevice, c->s));
    TD_CUDA(cudaMemcpyAsync(c->d_tri, c->tri.data(), 3 * sizeof(int32_t) * ns, cudaMemcpyHostToDevice, c->s));
    TD_CUDA(cudaMemcpyAsync(c->d_phi, c->phi.data(), ns, cudaMemcpyHostToDevice, c->s));
    TD_CUDA(launch_geometry(c));

    // spatial hierarchy of the FMM (also built for the direct path when a
    // depth is given, for inspection)
    if (c->P.algo == 1 && c->P.depth < 2) return fail(c, TDBEM_ERR_ARG, "the FMM needs depth >= 2");
    if (c->P.depth > 0) {
        if (c->P.depth > 10) return fail(c, TDBEM_ERR_ARG, "depth above 10");
        TD_CUDA(cudaMemsetAsync(c->d_flag, 0, 4 * sizeof(int), c->s));
        std::string why;
        TD_CUDA(build_tree(c, why));
        if (!why.empty()) return fail(c, TDBEM_ERR_ARG, why);
    }
    if (c->P.algo == 1) {
        std::string why;
        TD_CUDA(fmm_setup(c, why));
        if (!why.empty())
            return fail(c, why.find("infeasible") != std::string::npos ? TDBEM_ERR_INFEASIBLE_HIERARCHY : TDBEM_ERR_ARG,
                        why);
    }

    // pair lists: every pair (direct path) or the near pairs of the leaf
    // neighbour cells (FMM path)
    if (c->P.algo == 1) {
        TD_CUDA(build_near_lists(c));
    } else {
        std::vector<int64_t> prow(ns + 1), rowblk(ns + 1);
        const int64_t nbr = (ns + 31) / 32;
        for (int i = 0; i <= ns; ++i) {
            prow[i] = (int64_t)i * ns;
            rowblk[i] = (int64_t)i * nbr;
        }
        TD_CUDA(dalloc(c, &c->d_prow, (size_t)ns + 1));
        TD_CUDA(dalloc(c, &c->d_rowblk, (size_t)ns + 1));
        TD_CUDA(cudaMemcpyAsync(c->d_prow, prow.data(), (ns + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, c->s));
        TD_CUDA(cudaMemcpyAsync(c->d_rowblk, rowblk.data(), (ns + 1) * sizeof(int64_t), cudaMemcpyHostToDevice,
                                c->s));
        TD_CUDA(cudaStreamSynchronize(c->s));
        c->npairs = (int64_t)ns * ns;
        c->nbt = (int64_t)ns * nbr;
    }

    // lag windows of the pairs and coefficients per 32-pair block
    TD_CUDA(dalloc(c, &c->d_meta, (size_t)c->npairs));
    TD_CUDA(dalloc(c, &c->d_btot, (size_t)c->nbt));
    TD_CUDA(dalloc(c, &c->d_boff, (size_t)c->nbt + 1));
    int *d_m = c->d_flag + 1;  // flag[1..3]: max cnt, max g0, max lag
    TD_CUDA(cudaMemsetAsync(c->d_flag, 0, 4 * sizeof(int), c->s));
    TD_CUDA(launch_windows(c, d_m, d_m + 1, d_m + 2));
    int mx[3];
    TD_CUDA(cudaMemcpyAsync(mx, d_m, 3 * sizeof(int), cudaMemcpyDeviceToHost, c->s));
    TD_CUDA(cudaStreamSynchronize(c->s));
    if (mx[0] > kMaxCnt) return fail(c, TDBEM_ERR_ARG, "lag window longer than 15 (element larger than ~10 c*dt)");
    if (mx[1] > kMaxG0) return fail(c, TDBEM_ERR_ARG, "lag beyond 4095 (surface too large for c*dt)");
    c->smax = std::max(mx[0], 1);
    c->gmax = mx[2];
    // short rows (fewer than 8 blocks on average) get one warp per row; long
    // ones (all pairs) four warps sharing a row's blocks
    c->near_wpr = (c->nbt < (int64_t)8 * ns) ? 1 : 4;

    // packed coefficient layout: block offsets by a prefix on the host
    {
        size_t nb = (size_t)c->nbt;
        std::vector<int32_t> tot(nb);
        std::vector<int64_t> off(nb);
        TD_CUDA(cudaMemcpyAsync(tot.data(), c->d_btot, nb * sizeof(int32_t), cudaMemcpyDeviceToHost, c->s));
        TD_CUDA(cudaStreamSynchronize(c->s));
        int64_t run = 0;
        for (size_t k = 0; k < nb; ++k) {
            off[k] = run;
            run += tot[k];
        }
        c->ncoef = run;
        off.push_back(run);
        TD_CUDA(cudaMemcpyAsync(c->d_boff, off.data(), (nb + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, c->s));
        TD_CUDA(cudaStreamSynchronize(c->s));
    }

    // influence coefficients
    if (c->ku_kind >= 0) TD_CUDA(dalloc(c, &c->d_ku, (size_t)c->ncoef + 2));
    if (c->kw_kind >= 0) TD_CUDA(dalloc(c, &c->d_kw, (size_t)c->ncoef + 2));

    TD_CUDA(launch_coefficients(c));

    // zero-lag matrix (width of its ELL store counted first) and the Jacobi
    // contraction factor
    TD_CUDA(cudaMemsetAsync(c->d_flag, 0, 4 * sizeof(int), c->s));
    TD_CUDA(dalloc(c, &c->d_ainv, (size_t)ns));
    TD_CUDA(launch_zero_lag(c, true));
    int cnt_w = 0;
    TD_CUDA(cudaMemcpyAsync(&cnt_w, c->d_flag + 1, sizeof(int), cudaMemcpyDeviceToHost, c->s));
    TD_CUDA(cudaStreamSynchronize(c->s));
    c->ell_w = std::max(cnt_w, 1);
    const int W = c->ell_w;
    TD_CUDA(dalloc(c, &c->d_aoff, (size_t)W * ns));
    TD_CUDA(dalloc(c, &c->d_acol, (size_t)W * ns));
    TD_CUDA(cudaMemsetAsync(c->d_flag, 0, 4 * sizeof(int), c->s));
    TD_CUDA(launch_zero_lag(c, false));
    std::vector<double> aoff((size_t)W * ns), ainv(ns);
    std::vector<int32_t> acol((size_t)W * ns);
    int fl = 0;
    TD_CUDA(cudaMemcpyAsync(aoff.data(), c->d_aoff, aoff.size() * sizeof(double), cudaMemcpyDeviceToHost, c->s));
    TD_CUDA(cudaMemcpyAsync(acol.data(), c->d_acol, acol.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, c->s));
    TD_CUDA(cudaMemcpyAsync(ainv.data(), c->d_ainv, ainv.size() * sizeof(double), cudaMemcpyDeviceToHost, c->s));
    TD_CUDA(cudaMemcpyAsync(&fl, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, c->s));
    TD_CUDA(cudaStreamSynchronize(c->s));
    if (fl & 2) return fail(c, TDBEM_ERR_ARG, "zero-lag row wider than its counted width");
    if (fl & 4) return fail(c, TDBEM_ERR_ARG, "zero-lag matrix has a zero diagonal entry");
    double qmax = 0.0;
    for (int i = 0; i < ns; ++i) {
        double s = 0.0;
        for (int k = 0; k < W; ++k)
            if (acol[(size_t)k * ns + i] >= 0) s += fabs(aoff[(size_t)k * ns + i]);
        qmax = std::max(qmax, s * fabs(ainv[i]));
    }
    c->contraction = qmax;
    double tol = c->P.solver_tol > 0 ? c->P.solver_tol : 1e-16;
    int maxit = c->P.solver_maxit > 0 ? c->P.solver_maxit : 200;
    if (!(qmax < 1.0))
        return fail(c, TDBEM_ERR_NOT_CONVERGED,
                    "zero-lag matrix not diagonally dominant (contraction " + std::to_string(qmax) + ")");
    // Jacobi error after K sweeps (the first gives D^-1 b) <= q^K |x|
    int K = (qmax > 0.0) ? (int)ceil(log(tol) / log(qmax)) : 1;
    if (K < 1) K = 1;
    if (K > maxit) return fail(c, TDBEM_ERR_NOT_CONVERGED, "zero-lag solve needs more sweeps than solver_maxit");
    c->solve_iters = K;

    // histories, initialised with the known data (unknown components zero).
    // Each is preceded by gmax zero rows: a lag g of step alpha reads row
    // alpha - g >= 1 - gmax, so the history sum needs no range test.
    size_t nh = (size_t)nt * ns;
    const size_t npad = (size_t)c->gmax * ns;
    TD_CUDA(dalloc(c, &c->d_u, npad + nh));
    TD_CUDA(dalloc(c, &c->d_q, npad + nh));
    TD_CUDA(cudaMemsetAsync(c->d_u, 0, npad * sizeof(double), c->s));
    TD_CUDA(cudaMemsetAsync(c->d_q, 0, npad * sizeof(double), c->s));
    c->d_u += npad;
    c->d_q += npad;
    if (c->split) {
        TD_CUDA(dalloc(c, &c->d_us, npad + nh));
        TD_CUDA(dalloc(c, &c->d_qs, npad + nh));
        TD_CUDA(cudaMemsetAsync(c->d_us, 0, npad * sizeof(float2), c->s));
        TD_CUDA(cudaMemsetAsync(c->d_qs, 0, npad * sizeof(float2), c->s));
        c->d_us += npad;
        c->d_qs += npad;
    }
    int rh = reset_histories(c);
    if (rh != TDBEM_OK) return rh;
    if (c->split) TD_CUDA(launch_split_coefficients(c));
    TD_CUDA(dalloc(c, &c->d_b, (size_t)ns));
    TD_CUDA(dalloc(c, &c->d_xa, (size_t)ns));
    TD_CUDA(dalloc(c, &c->d_xb, (size_t)ns));
    TD_CUDA(dalloc(c, &c->d_bar, 2));
    TD_CUDA(setup_jacobi_fused(c));
    TD_CUDA(dalloc(c, &c->d_r, (size_t)ns));
    TD_CUDA(cudaMemsetAsync(c->d_b, 0, ns * sizeof(double), c->s));
    TD_CUDA(cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->s));
    TD_CUDA(cudaStreamSynchronize(c->s));
    TD_CUDA(cudaGetLastError());
    c->prepared = true;
    c->alpha = 0;
    c->ms_prepare =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    TD_CUDA(join(c->s, c->user));
    return TDBEM_OK;
}

static int step_impl(tdbem_ctx *c, int nsteps, const double *d_exc, int64_t exc_stride)
{
    for (int n = 0; n < nsteps; ++n) {
        int alpha = c->alpha + 1;
        const double *far = nullptr;
        if (c->fmm.on) {
            // far field of the leaf interval that holds step alpha (Section 3)
            int kobs = (alpha - 1) / c->fmm.Lt;
            if (kobs != c->fmm.far_k) {
                if (kobs > 0) {
                    PhaseTimer t(c, PH_FAR);
                    TD_CUDA(fmm_boundary(c, kobs - 1));
                    c->launches[PH_FAR] += 1;
                }
                c->fmm.far_k = kobs;
            }
            far = c->fmm.far + (size_t)(alpha - 1 - kobs * c->fmm.Lt) * c->ns;
        }
        {
            PhaseTimer t(c, PH_NEAR);
            TD_CUDA(launch_near_sum(c, alpha, d_exc ? d_exc + n * exc_stride : nullptr, far));
        }
        c->launches[PH_NEAR] += 1;
        {
            PhaseTimer t(c, PH_SOLVE);
            if (c->sai_val && c->sai_grid > 0) {
                TD_CUDA(launch_sai_fused(c, alpha));
            } else if (c->sai_val) {
                for (int it = 0; it < c->sai_iters; ++it) TD_CUDA(launch_sai_sweep(c, alpha, it));
            } else if (c->jac_grid > 0) {
                TD_CUDA(launch_jacobi_fused(c, alpha));
            } else {
                for (int it = 0; it < c->solve_iters; ++it)
                    TD_CUDA(launch_jacobi(c, alpha, it, it == c->solve_iters - 1));
            }
        }
        c->launches[PH_SOLVE] += c->sai_val ? (c->sai_grid > 0 ? 1 : c->sai_iters) : (c->jac_grid > 0 ? 1 : c->solve_iters);
        c->alpha = alpha;
        c->steps_total += 1;
    }
    // the deferred far-field work of the last boundary is part of this call
    if (c->fmm.on) TD_CUDA(fmm_join(c));
    return TDBEM_OK;
}

// Kernels of one direct-path step reading the step index from d_alpha,
// launched on `st` (a stream being captured).
static cudaError_t launch_step_chain(tdbem_ctx *c, cudaStream_t st)
{
    cudaStream_t keep = c->s;
    c->s = st;
    c->alpha_dev_on = true;
    cudaError_t e = cudaSuccess;
    // FMM: every far-field pass, each deciding on the device whether this
    // step is one of its boundaries (Section 3), then the near sum reading
    // the far field of the step's position in its leaf interval
    if (c->fmm.on) e = fmm_boundary(c, 0, true);
    if (e == cudaSuccess) e = launch_near_sum(c, 0, nullptr, c->fmm.on ? c->fmm.far : nullptr);
    for (int it = 0; it < c->solve_iters && e == cudaSuccess; ++it) e = launch_jacobi(c, 0, it, it == c->solve_iters - 1);
    if (e == cudaSuccess) e = launch_alpha_next(c);
    c->alpha_dev_on = false;
    c->s = keep;
    return e;
}

// After graph-replayed steps: the far field in the buffer is the one of the
// leaf interval holding the last step (plain stepping resumes from there).
static void graph_steps_done(tdbem_ctx *c)
{
    if (c->fmm.on && c->alpha >= 1) c->fmm.far_k = (c->alpha - 1) / c->fmm.Lt;
}

static int graph_ready(tdbem_ctx *c)
{
    if (!c->prepared) return fail(c, TDBEM_ERR_STATE, "graph step before prepare");
    if (c->fmm.on && !c->split)
        return fail(c, TDBEM_ERR_ARG, "graph-replayed FMM steps need a precision from 1 to 5 (not the FP64 form)");
    if (c->sai_val) return fail(c, TDBEM_ERR_ARG, "graph-replayed steps use the Jacobi zero-lag solve");
    if (!c->d_alpha) TD_CUDA(dalloc(c, &c->d_alpha, 1));
    TD_CUDA(fmm_join(c));
    return TDBEM_OK;
}

int tdbem_step_graph(tdbem_ctx *c, int32_t nsteps)
{
    if (!c) return TDBEM_ERR_ARG;
    int r = graph_ready(c);
    if (r != TDBEM_OK) return r;
    if (nsteps < 0 || c->alpha + nsteps > c->P.nt - 1) return fail(c, TDBEM_ERR_ARG, "stepping past Nt-1");
    if (nsteps == 0) return TDBEM_OK;
    TD_CUDA(cudaSetDevice(c->dev));
    if (!c->graph) {
        cudaGraph_t g;
        TD_CUDA(cudaStreamBeginCapture(c->s, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = launch_step_chain(c, c->s);
        cudaError_t e2 = cudaStreamEndCapture(c->s, &g);
        TD_CUDA(e);
        TD_CUDA(e2);
        TD_CUDA(cudaGraphInstantiate(&c->graph, g, 0));
        cudaGraphDestroy(g);
    }
    TD_CUDA(join(c->user, c->s));
    int a = c->alpha + 1;
    TD_CUDA(cudaMemcpyAsync(c->d_alpha, &a, sizeof(int), cudaMemcpyHostToDevice, c->s));
    for (int n = 0; n < nsteps; ++n) TD_CUDA(cudaGraphLaunch(c->graph, c->s));
    c->launches[PH_NEAR] += nsteps;
    c->launches[PH_SOLVE] += (int64_t)nsteps * c->solve_iters;
    c->alpha += nsteps;
    c->steps_total += nsteps;
    graph_steps_done(c);
    TD_CUDA(join(c->s, c->user));
    return TDBEM_OK;
}

int tdbem_step(tdbem_ctx *c, int32_t nsteps)
{
    return tdbem_step_io(c, nsteps, nullptr, nullptr, 1);
}

int tdbem_step_io(tdbem_ctx *c, int32_t nsteps, const double *exc, double *x_out, int32_t on_device)
{
    if (!c) return TDBEM_ERR_ARG;
    if (!c->prepared) return fail(c, TDBEM_ERR_STATE, "step before prepare");
    if (nsteps < 0 || c->alpha + nsteps > c->P.nt - 1) return fail(c, TDBEM_ERR_ARG, "stepping past Nt-1");
    if (nsteps == 0) return TDBEM_OK;
    const int ns = c->ns;
    TD_CUDA(cudaSetDevice(c->dev));
    TD_CUDA(join(c->user, c->s));
    const double *d_exc = exc;
    if (exc && !on_device) {
        if (c->exc_cap < nsteps) {
            dfree(c, c->d_exc);
            c->d_exc = nullptr;
            TD_CUDA(dalloc(c, &c->d_exc, (size_t)nsteps * ns));
            c->exc_cap = nsteps;
        }
        TD_CUDA(cudaMemcpyAsync(c->d_exc, exc, (size_t)nsteps * ns * sizeof(double), cudaMemcpyHostToDevice, c->s));
        d_exc = c->d_exc;
    }
    int a0 = c->alpha;
    int r = step_impl(c, nsteps, d_exc, ns);
    if (r != TDBEM_OK) return r;
    if (x_out) {
        // x^{a-1}: u where phi = 1, q where phi = 0 (Eq. linear)
        if (on_device) {
            TD_CUDA(launch_gather_x(c, a0, nsteps, x_out));
        } else {
            if (c->xout_cap < nsteps) {
                dfree(c, c->d_xout);
                c->d_xout = nullptr;
                TD_CUDA(dalloc(c, &c->d_xout, (size_t)nsteps * ns));
                c->xout_cap = nsteps;
            }
            TD_CUDA(launch_gather_x(c, a0, nsteps, c->d_xout));
            TD_CUDA(cudaMemcpyAsync(x_out, c->d_xout, (size_t)nsteps * ns * sizeof(double), cudaMemcpyDeviceToHost,
                                    c->s));
            TD_CUDA(cudaStreamSynchronize(c->s));
        }
    } else if (exc && !on_device) {
        TD_CUDA(cudaStreamSynchronize(c->s));
    }
    TD_CUDA(join(c->s, c->user));
    return TDBEM_OK;
}

int tdbem_steps_done(const tdbem_ctx *c, int32_t *out)
{
    if (!c || !out) return TDBEM_ERR_ARG;
    *out = c->alpha;
    return TDBEM_OK;
}

int tdbem_get_solution(const tdbem_ctx *cc, double *u, double *q, int32_t beta0, int32_t nbeta, int32_t on_device)
{
    tdbem_ctx *c = const_cast<tdbem_ctx *>(cc);
    if (!c) return TDBEM_ERR_ARG;
    if (!c->prepared) return fail(c, TDBEM_ERR_STATE, "no solution before prepare");
    if (beta0 < 0 || nbeta < 0 || beta0 + nbeta > c->P.nt - 1) return fail(c, TDBEM_ERR_ARG, "beta range");
    size_t n = (size_t)nbeta * c->ns;
    size_t o = (size_t)beta0 * c->ns;
    cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    TD_CUDA(join(c->user, c->s));
    if (u) TD_CUDA(cudaMemcpyAsync(u, c->d_u + o, n * sizeof(double), k, c->s));
    if (q) TD_CUDA(cudaMemcpyAsync(q, c->d_q + o, n * sizeof(double), k, c->s));
    TD_CUDA(cudaStreamSynchronize(c->s));
    return check_flags(c);
}

int tdbem_get_rhs(const tdbem_ctx *cc, double *b)
{
    tdbem_ctx *c = const_cast<tdbem_ctx *>(cc);
    if (!c || !b) return TDBEM_ERR_ARG;
    if (!c->prepared) return fail(c, TDBEM_ERR_STATE, "no rhs before prepare");
    TD_CUDA(cudaMemcpyAsync(b, c->d_b, c->ns * sizeof(double), cudaMemcpyDeviceToHost, c->s));
    TD_CUDA(cudaStreamSynchronize(c->s));
    return TDBEM_OK;
}

int tdbem_get_coefficients(const tdbem_ctx *cc, int32_t kind, const int32_t *rows, int32_t nrows, int32_t gmax,
                           double *out)
{
    tdbem_ctx *c = const_cast<tdbem_ctx *>(cc);
    if (!c || !rows || !out || nrows < 0 || gmax < 0) return TDBEM_ERR_ARG;
    if (!c->prepared) return fail(c, TDBEM_ERR_STATE, "no coefficients before prepare");
    const double *src = nullptr;
    if (kind == c->ku_kind) src = c->d_ku;
    if (kind == c->kw_kind) src = c->d_kw;
    if (!src) return fail(c, TDBEM_ERR_ARG, "coefficient kind not stored by this run");
    const int ns = c->ns;
    memset(out, 0, sizeof(double) * (size_t)nrows * (gmax + 1) * ns);
    std::vector<int64_t> prow(ns + 1), rowblk(ns + 1);
    TD_CUDA(cudaMemcpy(prow.data(), c->d_prow, (ns + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
    TD_CUDA(cudaMemcpy(rowblk.data(), c->d_rowblk, (ns + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
    std::vector<uint16_t> meta;
    std::vector<int32_t> cols, tot;
    std::vector<int64_t> off;
    std::vector<double> vals;
    for (int r = 0; r < nrows; ++r) {
        int i = rows[r];
        if (i < 0 || i >= ns) return fail(c, TDBEM_ERR_ARG, "row out of range");
        int64_t np = prow[i + 1] - prow[i], nb = rowblk[i + 1] - rowblk[i];
        meta.resize(np);
        cols.resize(np);
        off.resize(nb);
        tot.resize(nb);
        if (np == 0) continue;
        TD_CUDA(cudaMemcpy(meta.data(), c->d_meta + prow[i], np * sizeof(uint16_t), cudaMemcpyDeviceToHost));
        if (c->d_col) TD_CUDA(cudaMemcpy(cols.data(), c->d_col + prow[i], np * sizeof(int32_t), cudaMemcpyDeviceToHost));
        TD_CUDA(cudaMemcpy(off.data(), c->d_boff + rowblk[i], nb * sizeof(int64_t), cudaMemcpyDeviceToHost));
        TD_CUDA(cudaMemcpy(tot.data(), c->d_btot + rowblk[i], nb * sizeof(int32_t), cudaMemcpyDeviceToHost));
        int64_t first = off[0], last = off[nb - 1] + tot[nb - 1];
        vals.resize((size_t)(last - first));
        if (last > first)
            TD_CUDA(cudaMemcpy(vals.data(), src + first, (last - first) * sizeof(double), cudaMemcpyDeviceToHost));
        if (c->split)
            for (auto &v : vals) {
                float hl[2];
                memcpy(hl, &v, sizeof(hl));
                v = (double)hl[0] + (double)hl[1];
            }
        for (int64_t b = 0; b < nb; ++b) {
            int64_t pos = off[b] - first;
            int cnt[32], g0[32], jj[32];
            for (int l = 0; l < 32; ++l) {
                int64_t pr = b * 32 + l;
                unsigned m = pr < np ? meta[pr] : 0u;
                cnt[l] = m >> kG0Bits;
                g0[l] = m & kMaxG0;
                jj[l] = pr < np ? (c->d_col ? cols[pr] : (int)pr) : 0;
            }
            for (int s = 0; s < kMaxCnt; ++s)
                for (int l = 0; l < 32; ++l) {
                    if (cnt[l] <= s) continue;
                    int g = g0[l] + s;
                    if (g <= gmax) out[((size_t)r * (gmax + 1) + g) * ns + jj[l]] = vals[pos];
                    ++pos;
                }
        }
    }
    return TDBEM_OK;
}

int tdbem_get_far(const tdbem_ctx *cc, double *out, int32_t *first_step, int32_t *nsteps)
{
    tdbem_ctx *c = const_cast<tdbem_ctx *>(cc);
    if (!c || !first_step || !nsteps) return TDBEM_ERR_ARG;
    if (!c->prepared || !c->fmm.on) return fail(c, TDBEM_ERR_STATE, "no far field (algo 0 or not prepared)");
    const int k = std::max(c->fmm.far_k, 0);
    *first_step = k * c->fmm.Lt + 1;
    *nsteps = c->fmm.Lt;
    if (out) {
        TD_CUDA(cudaStreamSynchronize(c->s));
        TD_CUDA(cudaMemcpy(out, c->fmm.far, (size_t)c->fmm.Lt * c->ns * sizeof(double), cudaMemcpyDeviceToHost));
    }
    return TDBEM_OK;
}

int tdbem_get_zero_lag(const tdbem_ctx *cc, double *out)
{
    tdbem_ctx *c = const_cast<tdbem_ctx *>(cc);
    if (!c || !out) return TDBEM_ERR_ARG;
    if (!c->prepared) return fail(c, TDBEM_ERR_STATE, "no matrix before prepare");
    const int ns = c->ns;
    const int W = c->ell_w;
    std::vector<double> aoff((size_t)W * ns), ainv(ns);
    std::vector<int32_t> acol((size_t)W * ns);
    TD_CUDA(cudaMemcpyAsync(aoff.data(), c->d_aoff, aoff.size() * sizeof(double), cudaMemcpyDeviceToHost, c->s));
    TD_CUDA(cudaMemcpyAsync(acol.data(), c->d_acol, acol.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, c->s));
    TD_CUDA(cudaMemcpyAsync(ainv.data(), c->d_ainv, ainv.size() * sizeof(double), cudaMemcpyDeviceToHost, c->s));
    TD_CUDA(cudaStreamSynchronize(c->s));
    memset(out, 0, sizeof(double) * (size_t)ns * ns);
    for (int i = 0; i < ns; ++i) {
        out[(size_t)i * ns + i] = 1.0 / ainv[i];
        for (int k = 0; k < W; ++k) {
            int j = acol[(size_t)k * ns + i];
            if (j >= 0) out[(size_t)i * ns + j] = aoff[(size_t)k * ns + i];
        }
    }
    return TDBEM_OK;
}

int tdbem_get_tree(const tdbem_ctx *cc, int32_t what, int32_t level, void *out, int64_t *count)
{
    tdbem_ctx *c = const_cast<tdbem_ctx *>(cc);
    if (!c || !count) return TDBEM_ERR_ARG;
    if (!c->prepared || c->tree.levels.empty()) return fail(c, TDBEM_ERR_STATE, "no hierarchy (depth 0)");
    const int ns = c->ns;
    if (what == TDBEM_TREE_BOX) {
        *count = 4;
        if (out) TD_CUDA(cudaMemcpy(out, c->tree.box, 4 * sizeof(double), cudaMemcpyDeviceToHost));
        return TDBEM_OK;
    }
    if (what == TDBEM_TREE_PERM) {
        *count = ns;
        if (out) TD_CUDA(cudaMemcpy(out, c->tree.perm, ns * sizeof(int32_t), cudaMemcpyDeviceToHost));
        return TDBEM_OK;
    }
    if (what == TDBEM_TREE_NEAR_OFF || what == TDBEM_TREE_NEAR) {
        if (!c->d_col) return fail(c, TDBEM_ERR_STATE, "no near lists (algo 0)");
        if (what == TDBEM_TREE_NEAR_OFF) {
            *count = ns + 1;
            if (out) {
                std::vector<int64_t> pr(ns + 1);
                TD_CUDA(cudaMemcpy(pr.data(), c->d_prow, (ns + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
                for (int i = 0; i <= ns; ++i) ((int64_t *)out)[i] = pr[i];
            }
        } else {
            *count = c->npairs;
            if (out) TD_CUDA(cudaMemcpy(out, c->d_col, c->npairs * sizeof(int32_t), cudaMemcpyDeviceToHost));
        }
        return TDBEM_OK;
    }
    if (level < 0 || level >= (int)c->tree.levels.size()) return fail(c, TDBEM_ERR_ARG, "level out of range");
    const TreeLevel &T = c->tree.levels[level];
    const int nc = T.nc;
    auto csr = [&](const int32_t *dlist, const int32_t *dcount, int stride, bool offsets) -> int {
        std::vector<int32_t> cnt(nc), lst((size_t)nc * stride);
        if (dcount) {
            TD_CUDA(cudaMemcpy(cnt.data(), dcount, nc * sizeof(int32_t), cudaMemcpyDeviceToHost));
            TD_CUDA(cudaMemcpy(lst.data(), dlist, lst.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
        }
        int64_t tot = 0;
        for (int k = 0; k < nc; ++k) tot += cnt[k];
        *count = offsets ? nc + 1 : tot;
        if (!out) return TDBEM_OK;
        int32_t *o = (int32_t *)out;
        int64_t run = 0;
        for (int k = 0; k < nc; ++k) {
            if (offsets)
                o[k] = (int32_t)run;
            else
                for (int a = 0; a < cnt[k]; ++a) o[run + a] = lst[(size_t)k * stride + a];
            run += cnt[k];
        }
        if (offsets) o[nc] = (int32_t)run;
        return TDBEM_OK;
    };
    switch (what) {
    case TDBEM_TREE_KEYS:
        *count = nc;
        if (out) TD_CUDA(cudaMemcpy(out, T.ckey, nc * sizeof(uint64_t), cudaMemcpyDeviceToHost));
        return TDBEM_OK;
    case TDBEM_TREE_START:
        *count = nc + 1;
        if (out) TD_CUDA(cudaMemcpy(out, T.cstart, (nc + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost));
        return TDBEM_OK;
    case TDBEM_TREE_NBR_OFF: return csr(T.nbr, T.ncount, 27, true);
    case TDBEM_TREE_NBR: return csr(T.nbr, T.ncount, 27, false);
    case TDBEM_TREE_IL_OFF: return csr(T.il, T.ilcount, 189, true);
    case TDBEM_TREE_IL: return csr(T.il, T.ilcount, 189, false);
    default: return fail(c, TDBEM_ERR_ARG, "unknown tree item");
    }
}

// Checkpoint layout: header (8 int64: magic, version, ns, nt, alpha, algo,
// precision, far_k), u and q rows [0, alpha), then for the FMM, per level
// 2..L: M, ring, D, A; then the current far field [Lt][ns].
namespace {
constexpr int64_t kCkptMagic = 0x544442454d434b50LL;  // "TDBEMCKP"

struct CkptPart {
    void *dev;
    size_t bytes;
};

std::vector<CkptPart> ckpt_parts(tdbem_ctx *c)
{
    std::vector<CkptPart> v;
    size_t rows = (size_t)c->alpha * c->ns * sizeof(double);
    v.push_back({c->d_u, rows});
    v.push_back({c->d_q, rows});
    if (c->fmm.on) {
        const size_t P = c->fmm.P;
        for (int l = 2; l <= c->fmm.L; ++l) {
            FmmLevel &V = c->fmm.lev[l];
            v.push_back({V.M, (size_t)V.nc * P * sizeof(double)});
            v.push_back({V.ring, (size_t)c->fmm.nslot * V.nc * P * sizeof(double)});
            v.push_back({V.D, (size_t)std::max(c->P.d, 1) * V.nc * P * sizeof(double)});
            v.push_back({V.A, (size_t)std::max(c->fmm.nd, 1) * V.nc * P * sizeof(double)});
        }
        v.push_back({c->fmm.far, (size_t)c->fmm.Lt * c->ns * sizeof(double)});
    }
    return v;
}
}  // namespace

int tdbem_checkpoint(const tdbem_ctx *cc, void *buf, size_t *len)
{
    tdbem_ctx *c = const_cast<tdbem_ctx *>(cc);
    if (!c || !len) return TDBEM_ERR_ARG;
    if (!c->prepared) return fail(c, TDBEM_ERR_STATE, "checkpoint before prepare");
    auto parts = ckpt_parts(c);
    size_t need = 8 * sizeof(int64_t);
    for (auto &p : parts) need += p.bytes;
    if (!buf) {
        *len = need;
        return TDBEM_OK;
    }
    if (*len < need) return fail(c, TDBEM_ERR_ARG, "checkpoint buffer too small");
    TD_CUDA(fmm_join(c));
    TD_CUDA(cudaStreamSynchronize(c->s));
    int64_t h[8] = {kCkptMagic, 1, c->ns, c->P.nt, c->alpha, c->P.algo, c->P.precision, c->fmm.far_k};
    char *o = (char *)buf;
    memcpy(o, h, sizeof(h));
    o += sizeof(h);
    for (auto &p : parts) {
        if (p.bytes) TD_CUDA(cudaMemcpy(o, p.dev, p.bytes, cudaMemcpyDeviceToHost));
        o += p.bytes;
    }
    *len = need;
    return TDBEM_OK;
}

int tdbem_restore(tdbem_ctx *c, const void *buf, size_t len)
{
    if (!c || !buf) return TDBEM_ERR_ARG;
    if (!c->prepared) return fail(c, TDBEM_ERR_STATE, "restore before prepare");
    int64_t h[8];
    if (len < sizeof(h)) return fail(c, TDBEM_ERR_ARG, "checkpoint too short");
    memcpy(h, buf, sizeof(h));
    if (h[0] != kCkptMagic || h[1] != 1 || h[2] != c->ns || h[3] != c->P.nt || h[5] != c->P.algo ||
        h[6] != c->P.precision || h[4] < 0 || h[4] > c->P.nt - 1)
        return fail(c, TDBEM_ERR_ARG, "checkpoint of another problem or format");
    TD_CUDA(fmm_join(c));
    int keep = c->alpha;
    c->alpha = (int)h[4];
    auto parts = ckpt_parts(c);
    size_t need = sizeof(h);
    for (auto &p : parts) need += p.bytes;
    if (len < need) {
        c->alpha = keep;
        return fail(c, TDBEM_ERR_ARG, "checkpoint truncated");
    }
    // steps past the restore point go back to their initial state (known
    // data only), so a context can also be rewound
    int rh = reset_histories(c);
    if (rh != TDBEM_OK) return rh;
    TD_CUDA(cudaStreamSynchronize(c->s));
    const char *o = (const char *)buf + sizeof(h);
    for (auto &p : parts) {
        if (p.bytes) TD_CUDA(cudaMemcpy(p.dev, o, p.bytes, cudaMemcpyHostToDevice));
        o += p.bytes;
    }
    c->fmm.far_k = (int)h[7];
    if (c->split) TD_CUDA(launch_split_histories(c));
    TD_CUDA(cudaStreamSynchronize(c->s));
    return TDBEM_OK;
}

int tdbem_get_stats(const tdbem_ctx *cc, tdbem_stats *o)
{
    tdbem_ctx *c = const_cast<tdbem_ctx *>(cc);
    if (!c || !o) return TDBEM_ERR_ARG;
    TD_CUDA(cudaStreamSynchronize(c->s));
    harvest(c);
    memset(o, 0, sizeof(*o));
    o->ms_rhs = c->ms[PH_RHS];
    o->ms_near = c->ms[PH_NEAR];
    o->ms_solve = c->ms[PH_SOLVE];
    o->ms_far = c->ms[PH_FAR];
    o->ms_m2l = c->ms[PH_M2L];
    o->launches_m2l = c->launches[PH_M2L];
    o->m2l_flops = c->m2l_flops;
    o->ms_gemm = c->ms[PH_GEMM];
    o->launches_gemm = c->launches[PH_GEMM];
    o->gemm_tc_flops = c->gemm_tc_flops;
    o->m2l_products = c->fmm.on ? (c->split ? c->fmm.nprod : 1) : 0;
    o->launches_far_kernels = c->far_kernels;
    for (int l = 0; l < 11 && l < (int)c->fmm.lev.size(); ++l) o->m2l_tile_n[l] = c->fmm.lev[l].np ? c->fmm.lev[l].tile_n : 0;
    o->launches_far = c->launches[PH_FAR];
    o->fmm_lt = c->fmm.Lt;
    o->fmm_mu = c->fmm.mu;
    o->ms_total = c->ms[PH_RHS] + c->ms[PH_NEAR] + c->ms[PH_SOLVE] + c->ms[PH_FAR];
    o->launches_rhs = c->launches[PH_RHS];
    o->launches_near = c->launches[PH_NEAR];
    o->launches_solve = c->launches[PH_SOLVE];
    o->steps = c->steps_total;
    o->n_pairs = c->npairs;
    o->n_coef = c->ncoef;
    int kinds = (c->ku_kind >= 0) + (c->kw_kind >= 0);
    // one full history sum at steady state (every lag of every window in use)
    o->near_bytes_per_step = c->ncoef * 8 * kinds + c->npairs * (c->d_col ? 6 : 2) + c->nbt * 8 +
                             (int64_t)c->gmax * c->ns * 8 * kinds + (int64_t)c->ns * 8;
    o->gamma_max = c->gmax;
    // the zero-lag solver in use: the learned SAI once installed, else Jacobi
    o->solve_iters = c->sai_val ? c->sai_iters : c->solve_iters;
    o->solve_contraction = c->sai_val ? c->sai_contraction : c->contraction;
    o->ms_prepare = c->ms_prepare;
    return TDBEM_OK;
}

int tdbem_reset_stats(tdbem_ctx *c)
{
    if (!c) return TDBEM_ERR_ARG;
    TD_CUDA(cudaStreamSynchronize(c->s));
    harvest(c);
    for (int k = 0; k < PH_COUNT; ++k) {
        c->ms[k] = 0;
        c->launches[k] = 0;
    }
    c->steps_total = 0;
    c->m2l_flops = 0.0;
    c->gemm_tc_flops = 0.0;
    c->far_kernels = 0;
    return TDBEM_OK;
}

int tdbem_set_overlap(tdbem_ctx *c, int32_t overlap)
{
    if (!c || (overlap != 0 && overlap != 1)) return TDBEM_ERR_ARG;
    if (!c->prepared) return fail(c, TDBEM_ERR_STATE, "overlap before prepare");
    TD_CUDA(fmm_join(c));
    c->fmm.overlap = overlap != 0;
    return TDBEM_OK;
}

int tdbem_sync(tdbem_ctx *c)
{
    if (!c) return TDBEM_ERR_ARG;
    TD_CUDA(fmm_join(c));
    TD_CUDA(cudaStreamSynchronize(c->s));
    TD_CUDA(cudaGetLastError());
    return check_flags(c);
}

struct tdbem_batch {
    std::vector<tdbem_ctx *> ctx;
    cudaStream_t s = nullptr;
    cudaGraphExec_t graph = nullptr;   // one step of every instance
    cudaGraphExec_t graphk = nullptr;  // k consecutive steps of every instance (k > 1)
    int k = 1;
    std::vector<cudaEvent_t> ev;
    std::string err;
};

// Captures `steps` consecutive steps of every instance into one graph, each
// instance an independent branch (fork from and join into B->s).
static cudaError_t batch_capture(tdbem_batch *B, int steps, cudaGraphExec_t *out)
{
    const int n = (int)B->ctx.size();
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(B->s, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaEventRecord(B->ev[n], B->s);
    for (int k = 0; k < n && e == cudaSuccess; ++k) {
        tdbem_ctx *c = B->ctx[k];
        e = cudaStreamWaitEvent(c->s, B->ev[n], 0);
        for (int t = 0; t < steps && e == cudaSuccess; ++t) e = launch_step_chain(c, c->s);
        if (e == cudaSuccess) e = cudaEventRecord(B->ev[k], c->s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(B->s, B->ev[k], 0);
    }
    cudaError_t e2 = cudaStreamEndCapture(B->s, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    if (g) cudaGraphDestroy(g);
    return e;
}

int tdbem_batch_create_steps(tdbem_ctx *const *ctxs, int32_t n, int32_t steps_per_launch, tdbem_batch **out)
{
    if (!ctxs || n < 1 || !out || steps_per_launch < 1 || steps_per_launch > 1024) return TDBEM_ERR_ARG;
    *out = nullptr;
    int dev = ctxs[0] ? ctxs[0]->dev : -1;
    for (int k = 0; k < n; ++k) {
        tdbem_ctx *c = ctxs[k];
        if (!c || c->dev != dev) return TDBEM_ERR_ARG;
        for (int m = 0; m < k; ++m)
            if (ctxs[m] == c) return TDBEM_ERR_ARG;
        int r = graph_ready(c);
        if (r != TDBEM_OK) return r;
    }
    tdbem_batch *B = new tdbem_batch();
    B->ctx.assign(ctxs, ctxs + n);
    B->k = steps_per_launch;
    cudaError_t e = cudaStreamCreateWithFlags(&B->s, cudaStreamNonBlocking);
    B->ev.resize(n + 1);
    for (auto &x : B->ev)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
    if (e == cudaSuccess) e = batch_capture(B, 1, &B->graph);
    if (e == cudaSuccess && B->k > 1) e = batch_capture(B, B->k, &B->graphk);
    if (e != cudaSuccess) {
        tdbem_batch_destroy(B);
        return TDBEM_ERR_CUDA;
    }
    *out = B;
    return TDBEM_OK;
}

int tdbem_batch_create(tdbem_ctx *const *ctxs, int32_t n, tdbem_batch **out)
{
    return tdbem_batch_create_steps(ctxs, n, 1, out);
}

int tdbem_batch_step(tdbem_batch *B, int32_t nsteps)
{
    if (!B || nsteps < 0) return TDBEM_ERR_ARG;
    // instances of uneven Nt: one that reaches its step Nt-1 stops there (its
    // kernels test the device-side step counter and do nothing), the others
    // go on; the replay count is the largest number of steps any has left
    int left = 0;
    for (tdbem_ctx *c : B->ctx) left = std::max(left, std::min(nsteps, c->P.nt - 1 - c->alpha));
    if (left == 0) return TDBEM_OK;
    nsteps = left;
    for (tdbem_ctx *c : B->ctx) {
        cudaError_t e = join(c->user, B->s);
        int a = c->alpha + 1;
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_alpha, &a, sizeof(int), cudaMemcpyHostToDevice, B->s);
        if (e != cudaSuccess) {
            B->err = cudaGetErrorString(e);
            return TDBEM_ERR_CUDA;
        }
    }
    // k steps per replay of the long graph, the rest one step per replay
    for (int n = 0; n < nsteps;) {
        const bool big = B->graphk && nsteps - n >= B->k;
        cudaError_t e = cudaGraphLaunch(big ? B->graphk : B->graph, B->s);
        if (e != cudaSuccess) {
            B->err = cudaGetErrorString(e);
            return TDBEM_ERR_CUDA;
        }
        n += big ? B->k : 1;
    }
    for (tdbem_ctx *c : B->ctx) {
        const int done = std::min(nsteps, c->P.nt - 1 - c->alpha);
        c->alpha += done;
        c->steps_total += done;
        graph_steps_done(c);
        c->launches[PH_NEAR] += nsteps;
        c->launches[PH_SOLVE] += (int64_t)nsteps * c->solve_iters;
        cudaError_t e = join(B->s, c->user);
        if (e != cudaSuccess) {
            B->err = cudaGetErrorString(e);
            return TDBEM_ERR_CUDA;
        }
    }
    return TDBEM_OK;
}

int tdbem_batch_sync(tdbem_batch *B)
{
    if (!B) return TDBEM_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(B->s);
    if (e != cudaSuccess) {
        B->err = cudaGetErrorString(e);
        return TDBEM_ERR_CUDA;
    }
    for (tdbem_ctx *c : B->ctx) {
        int r = check_flags(c);
        if (r != TDBEM_OK) {
            B->err = c->err;
            return r;
        }
    }
    return TDBEM_OK;
}

void tdbem_batch_destroy(tdbem_batch *B)
{
    if (!B) return;
    if (B->s) cudaStreamSynchronize(B->s);
    if (B->graph) cudaGraphExecDestroy(B->graph);
    if (B->graphk) cudaGraphExecDestroy(B->graphk);
    for (auto e : B->ev)
        if (e) cudaEventDestroy(e);
    if (B->s) cudaStreamDestroy(B->s);
    delete B;
}

const char *tdbem_batch_last_error(const tdbem_batch *B) { return B ? B->err.c_str() : "null batch"; }

}  // extern "C"
