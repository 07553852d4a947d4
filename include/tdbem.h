/*
 * tdbem.h -- C ABI of the GB300 time-domain boundary element library.
 *
 * The library solves the exterior initial-boundary value problem of the 3-D
 * scalar wave equation (Section 2.1, Eq. ibvp) by the time-domain boundary
 * element method of Takahashi, Tanigawa & Miyazawa (arXiv 2111.05205):
 * piecewise-constant elements with centroid collocation in space and
 * uniform-knot B-splines of order d in time (Section 2.3, Eq. u_bspline), the
 * ordinary BIE (Eq. bie, "OBIE") or the Burton-Miller BIE (Eq. bmbie,
 * "BMBIE"), marched in time step by step (Section 2.5, Eq. linear).
 *
 * Conventions common to every call:
 *   - every call returns an int status (tdbem_status); nothing throws;
 *   - inputs are copied, the caller keeps ownership of its buffers;
 *   - outputs go to caller-allocated buffers (host, or device memory of the
 *     context's GPU when a call takes on_device = 1);
 *   - the CUDA stream given to tdbem_create is borrowed, never destroyed;
 *     all device work of a context is ordered after the work queued on that
 *     stream before the call and before work queued on it after the call;
 *   - a context owns all the device memory it allocates (cudaMalloc) and
 *     frees it in tdbem_destroy; there is no global mutable state;
 *   - tdbem_last_error returns a message for the last failed call of the
 *     context (a static string for a NULL context).
 *
 * Units and signs (readings of the paper where it is silent):
 *   - mesh triangles are ordered counter-clockwise seen from outside the
 *     scatterer V; the paper's normal n (Eq. bie) points INTO V, i.e. it is
 *     minus the geometric normal (v1-v0)x(v2-v0) normalised;
 *   - q = du/dn with that n;
 *   - the collocation point x_i is the centroid (v0+v1+v2)/3 of element i;
 *   - the free term is absorbed into the double layer by evaluating every
 *     coefficient as the limit of x_i approaching S from outside V
 *     (Section 2.4, below Eq. bie_disc').
 *   - the incident wave (omitted from the formulation in Section 2.1) enters
 *     as the total-field term: 0 = e_i(t_a) + sum_j sum_b (Ubar q - Wbar u),
 *     with e = u_in (OBIE) or e = (d/dn_x - c^-1 d/dt) u_in (BMBIE).
 */
#ifndef TDBEM_H
#define TDBEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tdbem_ctx tdbem_ctx;

typedef enum {
    TDBEM_OK = 0,
    TDBEM_ERR_ARG = -1,        /* invalid argument or size */
    TDBEM_ERR_CUDA = -2,       /* a CUDA runtime call failed */
    TDBEM_ERR_OOM = -3,        /* device allocation failed */
    TDBEM_ERR_NOT_CONVERGED = -4,
    TDBEM_ERR_DIVERGED = -5,   /* solution norm grew past the guard */
    TDBEM_ERR_TIMEOUT = -6,
    TDBEM_ERR_INFEASIBLE_HIERARCHY = -7,
    TDBEM_ERR_STATE = -8       /* call out of order (e.g. step before prepare) */
} tdbem_status;

/* Problem and method parameters (Section 2, Section 5.1 for the values the
 * paper uses). */
typedef struct {
    double c;             /* wave speed c > 0 */
    double dt;            /* time-step length Delta_t > 0 */
    int32_t nt;           /* number of time steps Nt >= 2; collocation at t_a, a = 1..Nt-1 */
    int32_t d;            /* B-spline order d, 1 <= d <= 4 (Eq. decompose) */
    int32_t bie;          /* 0 = OBIE (Eq. bie), 1 = BMBIE (Eq. bmbie) */
    int32_t algo;         /* 0 = direct history sum over all element pairs (Eq. linear);
                             1 = near pairs (leaf neighbours) direct + the far part by the
                             interpolation-based space-time FMM (Sections 3-4, Formula 1) */
    int32_t precision;    /* 0 = FP64 throughout; 1..5 = split: the history sum stores every
                             coefficient and history value as an FP32 pair (hi, lo) (48
                             significant bits) and sums in double-float arithmetic on the
                             FP32 pipes; coefficients, the zero-lag matrix and the solve
                             are computed in FP64 either way.  The FMM's near-future M2L
                             blocks run on the tensor cores (FP32 accumulation) with
                             operators and moments split into 16-bit terms: 1 = three BF16
                             terms, six products (FP32-grade); 2 = BF16x3 (two terms,
                             three products); 3 = one BF16 product; 4 = two FP16 terms
                             scaled by powers of two per operator row and per cell's
                             moment, three products (about 22 bits); 5 = the near-future
                             blocks by the FFT (Section 4, the estimate after Algorithm 1):
                             equispaced nodes, the observation box equal to the source
                             box, so each block is a Toeplitz matrix applied as a circular
                             convolution on a 2ps x 2ps x 2ps x 2pt grid, FP32 transforms
                             and products on the CUDA cores.  The last near-future
                             block, the derivative rows and the recurrence of Formula 1
                             stay FP64 / double-float in every form. */
    int32_t ps, pt;       /* FMM: interpolation points per space / time dimension (2..8,
                             ps^3 pt <= 4096) */
    int32_t mu;           /* FMM: near-future intervals (Section 4.2); 0 = the smallest value
                             for which the kernel is a polynomial over every distant-future
                             interval (the paper uses 8) */
    int32_t depth;        /* leaf level L of the spatial hierarchy (root = 0); 0 = none */
    double solver_tol;    /* bound on the zero-lag solve's relative error (0: 1e-16) */
    int32_t solver_maxit; /* cap on zero-lag iterations (0: 200) */
    int32_t precond;      /* zero-lag solver: 0 = Jacobi sweeps; 1 = the learned sparse
                             approximate inverse that tdbem_set_precond installs where it
                             needs fewer sweeps than Jacobi (Jacobi stays its fallback) */
} tdbem_params;

/* Per-phase device time (ms) and launch counts accumulated since the last
 * tdbem_reset_stats; filled by tdbem_get_stats, which synchronises. */
typedef struct {
    double ms_rhs, ms_near, ms_solve, ms_total;
    int64_t launches_rhs, launches_near, launches_solve;
    int64_t steps;                 /* time steps taken in total */
    int64_t n_pairs;               /* element pairs with a non-empty lag window */
    int64_t n_coef;                /* stored coefficients per kind */
    int64_t near_bytes_per_step;   /* algorithmic HBM bytes of one full history sum: every
                                      stored coefficient, the pair windows (2 B per pair),
                                      block offsets (8 B per 32 pairs), the history window
                                      (gamma_max x ns x 8 B per history kind) and b */
    int32_t gamma_max;             /* largest lag stored */
    int32_t solve_iters;           /* zero-lag sweeps per step of the solver in use (Jacobi, or the
                                      learned SAI once tdbem_set_precond installed it) */
    double solve_contraction;      /* its contraction: max_i sum_{j!=i} |A_ij / A_ii| for Jacobi,
                                      ||I - M A||_inf for the SAI */
    double ms_prepare;             /* wall time of tdbem_prepare */
    double ms_far;                 /* FMM: P2M..L2P at leaf-interval boundaries */
    int64_t launches_far;          /* FMM: boundaries processed */
    int32_t fmm_lt, fmm_mu;        /* FMM: steps per leaf interval, near-future intervals */
    double ms_m2l;                 /* FMM: gather + M2L GEMMs + reduction, all levels */
    int64_t launches_m2l;          /* FMM: level M2L applications */
    double m2l_flops;              /* FMM: algorithmic M2L flops, 2 P per operator row and pair and
                                      application (rows of all-zero operator blocks not counted in
                                      the tensor-core forms) */
    int32_t m2l_tile_n[11];        /* FMM, tensor-core forms: GEMM tile width (columns) per level
                                      chosen by the setup-time tuner (0 for levels without
                                      interaction pairs or in the FP64 form) */
    double ms_gemm;                /* FMM: the M2L GEMM launches alone (tensor-core kernel, or the
                                      FP64 form's DGEMMs) */
    int64_t launches_gemm;         /* FMM: GEMM launches */
    double gemm_tc_flops;          /* FMM: tensor-pipe flops the split requires, m2l_flops x
                                      m2l_products (K and tile padding not counted) */
    int32_t m2l_products;          /* FMM: BF16 products per FP64 product (6, 3, 1; 1 = FP64 form) */
    int32_t reserved2;
    int64_t launches_far_kernels;  /* FMM: kernel launches of the far-field passes (P2M, M2L gather,
                                      GEMM, reduction, recurrence, M2M, L2L, L2P) */
} tdbem_stats;

/* Creates a context on the current CUDA device.  `stream` is a cudaStream_t
 * (NULL = legacy default stream) on which the caller orders its work. */
int tdbem_create(const tdbem_params *params, void *stream, tdbem_ctx **out);

/* Frees all device and host memory of the context (NULL is a no-op). */
void tdbem_destroy(tdbem_ctx *ctx);

/* Message of the last failed call ("" if none). */
const char *tdbem_last_error(const tdbem_ctx *ctx);

/* Surface mesh (Section 2.3): xyz[nv*3] vertex coordinates, tri[ns*3]
 * vertex indices of the ns flat triangular elements, counter-clockwise seen
 * from outside V.  Host pointers, copied.  ERR_ARG on an index out of range
 * or a degenerate triangle. */
int tdbem_set_mesh(tdbem_ctx *ctx, const double *xyz, int32_t nv, const int32_t *tri, int32_t ns);

/* Boundary condition per element (Section 2.5, phi_j): phi[ns] host, 1 =
 * Neumann (q given, u unknown), 0 = Dirichlet (u given, q unknown).
 * Default: all 0. */
int tdbem_set_bc(tdbem_ctx *ctx, const int8_t *phi);

/* Known boundary data sampled at the collocation times: f[(Nt-1)*ns] host,
 * row a-1 (a = 1..Nt-1) holds u_j(t_a) where phi_j = 0 and q_j(t_a) where
 * phi_j = 1.  tdbem_prepare converts the samples to B-spline coefficients
 * (Eq. u_bspline) by collocation, sum_{g=1..d} N^{0,d}(g) fbar^{a-g} = f(t_a),
 * marched in a (a reading: the paper does not say how known data is
 * expanded; for d = 1 it gives fbar^{a-1} = f(t_a)).  NULL = homogeneous
 * (the default).  ERR_ARG on a non-finite sample. */
int tdbem_set_known(tdbem_ctx *ctx, const double *f);

/* Incident plane pulse u_in(x,t) = f(t - t0 - k.x/c), k = dir normalised:
 * shape 0, the Gaussian f(s) = exp(-(s/width)^2); shape 1, the raised cosine
 * of Section 5.1.1 (Eq. uin), f(s) = 0.5 (1 - cos(2 pi c s / width)) for
 * 0 <= c s <= width and 0 otherwise (width = the pulse length Lambda; with
 * t0 = 0 and dir = +x_1 this is the paper's 0.5 (1 - Cos(2 pi (ct - x_1) /
 * Lambda))).  Replaces nothing else; without this call there is no incident
 * wave.  ERR_ARG for another shape, a zero direction or width <= 0. */
int tdbem_set_incident_plane(tdbem_ctx *ctx, const double dir[3], double t0, double width, int32_t shape);

/* Builds everything the marching needs on the device: element geometry,
 * lag windows, influence coefficients (Section 2.4, Appendix B), the
 * zero-lag matrix A (Eq. linear).  Synchronous. */
int tdbem_prepare(tdbem_ctx *ctx);

/* Advances nsteps time steps (Eq. linear at a = a_cur+1 .. a_cur+nsteps,
 * a <= Nt-1).  Asynchronous on the context's stream; ERR_ARG past Nt-1. */
int tdbem_step(tdbem_ctx *ctx, int32_t nsteps);

/* Advances nsteps time steps with the excitation supplied by the caller:
 * exc[nsteps*ns] holds the excitation e_i(t_a) of the steps taken (used in
 * place of the configured incident-wave term), and x_out[nsteps*ns]
 * receives the unknown x^{a-1}
 * of each step.  on_device = 0: both are host buffers (pinned or pageable)
 * and the call copies in and out on the stream and returns after the
 * copies completed; on_device = 1: device buffers, asynchronous.  exc may
 * be NULL (the configured incident wave, if any, is used); x_out may be
 * NULL. */
int tdbem_step_io(tdbem_ctx *ctx, int32_t nsteps, const double *exc, double *x_out, int32_t on_device);

/* Same as tdbem_step but every step is one replay of a CUDA graph that holds
 * the step's kernels (history sum, Jacobi sweeps and a device-side step
 * counter), captured at the first call: no per-kernel launch cost.  With the
 * FMM (algo 1) the graph also holds every far-field pass of every level
 * (Section 3: P2M, M2L, Formula 1, M2M, L2L, L2P); each of those kernels
 * reads the step from the device counter and does its work only at the
 * steps where plain stepping would run it (leaf-interval boundaries, and for
 * level l every 2^(L-l)-th of them), so the graph is the same for every
 * step.  Results are identical to tdbem_step (bit for bit).  ERR_ARG for
 * the FP64 FMM form (precision 0: its GEMMs are library calls that cannot
 * test the step) and with a learned SAI installed. */
int tdbem_step_graph(tdbem_ctx *ctx, int32_t nsteps);

/* Batched driver: several independent instances (contexts on one device,
 * direct path or FMM in a precision from 1 to 5, e.g. scatterers of
 * different size, order and BIE)
 * advanced together, each step of all of them one replay of a single CUDA
 * graph in which every instance's step is an independent branch, so that
 * small instances share the GPU.  tdbem_batch_create captures the graph
 * (the contexts must outlive the batch and not be stepped otherwise while
 * it exists); tdbem_batch_step advances every instance nsteps steps, or
 * to its last step Nt-1 if that comes first (instances may have different
 * Nt: one at its end stops, its kernels in later replays test the
 * device-side step counter and do nothing; stepping with every instance at
 * its end is a no-op; asynchronous; ordered after and before each
 * context's stream);
 * tdbem_batch_sync waits and reports the first device-side error.  Results
 * are identical to stepping each context alone. */
typedef struct tdbem_batch tdbem_batch;
int tdbem_batch_create(tdbem_ctx *const *ctxs, int32_t n, tdbem_batch **out);
/* As tdbem_batch_create, and a second graph holds steps_per_launch
 * (1..1024) consecutive steps of every instance, so that one graph launch
 * advances the whole batch that many steps; tdbem_batch_step replays it as
 * often as the requested steps allow and the one-step graph for the rest. */
int tdbem_batch_create_steps(tdbem_ctx *const *ctxs, int32_t n, int32_t steps_per_launch, tdbem_batch **out);
int tdbem_batch_step(tdbem_batch *batch, int32_t nsteps);
int tdbem_batch_sync(tdbem_batch *batch);
void tdbem_batch_destroy(tdbem_batch *batch);
const char *tdbem_batch_last_error(const tdbem_batch *batch);

/* Self-check of the bounded grid barrier used by the fused zero-lag solve
 * (plain stepping runs the solve's K Jacobi sweeps in one cooperative
 * launch with a grid barrier between sweeps; every wait in it gives up
 * after a bounded number of polls, about 0.3 s, and the step then reports
 * TDBEM_ERR_TIMEOUT at the next synchronisation instead of hanging).  Runs
 * three barriers over nblocks CTAs (cooperative launch, so nblocks must fit
 * on the device at once); starve != 0 starts the arrival count where no CTA
 * can complete it, so every wait runs out.  *timed_out (host) = 1 if a wait
 * gave up.  ERR_ARG for nblocks < 1, ERR_CUDA if the launch fails.
 * Synchronises the device. */
int tdbem_grid_barrier_probe(int32_t nblocks, int32_t starve, int32_t *timed_out);

/* Self-check of the split-precision tensor-core GEMM that evaluates the
 * M2L contraction (Section 4.2, Eq. m2l_actual written as operator stack x
 * moments; the paper gives no kernel).  Computes, on the current device,
 *   c[j*m + i] = sum_{p < nprod} A_{s_p}[i, :] . B_{t_p}[j, :],
 * s_p = prod[p] >> 4, t_p = prod[p] & 15, for i < m, j < n, where the terms
 * A_s are a[(s*m + i)*k + x] (nta terms, 1..3) and B_t are b[(t*n + j)*k + x]
 * (ntb terms, 1..3), all 16-bit floating-point numbers (fmt 1 = BF16, 0 =
 * FP16) given as their bit patterns, with FP32 accumulation in tensor
 * memory (tcgen05.mma, operands loaded by TMA; bn = 128 or 256 columns per
 * tile).  Host buffers a[nta*m*k], b[ntb*n*k] (copied) and c[m*n] (FP32
 * out).  ERR_ARG on a bad size or product; ERR_CUDA on a CUDA failure;
 * ERR_TIMEOUT if a pipeline wait of the kernel gave up (every wait is
 * bounded by about 2 s).  Synchronous.  For tests of the kernel only. */
int tdbem_tc_gemm_check(int32_t m, int32_t n, int32_t k, int32_t nta, int32_t ntb, const int32_t *prod, int32_t nprod,
                        int32_t fmt, int32_t bn, const uint16_t *a, const uint16_t *b, float *c);

/* Learned sparse approximate inverse for the zero-lag solve (an addition
 * of this library; the paper only states that the system is sparse).  A
 * trainer holds a 2-layer network (5*width inputs -> hidden ReLU -> width
 * outputs, FP16 weights, FP32 arithmetic) that maps the features of row i
 * of A (per slot k, the diagonal first and then the off-diagonal entries
 * with |A_ij| >= 1e-12 |A_ii| by decreasing |A_ij|: A_ij/A_ii, A_jj/A_ii,
 * A_ji/A_ii, |x_i - x_j|/(c dt), 1) to a correction of the row of a left
 * SAI M on that pattern: M_ij = (base_k + output_k) / A_ii with base 1 on the
 * diagonal and the first Neumann term -A_ij/A_jj off it.  Training minimises
 * sum_i ||e_i^T - m_i^T A||^2 over the rows of prepared contexts (their
 * zero-lag matrices; a context with nt = 2 computes only those) with Adam,
 * one update per context and pass, all on the GPU.  width 2..16, hidden
 * 1..64; the output layer starts near zero (M = the Neumann SAI). */
typedef struct tdbem_sai tdbem_sai;
int tdbem_sai_create(int32_t width, int32_t hidden, uint64_t seed, tdbem_sai **out);
void tdbem_sai_destroy(tdbem_sai *sai);
const char *tdbem_sai_last_error(const tdbem_sai *sai);
int tdbem_sai_train(tdbem_sai *sai, tdbem_ctx *const *ctxs, int32_t n, int32_t epochs, float lr, float *loss_out);
/* Loss (sum over rows) and gradient (grad[count], FP32) at the current weights. */
int tdbem_sai_gradient(tdbem_sai *sai, tdbem_ctx *ctx, float *grad, float *loss);
/* Weights: *count = their number; set = 0 copies the FP16 weights (as
 * floats) to inout, set = 1 loads inout (and resets the optimiser). */
int tdbem_sai_weights(tdbem_sai *sai, float *inout, int64_t *count, int32_t set);
/* Installs the network's M as the context's zero-lag solver (sweeps
 * x <- x + M (b - A x), run as x_0 = M b, x <- M b + (I - M A) x with I - M A
 * formed once at installation; all K of a step in one cooperative launch with a
 * bounded grid barrier where the device supports it, else one launch each;
 * K from ||I - M A||_inf so that the error stays below solver_tol) when that
 * takes fewer sweeps than Jacobi; otherwise Jacobi stays.  *use_sai,
 * *sweeps, *contraction report the choice (tdbem_get_stats then reports the
 * SAI's sweeps and contraction as solve_iters / solve_contraction).
 * ERR_STATE for a context created with precond = 0 (Jacobi only) or not prepared. */
int tdbem_set_precond(tdbem_ctx *ctx, const tdbem_sai *sai, int32_t *use_sai, int32_t *sweeps, double *contraction);

/* Checkpoint and resume at any step boundary (an addition of the library).
 * The state is the u and q histories of the steps taken and, for the FMM,
 * every level's moment accumulator, locals L_k..L_{k+mu+1}, derivative and
 * auxiliary locals of Formula 1 and the current leaf far field.
 * tdbem_checkpoint: buf = NULL sets *len to the size needed; otherwise buf
 * (host, *len bytes) receives the state (synchronises).  tdbem_restore
 * loads it into a context prepared for the same problem (same mesh, BC,
 * known data, incident wave and parameters; ERR_ARG otherwise), which may
 * be the checkpointed context itself at a later step (a rewind: the steps
 * after the checkpoint return to their initial state); stepping then
 * continues exactly as the checkpointed context would. */
int tdbem_checkpoint(const tdbem_ctx *ctx, void *buf, size_t *len);
int tdbem_restore(tdbem_ctx *ctx, const void *buf, size_t len);

/* Number of time steps taken so far (a_cur). */
int tdbem_steps_done(const tdbem_ctx *ctx, int32_t *out);

/* B-spline coefficient histories u_j^beta, q_j^beta for beta = beta0 ..
 * beta0+nbeta-1 (each [nbeta*ns], either may be NULL).  Synchronises. */
int tdbem_get_solution(const tdbem_ctx *ctx, double *u, double *q, int32_t beta0, int32_t nbeta, int32_t on_device);

/* Right-hand side b^{a-1} of the last step taken (Eq. linear, incident term
 * included), b[ns] host.  Synchronises. */
int tdbem_get_rhs(const tdbem_ctx *ctx, double *b);

/* Stored influence coefficients of selected rows, expanded to dense form:
 * kind 0 = C_U, 1 = C_W, 2 = Ubar, 3 = Wbar (only the kinds the run needs are
 * stored; ERR_ARG for another); rows[nrows] element indices;
 * out[nrows*(gmax+1)*ns] host, out[(r*(gmax+1)+g)*ns + j], zero outside the
 * stored windows and at g = 0. */
int tdbem_get_coefficients(const tdbem_ctx *ctx, int32_t kind, const int32_t *rows, int32_t nrows,
                           int32_t gmax, double *out);

/* FMM far field of the current leaf interval: out[Lt*ns] host (row t = step
 * first_step + t), the interpolated far part of the history sum (Eq. target,
 * Eq. target_m2l; with the Burton-Miller operator for BMBIE).  out may be NULL
 * to query first_step and nsteps (= Lt).  ERR_STATE without algo 1. */
int tdbem_get_far(const tdbem_ctx *ctx, double *out, int32_t *first_step, int32_t *nsteps);

/* Field off the boundary (Section 2.1: the representation formula of the
 * exterior problem, of which Eq. bie is the limit on S), discretised like the
 * boundary equation:
 *   u(x_p, t_a) = u_in(x_p, t_a) + sum_j sum_{g=1}^{a} (C_U^(g)(x_p, E_j) q_j^{a-g}
 *                                                     - C_W^(g)(x_p, E_j) u_j^{a-g})
 * with the compact coefficients of the marching evaluated at x_p and the
 * solution histories of the steps taken; u_in is the incident pulse, if any.
 * points[npts*3] host (copied), points of the exterior domain off S;
 * out[na*npts] host, out[(a - a0)*npts + p] for steps a = a0 .. a0+na-1,
 * 1 <= a0, a0+na-1 <= steps taken.  Whatever the BIE used to solve, the field
 * is the single- and double-layer representation.  ERR_ARG for an empty set,
 * steps outside that range or a point on S; synchronous. */
int tdbem_eval_field(const tdbem_ctx *ctx, const double *points, int32_t npts, int32_t a0, int32_t na, double *out);

/* Zero-lag matrix A of Eq. linear as dense host rows out[ns*ns] (small ns only). */
int tdbem_get_zero_lag(const tdbem_ctx *ctx, double *out);

/* Spatial hierarchy of the space-time FMM (Section 3, Fig. 2; interaction
 * lists of Section 4.2, Remark precomp), built by tdbem_prepare when
 * params.depth = L > 0.  Definition (the paper defers it to its earlier
 * study): root cube lo = componentwise minimum of the collocation points,
 * side = largest extent x (1 + 2^-20); element i lies in the leaf cell
 * floor((x_i - lo) / side * 2^L) (FP64, each operation rounded separately,
 * clamped to [0, 2^L - 1]); cells are numbered by Morton key (bit b of
 * x, y, z at 3b, 3b+1, 3b+2) and elements ordered by (leaf key, index); the
 * occupied cells of level l are the distinct keys >> 3(L - l).  Neighbours
 * of a cell: occupied cells within one cell in every axis (itself
 * included); interaction list (levels >= 2): occupied children of the
 * parent's neighbours that are not neighbours (at most 189).  Lists are
 * ordered by key and given as cell indices of the level.
 * what: TDBEM_TREE_BOX (double[4]: lo, side; level ignored), _PERM (int32
 * [ns]: element at each sorted position), _KEYS (uint64 [ncells]), _START
 * (int32 [ncells+1]: first sorted position of each cell), _NBR_OFF /
 * _IL_OFF (int32 [ncells+1] CSR offsets), _NBR / _IL (int32 entries),
 * _NEAR_OFF (int64 [ns+1], algo 1: row offsets in element numbering) and
 * _NEAR (int32: for each element, every element of the leaf cells that
 * neighbour its own, cells by key and elements in sorted order).
 * *count receives the number of entries; out may be NULL to query it;
 * otherwise out is a host buffer of that many entries.  ERR_STATE without a
 * hierarchy. */
enum {
    TDBEM_TREE_BOX = 0, TDBEM_TREE_PERM = 1, TDBEM_TREE_KEYS = 2, TDBEM_TREE_START = 3,
    TDBEM_TREE_NBR_OFF = 4, TDBEM_TREE_NBR = 5, TDBEM_TREE_IL_OFF = 6, TDBEM_TREE_IL = 7,
    TDBEM_TREE_NEAR_OFF = 8, TDBEM_TREE_NEAR = 9
};
int tdbem_get_tree(const tdbem_ctx *ctx, int32_t what, int32_t level, void *out, int64_t *count);

int tdbem_get_stats(const tdbem_ctx *ctx, tdbem_stats *out);
int tdbem_reset_stats(tdbem_ctx *ctx);

/* Blocks until all work of the context has finished; reports a device-side
 * error (divergence guard) raised since the last check. */
int tdbem_sync(tdbem_ctx *ctx);

/* Schedule of the FMM's far field in plain stepping (tensor-core forms):
 * overlap = 1 (the default) runs the part of each leaf-interval boundary's
 * work that later boundaries need (M2L blocks 2..mu, the exact rows, the
 * recurrence of Formula 1) on a second, lower-priority stream under the
 * following steps' history sums; overlap = 0 runs every pass in order on the
 * context's stream (every kernel then has the GPU to itself, e.g. to time
 * it).  Results are the same bit for bit.  Takes effect at the next step;
 * ERR_STATE before prepare. */
int tdbem_set_overlap(tdbem_ctx *ctx, int32_t overlap);

/* Zero-lag solve that allocates no device memory (the paper has no
 * counterpart: it is a service for callers that cannot call cudaMalloc at the
 * point where they solve, e.g. code that runs while someone else captures a
 * CUDA graph, or hosts that forbid allocation after start-up).  Solves
 * A x = b with the context's zero-lag matrix (Eq. linear, built by
 * tdbem_prepare) by the Jacobi sweeps tdbem_step uses (always plain Jacobi:
 * a learned SAI preconditioner installed by tdbem_set_precond is ignored, so
 * then the two solutions agree to solver_tol, not bit for bit), with its
 * scratch (b and two iterates) in a fixed file-scope device array of
 * 3 x 262144 doubles (6 MiB) that every GPU loading the library keeps until
 * exit.  b[ns] in, x[ns] out: host buffers (on_device = 0; the call returns
 * after the copy back) or device buffers (on_device = 1; asynchronous); b
 * and x must not overlap.  Work goes on the stream given to tdbem_create.
 * ERR_ARG if ns exceeds 262144 (checked first, x untouched).  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress,
 * with that device current) and should come before any stream capture.  All calls on one device share
 * the array and it keeps the last call's contents: calls that overlap on the
 * GPU race.  No cudaMalloc, cudaFree or allocating library call is made. */
int tdbem_zero_lag_solve_static(const tdbem_ctx *ctx, const double *b, double *x, int32_t on_device);

#ifdef __cplusplus
}
#endif
#endif /* TDBEM_H */
