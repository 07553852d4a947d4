// Internal declarations shared by the translation units of libtdbem.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/tdbem.h"
#include "coef_math.cuh"

namespace tdbem {

// Pair metadata: lag window start g0 (12 bits) and length cnt (4 bits).
constexpr int kG0Bits = 12;
constexpr int kMaxG0 = (1 << kG0Bits) - 1;
constexpr int kMaxIL = 189;  // cells in one interaction list: 7^3 - 3^3 offsets, at most 189 occupied
constexpr int kMaxCnt = 15;

// Coefficient kinds (bit positions in a kinds mask).
enum { KIND_CU = 0, KIND_CW = 1, KIND_UB = 2, KIND_WB = 3 };

struct Incident {
    int on;
    int bie;
    int shape;  // 0: Gaussian exp(-(s/width)^2); 1: raised cosine of length width (Section 5.1.1)
    double k[3];
    double t0, width, c, dt;
};

// One level of the spatial hierarchy (device arrays).
struct TreeLevel {
    int nc = 0;                   // occupied cells
    uint64_t *ckey = nullptr;     // [nc] Morton keys, increasing
    int32_t *cstart = nullptr;    // [nc+1] first sorted position of each cell
    int32_t *ecell = nullptr;     // [ns] cell of each sorted position
    int32_t *nbr = nullptr;       // [nc][27] neighbour cells, by key
    int32_t *ncount = nullptr;    // [nc]
    int32_t *il = nullptr;        // [nc][189] interaction list, by key (levels >= 2)
    int32_t *ilcount = nullptr;   // [nc]
};

struct Tree {
    double *box = nullptr;        // lo[3], side
    uint64_t *key = nullptr;      // [ns] leaf keys (element numbering)
    int32_t *perm = nullptr;      // [ns] element at each sorted position
    int32_t *e2c = nullptr;       // [ns] leaf cell of each element (element numbering)
    std::vector<TreeLevel> levels;
};

// Graph-replayed steps (tdbem_step_graph, tdbem_batch_*): every kernel of
// the far field reads the step alpha from the device counter and works out
// there whether its pass runs at this step and for which interval (the host
// decides both in plain stepping).  A boundary step is the first step of a
// leaf interval: alpha - 1 = k1 Lt, k1 >= 1 leaf intervals completed.
struct StepWhen {
    const int *alpha = nullptr;  // device step counter; nullptr: plain stepping
    int alim = 0;                // last step, Nt - 1
    int lt = 1;                  // steps per leaf interval
    int span = 1;                // leaf intervals per interval of the pass's level
};

// The index of the level's interval that ended just before this step, or -1
// when the pass does not run at this step.
__device__ __forceinline__ int when_interval(const StepWhen w)
{
    const int a = *w.alpha;
    if (a > w.alim || a < 2 || (a - 1) % w.lt) return -1;
    const int k1 = (a - 1) / w.lt;
    if (k1 % w.span) return -1;
    return k1 / w.span - 1;
}

// Grid-wide barrier of a cooperative launch (every CTA resident): arrival
// counter bar[0], generation bar[1].  The wait is bounded: after
// kBarrierPolls polls the CTA records a timeout (flag bit 4) and goes on,
// so a barrier that cannot complete ends the kernel with an error that the
// host reports, never with a hang.
constexpr unsigned kBarrierPolls = 1u << 22;  // with 64 ns sleeps: about 0.3 s

__device__ __forceinline__ void grid_barrier(unsigned *bar, int *flag)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = bar + 1;
        const unsigned g = *gen;
        __threadfence();
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            // poll with short sleeps (polling without them measured slower:
            // every waiting CTA then hammers the same word)
            unsigned polls = 0;
            while (*gen == g) {
                if (++polls > kBarrierPolls) {
                    atomicOr(flag, 4);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
}

// Split-precision tensor-core GEMM (tc_gemm.cu): one output tile of at most
// 128 rows (A rows) x BN columns (B rows), C[c_off + j ldc + i].
constexpr int kTcBM = 128;
constexpr int kTcBK = 64;          // K elements per 128-byte swizzle row
constexpr int kTcMaxTerms = 3;
constexpr int kTcMaxProd = 6;
constexpr int kTcSmemBudget = 232448;  // dynamic shared memory per CTA (227 KB)

struct TcTile {
    int32_t a_row, b_row;  // first row of the tile in term 0 of A and B
    int32_t rows, cols;    // valid rows (<= 128) and columns (<= BN)
    int64_t c_off;         // C index of (row 0, column 0)
};

struct TcGemmArgs {
    int32_t nta, ntb;                 // terms of A and B
    int32_t a_term_rows, b_term_rows; // row distance between consecutive terms
    int32_t nprod;
    int32_t prod[kTcMaxProd];         // (A term << 4) | B term
    int32_t kchunks;                  // K / 64
    int32_t nstage;                   // shared-memory pipeline stages
    int32_t fmt;                      // 0 = FP16, 1 = BF16
    int64_t ldc;
    float *C;
    const TcTile *tiles;
    int32_t ntiles;
    int *err;                         // bit 3 (value 8) is set when a pipeline wait gave up
    StepWhen when;                    // graph-replayed steps: run only at the level's M2L steps
    const float *a_scale;             // per A row (term-0 row index) and per B row: the result is
    const float *b_scale;             // multiplied by both in the epilogue (nullptr: no scaling)
};

cudaError_t tc_make_map(CUtensorMap *map, const void *base, int64_t rows, int kp, int box_rows);
int tc_stages(int nta, int ntb, int bn);
size_t tc_smem_bytes(int nta, int ntb, int bn, int nstage);
// sm_div: the persistent grid takes 1/sm_div of the SMs (1: all)
cudaError_t tc_gemm_launch(const CUtensorMap &ta, const CUtensorMap &tb, const TcGemmArgs &a, int ntiles, int bn,
                           cudaStream_t s, int sm_div = 1);

// One level of the space-time FMM (device arrays; levels 2..L).
//
// M2L layout: the cell offsets o = S - O of the level's interaction pairs
// fall into classes of the cube's symmetry group (axis permutations and
// reflections); every offset is g(c) for the class's canonical offset c
// (|c_0| >= |c_1| >= |c_2| >= 0) and one fixed element g.  Because g maps
// the interpolation nodes onto themselves, the operator of o is the
// canonical one with its node indices permuted, so one operator per class
// serves all its offsets: a pair's moment enters the GEMM permuted by g and
// its product leaves it permuted back (see fmm.cu).
struct FmmLevel {
    int nc = 0;
    double s = 0, hs = 0, ho = 0;  // cell side, source / observation interpolation half-widths
    int T = 0;                   // steps per interval
    double Tlen = 0;             // c x interval length (T of Formula 1)
    double *M = nullptr;         // [nc][P] moment of the current source interval
    double *ring = nullptr;      // [mu+2][nc][P] locals L_k .. L_{k+mu+1}
    double *D = nullptr;         // [d][nc][P] derivative locals L^(p)
    double *A = nullptr;         // [n_d][nc][P] auxiliary locals L^(p,m)
    double *G = nullptr;         // [d][nc][P] contributions L^(p)_{k+mu+1,k}
    double *Sm = nullptr;        // [2][ps][ps] source-box transfer to the parent level (M2M)
    double *So = nullptr;        // [2][ps][ps] observation-box transfer from the parent level (L2L)
    // interaction pairs in GEMM column order: grouped by symmetry class
    int64_t np = 0;              // pairs (= GEMM columns)
    int ncls = 0;                // classes with pairs
    std::vector<int64_t> cbase;  // [ncls+1] first column of each class
    int32_t *pS = nullptr;       // [np] source cell of each column
    uint8_t *pg = nullptr;       // [np] symmetry element of each column
    uint8_t *pc = nullptr;       // [np] class of each column
    void *kr = nullptr;          // [ncls][d+1][P3][P3] r_ab^(e-1) between the canonical nodes (e = 0..d;
                                 // e = 1 unused): FP64, or float pairs in the tensor-core forms
    void *dmu = nullptr;         // [np][d+1][P3] time moments of the columns (exact rows: the block
                                 // L_{k+mu+1,k} and the derivative rows)
    void *dF = nullptr;          // [np][d+1][d+1][P3] their distance-power products
    double *dss = nullptr;       // [np][d+1] sums of the time moments
    int4 *djobs = nullptr;       // [njobs] (class, first column, columns) of the products kernel
    double *dcoef = nullptr;     // [d+1][pt][d+1][d+1] binomial-expansion coefficients of the exact rows
    int njobs = 0;
    int64_t *ooff = nullptr;     // [nc+1] columns of each observation cell (CSR)
    int64_t *oidx = nullptr;     // [np] their columns, in interaction-list order
    uint8_t *og = nullptr;       // [np] their symmetry elements
    double *op = nullptr;        // FP64 form: [ncls][mu P][P] canonical operator stacks (near future 1..mu)
    double *Bbuf = nullptr;      // FP64 form: [np][P] gathered (permuted) moments
    double *Cbuf = nullptr;      // FP64 form: [np][mu P] products
    // tensor-core forms: split terms of operators and moments, FP32 products
    uint16_t *opt = nullptr;     // [nta][ncls][Rp][Kp] BF16 operator terms
    uint16_t *Bt = nullptr;      // [ntb][np][Kp] BF16 moment terms
    float *ascale = nullptr;     // scaled FP16 form: [ncls][Rp] row scales of the operator terms
    float *bscale = nullptr;     // scaled FP16 form: [np] column scales of the moment terms
    int *cexp = nullptr;         // scaled FP16 form: [nc] scale exponent of each cell's moment
    float *C32 = nullptr;        // [np][mu P] products
    TcTile *tiles = nullptr;     // [ntiles] GEMM tiles (zero operator blocks skipped); the ntiles_u
    int ntiles = 0;              // tiles of the first near-future block's rows come first
    int ntiles_u = 0;
    double flops_u = 0;          // algorithmic flops of those tiles
    int tile_n = 128;            // tile width chosen by the setup-time tuner
    std::vector<std::pair<int, float>> tune;  // (tile width, ms) measured at setup
    CUtensorMap mapA{}, mapB{};
    double flops_app = 0;        // algorithmic flops of one application's GEMMs: 2 P per kept operator row and pair
    double flops_deriv = 0;      // and of its derivative rows: 2 P3^2 per spatial product and pair
    // FFT form: pairs per observation cell in interaction-list order (CSR ooff)
    int32_t *fS = nullptr;       // [np] source cell of each pair
    int16_t *fo = nullptr;       // [np] its offset's index into the spectra
    int nfo = 0;                 // distinct offsets of the level
    int fC = 0;                  // frequencies per CTA of the products
    float2 *Khat = nullptr;      // [nfo][mu][fN] spectra of the circulant kernel samples, near future 1..mu
    float2 *Mhat = nullptr;      // [nc][fN] spectra of the moments of the current source interval
    float2 *Yhat = nullptr;      // [nc][mu][fN] products summed over each cell's interaction list
};

struct Fmm {
    bool on = false;
    struct cublasContext *blas = nullptr;  // cuBLAS handle (FP64 form)
    int L = 0, ps = 0, pt = 0, P3 = 0, P = 0, mu = 0, Lt = 0, nblk = 0, nd = 0, nslot = 0;
    int ngb = 0;                            // operator blocks applied as GEMMs (near future 1..mu)
    int R = 0, Rp = 0, Kp = 0;              // their rows ngb P, rows padded to 128, K padded to 64
    int nta = 0, ntb = 0, nprod = 0;        // tensor-core forms: split terms and products
    bool f16 = false;                       // precision 4: two FP16 terms with power-of-two scales
    bool fft = false;                       // precision 5: M2L blocks by the FFT (equispaced nodes, equal boxes)
    int fNs = 0, fNt = 0;                   // FFT form: grid points per spatial axis and in time
    int64_t fN = 0;                         // FFT form: grid points of one transform, fNs^3 fNt
    int prod[kTcMaxProd] = {0};
    int16_t *perm = nullptr;                // [48][P3] node permutation of each symmetry element
    int16_t *iperm = nullptr;               // [48][P3] its inverse
    double rho = 0;
    std::vector<FmmLevel> lev;
    double *At = nullptr, *As = nullptr, *Dv = nullptr, *Dn = nullptr;  // [ns][P3]
    double *tl = nullptr, *dtl = nullptr;  // [Lt][8] time basis at the interval's positions
    double *wk = nullptr;                   // [d+2] w^{kappa,d}
    double *Tm = nullptr;                   // [2][pt][pt] time transfer
    double *wt = nullptr;                   // [pt] time nodes (Chebyshev, or equispaced in the FFT form)
    double *far = nullptr;                  // [Lt][ns] far field of the current leaf interval
    double *Tq = nullptr, *Tu = nullptr;    // [ns][pt] P2M time sums of the folded histories (sorted order)
    int far_k = -1;                         // leaf interval the far field belongs to
    // plain stepping in the tensor-core forms: the deferred part of each
    // boundary's work runs on this second stream (fmm_boundary)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_urgent = nullptr, ev_deferred = nullptr;
    bool overlap = true;                    // tdbem_set_overlap
};

struct Pending {
    int phase;
    cudaEvent_t a, b;
};

enum { PH_RHS = 0, PH_NEAR = 1, PH_SOLVE = 2, PH_FAR = 3, PH_M2L = 4, PH_GEMM = 5, PH_COUNT = 6 };

struct Status {
    int code = TDBEM_OK;
    std::string msg;
};

}  // namespace tdbem

struct tdbem_ctx {
    tdbem_params P{};
    double cdt = 0.0;
    cudaStream_t user = nullptr;  // borrowed
    cudaStream_t s = nullptr;     // the context's own stream
    int dev = 0;
    std::string err;

    // host-side problem description
    int ns = 0, nv = 0;
    std::vector<double> xyz;
    std::vector<int32_t> tri;
    std::vector<int8_t> phi;
    std::vector<double> kbar;  // known-data samples f(t_a), a = 1..Nt-1
    tdbem::Incident inc{};
    tdbem::BsTable bs{};

    bool prepared = false;
    int alpha = 0;  // steps taken: the next step solves at t_{alpha+1}

    // device data
    double *d_xyz = nullptr;
    int32_t *d_tri = nullptr;
    double *d_V = nullptr;   // [ns][9] vertices / cdt
    double *d_X = nullptr;   // [ns][3] centroids / cdt
    double *d_xc = nullptr;  // [ns][3] centroids (physical)
    double *d_n = nullptr;   // [ns][3] the paper's normal (into V)
    int8_t *d_phi = nullptr;
    // pair lists: row i owns pairs [prow[i], prow[i+1]) with columns col[p]
    // (nullptr: all columns, j = p - prow[i]), cut into 32-pair blocks
    // [rowblk[i], rowblk[i+1])
    int64_t *d_prow = nullptr;   // [ns+1]
    int32_t *d_col = nullptr;    // [npairs] or nullptr
    int64_t *d_rowblk = nullptr; // [ns+1]
    int64_t nbt = 0;             // blocks in total
    uint16_t *d_meta = nullptr;  // [npairs] lag windows
    int32_t *d_btot = nullptr;   // [nbt] coefficients per 32-pair block
    int64_t *d_boff = nullptr;   // [nbt+1] first coefficient of each block (last: ncoef)
    int smax = 0;                // largest window length
    int gmax = 0;                // largest lag stored
    int near_wpr = 4;            // history sum: warps per row (1 for short rows)
    int64_t npairs = 0, ncoef = 0;
    int ku_kind = -1, kw_kind = -1;
    double *d_ku = nullptr, *d_kw = nullptr;
    double *d_u = nullptr, *d_q = nullptr;  // [nt][ns] histories
    bool split = false;                     // split-precision history sum
    float2 *d_us = nullptr, *d_qs = nullptr; // [nt][ns] float-pair copies (split only)
    // split form with near lists (FMM): the float-pair copies hold element
    // perm[p] at position p (the octree's Morton order), so a near list's
    // history gathers are contiguous runs; d_hpos[i] = position of element i,
    // d_hcol = the near pairs' columns as positions (nullptr otherwise)
    int32_t *d_hpos = nullptr, *d_hcol = nullptr;
    // near lists per leaf cell (every element of a cell has the same list):
    // element numbers d_ccol, sorted positions d_chcol, cell c from d_coff[c]
    int64_t *d_coff = nullptr;
    int32_t *d_ccol = nullptr, *d_chcol = nullptr;
    double *d_b = nullptr, *d_xa = nullptr, *d_xb = nullptr;
    int ell_w = 0;               // off-diagonal entries per row of the zero-lag store
    int jac_grid = 0;            // CTAs of the fused Jacobi launch (0: one launch per sweep)
    unsigned *d_bar = nullptr;   // its grid barrier: arrival count, generation
    double *d_aoff = nullptr;    // [ell_w][ns]
    int32_t *d_acol = nullptr;   // [ell_w][ns]
    double *d_ainv = nullptr;    // [ns]
    int solve_iters = 0;
    double contraction = 0.0;
    double *d_exc = nullptr;
    int exc_cap = 0;
    double *d_xout = nullptr;
    int xout_cap = 0;
    int *d_flag = nullptr;       // device error flags
    // learned SAI for the zero-lag solve (nullptr: Jacobi)
    double *sai_val = nullptr;   // [sai_w][ns]
    int32_t *sai_col = nullptr;  // [sai_w][ns]
    int sai_w = 0, sai_iters = 0;
    int sai_grid = 0;            // CTAs of the fused SAI launch (0: one launch per sweep)
    double *sai_gval = nullptr;  // [sai_gw][ns] G = I - M A (ELL)
    int32_t *sai_gcol = nullptr; // [sai_gw][ns] its columns (-1: unused slot)
    int sai_gw = 0;
    double *sai_cb = nullptr;    // [ns] c = M b of the current step
    double sai_contraction = 0.0;
    double *d_r = nullptr;       // [ns] residual
    int *d_alpha = nullptr;      // device-side step counter for graph-replayed steps
    bool alpha_dev_on = false;   // kernels read the step from d_alpha (while capturing)
    cudaGraphExec_t graph = nullptr;  // one captured step (direct path)
    std::vector<void *> allocs;  // every cudaMalloc of the context

    tdbem::Tree tree;  // built when P.depth > 0
    tdbem::Fmm fmm;    // algo 1

    // timing
    std::vector<tdbem::Pending> pending;
    std::vector<cudaEvent_t> pool;
    double ms[tdbem::PH_COUNT] = {0, 0, 0, 0, 0, 0};
    int64_t launches[tdbem::PH_COUNT] = {0, 0, 0, 0, 0, 0};
    double m2l_flops = 0.0;  // algorithmic flops of the M2L GEMMs since the last reset
    double gemm_tc_flops = 0.0;  // tensor-pipe flops the split requires (products x algorithmic)
    int64_t far_kernels = 0;     // kernel launches of the far-field passes (FP64 form: DGEMMs count once)
    int64_t steps_total = 0;
    double ms_prepare = 0.0;
};

namespace tdbem {

// Kernel launchers (coef.cu)
cudaError_t launch_geometry(tdbem_ctx *c);
cudaError_t launch_windows(tdbem_ctx *c, int *d_maxcnt, int *d_maxg0, int *d_gtop);
cudaError_t launch_coefficients(tdbem_ctx *c);
cudaError_t launch_zero_lag(tdbem_ctx *c, bool count_only);
void set_bspline_table(const BsTable &T, cudaStream_t s);
cudaError_t launch_known_collocation(tdbem_ctx *c, const double *d_f);

// Hierarchy (tree.cu)
cudaError_t build_tree(tdbem_ctx *c, std::string &why);
cudaError_t build_near_lists(tdbem_ctx *c);

// Space-time FMM (fmm.cu)
cudaError_t fmm_setup(tdbem_ctx *c, std::string &why);
cudaError_t fmm_boundary(tdbem_ctx *c, int k, bool graph = false);
cudaError_t fmm_join(tdbem_ctx *c);
cudaError_t fft_m2l_level_setup(tdbem_ctx *c, FmmLevel &V, const std::vector<int32_t> &pS,
                                const std::vector<int16_t> &po, const std::vector<int32_t> &codes, double Tdt,
                                std::string &why);
cudaError_t fft_m2l_forward(tdbem_ctx *c, FmmLevel &V, cudaStream_t s, const StepWhen &w);
cudaError_t fft_m2l_apply(tdbem_ctx *c, FmmLevel &V, int kl, int lb, int le, cudaStream_t s, const StepWhen &w);
// Phase timer hooks for fmm.cu (events on the context's stream).
void phase_begin(tdbem_ctx *c, cudaEvent_t *e);
void phase_end(tdbem_ctx *c, int phase, cudaEvent_t e);
void fmm_free(tdbem_ctx *c);
void free_tree(tdbem_ctx *c);

// Kernel launchers (march.cu)
cudaError_t launch_near_sum(tdbem_ctx *c, int alpha, const double *d_exc, const double *d_far);
cudaError_t launch_jacobi(tdbem_ctx *c, int alpha, int it, int last);
cudaError_t setup_jacobi_fused(tdbem_ctx *c);
cudaError_t launch_jacobi_fused(tdbem_ctx *c, int alpha);
cudaError_t launch_gather_x(tdbem_ctx *c, int a0, int nsteps, double *x);
cudaError_t launch_alpha_next(tdbem_ctx *c);
cudaError_t launch_sai_sweep(tdbem_ctx *c, int alpha, int it);
cudaError_t launch_sai_fused(tdbem_ctx *c, int alpha);
cudaError_t launch_split_coefficients(tdbem_ctx *c);
cudaError_t launch_split_histories(tdbem_ctx *c);

}  // namespace tdbem
