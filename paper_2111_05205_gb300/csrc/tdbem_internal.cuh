// Internal declarations shared by the translation units of libtdbem.
#pragma once

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
constexpr int kMaxCnt = 15;
// Zero-lag matrix: off-diagonal entries per row (ELL width).
constexpr int kEllWidth = 8;

// Coefficient kinds (bit positions in a kinds mask).
enum { KIND_CU = 0, KIND_CW = 1, KIND_UB = 2, KIND_WB = 3 };

struct Incident {
    int on;
    int bie;
    double k[3];
    double t0, width, c, dt;
};

struct Pending {
    int phase;
    cudaEvent_t a, b;
};

enum { PH_RHS = 0, PH_NEAR = 1, PH_SOLVE = 2, PH_COUNT = 3 };

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
    uint16_t *d_meta = nullptr;  // [ns][ns] lag windows
    int32_t *d_btot = nullptr;   // [ns][nblk] coefficients per 32-pair block
    int64_t *d_boff = nullptr;   // [ns][nblk] first coefficient of each block
    int nblk = 0;
    int smax = 0;                // largest window length
    int gmax = 0;                // largest lag stored
    int64_t npairs = 0, ncoef = 0;
    int ku_kind = -1, kw_kind = -1;
    double *d_ku = nullptr, *d_kw = nullptr;
    double *d_u = nullptr, *d_q = nullptr;  // [nt][ns] histories
    double *d_b = nullptr, *d_xa = nullptr, *d_xb = nullptr;
    double *d_aoff = nullptr;    // [kEllWidth][ns]
    int32_t *d_acol = nullptr;   // [kEllWidth][ns]
    double *d_ainv = nullptr;    // [ns]
    int solve_iters = 0;
    double contraction = 0.0;
    double *d_exc = nullptr;
    int exc_cap = 0;
    double *d_xout = nullptr;
    int xout_cap = 0;
    int *d_flag = nullptr;       // device error flags
    std::vector<void *> allocs;  // every cudaMalloc of the context

    // timing
    std::vector<tdbem::Pending> pending;
    std::vector<cudaEvent_t> pool;
    double ms[tdbem::PH_COUNT] = {0, 0, 0};
    int64_t launches[tdbem::PH_COUNT] = {0, 0, 0};
    int64_t steps_total = 0;
    double ms_prepare = 0.0;
};

namespace tdbem {

// Kernel launchers (coef.cu)
cudaError_t launch_geometry(tdbem_ctx *c);
cudaError_t launch_windows(tdbem_ctx *c, int *d_maxcnt, int *d_maxg0, int *d_gtop);
cudaError_t launch_block_totals(tdbem_ctx *c);
cudaError_t launch_coefficients(tdbem_ctx *c);
cudaError_t launch_zero_lag(tdbem_ctx *c);
void set_bspline_table(const BsTable &T, cudaStream_t s);
cudaError_t launch_known_collocation(tdbem_ctx *c, const double *d_f);

// Kernel launchers (march.cu)
cudaError_t launch_near_sum(tdbem_ctx *c, int alpha, const double *d_exc);
cudaError_t launch_jacobi(tdbem_ctx *c, int alpha, int it, int last);
cudaError_t launch_gather_x(tdbem_ctx *c, int a0, int nsteps, double *x);

}  // namespace tdbem
