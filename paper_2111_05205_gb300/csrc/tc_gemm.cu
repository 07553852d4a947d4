// Split-precision GEMM on the 5th-generation tensor cores (tcgen05) for the
// M2L contraction of the space-time FMM (Section 4.2, Eq. m2l_actual in
// matrix form: the operator stack of one cell offset times the moments of
// every interaction pair with that offset).
//
//   C[c_off + j ldc + i] = sum_{(s,t) in products} A_s[a_row + i, :] . B_t[b_row + j, :]
//
// for i < rows (<= 128), j < cols (<= BN) of every tile.  A_s and B_t are
// the terms of a split of FP64 operands into BF16 (or FP16) numbers,
// x ~ x_0 + x_1 + x_2 with x_k = round(x - x_0 - .. - x_{k-1}); products
// (s, t) with s + t < n give about 8n significant bits.  Both operands are
// K-major (each row holds its K values contiguously), so one 128-byte row of
// a 64-wide K chunk is one swizzle row of the SW128 layout.
//
// Persistent: one CTA per SM, each taking tiles blockIdx.x, blockIdx.x +
// gridDim.x, ...; 6 warps:
//   warp 0 (one thread): TMA producer; per K chunk it loads every term's
//     128 x 64 A tile and BN x 64 B tile into a ring of shared-memory stages
//     (cp.async.bulk.tensor, 128-byte swizzle, completion on an mbarrier),
//     running ahead across tile boundaries;
//   warp 1: allocates 2 BN TMEM columns (two accumulators); one thread
//     issues tcgen05.mma (M = 128, N = BN, K = 16, FP32 accumulate in TMEM)
//     for every product and K step of a stage, tcgen05.commit frees the
//     stage, and a commit per tile hands the accumulator to the epilogue;
//   warps 2-5: epilogue; each reads its 32 TMEM lanes (tcgen05.ld 32x32b),
//     returns the accumulator to the MMA warp and stores the FP32 results,
//     one coalesced 128-byte row per column, while the MMAs of the next
//     tile run in the other accumulator.
// Every mbarrier wait gives up after kWaitNs of global time, sets bit 3 of
// *err and lets the CTA finish: TMA copies in flight are waited for (with
// the same bound), the MMAs issued are drained and the TMEM columns are
// freed before the CTA exits.
#include <cuda.h>

#include <algorithm>

#include "tdbem_internal.cuh"

namespace tdbem {

namespace {

constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits until the phase of the given parity completed; false after kWaitNs.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_test(bar, parity))
        if (global_ns() - t0 > kWaitNs) return false;
    return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows
// of 128 bytes, 8-row groups 1024 bytes apart (stride byte offset), tile
// base 1024-byte aligned; bits 46-47 hold the descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1u << 16) | ((uint64_t)(1024u >> 4) << 32) |
           ((uint64_t)1u << 46) | ((uint64_t)2u << 61);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A and
// B format (bits 7-9, 10-12: 0 = FP16, 1 = BF16), both K-major (bits 15, 16 =
// 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t f16_idesc(int fmt, int m, int n)
{
    return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

}  // namespace

template <int BN>
__global__ void __launch_bounds__(192, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const TcGemmArgs g)
{
    // graph-replayed steps: the whole grid leaves before touching shared
    // memory or TMEM when this step has no M2L at the GEMM's level
    if (g.when.alpha && when_interval(g.when) < 0) return;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    constexpr uint32_t kATile = kTcBM * 128, kBTile = BN * 128;
    const uint32_t stage_bytes = g.nta * kATile + g.ntb * kBTile;
    const int nstage = g.nstage;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)nstage * stage_bytes);
    // full[s], empty[s]; accumulator full[2] / empty[2]; MMA drain
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + nstage), accf0 = smem_u32(bars + 2 * nstage),
                   acce0 = smem_u32(bars + 2 * nstage + 2), drain = smem_u32(bars + 2 * nstage + 4);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * nstage + 5);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < nstage; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(accf0 + 8 * b, 1);
            mbar_init(acce0 + 8 * b, 4);  // one arrival per epilogue warp
        }
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"((uint32_t)(2 * BN))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int K = g.kchunks;
    const int ntiles = g.ntiles;

    if (warp == 0) {
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
            int it = 0;  // K chunks issued by this CTA
            bool ok = true;
            for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
                const TcTile t = g.tiles[tile];
                for (int kc = 0; kc < K; ++kc, ++it) {
                    const int s = it % nstage;
                    if (it >= nstage && !mbar_wait(empty0 + 8 * s, ((it / nstage) - 1) & 1)) {
                        atomicOr(g.err, 8);
                        ok = false;
                        break;
                    }
                    const uint32_t st = smem_u32(smem + (size_t)s * stage_bytes);
                    mbar_expect_tx(full0 + 8 * s, stage_bytes);
                    for (int a = 0; a < g.nta; ++a)
                        tma_load_2d(st + a * kATile, &tmA, kc * kTcBK, t.a_row + a * g.a_term_rows, full0 + 8 * s);
                    for (int b = 0; b < g.ntb; ++b)
                        tma_load_2d(st + g.nta * kATile + b * kBTile, &tmB, kc * kTcBK, t.b_row + b * g.b_term_rows,
                                    full0 + 8 * s);
                }
            }
            // every copy issued has landed before the CTA may exit
            for (int k = (it > nstage ? it - nstage : 0); k < it; ++k)
                if (!mbar_wait(full0 + 8 * (k % nstage), (k / nstage) & 1)) atomicOr(g.err, 8);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = f16_idesc(g.fmt, kTcBM, BN);
            int it = 0, j = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++j) {
                const int b = j & 1;
                // the epilogue has read this accumulator's previous tile
                if (j >= 2 && !mbar_wait(acce0 + 8 * b, ((j >> 1) - 1) & 1)) {
                    atomicOr(g.err, 8);
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(b * BN);
                for (int kc = 0; kc < K; ++kc, ++it) {
                    const int s = it % nstage;
                    if (!mbar_wait(full0 + 8 * s, (it / nstage) & 1)) {
                        atomicOr(g.err, 8);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t st = smem_u32(smem + (size_t)s * stage_bytes);
                    for (int p = 0; p < g.nprod; ++p) {
                        const uint64_t da = sw128_desc(st + (g.prod[p] >> 4) * kATile);
                        const uint64_t db = sw128_desc(st + g.nta * kATile + (g.prod[p] & 15) * kBTile);
#pragma unroll
                        for (int kk = 0; kk < kTcBK / 16; ++kk)
                            tc_mma(d, da + 2 * kk, db + 2 * kk, idesc, (kc | p | kk) != 0);
                    }
                    tc_commit(empty0 + 8 * s);
                }
                if (ok) tc_commit(accf0 + 8 * b);
            }
            // every MMA issued has completed before the columns are freed
            tc_commit(drain);
            if (!mbar_wait(drain, 0)) atomicOr(g.err, 8);
        }
    } else {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. 32 (w % 4) + 31 of
        // the tile's accumulator, then hands the columns back to the MMA
        // warp, so the next-but-one tile's MMAs overlap these stores
        const int q = warp & 3, row = 32 * q + lane;
        int j = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++j) {
            const int b = j & 1;
            // warp-uniform decision: the TMEM loads below are .sync.aligned
            const bool ok = __all_sync(0xffffffffu, mbar_wait(accf0 + 8 * b, (j >> 1) & 1));
            tc_fence_after();
            if (!ok) {
                if (lane == 0) atomicOr(g.err, 8);
                break;
            }
            const TcTile t = g.tiles[tile];
            float *out = g.C + t.c_off + row;
            const float sa = (g.a_scale && row < t.rows) ? g.a_scale[t.a_row + row] : 1.f;
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 32) {
                uint32_t r[32];
                tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * BN + c0), r);
                if (row < t.rows) {
                    if (g.a_scale) {
#pragma unroll
                        for (int x = 0; x < 32; ++x)
                            if (c0 + x < t.cols)
                                out[(int64_t)(c0 + x) * g.ldc] =
                                    __uint_as_float(r[x]) * sa * g.b_scale[t.b_row + c0 + x];
                    } else {
#pragma unroll
                        for (int x = 0; x < 32; ++x)
                            if (c0 + x < t.cols) out[(int64_t)(c0 + x) * g.ldc] = __uint_as_float(r[x]);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acce0 + 8 * b);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)(2 * BN))
                     : "memory");
    }
}

namespace {

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn()
{
    static EncodeTiled fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    }
    return fn;
}

}  // namespace

cudaError_t tc_make_map(CUtensorMap *map, const void *base, int64_t rows, int kp, int box_rows)
{
    EncodeTiled fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    if (((uintptr_t)base & 15) || kp % kTcBK || rows < 1 || rows > 0x7fffffffLL) return cudaErrorInvalidValue;
    cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)kp * 2};
    cuuint32_t box[2] = {(cuuint32_t)kTcBK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

int tc_stages(int nta, int ntb, int bn)
{
    const int stage = nta * kTcBM * 128 + ntb * bn * 128;
    int n = (kTcSmemBudget - 1024 - 256) / stage;
    return n > 6 ? 6 : n;
}

size_t tc_smem_bytes(int nta, int ntb, int bn, int nstage)
{
    return 1024 + (size_t)nstage * (nta * kTcBM * 128 + ntb * bn * 128) + 8 * (2 * nstage + 5) + 16;
}

cudaError_t tc_gemm_launch(const CUtensorMap &ta, const CUtensorMap &tb, const TcGemmArgs &a, int ntiles, int bn,
                           cudaStream_t s, int sm_div)
{
    if (ntiles <= 0) return cudaSuccess;
    if (a.nstage < 1 || a.nta < 1 || a.nta > kTcMaxTerms || a.ntb < 1 || a.ntb > kTcMaxTerms || a.nprod < 1 ||
        a.nprod > kTcMaxProd || (a.fmt != 0 && a.fmt != 1))
        return cudaErrorInvalidValue;
    for (int p = 0; p < a.nprod; ++p)
        if ((a.prod[p] >> 4) >= a.nta || (a.prod[p] & 15) >= a.ntb) return cudaErrorInvalidValue;
    const size_t shm = tc_smem_bytes(a.nta, a.ntb, bn, a.nstage);
    if (shm > (size_t)kTcSmemBudget) return cudaErrorInvalidValue;
    // persistent: one CTA per SM (the shared-memory ring fills the SM), each
    // taking every gridDim-th tile
    static int nsm = 0;
    if (!nsm) {
        int dev = 0;
        cudaError_t e0 = cudaGetDevice(&dev);
        if (e0 == cudaSuccess) e0 = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e0 != cudaSuccess || nsm < 1) return e0 != cudaSuccess ? e0 : cudaErrorInvalidValue;
    }
    TcGemmArgs g = a;
    g.ntiles = ntiles;
    const int grid = std::min(ntiles, std::max(1, nsm / std::max(sm_div, 1)));
    cudaError_t e;
    if (bn == 128) {
        e = cudaFuncSetAttribute(k_tc_gemm<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemBudget);
        if (e != cudaSuccess) return e;
        k_tc_gemm<128><<<grid, 192, shm, s>>>(ta, tb, g);
    } else if (bn == 256) {
        e = cudaFuncSetAttribute(k_tc_gemm<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemBudget);
        if (e != cudaSuccess) return e;
        k_tc_gemm<256><<<grid, 192, shm, s>>>(ta, tb, g);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace tdbem

// Self-check of the kernel on caller data (see tdbem.h).
extern "C" int tdbem_tc_gemm_check(int32_t m, int32_t n, int32_t k, int32_t nta, int32_t ntb, const int32_t *prod,
                                   int32_t nprod, int32_t fmt, int32_t bn, const uint16_t *a, const uint16_t *b,
                                   float *c)
{
    using namespace tdbem;
    if (m < 1 || n < 1 || k < 1 || nta < 1 || nta > kTcMaxTerms || ntb < 1 || ntb > kTcMaxTerms || nprod < 1 ||
        nprod > kTcMaxProd || (fmt != 0 && fmt != 1) || (bn != 128 && bn != 256) || !prod || !a || !b || !c)
        return TDBEM_ERR_ARG;
    if ((int64_t)m * nta > 0x7fffffff || (int64_t)n * ntb > 0x7fffffff || (int64_t)m * n > (1LL << 31))
        return TDBEM_ERR_ARG;
    for (int p = 0; p < nprod; ++p)
        if ((prod[p] >> 4) >= nta || (prod[p] & 15) >= ntb || prod[p] < 0) return TDBEM_ERR_ARG;
    const int kp = (k + kTcBK - 1) / kTcBK * kTcBK;
    std::vector<uint16_t> ha((size_t)nta * m * kp, 0), hb((size_t)ntb * n * kp, 0);
    for (int64_t r = 0; r < (int64_t)nta * m; ++r)
        for (int x = 0; x < k; ++x) ha[r * kp + x] = a[r * k + x];
    for (int64_t r = 0; r < (int64_t)ntb * n; ++r)
        for (int x = 0; x < k; ++x) hb[r * kp + x] = b[r * k + x];
    std::vector<TcTile> tiles;
    for (int i0 = 0; i0 < m; i0 += kTcBM)
        for (int j0 = 0; j0 < n; j0 += bn)
            tiles.push_back({i0, j0, std::min(kTcBM, m - i0), std::min(bn, n - j0), (int64_t)j0 * m + i0});
    void *da = nullptr, *db = nullptr, *dc = nullptr, *dt = nullptr;
    int *derr = nullptr;
    cudaStream_t s = nullptr;
    int status = TDBEM_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&da, ha.size() * 2);
    if (e == cudaSuccess) e = cudaMalloc(&db, hb.size() * 2);
    if (e == cudaSuccess) e = cudaMalloc(&dc, (size_t)m * n * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&dt, tiles.size() * sizeof(TcTile));
    if (e == cudaSuccess) e = cudaMalloc(&derr, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyAsync(da, ha.data(), ha.size() * 2, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(db, hb.data(), hb.size() * 2, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dt, tiles.data(), tiles.size() * sizeof(TcTile), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(dc, 0, (size_t)m * n * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(derr, 0, sizeof(int), s);
    CUtensorMap ta, tb;
    if (e == cudaSuccess) e = tc_make_map(&ta, da, (int64_t)nta * m, kp, kTcBM);
    if (e == cudaSuccess) e = tc_make_map(&tb, db, (int64_t)ntb * n, kp, bn);
    if (e == cudaSuccess) {
        TcGemmArgs g{};
        g.nta = nta;
        g.ntb = ntb;
        g.a_term_rows = m;
        g.b_term_rows = n;
        g.nprod = nprod;
        for (int p = 0; p < nprod; ++p) g.prod[p] = prod[p];
        g.kchunks = kp / kTcBK;
        g.nstage = tc_stages(nta, ntb, bn);
        g.fmt = fmt;
        g.ldc = m;
        g.C = (float *)dc;
        g.tiles = (const TcTile *)dt;
        g.err = derr;
        e = tc_gemm_launch(ta, tb, g, (int)tiles.size(), bn, s);
    }
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(c, dc, (size_t)m * n * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) status = TDBEM_ERR_CUDA;
    else if (herr) status = TDBEM_ERR_TIMEOUT;
    cudaFree(da);
    cudaFree(db);
    cudaFree(dc);
    cudaFree(dt);
    cudaFree(derr);
    if (s) cudaStreamDestroy(s);
    return status;
}
