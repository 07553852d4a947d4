// Spatial hierarchy of the space-time FMM (Section 3; interaction lists of
// Section 4.2, Remark precomp and Algorithm 1), built on the device:
//   root cube from the collocation points (lo = componentwise minimum,
//   side = largest extent x (1 + 2^-20)); leaf coordinates
//   floor((x - lo) / side * 2^L) in FP64 with every operation rounded on its
//   own (no contraction), clamped; Morton keys; element order by (key,
//   index); per level the occupied cells, their neighbours (|offset| <= 1)
//   and interaction lists (children of the parent's neighbours that are not
//   neighbours, offsets in [-3,3]^3 minus [-1,1]^3); leaf near lists.
// All of it is integer data that must match the reference definition bit
// for bit.
#include "tdbem_internal.cuh"

namespace tdbem {

constexpr int kScanThreads = 1024;

// lo[0..2] = min of the centroids, box[3] = side.
__global__ void k_root_box(int ns, const double *__restrict__ xc, double *box)
{
    __shared__ double smin[3][kScanThreads / 32], smax[3][kScanThreads / 32];
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = threadIdx.x; i < ns; i += blockDim.x)
        for (int a = 0; a < 3; ++a) {
            double v = xc[3 * i + a];
            mn[a] = fmin(mn[a], v);
            mx[a] = fmax(mx[a], v);
        }
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int a = 0; a < 3; ++a) {
        for (int o = 16; o; o >>= 1) {
            mn[a] = fmin(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
            mx[a] = fmax(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
        }
        if (lane == 0) {
            smin[a][w] = mn[a];
            smax[a][w] = mx[a];
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ext = 0.0;
        for (int a = 0; a < 3; ++a) {
            double lo = INFINITY, hi = -INFINITY;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
                lo = fmin(lo, smin[a][k]);
                hi = fmax(hi, smax[a][k]);
            }
            box[a] = lo;
            ext = fmax(ext, __dsub_rn(hi, lo));
        }
        box[3] = __dmul_rn(ext, 1.0 + 0x1p-20);
    }
}

__device__ __forceinline__ uint64_t morton3(uint32_t x, uint32_t y, uint32_t z, int bits)
{
    uint64_t k = 0;
    for (int b = 0; b < bits; ++b) {
        k |= (uint64_t)((x >> b) & 1u) << (3 * b);
        k |= (uint64_t)((y >> b) & 1u) << (3 * b + 1);
        k |= (uint64_t)((z >> b) & 1u) << (3 * b + 2);
    }
    return k;
}

__device__ __forceinline__ void demorton3(uint64_t k, int bits, int c[3])
{
    c[0] = c[1] = c[2] = 0;
    for (int b = 0; b < bits; ++b)
        for (int a = 0; a < 3; ++a) c[a] |= (int)((k >> (3 * b + a)) & 1u) << b;
}

__global__ void k_leaf_keys(int ns, int L, const double *__restrict__ xc, const double *__restrict__ box,
                            uint64_t *key)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns) return;
    const double n = (double)(1 << L);
    uint32_t c[3];
    for (int a = 0; a < 3; ++a) {
        double t = __dmul_rn(__ddiv_rn(__dsub_rn(xc[3 * i + a], box[a]), box[3]), n);
        long long v = (long long)floor(t);
        v = v < 0 ? 0 : (v > (1 << L) - 1 ? (1 << L) - 1 : v);
        c[a] = (uint32_t)v;
    }
    key[i] = morton3(c[0], c[1], c[2], L);
}

// Rank of element i in the order (key, index): the number of elements that
// precede it; perm[rank] = i.  Composite keys are unique, so the counting
// is exact and the result does not depend on the schedule.
__global__ void k_rank(int ns, const uint64_t *__restrict__ key, int32_t *perm)
{
    __shared__ uint64_t tile[256];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t ki = (i < ns) ? key[i] : 0;
    int r = 0;
    for (int base = 0; base < ns; base += 256) {
        int j = base + threadIdx.x;
        tile[threadIdx.x] = (j < ns) ? key[j] : 0;
        __syncthreads();
        int lim = min(256, ns - base);
        for (int t = 0; t < lim; ++t) {
            uint64_t kj = tile[t];
            int jj = base + t;
            r += (kj < ki) || (kj == ki && jj < i);
        }
        __syncthreads();
    }
    if (i < ns) perm[r] = i;
}

// Single-block exclusive scan of flags[0..n) into out[0..n], out[n] = total.
__global__ void k_scan(int n, const int32_t *__restrict__ in, int32_t *out)
{
    __shared__ int32_t part[kScanThreads];
    int per = (n + kScanThreads - 1) / kScanThreads;
    int b = threadIdx.x * per, e = min(n, b + per);
    int s = 0;
    for (int k = b; k < e; ++k) s += in[k];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < kScanThreads; o <<= 1) {
        int v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int run = part[threadIdx.x] - s;
    for (int k = b; k < e; ++k) {
        out[k] = run;
        run += in[k];
    }
    if (threadIdx.x == kScanThreads - 1) out[n] = part[kScanThreads - 1];
}

// Cell boundaries of a level in the sorted element order.
__global__ void k_cell_flags(int ns, int shift, const uint64_t *__restrict__ key, const int32_t *__restrict__ perm,
                             int32_t *flag)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= ns) return;
    uint64_t k = key[perm[p]] >> shift;
    flag[p] = (p == 0) || (k != (key[perm[p - 1]] >> shift));
}

__global__ void k_cell_fill(int ns, int shift, const uint64_t *__restrict__ key, const int32_t *__restrict__ perm,
                            const int32_t *__restrict__ flag, const int32_t *__restrict__ pos, uint64_t *ckey,
                            int32_t *cstart, int32_t *ecell)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= ns) return;
    int c = pos[p] + flag[p] - 1;  // cell index of position p
    ecell[p] = c;
    if (flag[p]) {
        ckey[c] = key[perm[p]] >> shift;
        cstart[c] = p;
    }
}

__device__ __forceinline__ int find_key(const uint64_t *__restrict__ keys, int n, uint64_t k)
{
    int lo = 0, hi = n - 1;
    while (lo <= hi) {
        int m = (lo + hi) >> 1;
        uint64_t v = keys[m];
        if (v == k) return m;
        if (v < k)
            lo = m + 1;
        else
            hi = m - 1;
    }
    return -1;
}

// Neighbours of every cell of a level: nbr[c*27 ..], ordered by key.
__global__ void k_neighbours(int nc, int lev, const uint64_t *__restrict__ ckey, int32_t *nbr, int32_t *ncount)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    int co[3];
    demorton3(ckey[c], lev, co);
    const int n = 1 << lev;
    int found[27];
    int m = 0;
    for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dz = -1; dz <= 1; ++dz) {
                int x = co[0] + dx, y = co[1] + dy, z = co[2] + dz;
                if (x < 0 || y < 0 || z < 0 || x >= n || y >= n || z >= n) continue;
                int idx = find_key(ckey, nc, morton3(x, y, z, lev));
                if (idx >= 0) found[m++] = idx;
            }
    // cell indices follow key order, so sorting indices sorts keys
    for (int a = 1; a < m; ++a)
        for (int b = a; b > 0 && found[b] < found[b - 1]; --b) {
            int t = found[b];
            found[b] = found[b - 1];
            found[b - 1] = t;
        }
    for (int a = 0; a < m; ++a) nbr[(int64_t)c * 27 + a] = found[a];
    ncount[c] = m;
}

// Interaction list of every cell of level lev >= 2: il[c*189 ..], by key.
__global__ void k_interaction_list(int nc, int lev, const uint64_t *__restrict__ ckey, int npc,
                                   const uint64_t *__restrict__ pkey, const int32_t *__restrict__ pnbr,
                                   const int32_t *__restrict__ pncount, int32_t *il, int32_t *ilcount, int *flag)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    int co[3];
    demorton3(ckey[c], lev, co);
    int p = find_key(pkey, npc, ckey[c] >> 3);
    int m = 0;
    int32_t *out = il + (int64_t)c * 189;
    for (int a = 0; a < pncount[p]; ++a) {
        uint64_t pk = pkey[pnbr[(int64_t)p * 27 + a]];
        for (int ch = 0; ch < 8; ++ch) {
            uint64_t kk = (pk << 3) | (uint64_t)ch;
            int idx = find_key(ckey, nc, kk);
            if (idx < 0) continue;
            int q[3];
            demorton3(kk, lev, q);
            int d = max(abs(q[0] - co[0]), max(abs(q[1] - co[1]), abs(q[2] - co[2])));
            if (d <= 1) continue;
            if (m < 189)
                out[m++] = idx;
            else
                atomicOr(flag, 8);
        }
    }
    for (int a = 1; a < m; ++a)
        for (int b = a; b > 0 && out[b] < out[b - 1]; --b) {
            int t = out[b];
            out[b] = out[b - 1];
            out[b - 1] = t;
        }
    ilcount[c] = m;
}

// Builds the hierarchy of depth c->P.depth on the device (synchronous).
cudaError_t build_tree(tdbem_ctx *c, std::string &why)
{
    const int ns = c->ns, L = c->P.depth;
    cudaStream_t s = c->s;
    cudaError_t e;
#define TRY(x)                         \
    do {                               \
        e = (x);                       \
        if (e != cudaSuccess) return e; \
    } while (0)
    TRY(cudaMalloc(&c->tree.box, 4 * sizeof(double)));
    TRY(cudaMalloc(&c->tree.key, ns * sizeof(uint64_t)));
    TRY(cudaMalloc(&c->tree.perm, ns * sizeof(int32_t)));
    int32_t *flag = nullptr, *pos = nullptr;
    TRY(cudaMalloc(&flag, ns * sizeof(int32_t)));
    TRY(cudaMalloc(&pos, (ns + 1) * sizeof(int32_t)));
    k_root_box<<<1, kScanThreads, 0, s>>>(ns, c->d_xc, c->tree.box);
    k_leaf_keys<<<(ns + 127) / 128, 128, 0, s>>>(ns, L, c->d_xc, c->tree.box, c->tree.key);
    k_rank<<<(ns + 255) / 256, 256, 0, s>>>(ns, c->tree.key, c->tree.perm);
    TRY(cudaGetLastError());
    c->tree.levels.assign(L + 1, TreeLevel{});
    for (int lev = 0; lev <= L; ++lev) {
        TreeLevel &T = c->tree.levels[lev];
        int shift = 3 * (L - lev);
        k_cell_flags<<<(ns + 255) / 256, 256, 0, s>>>(ns, shift, c->tree.key, c->tree.perm, flag);
        k_scan<<<1, kScanThreads, 0, s>>>(ns, flag, pos);
        int nc = 0;
        TRY(cudaMemcpyAsync(&nc, pos + ns, sizeof(int), cudaMemcpyDeviceToHost, s));
        TRY(cudaStreamSynchronize(s));
        T.nc = nc;
        TRY(cudaMalloc(&T.ckey, nc * sizeof(uint64_t)));
        TRY(cudaMalloc(&T.cstart, (nc + 1) * sizeof(int32_t)));
        TRY(cudaMalloc(&T.ecell, ns * sizeof(int32_t)));
        TRY(cudaMalloc(&T.nbr, (size_t)nc * 27 * sizeof(int32_t)));
        TRY(cudaMalloc(&T.ncount, nc * sizeof(int32_t)));
        k_cell_fill<<<(ns + 255) / 256, 256, 0, s>>>(ns, shift, c->tree.key, c->tree.perm, flag, pos, T.ckey,
                                                    T.cstart, T.ecell);
        TRY(cudaMemcpyAsync(T.cstart + nc, &c->ns, sizeof(int32_t), cudaMemcpyHostToDevice, s));
        k_neighbours<<<(nc + 127) / 128, 128, 0, s>>>(nc, lev, T.ckey, T.nbr, T.ncount);
        if (lev >= 2) {
            TreeLevel &P = c->tree.levels[lev - 1];
            TRY(cudaMalloc(&T.il, (size_t)nc * 189 * sizeof(int32_t)));
            TRY(cudaMalloc(&T.ilcount, nc * sizeof(int32_t)));
            k_interaction_list<<<(nc + 127) / 128, 128, 0, s>>>(nc, lev, T.ckey, P.nc, P.ckey, P.nbr, P.ncount,
                                                                T.il, T.ilcount, c->d_flag);
        }
        TRY(cudaGetLastError());
        TRY(cudaStreamSynchronize(s));
    }
    cudaFree(flag);
    cudaFree(pos);
    int fl = 0;
    TRY(cudaMemcpy(&fl, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (fl & 8) why = "interaction list longer than 189";
#undef TRY
    return cudaSuccess;
}

// Leaf cell (cell index at level L) of each element, in element numbering.
__global__ void k_elem_cell(int ns, const int32_t *__restrict__ perm, const int32_t *__restrict__ ecell, int32_t *e2c)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < ns) e2c[perm[p]] = ecell[p];
}

// Near pairs of element i: every element of the leaf cells neighbouring
// leaf(i), cells in key order and elements in sorted order within a cell.
__global__ void k_near_count(int ns, const int32_t *__restrict__ e2c, const int32_t *__restrict__ nbr,
                             const int32_t *__restrict__ ncount, const int32_t *__restrict__ cstart, int64_t *cnt)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns) return;
    int c = e2c[i];
    int64_t n = 0;
    for (int a = 0; a < ncount[c]; ++a) {
        int m = nbr[(int64_t)c * 27 + a];
        n += cstart[m + 1] - cstart[m];
    }
    cnt[i] = n;
}

__global__ void k_near_fill(int ns, const int32_t *__restrict__ e2c, const int32_t *__restrict__ nbr,
                            const int32_t *__restrict__ ncount, const int32_t *__restrict__ cstart,
                            const int32_t *__restrict__ perm, const int64_t *__restrict__ prow, int32_t *col,
                            int32_t *hcol)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns) return;
    int c = e2c[i];
    int64_t o = prow[i];
    for (int a = 0; a < ncount[c]; ++a) {
        int m = nbr[(int64_t)c * 27 + a];
        for (int p = cstart[m]; p < cstart[m + 1]; ++p) {
            if (hcol) hcol[o] = p;  // the element's position in the sorted order
            col[o++] = perm[p];
        }
    }
}

// The near list is the same for every element of a leaf cell: per cell c,
// the elements of its neighbour cells (key order, sorted order within a
// cell) as element numbers ccol and as sorted positions chcol, from
// coff[c].  (The per-step history sum reads these instead of per-pair
// columns.)
__global__ void k_cell_near_count(int nc, const int32_t *__restrict__ nbr, const int32_t *__restrict__ ncount,
                                  const int32_t *__restrict__ cstart, int64_t *cnt)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    int64_t n = 0;
    for (int a = 0; a < ncount[c]; ++a) {
        int m = nbr[(int64_t)c * 27 + a];
        n += cstart[m + 1] - cstart[m];
    }
    cnt[c] = n;
}

__global__ void k_cell_near_fill(int nc, const int32_t *__restrict__ nbr, const int32_t *__restrict__ ncount,
                                 const int32_t *__restrict__ cstart, const int32_t *__restrict__ perm,
                                 const int64_t *__restrict__ coff, int32_t *ccol, int32_t *chcol)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    int64_t o = coff[c];
    for (int a = 0; a < ncount[c]; ++a) {
        int m = nbr[(int64_t)c * 27 + a];
        for (int p = cstart[m]; p < cstart[m + 1]; ++p) {
            chcol[o] = p;
            ccol[o++] = perm[p];
        }
    }
}

__global__ void k_invert_perm(int ns, const int32_t *__restrict__ perm, int32_t *pos)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < ns) pos[perm[p]] = p;
}

cudaError_t build_near_lists(tdbem_ctx *c)
{
    const int ns = c->ns;
    if (c->tree.levels.empty()) return cudaErrorInvalidValue;
    const TreeLevel &T = c->tree.levels.back();
    cudaStream_t s = c->s;
    cudaError_t e;
    int32_t *e2c = nullptr;
    int64_t *cnt = nullptr;
    if ((e = cudaMalloc(&e2c, ns * sizeof(int32_t))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&cnt, ns * sizeof(int64_t))) != cudaSuccess) return e;
    k_elem_cell<<<(ns + 255) / 256, 256, 0, s>>>(ns, c->tree.perm, T.ecell, e2c);
    k_near_count<<<(ns + 127) / 128, 128, 0, s>>>(ns, e2c, T.nbr, T.ncount, T.cstart, cnt);
    std::vector<int64_t> hc(ns), prow(ns + 1), rowblk(ns + 1);
    if ((e = cudaMemcpyAsync(hc.data(), cnt, ns * sizeof(int64_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    prow[0] = rowblk[0] = 0;
    for (int i = 0; i < ns; ++i) {
        prow[i + 1] = prow[i] + hc[i];
        rowblk[i + 1] = rowblk[i] + (hc[i] + 31) / 32;
    }
    c->npairs = prow[ns];
    c->nbt = rowblk[ns];
    c->tree.e2c = e2c;
    cudaFree(cnt);
    void *p1, *p2, *p3;
    if ((e = cudaMalloc(&p1, (ns + 1) * sizeof(int64_t))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&p2, (ns + 1) * sizeof(int64_t))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&p3, std::max<int64_t>(c->npairs, 1) * sizeof(int32_t))) != cudaSuccess) return e;
    c->allocs.push_back(p1);
    c->allocs.push_back(p2);
    c->allocs.push_back(p3);
    c->d_prow = (int64_t *)p1;
    c->d_rowblk = (int64_t *)p2;
    c->d_col = (int32_t *)p3;
    if (c->split) {
        // the split form's float-pair histories are kept in the sorted order
        void *p4, *p5;
        if ((e = cudaMalloc(&p4, std::max<int64_t>(c->npairs, 1) * sizeof(int32_t))) != cudaSuccess) return e;
        if ((e = cudaMalloc(&p5, ns * sizeof(int32_t))) != cudaSuccess) return e;
        c->allocs.push_back(p4);
        c->allocs.push_back(p5);
        c->d_hcol = (int32_t *)p4;
        c->d_hpos = (int32_t *)p5;
        k_invert_perm<<<(ns + 255) / 256, 256, 0, s>>>(ns, c->tree.perm, c->d_hpos);
    }
    cudaMemcpyAsync(c->d_prow, prow.data(), (ns + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(c->d_rowblk, rowblk.data(), (ns + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    k_near_fill<<<(ns + 127) / 128, 128, 0, s>>>(ns, e2c, T.nbr, T.ncount, T.cstart, c->tree.perm, c->d_prow,
                                                c->d_col, c->d_hcol);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // per-cell near lists for the history sum
    {
        const int nc = T.nc;
        int64_t *ccnt = nullptr;
        if ((e = cudaMalloc(&ccnt, nc * sizeof(int64_t))) != cudaSuccess) return e;
        k_cell_near_count<<<(nc + 127) / 128, 128, 0, s>>>(nc, T.nbr, T.ncount, T.cstart, ccnt);
        std::vector<int64_t> hcc(nc), coff(nc + 1, 0);
        if ((e = cudaMemcpyAsync(hcc.data(), ccnt, nc * sizeof(int64_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return e;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
        cudaFree(ccnt);
        for (int k = 0; k < nc; ++k) coff[k + 1] = coff[k] + hcc[k];
        void *q1, *q2, *q3;
        if ((e = cudaMalloc(&q1, (nc + 1) * sizeof(int64_t))) != cudaSuccess) return e;
        if ((e = cudaMalloc(&q2, std::max<int64_t>(coff[nc], 1) * sizeof(int32_t))) != cudaSuccess) return e;
        if ((e = cudaMalloc(&q3, std::max<int64_t>(coff[nc], 1) * sizeof(int32_t))) != cudaSuccess) return e;
        c->allocs.push_back(q1);
        c->allocs.push_back(q2);
        c->allocs.push_back(q3);
        c->d_coff = (int64_t *)q1;
        c->d_ccol = (int32_t *)q2;
        c->d_chcol = (int32_t *)q3;
        if ((e = cudaMemcpyAsync(c->d_coff, coff.data(), (nc + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s)) !=
            cudaSuccess)
            return e;
        k_cell_near_fill<<<(nc + 127) / 128, 128, 0, s>>>(nc, T.nbr, T.ncount, T.cstart, c->tree.perm, c->d_coff,
                                                         c->d_ccol, c->d_chcol);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaStreamSynchronize(s);
}

void free_tree(tdbem_ctx *c)
{
    cudaFree(c->tree.box);
    cudaFree(c->tree.key);
    cudaFree(c->tree.perm);
    cudaFree(c->tree.e2c);
    for (auto &T : c->tree.levels) {
        cudaFree(T.ckey);
        cudaFree(T.cstart);
        cudaFree(T.ecell);
        cudaFree(T.nbr);
        cudaFree(T.ncount);
        cudaFree(T.il);
        cudaFree(T.ilcount);
    }
    c->tree = Tree{};
}

}  // namespace tdbem
