// Levels 1 and 0 of the V-cycle (Alg. 1 below the second-coarsest grid) in ONE thread block.
//
// With the paper's coarsest grid (8 x 8) level 1 is 16 x 16: 768 unknowns.  Run as separate
// kernels, its smoothing sweeps, IB passes, residual, restriction, the dense coarsest solve and the
// prolongation are a chain of 11 (Vanka) to 45 (Schur complement) dependent launches, each costing
// a launch and a round trip to L2 for almost no work.  Here one block of 1024 threads keeps the
// whole level in shared memory -- iterates, right-hand side, IB force, the patch entries, the SC
// diagonals and the assembled IB windows -- and separates the same steps by __syncthreads().
// The set-up data is copied in before the wait on the preceding kernel; only the right-hand side
// is read after it, and only the level's solution is written back.
//
// Every step evaluates the same point-wise formulas as the per-level kernels (grid_cells.cuh),
// in the same order, on shared-memory copies of the same arrays.
#include <cooperative_groups.h>

#include "grid_cells.cuh"

namespace cg = cooperative_groups;

namespace sib {

namespace {

template <typename T>
struct SmallSmem {
    T *x, *xt, *b, *r, *fib, *pf, *dinv, *pd;
    T *y, *d, *gq, *ya, *gq2, *dA2, *dA, *sv, *dp, *dM;
    T *b0, *x0, *win;
    int* tiles;
    unsigned char* tile;
};

// shared-memory layout of block 0: T arrays (the Vanka patch corrections share their space with
// the SC temporaries), then the active-tile list, then the tile flags
template <typename T>
__host__ __device__ inline size_t small_layout(int n, int n0, int nTiles, int per, int ntiles, SmallSmem<T>* s,
                                               unsigned char* base) {
    size_t off = 0;
    SmallSmem<T> dummy;
    SmallSmem<T>* q = s ? s : &dummy;
    auto take = [&](T** p, size_t cnt) {
        *p = reinterpret_cast<T*>(base + off);
        off += sizeof(T) * cnt;
    };
    take(&q->x, 3 * n);
    take(&q->xt, 3 * n);
    take(&q->b, 3 * n);
    take(&q->r, 3 * n);
    take(&q->fib, 2 * n);
    take(&q->pf, 7 * n);
    take(&q->dinv, 3 * n);
    const size_t tmp = off;   // SC temporaries, or the Vanka corrections (5 n <= 17 n)
    take(&q->y, 2 * n);
    take(&q->d, 2 * n);
    take(&q->gq, 2 * n);
    take(&q->ya, 2 * n);
    take(&q->gq2, 2 * n);
    take(&q->dA2, 2 * n);
    take(&q->dA, 2 * n);
    take(&q->sv, n);
    take(&q->dp, n);
    take(&q->dM, n);
    q->pd = reinterpret_cast<T*>(base + tmp);
    take(&q->b0, n0);
    take(&q->x0, n0);
    take(&q->win, (size_t)nTiles * 2 * WIN_SIZE * per);
    off = (off + 15) & ~(size_t)15;
    q->tiles = reinterpret_cast<int*>(base + off);
    off += sizeof(int) * (size_t)(nTiles > 0 ? nTiles : 1);
    q->tile = base + off;
    off += (size_t)ntiles;
    return (off + 15) & ~(size_t)15;
}

constexpr int NT = 1024;

__device__ __forceinline__ int ilog2(int v) { return 31 - __clz(v); }
constexpr int SMALL_CLUSTER = 8;

// Block-wide copy of `bytes` (a multiple of 16; both addresses 16-byte aligned) in 16-byte words,
// eight loads in flight per thread before their stores.
__device__ __forceinline__ void block_copy16(void* dst, const void* src, size_t bytes) {
    constexpr int U = 8;
    const int4* __restrict__ s = static_cast<const int4*>(src);
    int4* __restrict__ d = static_cast<int4*>(dst);
    const size_t n = bytes / 16;
    for (size_t q0 = 0; q0 < n; q0 += (size_t)NT * U) {
        int4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const size_t q = q0 + threadIdx.x + (size_t)u * NT;
            if (q < n) v[u] = s[q];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const size_t q = q0 + threadIdx.x + (size_t)u * NT;
            if (q < n) d[q] = v[u];
        }
    }
}


// f = [S K J] u on the active tiles: one thread per (slot, component, face), window rows summed in
// the per-level kernel's order.  Tile sizes, tile counts and N are powers of two: index arithmetic
// by shifts.  (The pass is bound by shared-memory bandwidth: 81 coefficients and 81 values a face.)
template <typename T>
__device__ void sm_ib(const GridK<T>& g, const SmallSmem<T>& s, int nTiles, const T* u, T* f) {
    const int N = g.N, lgN = ilog2(N), mk = N - 1, lgtx = g.lgtx, lgty = g.lgty;
    const int lgper = lgtx + lgty, per = 1 << lgper, lgntx = lgN - lgtx;
    const int items = nTiles * 2 * per;
    for (int item = threadIdx.x; item < items; item += NT) {
        const int q = item & (per - 1), rest = item >> lgper;
        const int c = rest & 1, slot = rest >> 1;
        const int t = s.tiles[slot];
        const int i = ((t & ((1 << lgntx) - 1)) << lgtx) + (q & ((1 << lgtx) - 1));
        const int j = ((t >> lgntx) << lgty) + (q >> lgtx);
        const T* w = s.win + (((slot * 2 + c) * WIN_SIZE) << lgper) + q;
        const T* uc = u + (c << (2 * lgN));
        T sum = T(0);
#pragma unroll
        for (int r = 0; r < WD; ++r) {
            const T* row = uc + (((j + r - WR) & mk) << lgN);
            T acc = T(0);
#pragma unroll
            for (int ox = -WR; ox <= WR; ++ox) acc += w[(r * WD + ox + WR) << lgper] * row[(i + ox) & mk];
            sum += acc;
        }
        f[(c << (2 * lgN)) + (j << lgN) + i] = sum;
    }
}

// one additive Vanka sweep xo = x + omega sum_c W_c R_c^T L_c^{-1} R_c (b - L x) (x == nullptr:
// zero start); g.fib holds [SKJ] x
template <typename T>
__device__ void sm_vanka(const GridK<T>& g, const SmallSmem<T>& s, const T* x, const T* b, T* xo) {
    const int N = g.N, n = N * N, m = N - 1;
    for (int c = threadIdx.x; c < n; c += NT) {
        const int i = c & m, j = c >> ilog2(N);
        if (x) {
            s.r[c] = res_u(g, x, b, i, j);
            s.r[n + c] = res_v(g, x, b, i, j);
            s.r[2 * n + c] = res_p(g, x, b, i, j);
        } else {
            s.r[c] = b[c];
            s.r[n + c] = b[n + c];
            s.r[2 * n + c] = b[2 * n + c];
        }
    }
    __syncthreads();
    const T ih = g.inv_h;
    for (int c = threadIdx.x; c < n; c += NT) {
        const int i = c & m, j = c >> ilog2(N);
        const int ce = j * N + ((i + 1) & m), cn = ((j + 1) & m) * N + i;
        const T r0 = s.r[c], r1 = s.r[ce], r2 = s.r[n + c], r3 = s.r[n + cn], r4 = s.r[2 * n + c];
        T f[7];
#pragma unroll
        for (int k = 0; k < 7; ++k) f[k] = g.pf[k * n + c];   // the cell's set-up patch factors
        T d0, d1, d2, d3, dp;
        patch_solve(f, ih, r0, r1, r2, r3, r4, d0, d1, d2, d3, dp);
        s.pd[c] = d0;
        s.pd[n + c] = d1;
        s.pd[2 * n + c] = d2;
        s.pd[3 * n + c] = d3;
        s.pd[4 * n + c] = dp;
    }
    __syncthreads();
    const T hw = T(0.5) * g.omega;
    for (int c = threadIdx.x; c < n; c += NT) {
        const int i = c & m, j = c >> ilog2(N);
        const int cw = j * N + ((i - 1) & m), cs = ((j - 1) & m) * N + i;
        const T du = hw * (s.pd[c] + s.pd[n + cw]);
        const T dv = hw * (s.pd[2 * n + c] + s.pd[3 * n + cs]);
        const T dq = g.omega * s.pd[4 * n + c];
        xo[c] = x ? x[c] + du : du;
        xo[n + c] = x ? x[n + c] + dv : dv;
        xo[2 * n + c] = x ? x[2 * n + c] + dq : dq;
    }
    __syncthreads();
}

// one Schur-complement sweep with two Chebyshev iterations per inner solve (x == nullptr: zero start)
template <typename T>
__device__ void sm_sc(const GridK<T>& g, const SmallArgs<T>& a, const SmallSmem<T>& s, const T* x, const T* b,
                      T* xo) {
    const int N = g.N, n = N * N, m = N - 1;
    const bool ib = a.nTiles > 0 && g.tile != nullptr;
    T* fib = const_cast<T*>(g.fib);
    if (x && ib) {
        sm_ib(g, s, a.nTiles, x, fib);
        __syncthreads();
    }
    for (int c = threadIdx.x; c < n; c += NT) sc_start_cell(g, a.ka, x, b, s.r, s.d, c & m, c >> ilog2(N), sc_pre<T, false>(g, c & m, c >> ilog2(N)));
    __syncthreads();
    if (ib) {
        sm_ib(g, s, a.nTiles, s.d, fib);
        __syncthreads();
    }
    for (int c = threadIdx.x; c < n; c += NT) sc_chebA_cell(g, a.ka, s.r, s.d, s.y, c & m, c >> ilog2(N), sc_pre<T, false>(g, c & m, c >> ilog2(N)));
    __syncthreads();
    for (int c = threadIdx.x; c < n; c += NT)
        sc_mstart_cell(g, a.ka, a.km, s.r + 2 * n, s.y, s.sv, s.dM, s.gq, s.dA, c & m, c >> ilog2(N),
                       sc_pre<T, true>(g, c & m, c >> ilog2(N)));
    __syncthreads();
    if (ib) {
        sm_ib(g, s, a.nTiles, s.dA, fib);
        __syncthreads();
    }
    for (int c = threadIdx.x; c < n; c += NT) sc_chebA_cell(g, a.ka, s.gq, s.dA, s.ya, c & m, c >> ilog2(N), sc_pre<T, false>(g, c & m, c >> ilog2(N)));
    __syncthreads();
    for (int c = threadIdx.x; c < n; c += NT)
        sc_mfinish_cell(g, a.ka, a.km, s.sv, s.dM, s.ya, s.dp, s.gq2, s.dA2, c & m, c >> ilog2(N),
                        sc_pre<T, true>(g, c & m, c >> ilog2(N)));
    __syncthreads();
    if (ib) {
        sm_ib(g, s, a.nTiles, s.dA2, fib);
        __syncthreads();
    }
    for (int c = threadIdx.x; c < n; c += NT) sc_finish_cell(g, a.ka, x, s.y, s.gq2, s.dA2, s.dp, xo, c & m, c >> ilog2(N),
                       sc_pre<T, false>(g, c & m, c >> ilog2(N)));
    __syncthreads();
}

template <typename T>
__device__ void sm_sweep(const GridK<T>& g, const SmallArgs<T>& a, const SmallSmem<T>& s, const T* x, const T* b,
                         T* xo) {
    if (a.smoother == SIB_SMOOTHER_SC) {
        sm_sc(g, a, s, x, b, xo);
        return;
    }
    if (x && a.nTiles > 0 && g.tile != nullptr) {
        sm_ib(g, s, a.nTiles, x, const_cast<T*>(g.fib));
        __syncthreads();
    }
    sm_vanka(g, s, x, b, xo);
}

// Block 0 runs level 1; blocks 1 .. csize-1 hold slices of the coarsest pseudo-inverse in shared
// memory (loaded before the wait) and apply it when block 0 has formed b0: each reads b0 from
// block 0's shared memory and writes its rows of x0 there, between two cluster barriers.
template <typename T>
__device__ void coarse_helper(const SmallArgs<T>& a, unsigned char* smraw, cg::cluster_group& cl) {
    const int rank = (int)cl.block_rank(), nh = (int)cl.num_blocks() - 1;
    const int rows = (a.n0 + nh - 1) / nh;
    const int r0 = (rank - 1) * rows, r1 = r0 + rows < a.n0 ? r0 + rows : a.n0;
    double* P = reinterpret_cast<double*>(smraw);                 // rows r0 .. r1-1
    double* bl = P + (size_t)rows * a.n0;                         // local copy of b0
    if (r1 > r0) block_copy16(P, a.Pinv + (size_t)r0 * a.n0, sizeof(double) * (size_t)(r1 - r0) * a.n0);
    pdl_entry();
    __syncthreads();
    SmallSmem<T> lay;
    const int N = a.g.N;
    small_layout<T>(N * N, a.n0, a.nTiles, a.g.tx * a.g.ty, a.ntiles, &lay, smraw);
    cl.sync();   // b0 formed by block 0
    const T* b0 = cl.map_shared_rank(lay.b0, 0);
    T* x0 = cl.map_shared_rank(lay.x0, 0);
    for (int c = threadIdx.x; c < a.n0; c += NT) bl[c] = (double)b0[c];
    __syncthreads();
    // four lanes a row: strided partial sums, then two butterfly steps.  The loop runs over
    // groups of eight rows, one group per warp, so every lane of a warp takes the same trip count
    // and reaches the shuffles; lanes of rows past r1 contribute nothing and store nothing.
    const int sub = threadIdx.x & 3;
    for (int rb = r0 + (int)(threadIdx.x >> 5) * 8; rb < r1; rb += (NT / 32) * 8) {
        const int r = rb + (int)((threadIdx.x & 31) >> 2);
        double acc = 0.0;
        if (r < r1) {
            const double* row = P + (size_t)(r - r0) * a.n0;
            for (int c = sub; c < a.n0; c += 4) acc += row[c] * bl[c];
        }
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        if (sub == 0 && r < r1) x0[r] = (T)acc;
    }
    cl.sync();   // x0 complete in block 0
}

template <typename T>
__global__ void __launch_bounds__(NT, 1) k_vcycle_small(const __grid_constant__ SmallArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    cg::cluster_group cl = cg::this_cluster();
    if (cl.block_rank() != 0) {
        coarse_helper(a, smraw, cl);
        return;
    }
    const GridK<T>& G = a.g;
    const int N = G.N, n = N * N, per = G.tx * G.ty;
    SmallSmem<T> s;
    small_layout<T>(n, a.n0, a.nTiles, per, a.ntiles, &s, smraw);
    // set-up data: not written by the kernels this one waits for (every array is a multiple of
    // 16 bytes: n is a multiple of 16)
    if (a.smoother == SIB_SMOOTHER_VANKA) block_copy16(s.pf, G.pf, sizeof(T) * 7 * n);
    if (a.smoother == SIB_SMOOTHER_SC) block_copy16(s.dinv, G.dinv, sizeof(T) * 3 * n);
    if (a.nTiles > 0) block_copy16(s.win, a.win, sizeof(T) * (size_t)a.nTiles * 2 * WIN_SIZE * per);
    for (int q = threadIdx.x; q < a.nTiles; q += NT) s.tiles[q] = a.tiles[q];
    if (G.tile)
        for (int q = threadIdx.x; q < a.ntiles; q += NT) s.tile[q] = G.tile[q];
    pdl_entry();
    block_copy16(s.b, a.b, sizeof(T) * 3 * n);
    __syncthreads();
    GridK<T> g = G;
    g.fib = s.fib;
    g.pf = s.pf;
    g.dinv = s.dinv;
    g.tile = G.tile ? s.tile : nullptr;
    const bool ib = a.nTiles > 0 && g.tile != nullptr;
    const int m = N - 1;

    T* x = s.x;
    T* xt = s.xt;
    int k0 = 0;
    if (a.nu1 > 0) {
        sm_sweep(g, a, s, (const T*)nullptr, s.b, xt);   // first sweep from w = 0
        T* t = x;
        x = xt;
        xt = t;
        k0 = 1;
    } else {
        for (int q = threadIdx.x; q < 3 * n; q += NT) x[q] = T(0);
        __syncthreads();
    }
    for (int k = k0; k < a.nu1; ++k) {
        sm_sweep(g, a, s, x, s.b, xt);
        T* t = x;
        x = xt;
        xt = t;
    }
    if (ib) {
        sm_ib(g, s, a.nTiles, x, s.fib);
        __syncthreads();
    }
    const int Nc = N / 2;
    for (int c = threadIdx.x; c < n; c += NT) {
        const int i = c & m, j = c >> ilog2(N);
        s.r[c] = res_u(g, x, s.b, i, j);
        s.r[n + c] = res_v(g, x, s.b, i, j);
        s.r[2 * n + c] = res_p(g, x, s.b, i, j);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < Nc * Nc; c += NT) restrict_cell(Nc, (const T*)s.r, s.b0, c & (Nc - 1), c >> ilog2(Nc));
    __syncthreads();
    cl.sync();   // b0 to the helpers
    cl.sync();   // x0 = Pinv b0 back from them
    for (int c = threadIdx.x; c < n; c += NT) prolong_add_cell(Nc, (const T*)s.x0, x, c & m, c >> ilog2(N));
    __syncthreads();
    for (int k = 0; k < a.nu2; ++k) {
        sm_sweep(g, a, s, x, s.b, xt);
        T* t = x;
        x = xt;
        xt = t;
    }
    block_copy16(a.out, x, sizeof(T) * 3 * n);
}

}  // namespace

template <typename T>
size_t vcycle_small_smem(int N1, int n0, int nTiles, int per, int ntiles) {
    return small_layout<T>(N1 * N1, n0, nTiles, per, ntiles, nullptr, nullptr);
}

// Cluster size of the launch: block 0 and the coarse-solve helpers (8, the portable maximum), 0
// if such a cluster cannot be resident with `smem` bytes per block.
template <typename T>
int vcycle_small_cluster(size_t smem) {
    if (cudaFuncSetAttribute(k_vcycle_small<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(SMALL_CLUSTER);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = SMALL_CLUSTER;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, k_vcycle_small<T>, &cfg) != cudaSuccess || clusters < 1) {
        cudaGetLastError();
        return 0;
    }
    return SMALL_CLUSTER;
}

template <typename T>
cudaError_t launch_vcycle_small(const SmallArgs<T>& a, size_t smem, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(k_vcycle_small<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(SMALL_CLUSTER);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = SMALL_CLUSTER;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, k_vcycle_small<T>, a);
}

template size_t vcycle_small_smem<float>(int, int, int, int, int);
template size_t vcycle_small_smem<double>(int, int, int, int, int);
template int vcycle_small_cluster<float>(size_t);
template int vcycle_small_cluster<double>(size_t);
template cudaError_t launch_vcycle_small<float>(const SmallArgs<float>&, size_t, cudaStream_t);
template cudaError_t launch_vcycle_small<double>(const SmallArgs<double>&, size_t, cudaStream_t);

}  // namespace sib
