// Lagrangian-Eulerian kernels: Peskin four-point stencils and their Galerkin coarsening, marker
// binning (Morton-ordered stable sort), interpolation J, spring forces K, spreading S as a
// cell-binned gather, and the set-up assembly of IB operator entries.
//
// Interpolation / spreading (Appendix, "Lagrangian-Eulerian interaction"):
//   U_l = sum_f u_f phi((x_f - X_l)/h) phi((y_f - Y_l)/h),   f_f = (1/h^2) sum_l F_l phi(.) phi(.)
// i.e. S = J^T / h^2 for a spring force F given in force units.  On coarse levels the composite
// stencil J_l = J P_u^(lmax<-l) is used, so that (1/h_l^2) J_l^T K J_l equals the Galerkin
// operator R_u [S K J]^(l+1) P_u of Sec. 3.1 (R_u = P_u^T / 4).
#include <cmath>

#include "sib_internal.h"

namespace sib {

// Peskin's four-point kernel phi(r) (Appendix): piecewise in |r| with square roots, support |r| < 2.
__device__ __forceinline__ double phi4(double r) {
    const double a = fabs(r);
    if (a < 1.0) return 0.125 * (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a));
    if (a < 2.0) return 0.125 * (5.0 - 2.0 * a - sqrt(-7.0 + 12.0 * a - 4.0 * a * a));
    return 0.0;
}
// d phi / d r
__device__ __forceinline__ double dphi4(double r) {
    const double a = fabs(r);
    const double sg = r < 0.0 ? -1.0 : 1.0;
    if (a < 1.0) return sg * 0.125 * (-2.0 + (2.0 - 4.0 * a) / sqrt(1.0 + 4.0 * a - 4.0 * a * a));
    if (a < 2.0) return sg * 0.125 * (-2.0 - (6.0 - 4.0 * a) / sqrt(-7.0 + 12.0 * a - 4.0 * a * a));
    return 0.0;
}

struct StencilOut {
    int* base[SIB_MAX_LEVELS][2];
    double* w64[SIB_MAX_LEVELS][2];
    float* w32[SIB_MAX_LEVELS][2];
};

// 1-D restriction of a row of interpolation weights by one level, w <- w P (P = RT0 prolongation):
// linear in the face-normal direction (fine face 2I -> I; 2I+1 -> I and I+1 with 1/2) ...
__device__ __forceinline__ void coarsen_linear(int& b0, double w[4]) {
    const int nb = b0 >> 1;   // floor(b0 / 2) for negative b0 as well
    double c[4] = {0.0, 0.0, 0.0, 0.0};
    for (int a = 0; a < 4; ++a) {
        const int idx = b0 + a;
        const int k = (idx >> 1) - nb;
        if ((idx & 1) == 0) {
            c[k] += w[a];
        } else {
            c[k] += 0.5 * w[a];
            c[k + 1] += 0.5 * w[a];
        }
    }
    b0 = nb;
    for (int a = 0; a < 4; ++a) w[a] = c[a];
}
// ... and constant in the tangential direction (fine index j -> floor(j/2)).
__device__ __forceinline__ void coarsen_const(int& b0, double w[4]) {
    const int nb = b0 >> 1;
    double c[4] = {0.0, 0.0, 0.0, 0.0};
    for (int a = 0; a < 4; ++a) c[((b0 + a) >> 1) - nb] += w[a];
    b0 = nb;
    for (int a = 0; a < 4; ++a) w[a] = c[a];
}

__global__ void k_stencils(const double* __restrict__ X, int M, int Nf, int lmax, StencilOut out) {
    pdl_entry();
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int comp = blockIdx.y;
    if (m >= M) return;
    const double ox = comp == 0 ? 0.0 : 0.5, oy = comp == 0 ? 0.5 : 0.0;
    const double sx = X[2 * m] * Nf - ox, sy = X[2 * m + 1] * Nf - oy;
    int bi = (int)floor(sx) - 1, bj = (int)floor(sy) - 1;
    double wx[4], wy[4];
    for (int a = 0; a < 4; ++a) {
        wx[a] = phi4((double)(bi + a) - sx);
        wy[a] = phi4((double)(bj + a) - sy);
    }
    int N = Nf;
    for (int l = lmax; l >= 0; --l) {
        if (l < lmax) {
            if (comp == 0) {
                coarsen_linear(bi, wx);
                coarsen_const(bj, wy);
            } else {
                coarsen_const(bi, wx);
                coarsen_linear(bj, wy);
            }
            N >>= 1;
        }
        out.base[l][comp][m] = ((bj & (N - 1)) << 16) | (bi & (N - 1));
        for (int a = 0; a < 4; ++a) {
            out.w64[l][comp][8 * m + a] = wx[a];
            out.w64[l][comp][8 * m + 4 + a] = wy[a];
            out.w32[l][comp][8 * m + a] = (float)wx[a];
            out.w32[l][comp][8 * m + 4 + a] = (float)wy[a];
        }
    }
}

void launch_stencils(const double* X, int M, int Nf, int lmax, int** base, double** w64, float** w32,
                     cudaStream_t s) {
    if (M == 0) return;
    StencilOut o;
    for (int l = 0; l <= lmax; ++l)
        for (int c = 0; c < 2; ++c) {
            o.base[l][c] = base[2 * l + c];
            o.w64[l][c] = w64[2 * l + c];
            o.w32[l][c] = w32[2 * l + c];
        }
    launch_pdl(k_stencils, dim3((M + 127) / 128, 2), 128, 0, s, X, M, Nf, lmax, o);
}

// ------------------------------------------------------------------------------------------
// Stable ordering of markers by the Morton code of their fine stencil origin: keys
// (morton << 32 | id) sorted by a bitonic network (ties cannot occur, ids are distinct).
__global__ void k_sort_keys(const int* __restrict__ base, int M, int Mpad, uint64_t* __restrict__ keys) {
    pdl_entry();
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= Mpad) return;
    if (m < M) {
        const int b = base[m];
        keys[m] = ((uint64_t)morton(b & 0xffff, (b >> 16) & 0xffff) << 32) | (uint32_t)m;
    } else {
        keys[m] = ~0ull;
    }
}
void launch_sort_keys(const int* baseFine, int M, int Mpad, uint64_t* keys, cudaStream_t s) {
    launch_pdl(k_sort_keys, (Mpad + 255) / 256, 256, 0, s, baseFine, M, Mpad, keys);
}

__global__ void k_bitonic_step(uint64_t* __restrict__ a, int Mpad, int j, int k) {
    pdl_entry();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Mpad) return;
    const int l = i ^ j;
    if (l > i) {
        const uint64_t x = a[i], y = a[l];
        const bool up = (i & k) == 0;
        if ((up && x > y) || (!up && x < y)) {
            a[i] = y;
            a[l] = x;
        }
    }
}
// all steps with j < 1024 of stage k run in shared memory
__global__ void k_bitonic_smem(uint64_t* __restrict__ a, int Mpad, int k, int jstart) {
    pdl_entry();
    __shared__ uint64_t sh[2048];
    const int base = blockIdx.x * 2048;
    for (int t = threadIdx.x; t < 2048; t += blockDim.x) sh[t] = a[base + t];
    __syncthreads();
    for (int j = jstart; j > 0; j >>= 1) {
        for (int t = threadIdx.x; t < 2048; t += blockDim.x) {
            const int i = base + t, l = i ^ j;
            if (l > i) {
                const uint64_t x = sh[t], y = sh[l - base];
                const bool up = (i & k) == 0;
                if ((up && x > y) || (!up && x < y)) {
                    sh[t] = y;
                    sh[l - base] = x;
                }
            }
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < 2048; t += blockDim.x) a[base + t] = sh[t];
}
void launch_bitonic(uint64_t* keys, int Mpad, cudaStream_t s) {
    for (int k = 2; k <= Mpad; k <<= 1) {
        int j = k >> 1;
        if (Mpad >= 2048) {
            for (; j >= 1024; j >>= 1) launch_pdl(k_bitonic_step, (Mpad + 255) / 256, 256, 0, s, keys, Mpad, j, k);
            launch_pdl(k_bitonic_smem, Mpad / 2048, 1024, 0, s, keys, Mpad, k, j);
        } else {
            for (; j >= 1; j >>= 1) launch_pdl(k_bitonic_step, (Mpad + 255) / 256, 256, 0, s, keys, Mpad, j, k);
        }
    }
}

__global__ void k_unpack_sorted(const uint64_t* __restrict__ keys, int M, int* __restrict__ sorted,
                                uint32_t* __restrict__ mkey) {
    pdl_entry();
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    sorted[m] = (int)(keys[m] & 0xffffffffu);
    mkey[m] = (uint32_t)(keys[m] >> 32);
}
void launch_unpack_sorted(const uint64_t* keys, int M, int* sorted, uint32_t* mkey, cudaStream_t s) {
    if (M == 0) return;
    launch_pdl(k_unpack_sorted, (M + 255) / 256, 256, 0, s, keys, M, sorted, mkey);
}

// binStart[b] = first position p with (mkey[p] >> shift) >= b, for b = 0..nbins
__global__ void k_bins(const uint32_t* __restrict__ mkey, int M, int nbins, int shift, int* __restrict__ binStart) {
    pdl_entry();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b > nbins) return;
    int lo = 0, hi = M;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((int)(mkey[mid] >> shift) < b)
            lo = mid + 1;
        else
            hi = mid;
    }
    binStart[b] = lo;
}
void launch_bins(const uint32_t* mkey, int M, int nbins, int shift, int* binStart, cudaStream_t s) {
    launch_pdl(k_bins, (nbins + 1 + 255) / 256, 256, 0, s, mkey, M, nbins, shift, binStart);
}

// ------------------------------------------------------------------------------------------
// IB-active tiles: every tile containing a face of some marker's stencil (either component),
// then dilated by one tile (so that a tile's one-cell halo is covered by its own flag) and
// compacted into an ordered list.
__global__ void k_tile_mark(const int* __restrict__ base, int M, int W, int N, int tx, int ty, int ntx,
                            unsigned char* __restrict__ flag) {
    pdl_entry();
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const int b = base[m], bi = b & 0xffff, bj = (b >> 16) & 0xffff, mk = N - 1;
    for (int q = 0; q < W; ++q)
        for (int p = 0; p < W; ++p) {
            const int i = (bi + p) & mk, j = (bj + q) & mk;
            flag[(j / ty) * ntx + i / tx] = 1;
        }
}
void launch_tile_flags(const int* base, int M, int W, int N, int tx, int ty, int ntx, unsigned char* flag,
                       cudaStream_t s) {
    if (M == 0) return;
    launch_pdl(k_tile_mark, (M + 127) / 128, 128, 0, s, base, M, W, N, tx, ty, ntx, flag);
}

// single block: raw flags in flag[0..nt), dilated flags written to flag[nt..2nt), list of
// active tiles (ascending) to tiles[], count to *nTiles
__global__ void k_tile_finish(unsigned char* __restrict__ flag, int ntx, int nty, int* __restrict__ tiles,
                              int* __restrict__ nTiles) {
    pdl_entry();
    __shared__ int warpSums[32];
    __shared__ int carry;
    const int nt = ntx * nty;
    unsigned char* dil = flag + nt;
    for (int t = threadIdx.x; t < nt; t += blockDim.x) {
        const int ti = t % ntx, tj = t / ntx;
        unsigned char f = 0;
        for (int dj = -1; dj <= 1; ++dj)
            for (int di = -1; di <= 1; ++di) {
                const int a = (ti + di + ntx) % ntx, bq = (tj + dj + nty) % nty;
                f |= flag[bq * ntx + a];
            }
        dil[t] = f;
    }
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int t0 = 0; t0 < nt; t0 += blockDim.x) {
        const int t = t0 + threadIdx.x;
        const int f = (t < nt && dil[t]) ? 1 : 0;
        // block-wide inclusive scan of f
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        int v = f;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (lane == 31) warpSums[wid] = v;
        __syncthreads();
        if (wid == 0) {
            int w = (lane < (int)(blockDim.x >> 5)) ? warpSums[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            warpSums[lane] = w;
        }
        __syncthreads();
        const int incl = v + (wid > 0 ? warpSums[wid - 1] : 0);
        if (f) tiles[carry + incl - 1] = t;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) *nTiles = carry;
}
void launch_tile_finish(unsigned char* flag, int ntx, int nty, int* tiles, int* nTiles, cudaStream_t s) {
    launch_pdl(k_tile_finish, 1, 1024, 0, s, flag, ntx, nty, tiles, nTiles);
}

// single block: the slots (indices into the active-tile list, ascending) of the active tiles whose
// raw flag is set, and their count
__global__ void k_row_slots(const unsigned char* __restrict__ flag, const int* __restrict__ tiles,
                            const int* __restrict__ nTiles, int* __restrict__ rowSlots, int* __restrict__ nRow) {
    pdl_entry();
    __shared__ int warpSums[32];
    __shared__ int carry;
    const int nt = *nTiles;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int s0 = 0; s0 < nt; s0 += blockDim.x) {
        const int sl = s0 + threadIdx.x;
        const int f = (sl < nt && flag[tiles[sl]]) ? 1 : 0;
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        int v = f;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (lane == 31) warpSums[wid] = v;
        __syncthreads();
        if (wid == 0) {
            int w = (lane < (int)(blockDim.x >> 5)) ? warpSums[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            warpSums[lane] = w;
        }
        __syncthreads();
        const int incl = v + (wid > 0 ? warpSums[wid - 1] : 0);
        if (f) rowSlots[carry + incl - 1] = sl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) *nRow = carry;
}
void launch_row_slots(const unsigned char* flag, const int* tiles, const int* nTiles, int* rowSlots, int* nRow,
                      cudaStream_t s) {
    launch_pdl(k_row_slots, 1, 1024, 0, s, flag, tiles, nTiles, rowSlots, nRow);
}

// ------------------------------------------------------------------------------------------
// Spring adjacency (CSR, deterministic): each marker's incident springs ordered by edge id.
__global__ void k_degree(const int* __restrict__ edges, int E, int* __restrict__ deg) {
    pdl_entry();
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    atomicAdd(&deg[edges[2 * e]], 1);
    atomicAdd(&deg[edges[2 * e + 1]], 1);
}
// single block exclusive scan of deg[0..M) into start[0..M]
__global__ void k_scan_single(const int* __restrict__ deg, int M, int* __restrict__ start) {
    pdl_entry();
    __shared__ int partial[1024];
    const int T = blockDim.x;
    const int chunk = (M + T - 1) / T;
    const int lo = threadIdx.x * chunk, hi = min(M, lo + chunk);
    int s = 0;
    for (int k = lo; k < hi; ++k) s += deg[k];
    partial[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int t = 0; t < T; ++t) {
            const int v = partial[t];
            partial[t] = acc;
            acc += v;
        }
        start[M] = acc;
    }
    __syncthreads();
    int acc = partial[threadIdx.x];
    for (int k = lo; k < hi; ++k) {
        start[k] = acc;
        acc += deg[k];
    }
}
__global__ void k_adj_fill(const int* __restrict__ edges, int E, const int* __restrict__ start, int* __restrict__ cursor,
                           int* __restrict__ nbr, int* __restrict__ eid) {
    pdl_entry();
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const int a = edges[2 * e], b = edges[2 * e + 1];
    int pa = start[a] + atomicAdd(&cursor[a], 1);
    nbr[pa] = b;
    eid[pa] = e;
    int pb = start[b] + atomicAdd(&cursor[b], 1);
    nbr[pb] = a;
    eid[pb] = e;
}
__global__ void k_adj_sort(int M, const int* __restrict__ start, int* __restrict__ nbr, int* __restrict__ eid) {
    pdl_entry();
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const int s = start[m], e = start[m + 1];
    for (int p = s + 1; p < e; ++p) {
        const int ke = eid[p], kn = nbr[p];
        int q = p - 1;
        while (q >= s && (eid[q] > ke || (eid[q] == ke && nbr[q] > kn))) {
            eid[q + 1] = eid[q];
            nbr[q + 1] = nbr[q];
            --q;
        }
        eid[q + 1] = ke;
        nbr[q + 1] = kn;
    }
}
void launch_adjacency(const int* edges, int E, int M, int* deg, int* start, int* nbr, int* eid, cudaStream_t s) {
    cudaMemsetAsync(deg, 0, sizeof(int) * (size_t)(M > 0 ? M : 1), s);
    if (E > 0) launch_pdl(k_degree, (E + 255) / 256, 256, 0, s, edges, E, deg);
    launch_pdl(k_scan_single, 1, 1024, 0, s, deg, M, start);
    cudaMemsetAsync(deg, 0, sizeof(int) * (size_t)(M > 0 ? M : 1), s);   // reused as cursor
    if (E > 0) launch_pdl(k_adj_fill, (E + 255) / 256, 256, 0, s, edges, E, start, deg, nbr, eid);
    if (M > 0) launch_pdl(k_adj_sort, (M + 255) / 256, 256, 0, s, M, start, nbr, eid);
}

template <typename T>
__global__ void k_adj_kappa(const int* __restrict__ eid, const double* __restrict__ kappa, int n2E, T* __restrict__ kap) {
    pdl_entry();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n2E) return;
    kap[p] = (T)kappa[eid[p]];
}
template <typename T>
void launch_adj_kappa(const int* eid, const double* kappa, int n2E, T* kap, cudaStream_t s) {
    if (n2E == 0) return;
    launch_pdl(k_adj_kappa<T>, (n2E + 255) / 256, 256, 0, s, eid, kappa, n2E, kap);
}

// ------------------------------------------------------------------------------------------
// Interpolation U^c_m = sum_{a,b < W} wx[a] wy[b] u^c[(bj+b) mod N][(bi+a) mod N]  (one thread per
// marker and component; U, F are stored component-major: U[c*M + m]).
template <typename T>
__global__ void k_interp(IBK<T> k, const T* __restrict__ u, T* __restrict__ U) {
    pdl_entry();
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (m >= k.M) return;
    const int N = k.N, mk = N - 1;
    // the component's arrays chosen by selects: indexing the parameter arrays by c would copy the
    // parameters to local memory
    const int b = (c ? k.base[1] : k.base[0])[m], bi = b & 0xffff, bj = (b >> 16) & 0xffff;
    const T* w = (c ? k.wgt[1] : k.wgt[0]) + 8 * m;
    const T* uc = u + (size_t)c * N * N;
    // W <= 4: the loops unrolled to four, so that every load of the stencil is in flight at once
    T acc = T(0);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (q >= k.W) break;
        const int row = ((bj + q) & mk) * N;
        T s = T(0);
#pragma unroll
        for (int p = 0; p < 4; ++p)
            if (p < k.W) s += w[p] * uc[row + ((bi + p) & mk)];
        acc += w[4 + q] * s;
    }
    U[c * k.M + m] = acc;
}
template <typename T>
void launch_interp(const IBK<T>& k, const T* u, T* U, cudaStream_t s) {
    if (k.M == 0) return;
    launch_pdl(k_interp<T>, dim3((k.M + 127) / 128, 2), 128, 0, s, k, u, U);
}

// Spring forces F_a = sum_{springs (a,b)} kappa_ab (U_b - U_a), per component (Appendix,
// "Lagrangian discretization", zero rest length).
template <typename T>
__global__ void k_spring(const int* __restrict__ start, const int* __restrict__ nbr, const T* __restrict__ kap, int M,
                         const T* __restrict__ U, T* __restrict__ F) {
    pdl_entry();
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (m >= M) return;
    const T* Uc = U + c * M;
    const T um = Uc[m];
    T acc = T(0);
    for (int p = start[m]; p < start[m + 1]; ++p) acc += kap[p] * (Uc[nbr[p]] - um);
    F[c * M + m] = acc;
}
template <typename T>
void launch_spring(const int* start, const int* nbr, const T* kap, int M, const T* U, T* F, cudaStream_t s) {
    if (M == 0) return;
    launch_pdl(k_spring<T>, dim3((M + 127) / 128, 2), 128, 0, s, start, nbr, kap, M, U, F);
}

// Spreading as a cell-binned gather: face (i, j) of component c collects every marker whose
// level-l stencil origin is (i - a, j - b), a, b < W, from the Morton-ordered bin of that origin:
//   f^c_ij = (1/h^2) sum_{a,b} sum_{m in bin(i-a, j-b)} wx_m[a] wy_m[b] F^c_m.
// No atomics; the summation order is fixed.  Only IB-active tiles are written.
template <typename T>
__device__ __forceinline__ T gather_face(const IBK<T>& k, const T* __restrict__ F, int c, int i, int j, int lane,
                                         int stride) {
    const int mk = k.N - 1;
    const int* bs = c ? k.binStart[1] : k.binStart[0];
    const int* srt = c ? k.sorted[1] : k.sorted[0];
    const T* wg = c ? k.wgt[1] : k.wgt[0];
    const T* Fc = F + c * k.M;
    // the W x W bin ranges first (independent loads, W <= 4), then the markers of each bin in the
    // same order (b, a, q) as a bin-by-bin walk
    int s[16], e[16];
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            s[4 * b + a] = 0;
            e[4 * b + a] = 0;
            if (a < k.W && b < k.W) {
                const uint32_t bin = morton((i - a) & mk, (j - b) & mk);
                s[4 * b + a] = bs[bin];
                e[4 * b + a] = bs[bin + 1];
            }
        }
    T acc = T(0);
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int a = 0; a < 4; ++a)
            for (int q = s[4 * b + a] + lane; q < e[4 * b + a]; q += stride) {
                const int m = srt[q];
                acc += wg[8 * m + a] * wg[8 * m + 4 + b] * Fc[m];
            }
    return acc;
}

// rowSlots != nullptr: block b takes the tile of slot rowSlots[b] (b < *nTiles, the count of that
// list), the tiles that a marker stencil touches; otherwise tile b of the active-tile list.  One thread
// per face of component blockIdx.y.
template <typename T>
__global__ void __launch_bounds__(256) k_spread_thread(IBK<T> k, const T* __restrict__ F, T* __restrict__ f,
                                                       const int* __restrict__ tiles, const int* __restrict__ nTiles,
                                                       const int* __restrict__ rowSlots, int tx, int ty, int ntx) {
    pdl_entry();
    if ((int)blockIdx.x >= *nTiles) return;
    const int t = tiles[rowSlots ? rowSlots[blockIdx.x] : blockIdx.x];
    const int i = (t % ntx) * tx + threadIdx.x, j = (t / ntx) * ty + threadIdx.y;
    const int n = k.N * k.N, c = blockIdx.y;
    f[c * n + j * k.N + i] = k.inv_h2 * gather_face(k, F, c, i, j, 0, 1);
}

template <typename T>
__global__ void __launch_bounds__(256) k_spread_warp(IBK<T> k, const T* __restrict__ F, T* __restrict__ f,
                                                     const int* __restrict__ tiles, const int* __restrict__ nTiles,
                                                     const int* __restrict__ rowSlots, int tx, int ty, int ntx) {
    pdl_entry();
    if ((int)blockIdx.x >= *nTiles) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int face = blockIdx.y * 8 + warp;
    const int per = tx * ty;
    if (face >= 2 * per) return;
    const int c = face / per, q = face % per;
    const int t = tiles[rowSlots ? rowSlots[blockIdx.x] : blockIdx.x];
    const int i = (t % ntx) * tx + q % tx, j = (t / ntx) * ty + q / tx;
    T acc = gather_face(k, F, c, i, j, lane, 32);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) f[c * k.N * k.N + j * k.N + i] = k.inv_h2 * acc;
}

// With rowSlots (nRow its count, maxTiles its host bound) only the tiles that a marker stencil touches
// are written; the caller keeps f at zero on the other active tiles.
template <typename T>
void launch_spread(const IBK<T>& k, const T* F, T* f, const int* tiles, const int* nTiles, int maxTiles, int tx,
                   int ty, int ntx, int warpPerFace, cudaStream_t s, const int* rowSlots, const int* nRow) {
    if (maxTiles == 0) return;
    const int* cnt = rowSlots ? nRow : nTiles;
    if (warpPerFace) {
        const int groups = (2 * tx * ty + 7) / 8;
        launch_pdl(k_spread_warp<T>, dim3(maxTiles, groups), 256, 0, s, k, F, f, tiles, cnt, rowSlots, tx, ty, ntx);
    } else {
        launch_pdl(k_spread_thread<T>, dim3(maxTiles, 2), dim3(tx, ty), 0, s, k, F, f, tiles, cnt, rowSlots, tx, ty,
                   ntx);
    }
}

// ------------------------------------------------------------------------------------------
// Spreading as a stored sparse product.  The gather's walk is done once per set-up: for every face of
// a stencil-touched tile and component, the markers it collects, in the gather's order (b, then a,
// then the bin's Morton order), with their weight products wx[a] wy[b] in FP64 and in FP32 (each
// formed as gather_face forms it).  Every (marker, a, b) pair lands on exactly one face, so a
// component holds M W^2 entries.  Row R = (c maxRow + r) tx ty + q: row tile r of the list, face q of
// the tile (row by row), component c.  Applying it, f = (1/h^2) S F is one ordered dot product per
// face, with the gather's rounding.
__device__ __forceinline__ void spread_face(int tile, int tx, int ty, int ntx, int q, int& i, int& j) {
    i = (tile % ntx) * tx + q % tx;
    j = (tile / ntx) * ty + q / tx;
}
// counts per face, their exclusive prefix within the tile (loc) and the tile's total (tileCnt)
__global__ void __launch_bounds__(256) k_spread_count(IBK<double> k, const int* __restrict__ tiles,
                                                      const int* __restrict__ rowSlots, const int* __restrict__ nRow,
                                                      int maxRow, int tx, int ty, int ntx, int* __restrict__ loc,
                                                      int* __restrict__ tileCnt) {
    pdl_entry();
    __shared__ int wsum[8];
    const int per = tx * ty, q = threadIdx.x, c = blockIdx.y, r = blockIdx.x;
    const int mk = k.N - 1;
    int cnt = 0;
    if (r < *nRow && q < per) {
        int i, j;
        spread_face(tiles[rowSlots[r]], tx, ty, ntx, q, i, j);
        const int* bs = c ? k.binStart[1] : k.binStart[0];
        for (int b = 0; b < k.W; ++b)
            for (int a = 0; a < k.W; ++a) {
                const uint32_t bin = morton((i - a) & mk, (j - b) & mk);
                cnt += bs[bin + 1] - bs[bin];
            }
    }
    // exclusive block scan of the 256 counts
    const int lane = q & 31, w = q >> 5;
    int x = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    int before = 0;
    for (int v = 0; v < w; ++v) before += wsum[v];
    if (q < per) loc[(size_t)(c * maxRow + r) * per + q] = before + x - cnt;
    if (q == 255) tileCnt[c * maxRow + r] = before + x;
}
template <typename T>
__device__ __forceinline__ T spread_product(const T* w, int m, int a, int b) {
    return w[8 * m + a] * w[8 * m + 4 + b];
}
// the rows' absolute offsets (off[R] = tileOff[tile] + loc[R], off[rows] = the total) and the entries
__global__ void __launch_bounds__(256) k_spread_fill(IBK<double> k, const float* __restrict__ w32u,
                                                     const float* __restrict__ w32v, const int* __restrict__ tiles,
                                                     const int* __restrict__ rowSlots, const int* __restrict__ nRow,
                                                     int maxRow, int tx, int ty, int ntx, const int* __restrict__ loc,
                                                     const int* __restrict__ tileOff, int64_t cap, int* __restrict__ off,
                                                     int* __restrict__ col, double* __restrict__ v64,
                                                     float* __restrict__ v32) {
    pdl_entry();
    const int per = tx * ty, q = threadIdx.x, c = blockIdx.y, r = blockIdx.x;
    if (q >= per) return;
    const size_t R = (size_t)(c * maxRow + r) * per + q;
    int p = tileOff[c * maxRow + r] + loc[R];
    off[R] = p;
    if (R + 1 == (size_t)2 * maxRow * per) off[R + 1] = tileOff[2 * maxRow];
    if (r >= *nRow) return;
    int i, j;
    spread_face(tiles[rowSlots[r]], tx, ty, ntx, q, i, j);
    const int mk = k.N - 1;
    const int* bs = c ? k.binStart[1] : k.binStart[0];
    const int* srt = c ? k.sorted[1] : k.sorted[0];
    const double* wg = c ? k.wgt[1] : k.wgt[0];
    const float* w32 = c ? w32v : w32u;
    for (int b = 0; b < k.W; ++b)
        for (int a = 0; a < k.W; ++a) {
            const uint32_t bin = morton((i - a) & mk, (j - b) & mk);
            for (int s = bs[bin]; s < bs[bin + 1]; ++s, ++p) {
                if (p >= cap) continue;   // cannot happen: a component holds exactly M W^2 entries
                const int m = srt[s];
                col[p] = m;
                v64[p] = spread_product(wg, m, a, b);
                v32[p] = spread_product(w32, m, a, b);
            }
        }
}
void launch_spread_store(const IBK<double>& k, const float* w32u, const float* w32v, const int* tiles,
                         const int* rowSlots, const int* nRow, int maxRow, int tx, int ty, int ntx, int* loc,
                         int* tileCnt, int* tileOff, int64_t cap, int* off, int* col, double* v64, float* v32,
                         cudaStream_t s) {
    if (maxRow == 0) return;
    const dim3 grd(maxRow, 2);
    launch_pdl(k_spread_count, grd, 256, 0, s, k, tiles, rowSlots, nRow, maxRow, tx, ty, ntx, loc, tileCnt);
    launch_pdl(k_scan_single, 1, 1024, 0, s, (const int*)tileCnt, 2 * maxRow, tileOff);
    launch_pdl(k_spread_fill, grd, 256, 0, s, k, w32u, w32v, tiles, rowSlots, nRow, maxRow, tx, ty, ntx,
               (const int*)loc, (const int*)tileOff, cap, off, col, v64, v32);
}
// f = (1/h^2) S F from the stored product: one thread per face of a stencil-touched tile and component
template <typename T>
__global__ void __launch_bounds__(256) k_spread_stored(const int* __restrict__ off, const int* __restrict__ col,
                                                       const T* __restrict__ val, const T* __restrict__ F, int M,
                                                       T inv_h2, const int* __restrict__ tiles,
                                                       const int* __restrict__ rowSlots, const int* __restrict__ nRow,
                                                       int maxRow, int N, int tx, int ty, int ntx, T* __restrict__ f) {
    pdl_entry();
    const int per = tx * ty, q = threadIdx.x, c = blockIdx.y, r = blockIdx.x;
    if (r >= *nRow || q >= per) return;
    const size_t R = (size_t)(c * maxRow + r) * per + q;
    const T* Fc = F + (size_t)c * M;
    T acc = T(0);
    const int e1 = off[R + 1];
    for (int e = off[R]; e < e1; ++e) acc += val[e] * Fc[col[e]];
    int i, j;
    spread_face(tiles[rowSlots[r]], tx, ty, ntx, q, i, j);
    f[(size_t)c * N * N + (size_t)j * N + i] = inv_h2 * acc;
}
template <typename T>
void launch_spread_stored(const int* off, const int* col, const T* val, const T* F, int M, T inv_h2, const int* tiles,
                          const int* rowSlots, const int* nRow, int maxRow, int N, int tx, int ty, int ntx, T* f,
                          cudaStream_t s) {
    if (maxRow == 0) return;
    launch_pdl(k_spread_stored<T>, dim3(maxRow, 2), 256, 0, s, off, col, val, F, M, inv_h2, tiles, rowSlots, nRow,
               maxRow, N, tx, ty, ntx, f);
}
template void launch_spread_stored<float>(const int*, const int*, const float*, const float*, int, float, const int*,
                                          const int*, const int*, int, int, int, int, int, float*, cudaStream_t);
template void launch_spread_stored<double>(const int*, const int*, const double*, const double*, int, double,
                                           const int*, const int*, const int*, int, int, int, int, int, double*,
                                           cudaStream_t);

// ------------------------------------------------------------------------------------------
// Set-up assembly of IB operator entries from the markers, B = [S K J]^l =
// -(1/h^2) sum_e kappa_e d_e d_e^T with d_e = J_l[a] - J_l[b] (the level-l stencil rows of the
// spring's two markers), used where the assembled windows overflow.
// Weight J_mf of marker m's level stencil at face (fi, fj), or 0 outside the stencil (covered = false).
__device__ __forceinline__ double stencil_weight(const IBK<double>& k, int c, int m, int fi, int fj, bool& covered) {
    const int mk = k.N - 1, bb = k.base[c][m];
    const int a = (fi - (bb & 0xffff)) & mk, b = (fj - ((bb >> 16) & 0xffff)) & mk;
    covered = a < k.W && b < k.W;
    return covered ? k.wgt[c][8 * m + a] * k.wgt[c][8 * m + 4 + b] : 0.0;
}

// Diagonal B(f, f) and the patch off-diagonal B(f, f + e) (e = +x for u faces, +y for v faces) of
// [S K J] on one level, where the assembled windows are not available:
//   B(f, g) = -(1/h^2) sum_e kappa_e d_e(f) d_e(g),   d_e(f) = J_af - J_bf  (spring e = (a, b), a != b).
// One thread per face of the tiles a marker stencil touches, per component.  The face gathers the
// markers whose stencil covers it from the level's cell bins (bin offsets in a fixed order, markers of a
// bin in Morton order) and each marker's springs from its adjacency list (ordered by spring id); a
// spring whose two markers both cover f is taken once, from the marker with the smaller index.  The
// summation order is fixed: repeated set-ups give the same bits.
__global__ void k_patch_entries(IBK<double> k, const int* __restrict__ adjStart, const int* __restrict__ adjNbr,
                                const double* __restrict__ adjKap, const int* __restrict__ tiles,
                                const int* __restrict__ rowSlots, const int* __restrict__ nRow, int tx, int ty,
                                int ntx, double* __restrict__ ibd) {
    pdl_entry();
    if ((int)blockIdx.x >= *nRow) return;
    const int c = blockIdx.y;
    const int t = tiles[rowSlots[blockIdx.x]];
    const int N = k.N, n = N * N, mk = N - 1;
    const int fi = (t % ntx) * tx + threadIdx.x, fj = (t / ntx) * ty + threadIdx.y;
    const int ni = c == 0 ? ((fi + 1) & mk) : fi, nj = c == 0 ? fj : ((fj + 1) & mk);   // f + e
    const int* bs = k.binStart[c];
    const int* srt = k.sorted[c];
    double dsum = 0.0, osum = 0.0;
    for (int b = 0; b < k.W; ++b)
        for (int a = 0; a < k.W; ++a) {
            const uint32_t bin = morton((fi - a) & mk, (fj - b) & mk);
            for (int q = bs[bin]; q < bs[bin + 1]; ++q) {
                const int m = srt[q];
                bool cm, cmn;
                const double jm = stencil_weight(k, c, m, fi, fj, cm);
                const double jmn = stencil_weight(k, c, m, ni, nj, cmn);
                if (!cm) continue;   // another level's origin bin (cannot happen on a consistent set-up)
                for (int p = adjStart[m]; p < adjStart[m + 1]; ++p) {
                    const int o = adjNbr[p];
                    if (o == m) continue;
                    bool co, con;
                    const double jo = stencil_weight(k, c, o, fi, fj, co);
                    if (co && o < m) continue;   // taken from o
                    const double jon = stencil_weight(k, c, o, ni, nj, con);
                    const double d = jm - jo, dn = jmn - jon;
                    dsum += adjKap[p] * d * d;
                    osum += adjKap[p] * d * dn;
                }
            }
        }
    const int f = fj * N + fi;
    ibd[(size_t)2 * c * n + f] = -dsum * k.inv_h2;
    ibd[(size_t)(2 * c + 1) * n + f] = -osum * k.inv_h2;
}
void launch_patch_entries(const IBK<double>& k, const int* adjStart, const int* adjNbr, const double* adjKap,
                          const int* tiles, const int* rowSlots, const int* nRow, int maxRow, int tx, int ty, int ntx,
                          double* ibd, cudaStream_t s) {
    if (maxRow == 0) return;
    launch_pdl(k_patch_entries, dim3(maxRow, 2), dim3(tx, ty), 0, s, k, adjStart, adjNbr, adjKap, tiles, rowSlots,
               nRow, tx, ty, ntx, ibd);
}

// Dense coarsest-level IB block B (2 x n0 x n0, per component), where the assembled windows are not
// available.  One block per row face p and component: its threads take the markers covering p (the
// markers of each bin in a fixed strided assignment) and their springs, as k_patch_entries does, and
// add kappa_e d_e(p) d_e(q) for the faces q of both markers' stencils into a row of their own in
// shared memory; the rows are then summed over the threads in thread order.  No atomics.
__global__ void k_dense_ib(IBK<double> k, const int* __restrict__ adjStart, const int* __restrict__ adjNbr,
                           const double* __restrict__ adjKap, double* __restrict__ B) {
    pdl_entry();
    extern __shared__ double rowacc[];   // blockDim.x x n0
    const int N = k.N, n0 = N * N, mk = N - 1, T = blockDim.x, tid = threadIdx.x;
    const int p = blockIdx.x, c = blockIdx.y;
    const int pi = p % N, pj = p / N;
    double* acc = rowacc + (size_t)tid * n0;
    for (int q = 0; q < n0; ++q) acc[q] = 0.0;
    const int* bs = k.binStart[c];
    const int* srt = k.sorted[c];
    for (int b = 0; b < k.W; ++b)
        for (int a = 0; a < k.W; ++a) {
            const uint32_t bin = morton((pi - a) & mk, (pj - b) & mk);
            for (int q = bs[bin] + tid; q < bs[bin + 1]; q += T) {
                const int m = srt[q];
                bool cm;
                const double jm = stencil_weight(k, c, m, pi, pj, cm);
                if (!cm) continue;
                const int bm = k.base[c][m];
                for (int e = adjStart[m]; e < adjStart[m + 1]; ++e) {
                    const int o = adjNbr[e];
                    if (o == m) continue;
                    bool co;
                    const double jo = stencil_weight(k, c, o, pi, pj, co);
                    if (co && o < m) continue;
                    const double kd = adjKap[e] * (jm - jo);
                    if (kd == 0.0) continue;
                    const int bo = k.base[c][o];
                    for (int y = 0; y < k.W; ++y)      // + kappa d_e(p) J_mq over m's stencil
                        for (int x = 0; x < k.W; ++x) {
                            const int qf = (((bm >> 16) + y) & mk) * N + (((bm & 0xffff) + x) & mk);
                            acc[qf] += kd * k.wgt[c][8 * m + x] * k.wgt[c][8 * m + 4 + y];
                        }
                    for (int y = 0; y < k.W; ++y)      // - kappa d_e(p) J_oq over o's stencil
                        for (int x = 0; x < k.W; ++x) {
                            const int qf = (((bo >> 16) + y) & mk) * N + (((bo & 0xffff) + x) & mk);
                            acc[qf] -= kd * k.wgt[c][8 * o + x] * k.wgt[c][8 * o + 4 + y];
                        }
                }
            }
        }
    __syncthreads();
    for (int q = tid; q < n0; q += T) {
        double sum = 0.0;
        for (int r = 0; r < T; ++r) sum += rowacc[(size_t)r * n0 + q];
        B[(size_t)c * n0 * n0 + (size_t)p * n0 + q] = -sum * k.inv_h2;
    }
}
void launch_dense_ib(const IBK<double>& k, const int* adjStart, const int* adjNbr, const double* adjKap, double* B,
                     cudaStream_t s) {
    if (k.M == 0) return;
    const int n0 = k.N * k.N;
    int threads = 256;
    while (threads > 32 && (size_t)threads * n0 * sizeof(double) > 128 * 1024) threads /= 2;
    const size_t smem = (size_t)threads * n0 * sizeof(double);
    cudaFuncSetAttribute(k_dense_ib, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    launch_pdl(k_dense_ib, dim3(n0, 2), dim3(threads), smem, s, k, adjStart, adjNbr, adjKap, B);
}

// ------------------------------------------------------------------------------------------
// Assembled Galerkin IB operator.  On a level where every spring joins markers whose stencil
// origins differ by at most WR - W + 1 cells, [S K J]^l couples a face only to faces within
// +-WR in each direction, so it is stored per face as a (2 WR + 1)^2 window of coefficients
//   B(f, f + o) = (1/h^2) sum_a J_l[a, f] sum_b K_ab J_l[b, f + o]
// (the same sum as the marker path, regrouped by face).  Windows exist for the faces of the
// IB-active tiles only, laid out [slot][comp][o][face in tile] (slot = index in the tile list).
__device__ __forceinline__ int wrapdiff(int d, int N) {
    d &= N - 1;
    return d >= N / 2 ? d - N : d;
}

// Faster set-up of the same windows.  Finest level: (1) per marker a the row (K J)_a =
// sum_b K_ab J[b, .] on a 6 x 6 patch anchored at a's stencil origin minus one (springs whose
// markers' origins differ by more than one cell set *overflow); (2) one thread per (face, window
// row oy) accumulates B(f, f+o) = (1/h^2) sum_{a: f in stencil(a)} J[a, f] (K J)_a(f + o) over
// the nine o of its row, in registers (the window index is static under full unrolling).
__global__ void k_kj_patch(IBK<double> k, const int* __restrict__ adjStart, const int* __restrict__ adjNbr,
                           const double* __restrict__ adjKap, double* __restrict__ KJ, int* __restrict__ overflow) {
    pdl_entry();
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (m >= k.M) return;
    const int N = k.N;
    const double* wg = k.wgt[c];
    const int* bse = k.base[c];
    double acc[36];
    for (int e = 0; e < 36; ++e) acc[e] = 0.0;
    const int om = bse[m], mi = om & 0xffff, mj = (om >> 16) & 0xffff;
    double ksum = 0.0;
    int ovf = 0;
    for (int p = adjStart[m]; p < adjStart[m + 1]; ++p) {
        const double kap = adjKap[p];
        ksum += kap;
        const int b = adjNbr[p];
        const int ob = bse[b];
        const int dx = wrapdiff((ob & 0xffff) - mi, N), dy = wrapdiff(((ob >> 16) & 0xffff) - mj, N);
        if (dx < -1 || dx > 1 || dy < -1 || dy > 1) {
            ovf = 1;
            continue;
        }
        for (int y = 0; y < 4; ++y)
            for (int x = 0; x < 4; ++x) acc[(dy + 1 + y) * 6 + dx + 1 + x] += kap * wg[8 * b + x] * wg[8 * b + 4 + y];
    }
    for (int y = 0; y < 4; ++y)
        for (int x = 0; x < 4; ++x) acc[(1 + y) * 6 + 1 + x] -= ksum * wg[8 * m + x] * wg[8 * m + 4 + y];
    double* out = KJ + ((size_t)c * k.M + m) * 36;
    for (int e = 0; e < 36; ++e) out[e] = acc[e];
    if (ovf) atomicOr(overflow, 1);
}
void launch_kj_patch(const IBK<double>& k, const int* adjStart, const int* adjNbr, const double* adjKap, double* KJ,
                     int* overflow, cudaStream_t s) {
    if (k.M == 0) return;
    launch_pdl(k_kj_patch, dim3((k.M + 127) / 128, 2), 128, 0, s, k, adjStart, adjNbr, adjKap, KJ, overflow);
}

__global__ void __launch_bounds__(256) k_window_fine(IBK<double> k, const double* __restrict__ KJ,
                                                     const int* __restrict__ tiles, int nTiles, int tx, int ty, int ntx,
                                                     double* __restrict__ win) {
    pdl_entry();
    const int slot = blockIdx.x;
    if (slot >= nTiles) return;
    const int c = blockIdx.y / WD, oy = (int)(blockIdx.y % WD) - WR;
    const int per = tx * ty, q = threadIdx.y * tx + threadIdx.x;
    const int t = tiles[slot];
    const int N = k.N, mk = N - 1;
    const int i = (t % ntx) * tx + threadIdx.x, j = (t / ntx) * ty + threadIdx.y;
    const int* bs = k.binStart[c];
    const int* srt = k.sorted[c];
    const double* wg = k.wgt[c];
    const double* kj = KJ + (size_t)c * k.M * 36;
    double acc[WD];
#pragma unroll
    for (int e = 0; e < WD; ++e) acc[e] = 0.0;
    for (int bo = 0; bo < 4; ++bo) {
        const int py = oy + 1 + bo;   // patch row holding f + o for markers with f in stencil row bo
        if (py < 0 || py > 5) continue;
#pragma unroll
        for (int ao = 0; ao < 4; ++ao) {
            const uint32_t bin = morton((i - ao) & mk, (j - bo) & mk);
            const int s0 = bs[bin], e0 = bs[bin + 1];
            for (int qq = s0; qq < e0; ++qq) {
                const int m = srt[qq];
                const double jf = wg[8 * m + ao] * wg[8 * m + 4 + bo] * k.inv_h2;
                const double* row = kj + (size_t)m * 36 + py * 6;
#pragma unroll
                for (int px = 0; px < 6; ++px) {
                    const int e = px - 1 - ao + WR;   // ox + WR, in [0, 8]
                    if (e >= 0 && e < WD) acc[e] += jf * row[px];
                }
            }
        }
    }
    double* wout = win + ((size_t)(slot * 2 + c) * WIN_SIZE + (size_t)(oy + WR) * WD) * per + q;
#pragma unroll
    for (int e = 0; e < WD; ++e) wout[(size_t)e * per] = acc[e];
}
void launch_window_fine(const IBK<double>& k, const double* KJ, const int* tiles, int nTiles, int tx, int ty, int ntx,
                        double* win, cudaStream_t s) {
    if (nTiles == 0 || k.M == 0) return;
    launch_pdl(k_window_fine, dim3(nTiles, 2 * WD), dim3(tx, ty), 0, s, k, KJ, tiles, nTiles, tx, ty, ntx, win);
}

// Coarse levels: the Galerkin product of Sec. 3.1 applied window to window,
//   B_c(F, G) = sum_f R_u(F, f) sum_g B_f(f, g) P_u(g, G),  R_u = P_u^T / 4,
// one thread per (coarse face, window row OY).  For x-faces R_u takes 1/4 of the two coincident
// fine faces and 1/8 of the four faces half a coarse cell away in x, and P_u is linear in x and
// constant in y; for y-faces the roles of x and y swap.
__global__ void __launch_bounds__(256) k_window_rap(const double* __restrict__ winF, const int* __restrict__ slotF,
                                                    int Nf, int txf, int tyf, int ntxf, const int* __restrict__ tilesC,
                                                    int nTilesC, int Nc, int txc, int tyc, int ntxc,
                                                    double* __restrict__ winC) {
    pdl_entry();
    const int slot = blockIdx.x;
    if (slot >= nTilesC) return;
    const int c = blockIdx.y / WD, OY = (int)(blockIdx.y % WD) - WR;
    const int perc = txc * tyc, perf = txf * tyf, q = threadIdx.y * txc + threadIdx.x;
    const int t = tilesC[slot];
    const int I = (t % ntxc) * txc + threadIdx.x, J = (t / ntxc) * tyc + threadIdx.y;
    const int mkf = Nf - 1;
    double acc[WD];
    for (int e = 0; e < WD; ++e) acc[e] = 0.0;
    for (int r = 0; r < 6; ++r) {
        int dx, dy;
        double wr;
        if (c == 0) {
            dx = r < 2 ? 0 : (r < 4 ? 1 : -1);
            dy = r & 1;
            wr = r < 2 ? 0.25 : 0.125;
        } else {
            dy = r < 2 ? 0 : (r < 4 ? 1 : -1);
            dx = r & 1;
            wr = r < 2 ? 0.25 : 0.125;
        }
        const int fx = 2 * I + dx, fy = 2 * J + dy;                 // unwrapped fine face
        const int wx = fx & mkf, wy = fy & mkf;
        const int sf = slotF[(wy / tyf) * ntxf + wx / txf];
        if (sf < 0) continue;
        const int qf = (wy % tyf) * txf + (wx % txf);
        const double* w = winF + ((size_t)(sf * 2 + c) * WIN_SIZE) * perf + qf;
        for (int oy = -WR; oy <= WR; ++oy) {
            const int gy = fy + oy;
            // targets of gy in y: constant (c == 0) or linear (c == 1)
            int Gy[2];
            double wyv[2];
            int ny;
            if (c == 0 || (gy & 1) == 0) {
                Gy[0] = gy >> 1;
                wyv[0] = 1.0;
                ny = 1;
            } else {
                Gy[0] = (gy - 1) >> 1;
                Gy[1] = (gy + 1) >> 1;
                wyv[0] = wyv[1] = 0.5;
                ny = 2;
            }
            double wsum = 0.0;
            for (int a = 0; a < ny; ++a)
                if (wrapdiff(Gy[a] - J, Nc) == OY) wsum += wyv[a];
            if (wsum == 0.0) continue;
            for (int ox = -WR; ox <= WR; ++ox) {
                const double b = w[(size_t)((oy + WR) * WD + ox + WR) * perf];
                if (b == 0.0) continue;
                const int gx = fx + ox;
                const double v = wr * wsum * b;
                if (c == 1 || (gx & 1) == 0) {
                    const int OX = wrapdiff((gx >> 1) - I, Nc);
                    acc[OX + WR] += v;
                } else {
                    acc[wrapdiff(((gx - 1) >> 1) - I, Nc) + WR] += 0.5 * v;
                    acc[wrapdiff(((gx + 1) >> 1) - I, Nc) + WR] += 0.5 * v;
                }
            }
        }
    }
    double* wout = winC + ((size_t)(slot * 2 + c) * WIN_SIZE + (size_t)(OY + WR) * WD) * perc + q;
    for (int e = 0; e < WD; ++e) wout[(size_t)e * perc] = acc[e];
}
void launch_window_rap(const double* winF, const int* slotF, int Nf, int txf, int tyf, int ntxf, const int* tilesC,
                       int nTilesC, int Nc, int txc, int tyc, int ntxc, double* winC, cudaStream_t s) {
    if (nTilesC == 0) return;
    launch_pdl(k_window_rap, dim3(nTilesC, 2 * WD), dim3(txc, tyc), 0, s, winF, slotF, Nf, txf, tyf, ntxf, tilesC, nTilesC, Nc,
                                                                 txc, tyc, ntxc, winC);
}

// slot of every tile of a level (-1 when the tile is not IB-active)
__global__ void k_slot_map(const int* __restrict__ tiles, const int* __restrict__ nTiles, int* __restrict__ slotOf) {
    pdl_entry();
    const int s2 = blockIdx.x * blockDim.x + threadIdx.x;
    if (s2 < *nTiles) slotOf[tiles[s2]] = s2;
}
void launch_slot_map(const int* tiles, const int* nTiles, int ntiles, int* slotOf, cudaStream_t s) {
    cudaMemsetAsync(slotOf, 0xff, sizeof(int) * (size_t)ntiles, s);
    launch_pdl(k_slot_map, (ntiles + 255) / 256, 256, 0, s, tiles, nTiles, slotOf);
}

// Patch entries of the Vanka/SC smoothers from the windows: B(f,f) and B(f, f+e), e = +x for u
// faces, +y for v faces; ibd is zero outside the active tiles.
__global__ void k_window_patch(const double* __restrict__ win, const int* __restrict__ tiles, int nTiles, int N,
                               int tx, int ty, int ntx, double* __restrict__ ibd) {
    pdl_entry();
    const int slot = blockIdx.x;
    if (slot >= nTiles) return;
    const int per = tx * ty;
    const int q = threadIdx.y * tx + threadIdx.x;
    const int t = tiles[slot];
    const int i = (t % ntx) * tx + threadIdx.x, j = (t / ntx) * ty + threadIdx.y;
    const int n = N * N, f = j * N + i;
    const double* wu = win + ((size_t)(slot * 2 + 0) * WIN_SIZE) * per;
    const double* wv = win + ((size_t)(slot * 2 + 1) * WIN_SIZE) * per;
    const int ctr = WR * WD + WR;
    ibd[f] = wu[(size_t)ctr * per + q];
    ibd[n + f] = wu[(size_t)(ctr + 1) * per + q];
    ibd[2 * n + f] = wv[(size_t)ctr * per + q];
    ibd[3 * n + f] = wv[(size_t)(ctr + WD) * per + q];
}
void launch_window_patch(const double* win, const int* tiles, int nTiles, int N, int tx, int ty, int ntx, double* ibd,
                         cudaStream_t s) {
    if (nTiles == 0) return;
    launch_pdl(k_window_patch, nTiles, dim3(tx, ty), 0, s, win, tiles, nTiles, N, tx, ty, ntx, ibd);
}

// Dense coarsest block B0 (per component, n0 x n0) from the level-0 windows (rows owned by one
// thread; window offsets that alias on the small grid add into the same entry).
__global__ void k_window_dense(const double* __restrict__ win, const int* __restrict__ tiles, int nTiles, int N,
                               int tx, int ty, int ntx, double* __restrict__ B) {
    pdl_entry();
    const int n0 = N * N;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= 2 * n0) return;
    const int c = r / n0, f = r % n0, i = f % N, j = f / N;
    const int t = (j / ty) * ntx + i / tx;
    int slot = -1;
    for (int s2 = 0; s2 < nTiles; ++s2)
        if (tiles[s2] == t) slot = s2;
    if (slot < 0) return;
    const int per = tx * ty, q = (j % ty) * tx + (i % tx), mk = N - 1;
    const double* w = win + ((size_t)(slot * 2 + c) * WIN_SIZE) * per;
    double* row = B + (size_t)c * n0 * n0 + (size_t)f * n0;
    for (int oy = -WR; oy <= WR; ++oy)
        for (int ox = -WR; ox <= WR; ++ox) {
            const double v = w[(size_t)((oy + WR) * WD + ox + WR) * per + q];
            if (v != 0.0) row[((j + oy) & mk) * N + ((i + ox) & mk)] += v;
        }
}
void launch_window_dense(const double* win, const int* tiles, int nTiles, int N, int tx, int ty, int ntx, double* B,
                         cudaStream_t s) {
    if (nTiles == 0) return;
    const int rows = 2 * N * N;
    launch_pdl(k_window_dense, (rows + 127) / 128, 128, 0, s, win, tiles, nTiles, N, tx, ty, ntx, B);
}

// Apply: f^c(face) = sum_o B(face, face + o) u^c(face + o) on the IB-active tiles.  A block
// takes 32 consecutive faces of one tile and component; thread (x, oy) sums window row oy of face
// x (nine terms), and the nine row sums are added in a fixed order.
// One block per (listed tile, group of 32 FV-face vectors, component): warp oy takes window row oy
// of every face of the group; each thread takes FV consecutive faces of one tile row (a 16-byte
// vector of coefficients per window entry), so a warp reads 512 contiguous bytes per entry.  The
// coefficients are set-up data, loaded before the dependency wait.
template <typename T>
struct WinVec;
template <>
struct WinVec<float> {
    using type = float4;
};
template <>
struct WinVec<double> {
    using type = double2;
};
template <typename T>
__global__ void __launch_bounds__(32 * WD) k_ib_window(const T* __restrict__ win, const int* __restrict__ tiles,
                                                       const int* __restrict__ rowSlots, const int* __restrict__ nRow,
                                                       int N, int tx, int ty, int ntx, const T* __restrict__ u,
                                                       T* __restrict__ f) {
    constexpr int FV = 16 / (int)sizeof(T);   // faces per thread
    static_assert(WR % FV == 0, "the u row's 16-byte loads start at i0 - WR");
    using VT = typename WinVec<T>::type;
    __shared__ __align__(16) T part[WD][32 * FV];
    if ((int)blockIdx.x >= *nRow) return;
    const int slot = rowSlots[blockIdx.x];
    const int per = tx * ty;
    const int q0 = (blockIdx.y * 32 + threadIdx.x) * FV;   // first face of the thread (tx is a multiple of FV)
    const int c = blockIdx.z;
    const int oy = (int)threadIdx.y - WR;
    const bool live = q0 < per;
    const int t = tiles[slot];
    const int i0 = (t % ntx) * tx + (live ? q0 % tx : 0), j = (t / ntx) * ty + (live ? q0 / tx : 0);
    const int n = N * N, mk = N - 1;
    VT wv[WD];
    if (live) {
        const T* w = win + ((size_t)(slot * 2 + c) * WIN_SIZE + (size_t)threadIdx.y * WD) * per + q0;
#pragma unroll
        for (int ox = 0; ox < WD; ++ox) wv[ox] = *reinterpret_cast<const VT*>(w + (size_t)ox * per);
    }
    pdl_entry();
    T acc[FV];
#pragma unroll
    for (int k = 0; k < FV; ++k) acc[k] = T(0);
    if (live) {
        const T* row = u + (size_t)c * n + (size_t)((j + oy) & mk) * N;
        T ur[FV + 2 * WR];   // u at i0 - WR .. i0 + FV + WR - 1 of the row
        if (i0 >= WR && i0 + FV + WR <= N) {   // inside the row: 16-byte loads (i0 - WR is a multiple of FV)
            constexpr int NV = (FV + 2 * WR) / FV;
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const VT q = *reinterpret_cast<const VT*>(row + i0 - WR + v * FV);
                const T* qv = reinterpret_cast<const T*>(&q);
#pragma unroll
                for (int k = 0; k < FV; ++k) ur[v * FV + k] = qv[k];
            }
        } else {   // across the periodic seam
#pragma unroll
            for (int k = 0; k < FV + 2 * WR; ++k) ur[k] = row[(i0 - WR + k) & mk];
        }
#pragma unroll
        for (int ox = 0; ox < WD; ++ox) {
            const T* wk = reinterpret_cast<const T*>(&wv[ox]);
#pragma unroll
            for (int k = 0; k < FV; ++k) acc[k] += wk[k] * ur[k + ox];
        }
    }
#pragma unroll
    for (int k = 0; k < FV; ++k) part[threadIdx.y][threadIdx.x * FV + k] = acc[k];
    __syncthreads();
    if (threadIdx.y == 0 && live) {
        VT out;
        T* o = reinterpret_cast<T*>(&out);
#pragma unroll
        for (int k = 0; k < FV; ++k) {
            T sum = T(0);
#pragma unroll
            for (int r = 0; r < WD; ++r) sum += part[r][threadIdx.x * FV + k];
            o[k] = sum;
        }
        *reinterpret_cast<VT*>(f + (size_t)c * n + (size_t)j * N + i0) = out;
    }
}
// Only the tiles a marker stencil touches have nonzero rows; the other active tiles keep the zero
// IB force written at set-up.
template <typename T>
void launch_ib_window(const T* win, const int* tiles, const int* rowSlots, const int* nRow, int maxRow, int N, int tx,
                      int ty, int ntx, const T* u, T* f, cudaStream_t s) {
    if (maxRow == 0) return;
    constexpr int FV = 16 / (int)sizeof(T);
    const int groups = (tx * ty + 32 * FV - 1) / (32 * FV);
    launch_pdl(k_ib_window<T>, dim3(maxRow, groups, 2), dim3(32, WD), 0, s, win, tiles, rowSlots, nRow, N, tx, ty, ntx,
               u, f);
}
template void launch_ib_window<float>(const float*, const int*, const int*, const int*, int, int, int, int, int,
                                      const float*, float*, cudaStream_t);
template void launch_ib_window<double>(const double*, const int*, const int*, const int*, int, int, int, int, int,
                                       const double*, double*, cudaStream_t);

// ------------------------------------------------------------------------------------------
// (M x 2) interleaved <-> component-major [x (M) | y (M)]
__global__ void k_deinterleave(const double* __restrict__ in, int M, double* __restrict__ out) {
    pdl_entry();
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    out[m] = in[2 * m];
    out[M + m] = in[2 * m + 1];
}
__global__ void k_interleave(const double* __restrict__ in, int M, double* __restrict__ out) {
    pdl_entry();
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    out[2 * m] = in[m];
    out[2 * m + 1] = in[M + m];
}
void launch_deinterleave(const double* in, int M, double* out, cudaStream_t s) {
    if (M == 0) return;
    launch_pdl(k_deinterleave, (M + 255) / 256, 256, 0, s, in, M, out);
}
void launch_interleave(const double* in, int M, double* out, cudaStream_t s) {
    if (M == 0) return;
    launch_pdl(k_interleave, (M + 255) / 256, 256, 0, s, in, M, out);
}

// Structure update of the semi-implicit scheme (Eq. imp-X-new): X^{n+1} = X^n + dt J^n u^{n+1}, with
// U = J^n u^{n+1} component-major [x (M) | y (M)] and X, X^{n+1} interleaved (M x 2).
__global__ void k_advance_markers(const double* __restrict__ X, const double* __restrict__ U, int M, double dt,
                                  double* __restrict__ Xn) {
    pdl_entry();
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    Xn[2 * m] = X[2 * m] + dt * U[m];
    Xn[2 * m + 1] = X[2 * m + 1] + dt * U[M + m];
}
void launch_advance_markers(const double* X, const double* U, int M, double dt, double* Xn, cudaStream_t s) {
    if (M == 0) return;
    launch_pdl(k_advance_markers, (M + 255) / 256, 256, 0, s, X, U, M, dt, Xn);
}

// Deterministic start vector of the power iterations: Knuth's multiplicative hash of k+1,
// (k+1) * 2654435761 mod 2^32, mapped to [-1/2, 1/2).
__global__ void k_hash_vector(double* __restrict__ x, int64_t n) {
    pdl_entry();
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t v = (uint32_t)(k + 1) * 2654435761u;
        x[k] = (double)v / 4294967296.0 - 0.5;
    }
}
void launch_hash_vector(double* x, int64_t n, cudaStream_t s) {
    launch_pdl(k_hash_vector, num_blocks_for(n), 256, 0, s, x, n);
}

// ------------------------------------------------------------------------------------------
// Gradients of the discrete adjoint (see sib_grad): per spring
//   dkappa_e = -(Lam_a - Lam_b) . (Y_a - Y_b)
// and per marker, with the interpolation weights and their derivatives recomputed from X:
//   dX_l^d = sum_c (d_d Lam_l^c) (K Y)_l^c + a (K Lam)_l^d + dt sum_c (K Lam)_l^c d_d U_l^c,
//   d_d J^c_{l,f} = -(1/h) phi'(r_x) phi(r_y)  (d = x),  -(1/h) phi(r_x) phi'(r_y)  (d = y).
// Lam, Y, KY, KL are component-major (M | M).
__global__ void k_grad_kappa(const int* __restrict__ edges, int E, int M, const double* __restrict__ Lam,
                             const double* __restrict__ Y, double* __restrict__ dkappa) {
    pdl_entry();
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const int a = edges[2 * e], b = edges[2 * e + 1];
    double s = 0.0;
    for (int c = 0; c < 2; ++c) s += (Lam[c * M + a] - Lam[c * M + b]) * (Y[c * M + a] - Y[c * M + b]);
    dkappa[e] = -s;
}
__global__ void k_grad_X(const double* __restrict__ X, int M, int N, const double* __restrict__ w,
                         const double* __restrict__ lam, const double* __restrict__ KY, const double* __restrict__ KL,
                         double dt, double acoef, double* __restrict__ dX) {
    pdl_entry();
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const int n = N * N, mk = N - 1;
    const double h = 1.0 / N, ih = (double)N, ih2 = ih * ih;
    double gd[2] = {acoef * KL[m], acoef * KL[M + m]};
    for (int c = 0; c < 2; ++c) {
        const double ox = c == 0 ? 0.0 : 0.5, oy = c == 0 ? 0.5 : 0.0;
        const double sx = X[2 * m] * N - ox, sy = X[2 * m + 1] * N - oy;
        const int bi = (int)floor(sx) - 1, bj = (int)floor(sy) - 1;
        double wx[4], wy[4], dx[4], dy[4];
        for (int a = 0; a < 4; ++a) {
            wx[a] = phi4((double)(bi + a) - sx);
            wy[a] = phi4((double)(bj + a) - sy);
            dx[a] = dphi4((double)(bi + a) - sx);
            dy[a] = dphi4((double)(bj + a) - sy);
        }
        const double* uc = w + c * n;
        const double* lc = lam + c * n;
        double gU[2] = {0.0, 0.0}, gL[2] = {0.0, 0.0};
        for (int q = 0; q < 4; ++q) {
            const int row = ((bj + q) & mk) * N;
            for (int p = 0; p < 4; ++p) {
                const int f = row + ((bi + p) & mk);
                const double jx = -dx[p] * wy[q] * ih;   // d J / d X^x
                const double jy = -wx[p] * dy[q] * ih;   // d J / d X^y
                gU[0] += jx * uc[f];
                gU[1] += jy * uc[f];
                gL[0] += jx * lc[f];
                gL[1] += jy * lc[f];
            }
        }
        (void)h;
        for (int d = 0; d < 2; ++d) gd[d] += gL[d] * ih2 * KY[c * M + m] + dt * KL[c * M + m] * gU[d];
    }
    dX[2 * m] = gd[0];
    dX[2 * m + 1] = gd[1];
}
void launch_grad_kappa(const int* edges, int E, int M, const double* Lam, const double* Y, double* dkappa,
                       cudaStream_t s) {
    if (E == 0) return;
    launch_pdl(k_grad_kappa, (E + 255) / 256, 256, 0, s, edges, E, M, Lam, Y, dkappa);
}
void launch_grad_X(const double* X, int M, int N, const double* w, const double* lam, const double* KY,
                   const double* KL, double dt, double acoef, double* dX, cudaStream_t s) {
    if (M == 0) return;
    launch_pdl(k_grad_X, (M + 127) / 128, 128, 0, s, X, M, N, w, lam, KY, KL, dt, acoef, dX);
}

// ------------------------------------------------------------------------------------------
#define SIB_IB_INST(T)                                                                                           \
    template void launch_adj_kappa<T>(const int*, const double*, int, T*, cudaStream_t);                        \
    template void launch_interp<T>(const IBK<T>&, const T*, T*, cudaStream_t);                                  \
    template void launch_spring<T>(const int*, const int*, const T*, int, const T*, T*, cudaStream_t);           \
    template void launch_spread<T>(const IBK<T>&, const T*, T*, const int*, const int*, int, int, int, int, int, \
                                   cudaStream_t, const int*, const int*);
SIB_IB_INST(float)
SIB_IB_INST(double)

}  // namespace sib
