// FP64 kernels of the outer flexible GMRES (dot products, classical Gram-Schmidt, gauge
// projection) and of the coarsest-grid exact solve (dense operator, Gauss-Jordan inverse,
// pseudo-inverse apply).  All reductions use a fixed block count and a fixed reduction tree,
// so results are bitwise reproducible run to run.
#include <cooperative_groups.h>

#include <cmath>

#include "sib_internal.h"

namespace cg = cooperative_groups;

namespace sib {

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double ws[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) ws[wid] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? ws[threadIdx.x] : 0.0;
    if (wid == 0)
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;   // valid in thread 0
}

__global__ void k_dot_partials(const double* __restrict__ x, const double* __restrict__ y, int64_t n,
                               double* __restrict__ partials) {
    pdl_entry();
    double s = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        s += x[k] * y[k];
    s = block_sum(s);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}
void launch_dot_partials(const double* x, const double* y, int64_t n, double* partials, int nblk, cudaStream_t s) {
    launch_pdl(k_dot_partials, nblk, 256, 0, s, x, y, n, partials);
}

// partials[i * nblk + b] = sum over block b's slice of V_i . w, for i < k
__global__ void k_multidot(const double* __restrict__ V, int64_t ld, const double* __restrict__ w, int64_t n,
                           double* __restrict__ partials) {
    pdl_entry();
    const int i = blockIdx.y;
    const double* v = V + (int64_t)i * ld;
    double s = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        s += v[k] * w[k];
    s = block_sum(s);
    if (threadIdx.x == 0) partials[(int64_t)i * gridDim.x + blockIdx.x] = s;
}
void launch_multidot(const double* V, int64_t ld, int k, const double* w, int64_t n, double* partials, int nblk,
                     cudaStream_t s) {
    launch_pdl(k_multidot, dim3(nblk, k), 256, 0, s, V, ld, w, n, partials);
}

__global__ void k_reduce_partials(const double* __restrict__ partials, int nblk, double* __restrict__ out) {
    pdl_entry();
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += partials[(int64_t)blockIdx.x * nblk + b];
    s = block_sum(s);
    if (threadIdx.x == 0) out[blockIdx.x] = s;
}
void launch_reduce_partials(const double* partials, int k, int nblk, double* out, cudaStream_t s) {
    launch_pdl(k_reduce_partials, k, 256, 0, s, partials, nblk, out);
}

// y += sign * sum_{i<k} coef[i] V_i
__global__ void k_multi_axpy(const double* __restrict__ V, int64_t ld, int k, const double* __restrict__ coef,
                             double sign, double* __restrict__ y, int64_t n) {
    pdl_entry();
    __shared__ double c[128];
    for (int t = threadIdx.x; t < k; t += blockDim.x) c[t] = sign * coef[t];
    __syncthreads();
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        double acc = y[e];
        for (int i = 0; i < k; ++i) acc += c[i] * V[(int64_t)i * ld + e];
        y[e] = acc;
    }
}
void launch_multi_axpy(const double* V, int64_t ld, int k, const double* coef, double sign, double* y, int64_t n,
                       cudaStream_t s) {
    launch_pdl(k_multi_axpy, num_blocks_for(n), 256, 0, s, V, ld, k, coef, sign, y, n);
}

// x *= 1 / sqrt(vals[idx])   (normalisation of the next Arnoldi vector)
__global__ void k_scale_rsqrt(double* __restrict__ x, const double* __restrict__ vals, int idx, int64_t n) {
    pdl_entry();
    const double nrm = sqrt(vals[idx]);
    const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        x[k] *= inv;
}
void launch_scale(double* x, const double* vals, int idx, int64_t n, cudaStream_t s) {
    launch_pdl(k_scale_rsqrt, num_blocks_for(n), 256, 0, s, x, vals, idx, n);
}

// gauge projection: means of the u, v, p blocks and their removal (mask bit b = block b)
__global__ void k_block_means(const double* __restrict__ x, int64_t n, double* __restrict__ partials) {
    pdl_entry();
    const double* xb = x + blockIdx.y * n;
    double s = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        s += xb[k];
    s = block_sum(s);
    if (threadIdx.x == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = s;
}
void launch_block_means(const double* x, int N, int nblocks_vec, double* partials, int nblk, cudaStream_t s) {
    launch_pdl(k_block_means, dim3(nblk, nblocks_vec), 256, 0, s, x, (int64_t)N * N, partials);
}
__global__ void k_subtract_means(double* __restrict__ x, int64_t n, const double* __restrict__ partials, int nblk,
                                 int mask) {
    pdl_entry();
    __shared__ double mean[3];
    if (threadIdx.x < 32) {
        for (int b = 0; b < 3; ++b) {
            double s = 0.0;
            for (int q = threadIdx.x; q < nblk; q += 32) s += partials[b * nblk + q];
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (threadIdx.x == 0) mean[b] = ((mask >> b) & 1) ? s / (double)n : 0.0;
        }
    }
    __syncthreads();
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < 3 * n; k += (int64_t)gridDim.x * blockDim.x)
        x[k] -= mean[k / n];
}
void launch_subtract_means(double* x, int N, const double* partials, int nblk, int mask, cudaStream_t s) {
    const int64_t n = (int64_t)N * N;
    launch_pdl(k_subtract_means, num_blocks_for(3 * n), 256, 0, s, x, n, partials, nblk, mask);
}

// ------------------------------------------------------------------------------------------
// Coarsest level: dense L^0 + Z Z^T (Z = orthonormal kernel basis: the constant pressure, and
// the constant velocity components when rho = 0), augmented with the identity: Aug = [L0+ZZ^T | I].
// One thread per entry: momentum rows hold A = a0 I - mu Lap (5-point, periodic), + G and - dt [SKJ]^0;
// pressure rows hold - D.  Coincident periodic neighbours add up (counted per offset).
__global__ void k_assemble_L0(int N, double rho, double mu, double dt, const double* __restrict__ B,
                              double* __restrict__ Aug) {
    pdl_entry();
    const int n0 = N * N, n = 3 * n0, mk = N - 1;
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= (int64_t)n * 2 * n) return;
    const int r = (int)(q / (2 * n)), col = (int)(q % (2 * n));
    if (col >= n) {
        Aug[q] = (col - n == r) ? 1.0 : 0.0;
        return;
    }
    const double h = 1.0 / N, ih = (double)N;
    const double a0 = rho / dt + 4.0 * mu / (h * h), cc = mu / (h * h);
    const int br = r / n0, f = r % n0, i = f % N, j = f / N;
    const int bc = col / n0, gcell = col % n0;
    double v = 0.0;
    if (br < 2) {
        if (bc == br) {
            if (gcell == f) v += a0;
            if (gcell == j * N + ((i + 1) & mk)) v -= cc;
            if (gcell == j * N + ((i - 1) & mk)) v -= cc;
            if (gcell == ((j + 1) & mk) * N + i) v -= cc;
            if (gcell == ((j - 1) & mk) * N + i) v -= cc;
            v -= dt * B[(int64_t)br * n0 * n0 + (int64_t)f * n0 + gcell];
        } else if (bc == 2) {   // G p: (p_ij - p_{i-1,j})/h on u faces, (p_ij - p_{i,j-1})/h on v faces
            if (gcell == f) v += ih;
            if (gcell == (br == 0 ? j * N + ((i - 1) & mk) : ((j - 1) & mk) * N + i)) v -= ih;
        }
    } else if (bc < 2) {        // - D u
        if (bc == 0) {
            if (gcell == f) v += ih;
            if (gcell == j * N + ((i + 1) & mk)) v -= ih;
        } else {
            if (gcell == f) v += ih;
            if (gcell == ((j + 1) & mk) * N + i) v -= ih;
        }
    }
    if (bc == br && (rho == 0.0 || br == 2)) v += 1.0 / (double)n0;
    Aug[q] = v;
}
void launch_assemble_L0(int N0, double rho, double mu, double dt, const double* B, double* Aug, cudaStream_t s) {
    const int64_t tot = (int64_t)3 * N0 * N0 * 6 * N0 * N0;
    launch_pdl(k_assemble_L0, (int)((tot + 255) / 256), 256, 0, s, N0, rho, mu, dt, B, Aug);
}

// In-place Gauss-Jordan elimination with partial pivoting on Aug (n x 2n, row-major) by one
// block; on exit the right half holds the inverse.  info = 0, or k+1 if pivot k is zero.
// (Fallback for coarsest grids too large for the cluster version below.)
__global__ void __launch_bounds__(1024) k_gauss_jordan(double* __restrict__ A, int n, int* __restrict__ info,
                                                       int* __restrict__ piv) {
    pdl_entry();
    extern __shared__ double fac[];   // n factors
    __shared__ int pivs;
    __shared__ double wv[32];
    __shared__ int wi[32];
    const int ld = 2 * n;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) *info = 0;
    for (int k = 0; k < n; ++k) {
        // pivot search over rows k..n-1 of column k
        double best = -1.0;
        int bi = k;
        for (int r = k + threadIdx.x; r < n; r += blockDim.x) {
            const double a = fabs(A[(int64_t)r * ld + k]);
            if (a > best) {
                best = a;
                bi = r;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) {
                best = ob;
                bi = oi;
            }
        }
        if (lane == 0) {
            wv[wid] = best;
            wi[wid] = bi;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = wv[0];
            int p = wi[0];
            for (int w = 1; w < nw; ++w)
                if (wv[w] > b || (wv[w] == b && wi[w] < p)) {
                    b = wv[w];
                    p = wi[w];
                }
            pivs = p;
            if (!(b > 0.0) && *info == 0) *info = k + 1;
        }
        __syncthreads();
        const int p = pivs;
        if (p != k)
            for (int c = threadIdx.x; c < ld; c += blockDim.x) {
                const double t = A[(int64_t)k * ld + c];
                A[(int64_t)k * ld + c] = A[(int64_t)p * ld + c];
                A[(int64_t)p * ld + c] = t;
            }
        __syncthreads();
        const double pv = A[(int64_t)k * ld + k];
        const double ipv = pv != 0.0 ? 1.0 / pv : 0.0;
        __syncthreads();
        for (int c = threadIdx.x; c < ld; c += blockDim.x) A[(int64_t)k * ld + c] *= ipv;
        for (int r = threadIdx.x; r < n; r += blockDim.x) fac[r] = (r == k) ? 0.0 : A[(int64_t)r * ld + k];
        __syncthreads();
        // eliminate column k from every other row (columns k.. of the left half, all of the right)
        for (int r = 0; r < n; ++r) {
            const double f = fac[r];
            if (f == 0.0) continue;
            for (int c = k + threadIdx.x; c < ld; c += blockDim.x) A[(int64_t)r * ld + c] -= f * A[(int64_t)k * ld + c];
        }
        __syncthreads();
    }
    for (int r = threadIdx.x; r < n; r += blockDim.x) piv[r] = r;
}
// Gauss-Jordan elimination with partial pivoting by one thread-block cluster: block r of the
// cluster keeps rows [r*rpc, (r+1)*rpc) of Aug in shared memory.  Pivot k: every block proposes
// its largest |A[row][k]| among rows not yet used as pivots (ties: lower row), the cluster picks
// the largest; every block copies the pivot row out of the owner's shared memory, and after a
// cluster barrier eliminates column k from its rows while the owner scales the pivot row.  Rows
// are not swapped: piv[k] records the pivot row of column k, so inverse row k = Aug[piv[k]][n:].
__global__ void __launch_bounds__(256) k_gauss_jordan_cluster(double* __restrict__ A, int n, int rpc,
                                                              int* __restrict__ info, int* __restrict__ piv) {
    pdl_entry();
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ double sm[];
    const int ld = 2 * n;
    double* rows = sm;                          // rpc x ld
    double* prow = sm + (size_t)rpc * ld;       // ld
    double* fac = prow + ld;                    // rpc
    __shared__ double candVal;
    __shared__ int candRow;
    __shared__ double pivVal;
    __shared__ int pivRow;
    __shared__ int usedLocal[64];
    const int rank = (int)cluster.block_rank();
    const int csize = (int)cluster.num_blocks();
    const int r0 = rank * rpc;
    for (int q = threadIdx.x; q < rpc * ld; q += blockDim.x) rows[q] = A[(size_t)r0 * ld + q];
    if (threadIdx.x < rpc) usedLocal[threadIdx.x] = 0;
    if (rank == 0 && threadIdx.x == 0) *info = 0;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (threadIdx.x < 32) {
            double best = -1.0;
            int bi = n;
            for (int r = threadIdx.x; r < rpc; r += 32) {
                if (usedLocal[r]) continue;
                const double a = fabs(rows[(size_t)r * ld + k]);
                if (a > best) {
                    best = a;
                    bi = r0 + r;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) {
                    best = ob;
                    bi = oi;
                }
            }
            if (threadIdx.x == 0) {
                candVal = best;
                candRow = bi;
            }
        }
        cluster.sync();
        // warp 0 gathers the cluster's candidates (lane b reads block b) and broadcasts the pivot
        if (threadIdx.x < 32) {
            double best = -1.0;
            int bi = n;
            if ((int)threadIdx.x < csize) {
                best = *cluster.map_shared_rank(&candVal, (int)threadIdx.x);
                bi = *cluster.map_shared_rank(&candRow, (int)threadIdx.x);
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) {
                    best = ob;
                    bi = oi;
                }
            }
            if (threadIdx.x == 0) {
                pivVal = best;
                pivRow = bi;
            }
        }
        __syncthreads();
        const double best = pivVal;
        const int p = pivRow;
        const int owner = p / rpc, pl = p - owner * rpc;
        const double* src = cluster.map_shared_rank(rows, owner) + (size_t)pl * ld;
        for (int c = k + threadIdx.x; c < ld; c += blockDim.x) prow[c] = src[c];
        for (int r = threadIdx.x; r < rpc; r += blockDim.x) fac[r] = (r0 + r == p) ? 0.0 : rows[(size_t)r * ld + k];
        if (rank == 0 && threadIdx.x == 0) {
            piv[k] = p;
            if (!(best > 0.0) && *info == 0) *info = k + 1;
        }
        cluster.sync();
        const double pv = prow[k];
        const double ipv = pv != 0.0 ? 1.0 / pv : 0.0;
        for (int r = 0; r < rpc; ++r) {
            if (r0 + r == p) {
                for (int c = k + threadIdx.x; c < ld; c += blockDim.x) rows[(size_t)r * ld + c] = prow[c] * ipv;
                if (threadIdx.x == 0) usedLocal[r] = 1;
                continue;
            }
            const double f = fac[r] * ipv;
            if (f == 0.0) continue;
            for (int c = k + threadIdx.x; c < ld; c += blockDim.x) rows[(size_t)r * ld + c] -= f * prow[c];
        }
        __syncthreads();
    }
    for (int q = threadIdx.x; q < rpc * ld; q += blockDim.x) A[(size_t)r0 * ld + q] = rows[q];
}

void launch_gauss_jordan(double* Aug, int n, int* info, int* piv, cudaStream_t s) {
    for (int cs : {16, 8}) {
        if (n % cs != 0) continue;
        const int rpc = n / cs;
        if (rpc > 64) continue;
        const size_t smem = sizeof(double) * ((size_t)rpc * 2 * n + 2 * n + rpc);
        if (smem > 200 * 1024) continue;
        cudaFuncSetAttribute(k_gauss_jordan_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (cs > 8) cudaFuncSetAttribute(k_gauss_jordan_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cs);
        cfg.blockDim = dim3(256);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int clusters = 0;
        if (cudaOccupancyMaxActiveClusters(&clusters, k_gauss_jordan_cluster, &cfg) != cudaSuccess || clusters < 1) {
            cudaGetLastError();
            continue;
        }
        if (cudaLaunchKernelEx(&cfg, k_gauss_jordan_cluster, Aug, n, rpc, info, piv) == cudaSuccess) return;
        cudaGetLastError();
    }
    launch_pdl(k_gauss_jordan, 1, 1024, sizeof(double) * n, s, Aug, n, info, piv);
}

// Pinv = (L0 + Z Z^T)^{-1} - Z Z^T, the pseudo-inverse of the symmetric L0 whose kernel is span Z;
// row r of the inverse is the right half of Aug's pivot row piv[r].
__global__ void k_extract_pinv(const double* __restrict__ Aug, const int* __restrict__ piv, int n, int N0, double rho,
                               double* __restrict__ P) {
    pdl_entry();
    const int r = blockIdx.y;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int n0 = N0 * N0;
    double v = Aug[(int64_t)piv[r] * 2 * n + n + c];
    const int br = r / n0, bc = c / n0;
    if (br == bc && (rho == 0.0 || br == 2)) v -= 1.0 / (double)n0;
    P[(int64_t)r * n + c] = v;
}
void launch_extract_pinv(const double* Aug, const int* piv, int n, int N0, double rho, double* Pinv, cudaStream_t s) {
    launch_pdl(k_extract_pinv, dim3((n + 127) / 128, n), 128, 0, s, Aug, piv, n, N0, rho, Pinv);
}

// x = Pinv b, one warp per row, FP64 accumulation for both precisions
template <typename T>
__global__ void k_coarse_apply(const double* __restrict__ P, int n, const T* __restrict__ b, T* __restrict__ x) {
    pdl_entry();
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= n) return;
    const double* row = P + (int64_t)r * n;
    double s = 0.0;
    for (int c = lane; c < n; c += 32) s += row[c] * (double)b[c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) x[r] = (T)s;
}
template <typename T>
void launch_coarse_apply(const double* Pinv, int n, const T* b, T* x, cudaStream_t s) {
    launch_pdl(k_coarse_apply<T>, (n + 7) / 8, 256, 0, s, Pinv, n, b, x);
}
template void launch_coarse_apply<float>(const double*, int, const float*, float*, cudaStream_t);
template void launch_coarse_apply<double>(const double*, int, const double*, double*, cudaStream_t);

__global__ void k_check_finite(const double* __restrict__ x, int64_t n, int* __restrict__ flag) {
    pdl_entry();
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(x[k])) *flag = 1;
}
void launch_check_finite(const double* x, int64_t n, int* flag, cudaStream_t s) {
    if (n == 0) return;
    launch_pdl(k_check_finite, num_blocks_for(n), 256, 0, s, x, n, flag);
}


// ------------------------------------------------------------------------------------------
// Flexible GMRES cycle on the device (the same recurrence as the host loop: CGS2 Arnoldi,
// Givens rotations, stop at ||r|| <= tol, at the cycle length or at the iteration cap).
__global__ void k_fg_init(FgDev* st, double beta, int m, int max_it, double tol) {
    pdl_entry();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    st->j = 0;
    st->jn = 0;
    st->its = 0;
    st->k = 0;
    st->converged = 0;
    st->m = m;
    st->max_it = max_it;
    st->tol = tol;
    st->est = beta;
    st->beta = beta;
    st->inv_hn = 0.0;
    for (int i = 0; i <= FG_MAXM; ++i) st->g[i] = 0.0;
    st->g[0] = beta;
    st->hist[0] = beta;
}
void launch_fg_init(FgDev* st, double beta, int m, int max_it, double tol, cudaStream_t s) {
    launch_pdl(k_fg_init, 1, 1, 0, s, st, beta, m, max_it, tol);
}

// Start of Arnoldi step j = st->jn: for j > 0 the new basis vector V_j = w / h_{j,j-1} (w, the
// orthogonalised product of the previous step, and 1/h from its norm) is stored; V_j, cast to
// the V-cycle precision, becomes the finest level's right-hand side.
template <typename T>
__global__ void k_fg_prep(double* __restrict__ V, const double* __restrict__ w, int64_t n, FgDev* st,
                          T* __restrict__ dst) {
    pdl_entry();
    const int j = st->jn;
    double* v = V + (int64_t)j * n;
    const double inv = st->inv_hn;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        double x;
        if (j == 0) {
            x = v[e];
        } else {
            x = w[e] * inv;
            v[e] = x;
        }
        dst[e] = (T)x;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) st->j = j;
}
template <typename T>
void launch_fg_prep(double* V, const double* w, int64_t n, FgDev* st, T* dst, cudaStream_t s) {
    launch_pdl(k_fg_prep<T>, num_blocks_for(n), 256, 0, s, V, w, n, st, dst);
}

template <typename T>
__global__ void k_fg_zstore(const T* __restrict__ src, double* __restrict__ Z, int64_t n, const FgDev* st,
                            double* __restrict__ zcur) {
    pdl_entry();
    double* z = Z + (int64_t)st->j * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const double v = (double)src[e];
        z[e] = v;
        zcur[e] = v;
    }
}
template <typename T>
void launch_fg_zstore(const T* src, double* Z, int64_t n, const FgDev* st, double* zcur, cudaStream_t s) {
    launch_pdl(k_fg_zstore<T>, num_blocks_for(n), 256, 0, s, src, Z, n, st, zcur);
}
template void launch_fg_prep<float>(double*, const double*, int64_t, FgDev*, float*, cudaStream_t);
template void launch_fg_prep<double>(double*, const double*, int64_t, FgDev*, double*, cudaStream_t);
template void launch_fg_zstore<float>(const float*, double*, int64_t, const FgDev*, double*, cudaStream_t);
template void launch_fg_zstore<double>(const double*, double*, int64_t, const FgDev*, double*, cudaStream_t);

// partials[i * S + s] = slice s of V_i . w for all i <= j, one warp per (vector, slice).  The
// launch has a fixed number of warps (MD_WARPS); the slice count S = md_slices(j) spreads them
// over the j + 1 vectors, so a short basis gets many short slices (latency) and a long one few
// long slices (the FP64 pipe is the limit there).  Lanes keep four independent sums.
constexpr int MD_BLOCKS = 202;
constexpr int MD_WARPS = MD_BLOCKS * 8;
__device__ __forceinline__ int md_slices(int j) {
    const int s = MD_WARPS / (j + 1);
    return s < 16 ? 16 : (s > 512 ? 512 : s);
}
__global__ void __launch_bounds__(256) k_multidot_dev(const double* __restrict__ V, int64_t ld,
                                                      const double* __restrict__ w, int64_t n,
                                                      double* __restrict__ partials, const FgDev* st) {
    pdl_entry();
    const int j = st->j;
    const int S = md_slices(j);
    const int lane = threadIdx.x & 31;
    const int lanes_total = MD_WARPS * 32;
    for (int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; gw < (j + 1) * S; gw += lanes_total >> 5) {
        const int i = gw / S, sl = gw - i * S;
        const int64_t len = (n + S - 1) / S;
        const int64_t e0 = sl * len, e1 = e0 + len < n ? e0 + len : n;
        const double* v = V + (int64_t)i * ld;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int64_t e = e0 + lane;
        for (; e + 96 < e1; e += 128) {
            a0 += v[e] * w[e];
            a1 += v[e + 32] * w[e + 32];
            a2 += v[e + 64] * w[e + 64];
            a3 += v[e + 96] * w[e + 96];
        }
        for (; e < e1; e += 32) a0 += v[e] * w[e];
        double t = (a0 + a1) + (a2 + a3);
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) partials[(int64_t)i * S + sl] = t;
    }
}
void launch_multidot_dev(const double* V, int64_t ld, const double* w, int64_t n, double* partials,
                         const FgDev* st, cudaStream_t s) {
    launch_pdl(k_multidot_dev, MD_BLOCKS, 256, 0, s, V, ld, w, n, partials, st);
}
// out[i] = sum of the partials of vector i in slice order: for i <= j with S = md_slices(j)
// partials each (nblk = 0), or for i < count with nblk partials each
__global__ void k_reduce_partials_dev(const double* __restrict__ partials, int nblk, double* __restrict__ out,
                                      const FgDev* st, int count) {
    pdl_entry();
    const int k = count > 0 ? count : st->j + 1;
    const int S = nblk > 0 ? nblk : md_slices(st->j);
    if ((int)blockIdx.x >= k) return;
    double s = 0.0;
    for (int b = threadIdx.x; b < S; b += blockDim.x) s += partials[(int64_t)blockIdx.x * S + b];
    s = block_sum(s);
    if (threadIdx.x == 0) out[blockIdx.x] = s;
}
void launch_reduce_partials_dev(const double* partials, int nblk, double* out, const FgDev* st, int count,
                                cudaStream_t s) {
    launch_pdl(k_reduce_partials_dev, count > 0 ? count : FG_MAXM + 1, 128, 0, s, partials, nblk, out, st, count);
}
// y += sign * sum_{i<k} coef[i] V_i with k = j + 1 (useK = 0) or k = st->k (useK = 1)
__global__ void k_multi_axpy_dev(const double* __restrict__ V, int64_t ld, const double* __restrict__ coef,
                                 double sign, double* __restrict__ y, int64_t n, const FgDev* st, int useK) {
    pdl_entry();
    __shared__ double c[FG_MAXM + 1];
    const int k = useK ? st->k : st->j + 1;
    for (int t = threadIdx.x; t < k; t += blockDim.x) c[t] = sign * coef[t];
    __syncthreads();
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        double acc = y[e];
        for (int i = 0; i < k; ++i) acc += c[i] * V[(int64_t)i * ld + e];
        y[e] = acc;
    }
}
void launch_multi_axpy_dev(const double* V, int64_t ld, const double* coef, double sign, double* y, int64_t n,
                           const FgDev* st, int useK, cudaStream_t s) {
    launch_pdl(k_multi_axpy_dev, num_blocks_for(n), 256, 0, s, V, ld, coef, sign, y, n, st, useK);
}

// The same update with k = j + 1, and the block partial sums of ||y||^2 of the result.
__global__ void k_multi_axpy_norm_dev(const double* __restrict__ V, int64_t ld, const double* __restrict__ coef,
                                      double sign, double* __restrict__ y, int64_t n, const FgDev* st,
                                      double* __restrict__ partials) {
    pdl_entry();
    __shared__ double c[FG_MAXM + 1];
    const int k = st->j + 1;
    for (int t = threadIdx.x; t < k; t += blockDim.x) c[t] = sign * coef[t];
    __syncthreads();
    double ss = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        double acc = y[e];
        for (int i = 0; i < k; ++i) acc += c[i] * V[(int64_t)i * ld + e];
        y[e] = acc;
        ss += acc * acc;
    }
    ss = block_sum(ss);
    if (threadIdx.x == 0) partials[blockIdx.x] = ss;
}
int launch_multi_axpy_norm_dev(const double* V, int64_t ld, const double* coef, double sign, double* y, int64_t n,
                               const FgDev* st, double* partials, cudaStream_t s) {
    const int nb = num_blocks_for(n);
    launch_pdl(k_multi_axpy_norm_dev, nb, 256, 0, s, V, ld, coef, sign, y, n, st, partials);
    return nb;
}

// One thread: Hessenberg column j from the two Gram-Schmidt passes, previous and new Givens
// rotation, residual estimate, and the loop decision (always terminates: the iteration cap and
// the cycle length bound it, and a non-finite estimate or a zero new norm stops it).
__global__ void k_fg_arnoldi(FgDev* st, const double* __restrict__ h1, const double* __restrict__ h2,
                             const double* __restrict__ nrm, cudaGraphConditionalHandle handle) {
    pdl_entry();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int j = st->j;
    double* Hj = st->H + (size_t)j * (FG_MAXM + 1);
    for (int i = 0; i <= j; ++i) Hj[i] = h1[i] + h2[i];
    const double hn = sqrt(nrm[0]);
    Hj[j + 1] = hn;
    for (int i = 0; i < j; ++i) {
        const double a = Hj[i], b = Hj[i + 1];
        Hj[i] = st->cs[i] * a + st->sn[i] * b;
        Hj[i + 1] = -st->sn[i] * a + st->cs[i] * b;
    }
    const double d = hypot(Hj[j], Hj[j + 1]);
    st->cs[j] = Hj[j] / d;
    st->sn[j] = Hj[j + 1] / d;
    Hj[j] = d;
    Hj[j + 1] = 0.0;
    st->g[j + 1] = -st->sn[j] * st->g[j];
    st->g[j] = st->cs[j] * st->g[j];
    const double est = fabs(st->g[j + 1]);
    st->its += 1;
    st->est = est;
    st->hist[j + 1] = est;
    const bool conv = est <= st->tol;
    const bool stop = conv || !(hn > 0.0) || !isfinite(est) || !isfinite(d) || st->its >= st->max_it || j + 1 >= st->m;
    st->inv_hn = hn > 0.0 ? 1.0 / hn : 0.0;
    st->jn = j + 1;
    if (stop) {
        st->k = j + 1;
        st->converged = (conv || hn == 0.0) ? 1 : 0;   // a zero new direction: the solution is exact
    }
    cudaGraphSetConditional(handle, stop ? 0u : 1u);
}
void launch_fg_arnoldi(FgDev* st, const double* h1, const double* h2, const double* nrm,
                       cudaGraphConditionalHandle handle, cudaStream_t s) {
    launch_pdl(k_fg_arnoldi, 1, 32, 0, s, st, h1, h2, nrm, handle);
}

// y = H^{-1} g on the k x k upper triangle (one thread)
__global__ void k_fg_backsolve(FgDev* st) {
    pdl_entry();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int k = st->k;
    for (int i = k - 1; i >= 0; --i) {
        double acc = st->g[i];
        for (int q = i + 1; q < k; ++q) acc -= st->H[(size_t)q * (FG_MAXM + 1) + i] * st->y[q];
        st->y[i] = acc / st->H[(size_t)i * (FG_MAXM + 1) + i];
    }
}
void launch_fg_backsolve(FgDev* st, cudaStream_t s) { launch_pdl(k_fg_backsolve, 1, 32, 0, s, st); }

}  // namespace sib
