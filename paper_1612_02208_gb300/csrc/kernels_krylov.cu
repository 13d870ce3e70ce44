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

// Blocked Gauss-Jordan inversion with partial pivoting of Aug = [A | I] (n x 2n, row-major), in
// panels of GJ_B columns.  For the panel Q = columns [c0, c0 + GJ_B):
//   1. one block selects the panel's pivot rows P by partial pivoting on a working copy of the
//      panel's candidate rows (largest |a| among rows not yet pivots, ties to the lower row, the
//      copy eliminated as unblocked elimination would), and inverts the pivot block A_PQ in FP64
//      with its pivots on the diagonal in selection order.  The working copy only chooses rows --
//      the result is computed from the FP64 panel and A_PQ^{-1} -- so it is kept in FP32: one SM's
//      FP64 rate made an FP64 copy cost ~120 us a panel, and FP32 can change a choice only between
//      candidates equal to rounding, which partial pivoting leaves free;
//   2. column slabs form the new pivot rows  W = A_PQ^{-1} A_P  on the columns right of Q;
//   3. every other row r becomes  A_r - A_rQ W  there (A_rQ: its panel entries before the panel's
//      elimination), and its panel entries 0 (the pivot rows' panel entries become unit vectors).
// Rows are never swapped: piv[k] is the pivot row of column k and row k of A^{-1} is
// Aug[piv[k]][n:].  info = 0, or k + 1 for the first pivot column without a nonzero candidate.
// The panel steps are sequential but tiny; the O(n^3) work of step 3 spreads over the GPU, whose
// FP64 rate is low per SM.
constexpr int GJ_B = 16;

struct GjWork {
    double* Q0;   // n x GJ_B: the panel before its elimination
    double* G;    // GJ_B x GJ_B: A_PQ^{-1}
    double* W;    // GJ_B x 2n: the new pivot rows
    int* used;    // n: row already a pivot
    int* prow;    // GJ_B: the panel's pivot rows in selection order
};
static GjWork gj_work(void* base, int n) {
    GjWork w;
    double* d = static_cast<double*>(base);
    w.Q0 = d;
    w.G = w.Q0 + (size_t)n * GJ_B;
    w.W = w.G + GJ_B * GJ_B;
    w.used = reinterpret_cast<int*>(w.W + (size_t)GJ_B * 2 * n);
    w.prow = w.used + n;
    return w;
}
size_t gauss_jordan_work_bytes(int n) {
    return sizeof(double) * ((size_t)n * GJ_B + GJ_B * GJ_B + (size_t)GJ_B * 2 * n) + sizeof(int) * (size_t)(n + GJ_B);
}

__global__ void __launch_bounds__(512) k_gj_panel(const double* __restrict__ A, int n, int c0, GjWork w,
                                                  int* __restrict__ piv, int* __restrict__ info) {
    pdl_entry();
    extern __shared__ float smf[];
    float* Wp = smf;                                      // n x GJ_B working copy of the panel
    float* fac = Wp + (size_t)n * GJ_B;                   // n: column t before the pivot's elimination
    int* usedS = reinterpret_cast<int*>(fac + n);         // n
    __shared__ float prowv[GJ_B];
    __shared__ double Mx[GJ_B][2 * GJ_B];
    __shared__ double colv[GJ_B], rowv[2 * GJ_B];
    __shared__ float wv[32];
    __shared__ int wi[32];
    __shared__ int pS[GJ_B];
    const int ld = 2 * n, lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (c0 == 0 && threadIdx.x == 0) *info = 0;
    for (int q = threadIdx.x; q < n * GJ_B; q += blockDim.x) {
        const double v = A[(size_t)(q / GJ_B) * ld + c0 + (q % GJ_B)];
        Wp[q] = (float)v;
        w.Q0[q] = v;
    }
    for (int r = threadIdx.x; r < n; r += blockDim.x) usedS[r] = c0 == 0 ? 0 : w.used[r];
    __syncthreads();
    for (int t = 0; t < GJ_B; ++t) {
        float best = -1.0f;
        int bi = n;
        for (int r = threadIdx.x; r < n; r += blockDim.x) {
            if (usedS[r]) continue;
            const float a = fabsf(Wp[r * GJ_B + t]);
            if (a > best) {
                best = a;
                bi = r;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, o);
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
        if (wid == 0) {
            best = lane < nw ? wv[lane] : -1.0f;
            bi = lane < nw ? wi[lane] : n;
            for (int o = 16; o > 0; o >>= 1) {
                const float ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) {
                    best = ob;
                    bi = oi;
                }
            }
            if (lane == 0) {
                pS[t] = bi;
                usedS[bi] = 1;
            }
        }
        __syncthreads();
        const int p = pS[t];
        for (int r = threadIdx.x; r < n; r += blockDim.x) fac[r] = Wp[r * GJ_B + t];
        if (threadIdx.x < GJ_B) prowv[threadIdx.x] = Wp[p * GJ_B + threadIdx.x];
        __syncthreads();
        const float pv = prowv[t];
        const float ipv = pv != 0.0f ? 1.0f / pv : 0.0f;
        for (int q = threadIdx.x; q < n * GJ_B; q += blockDim.x) {   // candidate rows only
            const int r = q / GJ_B, tt = q % GJ_B;
            if (tt <= t || usedS[r]) continue;
            const float f = fac[r] * ipv;
            if (f != 0.0f) Wp[q] -= f * prowv[tt];
        }
        __syncthreads();
    }
    // G = A_PQ^{-1} in FP64: Gauss-Jordan on [A_PQ | I] with the pivots on the diagonal.  At step t
    // the left columns < t are already unit vectors and the right columns > B + t still zero off
    // the diagonal, so only columns [t, B + t] change (besides the diagonal's own unit entries).
    for (int q = threadIdx.x; q < GJ_B * 2 * GJ_B; q += blockDim.x) {
        const int t = q / (2 * GJ_B), u = q % (2 * GJ_B);
        Mx[t][u] = u < GJ_B ? w.Q0[pS[t] * GJ_B + u] : (u - GJ_B == t ? 1.0 : 0.0);
    }
    __syncthreads();
    for (int t = 0; t < GJ_B; ++t) {
        if (threadIdx.x < GJ_B) colv[threadIdx.x] = Mx[threadIdx.x][t];
        if (threadIdx.x < 2 * GJ_B) rowv[threadIdx.x] = Mx[t][threadIdx.x];
        __syncthreads();
        if (threadIdx.x == 0 && !(colv[t] != 0.0) && *info == 0) *info = c0 + t + 1;
        const double ipv = colv[t] != 0.0 ? 1.0 / colv[t] : 0.0;
        for (int q = threadIdx.x; q < GJ_B * 2 * GJ_B; q += blockDim.x) {
            const int s2 = q / (2 * GJ_B), u = q % (2 * GJ_B);
            if (u < t || u > GJ_B + t) continue;
            if (s2 == t)
                Mx[s2][u] = rowv[u] * ipv;
            else
                Mx[s2][u] -= colv[s2] * ipv * rowv[u];
        }
        __syncthreads();
    }
    for (int q = threadIdx.x; q < GJ_B * GJ_B; q += blockDim.x) w.G[q] = Mx[q / GJ_B][GJ_B + q % GJ_B];
    if (threadIdx.x < GJ_B) {
        w.prow[threadIdx.x] = pS[threadIdx.x];
        piv[c0 + threadIdx.x] = pS[threadIdx.x];
    }
    for (int r = threadIdx.x; r < n; r += blockDim.x) w.used[r] = usedS[r];
}

// W = A_PQ^{-1} A_P on columns c >= c0 + GJ_B, written to the work array and into the pivot rows;
// block (16 x 16): a slab of 16 columns, thread (x, y) = (column, pivot t)
__global__ void __launch_bounds__(GJ_B * 16) k_gj_w(double* __restrict__ A, int n, int c0, GjWork w) {
    pdl_entry();
    __shared__ double ap[GJ_B][16];
    __shared__ double g[GJ_B][GJ_B];
    const int ld = 2 * n;
    const int c = c0 + GJ_B + blockIdx.x * 16 + threadIdx.x;
    const int t = threadIdx.y;
    g[t][threadIdx.x] = w.G[t * GJ_B + threadIdx.x];
    ap[t][threadIdx.x] = c < ld ? A[(size_t)w.prow[t] * ld + c] : 0.0;
    __syncthreads();
    if (c >= ld) return;
    double acc = 0.0;
#pragma unroll
    for (int u = 0; u < GJ_B; ++u) acc += g[t][u] * ap[u][threadIdx.x];
    w.W[(size_t)t * ld + c] = acc;
    A[(size_t)w.prow[t] * ld + c] = acc;
}

// Other rows: A_r -= A_rQ W on columns right of the panel, and their panel entries 0;
// the pivot rows' panel entries become unit vectors.  Block (row r, slab of 128 columns from c0).
__global__ void __launch_bounds__(128) k_gj_rows(double* __restrict__ A, int n, int c0, GjWork w) {
    pdl_entry();
    __shared__ double m[GJ_B];
    __shared__ int piv_t;
    const int ld = 2 * n, r = blockIdx.x;
    const int c = c0 + blockIdx.y * 128 + threadIdx.x;
    if (threadIdx.x == 0) {
        int pt = -1;
        for (int t = 0; t < GJ_B; ++t)
            if (w.prow[t] == r) pt = t;
        piv_t = pt;
    }
    if (threadIdx.x < GJ_B) m[threadIdx.x] = w.Q0[(size_t)r * GJ_B + threadIdx.x];
    __syncthreads();
    if (c >= ld) return;
    const int pt = piv_t;
    if (c < c0 + GJ_B) {
        A[(size_t)r * ld + c] = (pt >= 0 && c - c0 == pt) ? 1.0 : 0.0;
        return;
    }
    if (pt >= 0) return;   // pivot rows: written by k_gj_w
    double acc = A[(size_t)r * ld + c];
#pragma unroll
    for (int u = 0; u < GJ_B; ++u) acc -= m[u] * w.W[(size_t)u * ld + c];
    A[(size_t)r * ld + c] = acc;
}

void launch_gauss_jordan(double* Aug, int n, int* info, int* piv, void* work, cudaStream_t s) {
    const GjWork w = gj_work(work, n);
    const size_t smem = sizeof(float) * ((size_t)n * GJ_B + n) + sizeof(int) * (size_t)n;
    cudaFuncSetAttribute(k_gj_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int ld = 2 * n;
    for (int c0 = 0; c0 < n; c0 += GJ_B) {
        launch_pdl(k_gj_panel, 1, 512, smem, s, (const double*)Aug, n, c0, w, piv, info);
        const int R = ld - c0 - GJ_B;
        launch_pdl(k_gj_w, dim3((R + 15) / 16), dim3(16, GJ_B), 0, s, Aug, n, c0, w);
        launch_pdl(k_gj_rows, dim3(n, (ld - c0 + 127) / 128), dim3(128), 0, s, Aug, n, c0, w);
    }
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

// xo = x + omega P r, one warp per row, FP64 accumulation (x == nullptr: 0)
template <typename T>
__global__ void k_dense_correct(const double* __restrict__ P, int n, const T* __restrict__ r, const T* x, T omega,
                                T* xo) {
    pdl_entry();
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= n) return;
    const double* pr = P + (int64_t)row * n;
    double s = 0.0;
    for (int c = lane; c < n; c += 32) s += pr[c] * (double)r[c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) xo[row] = (T)((x ? (double)x[row] : 0.0) + (double)omega * s);
}
template <typename T>
void launch_dense_correct(const double* P, int n, const T* r, const T* x, T omega, T* xo, cudaStream_t s) {
    launch_pdl(k_dense_correct<T>, (n + 7) / 8, 256, 0, s, P, n, r, x, omega, xo);
}
template void launch_dense_correct<float>(const double*, int, const float*, const float*, float, float*, cudaStream_t);
template void launch_dense_correct<double>(const double*, int, const double*, const double*, double, double*,
                                           cudaStream_t);

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
