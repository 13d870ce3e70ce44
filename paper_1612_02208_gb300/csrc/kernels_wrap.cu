// Kernels of the Krylov-wrapped smoothing step (Sec. 3.3): a pre- or post-smoothing stage of nu
// sweeps becomes nu iterations of flexible GMRES on the level's residual equation, each
// preconditioned by one undamped sweep of the basic smoother.  The level vectors are in the
// V-cycle's precision T; inner products are summed in FP64 in a fixed order (block partials, then
// one block), the small Hessenberg least-squares problem is solved in FP64 by one thread.
#include "sib_internal.h"

namespace sib {

namespace {

__device__ __forceinline__ double wblock_sum(double v, double* ws) {
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

// partials[i * gridDim.x + block] = block's share of V_i . w, i < cnt (cnt <= WRAP_MAXK + 1)
template <typename T>
__global__ void __launch_bounds__(256) k_wdots(const T* __restrict__ V, int64_t ld, int cnt, const T* __restrict__ w,
                                               int64_t n, double* __restrict__ partials) {
    pdl_entry();
    __shared__ double ws[32];
    double acc[WRAP_MAXK + 1];
#pragma unroll
    for (int i = 0; i <= WRAP_MAXK; ++i) acc[i] = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const double we = (double)w[e];
#pragma unroll
        for (int i = 0; i <= WRAP_MAXK; ++i)
            if (i < cnt) acc[i] += (double)V[(int64_t)i * ld + e] * we;
    }
    for (int i = 0; i < cnt; ++i) {
        const double s = wblock_sum(acc[i], ws);
        if (threadIdx.x == 0) partials[(int64_t)i * gridDim.x + blockIdx.x] = s;
    }
}

// out[i] = sum over blocks of partials of vector i (block order), i < cnt; one block per vector
__global__ void k_wreduce(const double* __restrict__ partials, int nblk, double* __restrict__ out) {
    pdl_entry();
    __shared__ double ws[32];
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += partials[(int64_t)blockIdx.x * nblk + b];
    s = wblock_sum(s, ws);
    if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// yout = yin + sign * sum_{i < cnt} coef[i] V_i   (yin == nullptr: 0)
template <typename T>
__global__ void k_wmaxpy(const T* __restrict__ V, int64_t ld, int cnt, const double* __restrict__ coef, double sign,
                         const T* yin, T* yout, int64_t n) {
    pdl_entry();
    __shared__ T c[WRAP_MAXK + 1];
    if (threadIdx.x < cnt) c[threadIdx.x] = (T)(sign * coef[threadIdx.x]);
    __syncthreads();
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        T acc = yin ? yin[e] : T(0);
        for (int i = 0; i < cnt; ++i) acc += c[i] * V[(int64_t)i * ld + e];
        yout[e] = acc;
    }
}

// v = w / sqrt(nrm2[0]), or 0 when the norm is zero (a vanished Arnoldi vector)
template <typename T>
__global__ void k_wscale(const T* __restrict__ w, const double* __restrict__ nrm2, T* __restrict__ v, int64_t n) {
    pdl_entry();
    const double s = nrm2[0] > 0.0 ? 1.0 / sqrt(nrm2[0]) : 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        v[e] = (T)((double)w[e] * s);
}

// y = argmin || beta e1 - H y || for the (m + 1) x m Hessenberg matrix of the step (Givens
// rotations, back substitution).  H(i, j) = hA[j][i] + hB[j][i] for i <= j (the two Gram-Schmidt
// passes), H(j + 1, j) = sqrt(nr[j]); m stops at the first vanished subdiagonal entry.  y[m..k) = 0.
__global__ void k_wlsq(const double* __restrict__ hA, const double* __restrict__ hB, const double* __restrict__ nr,
                       const double* __restrict__ beta2, int k, double* __restrict__ y) {
    pdl_entry();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double H[WRAP_MAXK + 1][WRAP_MAXK];
    double g[WRAP_MAXK + 1];
    const double beta = sqrt(beta2[0]);
    int m = 0;
    for (int j = 0; j < k; ++j) {
        for (int i = 0; i <= j; ++i) H[i][j] = hA[j * (WRAP_MAXK + 1) + i] + hB[j * (WRAP_MAXK + 1) + i];
        H[j + 1][j] = sqrt(nr[j]);
        m = j + 1;
        if (!(H[j + 1][j] > 0.0)) break;
    }
    for (int j = 0; j < k; ++j) y[j] = 0.0;
    if (!(beta > 0.0)) return;
    for (int i = 0; i <= m; ++i) g[i] = i == 0 ? beta : 0.0;
    for (int j = 0; j < m; ++j) {   // rotate H(j, j), H(j + 1, j) to (r, 0)
        const double a = H[j][j], b = H[j + 1][j];
        const double d = hypot(a, b);
        const double cs = d > 0.0 ? a / d : 1.0, sn = d > 0.0 ? b / d : 0.0;
        for (int q = j; q < m; ++q) {
            const double u = H[j][q], v = H[j + 1][q];
            H[j][q] = cs * u + sn * v;
            H[j + 1][q] = -sn * u + cs * v;
        }
        const double gu = g[j], gv = g[j + 1];
        g[j] = cs * gu + sn * gv;
        g[j + 1] = -sn * gu + cs * gv;
    }
    for (int i = m - 1; i >= 0; --i) {
        double acc = g[i];
        for (int q = i + 1; q < m; ++q) acc -= H[i][q] * y[q];
        y[i] = H[i][i] != 0.0 ? acc / H[i][i] : 0.0;
    }
}

}  // namespace

template <typename T>
void launch_wdots(const T* V, int64_t ld, int cnt, const T* w, int64_t n, double* partials, cudaStream_t s) {
    launch_pdl(k_wdots<T>, WRAP_BLK, 256, 0, s, V, ld, cnt, w, n, partials);
}
void launch_wreduce(const double* partials, int cnt, double* out, cudaStream_t s) {
    launch_pdl(k_wreduce, cnt, 128, 0, s, partials, WRAP_BLK, out);
}
template <typename T>
void launch_wmaxpy(const T* V, int64_t ld, int cnt, const double* coef, double sign, const T* yin, T* yout, int64_t n,
                   cudaStream_t s) {
    launch_pdl(k_wmaxpy<T>, num_blocks_for(n), 256, 0, s, V, ld, cnt, coef, sign, yin, yout, n);
}
template <typename T>
void launch_wscale(const T* w, const double* nrm2, T* v, int64_t n, cudaStream_t s) {
    launch_pdl(k_wscale<T>, num_blocks_for(n), 256, 0, s, w, nrm2, v, n);
}
void launch_wlsq(const double* hA, const double* hB, const double* nr, const double* beta2, int k, double* y,
                 cudaStream_t s) {
    launch_pdl(k_wlsq, 1, 32, 0, s, hA, hB, nr, beta2, k, y);
}

#define SIB_WRAP_INST(T)                                                                                    \
    template void launch_wdots<T>(const T*, int64_t, int, const T*, int64_t, double*, cudaStream_t);          \
    template void launch_wmaxpy<T>(const T*, int64_t, int, const double*, double, const T*, T*, int64_t,      \
                                   cudaStream_t);                                                           \
    template void launch_wscale<T>(const T*, const double*, T*, int64_t, cudaStream_t);
SIB_WRAP_INST(float)
SIB_WRAP_INST(double)

}  // namespace sib
