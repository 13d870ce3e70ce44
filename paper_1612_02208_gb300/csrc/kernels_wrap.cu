// Kernels of the Krylov-wrapped smoothing step (Sec. 3.3): a pre- or post-smoothing stage of nu
// sweeps becomes nu iterations of flexible GMRES on the level's residual equation, each
// preconditioned by one undamped sweep of the basic smoother.  The level vectors are in the
// V-cycle's precision T.  Inner products are formed per thread over 16-byte vectors of T (products
// of one vector summed in T), accumulated in FP64, reduced per block, and the block partials are
// summed by one block per product in block order: a fixed order, so results do not depend on
// timing.  The classical Gram-Schmidt update of each pass is fused with the inner products that
// follow it (the second pass's coefficients, or the norm).  The small Hessenberg least-squares
// problem is solved in FP64 by one thread.
#include "sib_internal.h"

namespace sib {

namespace {

template <typename T>
struct WVec;
template <>
struct WVec<float> {
    using type = float4;
    static constexpr int n = 4;
};
template <>
struct WVec<double> {
    using type = double2;
    static constexpr int n = 2;
};
template <typename T>
__device__ __forceinline__ T wv(const typename WVec<T>::type& v, int c);
template <>
__device__ __forceinline__ float wv<float>(const float4& v, int c) {
    return c == 0 ? v.x : c == 1 ? v.y : c == 2 ? v.z : v.w;
}
template <>
__device__ __forceinline__ double wv<double>(const double2& v, int c) {
    return c == 0 ? v.x : v.y;
}
template <typename T>
__device__ __forceinline__ void wset(typename WVec<T>::type& v, int c, T x);
template <>
__device__ __forceinline__ void wset<float>(float4& v, int c, float x) {
    if (c == 0) v.x = x;
    else if (c == 1) v.y = x;
    else if (c == 2) v.z = x;
    else v.w = x;
}
template <>
__device__ __forceinline__ void wset<double>(double2& v, int c, double x) {
    if (c == 0) v.x = x;
    else v.y = x;
}

constexpr int WT = 256;           // threads per block
constexpr int WW = WT / 32;       // warps per block

// Block sums of acc[i], i < cnt, written to partials[i * gridDim.x + blockIdx.x]: warp shuffles,
// then the warps' values in warp order.
template <int KC>
__device__ __forceinline__ void block_partials(double (&acc)[KC], int cnt, double* __restrict__ partials) {
    __shared__ double ws[KC][WW];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < KC; ++i) {
        if (i < cnt) {
            double v = acc[i];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) ws[i][wid] = v;
        }
    }
    __syncthreads();
    if (threadIdx.x < cnt) {
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < WW; ++q) s += ws[threadIdx.x][q];
        partials[(int64_t)threadIdx.x * gridDim.x + blockIdx.x] = s;
    }
}

// partials of V_i . w, i < cnt (cnt <= KC <= WRAP_MAXK + 1)
template <typename T, int KC>
__global__ void __launch_bounds__(WT) k_wdots(const T* __restrict__ V, int64_t ld, int cnt, const T* __restrict__ w,
                                              int64_t n, double* __restrict__ partials) {
    using VT = typename WVec<T>::type;
    constexpr int VN = WVec<T>::n;
    pdl_entry();
    double acc[KC];
#pragma unroll
    for (int i = 0; i < KC; ++i) acc[i] = 0.0;
    const int64_t nv = n / VN;
    for (int64_t e = blockIdx.x * (int64_t)WT + threadIdx.x; e < nv; e += (int64_t)gridDim.x * WT) {
        const VT we = reinterpret_cast<const VT*>(w)[e];
#pragma unroll
        for (int i = 0; i < KC; ++i) {
            if (i < cnt) {
                const VT vi = reinterpret_cast<const VT*>(V + (int64_t)i * ld)[e];
                T s = T(0);
#pragma unroll
                for (int c = 0; c < VN; ++c) s = fma(wv<T>(vi, c), wv<T>(we, c), s);
                acc[i] += (double)s;
            }
        }
    }
    for (int64_t e = nv * VN + blockIdx.x * (int64_t)WT + threadIdx.x; e < n; e += (int64_t)gridDim.x * WT)
#pragma unroll
        for (int i = 0; i < KC; ++i)
            if (i < cnt) acc[i] += (double)V[(int64_t)i * ld + e] * (double)w[e];
    block_partials(acc, cnt, partials);
}

// wout = win - sum_{i < cnt} coef[i] V_i, and then (MODE 1) partials of V_i . wout, i < cnt, or
// (MODE 2) the partial of wout . wout; cnt <= KC
template <typename T, int MODE, int KC>
__global__ void __launch_bounds__(WT) k_wgs(const T* __restrict__ V, int64_t ld, int cnt,
                                            const double* __restrict__ coef, const T* win, T* wout, int64_t n,
                                            double* __restrict__ partials) {
    using VT = typename WVec<T>::type;
    constexpr int VN = WVec<T>::n;
    pdl_entry();
    T cf[KC];
#pragma unroll
    for (int i = 0; i < KC; ++i) cf[i] = i < cnt ? (T)coef[i] : T(0);
    double acc[KC];
#pragma unroll
    for (int i = 0; i < KC; ++i) acc[i] = 0.0;
    const int64_t nv = n / VN;
    for (int64_t e = blockIdx.x * (int64_t)WT + threadIdx.x; e < nv; e += (int64_t)gridDim.x * WT) {
        VT y = reinterpret_cast<const VT*>(win)[e];
        VT vi[KC];
#pragma unroll
        for (int i = 0; i < KC; ++i)
            if (i < cnt) vi[i] = reinterpret_cast<const VT*>(V + (int64_t)i * ld)[e];
#pragma unroll
        for (int i = 0; i < KC; ++i)
            if (i < cnt)
#pragma unroll
                for (int c = 0; c < VN; ++c) wset<T>(y, c, fma(-cf[i], wv<T>(vi[i], c), wv<T>(y, c)));
        reinterpret_cast<VT*>(wout)[e] = y;
        if (MODE == 1) {
#pragma unroll
            for (int i = 0; i < KC; ++i) {
                if (i < cnt) {
                    T s = T(0);
#pragma unroll
                    for (int c = 0; c < VN; ++c) s = fma(wv<T>(vi[i], c), wv<T>(y, c), s);
                    acc[i] += (double)s;
                }
            }
        } else if (MODE == 2) {
            T s = T(0);
#pragma unroll
            for (int c = 0; c < VN; ++c) s = fma(wv<T>(y, c), wv<T>(y, c), s);
            acc[0] += (double)s;
        }
    }
    for (int64_t e = nv * VN + blockIdx.x * (int64_t)WT + threadIdx.x; e < n; e += (int64_t)gridDim.x * WT) {
        T y = win[e];
#pragma unroll
        for (int i = 0; i < KC; ++i)
            if (i < cnt) y = fma(-cf[i], V[(int64_t)i * ld + e], y);
        wout[e] = y;
        if (MODE == 1) {
#pragma unroll
            for (int i = 0; i < KC; ++i)
                if (i < cnt) acc[i] += (double)V[(int64_t)i * ld + e] * (double)y;
        } else if (MODE == 2) {
            acc[0] += (double)y * (double)y;
        }
    }
    if (MODE == 1) block_partials(acc, cnt, partials);
    else if (MODE == 2) block_partials(acc, 1, partials);
}

// out[i] = sum over the nblk block partials of product i, in block order; one block per product
__global__ void __launch_bounds__(WT) k_wreduce(const double* __restrict__ partials, int nblk, double* __restrict__ out) {
    pdl_entry();
    __shared__ double ws[WW];
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += WT) s += partials[(int64_t)blockIdx.x * nblk + b];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) ws[wid] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < WW; ++q) t += ws[q];
        out[blockIdx.x] = t;
    }
}

// yout = yin + sign * sum_{i < cnt} coef[i] V_i   (yin == nullptr: 0); cnt <= KC
template <typename T, int KC>
__global__ void __launch_bounds__(WT) k_wmaxpy(const T* __restrict__ V, int64_t ld, int cnt,
                                               const double* __restrict__ coef, double sign, const T* yin, T* yout,
                                               int64_t n) {
    using VT = typename WVec<T>::type;
    constexpr int VN = WVec<T>::n;
    pdl_entry();
    T cf[KC];
#pragma unroll
    for (int i = 0; i < KC; ++i) cf[i] = i < cnt ? (T)(sign * coef[i]) : T(0);
    const int64_t nv = n / VN;
    for (int64_t e = blockIdx.x * (int64_t)WT + threadIdx.x; e < nv; e += (int64_t)gridDim.x * WT) {
        VT y;
        if (yin) {
            y = reinterpret_cast<const VT*>(yin)[e];
        } else {
#pragma unroll
            for (int c = 0; c < VN; ++c) wset<T>(y, c, T(0));
        }
#pragma unroll
        for (int i = 0; i < KC; ++i) {
            if (i < cnt) {
                const VT vi = reinterpret_cast<const VT*>(V + (int64_t)i * ld)[e];
#pragma unroll
                for (int c = 0; c < VN; ++c) wset<T>(y, c, fma(cf[i], wv<T>(vi, c), wv<T>(y, c)));
            }
        }
        reinterpret_cast<VT*>(yout)[e] = y;
    }
    for (int64_t e = nv * VN + blockIdx.x * (int64_t)WT + threadIdx.x; e < n; e += (int64_t)gridDim.x * WT) {
        T y = yin ? yin[e] : T(0);
#pragma unroll
        for (int i = 0; i < KC; ++i)
            if (i < cnt) y = fma(cf[i], V[(int64_t)i * ld + e], y);
        yout[e] = y;
    }
}

// v = w / sqrt(nrm2[0]), or 0 when the norm is zero (a vanished Arnoldi vector); the scale is
// formed once in FP64 and applied in T
template <typename T>
__global__ void __launch_bounds__(WT) k_wscale(const T* __restrict__ w, const double* __restrict__ nrm2,
                                               T* __restrict__ v, int64_t n) {
    using VT = typename WVec<T>::type;
    constexpr int VN = WVec<T>::n;
    pdl_entry();
    const T s = (T)(nrm2[0] > 0.0 ? 1.0 / sqrt(nrm2[0]) : 0.0);
    const int64_t nv = n / VN;
    for (int64_t e = blockIdx.x * (int64_t)WT + threadIdx.x; e < nv; e += (int64_t)gridDim.x * WT) {
        VT y = reinterpret_cast<const VT*>(w)[e];
#pragma unroll
        for (int c = 0; c < VN; ++c) wset<T>(y, c, wv<T>(y, c) * s);
        reinterpret_cast<VT*>(v)[e] = y;
    }
    for (int64_t e = nv * VN + blockIdx.x * (int64_t)WT + threadIdx.x; e < n; e += (int64_t)gridDim.x * WT)
        v[e] = w[e] * s;
}

// y = argmin || beta e1 - H y || for the (m + 1) x m Hessenberg matrix of the step (Givens
// rotations, back substitution).  H(i, j) = hA[j][i] + hB[j][i] for i <= j (the two Gram-Schmidt
// passes), H(j + 1, j) = sqrt(nr[j]); m stops at the first vanished subdiagonal entry.  y[m..k) = 0.
// One thread.  The loops run to a compile-time bound KM >= k, predicated on k and m, so that H stays in
// registers and every entry is loaded at once.
template <int KM>
__device__ void wlsq_solve_t(const double* __restrict__ hA, const double* __restrict__ hB,
                             const double* __restrict__ nr, const double* __restrict__ beta2, int k,
                             double* __restrict__ y) {
    double H[KM + 1][KM];
    double g[KM + 1], yv[KM];
#pragma unroll
    for (int j = 0; j < KM; ++j) {
        yv[j] = 0.0;
#pragma unroll
        for (int i = 0; i <= KM; ++i) H[i][j] = 0.0;
        if (j < k) {
#pragma unroll
            for (int i = 0; i <= j; ++i) H[i][j] = hA[j * (WRAP_MAXK + 1) + i] + hB[j * (WRAP_MAXK + 1) + i];
            H[j + 1][j] = sqrt(nr[j]);
        }
    }
    const double beta = sqrt(beta2[0]);
    int m = k;
#pragma unroll
    for (int j = KM - 1; j >= 0; --j)
        if (j < k && !(H[j + 1][j] > 0.0)) m = j + 1;
    if (beta > 0.0) {
#pragma unroll
        for (int i = 0; i <= KM; ++i) g[i] = i == 0 ? beta : 0.0;
#pragma unroll
        for (int j = 0; j < KM; ++j) {   // rotate H(j, j), H(j + 1, j) to (r, 0)
            if (j < m) {
                const double a = H[j][j], b = H[j + 1][j];
                const double d = hypot(a, b);
                const double cs = d > 0.0 ? a / d : 1.0, sn = d > 0.0 ? b / d : 0.0;
#pragma unroll
                for (int q = j; q < KM; ++q) {
                    if (q < m) {
                        const double u = H[j][q], v = H[j + 1][q];
                        H[j][q] = cs * u + sn * v;
                        H[j + 1][q] = -sn * u + cs * v;
                    }
                }
                const double gu = g[j], gv = g[j + 1];
                g[j] = cs * gu + sn * gv;
                g[j + 1] = -sn * gu + cs * gv;
            }
        }
#pragma unroll
        for (int i = KM - 1; i >= 0; --i) {
            if (i < m) {
                double acc = g[i];
#pragma unroll
                for (int q = i + 1; q < KM; ++q)
                    if (q < m) acc -= H[i][q] * yv[q];
                yv[i] = H[i][i] != 0.0 ? acc / H[i][i] : 0.0;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < KM; ++j)
        if (j < k) y[j] = yv[j];
}
__device__ void wlsq_solve(const double* __restrict__ hA, const double* __restrict__ hB,
                           const double* __restrict__ nr, const double* __restrict__ beta2, int k,
                           double* __restrict__ y) {
    if (k <= 2)
        wlsq_solve_t<2>(hA, hB, nr, beta2, k, y);
    else if (k <= 4)
        wlsq_solve_t<4>(hA, hB, nr, beta2, k, y);
    else
        wlsq_solve_t<WRAP_MAXK>(hA, hB, nr, beta2, k, y);
}

// The stage's last norm, out = sum of the nblk partials (as k_wreduce with one product), then the
// stage's least-squares solve into y by the thread that wrote it
__global__ void __launch_bounds__(WT) k_wreduce_lsq(const double* __restrict__ partials, int nblk, double* out,
                                                    const double* __restrict__ hA, const double* __restrict__ hB,
                                                    const double* nrAll, const double* __restrict__ beta2, int k,
                                                    double* __restrict__ y) {
    pdl_entry();
    __shared__ double ws[WW];
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += WT) s += partials[b];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) ws[wid] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < WW; ++q) t += ws[q];
        out[0] = t;
        wlsq_solve(hA, hB, nrAll, beta2, k, y);
    }
}

// Levels small enough for one block (n <= WRAP_ONE_MAX): each reduction finishes in the block that
// forms it, so no separate reduce kernel runs.  k_wnorm_one: beta2 = |r0|^2 and V0 = r0 / |r0|.
template <typename T>
__global__ void __launch_bounds__(WT) k_wnorm_one(const T* __restrict__ r0, int64_t n, double* __restrict__ beta2,
                                                  T* __restrict__ V0) {
    using VT = typename WVec<T>::type;
    constexpr int VN = WVec<T>::n;
    pdl_entry();
    __shared__ T scale;
    double acc[1] = {0.0};
    const int64_t nv = n / VN;
    for (int64_t e = threadIdx.x; e < nv; e += WT) {
        const VT y = reinterpret_cast<const VT*>(r0)[e];
        T s = T(0);
#pragma unroll
        for (int c = 0; c < VN; ++c) s = fma(wv<T>(y, c), wv<T>(y, c), s);
        acc[0] += (double)s;
    }
    for (int64_t e = nv * VN + threadIdx.x; e < n; e += WT) acc[0] += (double)r0[e] * (double)r0[e];
    block_partials<1>(acc, 1, beta2);
    __syncthreads();
    if (threadIdx.x == 0) scale = (T)(beta2[0] > 0.0 ? 1.0 / sqrt(beta2[0]) : 0.0);
    __syncthreads();
    const T sc = scale;
    for (int64_t e = threadIdx.x; e < nv; e += WT) {
        VT y = reinterpret_cast<const VT*>(r0)[e];
#pragma unroll
        for (int c = 0; c < VN; ++c) wset<T>(y, c, wv<T>(y, c) * sc);
        reinterpret_cast<VT*>(V0)[e] = y;
    }
    for (int64_t e = nv * VN + threadIdx.x; e < n; e += WT) V0[e] = r0[e] * sc;
}

// One block: w -= sum_{i < cnt} coef[i] V_i and nr = |w|^2 (the second Gram-Schmidt pass and the
// norm), then Vnext = w / sqrt(nr) (Vnext != nullptr) and, on the stage's last step (lsq_k > 0), the
// least-squares solve of the stage into y.
template <typename T, int KC>
__global__ void __launch_bounds__(WT) k_wgs2_one(const T* __restrict__ V, int64_t ld, int cnt,
                                                 const double* __restrict__ coef, T* w, int64_t n,
                                                 double* __restrict__ nr, T* __restrict__ Vnext, int lsq_k,
                                                 const double* __restrict__ hA, const double* __restrict__ hB,
                                                 const double* __restrict__ nrAll, const double* __restrict__ beta2,
                                                 double* __restrict__ y) {
    using VT = typename WVec<T>::type;
    constexpr int VN = WVec<T>::n;
    pdl_entry();
    __shared__ T scale;
    T cf[KC];
#pragma unroll
    for (int i = 0; i < KC; ++i) cf[i] = i < cnt ? (T)coef[i] : T(0);
    double acc[1] = {0.0};
    const int64_t nv = n / VN;
    for (int64_t e = threadIdx.x; e < nv; e += WT) {
        VT yv = reinterpret_cast<const VT*>(w)[e];
#pragma unroll
        for (int i = 0; i < KC; ++i) {
            if (i < cnt) {
                const VT vi = reinterpret_cast<const VT*>(V + (int64_t)i * ld)[e];
#pragma unroll
                for (int c = 0; c < VN; ++c) wset<T>(yv, c, fma(-cf[i], wv<T>(vi, c), wv<T>(yv, c)));
            }
        }
        reinterpret_cast<VT*>(w)[e] = yv;
        T s = T(0);
#pragma unroll
        for (int c = 0; c < VN; ++c) s = fma(wv<T>(yv, c), wv<T>(yv, c), s);
        acc[0] += (double)s;
    }
    for (int64_t e = nv * VN + threadIdx.x; e < n; e += WT) {
        T yv = w[e];
#pragma unroll
        for (int i = 0; i < KC; ++i)
            if (i < cnt) yv = fma(-cf[i], V[(int64_t)i * ld + e], yv);
        w[e] = yv;
        acc[0] += (double)yv * (double)yv;
    }
    block_partials<1>(acc, 1, nr);
    __syncthreads();
    if (threadIdx.x == 0) {
        scale = (T)(nr[0] > 0.0 ? 1.0 / sqrt(nr[0]) : 0.0);
        if (lsq_k > 0) wlsq_solve(hA, hB, nrAll, beta2, lsq_k, y);
    }
    __syncthreads();
    if (Vnext) {
        const T sc = scale;
        for (int64_t e = threadIdx.x; e < nv; e += WT) {
            VT yv = reinterpret_cast<const VT*>(w)[e];
#pragma unroll
            for (int c = 0; c < VN; ++c) wset<T>(yv, c, wv<T>(yv, c) * sc);
            reinterpret_cast<VT*>(Vnext)[e] = yv;
        }
        for (int64_t e = nv * VN + threadIdx.x; e < n; e += WT) Vnext[e] = w[e] * sc;
    }
}

}  // namespace

// blocks of the inner-product and update kernels for n values: one 16-byte vector per thread and
// pass, at most WRAP_BLK blocks (8 per SM)
template <typename T>
int wrap_blocks(int64_t n) {
    const int64_t per = (int64_t)WT * WVec<T>::n;
    const int64_t b = (n + per - 1) / per;
    return (int)(b < 1 ? 1 : (b > WRAP_BLK ? WRAP_BLK : b));
}

// the kernels hold their cnt coefficients and sums in registers, sized by a compile-time bound
#define SIB_WRAP_KC(cnt, CALL) \
    do {                       \
        if ((cnt) <= 2) {      \
            constexpr int KC = 2; \
            CALL;              \
        } else if ((cnt) <= 4) { \
            constexpr int KC = 4; \
            CALL;              \
        } else {               \
            constexpr int KC = WRAP_MAXK + 1; \
            CALL;              \
        }                      \
    } while (0)

template <typename T>
int launch_wdots(const T* V, int64_t ld, int cnt, const T* w, int64_t n, double* partials, cudaStream_t s) {
    const int nb = n <= WRAP_ONE_MAX ? 1 : wrap_blocks<T>(n);
    SIB_WRAP_KC(cnt, launch_pdl(k_wdots<T, KC>, nb, WT, 0, s, V, ld, cnt, w, n, partials));
    return nb;
}
template <typename T>
int launch_wgs(const T* V, int64_t ld, int cnt, const double* coef, const T* win, T* wout, int64_t n, int mode,
               double* partials, cudaStream_t s) {
    const int nb = n <= WRAP_ONE_MAX ? 1 : wrap_blocks<T>(n);
    if (mode == 1)
        SIB_WRAP_KC(cnt, launch_pdl(k_wgs<T, 1, KC>, nb, WT, 0, s, V, ld, cnt, coef, win, wout, n, partials));
    else
        SIB_WRAP_KC(cnt, launch_pdl(k_wgs<T, 2, KC>, nb, WT, 0, s, V, ld, cnt, coef, win, wout, n, partials));
    return nb;
}
template <typename T>
void launch_wnorm_one(const T* r0, int64_t n, double* beta2, T* V0, cudaStream_t s) {
    launch_pdl(k_wnorm_one<T>, 1, WT, 0, s, r0, n, beta2, V0);
}
template <typename T>
void launch_wgs2_one(const T* V, int64_t ld, int cnt, const double* coef, T* w, int64_t n, double* nr, T* Vnext,
                     int lsq_k, const double* hA, const double* hB, const double* nrAll, const double* beta2, double* y,
                     cudaStream_t s) {
    SIB_WRAP_KC(cnt, launch_pdl(k_wgs2_one<T, KC>, 1, WT, 0, s, V, ld, cnt, coef, w, n, nr, Vnext, lsq_k, hA, hB,
                                nrAll, beta2, y));
}
void launch_wreduce(const double* partials, int cnt, int nblk, double* out, cudaStream_t s) {
    launch_pdl(k_wreduce, cnt, WT, 0, s, partials, nblk, out);
}
template <typename T>
void launch_wmaxpy(const T* V, int64_t ld, int cnt, const double* coef, double sign, const T* yin, T* yout, int64_t n,
                   cudaStream_t s) {
    SIB_WRAP_KC(cnt, launch_pdl(k_wmaxpy<T, KC>, wrap_blocks<T>(n), WT, 0, s, V, ld, cnt, coef, sign, yin, yout, n));
}
template <typename T>
void launch_wscale(const T* w, const double* nrm2, T* v, int64_t n, cudaStream_t s) {
    launch_pdl(k_wscale<T>, wrap_blocks<T>(n), WT, 0, s, w, nrm2, v, n);
}
void launch_wreduce_lsq(const double* partials, int nblk, double* out, const double* hA, const double* hB,
                        const double* nrAll, const double* beta2, int k, double* y, cudaStream_t s) {
    launch_pdl(k_wreduce_lsq, 1, WT, 0, s, partials, nblk, out, hA, hB, nrAll, beta2, k, y);
}

#define SIB_WRAP_INST(T)                                                                                    \
    template int launch_wdots<T>(const T*, int64_t, int, const T*, int64_t, double*, cudaStream_t);           \
    template int launch_wgs<T>(const T*, int64_t, int, const double*, const T*, T*, int64_t, int, double*,     \
                               cudaStream_t);                                                               \
    template void launch_wmaxpy<T>(const T*, int64_t, int, const double*, double, const T*, T*, int64_t,      \
                                   cudaStream_t);                                                           \
    template void launch_wscale<T>(const T*, const double*, T*, int64_t, cudaStream_t);                      \
    template void launch_wnorm_one<T>(const T*, int64_t, double*, T*, cudaStream_t);                         \
    template void launch_wgs2_one<T>(const T*, int64_t, int, const double*, T*, int64_t, double*, T*, int,   \
                                     const double*, const double*, const double*, const double*, double*,     \
                                     cudaStream_t);
SIB_WRAP_INST(float)
SIB_WRAP_INST(double)

}  // namespace sib
