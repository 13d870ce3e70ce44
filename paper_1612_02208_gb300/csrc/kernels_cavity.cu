// The Stokes-IB operator of the lid-driven cavity (Sec. 5: no-slip walls; the lid enters only the
// right-hand side) on the periodic layout [u | v | p]: the seam faces u(0, j) (x = 0 = 1) and
// v(i, 0) (y = 0 = 1) are the wall faces, whose normal velocity is 0 and which are not unknowns.
//   - a neighbour along the component's own direction that is a wall face contributes 0;
//   - across a tangential wall the five-point Laplacian takes the ghost value -q (2 q_wall - q with
//     q_wall = 0; the lid's 2 q_wall part belongs to the right-hand side);
//   - G and D use the wall faces as zeros, so D = -G^T;
//   - the IB term is the level's [S K J] of the same field (the structure keeps its Peskin support
//     inside the domain, so it never touches a wall face).
// The wall-face entries of y are written as 0.
#include "grid_cells.cuh"

namespace sib {

namespace {

// (L x) at cell (i, j): the u row (i > 0), the v row (j > 0) and the -D row; the IB term from g.fib
template <typename T>
__device__ __forceinline__ void cavity_rows(const GridK<T>& g, const T* __restrict__ x, int i, int j, T& au, T& av,
                                            T& ap) {
    const int N = g.N, n = N * N, c = j * N + i;
    const T* u = x;
    const T* v = x + n;
    const T* p = x + 2 * n;
    au = av = T(0);
    if (i > 0) {
        const T uc = u[c];
        const T uE = i + 1 < N ? u[c + 1] : T(0);     // the x = 1 wall face
        const T uW = i - 1 >= 1 ? u[c - 1] : T(0);    // the x = 0 wall face
        const T uN = j + 1 < N ? u[c + N] : -uc;      // ghost across the lid
        const T uS = j - 1 >= 0 ? u[c - N] : -uc;     // ghost across the bottom wall
        au = g.a0 * uc - g.c * ((uE + uW) + (uN + uS)) + (p[c] - p[c - 1]) * g.inv_h;
        au -= g.dt * ibf(g, x, 0, i, j);
    }
    if (j > 0) {
        const T vc = v[c];
        const T vE = i + 1 < N ? v[c + 1] : -vc;
        const T vW = i - 1 >= 0 ? v[c - 1] : -vc;
        const T vN = j + 1 < N ? v[c + N] : T(0);
        const T vS = j - 1 >= 1 ? v[c - N] : T(0);
        av = g.a0 * vc - g.c * ((vE + vW) + (vN + vS)) + (p[c] - p[c - N]) * g.inv_h;
        av -= g.dt * ibf(g, x, 1, i, j);
    }
    const T ue = i + 1 < N ? u[c + 1] : T(0), uw = i >= 1 ? u[c] : T(0);
    const T vn = j + 1 < N ? v[c + N] : T(0), vs = j >= 1 ? v[c] : T(0);
    ap = -(((ue - uw) + (vn - vs)) * g.inv_h);
}

template <typename T>
__global__ void k_cavity_apply(GridK<T> g, const T* __restrict__ x, T* __restrict__ y) {
    pdl_entry();
    const int N = g.N, n = N * N;
    const int i = blockIdx.x * g.tx + threadIdx.x, j = blockIdx.y * g.ty + threadIdx.y;
    const int c = j * N + i;
    T au, av, ap;
    cavity_rows(g, x, i, j, au, av, ap);
    y[c] = au;          // 0 on the wall faces (i == 0, j == 0)
    y[n + c] = av;
    y[2 * n + c] = ap;
}

// r = b - L x on the unknowns, 0 on the wall faces
template <typename T>
__global__ void k_cavity_residual(GridK<T> g, const T* __restrict__ x, const T* __restrict__ b, T* __restrict__ r) {
    pdl_entry();
    const int N = g.N, n = N * N;
    const int i = blockIdx.x * g.tx + threadIdx.x, j = blockIdx.y * g.ty + threadIdx.y;
    const int c = j * N + i;
    T au, av, ap;
    cavity_rows(g, x, i, j, au, av, ap);
    r[c] = i > 0 ? b[c] - au : T(0);
    r[n + c] = j > 0 ? b[n + c] - av : T(0);
    r[2 * n + c] = b[2 * n + c] - ap;
}

// Vanka patch solve of cell (i, j) (Alg. 2, one-cell subdomain) with the wall rules: the 2 x 2
// velocity blocks carry the tangential ghost (+c on the diagonal of a face next to a tangential
// wall) and the IB entries; a wall face acts as an infinitely stiff block entry, so its inverse-block
// factors are 0, which zeroes its correction and drops it from the pressure Schur complement.
// d = (d0, d1, d2, d3, dp) per cell, 5 n values.
template <typename T>
__global__ void k_cavity_patch(GridK<T> g, const T* __restrict__ r, T* __restrict__ d) {
    pdl_entry();
    const int N = g.N, n = N * N, m = N - 1;
    const int i = blockIdx.x * g.tx + threadIdx.x, j = blockIdx.y * g.ty + threadIdx.y;
    const int c = j * N + i, ce = j * N + ((i + 1) & m), cn = ((j + 1) & m) * N + i;
    const bool wuL = i == 0, wuR = i == N - 1, wvB = j == 0, wvT = j == N - 1;
    const T tu = g.c * T(int(j == 0) + int(j == N - 1)), tv = g.c * T(int(i == 0) + int(i == N - 1));
    const T au00 = g.a0 + tu - g.dt * g.ibd[c], au11 = g.a0 + tu - g.dt * g.ibd[ce], au01 = -g.c - g.dt * g.ibd[n + c];
    const T av00 = g.a0 + tv - g.dt * g.ibd[2 * n + c], av11 = g.a0 + tv - g.dt * g.ibd[2 * n + cn],
            av01 = -g.c - g.dt * g.ibd[3 * n + c];
    auto block = [](T a00, T a11, T a01, bool wl, bool wr, T& A00, T& A01, T& A11) {
        if (wl && wr) {
            A00 = A01 = A11 = T(0);
        } else if (wl) {
            A00 = A01 = T(0);
            A11 = T(1) / a11;
        } else if (wr) {
            A00 = T(1) / a00;
            A01 = A11 = T(0);
        } else {
            const T idet = T(1) / (a00 * a11 - a01 * a01);
            A00 = a11 * idet;
            A01 = -a01 * idet;
            A11 = a00 * idet;
        }
    };
    T A00u, A01u, A11u, A00v, A01v, A11v;
    block(au00, au11, au01, wuL, wuR, A00u, A01u, A11u);
    block(av00, av11, av01, wvB, wvT, A00v, A01v, A11v);
    const T r0 = wuL ? T(0) : r[c], r1 = wuR ? T(0) : r[c + 1];
    const T r2 = wvB ? T(0) : r[n + c], r3 = wvT ? T(0) : r[n + c + N];
    const T r4 = r[2 * n + c];
    const T ih = g.inv_h;
    const T tu0 = A00u * r0 + A01u * r1, tu1 = A01u * r0 + A11u * r1;
    const T tv0 = A00v * r2 + A01v * r3, tv1 = A01v * r2 + A11v * r3;
    const T su0 = ih * (A00u - A01u), su1 = ih * (A01u - A11u);
    const T sv0 = ih * (A00v - A01v), sv1 = ih * (A01v - A11v);
    const T S = ih * ((su0 - su1) + (sv0 - sv1));
    const T dp = (ih * ((tu0 - tu1) + (tv0 - tv1)) - r4) / S;
    d[c] = tu0 - su0 * dp;
    d[n + c] = tu1 - su1 * dp;
    d[2 * n + c] = tv0 - sv0 * dp;
    d[3 * n + c] = tv1 - sv1 * dp;
    d[4 * n + c] = dp;
}

// xo = x + omega (1/2 (two cell corrections) on interior faces, the cell's on p); 0 on wall faces
template <typename T>
__global__ void k_cavity_update(GridK<T> g, T omega, const T* __restrict__ d, const T* __restrict__ x,
                                T* __restrict__ xo) {
    pdl_entry();
    const int N = g.N, n = N * N;
    const int i = blockIdx.x * g.tx + threadIdx.x, j = blockIdx.y * g.ty + threadIdx.y;
    const int c = j * N + i;
    const T hw = T(0.5) * omega;
    xo[c] = i >= 1 ? x[c] + hw * (d[c] + d[n + c - 1]) : T(0);
    xo[n + c] = j >= 1 ? x[n + c] + hw * (d[2 * n + c] + d[3 * n + c - N]) : T(0);
    xo[2 * n + c] = x[2 * n + c] + omega * d[4 * n + c];
}

}  // namespace

template <typename T>
void launch_cavity_apply(const GridK<T>& g, const T* x, T* y, cudaStream_t s) {
    launch_pdl(k_cavity_apply<T>, dim3(g.N / g.tx, g.N / g.ty), dim3(g.tx, g.ty), 0, s, g, x, y);
}
template <typename T>
void launch_cavity_vanka(const GridK<T>& g, const T* x, const T* b, T* r, T* d, T* xo, T omega, cudaStream_t s) {
    const dim3 grd(g.N / g.tx, g.N / g.ty), blk(g.tx, g.ty);
    launch_pdl(k_cavity_residual<T>, grd, blk, 0, s, g, x, b, r);
    launch_pdl(k_cavity_patch<T>, grd, blk, 0, s, g, (const T*)r, d);
    launch_pdl(k_cavity_update<T>, grd, blk, 0, s, g, omega, (const T*)d, x, xo);
}
template void launch_cavity_apply<float>(const GridK<float>&, const float*, float*, cudaStream_t);
template void launch_cavity_apply<double>(const GridK<double>&, const double*, double*, cudaStream_t);
template void launch_cavity_vanka<float>(const GridK<float>&, const float*, const float*, float*, float*, float*, float,
                                         cudaStream_t);
template void launch_cavity_vanka<double>(const GridK<double>&, const double*, const double*, double*, double*,
                                          double*, double, cudaStream_t);

}  // namespace sib
