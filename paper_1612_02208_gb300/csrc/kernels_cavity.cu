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

template <typename T>
__global__ void k_cavity_apply(GridK<T> g, const T* __restrict__ x, T* __restrict__ y) {
    pdl_entry();
    const int N = g.N, n = N * N;
    const int i = blockIdx.x * g.tx + threadIdx.x, j = blockIdx.y * g.ty + threadIdx.y;
    const int c = j * N + i;
    const T* u = x;
    const T* v = x + n;
    const T* p = x + 2 * n;
    if (i > 0) {
        const T uc = u[c];
        const T uE = i + 1 < N ? u[c + 1] : T(0);     // the x = 1 wall face
        const T uW = i - 1 >= 1 ? u[c - 1] : T(0);    // the x = 0 wall face
        const T uN = j + 1 < N ? u[c + N] : -uc;      // ghost across the lid
        const T uS = j - 1 >= 0 ? u[c - N] : -uc;     // ghost across the bottom wall
        T a = g.a0 * uc - g.c * ((uE + uW) + (uN + uS)) + (p[c] - p[c - 1]) * g.inv_h;
        a -= g.dt * ibf(g, x, 0, i, j);
        y[c] = a;
    } else {
        y[c] = T(0);
    }
    if (j > 0) {
        const T vc = v[c];
        const T vE = i + 1 < N ? v[c + 1] : -vc;
        const T vW = i - 1 >= 0 ? v[c - 1] : -vc;
        const T vN = j + 1 < N ? v[c + N] : T(0);
        const T vS = j - 1 >= 1 ? v[c - N] : T(0);
        T a = g.a0 * vc - g.c * ((vE + vW) + (vN + vS)) + (p[c] - p[c - N]) * g.inv_h;
        a -= g.dt * ibf(g, x, 1, i, j);
        y[n + c] = a;
    } else {
        y[n + c] = T(0);
    }
    const T ue = i + 1 < N ? u[c + 1] : T(0), uw = i >= 1 ? u[c] : T(0);
    const T vn = j + 1 < N ? v[c + N] : T(0), vs = j >= 1 ? v[c] : T(0);
    y[2 * n + c] = -(((ue - uw) + (vn - vs)) * g.inv_h);
}

}  // namespace

template <typename T>
void launch_cavity_apply(const GridK<T>& g, const T* x, T* y, cudaStream_t s) {
    launch_pdl(k_cavity_apply<T>, dim3(g.N / g.tx, g.N / g.ty), dim3(g.tx, g.ty), 0, s, g, x, y);
}
template void launch_cavity_apply<float>(const GridK<float>&, const float*, float*, cudaStream_t);
template void launch_cavity_apply<double>(const GridK<double>&, const double*, double*, cudaStream_t);

}  // namespace sib
