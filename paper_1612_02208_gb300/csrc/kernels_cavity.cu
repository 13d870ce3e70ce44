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

// Restriction for the cavity (Sec. 3.2 with walls): the periodic R_u = P_u^T / 4 and the pressure
// average, applied to a fine residual that holds 0 on its wall faces, with the coarse wall faces
// written as 0 (they are not unknowns).  The fine stencil of a coarse unknown never reaches a fine
// wall face or wraps across a wall.
template <typename T>
__global__ void k_cavity_restrict(int Nc, const T* __restrict__ rf, T* __restrict__ bc) {
    pdl_entry();
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    if (I >= Nc || J >= Nc) return;
    const int Nf = 2 * Nc, nf = Nf * Nf, nc = Nc * Nc, mf = Nf - 1;
    const T* ru = rf;
    const T* rv = rf + nf;
    const T* rp = rf + 2 * nf;
    const int i = 2 * I, j = 2 * J, ip = i + 1, jp = j + 1, im = (i - 1) & mf, jm = (j - 1) & mf;
    const T su = (ru[j * Nf + i] + ru[jp * Nf + i]) +
                 T(0.5) * ((ru[j * Nf + ip] + ru[jp * Nf + ip]) + (ru[j * Nf + im] + ru[jp * Nf + im]));
    const T sv = (rv[j * Nf + i] + rv[j * Nf + ip]) +
                 T(0.5) * ((rv[jp * Nf + i] + rv[jp * Nf + ip]) + (rv[jm * Nf + i] + rv[jm * Nf + ip]));
    const T sp = (rp[j * Nf + i] + rp[j * Nf + ip]) + (rp[jp * Nf + i] + rp[jp * Nf + ip]);
    const int c = J * Nc + I;
    bc[c] = I > 0 ? T(0.25) * su : T(0);
    bc[nc + c] = J > 0 ? T(0.25) * sv : T(0);
    bc[2 * nc + c] = T(0.25) * sp;
}

// xf += P ec for the cavity, one thread per fine cell: RT0 velocity exactly as on the periodic grid
// (the coarse wall faces hold 0, so fine wall faces receive 0 and the half-way faces next to a wall
// average with 0), bilinear pressure with a coarse neighbour outside the domain replaced by the cell
// itself (reflection across the wall).
template <typename T>
__global__ void k_cavity_prolong_add(int Nc, const T* __restrict__ ec, T* __restrict__ xf) {
    pdl_entry();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int Nf = 2 * Nc;
    if (i >= Nf || j >= Nf) return;
    const int nf = Nf * Nf, nc = Nc * Nc, mc = Nc - 1;
    const T* eu = ec;
    const T* ev = ec + nc;
    const T* ep = ec + 2 * nc;
    const int I = i >> 1, J = j >> 1;
    const T pu = (i & 1) ? T(0.5) * (eu[J * Nc + I] + eu[J * Nc + ((I + 1) & mc)]) : eu[J * Nc + I];
    const T pv = (j & 1) ? T(0.5) * (ev[J * Nc + I] + ev[((J + 1) & mc) * Nc + I]) : ev[J * Nc + I];
    int I2 = I + ((i & 1) ? 1 : -1), J2 = J + ((j & 1) ? 1 : -1);
    if (I2 < 0 || I2 > mc) I2 = I;
    if (J2 < 0 || J2 > mc) J2 = J;
    const T pp = T(9.0 / 16.0) * ep[J * Nc + I] + T(3.0 / 16.0) * (ep[J * Nc + I2] + ep[J2 * Nc + I]) +
                 T(1.0 / 16.0) * ep[J2 * Nc + I2];
    const int c = j * Nf + i;
    xf[c] += pu;
    xf[nf + c] += pv;
    xf[2 * nf + c] += pp;
}

// The cavity's coarsest operator bordered for its gauge, Aug = [L0 + Z Z^T | I] (3 n0 x 6 n0, row-major),
// with Z the normalised constant pressure (the operator's kernel).  A wall face's row and column are
// those of the identity: the face is not an unknown, and the right-hand side and the solution hold 0
// there.  Unknown rows follow cavity_rows: the tangential ghost -q adds c to the diagonal of a face next
// to a tangential wall, a wall neighbour along the component's own direction contributes nothing, and
// the IB block B (2 n0 x n0 per component, from the level-0 windows) enters as -dt B.
__global__ void k_cavity_assemble_L0(int N, double rho, double mu, double dt, const double* __restrict__ B,
                                     double* __restrict__ Aug) {
    pdl_entry();
    const int n0 = N * N, n = 3 * n0;
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= (int64_t)n * 2 * n) return;
    const int r = (int)(q / (2 * n)), col = (int)(q % (2 * n));
    if (col >= n) {
        Aug[q] = (col - n == r) ? 1.0 : 0.0;
        return;
    }
    const int br = r / n0, f = r % n0, i = f % N, j = f / N;
    const int bc = col / n0, g = col % n0, gi = g % N, gj = g / N;
    const bool wallR = (br == 0 && i == 0) || (br == 1 && j == 0);
    const bool wallC = (bc == 0 && gi == 0) || (bc == 1 && gj == 0);
    if (wallR || wallC) {
        Aug[q] = (r == col) ? 1.0 : 0.0;
        return;
    }
    const double h = 1.0 / N, ih = (double)N;
    const double a0 = rho / dt + 4.0 * mu / (h * h), cc = mu / (h * h);
    double v = 0.0;
    if (br < 2) {
        if (bc == br) {
            // normal direction of the component: x for u, y for v; tangential: the other one
            const int a = br == 0 ? i : j, t = br == 0 ? j : i;   // row face along (normal, tangential)
            const int ga = br == 0 ? gi : gj, gt = br == 0 ? gj : gi;
            if (g == f) v += a0 + cc * (double)((t == 0) + (t == N - 1));
            if (gt == t && (ga == a + 1 || ga == a - 1)) v -= cc;   // in-domain normal neighbours only
            if (ga == a && (gt == t + 1 || gt == t - 1)) v -= cc;   // tangential neighbours inside
            v -= dt * B[(int64_t)br * n0 * n0 + (int64_t)f * n0 + g];
        } else if (bc == 2) {   // G p: (p_ij - p_{i-1,j})/h on u faces, (p_ij - p_{i,j-1})/h on v faces
            if (g == f) v += ih;
            if (g == (br == 0 ? j * N + i - 1 : (j - 1) * N + i)) v -= ih;
        }
    } else if (bc < 2) {        // -D u with the wall faces as zeros
        if (bc == 0) {
            if (g == f) v += ih;
            if (i + 1 < N && g == j * N + i + 1) v -= ih;
        } else {
            if (g == f) v += ih;
            if (j + 1 < N && g == (j + 1) * N + i) v -= ih;
        }
    } else {
        v = 1.0 / (double)n0;   // Z Z^T on the pressure block
    }
    Aug[q] = v;
}

// Cavity windows of one level: the entries in a wall face's row or column are set to 0.  Applied after
// each level's Galerkin product (and to the finest windows), this gives the cavity's R_u B P_u with
// P_u restricted to the unknowns.  Columns are taken modulo N, as the windows store them: on an 8 x 8
// level the offsets +4 and -4 name the same face.  No entry couples two unknowns through a wall:
// the finest windows join faces within one marker's support, which stays inside the domain, and
// the product for an unknown row only reaches fine faces inside the domain, so every coupling it
// forms runs inside the domain or ends on a wall face, which this mask removes.
__global__ void k_cavity_mask_windows(double* __restrict__ win, const int* __restrict__ tiles, int N, int tx, int ty,
                                      int ntx) {
    const int slot = blockIdx.x, comp = blockIdx.y;
    const int per = tx * ty, q = threadIdx.x;
    if (q >= per) return;
    const int t = tiles[slot];
    const int i = (t % ntx) * tx + q % tx, j = (t / ntx) * ty + q / tx;
    double* w = win + ((size_t)(slot * 2 + comp) * WIN_SIZE) * per + q;
    const int m = N - 1;
    const bool wallRow = comp == 0 ? i == 0 : j == 0;
    for (int kw = 0; kw < WIN_SIZE; ++kw) {
        const int ox = kw % WD - WR, oy = kw / WD - WR;
        const bool wallCol = comp == 0 ? ((i + ox) & m) == 0 : ((j + oy) & m) == 0;
        if (wallRow || wallCol) w[(size_t)kw * per] = 0.0;
    }
}

// x <- 0 on the wall faces u(0, j), v(i, 0)
template <typename T>
__global__ void k_cavity_zero_walls(T* __restrict__ x, int N) {
    pdl_entry();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    x[k * N] = T(0);
    x[N * N + k] = T(0);
}

// rhs(u(i, N-1)) += 2 mu u_lid(i h) / h^2 for i = 1 .. N-1: the known part of the ghost value across
// the lid, u_lid(x) = (1 - cos 2 pi x) / 2 (the regularised lid of Sec. 5)
__global__ void k_cavity_add_lid(double* __restrict__ rhs, int N, double mu) {
    pdl_entry();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 1 || i >= N) return;
    const double h = 1.0 / N, x = i * h;
    const double ulid = 0.5 * (1.0 - cospi(2.0 * x));
    rhs[(N - 1) * N + i] += 2.0 * mu * ulid / (h * h);
}

}  // namespace

void launch_cavity_add_lid(double* rhs, int N, double mu, cudaStream_t s) {
    launch_pdl(k_cavity_add_lid, dim3((N + 127) / 128), dim3(128), 0, s, rhs, N, mu);
}

template <typename T>
void launch_cavity_residual(const GridK<T>& g, const T* x, const T* b, T* r, cudaStream_t s) {
    launch_pdl(k_cavity_residual<T>, dim3(g.N / g.tx, g.N / g.ty), dim3(g.tx, g.ty), 0, s, g, x, b, r);
}
template <typename T>
void launch_cavity_zero_walls(T* x, int N, cudaStream_t s) {
    launch_pdl(k_cavity_zero_walls<T>, dim3((N + 127) / 128), dim3(128), 0, s, x, N);
}

template <typename T>
void launch_cavity_restrict(int Nc, const T* rf, T* bc, cudaStream_t s) {
    dim3 blk(Nc < 32 ? Nc : 32, Nc < 8 ? Nc : 8);
    dim3 grd((Nc + blk.x - 1) / blk.x, (Nc + blk.y - 1) / blk.y);
    launch_pdl(k_cavity_restrict<T>, grd, blk, 0, s, Nc, rf, bc);
}
template <typename T>
void launch_cavity_prolong_add(int Nc, const T* ec, T* xf, cudaStream_t s) {
    const int Nf = 2 * Nc;
    dim3 blk(Nf < 32 ? Nf : 32, Nf < 8 ? Nf : 8);
    dim3 grd((Nf + blk.x - 1) / blk.x, (Nf + blk.y - 1) / blk.y);
    launch_pdl(k_cavity_prolong_add<T>, grd, blk, 0, s, Nc, ec, xf);
}
void launch_cavity_assemble_L0(int N0, double rho, double mu, double dt, const double* B, double* Aug,
                               cudaStream_t s) {
    const int64_t tot = (int64_t)3 * N0 * N0 * 6 * N0 * N0;
    launch_pdl(k_cavity_assemble_L0, (int)((tot + 255) / 256), 256, 0, s, N0, rho, mu, dt, B, Aug);
}
void launch_cavity_mask_windows(double* win, const int* tiles, int nTiles, int N, int tx, int ty, int ntx,
                                cudaStream_t s) {
    if (nTiles == 0) return;
    k_cavity_mask_windows<<<dim3(nTiles, 2), tx * ty, 0, s>>>(win, tiles, N, tx, ty, ntx);
}

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
template void launch_cavity_residual<float>(const GridK<float>&, const float*, const float*, float*, cudaStream_t);
template void launch_cavity_residual<double>(const GridK<double>&, const double*, const double*, double*,
                                             cudaStream_t);
template void launch_cavity_zero_walls<float>(float*, int, cudaStream_t);
template void launch_cavity_zero_walls<double>(double*, int, cudaStream_t);
template void launch_cavity_restrict<float>(int, const float*, float*, cudaStream_t);
template void launch_cavity_restrict<double>(int, const double*, double*, cudaStream_t);
template void launch_cavity_prolong_add<float>(int, const float*, float*, cudaStream_t);
template void launch_cavity_prolong_add<double>(int, const double*, double*, cudaStream_t);

}  // namespace sib
