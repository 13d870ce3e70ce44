// Point-wise pieces of the MAC-grid operators, shared by the per-level kernels (one thread per
// cell) and the single-block kernel of the small levels (shared-memory copies of the same arrays:
// every function here reads and writes through the pointers it is given, GridK's included).
//
// Layout: a level vector is [u | v | p], each N*N row-major [j][i]; u[j][i] on the x-face
// (i-1/2, j), v[j][i] on the y-face (i, j-1/2), p[j][i] at the cell centre (Appendix,
// "Eulerian discretization").  N is a power of two, so periodic wrap is a mask.
#pragma once
#include "sib_internal.h"

namespace sib {

// IB force ([S K J]^l fld) at face (i, j) of component comp, precomputed into g.fib by the IB
// pass for the same field; zero outside IB-active tiles.
template <typename T>
__device__ __forceinline__ T ibf(const GridK<T>& g, const T* __restrict__ fld, int comp, int i, int j) {
    (void)fld;
    if (g.tile == nullptr) return T(0);
    const int tile = (j >> g.lgty) * g.ntx + (i >> g.lgtx);
    if (!g.tile[tile]) return T(0);
    return g.fib[(size_t)comp * g.N * g.N + j * g.N + i];
}

// diagonal of A_IB on a face: a0 - dt B(f,f) (B(f,f) is zero outside IB-active tiles)
template <typename T>
__device__ __forceinline__ T diag_face(const GridK<T>& g, int comp, int i, int j) {
    if (g.tile == nullptr) return g.a0;
    const int tile = (j >> g.lgty) * g.ntx + (i >> g.lgtx);
    if (!g.tile[tile]) return g.a0;
    return g.a0 - g.dt * g.ibd[(size_t)2 * comp * g.N * g.N + j * g.N + i];
}

// ------------------------------------------------------------------------------------------
// Residual entries r = b - L x at one face / cell (Eq. matrix-h-impib); the IB term through g.fib.
template <typename T>
__device__ __forceinline__ T res_u(const GridK<T>& g, const T* __restrict__ x, const T* __restrict__ b, int i, int j) {
    const int N = g.N, m = N - 1;
    const T* u = x;
    const T* p = x + 2 * N * N;
    i &= m;
    j &= m;
    const int c = j * N + i;
    T Au = g.a0 * u[c] - g.c * ((u[j * N + ((i + 1) & m)] + u[j * N + ((i - 1) & m)]) +
                                (u[((j + 1) & m) * N + i] + u[((j - 1) & m) * N + i])) +
           (p[c] - p[j * N + ((i - 1) & m)]) * g.inv_h;
    Au -= g.dt * ibf(g, x, 0, i, j);
    return b[c] - Au;
}
template <typename T>
__device__ __forceinline__ T res_v(const GridK<T>& g, const T* __restrict__ x, const T* __restrict__ b, int i, int j) {
    const int N = g.N, n = N * N, m = N - 1;
    const T* v = x + n;
    const T* p = x + 2 * n;
    i &= m;
    j &= m;
    const int c = j * N + i;
    T Av = g.a0 * v[c] - g.c * ((v[j * N + ((i + 1) & m)] + v[j * N + ((i - 1) & m)]) +
                                (v[((j + 1) & m) * N + i] + v[((j - 1) & m) * N + i])) +
           (p[c] - p[((j - 1) & m) * N + i]) * g.inv_h;
    Av -= g.dt * ibf(g, x, 1, i, j);
    return b[n + c] - Av;
}
template <typename T>
__device__ __forceinline__ T res_p(const GridK<T>& g, const T* __restrict__ x, const T* __restrict__ b, int i, int j) {
    const int N = g.N, n = N * N, m = N - 1;
    i &= m;
    j &= m;
    const int c = j * N + i;
    return b[2 * n + c] + ((x[j * N + ((i + 1) & m)] - x[c]) + (x[n + ((j + 1) & m) * N + i] - x[n + c])) * g.inv_h;
}

// The same residual entries at a face of a tile whose IB flag `act` the caller has already read.
template <typename T>
__device__ __forceinline__ T ibf_act(const GridK<T>& g, bool act, int comp, int i, int j) {
    return act ? g.fib[(size_t)comp * g.N * g.N + j * g.N + i] : T(0);
}
template <typename T>
__device__ __forceinline__ T res_u_act(const GridK<T>& g, bool act, const T* __restrict__ x, const T* __restrict__ b,
                                       int i, int j) {
    const int N = g.N, m = N - 1;
    const T* u = x;
    const T* p = x + 2 * N * N;
    const int c = j * N + i;
    T Au = g.a0 * u[c] - g.c * ((u[j * N + ((i + 1) & m)] + u[j * N + ((i - 1) & m)]) +
                                (u[((j + 1) & m) * N + i] + u[((j - 1) & m) * N + i])) +
           (p[c] - p[j * N + ((i - 1) & m)]) * g.inv_h;
    Au -= g.dt * ibf_act(g, act, 0, i, j);
    return b[c] - Au;
}
template <typename T>
__device__ __forceinline__ T res_v_act(const GridK<T>& g, bool act, const T* __restrict__ x, const T* __restrict__ b,
                                       int i, int j) {
    const int N = g.N, n = N * N, m = N - 1;
    const T* v = x + n;
    const T* p = x + 2 * n;
    const int c = j * N + i;
    T Av = g.a0 * v[c] - g.c * ((v[j * N + ((i + 1) & m)] + v[j * N + ((i - 1) & m)]) +
                                (v[((j + 1) & m) * N + i] + v[((j - 1) & m) * N + i])) +
           (p[c] - p[((j - 1) & m) * N + i]) * g.inv_h;
    Av -= g.dt * ibf_act(g, act, 1, i, j);
    return b[n + c] - Av;
}

// Coarse right-hand side of coarse cell (I, J): R (b - L x) from the sixteen fine residuals that
// R = diag(P_u^T / 4, P_v^T / 4, average) combines (Sec. 3.2, Alg. 1).
template <typename T>
__device__ __forceinline__ void residual_restrict_cell(const GridK<T>& g, const T* __restrict__ x,
                                                       const T* __restrict__ b, T* __restrict__ bc, int I, int J) {
    const int Nc = g.N / 2;
    const int i = 2 * I, j = 2 * J;
    const T su = (res_u(g, x, b, i, j) + res_u(g, x, b, i, j + 1)) +
                 T(0.5) * ((res_u(g, x, b, i + 1, j) + res_u(g, x, b, i + 1, j + 1)) +
                           (res_u(g, x, b, i - 1, j) + res_u(g, x, b, i - 1, j + 1)));
    const T sv = (res_v(g, x, b, i, j) + res_v(g, x, b, i + 1, j)) +
                 T(0.5) * ((res_v(g, x, b, i, j + 1) + res_v(g, x, b, i + 1, j + 1)) +
                           (res_v(g, x, b, i, j - 1) + res_v(g, x, b, i + 1, j - 1)));
    const T sp = (res_p(g, x, b, i, j) + res_p(g, x, b, i + 1, j)) + (res_p(g, x, b, i, j + 1) + res_p(g, x, b, i + 1, j + 1));
    const int nc = Nc * Nc, c = J * Nc + I;
    bc[c] = T(0.25) * su;
    bc[nc + c] = T(0.25) * sv;
    bc[2 * nc + c] = T(0.25) * sp;
}

// Coarse right-hand side of coarse cell (I, J) from a fine residual rf (Sec. 3.2): a coarse x-face
// takes 1/4 of the two coincident fine faces plus 1/8 of the four fine faces half a coarse cell
// away in x (R_u = P_u^T / 4); pressure: the average of the four fine cells.
template <typename T>
__device__ __forceinline__ void restrict_cell(int Nc, const T* __restrict__ rf, T* __restrict__ bc, int I, int J) {
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
    bc[c] = T(0.25) * su;
    bc[nc + c] = T(0.25) * sv;
    bc[2 * nc + c] = T(0.25) * sp;
}

// xf += P ec at fine cell (i, j) (Sec. 3.2): RT0 for velocity (fine faces that coincide with
// coarse faces copy, faces half-way between two coarse faces average them, constant in the
// tangential direction), bilinear cell-centred interpolation for pressure (9/16, 3/16, 3/16, 1/16).
template <typename T>
__device__ __forceinline__ void prolong_add_cell(int Nc, const T* __restrict__ ec, T* __restrict__ xf, int i, int j) {
    const int Nf = 2 * Nc;
    const int nf = Nf * Nf, nc = Nc * Nc, mc = Nc - 1;
    const T* eu = ec;
    const T* ev = ec + nc;
    const T* ep = ec + 2 * nc;
    const int I = i >> 1, J = j >> 1;
    const T pu = (i & 1) ? T(0.5) * (eu[J * Nc + I] + eu[J * Nc + ((I + 1) & mc)]) : eu[J * Nc + I];
    const T pv = (j & 1) ? T(0.5) * (ev[J * Nc + I] + ev[((J + 1) & mc) * Nc + I]) : ev[J * Nc + I];
    const int I2 = (I + ((i & 1) ? 1 : -1)) & mc, J2 = (J + ((j & 1) ? 1 : -1)) & mc;
    const T pp = T(9.0 / 16.0) * ep[J * Nc + I] + T(3.0 / 16.0) * (ep[J * Nc + I2] + ep[J2 * Nc + I]) +
                 T(1.0 / 16.0) * ep[J2 * Nc + I2];
    const int c = j * Nf + i;
    xf[c] += pu;
    xf[nf + c] += pv;
    xf[2 * nf + c] += pp;
}

// ------------------------------------------------------------------------------------------
// Vanka patch solve from the cell's set-up factors (Alg. 2, one-cell subdomain): with
// A_u^{-1} = [[a00u, a01u], [a01u, a11u]] and A_v^{-1} likewise (the inverses of the 2 x 2 velocity
// blocks) and invS = 1 / (g^T A_u^{-1} g + g^T A_v^{-1} g), g = (1/h, -1/h), the patch system
// [[A_u, 0, g], [0, A_v, g], [g^T, g^T, 0]] (d0, d1, d2, d3, dp) = (r0, r1, r2, r3, r4) is solved by
// block elimination on the pressure: t = A^{-1} r, s = A^{-1} g, dp = (g^T t - r4) invS, d = t - s dp.
template <typename T>
__device__ __forceinline__ void patch_solve(const T* f, T ih, T r0, T r1, T r2, T r3, T r4, T& d0, T& d1, T& d2,
                                            T& d3, T& dp) {
    const T a00u = f[0], a01u = f[1], a11u = f[2], a00v = f[3], a01v = f[4], a11v = f[5], invS = f[6];
    const T tu0 = a00u * r0 + a01u * r1, tu1 = a01u * r0 + a11u * r1;
    const T tv0 = a00v * r2 + a01v * r3, tv1 = a01v * r2 + a11v * r3;
    const T su0 = ih * (a00u - a01u), su1 = ih * (a01u - a11u);
    const T sv0 = ih * (a00v - a01v), sv1 = ih * (a01v - a11v);
    dp = (ih * ((tu0 - tu1) + (tv0 - tv1)) - r4) * invS;
    d0 = tu0 - su0 * dp;
    d1 = tu1 - su1 * dp;
    d2 = tv0 - sv0 * dp;
    d3 = tv1 - sv1 * dp;
}

// ------------------------------------------------------------------------------------------
// Schur-complement smoother pieces (Eq. approx-fact-Stokes-IB).
// diag(A_IB) on a face: a0 - dt B(f,f) (B(f,f) read only in IB-active tiles).
template <typename T>
__device__ __forceinline__ T diagA(const GridK<T>& g, bool act, int comp, int c, int n) {
    return act ? g.a0 - g.dt * g.ibd[2 * comp * n + c] : g.a0;
}

// Schur-complement sweep with two Chebyshev iterations in each inner solve, in five point-wise
// stages separated by IB passes (Eq. approx-fact-Stokes-IB):
//   r = b - L x;  y = At^{-1} r_u;  s = r_p + D y;  dp = Mt^{-1} s;  yy = At^{-1} G dp;
//   xo = x + omega (y - yy, dp)
// with At^{-1} q = (1 + c1) d0 + c2 DA^{-1}(q - A_IB d0), d0 = DA^{-1} q / theta_A, and
// Mt^{-1} s = (1 + c1) e0 + c2 DM^{-1}(s - D At^{-1} G e0), e0 = DM^{-1} s / theta_M, where DA is
// diag(A_IB) and DM = diag(D DA^{-1} G).  A stage that needs G of a cell-centred quantity
// recomputes that quantity on the two neighbouring cells instead of synchronising.
template <typename T>
__device__ __forceinline__ T Aib(const GridK<T>& g, const T* __restrict__ d, int comp, int i, int j) {
    const int N = g.N, m = N - 1;
    const T* dc = d + (size_t)comp * N * N;
    const T a = g.a0 * dc[j * N + i] - g.c * ((dc[j * N + ((i + 1) & m)] + dc[j * N + ((i - 1) & m)]) +
                                             (dc[((j + 1) & m) * N + i] + dc[((j - 1) & m) * N + i]));
    return a - g.dt * ibf(g, d, comp, i, j);
}
template <typename T>
__device__ __forceinline__ T divg(const GridK<T>& g, const T* __restrict__ w, int i, int j) {
    const int N = g.N, m = N - 1;
    i &= m;
    j &= m;
    return ((w[j * N + ((i + 1) & m)] - w[j * N + i]) + (w[N * N + ((j + 1) & m) * N + i] - w[N * N + j * N + i])) *
           g.inv_h;
}
template <typename T>
__device__ __forceinline__ T dM_inv(const GridK<T>& g, int i, int j) {
    const int m = g.N - 1;
    i &= m;
    j &= m;
    const T s = T(1) / diag_face(g, 0, i, j) + T(1) / diag_face(g, 0, (i + 1) & m, j) + T(1) / diag_face(g, 1, i, j) +
                T(1) / diag_face(g, 1, i, (j + 1) & m);
    return T(1) / (-s * g.inv_h * g.inv_h);
}

// Set-up values an SC stage needs at cell (i, j): the IB flag of the cell's tile (the IB force of
// its faces is read only there) and the diagonal inverses of DA on its two faces and, with M, of DM
// on the cell and its west and south neighbours.  The per-level kernels load them before waiting
// for the stage's inputs.
template <typename T>
struct ScPre {
    bool act;
    T a0, a1, m, mw, ms;
};
template <typename T, bool M>
__device__ __forceinline__ ScPre<T> sc_pre(const GridK<T>& g, int i, int j) {
    const int N = g.N, n = N * N, mk = N - 1, c = j * N + i;
    ScPre<T> p;
    p.act = g.tile != nullptr && g.tile[(j >> g.lgty) * g.ntx + (i >> g.lgtx)];
    p.a0 = g.dinv[c];
    p.a1 = g.dinv[n + c];
    if (M) {
        p.m = g.dinv[2 * n + c];
        p.mw = g.dinv[2 * n + j * N + ((i - 1) & mk)];
        p.ms = g.dinv[2 * n + ((j - 1) & mk) * N + i];
    } else {
        p.m = p.mw = p.ms = T(0);
    }
    return p;
}
template <typename T>
__device__ __forceinline__ T Aib_act(const GridK<T>& g, bool act, const T* __restrict__ d, int comp, int i, int j) {
    const int N = g.N, m = N - 1;
    const T* dc = d + (size_t)comp * N * N;
    const T a = g.a0 * dc[j * N + i] - g.c * ((dc[j * N + ((i + 1) & m)] + dc[j * N + ((i - 1) & m)]) +
                                             (dc[((j + 1) & m) * N + i] + dc[((j - 1) & m) * N + i]));
    return a - g.dt * ibf_act(g, act, comp, i, j);
}

// r = b - L x (x == nullptr: zero initial guess, r = b);  d = DA^{-1} r_u / theta_A
template <typename T>
__device__ __forceinline__ void sc_start_cell(const GridK<T>& g, const Cheb2<T>& ka, const T* __restrict__ x,
                                              const T* __restrict__ b, T* __restrict__ r, T* __restrict__ d, int i,
                                              int j, const ScPre<T>& p) {
    const int N = g.N, n = N * N;
    const int c = j * N + i;
    const T ru = x ? res_u_act(g, p.act, x, b, i, j) : b[c], rv = x ? res_v_act(g, p.act, x, b, i, j) : b[n + c];
    r[c] = ru;
    r[n + c] = rv;
    r[2 * n + c] = x ? res_p(g, x, b, i, j) : b[2 * n + c];
    d[c] = ka.inv_theta * ru * p.a0;
    d[n + c] = ka.inv_theta * rv * p.a1;
}
// y = (1 + c1) d + c2 DA^{-1} (q - A_IB d)   (g.fib holds [SKJ] d)
template <typename T>
__device__ __forceinline__ void sc_chebA_cell(const GridK<T>& g, const Cheb2<T>& ka, const T* __restrict__ q,
                                              const T* __restrict__ d, T* __restrict__ y, int i, int j,
                                              const ScPre<T>& p) {
    const int N = g.N, n = N * N;
    const int c = j * N + i;
    for (int comp = 0; comp < 2; ++comp) {
        const int f = comp * n + c;
        const T rr = q[f] - Aib_act(g, p.act, d, comp, i, j);
        y[f] = ka.one_c1 * d[f] + ka.c2 * rr * (comp ? p.a1 : p.a0);
    }
}
// s = r_p + D y;  e0 = DM^{-1} s / theta_M;  gq = G e0;  dA = DA^{-1} gq / theta_A
template <typename T>
__device__ __forceinline__ void sc_mstart_cell(const GridK<T>& g, const Cheb2<T>& ka, const Cheb2<T>& km,
                                               const T* __restrict__ rp, const T* __restrict__ y, T* __restrict__ sv,
                                               T* __restrict__ dMo, T* __restrict__ gq, T* __restrict__ dA, int i,
                                               int j, const ScPre<T>& p) {
    const int N = g.N, n = N * N, m = N - 1;
    const int c = j * N + i;
    auto e0 = [&](int ii, int jj, T dm, T* sOut) {
        ii &= m;
        jj &= m;
        const T sval = rp[jj * N + ii] + divg(g, y, ii, jj);
        if (sOut) *sOut = sval;
        return km.inv_theta * sval * dm;
    };
    T sc;
    const T ec = e0(i, j, p.m, &sc), ew = e0(i - 1, j, p.mw, nullptr), es = e0(i, j - 1, p.ms, nullptr);
    sv[c] = sc;
    dMo[c] = ec;
    const T gu = (ec - ew) * g.inv_h, gv = (ec - es) * g.inv_h;
    gq[c] = gu;
    gq[n + c] = gv;
    dA[c] = ka.inv_theta * gu * p.a0;
    dA[n + c] = ka.inv_theta * gv * p.a1;
}
// dp = (1 + c1) e0 + c2 DM^{-1} (s - D ya);  gq = G dp;  dA = DA^{-1} gq / theta_A
template <typename T>
__device__ __forceinline__ void sc_mfinish_cell(const GridK<T>& g, const Cheb2<T>& ka, const Cheb2<T>& km,
                                                const T* __restrict__ sv, const T* __restrict__ dM,
                                                const T* __restrict__ ya, T* __restrict__ dp, T* __restrict__ gq,
                                                T* __restrict__ dA, int i, int j, const ScPre<T>& p) {
    const int N = g.N, n = N * N, m = N - 1;
    const int c = j * N + i;
    auto pval = [&](int ii, int jj, T dm) {
        ii &= m;
        jj &= m;
        const int cc = jj * N + ii;
        return km.one_c1 * dM[cc] + km.c2 * (sv[cc] - divg(g, ya, ii, jj)) * dm;
    };
    const T pc = pval(i, j, p.m), pw = pval(i - 1, j, p.mw), ps = pval(i, j - 1, p.ms);
    dp[c] = pc;
    const T gu = (pc - pw) * g.inv_h, gv = (pc - ps) * g.inv_h;
    gq[c] = gu;
    gq[n + c] = gv;
    dA[c] = ka.inv_theta * gu * p.a0;
    dA[n + c] = ka.inv_theta * gv * p.a1;
}
// yy = (1 + c1) dA + c2 DA^{-1} (gq - A_IB dA);  xo = x + omega (y - yy, dp)  (x == nullptr: x = 0)
template <typename T>
__device__ __forceinline__ void sc_finish_cell(const GridK<T>& g, const Cheb2<T>& ka, const T* __restrict__ x,
                                               const T* __restrict__ y, const T* __restrict__ gq,
                                               const T* __restrict__ dA, const T* __restrict__ dp, T* __restrict__ xo,
                                               int i, int j, const ScPre<T>& p) {
    const int N = g.N, n = N * N;
    const int c = j * N + i;
    for (int comp = 0; comp < 2; ++comp) {
        const int f = comp * n + c;
        const T yy = ka.one_c1 * dA[f] + ka.c2 * (gq[f] - Aib_act(g, p.act, dA, comp, i, j)) * (comp ? p.a1 : p.a0);
        xo[f] = (x ? x[f] : T(0)) + g.omega * (y[f] - yy);
    }
    xo[2 * n + c] = (x ? x[2 * n + c] : T(0)) + g.omega * dp[c];
}

}  // namespace sib
