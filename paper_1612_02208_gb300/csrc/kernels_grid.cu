// MAC-grid stencil kernels of one multigrid level: Stokes-IB residual, additive Vanka sweep,
// RT0 restriction / prolongation, precision casts, Schur-complement smoother pieces.
//
// Layout: a level vector is [u | v | p], each N*N row-major [j][i]; u[j][i] on the x-face
// (i-1/2, j), v[j][i] on the y-face (i, j-1/2), p[j][i] at the cell centre (Appendix,
// "Eulerian discretization").  N is a power of two, so periodic wrap is a mask.
#include <cstring>

#include "grid_cells.cuh"
#include "tma.cuh"

namespace sib {

// ------------------------------------------------------------------------------------------
// Residual r = b - L x, or y = L x when b == nullptr, with
//   (L x)_u = A u - dt [SKJ] u + G p,   (L x)_p = -D u     (Eq. matrix-impib / matrix-h-impib)
//   A u = a0 u - c (u_E + u_W + u_N + u_S),  (G p)_{i-1/2,j} = (p_ij - p_{i-1,j}) / h,
//   (D u)_ij = (u_{i+1/2,j} - u_{i-1/2,j} + v_{i,j+1/2} - v_{i,j-1/2}) / h.
// The IB term dt [SKJ]^l u enters through g.fib, computed beforehand for the same x.
template <typename T, bool HAS_B>
__global__ void __launch_bounds__(256) k_residual(GridK<T> g, const T* __restrict__ x, const T* __restrict__ b,
                                                  T* __restrict__ r) {
    const bool act = g.tile != nullptr && g.tile[blockIdx.y * g.ntx + blockIdx.x];   // set-up data, before the wait
    pdl_entry();
    const int N = g.N, n = N * N, m = N - 1;
    const int i = blockIdx.x * g.tx + threadIdx.x;
    const int j = blockIdx.y * g.ty + threadIdx.y;
    const int ip = (i + 1) & m, im = (i - 1) & m, jp = (j + 1) & m, jm = (j - 1) & m;
    const T* u = x;
    const T* v = x + n;
    const T* p = x + 2 * n;
    const int c = j * N + i;
    const T uc = u[c], vc = v[c], pc = p[c];
    const T uE = u[j * N + ip], uW = u[j * N + im], uN = u[jp * N + i], uS = u[jm * N + i];
    const T vE = v[j * N + ip], vW = v[j * N + im], vN = v[jp * N + i], vS = v[jm * N + i];
    const T pW = p[j * N + im], pS = p[jm * N + i];
    T Au = g.a0 * uc - g.c * ((uE + uW) + (uN + uS)) + (pc - pW) * g.inv_h;
    T Av = g.a0 * vc - g.c * ((vE + vW) + (vN + vS)) + (pc - pS) * g.inv_h;
    const T Dp = -((uE - uc) + (vN - vc)) * g.inv_h;
    Au -= g.dt * ibf_act(g, act, 0, i, j);
    Av -= g.dt * ibf_act(g, act, 1, i, j);
    if (HAS_B) {
        r[c] = b[c] - Au;
        r[n + c] = b[n + c] - Av;
        r[2 * n + c] = b[2 * n + c] - Dp;
    } else {
        r[c] = Au;
        r[n + c] = Av;
        r[2 * n + c] = Dp;
    }
}

template <typename T>
void launch_residual(const GridK<T>& g, const T* x, const T* b, T* r, cudaStream_t s) {
    dim3 blk(g.tx, g.ty), grd(g.N / g.tx, g.N / g.ty);
    if (b)
        launch_pdl(k_residual<T, true>, grd, blk, 0, s, g, x, b, r);
    else
        launch_pdl(k_residual<T, false>, grd, blk, 0, s, g, x, nullptr, r);
}

// ------------------------------------------------------------------------------------------
// One additive Vanka sweep (Alg. 2 with one-cell subdomains, corrections weighted and summed):
//   xo = x + omega * sum_c W_c R_c^T L_c^{-1} R_c (b - L x),  W = diag(1/2, 1/2, 1/2, 1/2, 1).
// Patch of cell (i,j): (u_{i-1/2,j}, u_{i+1/2,j}, v_{i,j-1/2}, v_{i,j+1/2}, p_ij) with
//   L_c = [[A_u, 0, g], [0, A_v, g], [g^T, g^T, 0]],  g = (1/h, -1/h),
//   A_u = [[a0 - dt B(uL,uL), -c - dt B(uL,uR)], [., a0 - dt B(uR,uR)]] (same for v),
// solved by block elimination on the pressure.  Phase 1 forms the residual on the tile plus a
// one-cell halo, phase 2 solves the patches of the tile plus its left/bottom halo cells,
// phase 3 adds to every face the average of the corrections of its two cells.
template <typename T, bool ZERO>
__global__ void __launch_bounds__(256) k_vanka(GridK<T> g, const T* __restrict__ x, const T* __restrict__ b,
                                               T* __restrict__ xo) {
    pdl_entry();
    __shared__ T sru[(TY + 2) * (TX + 2)];
    __shared__ T srv[(TY + 2) * (TX + 2)];
    __shared__ T srp[(TY + 2) * (TX + 2)];
    __shared__ T sd[5][(TY + 1) * (TX + 1)];
    const int N = g.N, n = N * N, m = N - 1;
    const int tx = g.tx, ty = g.ty;
    const int i0 = blockIdx.x * tx, j0 = blockIdx.y * ty;
    const int tid = threadIdx.y * tx + threadIdx.x, nth = tx * ty;
    const bool act = g.tile != nullptr && g.tile[blockIdx.y * g.ntx + blockIdx.x];
    const T* u = x;
    const T* v = x + n;
    const T* p = x + 2 * n;
    const int RW = tx + 2, RH = ty + 2;
    for (int q = tid; q < RW * RH; q += nth) {
        const int i = (i0 - 1 + q % RW) & m, j = (j0 - 1 + q / RW) & m;
        const int c = j * N + i;
        if (ZERO) {   // x = 0: the residual is b
            sru[q] = b[c];
            srv[q] = b[n + c];
            srp[q] = b[2 * n + c];
            continue;
        }
        const int ip = (i + 1) & m, im = (i - 1) & m, jp = (j + 1) & m, jm = (j - 1) & m;
        const T uc = u[c], vc = v[c], pc = p[c];
        const T uE = u[j * N + ip], uW = u[j * N + im], uN = u[jp * N + i], uS = u[jm * N + i];
        const T vE = v[j * N + ip], vW = v[j * N + im], vN = v[jp * N + i], vS = v[jm * N + i];
        T Au = g.a0 * uc - g.c * ((uE + uW) + (uN + uS)) + (pc - p[j * N + im]) * g.inv_h;
        T Av = g.a0 * vc - g.c * ((vE + vW) + (vN + vS)) + (pc - p[jm * N + i]) * g.inv_h;
        if (act) {   // fib holds [S K J] x (zero in inactive tiles; the flags are dilated by one tile)
            Au -= g.dt * g.fib[c];
            Av -= g.dt * g.fib[n + c];
        }
        sru[q] = b[c] - Au;
        srv[q] = b[n + c] - Av;
        srp[q] = b[2 * n + c] + ((uE - uc) + (vN - vc)) * g.inv_h;
    }
    __syncthreads();
    const int PW = tx + 1, PH = ty + 1;
    const T ih = g.inv_h;
    for (int q = tid; q < PW * PH; q += nth) {
        const int pi = q % PW, pj = q / PW;
        const int i = (i0 - 1 + pi) & m, j = (j0 - 1 + pj) & m;
        const T r0 = sru[pj * RW + pi], r1 = sru[pj * RW + pi + 1];
        const T r2 = srv[pj * RW + pi], r3 = srv[(pj + 1) * RW + pi];
        const T r4 = srp[pj * RW + pi];
        T f[7];
        const int cc = j * N + i;
#pragma unroll
        for (int k = 0; k < 7; ++k) f[k] = g.pf[(size_t)k * n + cc];
        T d0, d1, d2, d3, dp;
        patch_solve(f, ih, r0, r1, r2, r3, r4, d0, d1, d2, d3, dp);
        sd[0][q] = d0;
        sd[1][q] = d1;
        sd[2][q] = d2;
        sd[3][q] = d3;
        sd[4][q] = dp;
    }
    __syncthreads();
    const int ci = threadIdx.x, cj = threadIdx.y;
    const int c = (j0 + cj) * N + (i0 + ci);
    const int pc = (cj + 1) * PW + ci + 1, pl = (cj + 1) * PW + ci, pb = cj * PW + ci + 1;
    const T hw = T(0.5) * g.omega;
    if (ZERO) {
        xo[c] = hw * (sd[0][pc] + sd[1][pl]);
        xo[n + c] = hw * (sd[2][pc] + sd[3][pb]);
        xo[2 * n + c] = g.omega * sd[4][pc];
    } else {
        xo[c] = u[c] + hw * (sd[0][pc] + sd[1][pl]);
        xo[n + c] = v[c] + hw * (sd[2][pc] + sd[3][pb]);
        xo[2 * n + c] = p[c] + g.omega * sd[4][pc];
    }
}

// Tiled form of the same sweep for levels with N >= 32 (tiles exactly TX x TY): x is staged in
// shared memory with a two-cell halo by coalesced loads, index arithmetic uses compile-time tile
// sizes, and cells of tiles without IB entries use the constant patch inverse (no divisions).  FP64
// levels take k_vanka_tiled (one cell per thread), FP32 levels k_vanka_pair (two cells per thread).
template <typename T>
VankaBulk<T> vanka_bulk(double a0, double c, double inv_h) {
    const double det = a0 * a0 - c * c;
    const double s0 = inv_h / (a0 + c);
    VankaBulk<T> k;
    k.ai0 = (T)(a0 / det);
    k.ai1 = (T)(c / det);
    k.s0 = (T)s0;
    k.invS = (T)(1.0 / (4.0 * inv_h * s0));
    return k;
}

// Shared-memory layout of the tiled sweep.  Staged b: rows j0-1 .. j0+8, staged x: rows j0-2 ..
// j0+9, both over columns i0-4 .. i0+35 (40 wide, so that the TMA box starts on a 16-byte
// boundary); the residual overwrites the staged b in place, the patch corrections reuse the x area.
constexpr int VK_W = TX + 8;                   // staged row width
constexpr int VK_BR = TY + 2, VK_XR = TY + 4;  // staged rows of b and of x
constexpr int VK_PX = TX + 1, VK_PY = TY + 1;  // patches: tile plus its left and bottom neighbours
constexpr int VK_SB = 3 * VK_BR * VK_W;        // 1200 words of b
constexpr int VK_XOFF = ((VK_SB + 31) / 32) * 32;                       // x area, 128-byte aligned
constexpr int VK_STAGE = VK_XOFF + (3 * VK_XR * VK_W > 5 * VK_PY * VK_PX ? 3 * VK_XR * VK_W : 5 * VK_PY * VK_PX);
constexpr int VK_WAIT_LIMIT = 1 << 22;         // bounded wait for the tile copies

template <typename T, bool ZERO>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 8 : 4)
    k_vanka_tiled(GridK<T> g, VankaBulk<T> kb, const __grid_constant__ CUtensorMap mx,
                  const __grid_constant__ CUtensorMap mb, int tma, int first_wave, const T* __restrict__ x,
                  const T* __restrict__ b, T* __restrict__ xo) {
    __shared__ __align__(128) T stage[VK_STAGE];
    __shared__ T bs[7][VK_PY][VK_PX];   // patch factors of the patches of an active tile
    __shared__ uint64_t bar;
    T(*sb)[VK_BR][VK_W] = reinterpret_cast<T(*)[VK_BR][VK_W]>(stage);
    T(*sx)[VK_XR][VK_W] = reinterpret_cast<T(*)[VK_XR][VK_W]>(stage + VK_XOFF);
    T(*ds)[VK_PY][VK_PX] = reinterpret_cast<T(*)[VK_PY][VK_PX]>(stage + VK_XOFF);
    const int N = g.N, n = N * N, m = N - 1;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    // tiles whose staged window lies inside the grid take the TMA copies; the others (the periodic
    // wrap) and grids without tensor maps gather element by element
    const bool bulk = tma && i0 >= TX && i0 + 2 * TX <= N && j0 >= TY && j0 + 2 * TY <= N;
    // set-up data (tile flag, patch entries): blocks of the first wave load it before the wait for x
    // and b, hidden behind the preceding kernel; later blocks issue their tile copies first and load
    // it while the copies are in flight
    const bool early = (int)(blockIdx.y * gridDim.x + blockIdx.x) < first_wave;
    bool act = false;
    auto load_patch_ib = [&]() {
        for (int q = tid; q < VK_PY * VK_PX; q += TX * TY) {
            const int pj = q / VK_PX, pi = q - pj * VK_PX;
            const int cc = ((j0 - 1 + pj) & m) * N + ((i0 - 1 + pi) & m);
#pragma unroll
            for (int k = 0; k < 7; ++k) bs[k][pj][pi] = g.pf[(size_t)k * n + cc];
        }
    };
    if (early) {
        act = g.tile != nullptr && g.tile[blockIdx.y * g.ntx + blockIdx.x];
        if (act) load_patch_ib();
    }
    if (bulk && tid == 0) {
        tma_prefetch_map(&mb);
        if (!ZERO) tma_prefetch_map(&mx);
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    if (early) __syncthreads();   // patch entries and the barrier's initialisation complete
    pdl_entry();
    if (bulk && tid == 0) {
        constexpr uint32_t bb = 3 * VK_BR * VK_W * sizeof(T), bx = 3 * VK_XR * VK_W * sizeof(T);
        mbar_expect_tx(&bar, ZERO ? bb : bb + bx);
        tma_load_3d(&sb[0][0][0], &mb, &bar, i0 - 4, j0 - 1, 0);
        if (!ZERO) tma_load_3d(&sx[0][0][0], &mx, &bar, i0 - 4, j0 - 2, 0);
    }
    if (!early) {
        act = g.tile != nullptr && g.tile[blockIdx.y * g.ntx + blockIdx.x];
        if (act) load_patch_ib();
    }
    // residual cells: this thread's own (ri, rj) = (tx + 1, ty + 1) and, for the first
    // 2 (TX + TY) + 4 threads, one cell of the ring around the tile
    constexpr int RING = 2 * (TX + 2) + 2 * TY;
    int ri2 = 0, rj2 = 0;
    if (tid < TX + 2) {
        ri2 = tid;
    } else if (tid < 2 * (TX + 2)) {
        ri2 = tid - (TX + 2);
        rj2 = TY + 1;
    } else if (tid < 2 * (TX + 2) + TY) {
        rj2 = tid - 2 * (TX + 2) + 1;
    } else {
        ri2 = TX + 1;
        rj2 = tid - 2 * (TX + 2) - TY + 1;
    }
    // IB term of the residual cells of an active tile, fetched while the tile is in flight
    T fu0 = T(0), fv0 = T(0), fu1 = T(0), fv1 = T(0);
    if (!ZERO && act) {
        const int c0 = (j0 + ty) * N + (i0 + tx);
        fu0 = g.fib[c0];
        fv0 = g.fib[n + c0];
        if (tid < RING) {
            const int c1 = ((j0 - 1 + rj2) & m) * N + ((i0 - 1 + ri2) & m);
            fu1 = g.fib[c1];
            fv1 = g.fib[n + c1];
        }
    }
    if (!early) __syncthreads();   // the barrier's initialisation before the other threads wait on it
    if (bulk) {
        const bool ok = mbar_wait_bounded(&bar, 0, VK_WAIT_LIMIT);
        if (!__syncthreads_and(ok)) {   // copies never completed: report, let them drain, leave
            if (tid == 0 && g.err) *(volatile int*)g.err = SIB_DEV_ERR_TMA_WAIT;
            mbar_wait_bounded(&bar, 0, VK_WAIT_LIMIT);
            return;
        }
    } else {   // b at rows j0-1.., columns i0-1..i0+32; x at rows j0-2.., columns i0-2..i0+33
        constexpr int NB = VK_BR * (TX + 2), NX = VK_XR * (TX + 4), NT = TX * TY;
        static_assert(NB <= 2 * NT && NX <= 2 * NT, "two staging passes");
        T vb[2][3], vx[2][3];
#pragma unroll
        for (int k = 0; k < 2; ++k) {   // every load issued before the first store
            const int q = tid + k * NT;
            if (q < NB) {
                const int rj = q / (TX + 2), ri = q - rj * (TX + 2);
                const int gc = ((j0 - 1 + rj) & m) * N + ((i0 - 1 + ri) & m);
                vb[k][0] = b[gc];
                vb[k][1] = b[n + gc];
                vb[k][2] = b[2 * n + gc];
            }
            if (!ZERO && q < NX) {
                const int jj = q / (TX + 4), ii = q - jj * (TX + 4);
                const int gc = ((j0 - 2 + jj) & m) * N + ((i0 - 2 + ii) & m);
                vx[k][0] = x[gc];
                vx[k][1] = x[n + gc];
                vx[k][2] = x[2 * n + gc];
            }
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int q = tid + k * NT;
            if (q < NB) {
                const int rj = q / (TX + 2), ri = q - rj * (TX + 2);
                sb[0][rj][ri + 3] = vb[k][0];
                sb[1][rj][ri + 3] = vb[k][1];
                sb[2][rj][ri + 3] = vb[k][2];
            }
            if (!ZERO && q < NX) {
                const int jj = q / (TX + 4), ii = q - jj * (TX + 4);
                sx[0][jj][ii + 2] = vx[k][0];
                sx[1][jj][ii + 2] = vx[k][1];
                sx[2][jj][ii + 2] = vx[k][2];
            }
        }
        __syncthreads();
    }
    // residual r = b - L x on the tile plus one cell each side (rows rj = 0..TY+1 <-> j0-1+rj,
    // columns ri = 0..TX+1 <-> i0-1+ri), written over the staged b
    T xu = T(0), xv = T(0), xp = T(0);
    if (!ZERO) {
        auto residual = [&](int ri, int rj, T fu, T fv, bool own) {
            const int sxc = ri + 3, sy = rj + 1, sbc = ri + 3;
            const T uc = sx[0][sy][sxc], vc = sx[1][sy][sxc], pc = sx[2][sy][sxc];
            const T uE = sx[0][sy][sxc + 1], vN = sx[1][sy + 1][sxc];
            T Au = g.a0 * uc - g.c * ((uE + sx[0][sy][sxc - 1]) + (sx[0][sy + 1][sxc] + sx[0][sy - 1][sxc])) +
                   (pc - sx[2][sy][sxc - 1]) * g.inv_h;
            T Av = g.a0 * vc - g.c * ((sx[1][sy][sxc + 1] + sx[1][sy][sxc - 1]) + (vN + sx[1][sy - 1][sxc])) +
                   (pc - sx[2][sy - 1][sxc]) * g.inv_h;
            if (act) {
                Au -= g.dt * fu;
                Av -= g.dt * fv;
            }
            sb[0][rj][sbc] = sb[0][rj][sbc] - Au;
            sb[1][rj][sbc] = sb[1][rj][sbc] - Av;
            sb[2][rj][sbc] = sb[2][rj][sbc] + ((uE - uc) + (vN - vc)) * g.inv_h;
            if (own) {
                xu = uc;
                xv = vc;
                xp = pc;
            }
        };
        residual(tx + 1, ty + 1, fu0, fv0, true);
        if (tid < RING) residual(ri2, rj2, fu1, fv1, false);
        __syncthreads();
    }
    // patch solves for cells (i0-1+pi, j0-1+pj), pi = 0..TX, pj = 0..TY; the residual of patch
    // (pi, pj) sits at (ri, rj) = (pi, pj) of the staged area (column offset 3)
    const T ih = g.inv_h;
    auto patch = [&](int pi, int pj) {
        const T r0 = sb[0][pj][pi + 3], r1 = sb[0][pj][pi + 4];
        const T r2 = sb[1][pj][pi + 3], r3 = sb[1][pj + 1][pi + 3];
        const T r4 = sb[2][pj][pi + 3];
        T d0, d1, d2, d3, dp;
        if (!act) {
            const T tu0 = kb.ai0 * r0 + kb.ai1 * r1, tu1 = kb.ai1 * r0 + kb.ai0 * r1;
            const T tv0 = kb.ai0 * r2 + kb.ai1 * r3, tv1 = kb.ai1 * r2 + kb.ai0 * r3;
            dp = (ih * ((tu0 - tu1) + (tv0 - tv1)) - r4) * kb.invS;
            d0 = tu0 - kb.s0 * dp;
            d1 = tu1 + kb.s0 * dp;
            d2 = tv0 - kb.s0 * dp;
            d3 = tv1 + kb.s0 * dp;
        } else {
            T f[7];
#pragma unroll
            for (int k = 0; k < 7; ++k) f[k] = bs[k][pj][pi];
            patch_solve(f, ih, r0, r1, r2, r3, r4, d0, d1, d2, d3, dp);
        }
        ds[0][pj][pi] = d0;
        ds[1][pj][pi] = d1;
        ds[2][pj][pi] = d2;
        ds[3][pj][pi] = d3;
        ds[4][pj][pi] = dp;
    };
    patch(tx + 1, ty + 1);
    if (tid < VK_PX + TY) {   // bottom row pj = 0, then left column pi = 0 (one call: no divergent copies)
        const bool row = tid < VK_PX;
        patch(row ? tid : 0, row ? 0 : tid - VK_PX + 1);
    }
    __syncthreads();
    const int c = (j0 + ty) * N + (i0 + tx);
    const T hw = T(0.5) * g.omega;
    const T du = hw * (ds[0][ty + 1][tx + 1] + ds[1][ty + 1][tx]);
    const T dv = hw * (ds[2][ty + 1][tx + 1] + ds[3][ty][tx + 1]);
    const T dq = g.omega * ds[4][ty + 1][tx + 1];
    if (ZERO) {
        xo[c] = du;
        xo[n + c] = dv;
        xo[2 * n + c] = dq;
    } else {
        xo[c] = xu + du;
        xo[n + c] = xv + dv;
        xo[2 * n + c] = xp + dq;
    }
}

// FP32 form of the tiled sweep with two vertically adjacent cells per thread (TX x TY / 2 threads):
// the residual stencils of a pair share their x reads, and each thread keeps its cells' residuals
// and patch corrections in registers.  Shared memory carries only what a neighbour reads: the u
// residuals (read by the patch to the left), the lower cell's v residual (read by the pair below's
// upper patch), the corrections d1 (read by the cell to the right) and the upper cell's d3 (read by
// the pair above).  The ring of residual cells and the left / bottom ring of patches are formed by
// the first threads as in k_vanka_tiled; staging, set-up data and the arithmetic are the same.
constexpr int VK2_THREADS = TX * TY / 2;
template <typename T, bool ZERO>
__global__ void __launch_bounds__(VK2_THREADS, 8)
    k_vanka_pair(GridK<T> g, VankaBulk<T> kb, const __grid_constant__ CUtensorMap mx,
                 const __grid_constant__ CUtensorMap mb, int tma, int first_wave, const T* __restrict__ x,
                 const T* __restrict__ b, T* __restrict__ xo) {
    constexpr int NT = VK2_THREADS;
    __shared__ __align__(128) T stage[VK_STAGE];
    __shared__ T bs[7][VK_PY][VK_PX];   // patch factors of the patches of an active tile
    __shared__ uint64_t bar;
    T(*sb)[VK_BR][VK_W] = reinterpret_cast<T(*)[VK_BR][VK_W]>(stage);
    T(*sx)[VK_XR][VK_W] = reinterpret_cast<T(*)[VK_XR][VK_W]>(stage + VK_XOFF);
    T(*ds)[VK_PY][VK_PX] = reinterpret_cast<T(*)[VK_PY][VK_PX]>(stage + VK_XOFF);   // [0] d1, [1] d3
    const int N = g.N, n = N * N, m = N - 1;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;   // ty: pair row, cells 2 ty, 2 ty + 1
    const bool bulk = tma && i0 >= TX && i0 + 2 * TX <= N && j0 >= TY && j0 + 2 * TY <= N;
    const bool early = (int)(blockIdx.y * gridDim.x + blockIdx.x) < first_wave;
    bool act = false;
    auto load_patch_ib = [&]() {
        for (int q = tid; q < VK_PY * VK_PX; q += NT) {
            const int pj = q / VK_PX, pi = q - pj * VK_PX;
            const int cc = ((j0 - 1 + pj) & m) * N + ((i0 - 1 + pi) & m);
#pragma unroll
            for (int k = 0; k < 7; ++k) bs[k][pj][pi] = g.pf[(size_t)k * n + cc];
        }
    };
    if (early) {
        act = g.tile != nullptr && g.tile[blockIdx.y * g.ntx + blockIdx.x];
        if (act) load_patch_ib();
    }
    if (bulk && tid == 0) {
        tma_prefetch_map(&mb);
        if (!ZERO) tma_prefetch_map(&mx);
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    if (early) __syncthreads();
    pdl_entry();
    if (bulk && tid == 0) {
        constexpr uint32_t bb = 3 * VK_BR * VK_W * sizeof(T), bx = 3 * VK_XR * VK_W * sizeof(T);
        mbar_expect_tx(&bar, ZERO ? bb : bb + bx);
        tma_load_3d(&sb[0][0][0], &mb, &bar, i0 - 4, j0 - 1, 0);
        if (!ZERO) tma_load_3d(&sx[0][0][0], &mx, &bar, i0 - 4, j0 - 2, 0);
    }
    if (!early) {
        act = g.tile != nullptr && g.tile[blockIdx.y * g.ntx + blockIdx.x];
        if (act) load_patch_ib();
    }
    constexpr int RING = 2 * (TX + 2) + 2 * TY;
    static_assert(RING <= NT && VK_PX + TY <= NT, "one ring cell and one ring patch per thread");
    int ri2 = 0, rj2 = 0;
    if (tid < TX + 2) {
        ri2 = tid;
    } else if (tid < 2 * (TX + 2)) {
        ri2 = tid - (TX + 2);
        rj2 = TY + 1;
    } else if (tid < 2 * (TX + 2) + TY) {
        rj2 = tid - 2 * (TX + 2) + 1;
    } else {
        ri2 = TX + 1;
        rj2 = tid - 2 * (TX + 2) - TY + 1;
    }
    T fu[2] = {T(0), T(0)}, fv[2] = {T(0), T(0)}, fu1 = T(0), fv1 = T(0);
    if (!ZERO && act) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int cc = (j0 + 2 * ty + c) * N + (i0 + tx);
            fu[c] = g.fib[cc];
            fv[c] = g.fib[n + cc];
        }
        if (tid < RING) {
            const int c1 = ((j0 - 1 + rj2) & m) * N + ((i0 - 1 + ri2) & m);
            fu1 = g.fib[c1];
            fv1 = g.fib[n + c1];
        }
    }
    if (!early) __syncthreads();
    if (bulk) {
        const bool ok = mbar_wait_bounded(&bar, 0, VK_WAIT_LIMIT);
        if (!__syncthreads_and(ok)) {   // copies never completed: report, let them drain, leave
            if (tid == 0 && g.err) *(volatile int*)g.err = SIB_DEV_ERR_TMA_WAIT;
            mbar_wait_bounded(&bar, 0, VK_WAIT_LIMIT);
            return;
        }
    } else {   // b at rows j0-1.., columns i0-1..i0+32; x at rows j0-2.., columns i0-2..i0+33
        constexpr int NB = VK_BR * (TX + 2), NX = VK_XR * (TX + 4);
        constexpr int PB = (NB + NT - 1) / NT, PXN = (NX + NT - 1) / NT;
        T vb[PB][3], vx[PXN][3];
#pragma unroll
        for (int k = 0; k < PB; ++k) {   // every load issued before the first store
            const int q = tid + k * NT;
            if (q < NB) {
                const int rj = q / (TX + 2), ri = q - rj * (TX + 2);
                const int gc = ((j0 - 1 + rj) & m) * N + ((i0 - 1 + ri) & m);
                vb[k][0] = b[gc];
                vb[k][1] = b[n + gc];
                vb[k][2] = b[2 * n + gc];
            }
        }
        if (!ZERO) {
#pragma unroll
            for (int k = 0; k < PXN; ++k) {
                const int q = tid + k * NT;
                if (q < NX) {
                    const int jj = q / (TX + 4), ii = q - jj * (TX + 4);
                    const int gc = ((j0 - 2 + jj) & m) * N + ((i0 - 2 + ii) & m);
                    vx[k][0] = x[gc];
                    vx[k][1] = x[n + gc];
                    vx[k][2] = x[2 * n + gc];
                }
            }
        }
#pragma unroll
        for (int k = 0; k < PB; ++k) {
            const int q = tid + k * NT;
            if (q < NB) {
                const int rj = q / (TX + 2), ri = q - rj * (TX + 2);
                sb[0][rj][ri + 3] = vb[k][0];
                sb[1][rj][ri + 3] = vb[k][1];
                sb[2][rj][ri + 3] = vb[k][2];
            }
        }
        if (!ZERO) {
#pragma unroll
            for (int k = 0; k < PXN; ++k) {
                const int q = tid + k * NT;
                if (q < NX) {
                    const int jj = q / (TX + 4), ii = q - jj * (TX + 4);
                    sx[0][jj][ii + 2] = vx[k][0];
                    sx[1][jj][ii + 2] = vx[k][1];
                    sx[2][jj][ii + 2] = vx[k][2];
                }
            }
        }
        __syncthreads();
    }

    // residuals of the pair, staged coordinates (ri, rj) = (tx + 1, 2 ty + 1 + c), c = 0 lower, 1 upper
    const int ri = tx + 1, rj0 = 2 * ty + 1, sc = ri + 3;
    T ru[2], rv[2], rp[2], xu[2] = {T(0), T(0)}, xv[2] = {T(0), T(0)}, xp[2] = {T(0), T(0)};
    if (ZERO) {   // x = 0: the residual is b, already in place
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            ru[c] = sb[0][rj0 + c][sc];
            rv[c] = sb[1][rj0 + c][sc];
            rp[c] = sb[2][rj0 + c][sc];
        }
    } else {
        const int y0 = rj0 + 1;   // staged x row of the lower cell
        const T uS = sx[0][y0 - 1][sc], u0 = sx[0][y0][sc], u1 = sx[0][y0 + 1][sc], uN = sx[0][y0 + 2][sc];
        const T uE0 = sx[0][y0][sc + 1], uW0 = sx[0][y0][sc - 1], uE1 = sx[0][y0 + 1][sc + 1], uW1 = sx[0][y0 + 1][sc - 1];
        const T vS = sx[1][y0 - 1][sc], v0 = sx[1][y0][sc], v1 = sx[1][y0 + 1][sc], vN = sx[1][y0 + 2][sc];
        const T vE0 = sx[1][y0][sc + 1], vW0 = sx[1][y0][sc - 1], vE1 = sx[1][y0 + 1][sc + 1], vW1 = sx[1][y0 + 1][sc - 1];
        const T pS = sx[2][y0 - 1][sc], p0 = sx[2][y0][sc], p1 = sx[2][y0 + 1][sc];
        const T pW0 = sx[2][y0][sc - 1], pW1 = sx[2][y0 + 1][sc - 1];
        T Au0 = g.a0 * u0 - g.c * ((uE0 + uW0) + (u1 + uS)) + (p0 - pW0) * g.inv_h;
        T Av0 = g.a0 * v0 - g.c * ((vE0 + vW0) + (v1 + vS)) + (p0 - pS) * g.inv_h;
        T Au1 = g.a0 * u1 - g.c * ((uE1 + uW1) + (uN + u0)) + (p1 - pW1) * g.inv_h;
        T Av1 = g.a0 * v1 - g.c * ((vE1 + vW1) + (vN + v0)) + (p1 - p0) * g.inv_h;
        if (act) {
            Au0 -= g.dt * fu[0];
            Av0 -= g.dt * fv[0];
            Au1 -= g.dt * fu[1];
            Av1 -= g.dt * fv[1];
        }
        ru[0] = sb[0][rj0][sc] - Au0;
        rv[0] = sb[1][rj0][sc] - Av0;
        rp[0] = sb[2][rj0][sc] + ((uE0 - u0) + (v1 - v0)) * g.inv_h;
        ru[1] = sb[0][rj0 + 1][sc] - Au1;
        rv[1] = sb[1][rj0 + 1][sc] - Av1;
        rp[1] = sb[2][rj0 + 1][sc] + ((uE1 - u1) + (vN - v1)) * g.inv_h;
        xu[0] = u0;
        xu[1] = u1;
        xv[0] = v0;
        xv[1] = v1;
        xp[0] = p0;
        xp[1] = p1;
        // handed to the neighbours: both u residuals, the lower v residual
        sb[0][rj0][sc] = ru[0];
        sb[0][rj0 + 1][sc] = ru[1];
        sb[1][rj0][sc] = rv[0];
        if (tid < RING) {   // one ring cell, all three components in place
            const int sxc = ri2 + 3, sy = rj2 + 1;
            const T uc = sx[0][sy][sxc], vc = sx[1][sy][sxc], pc = sx[2][sy][sxc];
            const T uE = sx[0][sy][sxc + 1], vN1 = sx[1][sy + 1][sxc];
            T Au = g.a0 * uc - g.c * ((uE + sx[0][sy][sxc - 1]) + (sx[0][sy + 1][sxc] + sx[0][sy - 1][sxc])) +
                   (pc - sx[2][sy][sxc - 1]) * g.inv_h;
            T Av = g.a0 * vc - g.c * ((sx[1][sy][sxc + 1] + sx[1][sy][sxc - 1]) + (vN1 + sx[1][sy - 1][sxc])) +
                   (pc - sx[2][sy - 1][sxc]) * g.inv_h;
            if (act) {
                Au -= g.dt * fu1;
                Av -= g.dt * fv1;
            }
            sb[0][rj2][sxc] = sb[0][rj2][sxc] - Au;
            sb[1][rj2][sxc] = sb[1][rj2][sxc] - Av;
            sb[2][rj2][sxc] = sb[2][rj2][sxc] + ((uE - uc) + (vN1 - vc)) * g.inv_h;
        }
        __syncthreads();   // residuals handed over; the x area is free for the corrections
    }
    const T ih = g.inv_h;
    auto solve = [&](int pi, int pj, T r0, T r1, T r2, T r3, T r4, T& d0, T& d1, T& d2, T& d3, T& dp) {
        if (!act) {
            const T tu0 = kb.ai0 * r0 + kb.ai1 * r1, tu1 = kb.ai1 * r0 + kb.ai0 * r1;
            const T tv0 = kb.ai0 * r2 + kb.ai1 * r3, tv1 = kb.ai1 * r2 + kb.ai0 * r3;
            dp = (ih * ((tu0 - tu1) + (tv0 - tv1)) - r4) * kb.invS;
            d0 = tu0 - kb.s0 * dp;
            d1 = tu1 + kb.s0 * dp;
            d2 = tv0 - kb.s0 * dp;
            d3 = tv1 + kb.s0 * dp;
        } else {
            T f[7];
#pragma unroll
            for (int k = 0; k < 7; ++k) f[k] = bs[k][pj][pi];
            patch_solve(f, ih, r0, r1, r2, r3, r4, d0, d1, d2, d3, dp);
        }
    };
    // the pair's patches (pi, pj) = (tx + 1, 2 ty + 1 + c): r_u of the right face from the cell to the
    // right, r_v of the upper cell's top face from the pair above (or the ring)
    T d0[2], d1[2], d2[2], d3[2], dp[2];
    const T ruR0 = sb[0][rj0][sc + 1], ruR1 = sb[0][rj0 + 1][sc + 1], rvT = sb[1][rj0 + 2][sc];
    solve(ri, rj0, ru[0], ruR0, rv[0], rv[1], rp[0], d0[0], d1[0], d2[0], d3[0], dp[0]);
    solve(ri, rj0 + 1, ru[1], ruR1, rv[1], rvT, rp[1], d0[1], d1[1], d2[1], d3[1], dp[1]);
    // ring patches: bottom row pj = 0 (their d3 feeds the tile's bottom cells), then the left column
    // pi = 0 (their d1 feeds the tile's left cells); one call, no divergent copies
    T e0 = T(0), e1 = T(0), e2 = T(0), e3 = T(0), ep = T(0);
    const bool ringPatch = tid < VK_PX + TY;
    const bool rowPatch = tid < VK_PX;
    const int qi = rowPatch ? tid : 0, qj = rowPatch ? 0 : tid - VK_PX + 1;
    if (ringPatch)
        solve(qi, qj, sb[0][qj][qi + 3], sb[0][qj][qi + 4], sb[1][qj][qi + 3], sb[1][qj + 1][qi + 3],
              sb[2][qj][qi + 3], e0, e1, e2, e3, ep);
    ds[0][rj0][ri] = d1[0];   // the x area is no longer read
    ds[0][rj0 + 1][ri] = d1[1];
    ds[1][rj0 + 1][ri] = d3[1];
    if (ringPatch) {
        if (rowPatch)
            ds[1][qj][qi] = e3;
        else
            ds[0][qj][qi] = e1;
    }
    __syncthreads();
    const T hw = T(0.5) * g.omega;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const int cc = (j0 + 2 * ty + c) * N + (i0 + tx);
        const T du = hw * (d0[c] + ds[0][rj0 + c][ri - 1]);
        const T dv = hw * (d2[c] + (c == 0 ? ds[1][rj0 - 1][ri] : d3[0]));
        const T dq = g.omega * dp[c];
        if (ZERO) {
            xo[cc] = du;
            xo[n + cc] = dv;
            xo[2 * n + cc] = dq;
        } else {
            xo[cc] = xu[c] + du;
            xo[n + cc] = xv[c] + dv;
            xo[2 * n + cc] = xp[c] + dq;
        }
    }
}

// Tensor map of a level vector [u | v | p] (comps = 3) or of the IB force [f_u | f_v] (comps = 2)
// viewed as N x N x comps (column fastest) with a box of boxW x rows x comps; false if the base is not
// 16-byte aligned or the driver cannot encode it.  Encoded maps are kept per thread, keyed by (base, N,
// element size, rows, box width, components).
static bool field_map(CUtensorMap* out, const void* base, int N, int es, int rows, int boxW = VK_W, int comps = 3) {
    struct Entry {
        const void* p;
        int N, es, rows, boxW, comps;
        CUtensorMap m;
    };
    constexpr int CACHE = 32;
    static thread_local Entry cache[CACHE];
    static thread_local int used = 0, next = 0;
    for (int k = 0; k < used; ++k)
        if (cache[k].p == base && cache[k].N == N && cache[k].es == es && cache[k].rows == rows &&
            cache[k].boxW == boxW && cache[k].comps == comps) {
            *out = cache[k].m;
            return true;
        }
    static PFN_cuTensorMapEncodeTiled_v12000 enc = []() {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }();
    if (!enc || (reinterpret_cast<uintptr_t>(base) & 15) != 0) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)N, (cuuint64_t)N, (cuuint64_t)comps};
    const cuuint64_t strides[2] = {(cuuint64_t)N * es, (cuuint64_t)N * N * es};
    const cuuint32_t box[3] = {(cuuint32_t)boxW, (cuuint32_t)rows, (cuuint32_t)comps};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUtensorMap m;
    const CUresult r = enc(&m, es == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3,
                           const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
    Entry& e = cache[next];
    e = Entry{base, N, es, rows, boxW, comps, m};
    next = (next + 1) % CACHE;
    if (used < CACHE) ++used;
    *out = m;
    return true;
}

// blocks of a kernel that are resident on the GPU at once (occupancy x SM count); 0 if unknown
template <typename K>
int resident_blocks(K kern, int threads = TX * TY) {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, 0) != cudaSuccess)
        return 0;
    return sms * per;
}

template <typename T, bool ZERO>
void launch_vanka_any(const GridK<T>& g, const T* x, const T* b, T* xo, cudaStream_t s) {
    dim3 blk(g.tx, g.ty), grd(g.N / g.tx, g.N / g.ty);
    if (g.tx != TX || g.ty != TY) {
        launch_pdl(k_vanka<T, ZERO>, grd, blk, 0, s, g, x, b, xo);
        return;
    }
    const VankaBulk<T> kb = vanka_bulk<T>(g.a0, g.c, g.inv_h);
    CUtensorMap mx, mb;
    std::memset(&mx, 0, sizeof(mx));
    std::memset(&mb, 0, sizeof(mb));
    // interior tiles exist from N = 4 TX on; the maps are only read by those tiles
    const int tma = g.N >= 4 * TX && field_map(&mb, b, g.N, sizeof(T), VK_BR) &&
                    (ZERO || field_map(&mx, x, g.N, sizeof(T), VK_XR));
    if constexpr (sizeof(T) == 4) {   // FP32: two cells per thread
        static const int first_wave2 = resident_blocks(k_vanka_pair<T, ZERO>, VK2_THREADS);
        launch_pdl(k_vanka_pair<T, ZERO>, grd, dim3(TX, TY / 2), 0, s, g, kb, mx, mb, tma, first_wave2, x, b, xo);
        return;
    }
    static const int first_wave = resident_blocks(k_vanka_tiled<T, ZERO>);
    launch_pdl(k_vanka_tiled<T, ZERO>, grd, blk, 0, s, g, kb, mx, mb, tma, first_wave, x, b, xo);
}

template <typename T>
void launch_vanka(const GridK<T>& g, const T* x, const T* b, T* xo, cudaStream_t s) {
    launch_vanka_any<T, false>(g, x, b, xo, s);
}
// the first sweep from a zero initial guess (Alg. 1 recursion): no reads of x, residual = b
template <typename T>
void launch_vanka_zero(const GridK<T>& g, const T* b, T* xo, cudaStream_t s) {
    launch_vanka_any<T, true>(g, b, b, xo, s);   // x is never read
}

// ------------------------------------------------------------------------------------------
// Fine residual and its restriction in one pass (Sec. 3.2, Alg. 1): one thread per coarse cell.
template <typename T>
__global__ void k_residual_restrict(GridK<T> g, const T* __restrict__ x, const T* __restrict__ b, T* __restrict__ bc) {
    pdl_entry();
    const int Nc = g.N / 2;
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    if (I >= Nc || J >= Nc) return;
    residual_restrict_cell(g, x, b, bc, I, J);
}
// The same residual and restriction for N >= 64, tiled: one block per 32 x 8 coarse cells (64 x 16
// fine cells).  The block stages x (three components, fine rows fj0-2 .. fj0+17), b and the IB force
// (rows fj0-1 .. fj0+16), all over columns fi0-4 .. fi0+67, in shared memory.  Blocks whose staged
// rows and columns lie inside the grid load 16-byte vectors, every load issued before the first
// shared store; the others (the periodic wrap) gather element by element.  Each thread then forms, in
// registers, the fine residuals its coarse cell's restriction needs (u faces of columns 2I-1 .. 2I+1,
// v faces of rows 2J-1 .. 2J+1, p of its four cells; the faces it shares with a neighbour are formed
// by both) with the arithmetic of res_u / res_v / res_p, reading the staged rows as column pairs, and
// restricts them as residual_restrict_cell does.  The IB force is read where one of the tile's four
// fine tiles is IB-active: their flags are dilated by one tile and cover the one-cell halo, and the
// force is zero on inactive tiles.
constexpr int RR_CX = 32, RR_CY = 8;                 // coarse cells per block
constexpr int RR_FX = 2 * RR_CX, RR_FY = 2 * RR_CY;  // fine cells per block
constexpr int RR_W = RR_FX + 8;                      // staged row width (columns fi0-4 .. fi0+67)
constexpr int RR_XH = RR_FY + 4, RR_BH = RR_FY + 2;  // staged rows of x (fj0-2 ..) and of b, f (fj0-1 ..)
// staged x (3 x RR_XH rows), b (3 x RR_BH) and, from a 128-byte boundary, the IB force (2 x RR_BH)
constexpr int RR_FOFF = ((3 * RR_XH + 3 * RR_BH) * RR_W + 31) / 32 * 32;
constexpr int RR_WORDS = RR_FOFF + 2 * RR_BH * RR_W;
static_assert((3 * RR_XH * RR_W) % 32 == 0, "the staged b starts on a 128-byte boundary");
template <typename T>
struct RRVec;
template <>
struct RRVec<float> {
    using type = float4;
    using pair = float2;
};
template <>
struct RRVec<double> {
    using type = double2;
    using pair = double2;
};
template <typename T>
__global__ void __launch_bounds__(RR_CX * RR_CY) k_residual_restrict_tiled(GridK<T> g,
                                                                           const __grid_constant__ CUtensorMap mx,
                                                                           const __grid_constant__ CUtensorMap mb,
                                                                           const __grid_constant__ CUtensorMap mf,
                                                                           int tma, const T* __restrict__ x,
                                                                           const T* __restrict__ b,
                                                                           T* __restrict__ bc) {
    constexpr int NXB = 3 * RR_XH + 3 * RR_BH;                 // staged rows of x and b
    constexpr int NROWS = NXB + 2 * RR_BH;                     // and of the IB force
    constexpr int NT = RR_CX * RR_CY;
    extern __shared__ unsigned char rr_smem[];
    __shared__ __align__(8) uint64_t rr_bar;
    // the staged tile from a 128-byte boundary (the launch adds 128 bytes): the TMA boxes land there
    T* st = reinterpret_cast<T*>((reinterpret_cast<uintptr_t>(rr_smem) + 127) & ~(uintptr_t)127);
    T* sx = st;                       // 3 x RR_XH rows
    T* sb = st + 3 * RR_XH * RR_W;    // 3 x RR_BH rows
    T* sf = st + RR_FOFF;             // 2 x RR_BH rows
    const int N = g.N, n = N * N, m = N - 1, Nc = N / 2;
    const int tid = threadIdx.y * RR_CX + threadIdx.x;
    const int fi0 = blockIdx.x * RR_FX, fj0 = blockIdx.y * RR_FY;
    // IB flags of the four fine tiles (set-up data, read before the dependency wait)
    bool act = false;
    if (g.tile) {
        const int ti = fi0 >> g.lgtx, tj = fj0 >> g.lgty;
        act = g.tile[tj * g.ntx + ti] || g.tile[tj * g.ntx + ti + 1] || g.tile[(tj + 1) * g.ntx + ti] ||
              g.tile[(tj + 1) * g.ntx + ti + 1];
    }
    // tiles whose staged rows and columns lie inside the grid take three TMA box copies (x, b and the
    // IB force); the others (the periodic wrap) gather element by element
    const bool interior = fi0 >= 4 && fi0 + RR_FX + 4 <= N && fj0 >= 2 && fj0 + RR_FY + 2 <= N;
    const bool bulk = tma && interior;
    if (bulk) {
        if (tid == 0) {
            tma_prefetch_map(&mx);
            tma_prefetch_map(&mb);
            if (act) tma_prefetch_map(&mf);
            mbar_init(&rr_bar, 1);
            fence_mbar_init();
        }
        __syncthreads();
    }
    pdl_entry();
    if (bulk) {
        if (tid == 0) {
            constexpr uint32_t bx = 3 * RR_XH * RR_W * sizeof(T), bb3 = 3 * RR_BH * RR_W * sizeof(T),
                               bf = 2 * RR_BH * RR_W * sizeof(T);
            mbar_expect_tx(&rr_bar, bx + bb3 + (act ? bf : 0u));
            tma_load_3d(sx, &mx, &rr_bar, fi0 - 4, fj0 - 2, 0);
            tma_load_3d(sb, &mb, &rr_bar, fi0 - 4, fj0 - 1, 0);
            if (act) tma_load_3d(sf, &mf, &rr_bar, fi0 - 4, fj0 - 1, 0);
        }
        const bool ok = mbar_wait_bounded(&rr_bar, 0, VK_WAIT_LIMIT);
        if (!__syncthreads_and(ok)) {   // copies never completed: report, let them drain, leave
            if (tid == 0 && g.err) *(volatile int*)g.err = SIB_DEV_ERR_TMA_WAIT;
            mbar_wait_bounded(&rr_bar, 0, VK_WAIT_LIMIT);
            return;
        }
    } else {
        const int rows = act ? NROWS : NXB;
        for (int q = tid; q < rows * RR_W; q += NT) {
            const int r = q / RR_W, cc = q - r * RR_W;
            const T* base;
            int gj;
            T* dst;
            if (r < 3 * RR_XH) {
                const int comp = r / RR_XH;
                base = x + (size_t)comp * n;
                gj = fj0 - 2 + (r - comp * RR_XH);
                dst = sx + r * RR_W;
            } else if (r < NXB) {
                const int rr = r - 3 * RR_XH, comp = rr / RR_BH;
                base = b + (size_t)comp * n;
                gj = fj0 - 1 + (rr - comp * RR_BH);
                dst = sb + rr * RR_W;
            } else {
                const int rr = r - NXB, comp = rr / RR_BH;
                base = g.fib + (size_t)comp * n;
                gj = fj0 - 1 + (rr - comp * RR_BH);
                dst = sf + rr * RR_W;
            }
            dst[cc] = base[(size_t)(gj & m) * N + ((fi0 - 4 + cc) & m)];
        }
        __syncthreads();
    }
    using P2 = typename RRVec<T>::pair;
    const T* U = sx;
    const T* V = sx + RR_XH * RR_W;
    const T* P = sx + 2 * RR_XH * RR_W;
    const T* Bu = sb;
    const T* Bv = sb + RR_BH * RR_W;
    const T* Bp = sb + 2 * RR_BH * RR_W;
    const T* Fu = sf;
    const T* Fv = sf + RR_BH * RR_W;
    // coarse cell (I, J): fine cells 2I, 2I + 1 of rows 2J, 2J + 1 of the tile.  Staged column
    // c0 + k holds fine column 2I - 2 + k (k = 0 .. 5); staged x row 2J + r holds fine row 2J - 2 + r,
    // staged b / f row 2J + r fine row 2J - 1 + r.
    const int c0 = 2 * threadIdx.x + 2, r0 = 2 * threadIdx.y;
    auto pairs = [&](const T* a, int xr, int k0, int np, T* out) {   // np pairs of row xr from column c0 + k0
#pragma unroll
        for (int q = 0; q < np; ++q) {
            const P2 v = *reinterpret_cast<const P2*>(a + xr * RR_W + c0 + k0 + 2 * q);
            out[2 * q] = v.x;
            out[2 * q + 1] = v.y;
        }
    };
    // u residuals at fine columns 2I - 1 + a (k = 1 + a), rows 2J + r: x rows 2J + 2 + r (u rows 1 + r
    // of u[], loaded from staged rows 2J + 1 ..), b and f rows 2J + 1 + r
    T su, sv, sp;
    T du[2][2];   // U(xi + 1) - U(xi) of the p residuals, rows 2J, 2J + 1, columns 2I, 2I + 1
    {
        // u residuals at fine columns 2I - 1 + a (k = 1 + a), row 2J + r, one row at a time: x rows
        // 2J + 1 + r .. 2J + 3 + r (staged rows r0 + 1 + r ..), b and f row 2J + 1 + r
        T ru[2][3];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            T u[3][6], pp[4], bu[4], fu[4];
#pragma unroll
            for (int q = 0; q < 3; ++q) pairs(U, r0 + 1 + r + q, 0, 3, u[q]);
            pairs(P, r0 + 2 + r, 0, 2, pp);
            pairs(Bu, r0 + 1 + r, 0, 2, bu);
            if (act) pairs(Fu, r0 + 1 + r, 0, 2, fu);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const int k = 1 + a;
                T Au = g.a0 * u[1][k] - g.c * ((u[1][k + 1] + u[1][k - 1]) + (u[2][k] + u[0][k])) +
                       (pp[k] - pp[k - 1]) * g.inv_h;
                Au -= g.dt * (act ? fu[k] : T(0));
                ru[r][a] = bu[k] - Au;
            }
#pragma unroll
            for (int a = 0; a < 2; ++a) du[r][a] = u[1][3 + a] - u[1][2 + a];
        }
        // ru[r][a]: fine column 2I - 1 + a
        su = (ru[0][1] + ru[1][1]) + T(0.5) * ((ru[0][2] + ru[1][2]) + (ru[0][0] + ru[1][0]));
    }
    {
        // v residuals at fine columns 2I + a (k = 2 + a), row 2J - 1 + r, one row at a time: x rows
        // 2J + r .. 2J + 2 + r (staged rows r0 + r ..), b and f row 2J + r
        T rv[3][2], dv[2][2];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            T v[3][6], pc[2], pm[2], bv[2], fv[2];
#pragma unroll
            for (int q = 0; q < 3; ++q) pairs(V, r0 + r + q, 0, 3, v[q]);
            pairs(P, r0 + 1 + r, 2, 1, pc);   // P at the v face's row and the row below
            pairs(P, r0 + r, 2, 1, pm);
            pairs(Bv, r0 + r, 2, 1, bv);
            if (act) pairs(Fv, r0 + r, 2, 1, fv);
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const int k = 2 + a;
                T Av = g.a0 * v[1][k] - g.c * ((v[1][k + 1] + v[1][k - 1]) + (v[2][k] + v[0][k])) +
                       (pc[a] - pm[a]) * g.inv_h;
                Av -= g.dt * (act ? fv[a] : T(0));
                rv[r][a] = bv[a] - Av;
            }
            // V(xi, xj + 1) - V(xi, xj) of the p residual of row 2J - 2 + r (rows 2J and 2J + 1)
            if (r >= 1) {
#pragma unroll
                for (int a = 0; a < 2; ++a) dv[r - 1][a] = v[2][2 + a] - v[1][2 + a];
            }
        }
        // rv[r][a]: fine row 2J - 1 + r, column 2I + a
        sv = (rv[1][0] + rv[1][1]) + T(0.5) * ((rv[2][0] + rv[2][1]) + (rv[0][0] + rv[0][1]));
        T rp[2][2];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            T bp[2];
            pairs(Bp, r0 + 1 + r, 2, 1, bp);
#pragma unroll
            for (int a = 0; a < 2; ++a) rp[r][a] = bp[a] + (du[r][a] + dv[r][a]) * g.inv_h;
        }
        sp = (rp[0][0] + rp[0][1]) + (rp[1][0] + rp[1][1]);
    }
    const int I = blockIdx.x * RR_CX + threadIdx.x, J = blockIdx.y * RR_CY + threadIdx.y;
    const int nc = Nc * Nc, c = J * Nc + I;
    bc[c] = T(0.25) * su;
    bc[nc + c] = T(0.25) * sv;
    bc[2 * nc + c] = T(0.25) * sp;
}

template <typename T>
void launch_residual_restrict(const GridK<T>& g, const T* x, const T* b, T* bc, cudaStream_t s) {
    const int Nc = g.N / 2;
    if (Nc >= RR_CX && g.tx == TX && g.ty == TY) {   // fine tiles of 32 x 8: two by two per block
        const size_t smem = sizeof(T) * (size_t)RR_WORDS + 128;   // 128: room to align the staged tile
        static thread_local bool enabled = false;
        if (!enabled) {
            cudaFuncSetAttribute(k_residual_restrict_tiled<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            enabled = true;
        }
        CUtensorMap mx, mb, mf;
        std::memset(&mx, 0, sizeof(mx));
        std::memset(&mb, 0, sizeof(mb));
        std::memset(&mf, 0, sizeof(mf));
        // interior tiles exist from N = 4 RR_FX on (a tile's staged columns reach 4 beyond it on each side);
        // the maps are only read by those tiles, the IB force's only where a tile is IB-active
        const int es = (int)sizeof(T);
        const int tma = g.N >= 4 * RR_FX && field_map(&mx, x, g.N, es, RR_XH, RR_W, 3) &&
                        field_map(&mb, b, g.N, es, RR_BH, RR_W, 3) &&
                        (!g.tile || !g.fib || field_map(&mf, g.fib, g.N, es, RR_BH, RR_W, 2));
        launch_pdl(k_residual_restrict_tiled<T>, dim3(Nc / RR_CX, Nc / RR_CY), dim3(RR_CX, RR_CY), smem, s, g, mx, mb,
                   mf, tma, x, b, bc);
        return;
    }
    dim3 blk(Nc < 32 ? Nc : 32, Nc < 8 ? Nc : 8);
    dim3 grd((Nc + blk.x - 1) / blk.x, (Nc + blk.y - 1) / blk.y);
    launch_pdl(k_residual_restrict<T>, grd, blk, 0, s, g, x, b, bc);
}

// ------------------------------------------------------------------------------------------
// Restriction of a fine residual to the coarse right-hand side (Sec. 3.2):
//   velocity R_u = P_u^T / 4 (the h^2-weighted adjoint of RT0 prolongation): a coarse x-face
//   takes 1/4 of the two coincident fine faces plus 1/8 of the four fine faces half a coarse
//   cell away in x; pressure: average of the four fine cells.
template <typename T>
__global__ void k_restrict(int Nc, const T* __restrict__ rf, T* __restrict__ bc) {
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
    bc[c] = T(0.25) * su;
    bc[nc + c] = T(0.25) * sv;
    bc[2 * nc + c] = T(0.25) * sp;
}

template <typename T>
void launch_restrict(int Nc, const T* rf, T* bc, cudaStream_t s) {
    dim3 blk(Nc < 32 ? Nc : 32, Nc < 8 ? Nc : 8);
    dim3 grd((Nc + blk.x - 1) / blk.x, (Nc + blk.y - 1) / blk.y);
    launch_pdl(k_restrict<T>, grd, blk, 0, s, Nc, rf, bc);
}

// Prolongation and correction xf += P ec (Sec. 3.2): RT0 for velocity (fine faces that coincide
// with coarse faces copy, faces half-way between two coarse faces average them, constant in the
// tangential direction), bilinear cell-centred interpolation for pressure (9/16, 3/16, 3/16, 1/16).
template <typename T>
__global__ void k_prolong_add(int Nc, const T* __restrict__ ec, T* __restrict__ xf) {
    pdl_entry();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= 2 * Nc || j >= 2 * Nc) return;
    prolong_add_cell(Nc, ec, xf, i, j);
}

// The same correction with one thread per coarse cell (I, J) updating its 2 x 2 fine cells: the
// coarse neighbourhood is read once, and each fine row pair (2I, 2I + 1) is read and written as one
// two-word vector.  Each fine value is formed exactly as in prolong_add_cell.
template <typename T>
struct Vec2;
template <>
struct Vec2<float> {
    using type = float2;
};
template <>
struct Vec2<double> {
    using type = double2;
};
template <typename T>
__global__ void __launch_bounds__(256) k_prolong_add_quad(int Nc, const T* __restrict__ ec, T* __restrict__ xf) {
    using V2 = typename Vec2<T>::type;
    pdl_entry();
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    if (I >= Nc || J >= Nc) return;
    const int Nf = 2 * Nc, nf = Nf * Nf, nc = Nc * Nc, mc = Nc - 1;
    const int Ip = (I + 1) & mc, Im = (I - 1) & mc, Jp = (J + 1) & mc, Jm = (J - 1) & mc;
    const T* eu = ec;
    const T* ev = ec + nc;
    const T* ep = ec + 2 * nc;
    const T u0 = eu[J * Nc + I], u1 = T(0.5) * (eu[J * Nc + I] + eu[J * Nc + Ip]);
    const T v0 = ev[J * Nc + I], v1 = T(0.5) * (ev[J * Nc + I] + ev[Jp * Nc + I]);
    const T pc = ep[J * Nc + I];
    const T pW = ep[J * Nc + Im], pE = ep[J * Nc + Ip], pS = ep[Jm * Nc + I], pN = ep[Jp * Nc + I];
    const T pSW = ep[Jm * Nc + Im], pSE = ep[Jm * Nc + Ip], pNW = ep[Jp * Nc + Im], pNE = ep[Jp * Nc + Ip];
    // fine (2I, 2J) uses neighbours I-1, J-1; (2I+1, 2J): I+1, J-1; (2I, 2J+1): I-1, J+1; (2I+1, 2J+1): I+1, J+1
    const T p00 = T(9.0 / 16.0) * pc + T(3.0 / 16.0) * (pW + pS) + T(1.0 / 16.0) * pSW;
    const T p10 = T(9.0 / 16.0) * pc + T(3.0 / 16.0) * (pE + pS) + T(1.0 / 16.0) * pSE;
    const T p01 = T(9.0 / 16.0) * pc + T(3.0 / 16.0) * (pW + pN) + T(1.0 / 16.0) * pNW;
    const T p11 = T(9.0 / 16.0) * pc + T(3.0 / 16.0) * (pE + pN) + T(1.0 / 16.0) * pNE;
    const int r0 = (2 * J) * Nf + 2 * I, r1 = r0 + Nf;
    V2* xu0 = reinterpret_cast<V2*>(xf + r0);
    V2* xu1 = reinterpret_cast<V2*>(xf + r1);
    V2* xv0 = reinterpret_cast<V2*>(xf + nf + r0);
    V2* xv1 = reinterpret_cast<V2*>(xf + nf + r1);
    V2* xp0 = reinterpret_cast<V2*>(xf + 2 * nf + r0);
    V2* xp1 = reinterpret_cast<V2*>(xf + 2 * nf + r1);
    V2 a = *xu0, b = *xu1, c = *xv0, d = *xv1, e = *xp0, f = *xp1;
    a.x += u0;
    a.y += u1;
    b.x += u0;
    b.y += u1;
    c.x += v0;
    c.y += v0;
    d.x += v1;
    d.y += v1;
    e.x += p00;
    e.y += p10;
    f.x += p01;
    f.y += p11;
    *xu0 = a;
    *xu1 = b;
    *xv0 = c;
    *xv1 = d;
    *xp0 = e;
    *xp1 = f;
}

template <typename T>
void launch_prolong_add(int Nc, const T* ec, T* xf, cudaStream_t s) {
    // the two-word accesses need xf aligned to two elements (a caller's pointer may be offset by one)
    if (Nc >= 8 && (reinterpret_cast<uintptr_t>(xf) % (2 * sizeof(T))) == 0) {
        dim3 blk(Nc < 32 ? Nc : 32, 8);
        dim3 grd((Nc + blk.x - 1) / blk.x, (Nc + blk.y - 1) / blk.y);
        launch_pdl(k_prolong_add_quad<T>, grd, blk, 0, s, Nc, ec, xf);
        return;
    }
    const int Nf = 2 * Nc;
    dim3 blk(Nf < 32 ? Nf : 32, Nf < 8 ? Nf : 8);
    dim3 grd((Nf + blk.x - 1) / blk.x, (Nf + blk.y - 1) / blk.y);
    launch_pdl(k_prolong_add<T>, grd, blk, 0, s, Nc, ec, xf);
}

// ------------------------------------------------------------------------------------------
template <typename Ti, typename To>
__global__ void k_convert(const Ti* __restrict__ in, To* __restrict__ out, int64_t n) {
    pdl_entry();
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        out[k] = static_cast<To>(in[k]);
}

int num_blocks_for(int64_t n) {
    int64_t b = (n + 255) / 256;
    const int64_t cap = 152 * 16;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

template <typename Ti, typename To>
void launch_convert(const Ti* in, To* out, int64_t n, cudaStream_t s) {
    launch_pdl(k_convert<Ti, To>, num_blocks_for(n), 256, 0, s, in, out, n);
}

template <typename T>
__global__ void k_axpby(T a, const T* __restrict__ x, T b, const T* __restrict__ y, T* __restrict__ z, int64_t n) {
    pdl_entry();
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        z[k] = a * x[k] + (y ? b * y[k] : T(0));
}

template <typename T>
void launch_axpby(T a, const T* x, T b, const T* y, T* z, int64_t n, cudaStream_t s) {
    launch_pdl(k_axpby<T>, num_blocks_for(n), 256, 0, s, a, x, b, y, z, n);
}

// ------------------------------------------------------------------------------------------
// Schur-complement smoother pieces (Eq. approx-fact-Stokes-IB).
// z = scale * diag(A_IB)^{-1} r on both velocity components
template <typename T>
__global__ void k_jacobi_A(GridK<T> g, const T* __restrict__ r, T* __restrict__ z, T scale) {
    pdl_entry();
    const int N = g.N, n = N * N;
    const int i = blockIdx.x * g.tx + threadIdx.x, j = blockIdx.y * g.ty + threadIdx.y;
    const bool act = g.tile != nullptr && g.tile[blockIdx.y * g.ntx + blockIdx.x];
    const int c = j * N + i;
    z[c] = scale * r[c] / diagA(g, act, 0, c, n);
    z[n + c] = scale * r[n + c] / diagA(g, act, 1, c, n);
}
template <typename T>
void launch_sc_jacobi_A(const GridK<T>& g, const T* r, T* z, T scale, cudaStream_t s) {
    launch_pdl(k_jacobi_A<T>, dim3(g.N / g.tx, g.N / g.ty), dim3(g.tx, g.ty), 0, s, g, r, z, scale);
}

// y = A_IB u = A u - dt [SKJ] u on the velocity faces (fib holds [SKJ] u)
template <typename T>
__global__ void k_apply_AIB(GridK<T> g, const T* __restrict__ x, T* __restrict__ y) {
    pdl_entry();
    const int N = g.N, n = N * N, m = N - 1;
    const int i = blockIdx.x * g.tx + threadIdx.x, j = blockIdx.y * g.ty + threadIdx.y;
    const int ip = (i + 1) & m, im = (i - 1) & m, jp = (j + 1) & m, jm = (j - 1) & m;
    const int c = j * N + i;
    for (int comp = 0; comp < 2; ++comp) {
        const T* u = x + comp * n;
        T a = g.a0 * u[c] - g.c * ((u[j * N + ip] + u[j * N + im]) + (u[jp * N + i] + u[jm * N + i]));
        a -= g.dt * ibf(g, x, comp, i, j);
        y[comp * n + c] = a;
    }
}
template <typename T>
void launch_apply_AIB(const GridK<T>& g, const T* u, T* y, cudaStream_t s) {
    launch_pdl(k_apply_AIB<T>, dim3(g.N / g.tx, g.N / g.ty), dim3(g.tx, g.ty), 0, s, g, u, y);
}

// gu = G p on the velocity faces
template <typename T>
__global__ void k_gradient(GridK<T> g, const T* __restrict__ p, T* __restrict__ gu) {
    pdl_entry();
    const int N = g.N, n = N * N, m = N - 1;
    const int i = blockIdx.x * g.tx + threadIdx.x, j = blockIdx.y * g.ty + threadIdx.y;
    const int c = j * N + i;
    const T pc = p[c];
    gu[c] = (pc - p[j * N + ((i - 1) & m)]) * g.inv_h;
    gu[n + c] = (pc - p[((j - 1) & m) * N + i]) * g.inv_h;
}
template <typename T>
void launch_gradient(const GridK<T>& g, const T* p, T* gu, cudaStream_t s) {
    launch_pdl(k_gradient<T>, dim3(g.N / g.tx, g.N / g.ty), dim3(g.tx, g.ty), 0, s, g, p, gu);
}

// d = D u on the cells
template <typename T>
__global__ void k_divergence(GridK<T> g, const T* __restrict__ u, T* __restrict__ d) {
    pdl_entry();
    const int N = g.N, n = N * N, m = N - 1;
    const int i = blockIdx.x * g.tx + threadIdx.x, j = blockIdx.y * g.ty + threadIdx.y;
    const int c = j * N + i;
    d[c] = ((u[j * N + ((i + 1) & m)] - u[c]) + (u[n + ((j + 1) & m) * N + i] - u[n + c])) * g.inv_h;
}
template <typename T>
void launch_divergence(const GridK<T>& g, const T* u, T* d, cudaStream_t s) {
    launch_pdl(k_divergence<T>, dim3(g.N / g.tx, g.N / g.ty), dim3(g.tx, g.ty), 0, s, g, u, d);
}

// z = scale * diag(Mh)^{-1} r with Mh = D diag(A_IB)^{-1} G:
//   diag(Mh)_ij = -(1/h^2) (1/dA(u_ij) + 1/dA(u_i+1,j) + 1/dA(v_ij) + 1/dA(v_i,j+1))
// (the four neighbouring faces may belong to a neighbouring tile; the tile flags are dilated by
// one tile, so the flag of the cell's own tile covers them).
template <typename T>
__global__ void k_jacobi_M(GridK<T> g, const T* __restrict__ r, T* __restrict__ z, T scale) {
    pdl_entry();
    const int N = g.N, n = N * N, m = N - 1;
    const int i = blockIdx.x * g.tx + threadIdx.x, j = blockIdx.y * g.ty + threadIdx.y;
    const bool act = g.tile != nullptr && g.tile[blockIdx.y * g.ntx + blockIdx.x];
    const int c = j * N + i, ce = j * N + ((i + 1) & m), cn = ((j + 1) & m) * N + i;
    const T s = T(1) / diagA(g, act, 0, c, n) + T(1) / diagA(g, act, 0, ce, n) + T(1) / diagA(g, act, 1, c, n) +
                T(1) / diagA(g, act, 1, cn, n);
    const T dM = -s * g.inv_h * g.inv_h;
    z[c] = scale * r[c] / dM;
}
template <typename T>
void launch_jacobi_M(const GridK<T>& g, const T* r, T* z, T scale, cudaStream_t s) {
    launch_pdl(k_jacobi_M<T>, dim3(g.N / g.tx, g.N / g.ty), dim3(g.tx, g.ty), 0, s, g, r, z, scale);
}

// ------------------------------------------------------------------------------------------
// Symmetric multicolour Gauss-Seidel preconditioners of the SC smoother's Chebyshev iterations
// (Sec. 3.3, SC smoothing: Gauss-Seidel on A_IB and on Mh = D diag(A_IB)^{-1} G).  The dofs are
// coloured red-black by (i + j) mod 2 (u and v faces alike, and the cells of Mh), which separates
// every pair of unknowns coupled by the five-point stencils.  One pass updates one colour,
//   z_c <- z_c + (scale q - Op z)_c / diag_c,
// with Op z from the iterate at the start of the pass (for A_IB the IB term comes from g.fib,
// computed by an IB pass over that iterate: the IB couplings also link faces of one colour).  A
// sweep from zero runs passes 0, 1, 1, 0; the first pass writes every entry (colour 1 gets 0).
// Diagonal inverses come from g.dinv (faces: 1/diag(A_IB), cells: 1/diag(Mh)).
template <typename T>
__global__ void k_sgs_A_first(GridK<T> g, T scale, const T* __restrict__ q, T* __restrict__ z) {
    pdl_entry();
    const int N = g.N, n = N * N;
    const int i = blockIdx.x * g.tx + threadIdx.x, j = blockIdx.y * g.ty + threadIdx.y;
    const int c = j * N + i;
    const bool red = ((i + j) & 1) == 0;
    z[c] = red ? scale * q[c] * g.dinv[c] : T(0);
    z[n + c] = red ? scale * q[n + c] * g.dinv[n + c] : T(0);
}
// one pass over colour `colour`: thread (k, j) takes cell i = 2 k + ((j + colour) & 1) of row j
template <typename T>
__global__ void k_sgs_A_pass(GridK<T> g, int colour, T scale, const T* __restrict__ q, T* __restrict__ z) {
    pdl_entry();
    const int N = g.N, n = N * N;
    const int k = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (2 * k >= N || j >= N) return;
    const int i = 2 * k + ((j + colour) & 1);
    const int c = j * N + i;
    const T ru = scale * q[c] - Aib(g, z, 0, i, j);
    const T rv = scale * q[n + c] - Aib(g, z, 1, i, j);
    z[c] += ru * g.dinv[c];
    z[n + c] += rv * g.dinv[n + c];
}

// (Mh z) at cell (i, j): (1/h^2) sum over its faces f of a_f (z across f - z_ij), a = 1/diag(A_IB)
template <typename T>
__device__ __forceinline__ T mhat_cell(const GridK<T>& g, const T* __restrict__ z, int i, int j) {
    const int N = g.N, n = N * N, m = N - 1;
    const int ip = (i + 1) & m, im = (i - 1) & m, jp = (j + 1) & m, jm = (j - 1) & m;
    const int c = j * N + i;
    const T zc = z[c];
    const T fx = g.dinv[j * N + ip] * (z[j * N + ip] - zc) - g.dinv[c] * (zc - z[j * N + im]);
    const T fy = g.dinv[n + jp * N + i] * (z[jp * N + i] - zc) - g.dinv[n + c] * (zc - z[jm * N + i]);
    return (fx + fy) * g.inv_h * g.inv_h;
}
template <typename T>
__global__ void k_sgs_M_first(GridK<T> g, T scale, const T* __restrict__ q, T* __restrict__ z) {
    pdl_entry();
    const int N = g.N, n = N * N;
    const int i = blockIdx.x * g.tx + threadIdx.x, j = blockIdx.y * g.ty + threadIdx.y;
    const int c = j * N + i;
    z[c] = ((i + j) & 1) == 0 ? scale * q[c] * g.dinv[2 * n + c] : T(0);
}
template <typename T>
__global__ void k_sgs_M_pass(GridK<T> g, int colour, T scale, const T* __restrict__ q, T* __restrict__ z) {
    pdl_entry();
    const int N = g.N, n = N * N;
    const int k = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (2 * k >= N || j >= N) return;
    const int i = 2 * k + ((j + colour) & 1);
    const int c = j * N + i;
    z[c] += (scale * q[c] - mhat_cell(g, z, i, j)) * g.dinv[2 * n + c];
}

template <typename T>
void launch_sgs_pass(const GridK<T>& g, bool cells, int pass, T scale, const T* q, T* z, cudaStream_t s) {
    if (pass < 0) {   // the first pass of a sweep from zero
        const dim3 grd(g.N / g.tx, g.N / g.ty), blk(g.tx, g.ty);
        if (cells)
            launch_pdl(k_sgs_M_first<T>, grd, blk, 0, s, g, scale, q, z);
        else
            launch_pdl(k_sgs_A_first<T>, grd, blk, 0, s, g, scale, q, z);
        return;
    }
    const int half = g.N / 2;
    const dim3 blk(half < 32 ? half : 32, g.N < 8 ? g.N : 8);
    const dim3 grd((half + blk.x - 1) / blk.x, (g.N + blk.y - 1) / blk.y);
    if (cells)
        launch_pdl(k_sgs_M_pass<T>, grd, blk, 0, s, g, pass, scale, q, z);
    else
        launch_pdl(k_sgs_A_pass<T>, grd, blk, 0, s, g, pass, scale, q, z);
}

// Chebyshev direction update d = ra * d + rb * dinvr, then x += d
template <typename T>
__global__ void k_cheb_update(const T* __restrict__ dinvr, T* __restrict__ d, T* __restrict__ x, T ra, T rb,
                              int64_t n) {
    pdl_entry();
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const T dn = ra * d[k] + rb * dinvr[k];
        d[k] = dn;
        x[k] += dn;
    }
}
template <typename T>
void launch_cheb_update(const T* dinvr, T* d, T* x, T ra, T rb, int64_t n, cudaStream_t s) {
    launch_pdl(k_cheb_update<T>, num_blocks_for(n), 256, 0, s, dinvr, d, x, ra, rb, n);
}

// ------------------------------------------------------------------------------------------
// Schur-complement sweep with two Chebyshev iterations in each inner solve, fused into six
// kernels (Eq. approx-fact-Stokes-IB):
//   r = b - L x;  y = At^{-1} r_u;  s = r_p + D y;  dp = Mt^{-1} s;  yy = At^{-1} G dp;
//   xo = x + omega (y - yy, dp)
// with At^{-1} q = (1 + c1) d0 + c2 DA^{-1}(q - A_IB d0), d0 = DA^{-1} q / theta_A, and
// Mt^{-1} s = (1 + c1) e0 + c2 DM^{-1}(s - D At^{-1} G e0), e0 = DM^{-1} s / theta_M, where DA is
// diag(A_IB) and DM = diag(D DA^{-1} G).  A kernel that needs G of a cell-centred quantity
// recomputes that quantity on the two neighbouring cells instead of synchronising.
// The SC stage kernels read their set-up values (tile flag, diagonal inverses) before waiting for
// the stage's inputs.
template <typename T>
__global__ void __launch_bounds__(256) k_sc_start(GridK<T> g, Cheb2<T> ka, const T* __restrict__ x,
                                                  const T* __restrict__ b, T* __restrict__ r, T* __restrict__ d) {
    const int i = blockIdx.x * g.tx + threadIdx.x, j = blockIdx.y * g.ty + threadIdx.y;
    const ScPre<T> p = sc_pre<T, false>(g, i, j);
    pdl_entry();
    sc_start_cell(g, ka, x, b, r, d, i, j, p);
}

template <typename T>
__global__ void __launch_bounds__(256) k_sc_chebA(GridK<T> g, Cheb2<T> ka, const T* __restrict__ q,
                                                  const T* __restrict__ d, T* __restrict__ y) {
    const int i = blockIdx.x * g.tx + threadIdx.x, j = blockIdx.y * g.ty + threadIdx.y;
    const ScPre<T> p = sc_pre<T, false>(g, i, j);
    pdl_entry();
    sc_chebA_cell(g, ka, q, d, y, i, j, p);
}

template <typename T>
__global__ void __launch_bounds__(256) k_sc_mstart(GridK<T> g, Cheb2<T> ka, Cheb2<T> km, const T* __restrict__ rp,
                                                   const T* __restrict__ y, T* __restrict__ sv, T* __restrict__ dMo,
                                                   T* __restrict__ gq, T* __restrict__ dA) {
    const int i = blockIdx.x * g.tx + threadIdx.x, j = blockIdx.y * g.ty + threadIdx.y;
    const ScPre<T> p = sc_pre<T, true>(g, i, j);
    pdl_entry();
    sc_mstart_cell(g, ka, km, rp, y, sv, dMo, gq, dA, i, j, p);
}

template <typename T>
__global__ void __launch_bounds__(256) k_sc_mfinish(GridK<T> g, Cheb2<T> ka, Cheb2<T> km, const T* __restrict__ sv,
                                                    const T* __restrict__ dM, const T* __restrict__ ya,
                                                    T* __restrict__ dp, T* __restrict__ gq, T* __restrict__ dA) {
    const int i = blockIdx.x * g.tx + threadIdx.x, j = blockIdx.y * g.ty + threadIdx.y;
    const ScPre<T> p = sc_pre<T, true>(g, i, j);
    pdl_entry();
    sc_mfinish_cell(g, ka, km, sv, dM, ya, dp, gq, dA, i, j, p);
}

template <typename T>
__global__ void __launch_bounds__(256) k_sc_finish(GridK<T> g, Cheb2<T> ka, const T* __restrict__ x,
                                                   const T* __restrict__ y, const T* __restrict__ gq,
                                                   const T* __restrict__ dA, const T* __restrict__ dp,
                                                   T* __restrict__ xo) {
    const int i = blockIdx.x * g.tx + threadIdx.x, j = blockIdx.y * g.ty + threadIdx.y;
    const ScPre<T> p = sc_pre<T, false>(g, i, j);
    pdl_entry();
    sc_finish_cell(g, ka, x, y, gq, dA, dp, xo, i, j, p);
}

// power iterations: w = DA^{-1} A_IB v; gq = G v, dA = DA^{-1} gq / theta_A; w = DM^{-1} D ya
template <typename T>
__global__ void k_power_A(GridK<T> g, const T* __restrict__ v, T* __restrict__ w) {
    pdl_entry();
    const int N = g.N, n = N * N;
    const int i = blockIdx.x * g.tx + threadIdx.x, j = blockIdx.y * g.ty + threadIdx.y;
    const int c = j * N + i;
    for (int comp = 0; comp < 2; ++comp) w[comp * n + c] = Aib(g, v, comp, i, j) * g.dinv[comp * n + c];
}
template <typename T>
__global__ void k_power_Mstart(GridK<T> g, Cheb2<T> ka, const T* __restrict__ v, T* __restrict__ gq,
                               T* __restrict__ dA) {
    pdl_entry();
    const int N = g.N, n = N * N, m = N - 1;
    const int i = blockIdx.x * g.tx + threadIdx.x, j = blockIdx.y * g.ty + threadIdx.y;
    const int c = j * N + i;
    const T gu = (v[c] - v[j * N + ((i - 1) & m)]) * g.inv_h, gv = (v[c] - v[((j - 1) & m) * N + i]) * g.inv_h;
    gq[c] = gu;
    gq[n + c] = gv;
    dA[c] = ka.inv_theta * gu * g.dinv[c];
    dA[n + c] = ka.inv_theta * gv * g.dinv[n + c];
}
template <typename T>
__global__ void k_power_Mfinish(GridK<T> g, const T* __restrict__ ya, T* __restrict__ w) {
    pdl_entry();
    const int N = g.N;
    const int i = blockIdx.x * g.tx + threadIdx.x, j = blockIdx.y * g.ty + threadIdx.y;
    w[j * N + i] = divg(g, ya, i, j) * g.dinv[2 * N * N + j * N + i];
}

// set-up of the SC diagonals (FP64): 1/diag(A_IB) on both face sets and 1/diag(M^) on cells
__global__ void k_sc_diag(GridK<double> g, double* __restrict__ dinv) {
    pdl_entry();
    const int N = g.N, n = N * N;
    const int i = blockIdx.x * g.tx + threadIdx.x, j = blockIdx.y * g.ty + threadIdx.y;
    const int c = j * N + i;
    dinv[c] = 1.0 / diag_face(g, 0, i, j);
    dinv[n + c] = 1.0 / diag_face(g, 1, i, j);
    dinv[2 * n + c] = dM_inv(g, i, j);
}
void launch_sc_diag(const GridK<double>& g, double* dinv, cudaStream_t s) {
    launch_pdl(k_sc_diag, dim3(g.N / g.tx, g.N / g.ty), dim3(g.tx, g.ty), 0, s, g, dinv);
}

// Vanka patch factors of every cell (read by patch_solve): the 2 x 2 velocity blocks of the patch,
// A_u = [[a0 - dt B(uL,uL), -c - dt B(uL,uR)], [., a0 - dt B(uR,uR)]] and A_v likewise (B from the
// patch entries, zero outside IB-active tiles), inverted in closed form, and 1 / S with
// S = g^T A_u^{-1} g + g^T A_v^{-1} g, g = (1/h, -1/h).
__global__ void k_patch_factors(GridK<double> g, double* __restrict__ pf) {
    pdl_entry();
    const int N = g.N, n = N * N, m = N - 1;
    const int i = blockIdx.x * g.tx + threadIdx.x, j = blockIdx.y * g.ty + threadIdx.y;
    const int c = j * N + i, ce = j * N + ((i + 1) & m), cn = ((j + 1) & m) * N + i;
    const double au00 = g.a0 - g.dt * g.ibd[c], au11 = g.a0 - g.dt * g.ibd[ce], au01 = -g.c - g.dt * g.ibd[n + c];
    const double av00 = g.a0 - g.dt * g.ibd[2 * n + c], av11 = g.a0 - g.dt * g.ibd[2 * n + cn],
                 av01 = -g.c - g.dt * g.ibd[3 * n + c];
    const double idu = 1.0 / (au00 * au11 - au01 * au01), idv = 1.0 / (av00 * av11 - av01 * av01);
    const double a00u = au11 * idu, a01u = -au01 * idu, a11u = au00 * idu;
    const double a00v = av11 * idv, a01v = -av01 * idv, a11v = av00 * idv;
    const double ih = g.inv_h;
    const double S = ih * ih * ((a00u - 2.0 * a01u + a11u) + (a00v - 2.0 * a01v + a11v));
    pf[c] = a00u;
    pf[n + c] = a01u;
    pf[2 * n + c] = a11u;
    pf[3 * n + c] = a00v;
    pf[4 * n + c] = a01v;
    pf[5 * n + c] = a11v;
    pf[6 * n + c] = 1.0 / S;
}
void launch_patch_factors(const GridK<double>& g, double* pf, cudaStream_t s) {
    launch_pdl(k_patch_factors, dim3(g.N / g.tx, g.N / g.ty), dim3(g.tx, g.ty), 0, s, g, pf);
}

#define SIB_GRID_LAUNCH(kern, ...) launch_pdl(kern<T>, dim3(g.N / g.tx, g.N / g.ty), dim3(g.tx, g.ty), 0, s, __VA_ARGS__)
template <typename T>
void launch_sc_start(const GridK<T>& g, Cheb2<T> ka, const T* x, const T* b, T* r, T* d, cudaStream_t s) {
    SIB_GRID_LAUNCH(k_sc_start, g, ka, x, b, r, d);
}
template <typename T>
void launch_sc_chebA(const GridK<T>& g, Cheb2<T> ka, const T* q, const T* d, T* y, cudaStream_t s) {
    SIB_GRID_LAUNCH(k_sc_chebA, g, ka, q, d, y);
}
template <typename T>
void launch_sc_mstart(const GridK<T>& g, Cheb2<T> ka, Cheb2<T> km, const T* rp, const T* y, T* sv, T* dM, T* gq, T* dA,
                      cudaStream_t s) {
    SIB_GRID_LAUNCH(k_sc_mstart, g, ka, km, rp, y, sv, dM, gq, dA);
}
template <typename T>
void launch_sc_mfinish(const GridK<T>& g, Cheb2<T> ka, Cheb2<T> km, const T* sv, const T* dM, const T* ya, T* dp,
                       T* gq, T* dA, cudaStream_t s) {
    SIB_GRID_LAUNCH(k_sc_mfinish, g, ka, km, sv, dM, ya, dp, gq, dA);
}
template <typename T>
void launch_sc_finish(const GridK<T>& g, Cheb2<T> ka, const T* x, const T* y, const T* gq, const T* dA, const T* dp,
                      T* xo, cudaStream_t s) {
    SIB_GRID_LAUNCH(k_sc_finish, g, ka, x, y, gq, dA, dp, xo);
}
template <typename T>
void launch_power_A(const GridK<T>& g, const T* v, T* w, cudaStream_t s) {
    SIB_GRID_LAUNCH(k_power_A, g, v, w);
}
template <typename T>
void launch_power_Mstart(const GridK<T>& g, Cheb2<T> ka, const T* v, T* gq, T* dA, cudaStream_t s) {
    SIB_GRID_LAUNCH(k_power_Mstart, g, ka, v, gq, dA);
}
template <typename T>
void launch_power_Mfinish(const GridK<T>& g, const T* ya, T* w, cudaStream_t s) {
    SIB_GRID_LAUNCH(k_power_Mfinish, g, ya, w);
}

// ------------------------------------------------------------------------------------------
#define SIB_INST(T)                                                                                        \
    template void launch_residual<T>(const GridK<T>&, const T*, const T*, T*, cudaStream_t);              \
    template void launch_vanka<T>(const GridK<T>&, const T*, const T*, T*, cudaStream_t);                 \
    template void launch_restrict<T>(int, const T*, T*, cudaStream_t);                                    \
    template void launch_prolong_add<T>(int, const T*, T*, cudaStream_t);                                 \
    template void launch_axpby<T>(T, const T*, T, const T*, T*, int64_t, cudaStream_t);                   \
    template void launch_sc_jacobi_A<T>(const GridK<T>&, const T*, T*, T, cudaStream_t);                  \
    template void launch_apply_AIB<T>(const GridK<T>&, const T*, T*, cudaStream_t);                       \
    template void launch_gradient<T>(const GridK<T>&, const T*, T*, cudaStream_t);                        \
    template void launch_divergence<T>(const GridK<T>&, const T*, T*, cudaStream_t);                      \
    template void launch_jacobi_M<T>(const GridK<T>&, const T*, T*, T, cudaStream_t);                     \
    template void launch_sgs_pass<T>(const GridK<T>&, bool, int, T, const T*, T*, cudaStream_t);          \
    template void launch_cheb_update<T>(const T*, T*, T*, T, T, int64_t, cudaStream_t);                   \
    template void launch_vanka_zero<T>(const GridK<T>&, const T*, T*, cudaStream_t);                       \
    template void launch_residual_restrict<T>(const GridK<T>&, const T*, const T*, T*, cudaStream_t);       \
    template void launch_sc_start<T>(const GridK<T>&, Cheb2<T>, const T*, const T*, T*, T*, cudaStream_t);   \
    template void launch_sc_chebA<T>(const GridK<T>&, Cheb2<T>, const T*, const T*, T*, cudaStream_t);       \
    template void launch_sc_mstart<T>(const GridK<T>&, Cheb2<T>, Cheb2<T>, const T*, const T*, T*, T*, T*, T*, \
                                      cudaStream_t);                                                         \
    template void launch_sc_mfinish<T>(const GridK<T>&, Cheb2<T>, Cheb2<T>, const T*, const T*, const T*, T*, \
                                       T*, T*, cudaStream_t);                                                \
    template void launch_sc_finish<T>(const GridK<T>&, Cheb2<T>, const T*, const T*, const T*, const T*,     \
                                      const T*, T*, cudaStream_t);                                           \
    template void launch_power_A<T>(const GridK<T>&, const T*, T*, cudaStream_t);                          \
    template void launch_power_Mstart<T>(const GridK<T>&, Cheb2<T>, const T*, T*, T*, cudaStream_t);       \
    template void launch_power_Mfinish<T>(const GridK<T>&, const T*, T*, cudaStream_t);
SIB_INST(float)
SIB_INST(double)
template void launch_convert<double, float>(const double*, float*, int64_t, cudaStream_t);
template void launch_convert<float, double>(const float*, double*, int64_t, cudaStream_t);
template void launch_convert<double, double>(const double*, double*, int64_t, cudaStream_t);

}  // namespace sib
