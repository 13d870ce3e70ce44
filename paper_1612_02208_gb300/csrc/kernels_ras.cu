// Restricted additive Schwarz smoother over box subdomains (Sec. 3.3, Alg. 2 with b x b boxes and
// overlap o): every box solves its local saddle-point problem on the residual, and each dof takes
// the correction of the box whose core owns it.
//
// Subdomain of box (I, J): the e x e cells from (I b - o, J b - o), e = b + 2o (periodic), with
// all their faces and pressures, in the order
//   u(i0 + ii, j0 + jj), jj < e, ii <= e;   v(i0 + ii, j0 + jj), jj <= e, ii < e;   p, jj < e, ii < e
// (row-major within each); ne = 3 e^2 + 2 e dofs.  Owned dofs: the u, v and p of the core cells
// (o <= ii, jj < o + b), nown = 3 b^2, ordered u, v, p and row-major.
//
// Set-up (FP64): the local operator L_k = R_k L R_k^T is assembled from the stencil (A, G, -D) and the
// IB windows, inverted by Gauss-Jordan with partial pivoting, and the owned rows of the inverse are
// stored (column-major, FP64 and FP32).  Boxes whose subdomain meets no IB window all have the same
// operator (the grid is uniform and periodic): one shared inverse per level serves them.  Subdomains
// up to RAS_EMAX_SMEM cells wide are eliminated in shared memory and corrected by a persistent
// kernel; wider ones (the paper's 8 x 8 boxes with overlap 2 and up) are eliminated in a global
// workspace and corrected by a batched product over tiles of boxes.
#include <algorithm>

#include "sib_internal.h"
#include "tcgen05.cuh"
#include "tma.cuh"

namespace sib {

namespace {

struct RasGeo {
    int N, b, o, e, ne, nown, nbs;   // nbs = N / b boxes per side
};

__host__ __device__ inline RasGeo ras_geo(int N, int b, int o) {
    RasGeo g;
    g.N = N;
    g.b = b;
    g.o = o;
    g.e = b + 2 * o;
    g.ne = 3 * g.e * g.e + 2 * g.e;
    g.nown = 3 * b * b;
    g.nbs = N / b;
    return g;
}

// local dof q -> (component, ii, jj) in box coordinates
__device__ __forceinline__ void ras_dof(const RasGeo& G, int q, int& comp, int& ii, int& jj) {
    const int e = G.e, nu = e * (e + 1);
    if (q < nu) {
        comp = 0;
        jj = q / (e + 1);
        ii = q - jj * (e + 1);
    } else if (q < 2 * nu) {
        comp = 1;
        q -= nu;
        jj = q / e;
        ii = q - jj * e;
    } else {
        comp = 2;
        q -= 2 * nu;
        jj = q / e;
        ii = q - jj * e;
    }
}
// (component, ii, jj) -> local dof, or -1 outside the subdomain
__device__ __forceinline__ int ras_index(const RasGeo& G, int comp, int ii, int jj) {
    const int e = G.e, nu = e * (e + 1);
    if (comp == 0) return (ii >= 0 && ii <= e && jj >= 0 && jj < e) ? jj * (e + 1) + ii : -1;
    if (comp == 1) return (ii >= 0 && ii < e && jj >= 0 && jj <= e) ? nu + jj * e + ii : -1;
    return (ii >= 0 && ii < e && jj >= 0 && jj < e) ? 2 * nu + jj * e + ii : -1;
}
// owned dof r -> local dof
__device__ __forceinline__ int ras_owned(const RasGeo& G, int r) {
    const int bb = G.b * G.b, comp = r / bb, rem = r - comp * bb;
    return ras_index(G, comp, G.o + rem % G.b, G.o + rem / G.b);
}

// window slot of the tile holding face (i, j) of the level (-1: no IB entries in that row)
__device__ __forceinline__ int face_slot(const RasIB& ib, int i, int j) {
    if (!ib.slotOf) return -1;
    return ib.slotOf[(j / ib.ty) * ib.ntx + i / ib.tx];
}

// Box classification: box k is listed if some face of its subdomain has a nonzero row of the IB
// operator (a window entry != 0); the other boxes' local operators have no IB terms.  The list is
// filled through an atomic counter, so its order (and each box's storage slot) can differ between
// set-ups; every listed box's inverse depends only on that box, so the results do not.
__global__ void k_ras_classify(RasGeo G, RasIB ib, int* __restrict__ list, int* __restrict__ count) {
    const int k = blockIdx.x;
    const int I = k % G.nbs, J = k / G.nbs, m = G.N - 1;
    const int i0 = I * G.b - G.o, j0 = J * G.b - G.o;
    const int nu = G.e * (G.e + 1), per = ib.tx * ib.ty;
    int hit = 0;
    for (int t = threadIdx.x; t < 2 * nu * WIN_SIZE && !hit; t += blockDim.x) {
        const int q = t / WIN_SIZE, kw = t - q * WIN_SIZE;   // velocity dof q of the subdomain, window entry kw
        int comp, ii, jj;
        ras_dof(G, q, comp, ii, jj);
        const int gi = (i0 + ii) & m, gj = (j0 + jj) & m;
        const int slot = face_slot(ib, gi, gj);
        if (slot < 0) continue;
        const double* w = ib.win + ((size_t)(slot * 2 + comp) * WIN_SIZE) * per;
        if (w[(size_t)kw * per + (gj % ib.ty) * ib.tx + (gi % ib.tx)] != 0.0) hit = 1;
    }
    hit = __syncthreads_or(hit);
    if (hit && threadIdx.x == 0) list[atomicAdd(count, 1)] = k;
}

// Assembles L_k in shared memory (row-major, ne x ne), inverts it in place and stores the owned rows
// of the inverse.  Block 0 builds the shared IB-free operator (box 0 without IB terms); block s > 0
// builds box list[s - 1] with its IB terms.  info != 0 on a zero pivot.
__global__ void __launch_bounds__(256) k_ras_setup(RasGeo G, RasIB ib, double a0, double c, double inv_h, double dt,
                                                  const int* __restrict__ list, double* __restrict__ inv64,
                                                  float* __restrict__ inv32, int* __restrict__ info) {
    extern __shared__ double smem_ras[];
    const int n = G.ne, tid = threadIdx.x, nt = blockDim.x;
    double* A = smem_ras;                 // n x n
    double* colk = A + n * n;             // n
    double* redv = colk + n;              // 32
    int* redi = reinterpret_cast<int*>(redv + 32);   // 32
    int* perm = redi + 32;                // n
    const bool withIB = blockIdx.x > 0;
    const int k = withIB ? list[blockIdx.x - 1] : 0;
    const int I = k % G.nbs, J = k / G.nbs, m = G.N - 1;
    const int i0 = I * G.b - G.o, j0 = J * G.b - G.o;
    const int per = ib.tx * ib.ty;
    for (int t = tid; t < n * n; t += nt) A[t] = 0.0;
    __syncthreads();
    for (int q = tid; q < n; q += nt) {   // row q of L_k
        int comp, ii, jj;
        ras_dof(G, q, comp, ii, jj);
        double* row = A + (size_t)q * n;
        if (comp < 2) {
            row[q] = a0;
            // couplings to dofs of the subdomain, at local coordinates taken modulo N (on small grids a
            // neighbour or window offset can wrap around onto the far side of the same subdomain; the
            // subdomain itself never wraps onto itself, so the local index is unique)
            const int nb[4][2] = {{ii + 1, jj}, {ii - 1, jj}, {ii, jj + 1}, {ii, jj - 1}};
            for (int s2 = 0; s2 < 4; ++s2) {
                const int col = ras_index(G, comp, nb[s2][0] & m, nb[s2][1] & m);
                if (col >= 0) row[col] -= c;
            }
            // G p: u(i, j) -> (p(i, j) - p(i-1, j)) / h;  v(i, j) -> (p(i, j) - p(i, j-1)) / h
            const int pc = ras_index(G, 2, ii, jj);
            const int pm = comp == 0 ? ras_index(G, 2, ii - 1, jj) : ras_index(G, 2, ii, jj - 1);
            if (pc >= 0) row[pc] += inv_h;
            if (pm >= 0) row[pm] -= inv_h;
            if (withIB) {   // -dt B(f, g) for g of the same component in the subdomain (window offsets)
                const int gi = (i0 + ii) & m, gj = (j0 + jj) & m;
                const int slot = face_slot(ib, gi, gj);
                if (slot >= 0) {
                    const double* w = ib.win + ((size_t)(slot * 2 + comp) * WIN_SIZE) * per;
                    const int qt = (gj % ib.ty) * ib.tx + (gi % ib.tx);
                    for (int dj = -WR; dj <= WR; ++dj)
                        for (int di = -WR; di <= WR; ++di) {
                            const int col = ras_index(G, comp, (ii + di) & m, (jj + dj) & m);
                            if (col >= 0) row[col] -= dt * w[(size_t)((dj + WR) * WD + (di + WR)) * per + qt];
                        }
                }
            }
        } else {   // -D u: -(u(i+1, j) - u(i, j) + v(i, j+1) - v(i, j)) / h
            row[ras_index(G, 0, ii + 1, jj)] -= inv_h;
            row[ras_index(G, 0, ii, jj)] += inv_h;
            row[ras_index(G, 1, ii, jj + 1)] -= inv_h;
            row[ras_index(G, 1, ii, jj)] += inv_h;
        }
    }
    __syncthreads();
    // in-place Gauss-Jordan with partial (row) pivoting: A <- (P A)^{-1}
    const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    for (int kk = 0; kk < n; ++kk) {
        double best = -1.0;
        int bi = kk;
        for (int i = kk + tid; i < n; i += nt) {
            const double v = fabs(A[(size_t)i * n + kk]);
            if (v > best) {
                best = v;
                bi = i;
            }
        }
        for (int off = 16; off > 0; off >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, best, off);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
            if (ov > best || (ov == best && oi < bi)) {
                best = ov;
                bi = oi;
            }
        }
        if (lane == 0) {
            redv[wid] = best;
            redi[wid] = bi;
        }
        __syncthreads();
        if (tid == 0) {
            double bv = redv[0];
            int bx = redi[0];
            for (int w2 = 1; w2 < nw; ++w2)
                if (redv[w2] > bv || (redv[w2] == bv && redi[w2] < bx)) {
                    bv = redv[w2];
                    bx = redi[w2];
                }
            perm[kk] = bx;
            if (!(bv > 0.0)) atomicExch(info, 1);
        }
        __syncthreads();
        const int p = perm[kk];
        if (p != kk)
            for (int j = tid; j < n; j += nt) {
                const double t = A[(size_t)kk * n + j];
                A[(size_t)kk * n + j] = A[(size_t)p * n + j];
                A[(size_t)p * n + j] = t;
            }
        __syncthreads();
        const double piv = A[(size_t)kk * n + kk];
        const double pinv = piv != 0.0 ? 1.0 / piv : 0.0;
        for (int i = tid; i < n; i += nt) colk[i] = A[(size_t)i * n + kk];
        __syncthreads();
        for (int j = tid; j < n; j += nt) A[(size_t)kk * n + j] = (j == kk ? 1.0 : A[(size_t)kk * n + j]) * pinv;
        __syncthreads();
        for (int t = tid; t < n * n; t += nt) {
            const int i = t / n, j = t - i * n;
            if (i == kk) continue;
            A[t] = (j == kk ? 0.0 : A[t]) - colk[i] * A[(size_t)kk * n + j];
        }
        __syncthreads();
    }
    // (P A)^{-1} P = A^{-1}: swap columns back in reverse order of the row interchanges
    for (int kk = n - 1; kk >= 0; --kk) {
        const int p = perm[kk];
        if (p != kk)
            for (int i = tid; i < n; i += nt) {
                const double t = A[(size_t)i * n + kk];
                A[(size_t)i * n + kk] = A[(size_t)i * n + p];
                A[(size_t)i * n + p] = t;
            }
        __syncthreads();
    }
    // owned rows, column-major: out[q * nown + r] = A^{-1}(owned(r), q)
    const size_t base = (size_t)blockIdx.x * n * G.nown;
    for (int t = tid; t < n * G.nown; t += nt) {
        const int q = t / G.nown, r = t - q * G.nown;
        const double v = A[(size_t)ras_owned(G, r) * n + q];
        inv64[base + t] = v;
        inv32[base + t] = (float)v;
    }
}

// One RAS correction: xo(owned) = x(owned) + omega (Inv_k r_k)(owned) for every box k, with r the
// residual (x == nullptr: zero initial guess, xo = omega Inv r).  The boxes without IB terms
// (slotOfBox[k] < 0) share one inverse, staged once per block in shared memory (k_ras_apply); the
// others, listed at set-up, use their own (k_ras_apply_ib, one block per box).
// Every warp takes groups of RAS_GB consecutive boxes (grid-stride over the groups):
// the group's residuals are gathered into shared memory as [q][box], and lane l accumulates owned
// rows l and l + 32 for all boxes of the group, so one read of an inverse entry serves RAS_GB boxes.
constexpr int RAS_GB = 4;
constexpr int RAS_WARPS = 4;
constexpr int RAS_QL = 4;   // subdomain dofs per lane: ne <= 32 RAS_QL (ne <= 120 for b + 2o <= 6)
template <typename T>
struct alignas(4 * sizeof(T)) Quad {
    T v[4];
};
template <typename T>
__global__ void __launch_bounds__(32 * RAS_WARPS) k_ras_apply(RasGeo G, const int* __restrict__ slotOfBox,
                                                              const T* __restrict__ inv, T omega,
                                                              const T* __restrict__ r, const T* x, T* xo) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* Ms = reinterpret_cast<T*>(smem_raw);                                  // ne x nown, [q][row]
    T* rbAll = Ms + ((G.ne * G.nown + 3) & ~3);                              // per warp: ne x RAS_GB
    int* qtab = reinterpret_cast<int*>(rbAll + (size_t)RAS_WARPS * G.ne * RAS_GB);   // ne: comp | ii << 8 | jj << 16
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T* rb = rbAll + (size_t)warp * G.ne * RAS_GB;
    {   // stage the shared inverse (set-up data): 16-byte asynchronous copies, all in flight at once
        const int words = G.ne * G.nown, per16 = 16 / (int)sizeof(T), chunks = words / per16;
        for (int t = threadIdx.x; t < chunks; t += blockDim.x)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((uint32_t)__cvta_generic_to_shared(Ms + t * per16)),
                         "l"(inv + (size_t)t * per16)
                         : "memory");
        for (int t = chunks * per16 + threadIdx.x; t < words; t += blockDim.x) Ms[t] = inv[t];
        asm volatile("cp.async.wait_all;\n" ::: "memory");
    }
    for (int q = threadIdx.x; q < G.ne; q += blockDim.x) {
        int comp, ii, jj;
        ras_dof(G, q, comp, ii, jj);
        qtab[q] = comp | (ii << 8) | (jj << 16);
    }
    __syncthreads();
    pdl_entry();
    const int N = G.N, n = N * N, m = N - 1, bb = G.b * G.b;
    const int ngroups = G.nbs * G.nbs / RAS_GB;
    const int r0 = lane, r1 = lane + 32;
    for (int grp = blockIdx.x * RAS_WARPS + warp; grp < ngroups; grp += gridDim.x * RAS_WARPS) {
        const int k0 = grp * RAS_GB;
        // gather the group's residuals: every load of the lane is issued before the first store
        T gv[RAS_GB][RAS_QL];
#pragma unroll
        for (int j = 0; j < RAS_GB; ++j) {
            const int kb = k0 + j;
            const int ib0 = (kb % G.nbs) * G.b - G.o, jb0 = (kb / G.nbs) * G.b - G.o;
#pragma unroll
            for (int sq = 0; sq < RAS_QL; ++sq) {
                const int q = lane + 32 * sq;
                if (q < G.ne) {
                    const int code = qtab[q];
                    const int gi = (ib0 + ((code >> 8) & 0xff)) & m, gj = (jb0 + (code >> 16)) & m;
                    gv[j][sq] = r[(size_t)(code & 0xff) * n + gj * N + gi];
                }
            }
        }
#pragma unroll
        for (int j = 0; j < RAS_GB; ++j)
#pragma unroll
            for (int sq = 0; sq < RAS_QL; ++sq) {
                const int q = lane + 32 * sq;
                if (q < G.ne) rb[q * RAS_GB + j] = gv[j][sq];
            }
        __syncwarp();
        int sl[RAS_GB];
#pragma unroll
        for (int j = 0; j < RAS_GB; ++j) sl[j] = slotOfBox ? slotOfBox[k0 + j] : -1;
        T acc0[RAS_GB], acc1[RAS_GB];
#pragma unroll
        for (int j = 0; j < RAS_GB; ++j) acc0[j] = acc1[j] = T(0);
        {   // the shared inverse for the whole group (boxes with their own are stored by k_ras_apply_ib)
            const int c0 = r0 < G.nown ? r0 : 0, c1 = r1 < G.nown ? r1 : 0;   // rows past nown compute, unused
            const Quad<T>* rq = reinterpret_cast<const Quad<T>*>(rb);
#pragma unroll 8
            for (int q = 0; q < G.ne; ++q) {
                const T m0 = Ms[q * G.nown + c0];
                const T m1 = Ms[q * G.nown + c1];
                const Quad<T> v = rq[q];
#pragma unroll
                for (int j = 0; j < RAS_GB; ++j) {
                    acc0[j] += m0 * v.v[j];
                    acc1[j] += m1 * v.v[j];
                }
            }
        }
#pragma unroll
        for (int j = 0; j < RAS_GB; ++j) {
            if (sl[j] >= 0) continue;
            const int I = (k0 + j) % G.nbs, J = (k0 + j) / G.nbs;
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
                const int rr = h2 ? r1 : r0;
                if (rr >= G.nown) continue;
                const int comp = rr / bb, rem = rr - comp * bb;
                const int gi = I * G.b + rem % G.b, gj = J * G.b + rem / G.b;
                const size_t d = (size_t)comp * n + gj * N + gi;
                xo[d] = (x ? x[d] : T(0)) + omega * (h2 ? acc1[j] : acc0[j]);
            }
        }
        __syncwarp();   // the group's residual buffer is reused by the next group
    }
}

// One block per listed IB box: RAS_QS groups of threads each take a quarter of the q range for every
// owned row, and the partial sums are added in shared memory in a fixed order.
constexpr int RAS_QS = 4;
template <typename T>
__global__ void __launch_bounds__(64 * RAS_QS) k_ras_apply_ib(RasGeo G, const int* __restrict__ list,
                                                             const T* __restrict__ inv, T omega,
                                                             const T* __restrict__ r, const T* x, T* xo) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* rb = reinterpret_cast<T*>(smem_raw);   // ne
    T* part = rb + G.ne;                      // RAS_QS x 64
    const int s = blockIdx.x, k = list[s];    // set-up data
    pdl_entry();
    const int I = k % G.nbs, J = k / G.nbs, N = G.N, n = N * N, m = N - 1, bb = G.b * G.b;
    const int i0 = I * G.b - G.o, j0 = J * G.b - G.o;
    for (int q = threadIdx.x; q < G.ne; q += blockDim.x) {
        int comp, ii, jj;
        ras_dof(G, q, comp, ii, jj);
        rb[q] = r[(size_t)comp * n + ((j0 + jj) & m) * N + ((i0 + ii) & m)];
    }
    __syncthreads();
    const T* M = inv + (size_t)(s + 1) * G.ne * G.nown;
    const int rr = threadIdx.x & 63, part_id = threadIdx.x >> 6;
    const int qchunk = (G.ne + RAS_QS - 1) / RAS_QS;
    const int qa = part_id * qchunk, qb = min(G.ne, qa + qchunk);
    T acc = T(0);
    if (rr < G.nown) {
#pragma unroll 6
        for (int q = qa; q < qb; ++q) acc += M[(size_t)q * G.nown + rr] * rb[q];
    }
    part[part_id * 64 + rr] = acc;
    __syncthreads();
    if (part_id == 0 && rr < G.nown) {
        T sum = part[rr];
        for (int p2 = 1; p2 < RAS_QS; ++p2) sum += part[p2 * 64 + rr];
        const int comp = rr / bb, rem = rr - comp * bb;
        const size_t d = (size_t)comp * n + (J * G.b + rem / G.b) * N + I * G.b + rem % G.b;
        xo[d] = (x ? x[d] : T(0)) + omega * sum;
    }
}

__global__ void k_box_slots(const int* __restrict__ list, const int* __restrict__ count, int* __restrict__ slotOfBox) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < *count) slotOfBox[list[s]] = s;
}

// ---- subdomains wider than RAS_EMAX_SMEM cells (e <= RAS_EMAX, ne <= 800) ----------------------
// The local operator (up to 5 MB in FP64) no longer fits shared memory.  Each set-up block assembles
// its matrix in a global workspace and eliminates there, with the pivot column and the scaled pivot
// row in shared memory.  The shared-inverse correction becomes one batched product per level,
// C (nown x boxes) = Inv (nown x ne) R (ne x boxes), over tiles of boxes; the IB boxes keep one block
// each.

// Row q of L_k for the subdomain with corner cell (i0, j0), added into `row` (zeroed by the caller):
// the same stencil and window entries as the shared-memory set-up above.
__device__ void ras_assemble_row(const RasGeo& G, const RasIB& ib, double a0, double c, double inv_h, double dt,
                                 bool withIB, int i0, int j0, int q, double* row) {
    const int m = G.N - 1, per = ib.tx * ib.ty;
    int comp, ii, jj;
    ras_dof(G, q, comp, ii, jj);
    if (comp < 2) {
        row[q] = a0;
        const int nb[4][2] = {{ii + 1, jj}, {ii - 1, jj}, {ii, jj + 1}, {ii, jj - 1}};
        for (int s2 = 0; s2 < 4; ++s2) {
            const int col = ras_index(G, comp, nb[s2][0] & m, nb[s2][1] & m);
            if (col >= 0) row[col] -= c;
        }
        const int pc = ras_index(G, 2, ii, jj);
        const int pm = comp == 0 ? ras_index(G, 2, ii - 1, jj) : ras_index(G, 2, ii, jj - 1);
        if (pc >= 0) row[pc] += inv_h;
        if (pm >= 0) row[pm] -= inv_h;
        if (withIB) {
            const int gi = (i0 + ii) & m, gj = (j0 + jj) & m;
            const int slot = face_slot(ib, gi, gj);
            if (slot >= 0) {
                const double* w = ib.win + ((size_t)(slot * 2 + comp) * WIN_SIZE) * per;
                const int qt = (gj % ib.ty) * ib.tx + (gi % ib.tx);
                for (int dj = -WR; dj <= WR; ++dj)
                    for (int di = -WR; di <= WR; ++di) {
                        const int col = ras_index(G, comp, (ii + di) & m, (jj + dj) & m);
                        if (col >= 0) row[col] -= dt * w[(size_t)((dj + WR) * WD + (di + WR)) * per + qt];
                    }
            }
        }
    } else {
        row[ras_index(G, 0, ii + 1, jj)] -= inv_h;
        row[ras_index(G, 0, ii, jj)] += inv_h;
        row[ras_index(G, 1, ii, jj + 1)] -= inv_h;
        row[ras_index(G, 1, ii, jj)] += inv_h;
    }
}

// Block b of a launch inverts matrix first + b (0: the shared IB-free operator; s > 0: the operator
// of box list[s - 1]) in work + b ne^2 by Gauss-Jordan with partial (row) pivoting, then stores the
// owned rows of the inverse column-major at slot first + b, as the shared-memory set-up does.
constexpr int RAS_BIG_SETUP_THREADS = 512;
__global__ void __launch_bounds__(RAS_BIG_SETUP_THREADS)
    k_ras_setup_big(RasGeo G, RasIB ib, double a0, double c, double inv_h, double dt, const int* __restrict__ list,
                    int first, double* __restrict__ work, double* __restrict__ inv64, float* __restrict__ inv32,
                    int* __restrict__ info) {
    extern __shared__ double smem_big[];
    const int n = G.ne, tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    double* colk = smem_big;                          // n: column kk before the step
    double* rowk = colk + n;                          // n: row kk after scaling
    double* redv = rowk + n;                          // 32
    int* redi = reinterpret_cast<int*>(redv + 32);    // 32
    int* perm = redi + 32;                            // n
    const int mi = first + blockIdx.x;
    const bool withIB = mi > 0;
    const int k = withIB ? list[mi - 1] : 0;
    const int I = k % G.nbs, J = k / G.nbs;
    double* A = work + (size_t)blockIdx.x * n * n;
    for (size_t t = tid; t < (size_t)n * n; t += nt) A[t] = 0.0;
    __syncthreads();
    for (int q = tid; q < n; q += nt)   // every thread writes only its own rows
        ras_assemble_row(G, ib, a0, c, inv_h, dt, withIB, I * G.b - G.o, J * G.b - G.o, q, A + (size_t)q * n);
    __syncthreads();
    for (int kk = 0; kk < n; ++kk) {
        double best = -1.0;
        int bi = kk;
        for (int i = kk + tid; i < n; i += nt) {
            const double v = fabs(A[(size_t)i * n + kk]);
            if (v > best) {
                best = v;
                bi = i;
            }
        }
        for (int off = 16; off > 0; off >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, best, off);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
            if (ov > best || (ov == best && oi < bi)) {
                best = ov;
                bi = oi;
            }
        }
        if (lane == 0) {
            redv[wid] = best;
            redi[wid] = bi;
        }
        __syncthreads();
        if (tid == 0) {
            double bv = redv[0];
            int bx = redi[0];
            for (int w2 = 1; w2 < nw; ++w2)
                if (redv[w2] > bv || (redv[w2] == bv && redi[w2] < bx)) {
                    bv = redv[w2];
                    bx = redi[w2];
                }
            perm[kk] = bx;
            if (!(bv > 0.0)) atomicExch(info, 1);
        }
        __syncthreads();
        const int p = perm[kk];
        if (p != kk)
            for (int j = tid; j < n; j += nt) {
                const double t = A[(size_t)kk * n + j];
                A[(size_t)kk * n + j] = A[(size_t)p * n + j];
                A[(size_t)p * n + j] = t;
            }
        __syncthreads();
        const double piv = A[(size_t)kk * n + kk];
        const double pinv = piv != 0.0 ? 1.0 / piv : 0.0;
        for (int i = tid; i < n; i += nt) colk[i] = A[(size_t)i * n + kk];
        __syncthreads();
        for (int j = tid; j < n; j += nt) {
            const double v = (j == kk ? 1.0 : A[(size_t)kk * n + j]) * pinv;
            rowk[j] = v;
            A[(size_t)kk * n + j] = v;
        }
        __syncthreads();
        // rank-one update of the other rows, one warp per row (coalesced); a row with a zero entry in
        // column kk is unchanged (its column-kk entry stays 0), so it is skipped
        for (int i = wid; i < n; i += nw) {
            const double ci = colk[i];
            if (i == kk || ci == 0.0) continue;
            double* Ai = A + (size_t)i * n;
            for (int j = lane; j < n; j += 32) Ai[j] = (j == kk ? 0.0 : Ai[j]) - ci * rowk[j];
        }
        __syncthreads();
    }
    for (int kk = n - 1; kk >= 0; --kk) {   // (P A)^{-1} P = A^{-1}
        const int p = perm[kk];
        if (p != kk)
            for (int i = tid; i < n; i += nt) {
                const double t = A[(size_t)i * n + kk];
                A[(size_t)i * n + kk] = A[(size_t)i * n + p];
                A[(size_t)i * n + p] = t;
            }
        __syncthreads();
    }
    const size_t base = (size_t)mi * n * G.nown;
    for (int t = tid; t < n * G.nown; t += nt) {
        const int q = t / G.nown, r = t - q * G.nown;
        const double v = A[(size_t)ras_owned(G, r) * n + q];
        inv64[base + t] = v;
        inv32[base + t] = (float)v;
    }
}

// Batched shared-inverse correction.  A block takes a tile of RAS_NBX consecutive boxes and all their
// owned rows; the subdomain dofs q are taken in chunks of RAS_KC: the chunk of the inverse (rows
// [q][row], contiguous in memory) is copied to shared memory asynchronously while the chunk of the
// tile's residual windows is gathered, then warp w accumulates the owned rows lane + 32 a (a < RA)
// for its RAS_BPT boxes.  The window chunk is stored [q][box] in 16-byte slots of VW boxes, slot s of
// row q at position s ^ (q & 15): the gather's stores (8 dofs x 4 boxes per warp) and the product's
// 16-byte broadcast loads are both free of bank conflicts.
constexpr int RAS_KC = 32;
constexpr int RAS_BW = 8;   // warps per block
template <typename T>
struct RasTile {
    static constexpr int VW = 16 / (int)sizeof(T);   // boxes per 16-byte slot
    static constexpr int NBX = 16 * VW;              // boxes per tile (16 slots)
    static constexpr int BPT = NBX / RAS_BW;         // boxes per warp (two slots)
};
template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
    using type = float4;
};
template <>
struct Vec16<double> {
    using type = double2;
};
template <typename T>
__device__ __forceinline__ T vget(const typename Vec16<T>::type& v, int c);
template <>
__device__ __forceinline__ float vget<float>(const float4& v, int c) {
    return c == 0 ? v.x : c == 1 ? v.y : c == 2 ? v.z : v.w;
}
template <>
__device__ __forceinline__ double vget<double>(const double2& v, int c) {
    return c == 0 ? v.x : v.y;
}

template <typename T, int RA>
__global__ void __launch_bounds__(32 * RAS_BW) k_ras_apply_big(RasGeo G, const int* __restrict__ slotOfBox,
                                                              const T* __restrict__ inv, T omega,
                                                              const T* __restrict__ r, const T* x, T* xo) {
    using TL = RasTile<T>;
    using V = typename Vec16<T>::type;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* Ms = reinterpret_cast<T*>(smem_raw);                             // RAS_KC x nown, [q][row]
    T* Rc = Ms + (size_t)RAS_KC * G.nown;                               // RAS_KC x NBX, swizzled slots
    int* qtab = reinterpret_cast<int*>(Rc + (size_t)RAS_KC * TL::NBX);  // ne: comp | ii << 8 | jj << 16
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = threadIdx.x; q < G.ne; q += blockDim.x) {
        int comp, ii, jj;
        ras_dof(G, q, comp, ii, jj);
        qtab[q] = comp | (ii << 8) | (jj << 16);
    }
    pdl_entry();
    const int N = G.N, n = N * N, m = N - 1, bb = G.b * G.b, nown = G.nown;
    const int nboxes = G.nbs * G.nbs, k0 = blockIdx.x * TL::NBX;
    const int s0 = 2 * warp, s1 = 2 * warp + 1;   // the warp's two slots: boxes warp BPT .. warp BPT + BPT - 1
    // each chunk's products are summed apart and then added to the total: the terms cancel heavily
    // (their magnitudes sum to about 10^2 times the result), and blocked summation keeps the FP32
    // rounding error at about half that of one running sum over all ne terms
    T tot[RA][TL::BPT];
#pragma unroll
    for (int a = 0; a < RA; ++a)
#pragma unroll
        for (int c2 = 0; c2 < TL::BPT; ++c2) tot[a][c2] = T(0);
    int rowA[RA];
#pragma unroll
    for (int a = 0; a < RA; ++a) rowA[a] = lane + 32 * a < nown ? lane + 32 * a : 0;   // rows past nown: unused
    for (int q0 = 0; q0 < G.ne; q0 += RAS_KC) {
        const int kc = min(RAS_KC, G.ne - q0);
        __syncthreads();   // the previous chunk is consumed; qtab is complete on the first pass
        {   // the inverse's chunk: kc nown words from inv + q0 nown (16-byte aligned: RAS_KC nown words apart)
            const int words = kc * nown, per16 = 16 / (int)sizeof(T), chunks = words / per16;
            const T* src = inv + (size_t)q0 * nown;
            for (int t = threadIdx.x; t < chunks; t += blockDim.x)
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(
                                 (uint32_t)__cvta_generic_to_shared(Ms + t * per16)),
                             "l"(src + (size_t)t * per16)
                             : "memory");
            for (int t = chunks * per16 + threadIdx.x; t < words; t += blockDim.x) Ms[t] = src[t];
        }
        {   // the windows' chunk: blocks of 8 dofs x 4 boxes, one per warp and pass
            const int qi = lane & 7, bi = lane >> 3;
            constexpr int QB = RAS_KC / 8, NBLK = QB * (TL::NBX / 4);
            for (int blk = warp; blk < NBLK; blk += RAS_BW) {
                const int ql = (blk % QB) * 8 + qi, box = (blk / QB) * 4 + bi;
                const int q = q0 + ql, kb = k0 + box;
                T v = T(0);
                if (q < G.ne && kb < nboxes) {
                    const int code = qtab[q];
                    const int gi = ((kb % G.nbs) * G.b - G.o + ((code >> 8) & 0xff)) & m;
                    const int gj = ((kb / G.nbs) * G.b - G.o + (code >> 16)) & m;
                    v = r[(size_t)(code & 0xff) * n + (size_t)gj * N + gi];
                }
                Rc[ql * TL::NBX + (((box / TL::VW) ^ (ql & 15)) * TL::VW) + box % TL::VW] = v;
            }
        }
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        __syncthreads();
        T acc[RA][TL::BPT];
#pragma unroll
        for (int a = 0; a < RA; ++a)
#pragma unroll
            for (int c2 = 0; c2 < TL::BPT; ++c2) acc[a][c2] = T(0);
#pragma unroll 4
        for (int ql = 0; ql < kc; ++ql) {
            T mv[RA];
#pragma unroll
            for (int a = 0; a < RA; ++a) mv[a] = Ms[ql * nown + rowA[a]];
            const V v0 = *reinterpret_cast<const V*>(Rc + ql * TL::NBX + ((s0 ^ (ql & 15)) * TL::VW));
            const V v1 = *reinterpret_cast<const V*>(Rc + ql * TL::NBX + ((s1 ^ (ql & 15)) * TL::VW));
#pragma unroll
            for (int a = 0; a < RA; ++a)
#pragma unroll
                for (int c2 = 0; c2 < TL::VW; ++c2) {
                    acc[a][c2] += mv[a] * vget<T>(v0, c2);
                    acc[a][TL::VW + c2] += mv[a] * vget<T>(v1, c2);
                }
        }
#pragma unroll
        for (int a = 0; a < RA; ++a)
#pragma unroll
            for (int c2 = 0; c2 < TL::BPT; ++c2) tot[a][c2] += acc[a][c2];
    }
#pragma unroll
    for (int c2 = 0; c2 < TL::BPT; ++c2) {
        const int kb = k0 + warp * TL::BPT + c2;
        if (kb >= nboxes || (slotOfBox && slotOfBox[kb] >= 0)) continue;   // IB boxes: k_ras_apply_big_ib
        const int I = kb % G.nbs, J = kb / G.nbs;
#pragma unroll
        for (int a = 0; a < RA; ++a) {
            const int rr = lane + 32 * a;
            if (rr >= nown) continue;
            const int comp = rr / bb, rem = rr - comp * bb;
            const size_t d = (size_t)comp * n + (size_t)(J * G.b + rem / G.b) * N + I * G.b + rem % G.b;
            xo[d] = (x ? x[d] : T(0)) + omega * tot[a][c2];
        }
    }
}

// One block per listed IB box with a subdomain wider than RAS_EMAX_SMEM: four groups of 64 threads
// each take a quarter of the q range for the owned rows lane64, lane64 + 64, ...; the partial sums
// are added in shared memory in a fixed order.
template <typename T>
__global__ void __launch_bounds__(256) k_ras_apply_big_ib(RasGeo G, const int* __restrict__ list,
                                                         const T* __restrict__ inv, T omega,
                                                         const T* __restrict__ r, const T* x, T* xo) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* rb = reinterpret_cast<T*>(smem_raw);   // ne
    T* part = rb + G.ne;                      // 4 x nown
    const int s = blockIdx.x, k = list[s];    // set-up data
    pdl_entry();
    const int I = k % G.nbs, J = k / G.nbs, N = G.N, n = N * N, m = N - 1, bb = G.b * G.b, nown = G.nown;
    const int i0 = I * G.b - G.o, j0 = J * G.b - G.o;
    for (int q = threadIdx.x; q < G.ne; q += blockDim.x) {
        int comp, ii, jj;
        ras_dof(G, q, comp, ii, jj);
        rb[q] = r[(size_t)comp * n + (size_t)((j0 + jj) & m) * N + ((i0 + ii) & m)];
    }
    __syncthreads();
    const T* M = inv + (size_t)(s + 1) * G.ne * nown;
    const int lr = threadIdx.x & 63, part_id = threadIdx.x >> 6;
    const int qchunk = (G.ne + 3) / 4;
    const int qa = part_id * qchunk, qb = min(G.ne, qa + qchunk);
    for (int rr = lr; rr < nown; rr += 64) {
        T acc = T(0);
#pragma unroll 4
        for (int q = qa; q < qb; ++q) acc += M[(size_t)q * nown + rr] * rb[q];
        part[part_id * nown + rr] = acc;
    }
    __syncthreads();
    for (int rr = threadIdx.x; rr < nown; rr += blockDim.x) {
        const T sum = ((part[rr] + part[nown + rr]) + part[2 * nown + rr]) + part[3 * nown + rr];
        const int comp = rr / bb, rem = rr - comp * bb;
        const size_t d = (size_t)comp * n + (size_t)(J * G.b + rem / G.b) * N + I * G.b + rem % G.b;
        xo[d] = (x ? x[d] : T(0)) + omega * sum;
    }
}

// ---- tensor-core correction of the IB-free boxes on FP32 levels ---------------------------------
// The boxes without IB terms share one inverse, so their correction is the product
//   C^T (boxes x owned rows) = R^T (boxes x ne) Inv^T (ne x owned rows).
// A tile of RT_NB = 128 boxes is the M of a tcgen05 TF32 MMA, the owned rows (padded to npad, a multiple
// of 16) its N, the subdomain dofs its K, taken in chunks of RT_KC = 32.  Three TF32 products per pair
// keep FP32 accuracy: a b = a_hi b_hi + a_hi b_lo + a_lo b_hi, a_hi = tf32(a), a_lo = tf32(a - a_hi)
// (the dropped a_lo b_lo is below FP32 rounding).  The accumulator lives in TMEM.  Both operands use the
// K-major layout of tcgen05.cuh: the residual chunk with LBO = 144 bytes (a 128-byte row of core
// matrices plus 16 bytes, so that the gather stores into shared memory without bank conflicts) and
// SBO = 8 LBO; the inverse chunk, written by bulk copies, packed (LBO = 128, SBO = 1024).
constexpr int RT_NB = 128, RT_KC = 32;
constexpr int RT_LBO = 144, RT_SBO = 8 * RT_LBO;      // residual chunk (A): rows padded by 16 bytes
constexpr int RT_BLBO = 128, RT_BSBO = 8 * RT_BLBO;   // inverse chunk (B): packed
constexpr int RT_THREADS = 512, RT_WARPS = RT_THREADS / 32;
constexpr int RT_BPW = RT_NB / RT_WARPS;          // boxes per warp in the residual gather
constexpr int RT_MAXSB = 16;                      // inverse stages at most
constexpr int RT_WAIT = 1 << 22;   // bounded waits on the copies and the MMAs
constexpr uint32_t RT_SLEEP_NS = 2000;   // sleep hint of one attempt in the pipeline's waits
constexpr int RT_SLEEP_WAIT = 1 << 18;   // attempts: at most about half a second of sleeping
constexpr int RT_ABYTES = (RT_NB / 8) * RT_SBO;   // one of hi, lo of the residual tile's chunk

// byte offset of (row, k) in a residual chunk of RT_KC values per row
__host__ __device__ inline int rt_off(int row, int k) {
    return (row >> 3) * RT_SBO + (k >> 2) * RT_LBO + (row & 7) * 16 + (k & 3) * 4;
}
// bytes of one of hi, lo of an inverse chunk (npad rows)
__host__ __device__ inline int rt_bbytes(int npad) { return (npad / 8) * RT_BSBO; }

// Packs the shared inverse's owned rows (slot 0 of inv64, [q][row]) for k_ras_apply_tc: chunk c holds
// rows 0 .. npad - 1 and dofs q = 32 c .. 32 c + 31 in the packed K-major layout, its hi part then its
// lo part; rows past nown and dofs past ne hold zeros.
__global__ void k_ras_tc_pack(const double* __restrict__ inv64, int ne, int nown, int npad, int nch,
                              float* __restrict__ out) {
    const int chunkWords = rt_bbytes(npad) / 4;
    const int64_t total = (int64_t)nch * 2 * chunkWords;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(idx / (2 * chunkWords));
        const int rem = (int)(idx - (int64_t)c * 2 * chunkWords);
        const int part = rem / chunkWords, byte = (rem - part * chunkWords) * 4;
        const int grp = byte / RT_BSBO, b2 = byte - grp * RT_BSBO, k4 = b2 / RT_BLBO, b3 = b2 - k4 * RT_BLBO;
        const int row = grp * 8 + b3 / 16, q = c * RT_KC + k4 * 4 + (b3 & 15) / 4;
        float val = 0.0f;
        if (row < nown && q < ne) {
            const double v = inv64[(size_t)q * nown + row];
            const float hi = tf32_rna((float)v);
            val = part == 0 ? hi : tf32_rna((float)(v - (double)hi));
        }
        out[idx] = val;
    }
}

// One correction of the IB-free boxes: xo(owned) = x(owned) + omega (Inv r_k)(owned) (x == nullptr: 0).
// Persistent blocks over tiles of RT_NB boxes; 16 worker warps and one issuing warp.  The residual
// chunks go through ns shared-memory stages and as many TMEM accumulator slots (chunk g uses stage and
// slot g % ns; ns = 2 for 8 x 8 boxes, whose slots fill the TMEM, 4 for smaller ones), the inverse
// chunks through nsb stages of their own (chunk g uses stage g % nsb): with nsb = nch the whole inverse
// stays resident and is fetched once, otherwise a chunk's copy is issued nsb - 1 chunks ahead of its MMAs.
//   Workers, for chunk g: wait for chunk g - ns's MMAs, add its slot into FP32 totals in registers (and
// write the tile when g - ns was its last chunk); store chunk g's residuals, gathered earlier (warp w:
// boxes w + 16 j, lane: the chunk's dof), split into hi and lo, into stage g % ns, and arrive on the
// stage's barrier; issue the loads of chunk g + 1's residuals.
//   Issuer (one thread), for chunk g: wait for the stage and the inverse chunk, issue the chunk's 3 x 4
// MMAs into slot g % ns starting from zero, commit them to the slot's barrier; in the ring, once chunk
// g - 1's MMAs are complete, fetch chunk g + nsb - 1 of the inverse into their inverse stage.
// Each chunk is thus summed apart and added to the total, as in the CUDA-core form (one long
// accumulation over all ne terms loses accuracy to their cancellation).  The worker of warp w and lane t
// holds owned rows (w / 4) npad / 4 .. of box 32 (w % 4) + t, the TMEM lanes its warp may read.  Every
// wait is bounded: a thread that gives up raises the block's error flag, every other wait then ends
// within its own bound, the block writes SIB_DEV_ERR_TMA_WAIT into the error word, the issuer waits
// (bounded) for its last MMAs and its copies in flight, and the TMEM is freed.
constexpr int RT_MAXNS = 4;   // residual stages and TMEM slots at most

// barrier of the four worker warps that share TMEM lane quadrant q (named barriers 1 .. 4)
__device__ __forceinline__ void quad_bar(int q) { asm volatile("bar.sync %0, 128;\n" ::"r"(1 + q) : "memory"); }
static_assert(MAX_N <= (1 << 15), "k_ras_apply_tc packs a box origin's two coordinates into one word");
template <int NC, int PF>
__global__ void __launch_bounds__(RT_THREADS + 32, 1)
    k_ras_apply_tc(RasGeo G, const int* __restrict__ slotOfBox, const float* __restrict__ pack, int npad, int nch,
                   int nsb, int ns, int rowOff, long long groupFloats, float omega, const float* __restrict__ r,
                   const float* x, float* xo, int* err) {
    // row group blockIdx.y: the next npad owned rows, from its own packed slice of the inverse
    pack += (size_t)blockIdx.y * (size_t)groupFloats;
    rowOff += (int)blockIdx.y * npad;
    extern __shared__ __align__(1024) unsigned char rt_smem[];
    __shared__ __align__(8) uint64_t tma_bar[RT_MAXSB];
    __shared__ __align__(8) uint64_t mma_bar[RT_MAXNS];    // the slot's MMAs are complete (one commit)
    __shared__ __align__(8) uint64_t full_bar[RT_MAXNS];   // the stage is stored and the slot read (every worker)
    __shared__ uint32_t tmem_base;
    __shared__ int s_err;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int aStage = 2 * RT_ABYTES;                  // hi and lo of one residual chunk
    const int bB = rt_bbytes(npad), bChunk = 2 * bB;   // hi and lo of one inverse chunk
    const int nq = nch * RT_KC;                        // dofs, padded to whole chunks
    unsigned char* bBase = rt_smem + ns * aStage;
    int* qoff = reinterpret_cast<int*>(bBase + nsb * bChunk);   // dof q: comp n + jj N + ii (-1: padding)
    int* qcode = qoff + nq;                                     // dof q: comp | ii << 8 | jj << 16
    int2* rowtab = reinterpret_cast<int2*>(qcode + nq);         // owned row: {comp, dy N + dx}
    int* linTab = reinterpret_cast<int*>(rowtab + G.nown);      // 2 x RT_NB gathered-box origins
    const bool resident = nsb == nch;
    const int N = G.N, n = N * N, m = N - 1, b = G.b, bb = b * b, nown = G.nown, e = G.e;
    for (int q = tid; q < nq; q += blockDim.x) {
        int comp = 0, ii = 0, jj = 0;
        if (q < G.ne) ras_dof(G, q, comp, ii, jj);
        qoff[q] = q < G.ne ? comp * n + jj * N + ii : -1;
        qcode[q] = comp | (ii << 8) | (jj << 16);
    }
    for (int rr = tid; rr < nown; rr += blockDim.x) {
        const int comp = rr / bb, rem = rr - comp * bb;
        rowtab[rr] = make_int2(comp, (rem / b) * N + rem % b);
    }
    if (tid == 0) {
        for (int k = 0; k < nsb; ++k) mbar_init(&tma_bar[k], 1);
        for (int k = 0; k < ns; ++k) {
            mbar_init(&mma_bar[k], 1);
            mbar_init(&full_bar[k], RT_THREADS);
        }
        s_err = 0;
        fence_mbar_init();
    }
    // ns accumulator slots of npad columns each (a power of two, 32 at least)
    const uint32_t slotCols = npad <= 32 ? 32u : npad <= 64 ? 64u : npad <= 128 ? 128u : 256u;
    const uint32_t ncols = ns * slotCols <= 32 ? 32u : ns * slotCols <= 64 ? 64u : ns * slotCols <= 128 ? 128u
                           : ns * slotCols <= 256 ? 256u : 512u;
    if (warp == 0) tmem_alloc(&tmem_base, ncols);
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tmem = tmem_base;
    pdl_entry();
    const int nboxes = G.nbs * G.nbs, ntiles = (nboxes + RT_NB - 1) / RT_NB;
    const int myTiles = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const uint32_t gEnd = (uint32_t)myTiles * nch;   // this block's chunks
    volatile int* verr = &s_err;
    if (warp == RT_WARPS) {   // ---- the issuing warp
        if (lane == 0) {
            const uint32_t idesc = umma_idesc_tf32(RT_NB, npad);
            // descriptors of the stages' first K step; step t adds t * 2 LBO bytes (the 14-bit address
            // field holds every shared-memory address, so the sums never carry out of it)
            const uint64_t dA0 = umma_desc(tc_smem_u32(rt_smem), RT_LBO, RT_SBO);
            const uint64_t dB0 = umma_desc(tc_smem_u32(bBase), RT_BLBO, RT_BSBO);
            auto fetch_inverse = [&](int st, int c) {   // chunk c of the inverse into inverse stage st
                mbar_expect_tx(&tma_bar[st], (uint32_t)bChunk);
                bulk_load(bBase + st * bChunk, reinterpret_cast<const unsigned char*>(pack) + (size_t)c * bChunk,
                          (uint32_t)bChunk, &tma_bar[st]);
            };
            uint32_t nM = 0, nT = 0;   // MMA commits and inverse copies issued
            for (uint32_t gc = 0; gc < (uint32_t)nsb && gc < gEnd; ++gc) {
                fetch_inverse((int)gc, (int)(gc % nch));
                nT = gc + 1;
            }
            int sa = 0, sb = 0;                     // stage/slot g % ns, inverse stage g % nsb
            uint32_t pa = 0, pb = 0;                // phase parities (g / ns) & 1, (g / nsb) & 1
            int sbNext = nsb - 1, cNext = (nsb - 1) % nch;   // where chunk g + nsb - 1's inverse goes
            int saPrev = ns - 1;                    // slot of chunk g - 1 and its parity
            uint32_t paPrev = 1;
            for (uint32_t g = 0; g < gEnd && !*verr; ++g) {
                if (!mbar_wait_sleep_bounded(&full_bar[sa], pa, RT_SLEEP_NS, RT_SLEEP_WAIT) ||
                    !mbar_wait_sleep_bounded(&tma_bar[sb], resident ? 0u : pb, RT_SLEEP_NS, RT_SLEEP_WAIT)) {
                    *verr = 1;
                    break;
                }
                tc_fence_after_sync();
                const uint32_t d = tmem + (uint32_t)sa * slotCols;
                const uint64_t ah = dA0 + (uint64_t)((sa * aStage) >> 4), al = ah + (RT_ABYTES >> 4);
                const uint64_t bh = dB0 + (uint64_t)((sb * bChunk) >> 4), bl = bh + (uint64_t)(bB >> 4);
#pragma unroll
                for (int t = 0; t < RT_KC / 8; ++t) {
                    const uint64_t ta = (uint64_t)(t * 2 * RT_LBO / 16), tb = (uint64_t)(t * 2 * RT_BLBO / 16);
                    umma_tf32(d, ah + ta, bh + tb, idesc, t > 0);   // the chunk's slot starts from zero
                    umma_tf32(d, ah + ta, bl + tb, idesc, true);
                    umma_tf32(d, al + ta, bh + tb, idesc, true);
                }
                umma_commit(&mma_bar[sa]);   // arrives once the MMAs issued so far are complete
                nM = g + 1;
                if (!resident && g >= 1 && g + nsb - 1 < gEnd) {   // chunk g - 1's inverse stage
                    if (!mbar_wait_sleep_bounded(&mma_bar[saPrev], paPrev, RT_SLEEP_NS, RT_SLEEP_WAIT)) {
                        *verr = 1;
                        break;
                    }
                    fetch_inverse(sbNext, cNext);
                    nT = g + nsb;
                }
                if (++sbNext == nsb) sbNext = 0;   // the inverse stage and chunk of g + nsb, for the next fetch
                if (++cNext == nch) cNext = 0;
                saPrev = sa;
                paPrev = pa;
                if (++sa == ns) {
                    sa = 0;
                    pa ^= 1u;
                }
                if (++sb == nsb) {
                    sb = 0;
                    pb ^= 1u;
                }
            }
            if (*verr) {   // the last MMAs and the copies in flight drain before the TMEM is freed
                if (nM > 0) mbar_wait_bounded(&mma_bar[(nM - 1) % ns], ((nM - 1) / ns) & 1, RT_WAIT);
                for (uint32_t gc = nT > (uint32_t)nsb ? nT - nsb : 0; gc < nT; ++gc)
                    mbar_wait_bounded(&tma_bar[gc % nsb], resident ? 0u : (gc / nsb) & 1u, RT_WAIT);
            }
        }
        __syncwarp();
    } else {   // ---- the workers
        const int q4 = npad / 4;                         // owned rows per thread
        const int cbase = (warp >> 2) * q4;              // this thread's first owned row
        const uint32_t lanes = (uint32_t)(32 * (warp & 3)) << 16;
        // the gathered boxes' subdomain origins, one table per tile parity, each warp writing and reading
        // only its own boxes' entries: oy N + ox where the subdomain lies inside the grid; for the periodic
        // wrap 2^31 | x | y << 16 taken mod N (N <= 2^15); -1 past the last box
        float v0[RT_BPW], v1[RT_BPW];                    // gathered residuals: PF chunks in flight
        int* lt = linTab;                                // the table of the tile being gathered
        int tilePar = 0;
        auto origins = [&](int tile) {
            lt = linTab + tilePar * RT_NB;
            tilePar ^= 1;
            if (lane < RT_BPW) {
                const int kb = tile * RT_NB + warp + RT_WARPS * lane;
                const int J = kb / G.nbs;
                const int ox = (kb - J * G.nbs) * b - G.o, oy = J * b - G.o;
                const bool in = ox >= 0 && oy >= 0 && ox + e < N && oy + e < N;   // faces ox .. ox + e
                lt[warp + RT_WARPS * lane] =
                    kb >= nboxes ? -1
                    : in         ? oy * N + ox
                                 : (int)(0x80000000u | ((uint32_t)ox & m) | (((uint32_t)oy & m) << 16));
            }
            __syncwarp();
            // the tile's owned cells of x into L2, ahead of its writes (nch + ns chunks later): with rows
            // of boxes a multiple of RT_NB long, its 128 boxes cover 3 b rows of 128 b cells, 12 b^2 lines of
            // 128 bytes, spread over the workers
            if (x && (G.nbs % RT_NB) == 0) {
                const int J = (tile * RT_NB) / G.nbs, I0 = tile * RT_NB - J * G.nbs;
                for (int ln = tid; ln < 12 * b * b; ln += RT_THREADS) {
                    const int perRow = 4 * b;   // 128-byte lines in a row of 128 b FP32 cells
                    const int row = ln / perRow, k = ln - row * perRow;
                    const int comp = row / b, dy = row - comp * b;
                    const float* pa =
                        x + (size_t)comp * n + (size_t)(J * b + dy) * N + (size_t)I0 * b + (size_t)k * 32;
                    asm volatile("prefetch.global.L2 [%0];\n" ::"l"(pa));
                }
            }
        };
        auto gather = [&](int c, float (&v)[RT_BPW]) {
            const int q = c * RT_KC + lane;
            const int off = qoff[q];
#pragma unroll
            for (int j = 0; j < RT_BPW; ++j) {
                const int lin = lt[warp + RT_WARPS * j];
                v[j] = 0.0f;
                if (lin >= 0) {
                    if (off >= 0) v[j] = __ldg(r + (lin + off));
                } else if (lin != -1 && off >= 0) {
                    const int code = qcode[q];
                    const int ii = (code >> 8) & 0xff, jj = code >> 16;
                    const int gx = ((lin & 0xffff) + ii) & m, gy = ((((uint32_t)lin >> 16) & 0x7fffu) + jj) & m;
                    v[j] = __ldg(r + ((size_t)(code & 0xff) * n + (size_t)gy * N + gx));
                }
            }
        };
        // the gather cursor: the next chunk to gather (tile, chunk); origins() when it enters a tile
        int tileG = blockIdx.x, cG = 0;
        auto gather_next = [&](float (&v)[RT_BPW]) {
            if (tileG >= ntiles) return;
            if (cG == 0) origins(tileG);
            gather(cG, v);
            if (++cG == nch) {
                cG = 0;
                tileG += gridDim.x;
            }
        };
        float tot[NC];
#pragma unroll
        for (int j = 0; j < NC; ++j) tot[j] = 0.0f;
        int tileD = blockIdx.x, cD = 0;   // the chunk being added
        int sS = 0, sD = 0;               // their stages / slots
        uint32_t pD = 0;                  // the added chunk's phase parity
        bool ok = true;                   // warp-uniform; after a failed wait the workers only keep step
        const int lb = __ffs(b) - 1;      // b = 2^lb
        const int quad = warp & 3;        // TMEM lane quadrant: boxes 32 quad .. 32 quad + 31 of the tile
        const int boxl = 32 * quad + lane;
        // a quadrant's 32 boxes lie in one row of boxes, next to each other, when nbs is a multiple of 32:
        // the tile is then written row by row through the TMEM
        const bool rowWrite = (G.nbs & 31) == 0;
        gather_next(v0);
        if (PF == 2) gather_next(v1);
        // Every worker runs every iteration, so that the quadrant barriers of the tile writes are reached
        // by all of them whatever the waits returned.
        for (uint32_t g = 0; g < gEnd + ns; ++g) {
            if (g >= (uint32_t)ns) {   // chunk g - ns: its slot into the totals, then the tile after its last chunk
                // warp-uniform: the slot loads below are warp-collective
                const bool w = __all_sync(0xffffffffu, ok && !*verr &&
                                                           mbar_wait_sleep_bounded(&mma_bar[sD], pD, RT_SLEEP_NS,
                                                                                   RT_SLEEP_WAIT));
                if (!w && ok) {
                    ok = false;
                    *verr = 1;
                }
                const uint32_t slot = tmem + (uint32_t)sD * slotCols;   // free until chunk g's MMAs
                if (ok) {
                    tc_fence_after_sync();
                    const uint32_t base = slot + lanes + (uint32_t)cbase;
#pragma unroll
                    for (int c0 = 0; c0 < NC; c0 += 8) {
                        uint32_t a[8];
                        tmem_ld8(base + (uint32_t)c0, a);
#pragma unroll
                        for (int j = 0; j < 8; ++j) tot[c0 + j] += __uint_as_float(a[j]);
                    }
                }
                if (++sD == ns) {
                    sD = 0;
                    pD ^= 1u;
                }
                if (++cD == nch) {   // the tile
                    const int k0 = tileD * RT_NB;
                    const int kb = k0 + boxl;
                    const bool wr = ok && kb < nboxes && !(slotOfBox && slotOfBox[kb] >= 0);
                    if (rowWrite) {
                        // the totals back into the slot, then read 16 boxes x 8 rows at a time: consecutive
                        // threads hold consecutive rows of a box, consecutive boxes follow, so the writes run
                        // along x
                        const unsigned wmask = __ballot_sync(0xffffffffu, wr);
                        if (ok) {
#pragma unroll
                            for (int j = 0; j < NC; j += 4)
                                if (j < q4) tmem_st4(slot + lanes + (uint32_t)(cbase + j), tot[j], tot[j + 1], tot[j + 2], tot[j + 3]);
                            tmem_wait_st();
                        }
                        tc_fence_before_sync();
                        quad_bar(quad);
                        tc_fence_after_sync();
                        const int kq = k0 + 32 * quad;
                        const int J = kq / G.nbs, I0 = kq - J * G.nbs;
                        const size_t rowBase = (size_t)(J * b) * N + (size_t)(I0 * b);
                        for (int grp = warp >> 2; grp < npad / 8 && ok; grp += 4) {
                            // both 16-lane halves of the group: the eight x loads go out before any store
                            uint32_t a[8];
                            tmem_ld16x256(slot + ((uint32_t)(32 * quad) << 16) + (uint32_t)(8 * grp), *(uint32_t(*)[4])a);
                            tmem_ld16x256(slot + ((uint32_t)(32 * quad + 16) << 16) + (uint32_t)(8 * grp),
                                          *(uint32_t(*)[4])(a + 4));
                            float xv[8];
                            int dd[8];   // offset within the component, or -1
                            int cc[8];
#pragma unroll
                            for (int u = 0; u < 8; ++u) {
                                const int l = 16 * (u >> 2) + (lane >> 2) + 8 * ((u >> 1) & 1);   // box in the quadrant
                                const int rr = rowOff + 8 * grp + 2 * (lane & 3) + (u & 1);           // owned row
                                const int comp = rr >> (2 * lb), rem = rr & (bb - 1);
                                cc[u] = comp;
                                dd[u] = (rr < nown && ((wmask >> l) & 1u))
                                            ? (int)rowBase + ((rem >> lb) * N) + l * b + (rem & (b - 1))
                                            : -1;
                                xv[u] = (dd[u] >= 0 && x) ? x[(size_t)comp * n + dd[u]] : 0.0f;
                            }
#pragma unroll
                            for (int u = 0; u < 8; ++u)
                                if (dd[u] >= 0) xo[(size_t)cc[u] * n + dd[u]] = xv[u] + omega * __uint_as_float(a[u]);
                        }
                    } else if (wr) {   // boxes across rows of boxes: each thread writes its own rows
                        const int J = kb / G.nbs, I = kb - J * G.nbs;
                        const size_t org0 = (size_t)(J * b) * N + (size_t)(I * b);
#pragma unroll
                        for (int j = 0; j < NC; ++j) {
                            const int rr = rowOff + cbase + j;
                            if (j < q4 && rr < nown) {
                                const int2 t = rowtab[rr];
                                const size_t d = (size_t)t.x * n + org0 + (size_t)t.y;
                                xo[d] = (x ? x[d] : 0.0f) + omega * tot[j];
                            }
                        }
                    }
#pragma unroll
                    for (int j = 0; j < NC; ++j) tot[j] = 0.0f;
                    cD = 0;
                    tileD += gridDim.x;
                }
            }
            if (g < gEnd) {   // chunk g into its stage (free: chunk g - ns's MMAs are complete)
                unsigned char* Ahi = rt_smem + sS * aStage;
                // chunk g's residuals are in v0 (in v1 for odd g when two chunks are in flight); their
                // array then takes the loads of chunk g + PF, in flight until its stores
                auto store_refill = [&](float (&v)[RT_BPW]) {
#pragma unroll
                    for (int j = 0; j < RT_BPW; ++j) {
                        const float hi = tf32_rna(v[j]);
                        const int off = rt_off(warp + RT_WARPS * j, lane);
                        *reinterpret_cast<float*>(Ahi + off) = hi;
                        *reinterpret_cast<float*>(Ahi + RT_ABYTES + off) = tf32_rna(v[j] - hi);
                    }
                    fence_proxy_async_smem();
                    tc_fence_before_sync();
                    mbar_arrive(&full_bar[sS]);
                    gather_next(v);
                };
                if (PF == 1 || (g & 1) == 0)
                    store_refill(v0);
                else
                    store_refill(v1);
                if (++sS == ns) sS = 0;
            }
        }
    }
    tc_fence_before_sync();
    __syncthreads();
    if (tid == 0 && s_err && err) *(volatile int*)err = SIB_DEV_ERR_TMA_WAIT;
    if (warp == 0) tmem_dealloc(tmem, ncols);
}

// ---- 16 x 16 boxes: the shared inverse by the blocked Gauss-Jordan, and a low-rank (Woodbury)
// update of it for the IB boxes ------------------------------------------------------------------
// An IB box's local operator is L_k = L_0 + P E P^T: P selects the subdomain's IB-touched velocity dofs
// T (rows with a nonzero window entry at a column of the subdomain), E = -dt B on T x T.  Then
//   L_k^{-1} = L_0^{-1} - L_0^{-1} P W P^T L_0^{-1},   W = (I + E Q)^{-1} E,   Q = P^T L_0^{-1} P,
// so an IB box's correction is the shared one minus (L_0^{-1})_{own,T} W (L_0^{-1})_{T,:} r_k.  Set-up
// costs |T|^3 flops per IB box instead of ne^3, and |T|^2 words instead of ne nown.

// Aug = [L_0 | I] (n x 2n, zeroed by the caller; n >= ne a multiple of 16, rows and columns past ne the
// identity).  L_0 is the IB-free subdomain operator, the same for every box of the level.
__global__ void k_ras_huge_assemble(RasGeo G, double a0, double c, double inv_h, int n, double* __restrict__ Aug) {
    const RasIB none{nullptr, nullptr, 1, 1, 1};
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        double* row = Aug + (size_t)q * 2 * n;
        if (q < G.ne)
            ras_assemble_row(G, none, a0, c, inv_h, 0.0, false, 0, 0, q, row);
        else
            row[q] = 1.0;
        row[n + q] = 1.0;
    }
}

// the full inverse, row-major ne x ne: row r is Aug[piv[r]][n ..] (the elimination swaps no rows)
__global__ void k_ras_huge_extract(const double* __restrict__ Aug, const int* __restrict__ piv, int n, int ne,
                                   double* __restrict__ inv64, float* __restrict__ inv32) {
    const int r = blockIdx.y;
    const double* src = Aug + (size_t)piv[r] * 2 * n + n;
    for (int cc = blockIdx.x * blockDim.x + threadIdx.x; cc < ne; cc += gridDim.x * blockDim.x) {
        const double v = src[cc];
        inv64[(size_t)r * ne + cc] = v;
        inv32[(size_t)r * ne + cc] = (float)v;
    }
}

// whether local dof q of the subdomain with corner (i0, j0) is IB-touched: a velocity face with a
// nonzero window entry at a column of the subdomain
__device__ bool ras_ib_row(const RasGeo& G, const RasIB& ib, int i0, int j0, int q) {
    int comp, ii, jj;
    ras_dof(G, q, comp, ii, jj);
    if (comp == 2) return false;
    const int m = G.N - 1, per = ib.tx * ib.ty;
    const int gi = (i0 + ii) & m, gj = (j0 + jj) & m;
    const int slot = face_slot(ib, gi, gj);
    if (slot < 0) return false;
    const double* w = ib.win + ((size_t)(slot * 2 + comp) * WIN_SIZE) * per;
    const int qt = (gj % ib.ty) * ib.tx + (gi % ib.tx);
    for (int dj = -WR; dj <= WR; ++dj)
        for (int di = -WR; di <= WR; ++di)
            if (w[(size_t)((dj + WR) * WD + (di + WR)) * per + qt] != 0.0 &&
                ras_index(G, comp, (ii + di) & m, (jj + dj) & m) >= 0)
                return true;
    return false;
}

// |T| of each listed IB box (one block per box)
__global__ void k_ras_wb_count(RasGeo G, RasIB ib, const int* __restrict__ list, int* __restrict__ cnt) {
    __shared__ int total;
    const int k = list[blockIdx.x];
    const int i0 = (k % G.nbs) * G.b - G.o, j0 = (k / G.nbs) * G.b - G.o;
    if (threadIdx.x == 0) total = 0;
    __syncthreads();
    int mine = 0;
    for (int q = threadIdx.x; q < 2 * G.e * (G.e + 1); q += blockDim.x) mine += ras_ib_row(G, ib, i0, j0, q) ? 1 : 0;
    if (mine) atomicAdd(&total, mine);
    __syncthreads();
    if (threadIdx.x == 0) cnt[blockIdx.x] = total;
}

// the T lists, ascending local dof (one block per box; an ordered compaction over chunks of dofs)
__global__ void k_ras_wb_fill(RasGeo G, RasIB ib, const int* __restrict__ list, const int* __restrict__ offT,
                              int* __restrict__ T) {
    __shared__ int wcount[32], woff[32], base;
    const int k = list[blockIdx.x];
    const int i0 = (k % G.nbs) * G.b - G.o, j0 = (k / G.nbs) * G.b - G.o;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nv = 2 * G.e * (G.e + 1);
    int* out = T + offT[blockIdx.x];
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    for (int q0 = 0; q0 < nv; q0 += blockDim.x) {
        const int q = q0 + threadIdx.x;
        const bool f = q < nv && ras_ib_row(G, ib, i0, j0, q);
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        if (lane == 0) wcount[warp] = __popc(bal);
        __syncthreads();
        if (threadIdx.x == 0) {
            int acc = base;
            for (int w = 0; w < nw; ++w) {
                woff[w] = acc;
                acc += wcount[w];
            }
            base = acc;
        }
        __syncthreads();
        if (f) out[woff[warp] + __popc(bal & ((1u << lane) - 1u))] = q;
        __syncthreads();
    }
}

// One block per IB box: Mx = [I + E Q | E] (m x 2m, row-major, at work + 2 offW), eliminated by
// Gauss-Jordan with partial (row) pivoting to [I | W]; W (m x m, row-major) is stored at offW.
// E = -dt B on T x T (the window entries), Q = (L_0^{-1})_{T,T} from the full shared inverse.
// info != 0 on a zero pivot.
constexpr int RAS_WB_THREADS = 256;
__global__ void __launch_bounds__(RAS_WB_THREADS)
    k_ras_wb_setup(RasGeo G, RasIB ib, double dt, const int* __restrict__ list, const int* __restrict__ offT,
                   const int* __restrict__ Tl, const long long* __restrict__ offW, const double* __restrict__ inv0,
                   double* __restrict__ work, double* __restrict__ W, int* __restrict__ info, int mOneMax) {
    extern __shared__ double smem_wb[];
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int k = list[blockIdx.x];
    const int i0 = (k % G.nbs) * G.b - G.o, j0 = (k / G.nbs) * G.b - G.o;
    const int t0 = offT[blockIdx.x], m = offT[blockIdx.x + 1] - t0, n2 = 2 * m;
    const int* Ts = Tl + t0;
    double* Mx = work + 2 * offW[blockIdx.x];
    double* rowk = smem_wb;                           // 2m: pivot row after scaling
    double* colk = rowk + n2;                         // m: pivot column before the step
    double* redv = colk + m;                          // 32
    int* redi = reinterpret_cast<int*>(redv + 32);    // 32
    int* ent = redi + 32;                             // nw x WIN_SIZE: a row's nonzero positions in T
    double* ev = reinterpret_cast<double*>(ent + nw * WIN_SIZE + (nw * WIN_SIZE & 1));   // nw x WIN_SIZE values
    __shared__ int pivS;
    for (size_t t = tid; t < (size_t)m * n2; t += nt) Mx[t] = 0.0;
    __syncthreads();
    const int mk = G.N - 1, per = ib.tx * ib.ty;
    for (int a = warp; a < m; a += nw) {   // one warp per row a: E's row, then I + E Q's row
        int* me = ent + warp * WIN_SIZE;
        double* mv = ev + warp * WIN_SIZE;
        int comp, ii, jj;
        ras_dof(G, Ts[a], comp, ii, jj);
        const int gi = (i0 + ii) & mk, gj = (j0 + jj) & mk;
        const int slot = face_slot(ib, gi, gj);
        int cnt = 0;
        if (slot >= 0) {
            const double* w = ib.win + ((size_t)(slot * 2 + comp) * WIN_SIZE) * per;
            const int qt = (gj % ib.ty) * ib.tx + (gi % ib.tx);
            for (int kw0 = 0; kw0 < WIN_SIZE; kw0 += 32) {   // window entries whose column is in T
                const int kw = kw0 + lane;
                int pos = -1;
                double coef = 0.0;
                if (kw < WIN_SIZE) {
                    const int dj = kw / WD - WR, di = kw % WD - WR;
                    coef = w[(size_t)kw * per + qt];
                    const int col = ras_index(G, comp, (ii + di) & mk, (jj + dj) & mk);
                    if (coef != 0.0 && col >= 0) {
                        int lo = 0, hi = m;   // lower bound of col in the ascending T
                        while (lo < hi) {
                            const int mid = (lo + hi) >> 1;
                            if (Ts[mid] < col) lo = mid + 1;
                            else hi = mid;
                        }
                        if (lo < m && Ts[lo] == col) pos = lo;
                    }
                }
                const unsigned bal = __ballot_sync(0xffffffffu, pos >= 0);
                if (pos >= 0) {
                    const int at = cnt + __popc(bal & ((1u << lane) - 1u));
                    me[at] = pos;
                    mv[at] = -dt * coef;
                }
                cnt += __popc(bal);
            }
        }
        __syncwarp();
        double* Ma = Mx + (size_t)a * n2;
        for (int t = lane; t < cnt; t += 32) Ma[m + me[t]] += mv[t];   // distinct positions per row
        for (int bcol = lane; bcol < m; bcol += 32) {
            const int Tb = Ts[bcol];
            double acc = a == bcol ? 1.0 : 0.0;
            for (int t = 0; t < cnt; ++t) acc += mv[t] * inv0[(size_t)Ts[me[t]] * G.ne + Tb];
            Ma[bcol] = acc;
        }
        __syncwarp();
    }
    __syncthreads();
    if (m > mOneMax) return;   // a large box: [I + E Q | E] is eliminated by the blocked Gauss-Jordan
    for (int kk = 0; kk < m; ++kk) {
        double best = -1.0;
        int bi = kk;
        for (int i = kk + tid; i < m; i += nt) {
            const double v = fabs(Mx[(size_t)i * n2 + kk]);
            if (v > best) {
                best = v;
                bi = i;
            }
        }
        for (int off = 16; off > 0; off >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, best, off);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
            if (ov > best || (ov == best && oi < bi)) {
                best = ov;
                bi = oi;
            }
        }
        if (lane == 0) {
            redv[warp] = best;
            redi[warp] = bi;
        }
        __syncthreads();
        if (tid == 0) {
            double bv = redv[0];
            int bx = redi[0];
            for (int w2 = 1; w2 < nw; ++w2)
                if (redv[w2] > bv || (redv[w2] == bv && redi[w2] < bx)) {
                    bv = redv[w2];
                    bx = redi[w2];
                }
            pivS = bx;
            if (!(bv > 0.0)) atomicExch(info, 1);
        }
        __syncthreads();
        const int p = pivS;
        if (p != kk)
            for (int j = kk + tid; j < n2; j += nt) {
                const double t = Mx[(size_t)kk * n2 + j];
                Mx[(size_t)kk * n2 + j] = Mx[(size_t)p * n2 + j];
                Mx[(size_t)p * n2 + j] = t;
            }
        __syncthreads();
        const double piv = Mx[(size_t)kk * n2 + kk];
        const double pinv = piv != 0.0 ? 1.0 / piv : 0.0;
        for (int i = tid; i < m; i += nt) colk[i] = Mx[(size_t)i * n2 + kk];
        for (int j = kk + tid; j < n2; j += nt) rowk[j] = Mx[(size_t)kk * n2 + j] * pinv;
        __syncthreads();
        for (size_t t = tid; t < (size_t)m * (n2 - kk); t += nt) {
            const int i = (int)(t / (n2 - kk)), j = kk + (int)(t % (n2 - kk));
            Mx[(size_t)i * n2 + j] = i == kk ? rowk[j] : Mx[(size_t)i * n2 + j] - colk[i] * rowk[j];
        }
        __syncthreads();
    }
    double* Wb = W + offW[blockIdx.x];
    for (size_t t = tid; t < (size_t)m * m; t += nt) Wb[t] = Mx[(t / m) * n2 + m + t % m];
}

// Shared correction of every box with 16 x 16 boxes, on the CUDA cores: a block takes RH_BX boxes,
// gathers their windows into shared memory, and each warp walks owned rows: row own(r) of the shared
// inverse, read once per block, against the RH_BX windows.  xo(owned) = x(owned) + omega c
// (x == nullptr: 0).  Blocks along y split the owned rows (rows blockIdx.y, blockIdx.y + gridDim.y, ...
// of the warps' walk), so that a level with few boxes still fills the GPU.
constexpr int RH_BX = 8, RH_THREADS = 256;
template <typename T>
__global__ void __launch_bounds__(RH_THREADS)
    k_ras_huge_apply(RasGeo G, const T* __restrict__ inv, T omega, const T* __restrict__ r, const T* x, T* xo) {
    extern __shared__ unsigned char smem_rh[];
    T* win = reinterpret_cast<T*>(smem_rh);   // RH_BX x ne
    const int N = G.N, n = N * N, m = N - 1, ne = G.ne;
    const int nboxes = G.nbs * G.nbs, k0 = blockIdx.x * RH_BX;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    pdl_entry();
    for (int t = threadIdx.x; t < RH_BX * ne; t += blockDim.x) {
        const int j = t / ne, q = t - j * ne, kb = k0 + j;
        T v = T(0);
        if (kb < nboxes) {
            int comp, ii, jj;
            ras_dof(G, q, comp, ii, jj);
            const int gi = ((kb % G.nbs) * G.b - G.o + ii) & m, gj = ((kb / G.nbs) * G.b - G.o + jj) & m;
            v = r[(size_t)comp * n + (size_t)gj * N + gi];
        }
        win[t] = v;
    }
    __syncthreads();
    for (int rr = (int)blockIdx.y * nw + warp; rr < G.nown; rr += nw * (int)gridDim.y) {
        const T* row = inv + (size_t)ras_owned(G, rr) * ne;
        T acc[RH_BX];
#pragma unroll
        for (int j = 0; j < RH_BX; ++j) acc[j] = T(0);
        for (int q = lane; q < ne; q += 32) {
            const T a = row[q];
#pragma unroll
            for (int j = 0; j < RH_BX; ++j) acc[j] += a * win[j * ne + q];
        }
#pragma unroll
        for (int j = 0; j < RH_BX; ++j)
            for (int off = 16; off > 0; off >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], off);
        if (lane < RH_BX && k0 + lane < nboxes) {
            T a = acc[0];
#pragma unroll
            for (int j = 1; j < RH_BX; ++j)
                if (lane == j) a = acc[j];
            const int kb = k0 + lane, bb = G.b * G.b;
            const int comp = rr / bb, rem = rr - comp * bb;
            const size_t d = (size_t)comp * n + (size_t)((kb / G.nbs) * G.b + rem / G.b) * N + (kb % G.nbs) * G.b +
                             rem % G.b;
            xo[d] = (x ? x[d] : T(0)) + omega * a;
        }
    }
}

// (L_k v)_q for the subdomain with corner (i0, j0): the entries of ras_assemble_row (withIB: with the IB
// windows' -dt B), applied to v without forming the row
__device__ double ras_row_dot(const RasGeo& G, const RasIB& ib, double a0, double c, double inv_h, double dt,
                              int i0, int j0, int q, const double* v) {
    const int m = G.N - 1, per = ib.tx * ib.ty;
    int comp, ii, jj;
    ras_dof(G, q, comp, ii, jj);
    double acc = 0.0;
    if (comp < 2) {
        acc = a0 * v[q];
        const int nb[4][2] = {{ii + 1, jj}, {ii - 1, jj}, {ii, jj + 1}, {ii, jj - 1}};
        for (int s2 = 0; s2 < 4; ++s2) {
            const int col = ras_index(G, comp, nb[s2][0] & m, nb[s2][1] & m);
            if (col >= 0) acc -= c * v[col];
        }
        const int pc = ras_index(G, 2, ii, jj);
        const int pm = comp == 0 ? ras_index(G, 2, ii - 1, jj) : ras_index(G, 2, ii, jj - 1);
        if (pc >= 0) acc += inv_h * v[pc];
        if (pm >= 0) acc -= inv_h * v[pm];
        const int gi = (i0 + ii) & m, gj = (j0 + jj) & m;
        const int slot = face_slot(ib, gi, gj);
        if (slot >= 0) {
            const double* w = ib.win + ((size_t)(slot * 2 + comp) * WIN_SIZE) * per;
            const int qt = (gj % ib.ty) * ib.tx + (gi % ib.tx);
            for (int dj = -WR; dj <= WR; ++dj)
                for (int di = -WR; di <= WR; ++di) {
                    const int col = ras_index(G, comp, (ii + di) & m, (jj + dj) & m);
                    if (col >= 0) acc -= dt * w[(size_t)((dj + WR) * WD + (di + WR)) * per + qt] * v[col];
                }
        }
    } else {
        acc = -inv_h * v[ras_index(G, 0, ii + 1, jj)] + inv_h * v[ras_index(G, 0, ii, jj)] -
              inv_h * v[ras_index(G, 1, ii, jj + 1)] + inv_h * v[ras_index(G, 1, ii, jj)];
    }
    return acc;
}

// IB boxes with 16 x 16 boxes, one block per box, in FP64, after the shared correction wrote
// xo = x + omega (L_0^{-1} r_k)(owned) for every box.  The box's own local solve is L_k^{-1} r_k = M r_k, the
// Woodbury form M r = y - (L_0^{-1})_{:,T} W y_T, y = L_0^{-1} r.
// FP64 levels: delta_0 = M r_k is refined once against the local operator itself, delta = delta_0 +
// M (r_k - L_k delta_0): with a stiff structure W is large and the two terms of M nearly cancel, and the
// refinement recovers the digits they lose; then xo(owned) += omega (delta - L_0^{-1} r_k)(owned).
// FP32 levels: the low-rank term alone, xo(owned) -= omega (L_0^{-1})_{own,T} W (L_0^{-1})_{T,:} r_k (what
// the cancellation costs stays below FP32 rounding; m (ne + nown) flops instead of 2 ne^2).
// L_0^{-1} is symmetric (L_0 is), so its columns T are read as rows.
template <typename T>
__global__ void __launch_bounds__(256)
    k_ras_wb_apply(RasGeo G, RasIB ib, double a0, double c, double inv_h, double dt, const int* __restrict__ list,
                   const int* __restrict__ offT, const int* __restrict__ Tl, const long long* __restrict__ offW,
                   const double* __restrict__ Wd, const double* __restrict__ inv0, T omega, const T* __restrict__ r,
                   T* xo) {
    extern __shared__ double smem_wa[];
    const int N = G.N, n = N * N, mk = N - 1, ne = G.ne;
    const int k = list[blockIdx.x];
    const int I = k % G.nbs, J = k / G.nbs, i0 = I * G.b - G.o, j0 = J * G.b - G.o;
    const int t0 = offT[blockIdx.x], m = offT[blockIdx.x + 1] - t0;
    const int* Ts = Tl + t0;
    const double* Wb = Wd + offW[blockIdx.x];
    double* rk = smem_wa;     // ne: r_k, then the refinement's residual
    double* y0 = rk + ne;     // ne: L_0^{-1} r_k
    double* d0 = y0 + ne;     // ne: delta_0
    double* y1 = d0 + ne;     // ne: L_0^{-1} of the residual
    double* z = y1 + ne;      // m
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    pdl_entry();
    for (int q = threadIdx.x; q < ne; q += blockDim.x) {
        int comp, ii, jj;
        ras_dof(G, q, comp, ii, jj);
        rk[q] = (double)r[(size_t)comp * n + (size_t)((j0 + jj) & mk) * N + ((i0 + ii) & mk)];
    }
    __syncthreads();
    // out = M in (full vector); y holds L_0^{-1} in on return
    auto woodbury = [&](const double* in, double* y, double* out) {
        for (int q = warp; q < ne; q += nw) {   // y = L_0^{-1} in
            const double* row = inv0 + (size_t)q * ne;
            double acc = 0.0;
            for (int t = lane; t < ne; t += 32) acc += row[t] * in[t];
            for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
            if (lane == 0) y[q] = acc;
        }
        __syncthreads();
        for (int a = warp; a < m; a += nw) {   // z = W y_T
            const double* row = Wb + (size_t)a * m;
            double acc = 0.0;
            for (int t = lane; t < m; t += 32) acc += row[t] * y[Ts[t]];
            for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
            if (lane == 0) z[a] = acc;
        }
        __syncthreads();
        for (int q = threadIdx.x; q < ne; q += blockDim.x) {   // out = y - (L_0^{-1})_{:,T} z
            double acc = 0.0;
            for (int a = 0; a < m; ++a) acc += inv0[(size_t)Ts[a] * ne + q] * z[a];
            out[q] = y[q] - acc;
        }
        __syncthreads();
    };
    const int bb = G.b * G.b;
    if constexpr (sizeof(T) == 4) {
        for (int a = warp; a < m; a += nw) {   // y_T = (L_0^{-1})_{T,:} r_k
            const double* row = inv0 + (size_t)Ts[a] * ne;
            double acc = 0.0;
            for (int t = lane; t < ne; t += 32) acc += row[t] * rk[t];
            for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
            if (lane == 0) y0[a] = acc;
        }
        __syncthreads();
        for (int a = warp; a < m; a += nw) {   // z = W y_T
            const double* row = Wb + (size_t)a * m;
            double acc = 0.0;
            for (int t = lane; t < m; t += 32) acc += row[t] * y0[t];
            for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
            if (lane == 0) z[a] = acc;
        }
        __syncthreads();
        for (int rr = threadIdx.x; rr < G.nown; rr += blockDim.x) {
            const double* row = inv0 + (size_t)ras_owned(G, rr) * ne;
            double acc = 0.0;
            for (int a = 0; a < m; ++a) acc += row[Ts[a]] * z[a];
            const int comp = rr / bb, rem = rr - comp * bb;
            const size_t d = (size_t)comp * n + (size_t)(J * G.b + rem / G.b) * N + I * G.b + rem % G.b;
            xo[d] = (T)((double)xo[d] - (double)omega * acc);
        }
        return;
    }
    woodbury(rk, y0, d0);
    for (int q = threadIdx.x; q < ne; q += blockDim.x)   // the residual of delta_0 in the local problem
        y1[q] = rk[q] - ras_row_dot(G, ib, a0, c, inv_h, dt, i0, j0, q, d0);
    __syncthreads();
    for (int q = threadIdx.x; q < ne; q += blockDim.x) rk[q] = y1[q];
    __syncthreads();
    woodbury(rk, y1, rk);   // rk <- M (residual)
    for (int rr = threadIdx.x; rr < G.nown; rr += blockDim.x) {
        const int q = ras_owned(G, rr);
        const int comp = rr / bb, rem = rr - comp * bb;
        const size_t d = (size_t)comp * n + (size_t)(J * G.b + rem / G.b) * N + I * G.b + rem % G.b;
        xo[d] = (T)((double)xo[d] + (double)omega * (d0[q] + rk[q] - y0[q]));
    }
}

// Packs owned rows rowOff .. rowOff + npad - 1 of the full shared inverse (row-major ne x ne) for the
// tensor-core correction, in the layout of k_ras_tc_pack (rows past nown hold zeros)
__global__ void k_ras_tc_pack_rows(RasGeo G, const double* __restrict__ inv0, int rowOff, int npad, int nch,
                                   float* __restrict__ out) {
    const int chunkWords = rt_bbytes(npad) / 4;
    const int64_t total = (int64_t)nch * 2 * chunkWords;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(idx / (2 * chunkWords));
        const int rem = (int)(idx - (int64_t)c * 2 * chunkWords);
        const int part = rem / chunkWords, byte = (rem - part * chunkWords) * 4;
        const int grp = byte / RT_BSBO, b2 = byte - grp * RT_BSBO, k4 = b2 / RT_BLBO, b3 = b2 - k4 * RT_BLBO;
        const int row = rowOff + grp * 8 + b3 / 16, q = c * RT_KC + k4 * 4 + (b3 & 15) / 4;
        float val = 0.0f;
        if (row < G.nown && q < G.ne) {
            const double v = inv0[(size_t)ras_owned(G, row) * G.ne + q];
            const float hi = tf32_rna((float)v);
            val = part == 0 ? hi : tf32_rna((float)(v - (double)hi));
        }
        out[idx] = val;
    }
}

}  // namespace

bool ras_big(int b, int o) { return b + 2 * o > RAS_EMAX_SMEM; }

size_t ras_setup_smem(int b, int o) {
    const RasGeo G = ras_geo(16, b, o);
    return sizeof(double) * ((size_t)G.ne * G.ne + G.ne + 32) + sizeof(int) * (32 + G.ne);
}
int ras_ne(int b, int o) { return ras_geo(16, b, o).ne; }

void launch_ras_classify(int N, int b, int o, const RasIB& ib, int* list, int* count, cudaStream_t s) {
    const RasGeo G = ras_geo(N, b, o);
    cudaMemsetAsync(count, 0, sizeof(int), s);
    if (!ib.slotOf) return;
    k_ras_classify<<<G.nbs * G.nbs, 128, 0, s>>>(G, ib, list, count);
}

void launch_box_slots(int nboxes, const int* list, const int* count, int* slotOfBox, cudaStream_t s) {
    cudaMemsetAsync(slotOfBox, 0xff, sizeof(int) * (size_t)nboxes, s);
    k_box_slots<<<(nboxes + 255) / 256, 256, 0, s>>>(list, count, slotOfBox);
}

void launch_ras_setup(int N, int b, int o, const RasIB& ib, double a0, double c, double inv_h, double dt,
                      const int* list, int nIB, double* inv64, float* inv32, int* info, cudaStream_t s) {
    const RasGeo G = ras_geo(N, b, o);
    const size_t smem = ras_setup_smem(b, o);
    cudaFuncSetAttribute(k_ras_setup, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_ras_setup<<<1 + nIB, 256, smem, s>>>(G, ib, a0, c, inv_h, dt, list, inv64, inv32, info);
}

void launch_ras_setup_big(int N, int b, int o, const RasIB& ib, double a0, double c, double inv_h, double dt,
                          const int* list, int first, int count, double* work, double* inv64, float* inv32, int* info,
                          cudaStream_t s) {
    const RasGeo G = ras_geo(N, b, o);
    const size_t smem = sizeof(double) * (2 * (size_t)G.ne + 32) + sizeof(int) * (32 + (size_t)G.ne);
    k_ras_setup_big<<<count, RAS_BIG_SETUP_THREADS, smem, s>>>(G, ib, a0, c, inv_h, dt, list, first, work, inv64,
                                                                inv32, info);
}

namespace {
template <typename T, int RA>
void launch_ras_apply_big(const RasGeo& G, const int* slotOfBox, const T* inv, T omega, const T* r, const T* x, T* xo,
                          cudaStream_t s) {
    using TL = RasTile<T>;
    const size_t smem = sizeof(T) * ((size_t)RAS_KC * G.nown + (size_t)RAS_KC * TL::NBX) + sizeof(int) * G.ne;
    static thread_local size_t allowed = 48 * 1024;   // dynamic shared memory the kernel is enabled for
    if (smem > allowed) {
        cudaFuncSetAttribute(k_ras_apply_big<T, RA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        allowed = smem;
    }
    const int tiles = (G.nbs * G.nbs + TL::NBX - 1) / TL::NBX;
    launch_pdl(k_ras_apply_big<T, RA>, dim3(tiles), dim3(32 * RAS_BW), smem, s, G, slotOfBox, inv, omega, r, x, xo);
}
}  // namespace

int ras_tc_npad(int b) { return (3 * b * b + 15) / 16 * 16; }
size_t ras_tc_pack_floats(int b, int o) {
    const RasGeo G = ras_geo(16, b, o);
    const int nch = (G.ne + RT_KC - 1) / RT_KC;
    return (size_t)nch * 2 * rt_bbytes(ras_tc_npad(b)) / 4;
}
void launch_ras_tc_pack(int b, int o, const double* inv64, float* pack, cudaStream_t s) {
    const RasGeo G = ras_geo(16, b, o);
    const int nch = (G.ne + RT_KC - 1) / RT_KC;
    const int64_t total = (int64_t)ras_tc_pack_floats(b, o);
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 8);
    k_ras_tc_pack<<<blocks, 256, 0, s>>>(inv64, G.ne, G.nown, ras_tc_npad(b), nch, pack);
}
// the IB-free boxes' correction on the tensor cores (FP32 levels): persistent blocks, one per SM, with
// as many inverse stages as the shared memory holds (all nch chunks where they fit).  False, and nothing
// launched, where the shared memory cannot hold two inverse stages.
bool launch_ras_apply_tc(int N, int b, int o, const int* slotOfBox, const float* pack, float omega, const float* r,
                         const float* x, float* xo, int* err, cudaStream_t s, int rowOff = 0, int npadGroup = 0,
                         int groups = 1, long long groupFloats = 0) {
    const RasGeo G = ras_geo(N, b, o);
    const int npad = npadGroup > 0 ? npadGroup : ras_tc_npad(b), nch = (G.ne + RT_KC - 1) / RT_KC;
    // owned rows per thread, rounded up to whole TMEM loads; narrow boxes keep two chunks of residual
    // loads in flight, 8 x 8 boxes (48 rows a thread) one
    const int nc = npad / 4 <= 16 ? 16 : 48;
    static thread_local int sms = 0, optin = 0, staticSmem[2] = {-1, -1};
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (sms <= 0) sms = 1;
        cudaFuncAttributes fa;
        staticSmem[0] = cudaFuncGetAttributes(&fa, k_ras_apply_tc<16, 2>) == cudaSuccess ? (int)fa.sharedSizeBytes : 1024;
        staticSmem[1] = cudaFuncGetAttributes(&fa, k_ras_apply_tc<48, 1>) == cudaSuccess ? (int)fa.sharedSizeBytes : 1024;
    }
    const size_t tables =
        2 * sizeof(int) * (size_t)nch * RT_KC + sizeof(int2) * (size_t)G.nown + 2 * sizeof(int) * RT_NB;
    const size_t aStage = 2 * (size_t)RT_ABYTES, bChunk = 2 * (size_t)rt_bbytes(npad);
    const size_t avail = (size_t)optin - (size_t)staticSmem[nc == 48];
    const int slotCols = npad <= 32 ? 32 : npad <= 64 ? 64 : npad <= 128 ? 128 : 256;
    // residual stages (= TMEM slots): as many as 512 TMEM columns and the shared memory left after the
    // whole inverse (or three of its stages) allow, 2 to RT_MAXNS
    int ns = std::min(RT_MAXNS, 512 / slotCols);
    const size_t bWant = (size_t)std::min(nch, 3) * bChunk;
    while (ns > 2 && tables + ns * aStage + bWant > avail) --ns;
    const size_t fixed = tables + (size_t)ns * aStage;
    int nsb = avail > fixed ? (int)std::min<size_t>((size_t)nch, (avail - fixed) / bChunk) : 0;
    nsb = std::min(nsb, RT_MAXSB);
    if (nsb < 2) return false;   // b + 2 o <= 16 leaves room for three inverse stages in 227 KB
    const size_t smem = fixed + (size_t)nsb * bChunk;
    static thread_local size_t allowed[2] = {48 * 1024, 48 * 1024};
    if (smem > allowed[nc == 48]) {
        if (nc == 48)
            cudaFuncSetAttribute(k_ras_apply_tc<48, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        else
            cudaFuncSetAttribute(k_ras_apply_tc<16, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        allowed[nc == 48] = smem;
    }
    const int ntiles = (G.nbs * G.nbs + RT_NB - 1) / RT_NB;
    // 16 worker warps and the issuing warp; row groups (16 x 16 boxes) side by side along y
    const dim3 grd(std::min(ntiles, sms), groups), blk(RT_THREADS + 32);
    if (nc == 16)
        launch_pdl(k_ras_apply_tc<16, 2>, grd, blk, smem, s, G, slotOfBox, pack, npad, nch, nsb, ns, rowOff,
                   groupFloats, omega, r, x, xo, err);
    else
        launch_pdl(k_ras_apply_tc<48, 1>, grd, blk, smem, s, G, slotOfBox, pack, npad, nch, nsb, ns, rowOff,
                   groupFloats, omega, r, x, xo, err);
    return true;
}

// ---- 16 x 16 boxes --------------------------------------------------------------------------
bool ras_huge(int b) { return b == RAS_BOX_HUGE; }
int ras_huge_n(int b, int o) { return (ras_ne(b, o) + 15) / 16 * 16; }
void launch_ras_huge_assemble(int N, int b, int o, double a0, double c, double inv_h, double* Aug, cudaStream_t s) {
    const RasGeo G = ras_geo(N, b, o);
    const int n = ras_huge_n(b, o);
    cudaMemsetAsync(Aug, 0, sizeof(double) * (size_t)n * 2 * n, s);
    k_ras_huge_assemble<<<(n + 255) / 256, 256, 0, s>>>(G, a0, c, inv_h, n, Aug);
}
void launch_ras_huge_extract(const double* Aug, const int* piv, int b, int o, double* inv64, float* inv32,
                             cudaStream_t s) {
    const int ne = ras_ne(b, o), n = ras_huge_n(b, o);
    k_ras_huge_extract<<<dim3((ne + 255) / 256, ne), 256, 0, s>>>(Aug, piv, n, ne, inv64, inv32);
}
void launch_ras_wb_count(int N, int b, int o, const RasIB& ib, const int* list, int nIB, int* cnt, cudaStream_t s) {
    if (nIB > 0) k_ras_wb_count<<<nIB, 256, 0, s>>>(ras_geo(N, b, o), ib, list, cnt);
}
void launch_ras_wb_fill(int N, int b, int o, const RasIB& ib, const int* list, int nIB, const int* offT, int* T,
                        cudaStream_t s) {
    if (nIB > 0) k_ras_wb_fill<<<nIB, 256, 0, s>>>(ras_geo(N, b, o), ib, list, offT, T);
}
void launch_ras_wb_setup(int N, int b, int o, const RasIB& ib, double dt, const int* list, int nIB, const int* offT,
                         const int* T, const long long* offW, const double* inv0, double* work, double* W, int* info,
                         int mmax, int mOneMax, cudaStream_t s) {
    if (nIB <= 0) return;
    const int nw = RAS_WB_THREADS / 32;
    const size_t smem = sizeof(double) * (3 * (size_t)mmax + 32) +
                        sizeof(int) * (32 + nw * WIN_SIZE + ((nw * WIN_SIZE) & 1)) + sizeof(double) * nw * WIN_SIZE;
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_ras_wb_setup, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_ras_wb_setup<<<nIB, RAS_WB_THREADS, smem, s>>>(ras_geo(N, b, o), ib, dt, list, offT, T, offW, inv0, work, W,
                                                     info, mOneMax);
}

// A large IB box's [I + E Q | E] (m x 2m, row-major) into the blocked Gauss-Jordan's layout, padded to
// m16 (a multiple of 16) with identity rows: Aug is m16 x 2 m16, [A | B] with A = I + E Q and B = E.
__global__ void k_ras_wb_pad(const double* __restrict__ Mx, int m, int m16, double* __restrict__ Aug) {
    const int i = blockIdx.y;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < 2 * m16; j += gridDim.x * blockDim.x) {
        double v = 0.0;
        if (i < m) {
            if (j < m) v = Mx[(size_t)i * 2 * m + j];
            else if (j >= m16 && j < m16 + m) v = Mx[(size_t)i * 2 * m + m + (j - m16)];
        } else if (j == i) {
            v = 1.0;
        }
        Aug[(size_t)i * 2 * m16 + j] = v;
    }
}
// W = A^{-1} B from the eliminated Aug: row a is the right half of pivot row piv[a]
__global__ void k_ras_wb_take(const double* __restrict__ Aug, const int* __restrict__ piv, int m, int m16,
                              double* __restrict__ Wb) {
    const int a = blockIdx.y;
    const double* row = Aug + (size_t)piv[a] * 2 * m16 + m16;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) Wb[(size_t)a * m + c] = row[c];
}
void launch_ras_wb_big(const double* Mx, int m, double* Aug, int* piv, void* work, int* info, double* Wb,
                       cudaStream_t s) {
    const int m16 = (m + 15) / 16 * 16;
    k_ras_wb_pad<<<dim3((2 * m16 + 255) / 256, m16), 256, 0, s>>>(Mx, m, m16, Aug);
    launch_gauss_jordan(Aug, m16, info, piv, work, s);
    k_ras_wb_take<<<dim3((m + 255) / 256, m), 256, 0, s>>>(Aug, piv, m, m16, Wb);
}
template <typename T>
void launch_ras_huge_apply(int N, int b, int o, const T* inv, T omega, const T* r, const T* x, T* xo, cudaStream_t s) {
    const RasGeo G = ras_geo(N, b, o);
    const size_t smem = sizeof(T) * RH_BX * (size_t)G.ne;
    static thread_local size_t allowed = 48 * 1024;
    if (smem > allowed) {
        cudaFuncSetAttribute(k_ras_huge_apply<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        allowed = smem;
    }
    // row splits: about two blocks per SM in all, at most one warp's row per split and warp
    const int boxBlocks = (G.nbs * G.nbs + RH_BX - 1) / RH_BX, nw = RH_THREADS / 32;
    const int splits = std::max(1, std::min((2 * 152 + boxBlocks - 1) / boxBlocks, (G.nown + nw - 1) / nw));
    launch_pdl(k_ras_huge_apply<T>, dim3(boxBlocks, splits), dim3(RH_THREADS), smem, s, G, inv, omega, r, x, xo);
}
template void launch_ras_huge_apply<float>(int, int, int, const float*, float, const float*, const float*, float*,
                                           cudaStream_t);
template void launch_ras_huge_apply<double>(int, int, int, const double*, double, const double*, const double*,
                                            double*, cudaStream_t);
// FP32 levels, spread over the GPU: every IB box's local solve in three launches over (box, chunk), so
// that the FP64 products run on every SM instead of one SM per IB box.
//   1. y = L_0^{-1} r_k on the rows T and on the owned rows, a warp per row;
//   2. z = W y_T, a warp per row;
//   3. xo(owned) = x(owned) + omega (y_own - (L_0^{-1})_{own,T} z), 32 owned rows per block and eight
//      partial sums per row, reading (L_0^{-1})_{T,own} (L_0 is symmetric) so that a warp's reads of one
//      row of the inverse are consecutive.
// The owned values of an IB box are written whole, from FP64 sums.  With a stiff structure the shared
// term y_own and the low-rank term nearly cancel, and the FP32 shared correction of those rows (already
// written by the kernel for all boxes) would carry its rounding, scaled by that cancellation, into the
// result.
constexpr int WB_ROWS = 32;   // rows per block in the first two launches
template <typename T>
__global__ void __launch_bounds__(256) k_ras_wb_y(RasGeo G, const int* __restrict__ list, const int* __restrict__ offT,
                                                  const int* __restrict__ Tl, const double* __restrict__ inv0,
                                                  const T* __restrict__ r, double* __restrict__ yT,
                                                  double* __restrict__ yOwn) {
    extern __shared__ double wb_rk[];   // ne: r_k
    pdl_entry();   // every block waits (a block with no rows too), so completion orders the three launches
    const int t0 = offT[blockIdx.x], m = offT[blockIdx.x + 1] - t0;
    const int a0 = blockIdx.y * WB_ROWS;   // rows a < m: T; a >= m: owned row a - m
    if (a0 >= m + G.nown) return;
    const int N = G.N, n = N * N, mk = N - 1, ne = G.ne;
    const int k = list[blockIdx.x];
    const int I = k % G.nbs, J = k / G.nbs, i0 = I * G.b - G.o, j0 = J * G.b - G.o;
    const int* Ts = Tl + t0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int q = threadIdx.x; q < ne; q += blockDim.x) {
        int comp, ii, jj;
        ras_dof(G, q, comp, ii, jj);
        wb_rk[q] = (double)r[(size_t)comp * n + (size_t)((j0 + jj) & mk) * N + ((i0 + ii) & mk)];
    }
    __syncthreads();
    const int a1 = min(m + G.nown, a0 + WB_ROWS);
    for (int a = a0 + warp; a < a1; a += nw) {
        const double* row = inv0 + (size_t)(a < m ? Ts[a] : ras_owned(G, a - m)) * ne;
        double acc = 0.0;
        for (int t = lane; t < ne; t += 32) acc += row[t] * wb_rk[t];
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0) {
            if (a < m)
                yT[t0 + a] = acc;
            else
                yOwn[(size_t)blockIdx.x * G.nown + (a - m)] = acc;
        }
    }
}
__global__ void __launch_bounds__(256) k_ras_wb_z(const int* __restrict__ offT, const long long* __restrict__ offW,
                                                  const double* __restrict__ Wd, const double* __restrict__ yT,
                                                  double* __restrict__ z) {
    pdl_entry();
    const int t0 = offT[blockIdx.x], m = offT[blockIdx.x + 1] - t0;
    const int a0 = blockIdx.y * WB_ROWS;
    if (a0 >= m) return;
    const double* Wb = Wd + offW[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int a1 = min(m, a0 + WB_ROWS);
    for (int a = a0 + warp; a < a1; a += nw) {
        const double* row = Wb + (size_t)a * m;
        double acc = 0.0;
        for (int t = lane; t < m; t += 32) acc += row[t] * yT[t0 + t];
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0) z[t0 + a] = acc;
    }
}
template <typename T>
__global__ void __launch_bounds__(256) k_ras_wb_out(RasGeo G, const int* __restrict__ list, const int* __restrict__ offT,
                                                    const int* __restrict__ Tl, const double* __restrict__ inv0,
                                                    const double* __restrict__ z, const double* __restrict__ yOwn,
                                                    T omega, const T* x, T* xo) {
    // 32 owned rows per block; warp w sums the terms a = w, w + 8, ... of each row (lane = row), and
    // the eight partial sums are added in warp order
    __shared__ double part[8][32];
    pdl_entry();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int rr = blockIdx.y * 32 + lane;
    const bool live = rr < G.nown;
    const int N = G.N, n = N * N, ne = G.ne, bb = G.b * G.b;
    const int t0 = offT[blockIdx.x], m = offT[blockIdx.x + 1] - t0;
    const int* Ts = Tl + t0;
    const int q = live ? ras_owned(G, rr) : 0;
    double acc = 0.0;
    if (live)
        for (int a = w; a < m; a += 8) acc += inv0[(size_t)Ts[a] * ne + q] * z[t0 + a];
    part[w][lane] = acc;
    __syncthreads();
    if (w != 0 || !live) return;
    double sum = part[0][lane];
#pragma unroll
    for (int v = 1; v < 8; ++v) sum += part[v][lane];
    const int k = list[blockIdx.x];
    const int I = k % G.nbs, J = k / G.nbs;
    const int comp = rr / bb, rem = rr - comp * bb;
    const size_t d = (size_t)comp * n + (size_t)(J * G.b + rem / G.b) * N + I * G.b + rem % G.b;
    const double delta = yOwn[(size_t)blockIdx.x * G.nown + rr] - sum;
    xo[d] = (T)((x ? (double)x[d] : 0.0) + (double)omega * delta);
}

template <typename T>
void launch_ras_wb_apply(int N, int b, int o, const RasIB& ib, double a0, double c, double inv_h, double dt,
                         const int* list, int nIB, const int* offT, const int* Tl, const long long* offW,
                         const double* W, const double* inv0, int mmax, T omega, const T* r, T* xo, cudaStream_t s,
                         double* scratch, const T* x) {
    if (nIB <= 0) return;
    const RasGeo G = ras_geo(N, b, o);
    if (sizeof(T) == 4 && scratch) {   // FP32: the IB boxes' local solves over the whole GPU
        // the caller's scratch holds (2 mmax + nown) nIB values
        double* yT = scratch;
        double* z = scratch + (size_t)mmax * nIB;
        double* yOwn = z + (size_t)mmax * nIB;
        const int chunks = (mmax + WB_ROWS - 1) / WB_ROWS, chunksY = (mmax + G.nown + WB_ROWS - 1) / WB_ROWS;
        const size_t smem = sizeof(double) * (size_t)G.ne;
        static thread_local size_t allowedY = 48 * 1024;
        if (smem > allowedY) {
            cudaFuncSetAttribute(k_ras_wb_y<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            allowedY = smem;
        }
        launch_pdl(k_ras_wb_y<T>, dim3(nIB, chunksY), dim3(256), smem, s, G, list, offT, Tl, inv0, r, yT, yOwn);
        launch_pdl(k_ras_wb_z, dim3(nIB, chunks), dim3(256), 0, s, offT, offW, W, (const double*)yT, z);
        launch_pdl(k_ras_wb_out<T>, dim3(nIB, (G.nown + 31) / 32), dim3(256), 0, s, G, list, offT, Tl, inv0,
                   (const double*)z, (const double*)yOwn, omega, x, xo);
        return;
    }
    const size_t smem = sizeof(double) * (4 * (size_t)G.ne + (size_t)mmax);
    static thread_local size_t allowed = 48 * 1024;
    if (smem > allowed) {
        cudaFuncSetAttribute(k_ras_wb_apply<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        allowed = smem;
    }
    launch_pdl(k_ras_wb_apply<T>, dim3(nIB), dim3(256), smem, s, G, ib, a0, c, inv_h, dt, list, offT, Tl, offW, W,
               inv0, omega, r, xo);
}
template void launch_ras_wb_apply<float>(int, int, int, const RasIB&, double, double, double, double, const int*, int,
                                         const int*, const int*, const long long*, const double*, const double*, int,
                                         float, const float*, float*, cudaStream_t, double*, const float*);
template void launch_ras_wb_apply<double>(int, int, int, const RasIB&, double, double, double, double, const int*,
                                          int, const int*, const int*, const long long*, const double*,
                                          const double*, int, double, const double*, double*, cudaStream_t, double*,
                                          const double*);
size_t ras_tc_group_floats(int b, int o) {
    const RasGeo G = ras_geo(16, b, o);
    const int nch = (G.ne + RT_KC - 1) / RT_KC;
    return (size_t)nch * 2 * rt_bbytes(RAS_TC_GROUP) / 4;
}
void launch_ras_tc_pack_rows(int b, int o, const double* inv0, int g, float* out, cudaStream_t s) {
    const RasGeo G = ras_geo(16, b, o);
    const int nch = (G.ne + RT_KC - 1) / RT_KC;
    const int64_t total = (int64_t)ras_tc_group_floats(b, o);
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 8);
    k_ras_tc_pack_rows<<<blocks, 256, 0, s>>>(G, inv0, g * RAS_TC_GROUP, RAS_TC_GROUP, nch, out);
}
bool launch_ras_apply_tc_groups(int N, int b, int o, const float* pack, int groups, float omega, const float* r,
                                const float* x, float* xo, int* err, cudaStream_t s) {
    return launch_ras_apply_tc(N, b, o, nullptr, pack, omega, r, x, xo, err, s, 0, RAS_TC_GROUP, groups,
                               (long long)ras_tc_group_floats(b, o));
}

template <typename T>
void launch_ras_apply(int N, int b, int o, const int* slotOfBox, const int* list, int nIB, const T* inv, T omega,
                      const T* r, const T* x, T* xo, cudaStream_t s, const float* tcPack, int* err) {
    const RasGeo G = ras_geo(N, b, o);
    if constexpr (sizeof(T) == 4) {
        // IB-free boxes on the tensor cores, IB boxes by their own inverses
        if (tcPack && launch_ras_apply_tc(N, b, o, slotOfBox, tcPack, omega, r, x, xo, err, s)) {
            if (nIB > 0) {
                if (G.e > RAS_EMAX_SMEM)
                    launch_pdl(k_ras_apply_big_ib<T>, dim3(nIB), dim3(256), sizeof(T) * ((size_t)G.ne + 4 * (size_t)G.nown),
                               s, G, list, inv, omega, r, x, xo);
                else
                    launch_pdl(k_ras_apply_ib<T>, dim3(nIB), dim3(64 * RAS_QS), sizeof(T) * (G.ne + 64 * RAS_QS), s, G, list,
                               inv, omega, r, x, xo);
            }
            return;
        }
    }
    if (G.e > RAS_EMAX_SMEM) {   // rows per lane: nown <= 32 RA
        if (G.nown <= 32)
            launch_ras_apply_big<T, 1>(G, slotOfBox, inv, omega, r, x, xo, s);
        else if (G.nown <= 64)
            launch_ras_apply_big<T, 2>(G, slotOfBox, inv, omega, r, x, xo, s);
        else
            launch_ras_apply_big<T, 6>(G, slotOfBox, inv, omega, r, x, xo, s);
        if (nIB > 0)
            launch_pdl(k_ras_apply_big_ib<T>, dim3(nIB), dim3(256), sizeof(T) * ((size_t)G.ne + 4 * (size_t)G.nown), s,
                       G, list, inv, omega, r, x, xo);
        return;
    }
    const size_t smem = sizeof(T) * (((size_t)G.ne * G.nown + 3) / 4 * 4 + (size_t)RAS_WARPS * G.ne * RAS_GB) +
                        sizeof(int) * G.ne;
    static thread_local size_t cachedSmem = 0;   // persistent grid: the blocks resident at once, per size
    static thread_local int resident = 1;
    if (smem != cachedSmem) {
        cudaFuncSetAttribute(k_ras_apply<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_ras_apply<T>, 32 * RAS_WARPS, smem);
        resident = (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
        cachedSmem = smem;
    }
    const int ngroups = G.nbs * G.nbs / RAS_GB;
    const int want = (ngroups + RAS_WARPS - 1) / RAS_WARPS;
    const int blocks = want < resident ? want : resident;
    launch_pdl(k_ras_apply<T>, dim3(blocks), dim3(32 * RAS_WARPS), smem, s, G, slotOfBox, inv, omega, r, x, xo);
    if (nIB > 0)
        launch_pdl(k_ras_apply_ib<T>, dim3(nIB), dim3(64 * RAS_QS), sizeof(T) * (G.ne + 64 * RAS_QS), s, G, list, inv,
                   omega, r, x, xo);
}
template void launch_ras_apply<float>(int, int, int, const int*, const int*, int, const float*, float, const float*,
                                      const float*, float*, cudaStream_t, const float*, int*);
template void launch_ras_apply<double>(int, int, int, const int*, const int*, int, const double*, double,
                                       const double*, const double*, double*, cudaStream_t, const float*, int*);

}  // namespace sib
