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
// K-major layout of tcgen05.cuh with LBO = 144 bytes (a 128-byte row of core matrices plus 16 bytes, so
// that the residual gather stores into shared memory without bank conflicts) and SBO = 8 LBO.
constexpr int RT_NB = 128, RT_KC = 32;
constexpr int RT_LBO = 144, RT_SBO = 8 * RT_LBO;
constexpr int RT_THREADS = 256;
constexpr int RT_WAIT = 1 << 22;   // bounded waits on the copies and the MMAs
constexpr int RT_ABYTES = (RT_NB / 8) * RT_SBO;   // one of hi, lo of the residual tile's chunk

// byte offset of (row, k) in a K-major chunk of RT_KC values per row
__host__ __device__ inline int rt_off(int row, int k) {
    return (row >> 3) * RT_SBO + (k >> 2) * RT_LBO + (row & 7) * 16 + (k & 3) * 4;
}

// Packs the shared inverse's owned rows (slot 0 of inv64, [q][row]) for k_ras_apply_tc: chunk c holds
// rows 0 .. npad - 1 and dofs q = 32 c .. 32 c + 31 in the K-major layout, its hi part then its lo
// part; rows past nown, dofs past ne and the 16-byte gaps hold zeros.
__global__ void k_ras_tc_pack(const double* __restrict__ inv64, int ne, int nown, int npad, int nch,
                              float* __restrict__ out) {
    const int chunkWords = (npad / 8) * RT_SBO / 4;
    const int64_t total = (int64_t)nch * 2 * chunkWords;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(idx / (2 * chunkWords));
        const int rem = (int)(idx - (int64_t)c * 2 * chunkWords);
        const int part = rem / chunkWords, byte = (rem - part * chunkWords) * 4;
        const int grp = byte / RT_SBO, b2 = byte - grp * RT_SBO, k4 = b2 / RT_LBO, b3 = b2 - k4 * RT_LBO;
        float val = 0.0f;
        if (b3 < 128) {
            const int row = grp * 8 + b3 / 16, q = c * RT_KC + k4 * 4 + (b3 & 15) / 4;
            if (row < nown && q < ne) {
                const double v = inv64[(size_t)q * nown + row];
                const float hi = tf32_rna((float)v);
                val = part == 0 ? hi : tf32_rna((float)(v - (double)hi));
            }
        }
        out[idx] = val;
    }
}

// One correction of the IB-free boxes: xo(owned) = x(owned) + omega (Inv r_k)(owned) (x == nullptr: 0).
// Persistent blocks over tiles of RT_NB boxes.  Per K chunk (two shared-memory stages): the block
// gathers the tile's residual windows (warp w: boxes w + 8 j, lane: the chunk's dof), split into hi and
// lo; one thread fetches the inverse's packed chunk by a bulk copy, waits for it, and issues the
// chunk's 3 x 4 MMAs into a TMEM slot of its own (two slots, alternating), committed to the stage's
// barrier.  While the next chunk's MMAs run, every thread adds the previous chunk's slot into FP32
// totals in registers: each chunk is summed apart and then added to the total, as the CUDA-core form
// does (one long accumulation over all ne terms loses accuracy to their cancellation).  Warps 0-3 hold
// the owned rows 0 .. npad/2 - 1 of boxes 32 w + lane, warps 4-7 the others.  After a tile, the totals
// are written.  Every wait is bounded: a block that gives up writes SIB_DEV_ERR_TMA_WAIT into the error
// word, waits again (bounded) for its last MMAs and copy, frees its TMEM and leaves.
constexpr int RT_MAXCOL = 96;   // owned rows per thread: npad / 2 <= 96 (npad <= 192)
template <int NC>
__global__ void __launch_bounds__(RT_THREADS, 1)
    k_ras_apply_tc(RasGeo G, const int* __restrict__ slotOfBox, const float* __restrict__ pack, int npad, int nch,
                   float omega, const float* __restrict__ r, const float* x, float* xo, int* err) {
    extern __shared__ __align__(1024) unsigned char rt_smem[];
    __shared__ __align__(8) uint64_t tma_bar[2];
    __shared__ __align__(8) uint64_t mma_bar[2];
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int bBytes = (npad / 8) * RT_SBO;
    const int stageBytes = 2 * RT_ABYTES + 2 * bBytes;
    int* qtab = reinterpret_cast<int*>(rt_smem + 2 * stageBytes);
    for (int q = tid; q < G.ne; q += RT_THREADS) {
        int comp, ii, jj;
        ras_dof(G, q, comp, ii, jj);
        qtab[q] = comp | (ii << 8) | (jj << 16);
    }
    if (tid == 0) {
        for (int k = 0; k < 2; ++k) {
            mbar_init(&tma_bar[k], 1);
            mbar_init(&mma_bar[k], 1);
        }
        fence_mbar_init();
    }
    // two accumulator slots of npad columns each
    const uint32_t slotCols = npad <= 32 ? 32u : npad <= 64 ? 64u : npad <= 128 ? 128u : 256u;
    const uint32_t ncols = 2 * slotCols;
    if (warp == 0) tmem_alloc(&tmem_base, ncols);
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = umma_idesc_tf32(RT_NB, npad);
    pdl_entry();
    const int N = G.N, n = N * N, m = N - 1, bb = G.b * G.b, nown = G.nown;
    const int nboxes = G.nbs * G.nbs, ntiles = (nboxes + RT_NB - 1) / RT_NB;
    const int half = npad / 2;                       // a multiple of 8
    const int cbase = warp < 4 ? 0 : half;           // this thread's first owned row
    const uint32_t lanes = (uint32_t)(32 * (warp & 3)) << 16;
    uint32_t g = 0;          // chunks this block has staged (stage and slot g & 1); every one is committed
    bool ok = true;
    // adds the accumulator slot of chunk gc into the totals (its MMAs complete and waited for)
    auto add_slot = [&](uint32_t gc, float (&tot)[NC]) {
        const uint32_t base = tmem + lanes + (gc & 1) * slotCols + (uint32_t)cbase;
#pragma unroll
        for (int c0 = 0; c0 < NC; c0 += 16) {
            if (c0 < half) {
                uint32_t a[16];
                tmem_ld16(base + (uint32_t)c0, a);
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (c0 + j < NC) tot[c0 + j] += __uint_as_float(a[j]);
            }
        }
    };
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int k0 = tile * RT_NB;
        float tot[NC];
#pragma unroll
        for (int j = 0; j < NC; ++j) tot[j] = 0.0f;
        for (int c = 0; c < nch; ++c, ++g) {
            const int st = g & 1;
            unsigned char* base = rt_smem + st * stageBytes;
            unsigned char* Ahi = base;
            unsigned char* Alo = base + RT_ABYTES;
            unsigned char* Bhi = base + 2 * RT_ABYTES;
            unsigned char* Blo = Bhi + bBytes;
            if (g >= 2) {   // the MMAs of chunk g - 2 read this stage (and its slot was added up)
                const bool w = mbar_wait_bounded(&mma_bar[st], ((g >> 1) - 1) & 1, RT_WAIT);
                if (!__syncthreads_and(w)) {
                    ok = false;
                    break;
                }
                tc_fence_after_sync();
            }
            if (tid == 0) {
                mbar_expect_tx(&tma_bar[st], (uint32_t)(2 * bBytes));
                bulk_load(Bhi, reinterpret_cast<const unsigned char*>(pack) + (size_t)c * 2 * bBytes,
                          (uint32_t)(2 * bBytes), &tma_bar[st]);
            }
            const int q = c * RT_KC + lane;
            const int code = q < G.ne ? qtab[q] : 0;
            float v[RT_NB / 8];
#pragma unroll
            for (int j = 0; j < RT_NB / 8; ++j) {   // every load issued before the first store
                const int kb = k0 + warp + 8 * j;
                v[j] = 0.0f;
                if (q < G.ne && kb < nboxes) {
                    const int gi = ((kb % G.nbs) * G.b - G.o + ((code >> 8) & 0xff)) & m;
                    const int gj = ((kb / G.nbs) * G.b - G.o + (code >> 16)) & m;
                    v[j] = r[(size_t)(code & 0xff) * n + (size_t)gj * N + gi];
                }
            }
#pragma unroll
            for (int j = 0; j < RT_NB / 8; ++j) {
                const float hi = tf32_rna(v[j]);
                const int off = rt_off(warp + 8 * j, lane);
                *reinterpret_cast<float*>(Ahi + off) = hi;
                *reinterpret_cast<float*>(Alo + off) = tf32_rna(v[j] - hi);
            }
            fence_proxy_async_smem();
            tc_fence_before_sync();
            __syncthreads();   // the stage is written; the slot of chunk g - 2 has been read by everyone
            bool w0 = true;
            if (tid == 0) {
                w0 = mbar_wait_bounded(&tma_bar[st], (g >> 1) & 1, RT_WAIT);
                if (w0) {
                    tc_fence_after_sync();
                    const uint32_t d = tmem + (uint32_t)st * slotCols;
                    const uint32_t ah = tc_smem_u32(Ahi), al = tc_smem_u32(Alo);
                    const uint32_t bh = tc_smem_u32(Bhi), bl = tc_smem_u32(Blo);
#pragma unroll
                    for (int t = 0; t < RT_KC / 8; ++t) {
                        const uint32_t o = (uint32_t)(t * 2 * RT_LBO);
                        const uint64_t dah = umma_desc(ah + o, RT_LBO, RT_SBO), dal = umma_desc(al + o, RT_LBO, RT_SBO);
                        const uint64_t dbh = umma_desc(bh + o, RT_LBO, RT_SBO), dbl = umma_desc(bl + o, RT_LBO, RT_SBO);
                        umma_tf32(d, dah, dbh, idesc, t > 0);   // the chunk's slot starts from zero
                        umma_tf32(d, dah, dbl, idesc, true);
                        umma_tf32(d, dal, dbh, idesc, true);
                    }
                }
                umma_commit(&mma_bar[st]);   // arrives once the MMAs issued so far are complete
            }
            if (!__syncthreads_and(w0)) {
                ok = false;
                ++g;   // this chunk's commit was issued
                break;
            }
            if (c > 0) {   // the previous chunk's slot, while this chunk's MMAs run
                const uint32_t gp = g - 1;
                const bool w = mbar_wait_bounded(&mma_bar[gp & 1], (gp >> 1) & 1, RT_WAIT);
                if (!__syncthreads_and(w)) {
                    ok = false;
                    ++g;
                    break;
                }
                tc_fence_after_sync();
                add_slot(gp, tot);
            }
        }
        if (!ok) break;
        // the tile's last chunk
        const uint32_t gl = g - 1;
        const bool w = mbar_wait_bounded(&mma_bar[gl & 1], (gl >> 1) & 1, RT_WAIT);
        if (!__syncthreads_and(w)) {
            ok = false;
            break;
        }
        tc_fence_after_sync();
        add_slot(gl, tot);
        const int kb = k0 + 32 * (warp & 3) + lane;
        if (kb < nboxes && !(slotOfBox && slotOfBox[kb] >= 0)) {
            const int I = kb % G.nbs, J = kb / G.nbs;
#pragma unroll
            for (int j = 0; j < NC; ++j) {
                const int rr = cbase + j;
                if (j < half && rr < nown) {
                    const int comp = rr / bb, rem = rr - comp * bb;
                    const size_t d = (size_t)comp * n + (size_t)(J * G.b + rem / G.b) * N + I * G.b + rem % G.b;
                    xo[d] = (x ? x[d] : 0.0f) + omega * tot[j];
                }
            }
        }
        tc_fence_before_sync();
        __syncthreads();   // the slots are read before the next tile's MMAs overwrite them
        tc_fence_after_sync();
    }
    if (!ok) {   // report, then let this block's last MMAs and copy drain before the TMEM is freed
        if (tid == 0 && err) *(volatile int*)err = SIB_DEV_ERR_TMA_WAIT;
        if (g > 0) {
            const uint32_t gl = g - 1;
            mbar_wait_bounded(&mma_bar[gl & 1], (gl >> 1) & 1, RT_WAIT);
            mbar_wait_bounded(&tma_bar[gl & 1], (gl >> 1) & 1, RT_WAIT);
        }
    }
    tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, ncols);
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
    return (size_t)nch * 2 * (ras_tc_npad(b) / 8) * RT_SBO / 4;
}
void launch_ras_tc_pack(int b, int o, const double* inv64, float* pack, cudaStream_t s) {
    const RasGeo G = ras_geo(16, b, o);
    const int nch = (G.ne + RT_KC - 1) / RT_KC;
    const int64_t total = (int64_t)ras_tc_pack_floats(b, o);
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 8);
    k_ras_tc_pack<<<blocks, 256, 0, s>>>(inv64, G.ne, G.nown, ras_tc_npad(b), nch, pack);
}
// the IB-free boxes' correction on the tensor cores (FP32 levels): persistent blocks, one per SM
void launch_ras_apply_tc(int N, int b, int o, const int* slotOfBox, const float* pack, float omega, const float* r,
                         const float* x, float* xo, int* err, cudaStream_t s) {
    const RasGeo G = ras_geo(N, b, o);
    const int npad = ras_tc_npad(b), nch = (G.ne + RT_KC - 1) / RT_KC;
    const size_t smem = 2 * (2 * (size_t)RT_ABYTES + 2 * (size_t)(npad / 8) * RT_SBO) + sizeof(int) * (size_t)G.ne;
    static thread_local size_t allowed = 48 * 1024;
    static thread_local int sms = 0;
    if (smem > allowed) {
        cudaFuncSetAttribute(k_ras_apply_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_ras_apply_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_ras_apply_tc<RT_MAXCOL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        allowed = smem;
    }
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    const int ntiles = (G.nbs * G.nbs + RT_NB - 1) / RT_NB;
    const dim3 grd(std::min(ntiles, sms)), blk(RT_THREADS);
    // each thread keeps npad / 2 owned rows of one box: a compile-time bound for the register totals
    if (npad <= 32)
        launch_pdl(k_ras_apply_tc<16>, grd, blk, smem, s, G, slotOfBox, pack, npad, nch, omega, r, x, xo, err);
    else if (npad <= 64)
        launch_pdl(k_ras_apply_tc<32>, grd, blk, smem, s, G, slotOfBox, pack, npad, nch, omega, r, x, xo, err);
    else
        launch_pdl(k_ras_apply_tc<RT_MAXCOL>, grd, blk, smem, s, G, slotOfBox, pack, npad, nch, omega, r, x, xo, err);
}

template <typename T>
void launch_ras_apply(int N, int b, int o, const int* slotOfBox, const int* list, int nIB, const T* inv, T omega,
                      const T* r, const T* x, T* xo, cudaStream_t s, const float* tcPack, int* err) {
    const RasGeo G = ras_geo(N, b, o);
    if constexpr (sizeof(T) == 4) {
        if (tcPack) {   // IB-free boxes on the tensor cores, IB boxes by their own inverses
            launch_ras_apply_tc(N, b, o, slotOfBox, tcPack, omega, r, x, xo, err, s);
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
