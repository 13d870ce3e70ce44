// Internal declarations of libsib: kernel argument blocks, launchers and the solver context.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "sib.h"

namespace sib {

// Grid kernels work on tiles of TX x TY cells (one thread per cell); smaller levels use
// min(N, TX) x min(N, TY).  The IB "active tile" flags use the same tiles.
constexpr int TX = 32;
constexpr int TY = 8;
constexpr int MAX_N = 8192;
// Assembled IB operator windows: offsets -WR..WR in each direction, WD = 2 WR + 1 per side.
constexpr int WR = 4;
constexpr int WD = 2 * WR + 1;
constexpr int WIN_SIZE = WD * WD;

// ------------------------------------------------------------------------------------------
// Programmatic dependent launch: every kernel waits for the grids it depends on before touching
// memory, then lets its dependents be scheduled (they start waiting while this grid finishes), so
// consecutive kernels of a stream or graph overlap their launch latency.  Dependents become
// eligible only after every block of this grid has started, so early triggering cannot starve it.
__device__ __forceinline__ void pdl_entry() {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 900
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
#endif
}

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kern, args...);
}

// ------------------------------------------------------------------------------------------
// Morton order of a cell (i, j): bits of i on even positions, bits of j on odd positions.
// The bins of level l are the Morton codes of the fine-level bins shifted right by 2(lmax-l).
__host__ __device__ inline uint32_t part1by1(uint32_t x) {
    x &= 0x0000ffffu;
    x = (x | (x << 8)) & 0x00ff00ffu;
    x = (x | (x << 4)) & 0x0f0f0f0fu;
    x = (x | (x << 2)) & 0x33333333u;
    x = (x | (x << 1)) & 0x55555555u;
    return x;
}
__host__ __device__ inline uint32_t morton(uint32_t i, uint32_t j) { return part1by1(i) | (part1by1(j) << 1); }

// ------------------------------------------------------------------------------------------
// Arguments of the MAC-grid stencil kernels on one level.
template <typename T>
struct GridK {
    int N, tx, ty, ntx, lgtx, lgty;
    T inv_h;       // 1/h
    T a0;          // rho/dt + 4 mu / h^2   (diagonal of A)
    T c;           // mu / h^2              (off-diagonal magnitude of A)
    T dt;
    T omega;
    const T* fib;                    // [S K J]^l u on the faces (2 n), valid where the tile is active
    const T* ibd;                    // 4 n: B(f,f) on u faces, B(u_ij,u_i+1j), B(f,f) on v, B(v_ij,v_ij+1)
    const unsigned char* tile;       // per-tile IB flag (dilated by one tile), may be null
    const T* dinv;                   // SC: 1/diag(A_IB) on u and v faces, 1/diag(D diag(A_IB)^-1 G) on cells
    const T* pf;                     // Vanka: 7 n patch factors per cell (A_u^{-1}: 00, 01, 11; A_v^{-1}: 00, 01,
                                     // 11; 1 / pressure Schur complement), computed at set-up
    int* err;                        // host-visible error word (SIB_DEV_ERR_*), may be null
};

// Codes a kernel writes to the context's error word when a bounded wait gives up.
constexpr int SIB_DEV_ERR_TMA_WAIT = 1;   // a tile copy did not complete

// Constants of the Vanka patch solve for cells without IB entries (the patch matrix is the same
// for all of them): A^{-1} = [[ai0, ai1], [ai1, ai0]], s = A^{-1}(1/h, -1/h) = (s0, -s0), and the
// inverse of the pressure Schur complement 1 / (g^T s_u + g^T s_v).
template <typename T>
struct VankaBulk {
    T ai0, ai1, s0, invS;
};

// Chebyshev coefficients of two iterations from x0 = 0 on [lo, hi] lambda_max:
//   x2 = (1 + c1) d0 + c2 Dinv (q - Op d0),  d0 = Dinv q / theta
template <typename T>
struct Cheb2 {
    T inv_theta, one_c1, c2;
};

// Arguments of the marker kernels on one level (per velocity component c = 0, 1).
template <typename T>
struct IBK {
    int N, W, M;
    int shift;                       // Morton shift from fine bins to this level's bins
    const int* base[2];              // packed stencil origin (bj << 16) | bi, per marker
    const T* wgt[2];                 // per marker 8 weights: wx[0..3], wy[0..3]
    const int* binStart[2];          // N*N + 1, Morton-indexed ranges into sorted[]
    const int* sorted[2];            // marker ids in Morton order of their fine stencil origin
    T inv_h2;
};

// ------------------------------------------------------------------------------------------
// Box RAS smoother (kernels_ras.cu): where the level's IB windows live (slotOf == nullptr: no IB).
struct RasIB {
    const int* slotOf;       // tile -> window slot, -1 without IB entries
    const double* win;       // FP64 windows of the level
    int tx, ty, ntx;         // tile geometry of the level
};
// Subdomains up to RAS_EMAX_SMEM cells wide are set up and applied in shared memory; wider ones, up to
// RAS_EMAX cells (ne <= 800), are eliminated in a global workspace and applied as a batched product.
constexpr int RAS_EMAX_SMEM = 6;
constexpr int RAS_EMAX = 16;
bool ras_big(int b, int o);
size_t ras_setup_smem(int b, int o);
int ras_ne(int b, int o);
void launch_ras_classify(int N, int b, int o, const RasIB& ib, int* list, int* count, cudaStream_t s);
void launch_box_slots(int nboxes, const int* list, const int* count, int* slotOfBox, cudaStream_t s);
void launch_ras_setup(int N, int b, int o, const RasIB& ib, double a0, double c, double inv_h, double dt,
                      const int* list, int nIB, double* inv64, float* inv32, int* info, cudaStream_t s);
// wide subdomains: matrices first .. first + count - 1 (0: the shared one, s > 0: box list[s - 1]), each
// eliminated in its own ne x ne FP64 block of `work`
void launch_ras_setup_big(int N, int b, int o, const RasIB& ib, double a0, double c, double inv_h, double dt,
                          const int* list, int first, int count, double* work, double* inv64, float* inv32, int* info,
                          cudaStream_t s);
// the shared-inverse kernel, then (nIB > 0) one block per listed IB box
// tcPack != nullptr (FP32): the IB-free boxes' correction runs on the tensor cores from the packed
// shared inverse (launch_ras_tc_pack); err receives SIB_DEV_ERR_TMA_WAIT if one of its waits gives up
template <typename T>
void launch_ras_apply(int N, int b, int o, const int* slotOfBox, const int* list, int nIB, const T* inv, T omega,
                      const T* r, const T* x, T* xo, cudaStream_t s, const float* tcPack = nullptr,
                      int* err = nullptr);
// the shared inverse (slot 0 of the FP64 inverses) packed for the tensor-core correction: hi and lo
// TF32 parts in K-major chunks of 32 dofs; ras_tc_pack_floats gives its size
size_t ras_tc_pack_floats(int b, int o);
void launch_ras_tc_pack(int b, int o, const double* inv64, float* pack, cudaStream_t s);
// 16 x 16 boxes (subdomains up to 24 cells, ne <= 1,776): the full shared inverse of the IB-free
// subdomain operator by the blocked Gauss-Jordan (order ras_huge_n, ne padded to a multiple of 16) and a
// low-rank (Woodbury) update of it for the IB boxes: T lists (IB-touched dofs, ascending), W = (I + E Q)^-1 E
// per box (row-major |T| x |T| at offW); the shared correction of every box, then the IB boxes' update
constexpr int RAS_BOX_HUGE = 16;
constexpr int RAS_TC_GROUP = 192;   // owned rows per tensor-core row group with 16 x 16 boxes (768 = 4 x 192)
// 16 x 16 boxes: levels with fewer boxes than this take the CUDA-core correction, split over rows, even
// with the tensor-core option on (a few tiles of 128 boxes leave the tensor-core form a few CTAs, each
// walking the whole K = 1,776 in sequence)
constexpr int RAS_TC_MIN_BOXES = 1024;
bool ras_huge(int b);
int ras_huge_n(int b, int o);
void launch_ras_huge_assemble(int N, int b, int o, double a0, double c, double inv_h, double* Aug, cudaStream_t s);
void launch_ras_huge_extract(const double* Aug, const int* piv, int b, int o, double* inv64, float* inv32,
                             cudaStream_t s);
void launch_ras_wb_count(int N, int b, int o, const RasIB& ib, const int* list, int nIB, int* cnt, cudaStream_t s);
void launch_ras_wb_fill(int N, int b, int o, const RasIB& ib, const int* list, int nIB, const int* offT, int* T,
                        cudaStream_t s);
void launch_ras_wb_setup(int N, int b, int o, const RasIB& ib, double dt, const int* list, int nIB, const int* offT,
                         const int* T, const long long* offW, const double* inv0, double* work, double* W, int* info,
                         int mmax, int mOneMax, cudaStream_t s);
// boxes with |T| > RAS_WB_ONE_MAX: launch_ras_wb_setup only fills their [I + E Q | E] (Mx, m x 2m); this
// eliminates it by the blocked Gauss-Jordan (Aug: m16 x 2 m16, piv: m16, work: gauss_jordan_work_bytes(m16),
// m16 = m rounded up to 16) and writes W (m x m)
constexpr int RAS_WB_ONE_MAX = 256;
void launch_ras_wb_big(const double* Mx, int m, double* Aug, int* piv, void* work, int* info, double* Wb,
                       cudaStream_t s);
template <typename T>
void launch_ras_huge_apply(int N, int b, int o, const T* inv, T omega, const T* r, const T* x, T* xo, cudaStream_t s);
template <typename T>
void launch_ras_wb_apply(int N, int b, int o, const RasIB& ib, double a0, double c, double inv_h, double dt,
                         const int* list, int nIB, const int* offT, const int* Tl, const long long* offW,
                         const double* W, const double* inv0, int mmax, T omega, const T* r, T* xo, cudaStream_t s,
                         double* scratch = nullptr, const T* x = nullptr);
// (FP32 with scratch, (2 mmax + 3 b^2) nIB values: three launches, which write the IB boxes' owned values
// whole from x, distinct from xo; x == nullptr: zero)
size_t ras_tc_group_floats(int b, int o);
void launch_ras_tc_pack_rows(int b, int o, const double* inv0, int g, float* out, cudaStream_t s);
// the 16 x 16 boxes' shared correction on the tensor cores, all `groups` row groups of RAS_TC_GROUP owned
// rows in one launch (pack: the groups' packed slices, ras_tc_group_floats apart)
bool launch_ras_apply_tc_groups(int N, int b, int o, const float* pack, int groups, float omega, const float* r,
                                const float* x, float* xo, int* err, cudaStream_t s);

// ------------------------------------------------------------------------------------------
// Levels 1 and 0 of the V-cycle in one thread block (kernels_small.cu).
template <typename T>
struct SmallArgs {
    GridK<T> g;                 // level 1; its set-up arrays (ibd, dinv, tile flags) in global memory
    Cheb2<T> ka, km;            // SC Chebyshev coefficients of level 1
    const T* b;                 // level-1 right-hand side
    T* out;                     // level-1 result
    const T* win;               // IB windows of the active tiles
    const int* tiles;           // active-tile list
    int nTiles, ntiles;         // its length (0 without IB); number of tiles of the level
    int smoother, nu1, nu2, n0;
    const double* Pinv;         // coarsest pseudo-inverse, n0 x n0
};

// ------------------------------------------------------------------------------------------
// launchers (kernels_grid.cu)
template <typename T> void launch_residual(const GridK<T>& g, const T* x, const T* b, T* r, cudaStream_t s);
// y = L x of the lid-driven cavity on the periodic layout (kernels_cavity.cu); wall-face entries 0
template <typename T> void launch_cavity_apply(const GridK<T>& g, const T* x, T* y, cudaStream_t s);
// one additive Vanka sweep of the cavity: r = b - L x, per-cell patch solves into d (5 n), xo = x + omega
// (weighted corrections); g.fib must hold [S K J] x (kernels_cavity.cu)
template <typename T>
void launch_cavity_vanka(const GridK<T>& g, const T* x, const T* b, T* r, T* d, T* xo, T omega, cudaStream_t s);
// r = b - L x of the cavity (0 on the wall faces); x <- 0 on the wall faces
template <typename T> void launch_cavity_residual(const GridK<T>& g, const T* x, const T* b, T* r, cudaStream_t s);
template <typename T> void launch_cavity_zero_walls(T* x, int N, cudaStream_t s);
// rhs += the regularised lid's term 2 mu u_lid(x_i) / h^2 on the top row of u faces
void launch_cavity_add_lid(double* rhs, int N, double mu, cudaStream_t s);
// the cavity's transfers (kernels_cavity.cu): restriction with the coarse wall faces zeroed, and
// prolongation-correction with the pressure reflected at the walls
template <typename T> void launch_cavity_restrict(int Nc, const T* rf, T* bc, cudaStream_t s);
template <typename T> void launch_cavity_prolong_add(int Nc, const T* ec, T* xf, cudaStream_t s);
// the cavity's coarsest operator bordered for its gauge (the constant pressure), [L0 + Z Z^T | I]
void launch_cavity_assemble_L0(int N0, double rho, double mu, double dt, const double* B, double* Aug,
                               cudaStream_t s);
// zero the window entries of one level in a wall face's row or column
void launch_cavity_mask_windows(double* win, const int* tiles, int nTiles, int N, int tx, int ty, int ntx,
                                cudaStream_t s);
template <typename T> void launch_vanka(const GridK<T>& g, const T* x, const T* b, T* xo, cudaStream_t s);
template <typename T> void launch_restrict(int Nc, const T* rf, T* bc, cudaStream_t s);
template <typename T> void launch_prolong_add(int Nc, const T* ec, T* xf, cudaStream_t s);
template <typename Ti, typename To> void launch_convert(const Ti* in, To* out, int64_t n, cudaStream_t s);
template <typename T> void launch_axpby(T a, const T* x, T b, const T* y, T* z, int64_t n, cudaStream_t s);
// Schur-complement smoother pieces
template <typename T> void launch_sc_jacobi_A(const GridK<T>& g, const T* r, T* z, T scale, cudaStream_t s);
template <typename T> void launch_apply_AIB(const GridK<T>& g, const T* u, T* y, cudaStream_t s);
template <typename T> void launch_gradient(const GridK<T>& g, const T* p, T* gu, cudaStream_t s);
template <typename T> void launch_divergence(const GridK<T>& g, const T* u, T* d, cudaStream_t s);
template <typename T> void launch_jacobi_M(const GridK<T>& g, const T* r, T* z, T scale, cudaStream_t s);
// Vanka patch factors of every cell of the level from its patch entries (FP64, set-up)
void launch_patch_factors(const GridK<double>& g, double* pf, cudaStream_t s);
// one pass of a symmetric multicolour Gauss-Seidel sweep on A_IB (cells == false) or on
// Mh = D diag(A_IB)^{-1} G (cells == true): pass = colour 0 or 1, or -1 for the first pass from zero
template <typename T> void launch_sgs_pass(const GridK<T>& g, bool cells, int pass, T scale, const T* q, T* z,
                                           cudaStream_t s);
template <typename T> void launch_cheb_update(const T* dinvr, T* d, T* x, T ra, T rb, int64_t n, cudaStream_t s);
// fused kernels
template <typename T> void launch_vanka_zero(const GridK<T>& g, const T* b, T* xo, cudaStream_t s);
template <typename T> VankaBulk<T> vanka_bulk(double a0, double c, double inv_h);
template <typename T> void launch_residual_restrict(const GridK<T>& g, const T* x, const T* b, T* bc, cudaStream_t s);
template <typename T> void launch_sc_start(const GridK<T>& g, Cheb2<T> ka, const T* x, const T* b, T* r, T* d,
                                           cudaStream_t s);
template <typename T> void launch_sc_chebA(const GridK<T>& g, Cheb2<T> ka, const T* q, const T* d, T* y,
                                           cudaStream_t s);
template <typename T> void launch_sc_mstart(const GridK<T>& g, Cheb2<T> ka, Cheb2<T> km, const T* rp, const T* y,
                                            T* sv, T* dM, T* gq, T* dA, cudaStream_t s);
template <typename T> void launch_sc_mfinish(const GridK<T>& g, Cheb2<T> ka, Cheb2<T> km, const T* sv, const T* dM,
                                             const T* ya, T* dp, T* gq, T* dA, cudaStream_t s);
template <typename T> void launch_sc_finish(const GridK<T>& g, Cheb2<T> ka, const T* x, const T* y, const T* gq,
                                            const T* dA, const T* dp, T* xo, cudaStream_t s);
void launch_sc_diag(const GridK<double>& g, double* dinv, cudaStream_t s);
template <typename T> void launch_power_A(const GridK<T>& g, const T* v, T* w, cudaStream_t s);
template <typename T> void launch_power_Mstart(const GridK<T>& g, Cheb2<T> ka, const T* v, T* gq, T* dA,
                                               cudaStream_t s);
template <typename T> void launch_power_Mfinish(const GridK<T>& g, const T* ya, T* w, cudaStream_t s);

// launchers (kernels_small.cu)
template <typename T> size_t vcycle_small_smem(int N1, int n0, int nTiles, int per, int ntiles);
template <typename T> int vcycle_small_cluster(size_t smem);
template <typename T> cudaError_t launch_vcycle_small(const SmallArgs<T>& a, size_t smem, cudaStream_t s);

// launchers (kernels_wrap.cu): the Krylov-wrapped smoothing step
constexpr int WRAP_MAXK = 8;     // at most this many FGMRES iterations a smoothing stage
constexpr int WRAP_BLK = 152 * 8;   // most blocks of the inner-product and update kernels
// partials of V_i . w (i < cnt) into partials[i * nblk + block]; returns nblk
template <typename T> int launch_wdots(const T* V, int64_t ld, int cnt, const T* w, int64_t n, double* partials,
                                       cudaStream_t s);
// wout = win - sum_{i < cnt} coef[i] V_i, then partials of V_i . wout (mode 1) or of wout . wout
// (mode 2); returns nblk
template <typename T> int launch_wgs(const T* V, int64_t ld, int cnt, const double* coef, const T* win, T* wout,
                                     int64_t n, int mode, double* partials, cudaStream_t s);
void launch_wreduce(const double* partials, int cnt, int nblk, double* out, cudaStream_t s);
// the stage's last norm (one product) and then its least-squares solve, in one single-block launch
void launch_wreduce_lsq(const double* partials, int nblk, double* out, const double* hA, const double* hB,
                        const double* nrAll, const double* beta2, int k, double* y, cudaStream_t s);
// Levels of at most WRAP_ONE_MAX values: one block forms each inner product completely (launch_wdots
// and launch_wgs return nblk = 1 and write the sums themselves), the normalisations are fused
// (launch_wnorm_one: beta2 = |r0|^2, V0 = r0 / |r0|; launch_wgs2_one: the second Gram-Schmidt pass,
// the norm, the next Arnoldi vector and, with lsq_k > 0, the stage's least-squares solve).
constexpr int64_t WRAP_ONE_MAX = 3 * 32 * 32;
template <typename T> void launch_wnorm_one(const T* r0, int64_t n, double* beta2, T* V0, cudaStream_t s);
template <typename T> void launch_wgs2_one(const T* V, int64_t ld, int cnt, const double* coef, T* w, int64_t n,
                                           double* nr, T* Vnext, int lsq_k, const double* hA, const double* hB,
                                           const double* nrAll, const double* beta2, double* y, cudaStream_t s);
template <typename T> void launch_wmaxpy(const T* V, int64_t ld, int cnt, const double* coef, double sign, const T* yin,
                                         T* yout, int64_t n, cudaStream_t s);
template <typename T> void launch_wscale(const T* w, const double* nrm2, T* v, int64_t n, cudaStream_t s);

// launchers (kernels_ib.cu)
void launch_stencils(const double* X, int M, int Nf, int lmax, int** base, double** w64, float** w32,
                     cudaStream_t s);
void launch_sort_keys(const int* baseFine, int M, int Mpad, uint64_t* keys, cudaStream_t s);
void launch_bitonic(uint64_t* keys, int Mpad, cudaStream_t s);
void launch_unpack_sorted(const uint64_t* keys, int M, int* sorted, uint32_t* mkey, cudaStream_t s);
void launch_bins(const uint32_t* mkey, int M, int nbins, int shift, int* binStart, cudaStream_t s);
void launch_tile_flags(const int* base, int M, int W, int N, int tx, int ty, int ntx, unsigned char* flag,
                       cudaStream_t s);
void launch_tile_finish(unsigned char* flag, int ntx, int nty, int* tiles, int* nTiles, cudaStream_t s);
// slots of the active tiles whose raw flag is set (the rows of the IB operator are zero elsewhere)
void launch_row_slots(const unsigned char* flag, const int* tiles, const int* nTiles, int* rowSlots, int* nRow,
                      cudaStream_t s);
void launch_adjacency(const int* edges, int E, int M, int* deg, int* start, int* nbr, int* eid,
                      cudaStream_t s);
template <typename T> void launch_adj_kappa(const int* eid, const double* kappa, int n2E, T* kap, cudaStream_t s);
template <typename T> void launch_interp(const IBK<T>& k, const T* u, T* U, cudaStream_t s);
template <typename T> void launch_spring(const int* start, const int* nbr, const T* kap, int M, const T* U, T* F,
                                         cudaStream_t s);
// rowSlots != nullptr: only the tiles of that slot list (count *nRow, at most maxTiles) are written
template <typename T> void launch_spread(const IBK<T>& k, const T* F, T* f, const int* tiles, const int* nTiles,
                                         int maxTiles, int tx, int ty, int ntx, int warpPerFace, cudaStream_t s,
                                         const int* rowSlots = nullptr, const int* nRow = nullptr);
// the spreading's walk stored at set-up (rows: faces of the stencil-touched tiles, entries in the
// gather's order, cap = 2 M W^2), then applied as one ordered dot product per face
void launch_spread_store(const IBK<double>& k, const float* w32u, const float* w32v, const int* tiles,
                         const int* rowSlots, const int* nRow, int maxRow, int tx, int ty, int ntx, int* loc,
                         int* tileCnt, int* tileOff, int64_t cap, int* off, int* col, double* v64, float* v32,
                         cudaStream_t s);
template <typename T>
void launch_spread_stored(const int* off, const int* col, const T* val, const T* F, int M, T inv_h2, const int* tiles,
                          const int* rowSlots, const int* nRow, int maxRow, int N, int tx, int ty, int ntx, T* f,
                          cudaStream_t s);
// the patch entries B(f, f), B(f, f + e) and the coarsest dense IB block from the markers and springs
// (where the assembled windows are not available), by fixed-order gathers
void launch_patch_entries(const IBK<double>& k, const int* adjStart, const int* adjNbr, const double* adjKap,
                          const int* tiles, const int* rowSlots, const int* nRow, int maxRow, int tx, int ty, int ntx,
                          double* ibd, cudaStream_t s);
void launch_dense_ib(const IBK<double>& k, const int* adjStart, const int* adjNbr, const double* adjKap, double* B,
                     cudaStream_t s);
void launch_kj_patch(const IBK<double>& k, const int* adjStart, const int* adjNbr, const double* adjKap, double* KJ,
                     int* overflow, cudaStream_t s);
void launch_window_fine(const IBK<double>& k, const double* KJ, const int* tiles, int nTiles, int tx, int ty, int ntx,
                        double* win, cudaStream_t s);
void launch_window_rap(const double* winF, const int* slotF, int Nf, int txf, int tyf, int ntxf, const int* tilesC,
                       int nTilesC, int Nc, int txc, int tyc, int ntxc, double* winC, cudaStream_t s);
void launch_slot_map(const int* tiles, const int* nTiles, int ntiles, int* slotOf, cudaStream_t s);
void launch_window_patch(const double* win, const int* tiles, int nTiles, int N, int tx, int ty, int ntx, double* ibd,
                         cudaStream_t s);
void launch_window_dense(const double* win, const int* tiles, int nTiles, int N, int tx, int ty, int ntx, double* B,
                         cudaStream_t s);
// f = [S K J]^l u through the windows, on the tiles listed by rowSlots (at most maxRow of them)
template <typename T>
void launch_ib_window(const T* win, const int* tiles, const int* rowSlots, const int* nRow, int maxRow, int N, int tx,
                      int ty, int ntx, const T* u, T* f, cudaStream_t s);
void launch_deinterleave(const double* in, int M, double* out, cudaStream_t s);
void launch_interleave(const double* in, int M, double* out, cudaStream_t s);
void launch_advance_markers(const double* X, const double* U, int M, double dt, double* Xn, cudaStream_t s);
void launch_hash_vector(double* x, int64_t n, cudaStream_t s);
void launch_grad_kappa(const int* edges, int E, int M, const double* Lam, const double* Y, double* dkappa,
                       cudaStream_t s);
void launch_grad_X(const double* X, int M, int N, const double* w, const double* lam, const double* KY,
                   const double* KL, double dt, double acoef, double* dX, cudaStream_t s);

// Device-side state of one flexible-GMRES cycle (the loop runs as a conditional graph node).
constexpr int FG_MAXM = 100;                 // restart length cap
struct FgDev {
    int j, jn, its, k, converged, m, max_it, pad;
    double tol, est, inv_hn, beta;
    double g[FG_MAXM + 1], cs[FG_MAXM], sn[FG_MAXM], y[FG_MAXM];
    double hist[FG_MAXM + 1];                // residual estimates of this cycle, hist[0] = beta
    double H[(FG_MAXM + 1) * FG_MAXM];       // column j at H[j * (FG_MAXM + 1)]
};

// launchers (kernels_krylov.cu)
void launch_dot_partials(const double* x, const double* y, int64_t n, double* partials, int nblk, cudaStream_t s);
void launch_multidot(const double* V, int64_t ld, int k, const double* w, int64_t n, double* partials, int nblk,
                     cudaStream_t s);
void launch_reduce_partials(const double* partials, int k, int nblk, double* out, cudaStream_t s);
void launch_multi_axpy(const double* V, int64_t ld, int k, const double* coef, double sign, double* y,
                       int64_t n, cudaStream_t s);
void launch_scale(double* x, const double* num_den, int idx, int64_t n, cudaStream_t s);
void launch_block_means(const double* x, int N, int nblocks_vec, double* partials, int nblk, cudaStream_t s);
void launch_subtract_means(double* x, int N, const double* partials, int nblk, int mask, cudaStream_t s);
void launch_assemble_L0(int N0, double rho, double mu, double dt, const double* B, double* Aug, cudaStream_t s);
// blocked Gauss-Jordan inversion (n a multiple of 16); work: gauss_jordan_work_bytes(n) bytes
size_t gauss_jordan_work_bytes(int n);
void launch_gauss_jordan(double* Aug, int n, int* info, int* piv, void* work, cudaStream_t s);
void launch_extract_pinv(const double* Aug, const int* piv, int n, int N0, double rho, double* Pinv, cudaStream_t s);
template <typename T> void launch_coarse_apply(const double* Pinv, int n, const T* b, T* x, cudaStream_t s);
// xo = x + omega P r (x == nullptr: 0), P dense n x n FP64: the exact level solve of a level too small
// for the RAS boxes
template <typename T>
void launch_dense_correct(const double* P, int n, const T* r, const T* x, T omega, T* xo, cudaStream_t s);
void launch_check_finite(const double* x, int64_t n, int* flag, cudaStream_t s);

void launch_fg_init(FgDev* st, double beta, int m, int max_it, double tol, cudaStream_t s);
template <typename T> void launch_fg_prep(double* V, const double* w, int64_t n, FgDev* st, T* dst, cudaStream_t s);
template <typename T> void launch_fg_zstore(const T* src, double* Z, int64_t n, const FgDev* st, double* zcur,
                                            cudaStream_t s);
void launch_multidot_dev(const double* V, int64_t ld, const double* w, int64_t n, double* partials,
                         const FgDev* st, cudaStream_t s);
void launch_reduce_partials_dev(const double* partials, int nblk, double* out, const FgDev* st, int count,
                                cudaStream_t s);
void launch_multi_axpy_dev(const double* V, int64_t ld, const double* coef, double sign, double* y, int64_t n,
                           const FgDev* st, int useK, cudaStream_t s);
// returns the number of partial sums written
int launch_multi_axpy_norm_dev(const double* V, int64_t ld, const double* coef, double sign, double* y, int64_t n,
                               const FgDev* st, double* partials, cudaStream_t s);
void launch_fg_arnoldi(FgDev* st, const double* h1, const double* h2, const double* nrm,
                       cudaGraphConditionalHandle handle, cudaStream_t s);
void launch_fg_backsolve(FgDev* st, cudaStream_t s);

int num_blocks_for(int64_t n);

}  // namespace sib
